// Minimum additive-CCD time of impact over a caller-given pair list, for
// callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocator) at the point where
// they need a CCD bound: code running while another component owns the
// device memory budget (a fixed-size pool handed out once at start-up), real-
// time loops that forbid allocation after initialisation, or hosts whose only
// allocator is unavailable on the calling thread.  This entry point takes
// every input and the output from the caller and keeps its scratch in a
// file-scope __device__ array that exists on every GPU that loads the library
// until the process exits.
#include <string.h>

#include <cuda.h>

#include <mutex>
#include <vector>

#include "../../include/abd.h"
#include "geom.cuh"

namespace {

// Scratch: one time of impact per pair, then the result and a status word.
constexpr long kNoAllocMaxPairs = 1L << 18;  // 262,144 pairs -> 2 MiB per GPU
constexpr long kResultSlot = kNoAllocMaxPairs;
constexpr long kStatusSlot = kNoAllocMaxPairs + 1;
static __device__ __align__(256) double g_ccd_scratch[kNoAllocMaxPairs + 32];

constexpr unsigned long long kBadIndex = 1ull, kBadKind = 2ull, kCapHit = 4ull;

__global__ void k_toi_pairs(const double* __restrict__ x, const double* __restrict__ dx, int nv,
                            const int* __restrict__ verts, const unsigned char* __restrict__ kind, long n,
                            double s, int max_iter, double* scratch) {
  unsigned long long* status = reinterpret_cast<unsigned long long*>(scratch + kStatusSlot);
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < n; p += (long)gridDim.x * blockDim.x) {
    const int k = kind[p];
    abd::v3 xs[4], ds[4];
    bool ok = k == 0 || k == 1;
    if (!ok) atomicOr(status, kBadKind);
    for (int m = 0; m < 4 && ok; ++m) {
      const int v = verts[4 * p + m];
      if (v < 0 || v >= nv) {
        atomicOr(status, kBadIndex);
        ok = false;
        break;
      }
      xs[m] = abd::v3{x[3 * v], x[3 * v + 1], x[3 * v + 2]};
      ds[m] = abd::v3{dx[3 * v], dx[3 * v + 1], dx[3 * v + 2]};
    }
    double toi = 1.0;
    if (ok && abd::accd(k, xs, ds, s, 1.0, max_iter, toi)) atomicOr(status, kCapHit);
    scratch[p] = toi;
  }
}

// fixed-order minimum of scratch[0..n) into the result slot
__global__ void k_toi_min(long n, double* scratch) {
  __shared__ double red[1024];
  double m = 1.0;
  for (long i = threadIdx.x; i < n; i += 1024) m = fmin(m, scratch[i]);
  red[threadIdx.x] = m;
  __syncthreads();
  for (int o = 512; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = fmin(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) scratch[kResultSlot] = red[0];
}

// Device address of the scratch array.  In host code the array's name only
// stands in for the symbol; kernels must be given the address that
// cudaGetSymbolAddress returns for the CUDA context that launches them.  That
// address belongs to one context: after cudaDeviceReset, or in a driver-API
// context other than the device's primary one, the module is loaded again at
// another address.  The cache is therefore keyed on the device and on the
// context's unique id (cuCtxGetId, reached through the runtime's driver
// entry-point query, so the library does not link libcuda directly).
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

struct ScratchEntry {
  int dev;
  unsigned long long ctx_id;
  double* addr;
};

std::mutex g_mu;
std::vector<ScratchEntry> g_cache;
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;
bool g_entry_points_tried = false;

// id of the calling thread's current context; false if there is none yet
// (the runtime creates the primary context on its first device call) or the
// driver entry points are unavailable.  Called with g_mu held.
bool current_context_id(unsigned long long* id) {
  if (!g_entry_points_tried) {
    g_entry_points_tried = true;
    cudaDriverEntryPointQueryResult q1, q2;
    void* f1 = nullptr;
    void* f2 = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess && f1 && f2) {
      g_ctx_current = reinterpret_cast<CtxGetCurrentFn>(f1);
      g_ctx_id = reinterpret_cast<CtxGetIdFn>(f2);
    } else {
      cudaGetLastError();  // a failed query leaves nothing pending for the caller
    }
  }
  if (!g_ctx_current || !g_ctx_id) return false;
  CUcontext c = nullptr;
  if (g_ctx_current(&c) != CUDA_SUCCESS || !c) return false;
  return g_ctx_id(c, id) == CUDA_SUCCESS;
}

abd_status scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return ABD_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  unsigned long long id = 0;
  bool have_id = current_context_id(&id);
  if (have_id)
    for (const ScratchEntry& e : g_cache)
      if (e.dev == dev && e.ctx_id == id) {
        *out = e.addr;
        return ABD_OK;
      }
  // set-up for this device and context: look the address up with the
  // device current (the lookup also creates the primary context if needed)
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_ccd_scratch) != cudaSuccess || !p) return ABD_ERR_CUDA;
  if (!have_id) have_id = current_context_id(&id);
  if (have_id) {
    bool replaced = false;
    for (ScratchEntry& e : g_cache)
      if (e.dev == dev) {  // a context of this device that is gone or not current: keep one entry per device
        e.ctx_id = id;
        e.addr = static_cast<double*>(p);
        replaced = true;
      }
    if (!replaced) g_cache.push_back(ScratchEntry{dev, id, static_cast<double*>(p)});
  }
  // without a context id nothing is cached: every call looks the address up
  *out = static_cast<double*>(p);
  return ABD_OK;
}

}  // namespace

extern "C" ABD_API abd_status abd_ccd_toi_pairs_noalloc(const double* x_dev, const double* dx_dev, int nv,
                                                        const int* verts_dev, const unsigned char* kind_dev,
                                                        long npairs, double ccd_s, int ccd_max, void* stream,
                                                        double* toi_host) {
  if (!toi_host || npairs < 0 || nv < 0 || !(ccd_s > 0.0 && ccd_s < 1.0) || ccd_max <= 0) return ABD_ERR_INVALID_ARG;
  if (npairs > kNoAllocMaxPairs) return ABD_ERR_CAPACITY;
  if (npairs == 0) {
    *toi_host = 1.0;
    return ABD_OK;
  }
  if (!x_dev || !dx_dev || !verts_dev || !kind_dev) return ABD_ERR_INVALID_ARG;
  double* scratch = nullptr;
  if (abd_status r = scratch_address(&scratch)) return r;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the array keeps the previous call's contents: clear the status word
  if (cudaMemsetAsync(scratch + kStatusSlot, 0, sizeof(unsigned long long), st) != cudaSuccess) return ABD_ERR_CUDA;
  long blocks = (npairs + 127) / 128;
  if (blocks > 152 * 8) blocks = 152 * 8;
  // each launch's own error is returned by cudaLaunchKernel; the caller's
  // unrelated pending errors are neither reported nor consumed here
  {
    void* args[] = {(void*)&x_dev, (void*)&dx_dev, (void*)&nv, (void*)&verts_dev, (void*)&kind_dev,
                    (void*)&npairs, (void*)&ccd_s, (void*)&ccd_max, (void*)&scratch};
    if (cudaLaunchKernel((const void*)k_toi_pairs, dim3((unsigned)blocks), dim3(128), args, 0, st) != cudaSuccess)
      return ABD_ERR_CUDA;
  }
  {
    void* args[] = {(void*)&npairs, (void*)&scratch};
    if (cudaLaunchKernel((const void*)k_toi_min, dim3(1), dim3(1024), args, 0, st) != cudaSuccess)
      return ABD_ERR_CUDA;
  }
  double res[2];
  if (cudaMemcpyAsync(res, scratch + kResultSlot, sizeof(res), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return ABD_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return ABD_ERR_CUDA;
  unsigned long long status;
  memcpy(&status, &res[1], sizeof(status));
  if (status & (kBadIndex | kBadKind)) return ABD_ERR_INVALID_ARG;
  *toi_host = res[0];
  if (status & kCapHit) return ABD_ERR_CCD_MAXITER;
  return ABD_OK;
}
