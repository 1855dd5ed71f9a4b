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

#include <mutex>

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

// Device address of the scratch array, looked up once per device with that
// device current.  In host code the array's name only stands in for the
// symbol; kernels must be given this address.
std::mutex g_mu;
double* g_addr[256] = {};

abd_status scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return ABD_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_ccd_scratch) != cudaSuccess || !p) return ABD_ERR_CUDA;
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
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
  k_toi_pairs<<<(int)blocks, 128, 0, st>>>(x_dev, dx_dev, nv, verts_dev, kind_dev, npairs, ccd_s, ccd_max, scratch);
  k_toi_min<<<1, 1024, 0, st>>>(npairs, scratch);
  double res[2];
  if (cudaMemcpyAsync(res, scratch + kResultSlot, sizeof(res), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return ABD_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) return ABD_ERR_CUDA;
  unsigned long long status;
  memcpy(&status, &res[1], sizeof(status));
  if (status & (kBadIndex | kBadKind)) return ABD_ERR_INVALID_ARG;
  *toi_host = res[0];
  if (status & kCapHit) return ABD_ERR_CCD_MAXITER;
  return ABD_OK;
}
