/* Second-order forward-mode automatic differentiation over up to 12 inputs.
 *
 * TEST INFRASTRUCTURE ONLY: part of the CPU oracle.  Only tests, the smoke
 * check and the benchmark's CPU baseline may load it; the CUDA library never
 * does.
 *
 * A jet carries a value, its gradient and its full (symmetric) Hessian with
 * respect to JET_N independent inputs.  The oracle uses jets so that every
 * gradient and Hessian it reports is the exact derivative of the energy as
 * written in the paper (orthogonality potential Eq. ortho-energy, clamped
 * barrier Eq. clamped-b), with no hand-derived derivative formula in between.
 */
#ifndef ORC_JET_H
#define ORC_JET_H

#define JET_N 12

typedef struct {
  double v;
  double g[JET_N];
  double h[JET_N * JET_N];
} jet;

void jet_const(jet* r, double c);
void jet_var(jet* r, double value, int index);
void jet_add(jet* r, const jet* a, const jet* b);
void jet_sub(jet* r, const jet* a, const jet* b);
void jet_mul(jet* r, const jet* a, const jet* b);
void jet_scale(jet* r, const jet* a, double c);
void jet_add_const(jet* r, const jet* a, double c);
/* r = f(a) given f(a.v), f'(a.v), f''(a.v) */
void jet_chain(jet* r, const jet* a, double f, double df, double d2f);
void jet_inv(jet* r, const jet* a);
void jet_div(jet* r, const jet* a, const jet* b);
void jet_sqrt(jet* r, const jet* a);
void jet_log(jet* r, const jet* a);
void jet_sq(jet* r, const jet* a);

/* 3-vectors of jets */
typedef struct {
  jet c[3];
} jet3;
void jet3_var(jet3* r, const double x[3], int first_index);
void jet3_sub(jet3* r, const jet3* a, const jet3* b);
void jet3_cross(jet3* r, const jet3* a, const jet3* b);
void jet3_dot(jet* r, const jet3* a, const jet3* b);

#endif
