/* Second-order forward-mode AD (see jet.h).  TEST INFRASTRUCTURE ONLY. */
#include "jet.h"

#include <math.h>
#include <string.h>

void jet_const(jet* r, double c) {
  memset(r, 0, sizeof(*r));
  r->v = c;
}

void jet_var(jet* r, double value, int index) {
  memset(r, 0, sizeof(*r));
  r->v = value;
  r->g[index] = 1.0;
}

void jet_add(jet* r, const jet* a, const jet* b) {
  jet t;
  t.v = a->v + b->v;
  for (int i = 0; i < JET_N; ++i) t.g[i] = a->g[i] + b->g[i];
  for (int i = 0; i < JET_N * JET_N; ++i) t.h[i] = a->h[i] + b->h[i];
  *r = t;
}

void jet_sub(jet* r, const jet* a, const jet* b) {
  jet t;
  t.v = a->v - b->v;
  for (int i = 0; i < JET_N; ++i) t.g[i] = a->g[i] - b->g[i];
  for (int i = 0; i < JET_N * JET_N; ++i) t.h[i] = a->h[i] - b->h[i];
  *r = t;
}

/* product rule: d(ab) = a db + b da; d2(ab) = a d2b + b d2a + da dbT + db daT */
void jet_mul(jet* r, const jet* a, const jet* b) {
  jet t;
  t.v = a->v * b->v;
  for (int i = 0; i < JET_N; ++i) t.g[i] = a->v * b->g[i] + b->v * a->g[i];
  for (int i = 0; i < JET_N; ++i)
    for (int j = 0; j < JET_N; ++j)
      t.h[i * JET_N + j] = a->v * b->h[i * JET_N + j] + b->v * a->h[i * JET_N + j] +
                           a->g[i] * b->g[j] + b->g[i] * a->g[j];
  *r = t;
}

void jet_scale(jet* r, const jet* a, double c) {
  jet t;
  t.v = a->v * c;
  for (int i = 0; i < JET_N; ++i) t.g[i] = a->g[i] * c;
  for (int i = 0; i < JET_N * JET_N; ++i) t.h[i] = a->h[i] * c;
  *r = t;
}

void jet_add_const(jet* r, const jet* a, double c) {
  *r = *a;
  r->v += c;
}

/* chain rule: d f(a) = f' da; d2 f(a) = f' d2a + f'' da daT */
void jet_chain(jet* r, const jet* a, double f, double df, double d2f) {
  jet t;
  t.v = f;
  for (int i = 0; i < JET_N; ++i) t.g[i] = df * a->g[i];
  for (int i = 0; i < JET_N; ++i)
    for (int j = 0; j < JET_N; ++j)
      t.h[i * JET_N + j] = df * a->h[i * JET_N + j] + d2f * a->g[i] * a->g[j];
  *r = t;
}

void jet_inv(jet* r, const jet* a) {
  double x = a->v;
  jet_chain(r, a, 1.0 / x, -1.0 / (x * x), 2.0 / (x * x * x));
}

void jet_div(jet* r, const jet* a, const jet* b) {
  jet ib;
  jet_inv(&ib, b);
  jet_mul(r, a, &ib);
}

void jet_sqrt(jet* r, const jet* a) {
  double s = sqrt(a->v);
  jet_chain(r, a, s, 0.5 / s, -0.25 / (s * a->v));
}

void jet_log(jet* r, const jet* a) {
  double x = a->v;
  jet_chain(r, a, log(x), 1.0 / x, -1.0 / (x * x));
}

void jet_sq(jet* r, const jet* a) { jet_mul(r, a, a); }

void jet3_var(jet3* r, const double x[3], int first_index) {
  for (int k = 0; k < 3; ++k) jet_var(&r->c[k], x[k], first_index + k);
}

void jet3_sub(jet3* r, const jet3* a, const jet3* b) {
  for (int k = 0; k < 3; ++k) jet_sub(&r->c[k], &a->c[k], &b->c[k]);
}

void jet3_cross(jet3* r, const jet3* a, const jet3* b) {
  jet3 t;
  jet p, q;
  jet_mul(&p, &a->c[1], &b->c[2]);
  jet_mul(&q, &a->c[2], &b->c[1]);
  jet_sub(&t.c[0], &p, &q);
  jet_mul(&p, &a->c[2], &b->c[0]);
  jet_mul(&q, &a->c[0], &b->c[2]);
  jet_sub(&t.c[1], &p, &q);
  jet_mul(&p, &a->c[0], &b->c[1]);
  jet_mul(&q, &a->c[1], &b->c[0]);
  jet_sub(&t.c[2], &p, &q);
  *r = t;
}

void jet3_dot(jet* r, const jet3* a, const jet3* b) {
  jet t, p;
  jet_mul(&t, &a->c[0], &b->c[0]);
  jet_mul(&p, &a->c[1], &b->c[1]);
  jet_add(&t, &t, &p);
  jet_mul(&p, &a->c[2], &b->c[2]);
  jet_add(r, &t, &p);
}
