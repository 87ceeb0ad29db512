/*
 * FP64 Schroedinger state-vector ORACLE -- test infrastructure only.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may load
 * this library.  It shares no code with the CUDA library: it is a plain,
 * deliberately unoptimised restatement of the definitions the paper uses.
 *
 * State: 2^n amplitudes alpha_i, stored as interleaved (re, im) doubles, in
 * LOGICAL order: index i = sum_q i_q 2^q (Sec. 2, representation of the state
 * as a vector of 2^n complex amplitudes).  Gate application updates amplitudes
 * in pairs / groups exactly as written in the definitions below (Sec. 2: the
 * simulator implements gates as linear manipulation of the amplitudes, 1-qubit
 * gates update pairs).  The outer loops are parallelised with OpenMP (the
 * paper's node-level threading) and are otherwise the textbook loops: no
 * blocking, fusion or reordering.
 *
 * Built with -O2 -fopenmp -ffp-contract=off so that every product and sum is
 * rounded separately (IEEE binary64, round to nearest).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { double re, im; } cpx;

static inline cpx cmul(cpx a, cpx b) {
  cpx r;
  r.re = a.re * b.re - a.im * b.im;
  r.im = a.re * b.im + a.im * b.re;
  return r;
}
static inline cpx cadd(cpx a, cpx b) {
  cpx r;
  r.re = a.re + b.re;
  r.im = a.im + b.im;
  return r;
}

/* |0...0>: alpha_0 = 1, all others 0 (state preparation, Sec. 2). */
void or_init_zero(double* psi, int n) {
  int64_t N = (int64_t)1 << n;
  memset(psi, 0, (size_t)N * 2 * sizeof(double));
  psi[0] = 1.0;
}

/* Arbitrary 1-qubit gate U (row-major 2x2, (re,im) pairs) on qubit q:
 * for every i with i_q = 0, (alpha_i, alpha_{i+2^q}) <- U (alpha_i, alpha_{i+2^q}). */
void or_apply_1q(double* psi, int n, const double* U, int q) {
  int64_t N = (int64_t)1 << n, s = (int64_t)1 << q;
  cpx u00 = {U[0], U[1]}, u01 = {U[2], U[3]}, u10 = {U[4], U[5]}, u11 = {U[6], U[7]};
  cpx* a = (cpx*)psi;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < N; i++) {
    if (i & s) continue;
    cpx x0 = a[i], x1 = a[i + s];
    a[i] = cadd(cmul(u00, x0), cmul(u01, x1));
    a[i + s] = cadd(cmul(u10, x0), cmul(u11, x1));
  }
}

/* Controlled 1-qubit gate: the pair update of or_apply_1q on the target,
 * restricted to indices whose control bit is 1 (Sec. 2, controlled 1-qubit
 * gates; CNOT is the case U = X). */
void or_apply_ctrl(double* psi, int n, const double* U, int c, int t) {
  int64_t N = (int64_t)1 << n, s = (int64_t)1 << t, cm = (int64_t)1 << c;
  cpx u00 = {U[0], U[1]}, u01 = {U[2], U[3]}, u10 = {U[4], U[5]}, u11 = {U[6], U[7]};
  cpx* a = (cpx*)psi;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < N; i++) {
    if ((i & s) || !(i & cm)) continue;
    cpx x0 = a[i], x1 = a[i + s];
    a[i] = cadd(cmul(u00, x0), cmul(u01, x1));
    a[i + s] = cadd(cmul(u10, x0), cmul(u11, x1));
  }
}

/* Dense k-qubit gate U (2^k x 2^k row-major, (re,im) pairs) on qubits
 * qs[0..k-1]: for every i with all target bits 0, gather the 2^k amplitudes
 * x_r = alpha_{i + sum_t r_t 2^{qs[t]}} (r = sum_t r_t 2^t), set x <- U x, scatter. */
void or_apply_dense(double* psi, int n, const double* U, int k, const int* qs) {
  int64_t N = (int64_t)1 << n;
  int64_t mask = 0;
  int K = 1 << k;
  for (int t = 0; t < k; t++) mask |= (int64_t)1 << qs[t];
  cpx* a = (cpx*)psi;
  const cpx* u = (const cpx*)U;
#pragma omp parallel
  {
    int64_t* off = (int64_t*)malloc(sizeof(int64_t) * K);
    cpx* x = (cpx*)malloc(sizeof(cpx) * K);
    cpx* y = (cpx*)malloc(sizeof(cpx) * K);
    for (int r = 0; r < K; r++) {
      off[r] = 0;
      for (int t = 0; t < k; t++)
        if ((r >> t) & 1) off[r] |= (int64_t)1 << qs[t];
    }
#pragma omp for schedule(static)
    for (int64_t i = 0; i < N; i++) {
      if (i & mask) continue;
      for (int r = 0; r < K; r++) x[r] = a[i + off[r]];
      for (int r = 0; r < K; r++) {
        cpx acc = {0.0, 0.0};
        for (int c = 0; c < K; c++) acc = cadd(acc, cmul(u[(int64_t)r * K + c], x[c]));
        y[r] = acc;
      }
      for (int r = 0; r < K; r++) a[i + off[r]] = y[r];
    }
    free(off);
    free(x);
    free(y);
  }
}

/* Two-qubit gate: the k = 2 case of or_apply_dense with r = b(q0) + 2 b(q1). */
void or_apply_2q(double* psi, int n, const double* U, int q0, int q1) {
  int qs[2] = {q0, q1};
  or_apply_dense(psi, n, U, 2, qs);
}

/* Storage index of amplitude i under qubit permutation sigma (Sec. 2):
 * j(i, sigma) = sum_q i_q 2^{sigma(q)}. */
static inline int64_t storage_index(int64_t i, int n, const int* sigma) {
  int64_t j = 0;
  for (int q = 0; q < n; q++)
    if ((i >> q) & 1) j |= (int64_t)1 << sigma[q];
  return j;
}

/* PermuteQubits(sigma'): `in` holds the state stored under sigma, `out` gets
 * the same state stored under sigma': out[j(i, sigma')] = in[j(i, sigma)]
 * for every logical index i (Sec. 2 and Appendix A). A pure copy. */
void or_permute(const double* in, double* out, int n, const int* sigma, const int* sigma_new) {
  int64_t N = (int64_t)1 << n;
  const cpx* a = (const cpx*)in;
  cpx* b = (cpx*)out;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < N; i++) b[storage_index(i, n, sigma_new)] = a[storage_index(i, n, sigma)];
}

/* Convert between storage order under sigma and logical order. */
void or_to_logical(const double* stored, double* logical, int n, const int* sigma) {
  int64_t N = (int64_t)1 << n;
  const cpx* a = (const cpx*)stored;
  cpx* b = (cpx*)logical;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < N; i++) b[i] = a[storage_index(i, n, sigma)];
}

/* p_i = |alpha_i|^2 (measurement probabilities). */
void or_probabilities(const double* psi, int n, double* p) {
  int64_t N = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < N; i++) p[i] = psi[2 * i] * psi[2 * i] + psi[2 * i + 1] * psi[2 * i + 1];
}

/* sum_i |alpha_i|^2, accumulated sequentially in index order. */
double or_norm2(const double* psi, int n) {
  int64_t N = (int64_t)1 << n;
  double s = 0.0;
  for (int64_t i = 0; i < N; i++) s += psi[2 * i] * psi[2 * i] + psi[2 * i + 1] * psi[2 * i + 1];
  return s;
}

/* <a|b> = sum_i conj(a_i) b_i, sequential. */
void or_inner(const double* a, const double* b, int n, double* out_re_im) {
  int64_t N = (int64_t)1 << n;
  double re = 0.0, im = 0.0;
  for (int64_t i = 0; i < N; i++) {
    double ar = a[2 * i], ai = a[2 * i + 1], br = b[2 * i], bi = b[2 * i + 1];
    re += ar * br + ai * bi;
    im += ar * bi - ai * br;
  }
  out_re_im[0] = re;
  out_re_im[1] = im;
}

int or_num_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}
