/* A C caller of libqs.so (no Python): GHZ states through every layer of the C ABI.
 *
 * H(0) then CNOT(0, k) for k = 1 .. n-1 gives (|0...0> + |1...1>) / sqrt(2), a closed form.
 * The program checks it (1) through qs_compile / qs_execute in every compile mode,
 * (2) through the per-gate calls, and (3) through the serving calls (qs_server_*) for
 * several n and both dtypes at once.  Prints "ok" and exits 0 on success.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "qs.h"

#define CHECK(call)                                                               \
  do {                                                                            \
    qs_status _s = (call);                                                        \
    if (_s != QS_OK) {                                                            \
      fprintf(stderr, "%s:%d %s -> %d (%s)\n", __FILE__, __LINE__, #call, (int)_s, qs_last_error()); \
      exit(1);                                                                    \
    }                                                                             \
  } while (0)

static int ghz_ops(int n, qs_op* ops) {
  memset(ops, 0, sizeof(qs_op) * (size_t)n);
  ops[0].kind = QS_OP_H;
  ops[0].nq = 1;
  ops[0].q[0] = 0;
  ops[0].mat = -1;
  for (int k = 1; k < n; k++) {
    ops[k].kind = QS_OP_CNOT;
    ops[k].nq = 2;
    ops[k].q[0] = 0;
    ops[k].q[1] = k;
    ops[k].mat = -1;
  }
  return n;
}

/* amplitudes as doubles (re, im) of either dtype */
static void amp(const void* buf, int dtype, size_t i, double* re, double* im) {
  if (dtype == QS_C128) {
    *re = ((const double*)buf)[2 * i];
    *im = ((const double*)buf)[2 * i + 1];
  } else {
    *re = ((const float*)buf)[2 * i];
    *im = ((const float*)buf)[2 * i + 1];
  }
}

static void check_ghz(const void* buf, int n, int dtype, size_t count) {
  const double tol = dtype == QS_C128 ? 1e-12 : 1e-6;
  const double h = 1.0 / sqrt(2.0);
  const size_t last = ((size_t)1 << n) - 1;
  for (size_t i = 0; i < count; i++) {
    double re, im;
    amp(buf, dtype, i, &re, &im);
    const double want = (i == 0 || i == last) ? h : 0.0;
    if (fabs(re - want) > tol || fabs(im) > tol) {
      fprintf(stderr, "n=%d dtype=%d amplitude %zu = (%g, %g), want %g\n", n, dtype, i, re, im, want);
      exit(1);
    }
  }
}

int main(void) {
  qs_op ops[32];
  double dummy = 0.0;
  /* (1) compiled plans, every mode and dtype */
  for (int dtype = 0; dtype < 2; dtype++)
    for (int mode = 0; mode < 3; mode++) {
      const int n = 14;
      qs_handle h;
      CHECK(qs_create(n, (qs_dtype)dtype, &h));
      qs_compile_opts o;
      memset(&o, 0, sizeof(o));
      o.mode = mode;
      o.dtype = dtype;
      o.tile_bits = mode == QS_MODE_PAPER ? 8 : 0;
      qs_plan_t p;
      CHECK(qs_compile(n, ops, (size_t)ghz_ops(n, ops), &dummy, 0, NULL, &o, &p));
      qs_plan_stats st;
      CHECK(qs_plan_get_stats(p, &st));
      CHECK(qs_execute(h, p));
      CHECK(qs_plan_destroy(p));
      const size_t N = (size_t)1 << n;
      void* buf = malloc(N * (dtype == QS_C128 ? 16 : 8));
      CHECK(qs_get_amplitudes(h, buf, 0, N, QS_ORDER_LOGICAL));
      check_ghz(buf, n, dtype, N);
      double nrm;
      CHECK(qs_norm(h, &nrm));
      if (fabs(nrm - 1.0) > 1e-6) return 1;
      free(buf);
      CHECK(qs_destroy(h));
    }
  /* (2) per-gate calls */
  {
    const int n = 10;
    qs_handle h;
    CHECK(qs_create(n, QS_C128, &h));
    const double hd = 1.0 / sqrt(2.0);
    const double H[8] = {hd, 0, hd, 0, hd, 0, -hd, 0};
    const double X[8] = {0, 0, 1, 0, 1, 0, 0, 0};
    CHECK(qs_apply_1q(h, H, 0));
    for (int k = 1; k < n; k++) CHECK(qs_apply_controlled(h, X, 0, k));
    double buf[2 * 1024];
    CHECK(qs_get_amplitudes(h, buf, 0, 1024, QS_ORDER_LOGICAL));
    check_ghz(buf, n, QS_C128, 1024);
    CHECK(qs_destroy(h));
  }
  /* (3) the server: 12 requests of 8..19 qubits, both dtypes, submitted at once */
  {
    qs_server_t s;
    qs_server_opts so;
    memset(&so, 0, sizeof(so));
    so.slots = 4;
    so.readout = 4;
    so.mem_budget = (int64_t)1 << 30;
    CHECK(qs_server_create(&so, &s));
    int64_t ids[12];
    int ns[12], dts[12];
    for (int r = 0; r < 12; r++) {
      ns[r] = 8 + r;
      dts[r] = r & 1;
      CHECK(qs_server_submit(s, ns[r], (qs_dtype)dts[r], ops, (size_t)ghz_ops(ns[r], ops), &dummy, 0, &ids[r]));
    }
    int done = 0;
    for (int tries = 0; done < 12 && tries < 600; tries++) {
      qs_server_result res[12];
      int cnt = 0;
      CHECK(qs_server_poll(s, res, 12, &cnt, 100));
      for (int i = 0; i < cnt; i++) {
        if (res[i].status != QS_OK) {
          fprintf(stderr, "request %lld failed: %s\n", (long long)res[i].id, res[i].error);
          return 1;
        }
        double buf[8];
        CHECK(qs_server_take(s, res[i].id, buf, res[i].amplitudes));
        check_ghz(buf, res[i].n, res[i].dtype, res[i].amplitudes);
        if (fabs(res[i].norm - 1.0) > 1e-6) return 1;
        done++;
      }
    }
    if (done != 12) {
      fprintf(stderr, "only %d of 12 requests finished\n", done);
      return 1;
    }
    qs_server_stats stt;
    CHECK(qs_server_get_stats(s, &stt));
    if (stt.completed != 12) return 1;
    CHECK(qs_server_destroy(s));
  }
  printf("ok\n");
  return 0;
}
