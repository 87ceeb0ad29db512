// Host build of the complex128 double-float arithmetic of the tile and per-gate kernels
// (paper_2010_09746_gb300/csrc/arith.cuh), checked against long double.  The formulas are
// the device ones; on the host every packed f32x2 step is two IEEE binary32 operations with
// round-to-nearest, which is what the f32x2 instructions compute lane by lane.
//
// Prints one line per formula: "<name> <worst error relative to the operand magnitudes>".
#include <cmath>
#include <complex>
#include <cstdio>
#include <random>
#include <vector>

#include "../paper_2010_09746_gb300/csrc/arith.cuh"
#include "../paper_2010_09746_gb300/csrc/qs_internal.h"

using namespace qs;
typedef std::complex<long double> cl;

static dfm entry(double re, double im) {   // through the pool's own serialisation
  Pool p;
  p.add(cd(re, im));
  std::vector<unsigned char> ser = p.serialise(POL_DF);
  dfm m;
  memcpy(&m, ser.data(), sizeof(m));
  return m;
}
static cl val(float4 v) { return cl((long double)v.x + (long double)v.z, (long double)v.y + (long double)v.w); }

int main() {
  std::mt19937_64 g(7);
  std::normal_distribution<double> nd;
  std::uniform_real_distribution<double> ud(-3.141592653589793, 3.141592653589793);
  double w_rt = 0, w_mul = 0, w_rx = 0, w_axpy = 0, w_axmy = 0, w_ymx = 0, w_rot = 0, w_q = 0, w_chain = 0;
  auto upd = [](double& w, long double e) { w = std::max(w, (double)e); };
  for (int it = 0; it < 100000; it++) {
    const double2 d = make_double2(nd(g), nd(g) * std::ldexp(1.0, -(int)(it % 40)));
    const double2 r = ADF::to_store(ADF::from_store(d));
    upd(w_rt, std::max(std::fabs(r.x - d.x) / std::fabs(d.x), std::fabs(r.y - d.y) / std::fabs(d.y)));
    const float4 a = ADF::from_store(make_double2(nd(g), nd(g))), b = ADF::from_store(make_double2(nd(g), nd(g)));
    const cl A = val(a), B = val(b);
    const long double na = std::abs(A), nb = std::abs(B);
    const double ur = nd(g), ui = nd(g);
    const cl U((long double)ur, (long double)ui);
    upd(w_mul, std::abs(val(ADF::mul(entry(ur, ui), a)) - U * A) / (std::abs(U) * na));
    const double th = ud(g), c = std::cos(th), s = std::sin(th);
    upd(w_rx, std::abs(val(ADF::rx(entry(c, s), a, b)) - ((long double)c * A - cl(0, 1) * (long double)s * B)) / (na + nb));
    double t = std::tan(th / 2);
    if (std::fabs(t) > 1) t = 1 / t;
    const dfr T = ADF::real_of(entry(t, 0.0));
    const long double tl = t, den = na + std::fabs(t) * nb;
    upd(w_axpy, std::abs(val(ADF::axpy_r(T, b, a)) - (A + tl * B)) / den);
    upd(w_axmy, std::abs(val(ADF::axmy_r(T, b, a)) - (A - tl * B)) / den);
    upd(w_ymx, std::abs(val(ADF::ymx_r(T, b, a)) - (tl * B - A)) / den);
    float4 a2, b2;
    ADF::rot_r(ADF::real_of(entry(c, 0.0)), ADF::real_of(entry(s, 0.0)), a, b, a2, b2);
    upd(w_rot, std::max(std::abs(val(a2) - ((long double)c * A + (long double)s * B)),
                        std::abs(val(b2) - ((long double)c * B - (long double)s * A))) / (na + nb));
    for (unsigned q = 0; q < 4; q++) {
      const cl f = q == 0 ? cl(1, 0) : q == 1 ? cl(0, -1) : q == 2 ? cl(-1, 0) : cl(0, 1);
      upd(w_q, std::abs(val(ADF::rot_q(a, q)) - f * A));
    }
  }
  // chains of 64 rotations and phases on unnormalised register values (no to_store between)
  for (int it = 0; it < 2000; it++) {
    float4 x0 = ADF::from_store(make_double2(nd(g), nd(g))), x1 = ADF::from_store(make_double2(nd(g), nd(g)));
    cl X0 = val(x0), X1 = val(x1);
    for (int k = 0; k < 64; k++) {
      const double th = ud(g);
      const double t = std::tan(th / 2);
      const dfr T = ADF::real_of(entry(std::fabs(t) <= 1 ? t : 1 / t, 0.0));
      const long double tl = std::fabs(t) <= 1 ? t : 1 / t;
      const float4 y0 = (k & 1) ? ADF::axpy_r(T, x1, x0) : ADF::axpy_r(T, x0, x1);
      const float4 y1 = (k & 1) ? ADF::axmy_r(T, x0, x1) : ADF::ymx_r(T, x1, x0);
      const cl Y0 = (k & 1) ? X0 + tl * X1 : X1 + tl * X0;
      const cl Y1 = (k & 1) ? X1 - tl * X0 : tl * X1 - X0;
      // keep the magnitudes bounded as the tangent-form pass does with its dropped factor
      const long double sc = 1.0L / std::sqrt(1.0L + tl * tl);
      const double ph = ud(g);
      const dfm P = entry(std::cos(ph) * (double)sc, std::sin(ph) * (double)sc);
      const cl Pl((long double)std::cos(ph) * (long double)(double)sc, (long double)std::sin(ph) * (long double)(double)sc);
      x0 = ADF::mul(P, y0);
      x1 = ADF::mul(P, y1);
      X0 = Pl * Y0;
      X1 = Pl * Y1;
    }
    const double2 s0 = ADF::to_store(x0), s1 = ADF::to_store(x1);
    const long double nrm = std::sqrt(std::norm(X0) + std::norm(X1));
    upd(w_chain, std::max(std::abs(cl(s0.x, s0.y) - X0), std::abs(cl(s1.x, s1.y) - X1)) / nrm);
  }
  printf("roundtrip %.6e\nmul %.6e\nrx %.6e\naxpy %.6e\naxmy %.6e\nymx %.6e\nrot %.6e\nrot_q %.6e\nchain64 %.6e\n", w_rt,
         w_mul, w_rx, w_axpy, w_axmy, w_ymx, w_rot, w_q, w_chain);
  return 0;
}
