// Complex arithmetic policies for the state-vector kernels.
//
// A kernel is written once over a policy A:
//   A::store_t  element as it sits in HBM (float2 for complex64, double2 for complex128)
//   A::reg_t    element as the kernel computes on it (registers and shared memory)
//   A::mat_t    gate-matrix entry in the policy's own format
//
// AF32  complex64 storage, FP32 arithmetic.
// AF64  complex128 storage, native FP64 arithmetic (reference policy; on GB300 the FP64
//       pipe issues about 2 DFMA per clock per SM, 1/64 of FP32, so this policy is
//       ALU-bound by a wide margin).
// ADF   complex128 storage, "double-float" arithmetic on the FP32 pipe: each real number is
//       an unevaluated sum hi + lo of two floats (Dekker 1971 TwoProduct via FMA; Knuth
//       TwoSum; Shewchuk 1997 renormalisation).  About 47-48 significant bits, relative
//       error ~1e-14 per operation.  The FP64 <-> (hi, lo) conversions are done with
//       integer bit manipulation so that no instruction touches the FP64 pipe.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace qs {

// ------------------------------------------------------------------------------------------
// complex64, FP32
// ------------------------------------------------------------------------------------------
struct AF32 {
  using store_t = float2;
  using reg_t = float2;
  using mat_t = float2;
  static constexpr int kStoreBytes = 8;
  static __device__ __forceinline__ reg_t from_store(store_t v) { return v; }
  static __device__ __forceinline__ store_t to_store(reg_t v) { return v; }
  static __device__ __forceinline__ reg_t zero() { return make_float2(0.f, 0.f); }
  // u*a + v*b
  static __device__ __forceinline__ reg_t mac2(mat_t u, reg_t a, mat_t v, reg_t b) {
    float re = u.x * a.x;
    re = fmaf(-u.y, a.y, re);
    re = fmaf(v.x, b.x, re);
    re = fmaf(-v.y, b.y, re);
    float im = u.x * a.y;
    im = fmaf(u.y, a.x, im);
    im = fmaf(v.x, b.y, im);
    im = fmaf(v.y, b.x, im);
    return make_float2(re, im);
  }
  // acc + u*a
  static __device__ __forceinline__ reg_t mac(reg_t acc, mat_t u, reg_t a) {
    float re = fmaf(u.x, a.x, acc.x);
    re = fmaf(-u.y, a.y, re);
    float im = fmaf(u.x, a.y, acc.y);
    im = fmaf(u.y, a.x, im);
    return make_float2(re, im);
  }
  static __device__ __forceinline__ reg_t mul(mat_t u, reg_t a) {
    return make_float2(fmaf(u.x, a.x, -u.y * a.y), fmaf(u.x, a.y, u.y * a.x));
  }
  // (c*a.re + s*b.im, c*a.im - s*b.re): the RX-type update c*a - i*s*b
  static __device__ __forceinline__ reg_t rx(mat_t cs, reg_t a, reg_t b) {
    return make_float2(fmaf(cs.x, a.x, cs.y * b.y), fmaf(cs.x, a.y, -cs.y * b.x));
  }
  // u + t v with the real t in t.x (tangent-form RX), and -i b
  static __device__ __forceinline__ reg_t axpy(mat_t t, reg_t v, reg_t u) {
    return make_float2(fmaf(t.x, v.x, u.x), fmaf(t.x, v.y, u.y));
  }
  static __device__ __forceinline__ reg_t mul_mi(reg_t b) { return make_float2(b.y, -b.x); }
  static __device__ __forceinline__ reg_t neg(reg_t a) { return make_float2(-a.x, -a.y); }
  static __device__ __forceinline__ double norm2(reg_t a) {
    return (double)a.x * (double)a.x + (double)a.y * (double)a.y;
  }
};

// ------------------------------------------------------------------------------------------
// complex128, native FP64
// ------------------------------------------------------------------------------------------
struct AF64 {
  using store_t = double2;
  using reg_t = double2;
  using mat_t = double2;
  static constexpr int kStoreBytes = 16;
  static __device__ __forceinline__ reg_t from_store(store_t v) { return v; }
  static __device__ __forceinline__ store_t to_store(reg_t v) { return v; }
  static __device__ __forceinline__ reg_t zero() { return make_double2(0.0, 0.0); }
  static __device__ __forceinline__ reg_t mac2(mat_t u, reg_t a, mat_t v, reg_t b) {
    double re = u.x * a.x;
    re = fma(-u.y, a.y, re);
    re = fma(v.x, b.x, re);
    re = fma(-v.y, b.y, re);
    double im = u.x * a.y;
    im = fma(u.y, a.x, im);
    im = fma(v.x, b.y, im);
    im = fma(v.y, b.x, im);
    return make_double2(re, im);
  }
  static __device__ __forceinline__ reg_t mac(reg_t acc, mat_t u, reg_t a) {
    double re = fma(u.x, a.x, acc.x);
    re = fma(-u.y, a.y, re);
    double im = fma(u.x, a.y, acc.y);
    im = fma(u.y, a.x, im);
    return make_double2(re, im);
  }
  static __device__ __forceinline__ reg_t mul(mat_t u, reg_t a) {
    return make_double2(fma(u.x, a.x, -u.y * a.y), fma(u.x, a.y, u.y * a.x));
  }
  static __device__ __forceinline__ reg_t rx(mat_t cs, reg_t a, reg_t b) {
    return make_double2(fma(cs.x, a.x, cs.y * b.y), fma(cs.x, a.y, -cs.y * b.x));
  }
  static __device__ __forceinline__ reg_t axpy(mat_t t, reg_t v, reg_t u) {
    return make_double2(fma(t.x, v.x, u.x), fma(t.x, v.y, u.y));
  }
  static __device__ __forceinline__ reg_t mul_mi(reg_t b) { return make_double2(b.y, -b.x); }
  static __device__ __forceinline__ reg_t neg(reg_t a) { return make_double2(-a.x, -a.y); }
  static __device__ __forceinline__ double norm2(reg_t a) { return a.x * a.x + a.y * a.y; }
};

// ------------------------------------------------------------------------------------------
// double-float building blocks (all explicitly rounded: no contraction changes them)
// ------------------------------------------------------------------------------------------
struct dfl { float hi, lo; };

// s + e == a + b exactly (Knuth TwoSum, 6 flops)
static __device__ __forceinline__ dfl two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
// s + e == a + b exactly when |a| >= |b| (Dekker FastTwoSum, 3 flops)
static __device__ __forceinline__ dfl fast_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}
// p + e == a * b exactly (TwoProduct with FMA)
static __device__ __forceinline__ dfl two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  float e = __fmaf_rn(a, b, -p);
  return {p, e};
}

// Split a binary64 value into hi + lo floats without FP64 instructions.
// hi keeps the leading 24 significant bits (truncated), lo = x - hi (its 29 bits rounded
// to 24): |x - (hi + lo)| <= 2^-47 |x|.  |x| < 2^-126 flushes to 0 (absolute error
// below 1.2e-38); the lo part flushes when it would leave the normal float range
// (|x| below about 2^-98; absolute error below 2^-120).
static __device__ __forceinline__ dfl split_double(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int w1 = (unsigned int)(b >> 32);
  const unsigned int w0 = (unsigned int)b;
  const unsigned int sign = w1 & 0x80000000u;
  const int e = (int)((w1 >> 20) & 0x7FFu);
  const int ef = e - 896;                                   // float biased exponent
  const unsigned int m23 = ((w1 & 0xFFFFFu) << 3) | (w0 >> 29);
  float hi = __uint_as_float(sign | ((unsigned int)ef << 23) | m23);
  hi = (ef > 0) ? hi : 0.0f;
  const unsigned int r = w0 & 0x1FFFFFFFu;                   // low 29 mantissa bits
  // lo = r * 2^(e - 1075): convert r exactly-rounded, then move its exponent field
  const unsigned int rb = __float_as_uint(__uint2float_rn(r));
  const int el = (int)(rb >> 23) + (e - 1075);               // biased exponent of lo
  float lo = __uint_as_float(sign | ((unsigned int)el << 23) | (rb & 0x7FFFFFu));
  lo = (r != 0u && el > 0 && ef > 0) ? lo : 0.0f;
  return {hi, lo};
}

// Join hi + lo (|lo| <= ulp(hi)/2, as produced by the arithmetic below) into a binary64
// with integer operations only: the binary64 pattern of hi plus lo counted in binary64 ulps
// (IEEE patterns are monotonic in magnitude for a fixed sign, so adding k to the pattern
// moves the value by k ulps, across a binade boundary included).
static __device__ __forceinline__ double join_double(float hi, float lo) {
  const unsigned int hb = __float_as_uint(hi);
  const unsigned int sign = hb & 0x80000000u;
  const int ef = (int)((hb >> 23) & 0xFFu);
  if (ef == 0) return 0.0;
  unsigned long long db = ((unsigned long long)(sign | ((unsigned int)(ef + 896) << 20) |
                                                ((hb & 0x7FFFFFu) >> 3)) << 32) |
                          ((unsigned long long)(hb & 7u) << 29);
  const unsigned int lb = __float_as_uint(lo);
  const int el = (int)((lb >> 23) & 0xFFu);
  // lo is counted in binary64 ulps of hi's binade, 2^(ef-179); when hi is a power of two and
  // lo points down, the result lies in the binade below, whose ulp is half as large
  const bool down = ((lb ^ hb) & 0x80000000u) && ((hb & 0x7FFFFFu) == 0u);
  const int ne = el + (down ? 180 : 179) - ef;             // exponent of lo / ulp
  int k = 0;
  if (el != 0 && ne > 0) {
    float ls = __uint_as_float((lb & 0x807FFFFFu) | ((unsigned int)ne << 23));
    k = __float2int_rn(ls);
  }
  long long delta = sign ? -(long long)k : (long long)k;
  db = (unsigned long long)((long long)db + delta);
  return __longlong_as_double((long long)db);
}

// ------------------------------------------------------------------------------------------
// complex128 storage, double-float arithmetic
// reg_t = (re.hi, re.lo, im.hi, im.lo); mat_t the same format (prepared on the host).
// ------------------------------------------------------------------------------------------
struct ADF {
  using store_t = double2;
  using reg_t = float4;
  using mat_t = float4;
  static constexpr int kStoreBytes = 16;
  static __device__ __forceinline__ reg_t from_store(store_t v) {
    dfl r = split_double(v.x), i = split_double(v.y);
    return make_float4(r.hi, r.lo, i.hi, i.lo);
  }
  // register values are kept unnormalised between operations (hi need not be the rounded
  // value of hi + lo); normalise once with TwoSum before the exact integer join
  static __device__ __forceinline__ store_t to_store(reg_t v) {
    const dfl r = two_sum(v.x, v.y), i = two_sum(v.z, v.w);
    return make_double2(join_double(r.hi, r.lo), join_double(i.hi, i.lo));
  }
  static __device__ __forceinline__ reg_t zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }

  // Sum of two products p0 + p1 where p_k = (a_k.hi + a_k.lo) * (b_k.hi + b_k.lo) (signs
  // folded into the a's): TwoProduct of the high parts, first-order cross terms in FP32,
  // TwoSum of the two leading terms.  The result is left unnormalised (lo collects the
  // TwoSum error and the first-order terms, |lo| ~ 2^-22 |hi|); the next operation uses lo
  // only in first-order terms, so accuracy stays near 2^-44 relative, and to_store
  // normalises before converting back to binary64.
  static __device__ __forceinline__ dfl dot2(float a0h, float a0l, float b0h, float b0l,
                                             float a1h, float a1l, float b1h, float b1l) {
    dfl p0 = two_prod(a0h, b0h);
    dfl p1 = two_prod(a1h, b1h);
    float err = __fmaf_rn(a0h, b0l, p0.lo);
    err = __fmaf_rn(a0l, b0h, err);
    err = __fadd_rn(err, p1.lo);
    err = __fmaf_rn(a1h, b1l, err);
    err = __fmaf_rn(a1l, b1h, err);
    dfl s = two_sum(p0.hi, p1.hi);
    return {s.hi, __fadd_rn(s.lo, err)};
  }
  static __device__ __forceinline__ dfl dot4(float a0h, float a0l, float b0h, float b0l,
                                             float a1h, float a1l, float b1h, float b1l,
                                             float a2h, float a2l, float b2h, float b2l,
                                             float a3h, float a3l, float b3h, float b3l) {
    dfl p0 = two_prod(a0h, b0h);
    dfl p1 = two_prod(a1h, b1h);
    dfl p2 = two_prod(a2h, b2h);
    dfl p3 = two_prod(a3h, b3h);
    float err = __fmaf_rn(a0h, b0l, p0.lo);
    err = __fmaf_rn(a0l, b0h, err);
    err = __fadd_rn(err, p1.lo);
    err = __fmaf_rn(a1h, b1l, err);
    err = __fmaf_rn(a1l, b1h, err);
    err = __fadd_rn(err, p2.lo);
    err = __fmaf_rn(a2h, b2l, err);
    err = __fmaf_rn(a2l, b2h, err);
    err = __fadd_rn(err, p3.lo);
    err = __fmaf_rn(a3h, b3l, err);
    err = __fmaf_rn(a3l, b3h, err);
    dfl s01 = two_sum(p0.hi, p1.hi);
    dfl s23 = two_sum(p2.hi, p3.hi);
    dfl s = two_sum(s01.hi, s23.hi);
    err = __fadd_rn(err, __fadd_rn(s01.lo, __fadd_rn(s23.lo, s.lo)));
    return {s.hi, err};
  }
  // acc + u*a (complex)
  static __device__ __forceinline__ reg_t mac(reg_t acc, mat_t u, reg_t a) {
    reg_t p = mul(u, a);
    dfl re = two_sum(acc.x, p.x);
    dfl im = two_sum(acc.z, p.z);
    return make_float4(re.hi, __fadd_rn(re.lo, __fadd_rn(acc.y, p.y)), im.hi, __fadd_rn(im.lo, __fadd_rn(acc.w, p.w)));
  }
  // u*a + v*b: re = u.re a.re - u.im a.im + v.re b.re - v.im b.im, im likewise
  static __device__ __forceinline__ reg_t mac2(mat_t u, reg_t a, mat_t v, reg_t b) {
    dfl re = dot4(u.x, u.y, a.x, a.y, -u.z, -u.w, a.z, a.w,
                  v.x, v.y, b.x, b.y, -v.z, -v.w, b.z, b.w);
    dfl im = dot4(u.x, u.y, a.z, a.w, u.z, u.w, a.x, a.y,
                  v.x, v.y, b.z, b.w, v.z, v.w, b.x, b.y);
    return make_float4(re.hi, re.lo, im.hi, im.lo);
  }
  static __device__ __forceinline__ reg_t mul(mat_t u, reg_t a) {
    dfl re = dot2(u.x, u.y, a.x, a.y, -u.z, -u.w, a.z, a.w);
    dfl im = dot2(u.x, u.y, a.z, a.w, u.z, u.w, a.x, a.y);
    return make_float4(re.hi, re.lo, im.hi, im.lo);
  }
  // c*a - i*s*b with cs = (c.hi, c.lo, s.hi, s.lo): re = c a.re + s b.im, im = c a.im - s b.re
  static __device__ __forceinline__ reg_t rx(mat_t cs, reg_t a, reg_t b) {
    dfl re = dot2(cs.x, cs.y, a.x, a.y, cs.z, cs.w, b.z, b.w);
    dfl im = dot2(cs.x, cs.y, a.z, a.w, -cs.z, -cs.w, b.x, b.y);
    return make_float4(re.hi, re.lo, im.hi, im.lo);
  }
  // u + t v for a real double-float t = (t.x, t.y): TwoProduct of the high parts, the two
  // first-order cross terms, TwoSum with u's high part (12 instructions per component
  // against 16 for a two-term dot product).  Used by the tangent-form RX, which applies
  // (I - i t X) or (t I - i X) and leaves the factor cos or sin to one full-form RX of the
  // pass.
  static __device__ __forceinline__ reg_t axpy(mat_t t, reg_t v, reg_t u) {
    const dfl pr = two_prod(t.x, v.x);
    float er = __fmaf_rn(t.x, v.y, pr.lo);
    er = __fmaf_rn(t.y, v.x, er);
    const dfl sr = two_sum(u.x, pr.hi);
    const dfl pi = two_prod(t.x, v.z);
    float ei = __fmaf_rn(t.x, v.w, pi.lo);
    ei = __fmaf_rn(t.y, v.z, ei);
    const dfl si = two_sum(u.z, pi.hi);
    return make_float4(sr.hi, __fadd_rn(sr.lo, __fadd_rn(u.y, er)), si.hi, __fadd_rn(si.lo, __fadd_rn(u.w, ei)));
  }
  static __device__ __forceinline__ reg_t mul_mi(reg_t b) { return make_float4(b.z, b.w, -b.x, -b.y); }
  static __device__ __forceinline__ reg_t neg(reg_t a) { return make_float4(-a.x, -a.y, -a.z, -a.w); }
  static __device__ __forceinline__ double norm2(reg_t a) {
    double r = (double)a.x + (double)a.y, i = (double)a.z + (double)a.w;
    return r * r + i * i;
  }
};

}  // namespace qs
