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
//       integer bit manipulation so that no instruction touches the FP64 pipe; the real
//       and imaginary lanes run through packed f32x2 instructions.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

namespace qs {

// ------------------------------------------------------------------------------------------
// complex64, FP32
// ------------------------------------------------------------------------------------------
struct AF32 {
  using store_t = float2;
  using reg_t = float2;
  using mat_t = float2;
  static constexpr int kStoreBytes = 8;
  static constexpr bool kFrame = false;
  static __device__ __forceinline__ mat_t ld(const mat_t* p) { return *p; }
  static __device__ __forceinline__ reg_t from_store(store_t v) { return v; }
  static __device__ __forceinline__ store_t to_store(reg_t v) { return v; }
  static __device__ __forceinline__ reg_t from_store_f(store_t v, bool) { return v; }
  static __device__ __forceinline__ store_t to_store_f(reg_t v, bool) { return v; }
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
  static constexpr bool kFrame = false;
  static __device__ __forceinline__ mat_t ld(const mat_t* p) { return *p; }
  static __device__ __forceinline__ reg_t from_store(store_t v) { return v; }
  static __device__ __forceinline__ store_t to_store(reg_t v) { return v; }
  static __device__ __forceinline__ reg_t from_store_f(store_t v, bool) { return v; }
  static __device__ __forceinline__ store_t to_store_f(reg_t v, bool) { return v; }
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
// double-float building blocks (all explicitly rounded: no contraction changes them).
// They are host-callable as well, so that the formulas can be checked on a CPU against
// binary64; on the host the float operations are plain IEEE binary32 with
// round-to-nearest (build with contraction off).
// ------------------------------------------------------------------------------------------
#define QS_HD __host__ __device__ __forceinline__

QS_HD float f_add(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
QS_HD float f_sub(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}
QS_HD float f_mul(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
QS_HD float f_fma(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return fmaf(a, b, c);
#endif
}
QS_HD unsigned int f_bits(float x) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(x);
#else
  unsigned int u;
  memcpy(&u, &x, 4);
  return u;
#endif
}
QS_HD float f_from_bits(unsigned int u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float x;
  memcpy(&x, &u, 4);
  return x;
#endif
}
QS_HD unsigned long long d_bits(double x) {
#ifdef __CUDA_ARCH__
  return (unsigned long long)__double_as_longlong(x);
#else
  unsigned long long u;
  memcpy(&u, &x, 8);
  return u;
#endif
}
QS_HD double d_from_bits(unsigned long long u) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)u);
#else
  double x;
  memcpy(&x, &u, 8);
  return x;
#endif
}
QS_HD float u32_to_f_rn(unsigned int r) {
#ifdef __CUDA_ARCH__
  return __uint2float_rn(r);
#else
  return (float)r;
#endif
}
QS_HD int f_to_i_rn(float x) {
#ifdef __CUDA_ARCH__
  return __float2int_rn(x);
#else
  return (int)lrintf(x);
#endif
}

// Packed lane pairs: one f32x2 instruction (FADD2 / FMUL2 / FFMA2 on sm_100 and later)
// does the same operation on both floats of a 64-bit register pair.
QS_HD float2 add2(float2 a, float2 b) {
#ifdef __CUDA_ARCH__
  return __fadd2_rn(a, b);
#else
  return make_float2(a.x + b.x, a.y + b.y);
#endif
}
QS_HD float2 sub2(float2 a, float2 b) {
#ifdef __CUDA_ARCH__
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\t"
      "mov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rd, ra, rb;\n\t"
      "mov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
#else
  return make_float2(a.x - b.x, a.y - b.y);
#endif
}
QS_HD float2 mul2(float2 a, float2 b) {
#ifdef __CUDA_ARCH__
  return __fmul2_rn(a, b);
#else
  return make_float2(a.x * b.x, a.y * b.y);
#endif
}
QS_HD float2 fma2(float2 a, float2 b, float2 c) {
#ifdef __CUDA_ARCH__
  return __ffma2_rn(a, b, c);
#else
  return make_float2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y));
#endif
}

struct dfl { float hi, lo; };

// s + e == a + b exactly (Knuth TwoSum, 6 flops)
QS_HD dfl two_sum(float a, float b) {
  float s = f_add(a, b);
  float bb = f_sub(s, a);
  float e = f_add(f_sub(a, f_sub(s, bb)), f_sub(b, bb));
  return {s, e};
}
// p + e == a * b exactly (TwoProduct with FMA)
QS_HD dfl two_prod(float a, float b) {
  float p = f_mul(a, b);
  float e = f_fma(a, b, -p);
  return {p, e};
}
// lane-wise TwoSum: s + e == a + b exactly in each lane
QS_HD void two_sum2(float2 a, float2 b, float2& s, float2& e) {
  s = add2(a, b);
  const float2 bb = sub2(s, a);
  e = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
}
// lane-wise TwoSum of a and -b: s + e == a - b exactly
QS_HD void two_diff2(float2 a, float2 b, float2& s, float2& e) {
  s = sub2(a, b);
  const float2 bb = sub2(s, a);
  e = sub2(sub2(a, sub2(s, bb)), add2(b, bb));
}
// Lane-wise double-float product of U = Uh + Ul (given as Uh, -Uh, -Ul) and v = vh + vl:
// p = Uh vh rounded, ne = -(TwoProduct error + Uh vl + Ul vh), so that U v ~= p - ne
// (the product of the low parts, ~2^-48 relative, is dropped).  The negated operands keep
// every step a plain packed FMA: FMA(-Uh, vh, p) is the exact negated TwoProduct error.
QS_HD void prod2(float2 Uh, float2 nUh, float2 nUl, float2 vh, float2 vl, float2& p, float2& ne) {
  p = mul2(Uh, vh);
  ne = fma2(nUh, vh, p);
  ne = fma2(nUh, vl, ne);
  ne = fma2(nUl, vh, ne);
}

// Split a binary64 value into hi + lo floats without FP64 instructions.
// hi keeps the leading 24 significant bits (truncated), lo = x - hi (its 29 bits rounded
// to 24): |x - (hi + lo)| <= 2^-47 |x|.  |x| < 2^-126 flushes to 0 (absolute error
// below 1.2e-38); the lo part flushes when it would leave the normal float range
// (|x| below about 2^-98; absolute error below 2^-120).
QS_HD dfl split_double(double x) {
  const unsigned long long b = d_bits(x);
  const unsigned int w1 = (unsigned int)(b >> 32);
  const unsigned int w0 = (unsigned int)b;
  const unsigned int sign = w1 & 0x80000000u;
  const int e = (int)((w1 >> 20) & 0x7FFu);
  const int ef = e - 896;                                   // float biased exponent
  const unsigned int m23 = ((w1 & 0xFFFFFu) << 3) | (w0 >> 29);
  float hi = f_from_bits(sign | ((unsigned int)ef << 23) | m23);
  hi = (ef > 0) ? hi : 0.0f;
  const unsigned int r = w0 & 0x1FFFFFFFu;                   // low 29 mantissa bits
  // lo = r * 2^(e - 1075): convert r exactly-rounded, then move its exponent field
  const unsigned int rb = f_bits(u32_to_f_rn(r));
  const int el = (int)(rb >> 23) + (e - 1075);               // biased exponent of lo
  float lo = f_from_bits(sign | ((unsigned int)el << 23) | (rb & 0x7FFFFFu));
  lo = (r != 0u && el > 0 && ef > 0) ? lo : 0.0f;
  return {hi, lo};
}

// Join hi + lo (|lo| <= ulp(hi)/2, as produced by the arithmetic below) into a binary64
// with integer operations only: the binary64 pattern of hi plus lo counted in binary64 ulps
// (IEEE patterns are monotonic in magnitude for a fixed sign, so adding k to the pattern
// moves the value by k ulps, across a binade boundary included).
QS_HD double join_double(float hi, float lo) {
  const unsigned int hb = f_bits(hi);
  const unsigned int sign = hb & 0x80000000u;
  const int ef = (int)((hb >> 23) & 0xFFu);
  if (ef == 0) return 0.0;
  unsigned long long db = ((unsigned long long)(sign | ((unsigned int)(ef + 896) << 20) |
                                                ((hb & 0x7FFFFFu) >> 3)) << 32) |
                          ((unsigned long long)(hb & 7u) << 29);
  const unsigned int lb = f_bits(lo);
  const int el = (int)((lb >> 23) & 0xFFu);
  // lo is counted in binary64 ulps of hi's binade, 2^(ef-179); when hi is a power of two and
  // lo points down, the result lies in the binade below, whose ulp is half as large
  const bool down = ((lb ^ hb) & 0x80000000u) && ((hb & 0x7FFFFFu) == 0u);
  const int ne = el + (down ? 180 : 179) - ef;             // exponent of lo / ulp
  int k = 0;
  if (el != 0 && ne > 0) {
    float ls = f_from_bits((lb & 0x807FFFFFu) | ((unsigned int)ne << 23));
    k = f_to_i_rn(ls);
  }
  long long delta = sign ? -(long long)k : (long long)k;
  db = (unsigned long long)((long long)db + delta);
  return d_from_bits(db);
}

// ------------------------------------------------------------------------------------------
// complex128 storage, double-float arithmetic, two lanes per instruction
//
// reg_t = (re.hi, im.hi, re.lo, im.lo): the (re, im) lanes of the high parts and of the
// low parts are each one 64-bit register pair, so each step of the complex arithmetic is
// one packed f32x2 instruction instead of two scalar ones.  Register values are kept
// unnormalised between operations (hi need not be the rounded value of hi + lo);
// to_store normalises once with TwoSum before the exact integer join.
//
// mat_t (48 bytes, prepared on the host) holds a complex u = ur + i ui as lane patterns:
//   a = ( ur.hi,  ur.hi, -ur.hi, -ur.hi)     ur on both lanes, and its negation
//   b = (-ui.hi,  ui.hi,  ui.hi, -ui.hi)     (-ui, ui): i ui acting on a swapped (im, re)
//   c = (-ur.lo, -ur.lo,  ui.lo, -ui.lo)     negated low parts of both patterns
// so that u a = ur (.) a + (-ui, ui) (.) swap(a) lane-wise and no packed operand needs a
// sign flip at run time.
//
// Tile passes run in a phase frame: amplitude i of a tile is held as (-i)^popcount(i)
// times its value (S^dagger on every tile bit).  Diagonal gates are unchanged, RX becomes
// the real rotation [[c, s], [-s, c]] (no lane swaps at all), X becomes [[0, i], [-i, 0]],
// and the host transforms the matrices of general gates (entry (r, c) times
// (-i)^(popcount r - popcount c)).  The per-gate kernels use the plain frame.
// ------------------------------------------------------------------------------------------
struct alignas(16) dfm {
  float4 a, b, c;
};
// a real double-float factor t as the three lane pairs the products need: (t.hi, t.hi),
// its negation, and the negated low part
struct dfr {
  float2 h, nh, nl;
};

struct ADF {
  using store_t = double2;
  using reg_t = float4;
  using mat_t = dfm;
  static constexpr int kStoreBytes = 16;
  static constexpr bool kFrame = true;

  static QS_HD float2 hi(reg_t v) { return make_float2(v.x, v.y); }
  static QS_HD float2 lo(reg_t v) { return make_float2(v.z, v.w); }
  static QS_HD float2 swp(float2 v) { return make_float2(v.y, v.x); }
  static QS_HD reg_t mk(float2 h, float2 l) { return make_float4(h.x, h.y, l.x, l.y); }

  // A 48-byte entry loaded where it is used: the loads are volatile so that the compiler
  // cannot hoist the entries of a whole matrix out of a loop (12 registers each).
  static QS_HD mat_t ld(const mat_t* p) {
#ifdef __CUDA_ARCH__
    mat_t m;
    asm volatile("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(m.a.x), "=f"(m.a.y), "=f"(m.a.z), "=f"(m.a.w) : "l"(p));
    asm volatile("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4+16];"
                 : "=f"(m.b.x), "=f"(m.b.y), "=f"(m.b.z), "=f"(m.b.w) : "l"(p));
    asm volatile("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4+32];"
                 : "=f"(m.c.x), "=f"(m.c.y), "=f"(m.c.z), "=f"(m.c.w) : "l"(p));
    return m;
#else
    return *p;
#endif
  }
  // the real part of an entry (t, 0): two of its three 16-byte words
  static QS_HD dfr ld_real(const mat_t* p) {
#ifdef __CUDA_ARCH__
    float4 a, c;
    asm volatile("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w) : "l"(p));
    asm volatile("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4+32];" : "=f"(c.x), "=f"(c.y), "=f"(c.z), "=f"(c.w) : "l"(p));
    return dfr{make_float2(a.x, a.y), make_float2(a.z, a.w), make_float2(c.x, c.y)};
#else
    return real_of(*p);
#endif
  }
  static QS_HD dfr real_of(const mat_t& m) {
    return dfr{make_float2(m.a.x, m.a.y), make_float2(m.a.z, m.a.w), make_float2(m.c.x, m.c.y)};
  }
  static QS_HD reg_t from_store(store_t v) {
    const dfl r = split_double(v.x), i = split_double(v.y);
    return make_float4(r.hi, i.hi, r.lo, i.lo);
  }
  static QS_HD store_t to_store(reg_t v) {
    const dfl r = two_sum(v.x, v.z), i = two_sum(v.y, v.w);
    return make_double2(join_double(r.hi, r.lo), join_double(i.hi, i.lo));
  }
  // The double-float storage form a plan keeps between consecutive tile passes: the four
  // floats of a normalised register value in the 16 bytes of an element (no binary64
  // split or join).  It exists only inside one plan execution; the state holds binary64
  // before and after.
  static QS_HD reg_t from_df(store_t v) {
    const unsigned long long a = d_bits(v.x), b = d_bits(v.y);
    return make_float4(f_from_bits((unsigned int)a), f_from_bits((unsigned int)(a >> 32)),
                       f_from_bits((unsigned int)b), f_from_bits((unsigned int)(b >> 32)));
  }
  static QS_HD store_t to_df(reg_t v) {
    float2 s, e;
    two_sum2(hi(v), lo(v), s, e);
    return make_double2(d_from_bits(((unsigned long long)f_bits(s.y) << 32) | f_bits(s.x)),
                        d_from_bits(((unsigned long long)f_bits(e.y) << 32) | f_bits(e.x)));
  }
  static QS_HD reg_t from_store_f(store_t v, bool df) { return df ? from_df(v) : from_store(v); }
  static QS_HD store_t to_store_f(reg_t v, bool df) { return df ? to_df(v) : to_store(v); }
  static QS_HD reg_t zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }

  // u a
  static QS_HD reg_t mul(const mat_t& u, reg_t a) {
    float2 p1, n1, p2, n2, s, e;
    prod2(make_float2(u.a.x, u.a.y), make_float2(u.a.z, u.a.w), make_float2(u.c.x, u.c.y), hi(a), lo(a), p1, n1);
    prod2(make_float2(u.b.x, u.b.y), make_float2(u.b.z, u.b.w), make_float2(u.c.z, u.c.w), swp(hi(a)), swp(lo(a)),
          p2, n2);
    two_sum2(p1, p2, s, e);
    return mk(s, sub2(e, add2(n1, n2)));
  }
  static QS_HD reg_t add(reg_t x, reg_t y) {
    float2 s, e;
    two_sum2(hi(x), hi(y), s, e);
    return mk(s, add2(e, add2(lo(x), lo(y))));
  }
  // acc + u a
  static QS_HD reg_t mac(reg_t acc, const mat_t& u, reg_t a) { return add(acc, mul(u, a)); }
  // u a + v b
  static QS_HD reg_t mac2(const mat_t& u, reg_t a, const mat_t& v, reg_t b) { return add(mul(u, a), mul(v, b)); }
  // c a - i s b for cs = (c, s), plain frame: c (.) a + (s, -s) (.) swap(b), and (s, -s) is
  // the negated (-ui, ui) pattern of the entry
  static QS_HD reg_t rx(const mat_t& cs, reg_t a, reg_t b) {
    float2 p1, n1, p2, n2, s, e;
    prod2(make_float2(cs.a.x, cs.a.y), make_float2(cs.a.z, cs.a.w), make_float2(cs.c.x, cs.c.y), hi(a), lo(a), p1, n1);
    prod2(make_float2(cs.b.x, cs.b.y), make_float2(cs.b.z, cs.b.w), make_float2(cs.c.z, cs.c.w), swp(hi(b)),
          swp(lo(b)), p2, n2);
    two_diff2(p1, p2, s, e);   // (p1 - n1) - (p2 - n2)
    return mk(s, add2(e, sub2(n2, n1)));
  }

  // ---- phase-frame updates with a real double-float factor t
  // u + t v
  static QS_HD reg_t axpy_r(const dfr& t, reg_t v, reg_t u) {
    float2 p, n, s, e;
    prod2(t.h, t.nh, t.nl, hi(v), lo(v), p, n);
    two_sum2(hi(u), p, s, e);
    return mk(s, add2(e, sub2(lo(u), n)));
  }
  // u - t v
  static QS_HD reg_t axmy_r(const dfr& t, reg_t v, reg_t u) {
    float2 p, n, s, e;
    prod2(t.h, t.nh, t.nl, hi(v), lo(v), p, n);
    two_diff2(hi(u), p, s, e);
    return mk(s, add2(e, add2(lo(u), n)));
  }
  // t v - u
  static QS_HD reg_t ymx_r(const dfr& t, reg_t v, reg_t u) {
    float2 p, n, s, e;
    prod2(t.h, t.nh, t.nl, hi(v), lo(v), p, n);
    two_diff2(p, hi(u), s, e);
    return mk(s, sub2(e, add2(n, lo(u))));
  }
  // (a, b) -> (c a + s b, c b - s a) with real c and s
  static QS_HD void rot_r(const dfr& c, const dfr& sn, reg_t a, reg_t b, reg_t& a2, reg_t& b2) {
    const float2 ch = c.h, nch = c.nh, ncl = c.nl;
    const float2 sh = sn.h, nsh = sn.nh, nsl = sn.nl;
    float2 p1, n1, p2, n2, s, e;
    prod2(ch, nch, ncl, hi(a), lo(a), p1, n1);
    prod2(sh, nsh, nsl, hi(b), lo(b), p2, n2);
    two_sum2(p1, p2, s, e);
    const reg_t ra = mk(s, sub2(e, add2(n1, n2)));
    prod2(ch, nch, ncl, hi(b), lo(b), p1, n1);
    prod2(sh, nsh, nsl, hi(a), lo(a), p2, n2);
    two_diff2(p1, p2, s, e);
    b2 = mk(s, add2(e, sub2(n2, n1)));
    a2 = ra;
  }
  // v (-i)^q, exact (a lane swap and sign flips); q in 0..3
  static QS_HD reg_t rot_q(reg_t v, unsigned int q) {
    const bool sw = (q & 1u) != 0u;
    const float r0 = sw ? v.y : v.x, r1 = sw ? v.x : v.y, l0 = sw ? v.w : v.z, l1 = sw ? v.z : v.w;
    const unsigned int n0 = (q >> 1) << 31, n1 = ((q ^ (q >> 1)) & 1u) << 31;
    return make_float4(f_from_bits(f_bits(r0) ^ n0), f_from_bits(f_bits(r1) ^ n1), f_from_bits(f_bits(l0) ^ n0),
                       f_from_bits(f_bits(l1) ^ n1));
  }
  static QS_HD reg_t neg(reg_t a) { return make_float4(-a.x, -a.y, -a.z, -a.w); }
  static QS_HD double norm2(reg_t a) {
    double r = (double)a.x + (double)a.z, i = (double)a.y + (double)a.w;
    return r * r + i * i;
  }
};

}  // namespace qs
