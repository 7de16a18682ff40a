// sun_device.cuh -- device primitives of the SU(Nc) link sweep (sm_103a).
//
// Complex Nc x Nc matrices in registers, SU(2) quaternions (Eq. 6 of
// Cardoso & Bicudo, arXiv:1112.4533), Philox4x32-10 (Salmon et al., SC'11),
// the Kennedy-Pendleton / Creutz draws of the SU(2) heatbath (Eqs. 12-13),
// structure-of-arrays link storage and even/odd site indexing.
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

#include "sun_runtime.h"

namespace sun {

// ------------------------------------------------------------------ math ----
__device__ __forceinline__ float d_log(float x) { return logf(x); }
__device__ __forceinline__ double d_log(double x) { return log(x); }
__device__ __forceinline__ float d_log1p(float x) { return log1pf(x); }
__device__ __forceinline__ double d_log1p(double x) { return log1p(x); }
__device__ __forceinline__ float d_expm1(float x) { return expm1f(x); }
__device__ __forceinline__ double d_expm1(double x) { return expm1(x); }
__device__ __forceinline__ float d_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double d_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float d_cospi(float x) { return cospif(x); }
__device__ __forceinline__ double d_cospi(double x) { return cospi(x); }
__device__ __forceinline__ void d_sincospi(float x, float* s, float* c) { sincospif(x, s, c); }
__device__ __forceinline__ void d_sincospi(double x, double* s, double* c) { sincospi(x, s, c); }
__device__ __forceinline__ bool d_isfinite(float x) { return isfinite(x); }
__device__ __forceinline__ bool d_isfinite(double x) { return isfinite(x); }

// --------------------------------------------------------------- complex ----
template <class R>
struct Cpx {
  R re, im;
};

// The library is compiled without floating-point contraction (-fmad=false), so
// every kernel that inlines these helpers rounds identically; the products
// below spell out their fused multiply-adds.
template <class R>
__device__ __forceinline__ Cpx<R> cmul(Cpx<R> a, Cpx<R> b) {
  return {fma(a.re, b.re, -(a.im * b.im)), fma(a.re, b.im, a.im * b.re)};
}
// a * conj(b)
template <class R>
__device__ __forceinline__ Cpx<R> cmulc(Cpx<R> a, Cpx<R> b) {
  return {fma(a.re, b.re, a.im * b.im), fma(a.im, b.re, -(a.re * b.im))};
}
// conj(a) * b
template <class R>
__device__ __forceinline__ Cpx<R> ccmul(Cpx<R> a, Cpx<R> b) {
  return {fma(a.re, b.re, a.im * b.im), fma(a.re, b.im, -(a.im * b.re))};
}
// acc += a * b
template <class R>
__device__ __forceinline__ void cfma(Cpx<R>& acc, Cpx<R> a, Cpx<R> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
}
// acc += a * conj(b)
template <class R>
__device__ __forceinline__ void cfmac(Cpx<R>& acc, Cpx<R> a, Cpx<R> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.im, b.re, acc.im);
  acc.im = fma(-a.re, b.im, acc.im);
}
// acc += conj(a) * b
template <class R>
__device__ __forceinline__ void ccfma(Cpx<R>& acc, Cpx<R> a, Cpx<R> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
}

// ----------------------------------------------------- packed FP32 pairs ----
// Two FP32 values handled by one packed instruction ({add,sub,mul,fma}.rn.f32x2,
// sm_100 and later): each lane is the same IEEE round-to-nearest operation as
// the float one, so code written for a real type R and run with R = F2 computes
// two independent problems (two links) with the results of the float code for
// each, in half the arithmetic instructions.
struct F2 {
  unsigned long long v;
  F2() = default;
  __device__ __forceinline__ explicit F2(float s) { asm("mov.b64 %0, {%1, %1};" : "=l"(v) : "f"(s)); }
};

using ::fma;  // the float and double overloads stay visible beside the F2 one

__device__ __forceinline__ F2 f2_pack(float lo, float hi) {
  F2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void f2_unpack(F2 a, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a.v));
}
__device__ __forceinline__ F2 operator+(F2 a, F2 b) {
  F2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ F2 operator-(F2 a, F2 b) {
  F2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ F2 operator*(F2 a, F2 b) {
  F2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
// negation flips the two sign bits (exact, as float negation)
__device__ __forceinline__ F2 operator-(F2 a) {
  F2 r;
  r.v = a.v ^ 0x8000000080000000ull;
  return r;
}
__device__ __forceinline__ F2 fma(F2 a, F2 b, F2 c) {
  F2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
  return r;
}

// -------------------------------------------------------------- matrices ----
template <class R, int N>
struct Mat {
  Cpx<R> e[N][N];
};

template <class R, int N>
__device__ __forceinline__ void mat_zero(Mat<R, N>& a) {
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) a.e[i][j] = {R(0), R(0)};
}

template <class R, int N>
__device__ __forceinline__ void mat_identity(Mat<R, N>& a) {
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) a.e[i][j] = {R(i == j ? 1 : 0), R(0)};
}

// C = A B
template <class R, int N>
__device__ __forceinline__ Mat<R, N> mul_nn(const Mat<R, N>& a, const Mat<R, N>& b) {
  Mat<R, N> c;
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) {
      Cpx<R> s = cmul(a.e[i][0], b.e[0][j]);
#pragma unroll
      for (int k = 1; k < N; ++k) cfma(s, a.e[i][k], b.e[k][j]);
      c.e[i][j] = s;
    }
  return c;
}

// C += A B^+
template <class R, int N>
__device__ __forceinline__ void acc_nd(Mat<R, N>& c, const Mat<R, N>& a, const Mat<R, N>& b) {
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j)
#pragma unroll
      for (int k = 0; k < N; ++k) cfmac(c.e[i][j], a.e[i][k], b.e[j][k]);
}

// C += A B
template <class R, int N>
__device__ __forceinline__ void acc_nn(Mat<R, N>& c, const Mat<R, N>& a, const Mat<R, N>& b) {
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j)
#pragma unroll
      for (int k = 0; k < N; ++k) cfma(c.e[i][j], a.e[i][k], b.e[k][j]);
}

// C = A^+ B
template <class R, int N>
__device__ __forceinline__ Mat<R, N> mul_dn(const Mat<R, N>& a, const Mat<R, N>& b) {
  Mat<R, N> c;
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) {
      Cpx<R> s = ccmul(a.e[0][i], b.e[0][j]);
#pragma unroll
      for (int k = 1; k < N; ++k) ccfma(s, a.e[k][i], b.e[k][j]);
      c.e[i][j] = s;
    }
  return c;
}

// C = A B^+
template <class R, int N>
__device__ __forceinline__ Mat<R, N> mul_nd(const Mat<R, N>& a, const Mat<R, N>& b) {
  Mat<R, N> c;
  mat_zero(c);
  acc_nd(c, a, b);
  return c;
}

// Re Tr(A B^+) = sum_ij Re(a_ij conj(b_ij))
template <class R, int N>
__device__ __forceinline__ R retr_nd(const Mat<R, N>& a, const Mat<R, N>& b) {
  R s = R(0);
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) {
      s = fma(a.e[i][j].re, b.e[i][j].re, s);
      s = fma(a.e[i][j].im, b.e[i][j].im, s);
    }
  return s;
}

// conj(a_k b_l - a_l b_k), entry (k, l) of conj(a x b), plus acc: each part is
// one chain of fused multiply-adds started from acc
template <class R>
__device__ __forceinline__ Cpx<R> conj_cross_acc(Cpx<R> ak, Cpx<R> bl, Cpx<R> al, Cpx<R> bk, Cpx<R> acc) {
  R re = fma(ak.re, bl.re, acc.re);
  re = fma(-ak.im, bl.im, re);
  re = fma(-al.re, bk.re, re);
  re = fma(al.im, bk.im, re);
  R im = fma(-ak.re, bl.im, acc.im);
  im = fma(-ak.im, bl.re, im);
  im = fma(al.re, bk.im, im);
  im = fma(al.im, bk.re, im);
  return {re, im};
}

// conj(a_k b_l - a_l b_k) alone: the chains start from the first product
template <class R>
__device__ __forceinline__ Cpx<R> conj_cross(Cpx<R> ak, Cpx<R> bl, Cpx<R> al, Cpx<R> bk) {
  R re = ak.re * bl.re;
  re = fma(-ak.im, bl.im, re);
  re = fma(-al.re, bk.re, re);
  re = fma(al.im, bk.im, re);
  R im = -(ak.re * bl.im);
  im = fma(-ak.im, bl.re, im);
  im = fma(al.re, bk.im, im);
  im = fma(al.im, bk.re, im);
  return {re, im};
}

// row 2 of an SU(3) matrix from rows 0 and 1: conj(row0 x row1)
template <class R>
__device__ __forceinline__ void su3_third_row(Mat<R, 3>& m) {
  const Cpx<R>* a = m.e[0];
  const Cpx<R>* b = m.e[1];
  m.e[2][0] = conj_cross(a[1], b[2], a[2], b[1]);
  m.e[2][1] = conj_cross(a[2], b[0], a[0], b[2]);
  m.e[2][2] = conj_cross(a[0], b[1], a[1], b[0]);
}

// ------------------------------------------- FP32 <-> FP64 conversions ----
// GB300 converts between FP32 and FP64 at its FP64 rate: about 2 conversions a
// clock per SM, the rate of its FP64 FMAs, against about 118 FP32 FMAs
// (measured).  to_f64 and to_f32 do these conversions with integer operations on
// the IEEE 754 binary32 and binary64 encodings (sign, biased exponent, fraction),
// and return exactly the hardware's result for every operand
// (sun_selftest_conversions checks this bit for bit).
//
// float -> double is exact: the fraction is extended by 29 zero bits and the
// exponent rebiased from 127 to 1023.  Every case is taken by selects, with no
// branch: +-0 keeps exponent 0; a subnormal float m 2^-149 is normalised (its top
// fraction bit p becomes the hidden bit, exponent p + 874); infinities keep a zero
// fraction and NaNs their payload with the quiet bit set, as the hardware does.
// A branch to the hardware conversion for the rare cases was if-converted by the
// compiler, which then issued that conversion for every operand.
__device__ __forceinline__ double to_f64(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t e = (b >> 23) & 0xffu;
  const uint32_t m = b & 0x007fffffu;
  const uint32_t p = 31u - uint32_t(__clz(m | 1u));  // top set bit of a subnormal's fraction
  uint32_t ed = e == 0u ? (m == 0u ? 0u : p + 874u) : (e == 0xffu ? 0x7ffu : e + 896u);
  uint32_t fr = e == 0u ? (m << (23u - p)) & 0x007fffffu : m;
  fr = (e == 0xffu && m != 0u) ? (fr | 0x00400000u) : fr;
  const uint32_t hi = (b & 0x80000000u) | (ed << 20) | (fr >> 3);
  return __hiloint2double(int(hi), int(fr << 29));
}
__device__ __forceinline__ double to_f64(double d) { return d; }

// double -> float keeps the top 23 fraction bits and rounds to nearest, ties to
// even, on the 29 bits dropped (a carry out of the fraction raises the exponent,
// 254 -> 255 being the overflow to infinity).  Doubles whose float is subnormal,
// infinite or NaN go to the hardware conversion in a function of its own, so that
// the common path issues no FP64-pipe instruction.
static __device__ __noinline__ float to_f32_rare(double d) { return float(d); }
__device__ __forceinline__ float to_f32(double d) {
  const uint32_t hi = uint32_t(__double2hiint(d)), lo = uint32_t(__double2loint(d));
  const uint32_t e = (hi >> 20) & 0x7ffu;
  if (e - 897u < 254u) {  // the float is normal before rounding: exponent e - 896 in [1, 254]
    uint32_t f = (hi & 0x80000000u) | ((e - 896u) << 23) | ((hi & 0x000fffffu) << 3) | (lo >> 29);
    const uint32_t rest = lo & 0x1fffffffu;
    f += (rest > 0x10000000u || (rest == 0x10000000u && (f & 1u) != 0u)) ? 1u : 0u;
    return __uint_as_float(f);
  }
  if (((hi << 1) | lo) == 0u) return __uint_as_float(hi & 0x80000000u);  // +-0
  return to_f32_rare(d);
}
__device__ __forceinline__ float to_f32(float f) { return f; }

// conversion between the storage and the FP64 working precision
template <class B>
__device__ __forceinline__ B convert_to(float x) {
  if constexpr (std::is_same<B, double>::value) return to_f64(x);
  else return B(x);
}
template <class B>
__device__ __forceinline__ B convert_to(double x) {
  if constexpr (std::is_same<B, float>::value) return to_f32(x);
  else return B(x);
}

// ------------------------------------------------------------ quaternions ----
// q = (a0, a1, a2, a3) <-> a0 1 + i (a1 s1 + a2 s2 + a3 s3)
//   = [[a0 + i a3, a2 + i a1], [-a2 + i a1, a0 - i a3]]
template <class R>
struct Quat {
  R a0, a1, a2, a3;
};

// product p q of the matrices p, q
template <class R>
__device__ __forceinline__ Quat<R> qmul(Quat<R> p, Quat<R> q) {
  // r0 = p0 q0 - p.q ; r = p0 q + q0 p - p x q
  Quat<R> r;
  r.a0 = fma(p.a0, q.a0, -fma(p.a1, q.a1, fma(p.a2, q.a2, p.a3 * q.a3)));
  r.a1 = fma(p.a0, q.a1, fma(q.a0, p.a1, fma(p.a3, q.a2, -(p.a2 * q.a3))));
  r.a2 = fma(p.a0, q.a2, fma(q.a0, p.a2, fma(p.a1, q.a3, -(p.a3 * q.a1))));
  r.a3 = fma(p.a0, q.a3, fma(q.a0, p.a3, fma(p.a2, q.a1, -(p.a1 * q.a2))));
  return r;
}
template <class R>
__device__ __forceinline__ Quat<R> qdag(Quat<R> p) {
  return {p.a0, -p.a1, -p.a2, -p.a3};
}
template <class R>
__device__ __forceinline__ Quat<R> qadd(Quat<R> p, Quat<R> q) {
  return {p.a0 + q.a0, p.a1 + q.a1, p.a2 + q.a2, p.a3 + q.a3};
}

// Overrelaxation element of one subgroup (Eq. 17), A = (vhat^+)^2, from v = c vhat
// (any c > 0) with n3 = |v_vec|^2 and k2 = v0^2 + n3.  A quaternion q = (q0, q)
// squares to (q0^2 - |q|^2, 2 q0 q), so with v^+ = (v0, -v_vec)
//   A = ((v0^2 - n3) / k2, -2 v0 v_vec / k2):
// no square root and one division; the scale c cancels, and a power-of-two c
// gives bitwise the same A.
template <class R>
__device__ __forceinline__ Quat<R> or_element(const Quat<R>& v, R n3, R k2) {
  const R inv = R(1) / k2;
  const R c = -(v.a0 + v.a0) * inv;
  return {fma(v.a0, v.a0, -n3) * inv, c * v.a1, c * v.a2, c * v.a3};
}

// projection of a 2x2 block [[w00, w01], [w10, w11]] onto the real span of SU(2)
template <class R>
__device__ __forceinline__ Quat<R> block_to_quat(Cpx<R> w00, Cpx<R> w01, Cpx<R> w10, Cpx<R> w11) {
  Quat<R> v;
  v.a0 = R(0.5) * (w00.re + w11.re);
  v.a3 = R(0.5) * (w00.im - w11.im);
  v.a1 = R(0.5) * (w01.im + w10.im);
  v.a2 = R(0.5) * (w01.re - w10.re);
  return v;
}
// twice that projection (exactly: no factor 1/2), for or_element
template <class R>
__device__ __forceinline__ Quat<R> block_to_quat2(Cpx<R> w00, Cpx<R> w01, Cpx<R> w10, Cpx<R> w11) {
  return {w00.re + w11.re, w01.im + w10.im, w01.re - w10.re, w00.im - w11.im};
}

// ---------------------------------------------------------------- Philox ----
// Philox4x32-10: ten rounds, multipliers 0xD2511F53 / 0xCD9E8D57, key bumped by
// the Weyl constants 0x9E3779B9 / 0xBB67AE85 before every round but the first.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// uniform in (0,1) with 2^23 levels, exact in float and double
template <class R>
__device__ __forceinline__ R u01(uint32_t u) {
  return (R(u >> 9) + R(0.5)) * R(1.1920928955078125e-07);
}

constexpr int kHeatbathAttempts = 64;
constexpr uint32_t kTagHeatbath = 1u;
constexpr uint32_t kTagInit = 2u;

// SU(2) heatbath element b with density sqrt(1-b0^2) exp(alpha b0) on b0 and an
// isotropic vector part of length sqrt(1-b0^2).  Kennedy-Pendleton draws
// delta = (1-b0)/2 from Gamma(3/2, 2 alpha) and accepts with sqrt(1-delta);
// below alpha = 1.5 Creutz inverts exp(alpha b0) and accepts with
// sqrt(1-b0^2).  Returns false (b untouched) after 64 rejected attempts.
// Not inlined: one copy of the draw serves all Nc(Nc-1)/2 subgroups of a pass
// (measured: the inlined copies of an SU(3) heatbath pass stalled on instruction
// fetch; 0.828 -> 0.808 ms at 48^3 x 96, the same arithmetic).
template <class R>
__device__ __noinline__ bool heatbath_su2(R alpha, uint2 key, uint32_t link, uint32_t step,
                                          uint32_t sub, Quat<R>& b) {
  R b0 = R(1);
  bool ok = false;
  if (alpha >= R(1.5)) {
    const R inv2a = R(1) / (R(2) * alpha);
    for (int att = 0; att < kHeatbathAttempts; ++att) {
      const uint4 u = philox4x32_10(make_uint4(link, step, (sub << 16) | uint32_t(att), kTagHeatbath), key);
      const R r0 = u01<R>(u.x), r1 = u01<R>(u.y), r2 = u01<R>(u.z), r3 = u01<R>(u.w);
      const R c = d_cospi(R(2) * r1);
      const R delta = -(d_log(r0) + c * c * d_log(r2)) * inv2a;
      if (r3 * r3 <= R(1) - delta) {
        b0 = R(1) - R(2) * delta;
        ok = true;
        break;
      }
    }
  } else {
    const R e = -d_expm1(R(-2) * alpha);
    for (int att = 0; att < kHeatbathAttempts; ++att) {
      const uint4 u = philox4x32_10(make_uint4(link, step, (sub << 16) | uint32_t(att), kTagHeatbath), key);
      const R r0 = u01<R>(u.x), r1 = u01<R>(u.y);
      // alpha = 0 (beta = 0): the limit of the inversion, 1 - 2 r0
      const R x = alpha > R(0) ? R(1) + d_log1p(-r0 * e) / alpha : R(1) - R(2) * r0;
      if (r1 * r1 <= R(1) - x * x) {
        b0 = x;
        ok = true;
        break;
      }
    }
  }
  if (!ok) return false;
  const uint4 u = philox4x32_10(make_uint4(link, step, (sub << 16) | uint32_t(kHeatbathAttempts), kTagHeatbath), key);
  const R cth = R(2) * u01<R>(u.x) - R(1);
  const R sth = d_sqrt(R(1) - cth * cth);
  R sphi, cphi;
  d_sincospi(R(2) * u01<R>(u.y), &sphi, &cphi);
  const R rho = d_sqrt(fmax(R(0), R(1) - b0 * b0));
  b.a0 = b0;
  b.a1 = rho * sth * cphi;
  b.a2 = rho * sth * sphi;
  b.a3 = rho * cth;
  return true;
}

// --------------------------------------------------------------- storage ----
// Links of one (direction, parity) block are stored as structure of arrays:
// component vectors of 16 bytes (float4 / double2), each array Vh long, then
// (float storage with 2 mod 4 reals) one array of float2.
enum StoreKind { kQuat = 0, kFull = 1, kTwoRow = 2 };

template <class R, int N, int S>
struct Layout {
  static constexpr int nreals = S == kQuat ? 4 : (S == kTwoRow ? 12 : 2 * N * N);
  static constexpr int bytes = nreals * int(sizeof(R));
  static constexpr int per16 = 16 / int(sizeof(R));
  static constexpr int n16 = nreals / per16;
  static constexpr bool tail = (nreals % per16) != 0;
};

template <class R>
struct Vec16;
template <>
struct Vec16<float> {
  using T = float4;
};
template <>
struct Vec16<double> {
  using T = double2;
};

__device__ __forceinline__ void unpack(float4 v, float* r) { r[0] = v.x; r[1] = v.y; r[2] = v.z; r[3] = v.w; }
__device__ __forceinline__ void unpack(double2 v, double* r) { r[0] = v.x; r[1] = v.y; }
__device__ __forceinline__ float4 pack4(const float* r) { return make_float4(r[0], r[1], r[2], r[3]); }
__device__ __forceinline__ double2 pack4(const double* r) { return make_double2(r[0], r[1]); }

// How a link is loaded: kLoadPlain (ld.global), kLoadNc (read-only data path,
// only for links no thread writes while the kernel runs), kLoadCg (cached in L2
// only: links another block of the same kernel may have written before a
// synchronisation)
enum LoadKind { kLoadPlain = 0, kLoadNc = 1, kLoadCg = 2 };

template <class V>
__device__ __forceinline__ V load_as(const V* p, int kind) {
  return kind == kLoadNc ? __ldg(p) : (kind == kLoadCg ? __ldcg(p) : *p);
}

// read the stored reals of half-site h of a block
template <class R, int NR, int kLoad>
__device__ __forceinline__ void load_reals(const char* __restrict__ blk, int64_t Vh, int64_t h, R (&r)[NR]) {
  constexpr int per16 = 16 / int(sizeof(R));
  constexpr int n16 = NR / per16;
  using V = typename Vec16<R>::T;
#pragma unroll
  for (int c = 0; c < n16; ++c) {
    const V* p = reinterpret_cast<const V*>(blk + (int64_t(c) * Vh + h) * 16);
    V v = load_as(p, kLoad);
    unpack(v, &r[c * per16]);
  }
  if constexpr (NR % per16 != 0) {
    const float2* p = reinterpret_cast<const float2*>(blk + int64_t(n16) * Vh * 16 + h * 8);
    float2 v = load_as(p, kLoad);
    r[NR - 2] = v.x;
    r[NR - 1] = v.y;
  }
}

template <class R, int NR>
__device__ __forceinline__ void store_reals(char* blk, int64_t Vh, int64_t h, const R (&r)[NR]) {
  constexpr int per16 = 16 / int(sizeof(R));
  constexpr int n16 = NR / per16;
  using V = typename Vec16<R>::T;
#pragma unroll
  for (int c = 0; c < n16; ++c) {
    V* p = reinterpret_cast<V*>(blk + (int64_t(c) * Vh + h) * 16);
    *p = pack4(&r[c * per16]);
  }
  if constexpr (NR % per16 != 0) {
    float2* p = reinterpret_cast<float2*>(blk + int64_t(n16) * Vh * 16 + h * 8);
    *p = make_float2(r[NR - 2], r[NR - 1]);
  }
}

// stored reals <-> matrix (full: row-major re,im; two-row: rows 0,1 then row 2 rebuilt)
template <class R, int N, int S>
__device__ __forceinline__ void reals_to_mat(const R (&r)[Layout<R, N, S>::nreals], Mat<R, N>& m) {
  if constexpr (S == kQuat) {
    // [[a0 + i a3, a2 + i a1], [-a2 + i a1, a0 - i a3]]
    m.e[0][0] = {r[0], r[3]};
    m.e[0][1] = {r[2], r[1]};
    m.e[1][0] = {-r[2], r[1]};
    m.e[1][1] = {r[0], -r[3]};
  } else if constexpr (S == kTwoRow) {
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) m.e[i][j] = {r[2 * (3 * i + j)], r[2 * (3 * i + j) + 1]};
    su3_third_row(m);
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
      for (int j = 0; j < N; ++j) m.e[i][j] = {r[2 * (N * i + j)], r[2 * (N * i + j) + 1]};
  }
}

template <class R, int N, int S>
__device__ __forceinline__ void mat_to_reals(const Mat<R, N>& m, R (&r)[Layout<R, N, S>::nreals]) {
  if constexpr (S == kQuat) {
    r[0] = m.e[0][0].re;
    r[3] = m.e[0][0].im;
    r[2] = m.e[0][1].re;
    r[1] = m.e[0][1].im;
  } else {
    constexpr int rows = S == kTwoRow ? 2 : N;
#pragma unroll
    for (int i = 0; i < rows; ++i)
#pragma unroll
      for (int j = 0; j < N; ++j) {
        r[2 * (N * i + j)] = m.e[i][j].re;
        r[2 * (N * i + j) + 1] = m.e[i][j].im;
      }
  }
}

template <class R, int N, int S, int kLoad = kLoadNc>
__device__ __forceinline__ Mat<R, N> load_mat(const char* blk, int64_t Vh, int64_t h) {
  R r[Layout<R, N, S>::nreals];
  load_reals<R, Layout<R, N, S>::nreals, kLoad>(blk, Vh, h, r);
  Mat<R, N> m;
  reals_to_mat<R, N, S>(r, m);
  return m;
}

template <class R, int N, int S>
__device__ __forceinline__ void store_mat(char* blk, int64_t Vh, int64_t h, const Mat<R, N>& m) {
  R r[Layout<R, N, S>::nreals];
  mat_to_reals<R, N, S>(m, r);
  store_reals<R, Layout<R, N, S>::nreals>(blk, Vh, h, r);
}

template <class R, int kLoad = kLoadNc>
__device__ __forceinline__ Quat<R> load_quat(const char* blk, int64_t Vh, int64_t h) {
  R r[4];
  load_reals<R, 4, kLoad>(blk, Vh, h, r);
  return {r[0], r[1], r[2], r[3]};
}

template <class R>
__device__ __forceinline__ void store_quat(char* blk, int64_t Vh, int64_t h, Quat<R> q) {
  const R r[4] = {q.a0, q.a1, q.a2, q.a3};
  store_reals<R, 4>(blk, Vh, h, r);
}

// -------------------------------------------------------------- geometry ----
// Even/odd ordering: site (x,y,z,t), lex = x + Nx(y + Ny(z + Nz t)), lives in the
// block of its parity (x+y+z+t)&1 at half index lex >> 1 (Nx is even).
struct Site {
  int c[4];      // x, y, z, t
  int64_t lex;
};

__device__ __forceinline__ uint32_t fdiv(const FastDiv& f, uint32_t n) {
  return (__umulhi(n, f.m) + n) >> f.s;
}

__device__ __forceinline__ Site decode_half(const Geom& g, int64_t h64, int parity) {
  Site s;
  const uint32_t h = uint32_t(h64);
  const uint32_t r1 = fdiv(g.div_nxh, h);
  const uint32_t xh = h - r1 * uint32_t(g.nxh);
  const uint32_t r2 = fdiv(g.div_ny, r1);
  s.c[1] = int(r1 - r2 * uint32_t(g.ny));
  const uint32_t t = fdiv(g.div_nz, r2);
  s.c[2] = int(r2 - t * uint32_t(g.nz));
  s.c[3] = int(t);
  s.c[0] = int(2 * xh) + ((parity + s.c[1] + s.c[2] + s.c[3]) & 1);
  s.lex = 2 * int64_t(h) + (s.c[0] & 1);
  return s;
}

__device__ __forceinline__ int dim_of(const Geom& g, int d) {
  return d == 0 ? g.nx : (d == 1 ? g.ny : (d == 2 ? g.nz : g.nt));
}

// lex of the neighbour one step forward / backward along d, given the coordinate along d
__device__ __forceinline__ int64_t lex_fwd(const Geom& g, int64_t lex, int coord, int d) {
  const int n = dim_of(g, d);
  return coord == n - 1 ? lex - int64_t(n - 1) * g.stride[d] : lex + g.stride[d];
}
__device__ __forceinline__ int64_t lex_bwd(const Geom& g, int64_t lex, int coord, int d) {
  const int n = dim_of(g, d);
  return coord == 0 ? lex + int64_t(n - 1) * g.stride[d] : lex - g.stride[d];
}

__device__ __forceinline__ int coord_of(const Site& s, int d) {
  return d == 0 ? s.c[0] : (d == 1 ? s.c[1] : (d == 2 ? s.c[2] : s.c[3]));
}

}  // namespace sun
