// sun_kernels.cuh -- kernel templates of the SU(Nc) chessboard link sweep and the
// per-(Nc, storage, precision) operation table built from them.
//
// Included by exactly one translation unit per Nc (ops_su*.cu), which
// instantiates the table entries it needs.
#pragma once

#include <type_traits>

#include "sun_device.cuh"

namespace sun {

constexpr int kMaxBlockThreads = 256;
// resident 128-thread blocks per SM the register-bounded kernels (variant bit 1)
// are compiled for: 5 measured fastest among 4..8 for the SU(3) FP32 passes on
// GB300 (more warps cost more spills than they hide latency); with the two-row
// staple products (bit 2) the overrelaxation passes need fewer registers and 7
// blocks (72 registers) are fastest, for the fused re-unitarizing pass too
// (48^3 x 96, against 6 blocks: 0.474 -> 0.467 ms, fused 0.709 -> 0.684 ms; 8
// blocks: 0.472 ms); the heatbath pass stays at 5
constexpr int kOccBlocks = 5;
constexpr int kOccBlocksTwoRowOR = 7;
constexpr int kOccBlocksTwoRowHB = 5;  // 6 blocks: 0.706 -> 0.743 ms
// the same bound for the SU(4) FP32 per-link passes: 4 blocks (128 registers)
constexpr int kOccBlocksSU4 = 4;
template <int N, int VAR = 1, int MODE = 0>
__host__ __device__ constexpr int occ_blocks() {
  return N == 4 ? kOccBlocksSU4
                : ((VAR & 2) != 0 ? (MODE == 1 ? kOccBlocksTwoRowOR : kOccBlocksTwoRowHB) : kOccBlocks);
}
constexpr int kHeatbathMode = 0;
constexpr int kOverrelaxMode = 1;

__device__ __forceinline__ uint32_t stride_of(const Geom& g, int d) {
  return uint32_t(d == 0 ? g.stride[0] : (d == 1 ? g.stride[1] : (d == 2 ? g.stride[2] : g.stride[3])));
}
// lex of the neighbour one step forward / backward along d (coord = the site's coordinate along d)
__device__ __forceinline__ uint32_t fwd(const Geom& g, uint32_t lex, int coord, int d) {
  const int n = dim_of(g, d);
  const uint32_t st = stride_of(g, d);
  return coord == n - 1 ? lex - uint32_t(n - 1) * st : lex + st;
}
__device__ __forceinline__ uint32_t bwd(const Geom& g, uint32_t lex, int coord, int d) {
  const int n = dim_of(g, d);
  const uint32_t st = stride_of(g, d);
  return coord == 0 ? lex + uint32_t(n - 1) * st : lex - st;
}

struct PassParams {
  char* links;
  int64_t block_bytes;  // bytes of one (direction, parity) block
  Geom g;
  int mu, parity;
  double alpha_coef;  // 2 beta / Nc: heatbath strength alpha = alpha_coef * k
  uint2 key;
  const uint32_t* hb_step;
  uint32_t step_offset;
  // FP64 re-unitarization right after the update of the links whose run of 32
  // half-site indices r = h >> 5 (of the whole lattice) has r % reunit_mod ==
  // reunit_rem (0 = none)
  uint32_t reunit_mod, reunit_rem;
  // The pass covers half-sites [h_begin, h_end) of this (local) lattice.  A slab
  // of a lattice cut into t-slabs is a local lattice with one halo slice on each
  // side: its site lex is site (lex + lex_offset) mod v_global of the whole
  // lattice, which keys the random numbers and the re-unitarization runs.
  int64_t h_begin, h_end;
  uint32_t lex_offset, v_global;
};

// index of a local site in the whole lattice
__device__ __forceinline__ uint32_t global_lex(const PassParams& p, uint32_t lex) {
  const uint32_t l = lex + p.lex_offset;
  return l >= p.v_global ? l - p.v_global : l;
}

// hg: the half-site index in the whole lattice
__device__ __forceinline__ bool reunit_selected(const PassParams& p, int64_t hg) {
  return p.reunit_mod != 0u && ((uint32_t(hg) >> 5) % p.reunit_mod) == p.reunit_rem;
}

__device__ __forceinline__ const char* block_ptr(const PassParams& p, int d, int par) {
  return p.links + (2 * d + par) * p.block_bytes;
}

// Left-multiply rows i, j of m by the SU(2) element a embedded in the (i,j) subgroup.
template <class R, int N>
__device__ __forceinline__ void apply_rows(Mat<R, N>& m, int i, int j, const Quat<R>& a) {
  const Cpx<R> A00 = {a.a0, a.a3}, A01 = {a.a2, a.a1}, A10 = {-a.a2, a.a1}, A11 = {a.a0, -a.a3};
#pragma unroll
  for (int c = 0; c < N; ++c) {
    const Cpx<R> ri = m.e[i][c], rj = m.e[j][c];
    Cpx<R> ni = cmul(A00, ri), nj = cmul(A10, ri);
    cfma(ni, A01, rj);
    cfma(nj, A11, rj);
    m.e[i][c] = ni;
    m.e[j][c] = nj;
  }
}

// ---------------------------------------------------------------------------
// FP64 re-unitarization of one matrix (Sec. 2).
// ---------------------------------------------------------------------------
// 1/sqrt(s).  Rows of links stored in FP32 are within ~1e-6 of unit norm, and
// there the binomial series (1 + d)^(-1/2) = 1 - d/2 + 3 d^2/8 - 5 d^3/16 + ...
// with d = s - 1, cut after d^3, is exact to FP64 rounding: the first omitted
// term, 35 d^4 / 128, is below 4e-18 for |d| < 2^-14.  Other rows use rsqrt().
__device__ __forceinline__ double rsqrt_near_one(double s) {
  const double d = s - 1.0;
  // |d| < 2^-14 read off the exponent bits: an integer compare instead of one on
  // the FP64 pipe, which bounds the re-unitarizing passes (fused SU(3) pass at
  // 48^3 x 96: 0.718 -> 0.709 ms)
  if ((uint32_t(__double2hiint(d)) & 0x7ff00000u) < (uint32_t(1023 - 14) << 20))
    return fma(fma(fma(-0.3125, d, 0.375), d, -0.5), d, 1.0);
  return rsqrt(s);
}

template <int N>
__device__ __forceinline__ void normalise_row(Mat<double, N>& m, int r) {
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < N; ++c) {
    s = fma(m.e[r][c].re, m.e[r][c].re, s);
    s = fma(m.e[r][c].im, m.e[r][c].im, s);
  }
  const double inv = rsqrt_near_one(s);
#pragma unroll
  for (int c = 0; c < N; ++c) {
    m.e[r][c].re *= inv;
    m.e[r][c].im *= inv;
  }
}

template <int N>
__device__ __forceinline__ Cpx<double> det_lu_inplace(Mat<double, N>& a) {
  Cpx<double> det = {1.0, 0.0};
#pragma unroll
  for (int c = 0; c < N; ++c) {
    // partial pivoting on |a_rc|
    int piv = c;
    double best = a.e[c][c].re * a.e[c][c].re + a.e[c][c].im * a.e[c][c].im;
#pragma unroll
    for (int r = c + 1; r < N; ++r) {
      const double m2 = a.e[r][c].re * a.e[r][c].re + a.e[r][c].im * a.e[r][c].im;
      if (m2 > best) {
        best = m2;
        piv = r;
      }
    }
    if (best == 0.0) return {0.0, 0.0};
    if (piv != c) {
#pragma unroll
      for (int r = c + 1; r < N; ++r) {
        if (r == piv) {
#pragma unroll
          for (int k = 0; k < N; ++k) {
            const Cpx<double> t = a.e[c][k];
            a.e[c][k] = a.e[r][k];
            a.e[r][k] = t;
          }
        }
      }
      det = {-det.re, -det.im};
    }
    const Cpx<double> d = a.e[c][c];
    det = cmul(det, d);
    const double inv2 = 1.0 / best;
    const Cpx<double> dinv = {d.re * inv2, -d.im * inv2};
#pragma unroll
    for (int r = c + 1; r < N; ++r) {
      const Cpx<double> f = cmul(a.e[r][c], dinv);
#pragma unroll
      for (int k = c; k < N; ++k) {
        const Cpx<double> t = cmul(f, a.e[c][k]);
        a.e[r][k].re -= t.re;
        a.e[r][k].im -= t.im;
      }
    }
  }
  return det;
}

template <int N>
__device__ __forceinline__ Cpx<double> det_lu(Mat<double, N> a) {
  return det_lu_inplace<N>(a);
}

// Gram-Schmidt of rows 0 .. ROWS-1 in order (Sec. 2)
template <int N, int ROWS>
__device__ __forceinline__ void gram_schmidt_rows(Mat<double, N>& m) {
#pragma unroll
  for (int r = 0; r < ROWS; ++r) {
#pragma unroll
    for (int q = 0; q < r; ++q) {
      Cpx<double> pr = {0.0, 0.0};
#pragma unroll
      for (int c = 0; c < N; ++c) ccfma(pr, m.e[q][c], m.e[r][c]);
      // row r -= pr * row q
#pragma unroll
      for (int c = 0; c < N; ++c) {
        const Cpx<double> a = m.e[q][c];
        m.e[r][c].re = fma(pr.im, a.im, fma(-pr.re, a.re, m.e[r][c].re));
        m.e[r][c].im = fma(-pr.im, a.re, fma(-pr.re, a.im, m.e[r][c].im));
      }
    }
    normalise_row<N>(m, r);
  }
}

template <int N>
__device__ __forceinline__ void reunit_d(Mat<double, N>& m) {
  if constexpr (N == 2) {
    normalise_row<2>(m, 0);
    m.e[1][0] = {-m.e[0][1].re, m.e[0][1].im};
    m.e[1][1] = {m.e[0][0].re, -m.e[0][0].im};
  } else {
    gram_schmidt_rows<N, (N == 3) ? 2 : N>(m);
    if constexpr (N == 3) {
      su3_third_row(m);
    } else {
      const Cpx<double> d = det_lu<N>(m);
      const double inv = 1.0 / sqrt(d.re * d.re + d.im * d.im);
      const Cpx<double> ph = {d.re * inv, -d.im * inv};
#pragma unroll
      for (int c = 0; c < N; ++c) m.e[N - 1][c] = cmul(m.e[N - 1][c], ph);
    }
  }
}

template <class A, class B, int N>
__device__ __forceinline__ Mat<B, N> mat_cast(const Mat<A, N>& m) {
  Mat<B, N> o;
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) o.e[i][j] = {B(m.e[i][j].re), B(m.e[i][j].im)};
  return o;
}

// mat_cast with the FP32 <-> FP64 conversions done on the integer pipe (to_f64,
// to_f32: the same bits).  For the re-unitarization kernels and the update
// passes that re-unitarize, whose time is the FP64 pipe's (measured: the fused
// SU(3) overrelaxation pass 0.807 -> 0.716 ms at 48^3 x 96, its FP64 pipe 83%
// busy before; the separate pass, SU(4) 32^4 4.19 -> 3.63 ms, SU(6) 24^4 4.05 ->
// 3.67 ms).  The plaquette, whose FP64 pipe is a third busy, keeps the hardware
// conversions.
template <class A, class B, int N>
__device__ __forceinline__ Mat<B, N> mat_cast_int(const Mat<A, N>& m) {
  Mat<B, N> o;
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) o.e[i][j] = {convert_to<B>(m.e[i][j].re), convert_to<B>(m.e[i][j].im)};
  return o;
}

// ---------------------------------------------------------------------------
// Staple terms (Eq. 9).  With ROWS2 (SU(3) two-row storage, kernel variant bit
// 1) only rows 0 and 1 of each term are multiplied out and the term's third row
// is taken as conj(row0 x row1), which holds for an exact SU(3) product: a third
// fewer products, at an extra error of the order of the links' unitarity drift.
// ---------------------------------------------------------------------------
template <class R>
struct Rows2 {
  Cpx<R> e[2][3];
};

template <class R>
__device__ __forceinline__ Rows2<R> load_rows2(const char* blk, int64_t Vh, int64_t h) {
  R r[12];
  load_reals<R, 12, kLoadNc>(blk, Vh, h, r);
  Rows2<R> m;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) m.e[i][j] = {r[2 * (3 * i + j)], r[2 * (3 * i + j) + 1]};
  return m;
}

// st += the SU(3) term with rows t[0], t[1] and third row conj(t0 x t1): rows 0
// and 1 added, the third row's entries accumulated into st by fused chains
template <class R>
__device__ __forceinline__ void add_two_row_term(Mat<R, 3>& st, const Cpx<R> (&t)[2][3]) {
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      st.e[i][j].re += t[i][j].re;
      st.e[i][j].im += t[i][j].im;
    }
  st.e[2][0] = conj_cross_acc(t[0][1], t[1][2], t[0][2], t[1][1], st.e[2][0]);
  st.e[2][1] = conj_cross_acc(t[0][2], t[1][0], t[0][0], t[1][2], st.e[2][1]);
  st.e[2][2] = conj_cross_acc(t[0][0], t[1][1], t[0][1], t[1][0], st.e[2][2]);
}

// U_nu(x) U_mu(x+nu) U_nu(x+mu)^+ added to st; BL: how U_mu is loaded
template <class R, int N, int S, bool ROWS2, int BL>
__device__ __forceinline__ void staple_forward(Mat<R, N>& st, const char* pa, int64_t ha, const char* pb, int64_t hb,
                                               const char* pc, int64_t hc, int64_t Vh) {
  if constexpr (S == kTwoRow && ROWS2) {
    const Rows2<R> a = load_rows2<R>(pa, Vh, ha);
    const Mat<R, 3> b = load_mat<R, 3, S, BL>(pb, Vh, hb);
    Cpx<R> ab[2][3];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        Cpx<R> x = cmul(a.e[i][0], b.e[0][j]);
        cfma(x, a.e[i][1], b.e[1][j]);
        cfma(x, a.e[i][2], b.e[2][j]);
        ab[i][j] = x;
      }
    const Mat<R, 3> c = load_mat<R, 3, S>(pc, Vh, hc);
    Cpx<R> t[2][3];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        Cpx<R> x = cmulc(ab[i][0], c.e[j][0]);
        cfmac(x, ab[i][1], c.e[j][1]);
        cfmac(x, ab[i][2], c.e[j][2]);
        t[i][j] = x;
      }
    add_two_row_term(st, t);
  } else {
    const Mat<R, N> a = load_mat<R, N, S>(pa, Vh, ha);
    const Mat<R, N> b = load_mat<R, N, S, BL>(pb, Vh, hb);
    const Mat<R, N> t = mul_nn(a, b);
    const Mat<R, N> c = load_mat<R, N, S>(pc, Vh, hc);
    acc_nd(st, t, c);
  }
}

// U_nu(x-nu)^+ U_mu(x-nu) U_nu(x-nu+mu) added to st; BL: how U_mu is loaded
template <class R, int N, int S, bool ROWS2, int BL>
__device__ __forceinline__ void staple_backward(Mat<R, N>& st, const char* pa, int64_t ha, const char* pb, int64_t hb,
                                                const char* pc, int64_t hc, int64_t Vh) {
  if constexpr (S == kTwoRow && ROWS2) {
    const Rows2<R> a = load_rows2<R>(pa, Vh, ha);
    // entries (2,0), (2,1) of the third row conj(row0 x row1) of a
    const Cpx<R> a20 = conj_cross(a.e[0][1], a.e[1][2], a.e[0][2], a.e[1][1]);
    const Cpx<R> a21 = conj_cross(a.e[0][2], a.e[1][0], a.e[0][0], a.e[1][2]);
    const Mat<R, 3> b = load_mat<R, 3, S, BL>(pb, Vh, hb);
    // rows 0,1 of a^+ b: (a^+ b)_ik = sum_m conj(a_mi) b_mk
    Cpx<R> d[2][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      Cpx<R> x = ccmul(a.e[0][0], b.e[0][k]);
      ccfma(x, a.e[1][0], b.e[1][k]);
      ccfma(x, a20, b.e[2][k]);
      d[0][k] = x;
      Cpx<R> y = ccmul(a.e[0][1], b.e[0][k]);
      ccfma(y, a.e[1][1], b.e[1][k]);
      ccfma(y, a21, b.e[2][k]);
      d[1][k] = y;
    }
    const Mat<R, 3> c = load_mat<R, 3, S>(pc, Vh, hc);
    Cpx<R> t[2][3];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        Cpx<R> x = cmul(d[i][0], c.e[0][j]);
        cfma(x, d[i][1], c.e[1][j]);
        cfma(x, d[i][2], c.e[2][j]);
        t[i][j] = x;
      }
    add_two_row_term(st, t);
  } else {
    const Mat<R, N> a = load_mat<R, N, S>(pa, Vh, ha);
    const Mat<R, N> b = load_mat<R, N, S, BL>(pb, Vh, hb);
    const Mat<R, N> t = mul_dn(a, b);
    const Mat<R, N> c = load_mat<R, N, S>(pc, Vh, hc);
    acc_nn(st, t, c);
  }
}

// (U St^+)_ab = sum_k U_ak conj(St_bk)
template <class R, int N>
__device__ __forceinline__ Cpx<R> row_dot_c(const Mat<R, N>& u, int a, const Mat<R, N>& st, int b) {
  Cpx<R> x = cmulc(u.e[a][0], st.e[b][0]);
#pragma unroll
  for (int k = 1; k < N; ++k) cfmac(x, u.e[a][k], st.e[b][k]);
  return x;
}
// twice the SU(2) projection of the (i,j) block of W = U St^+, from the current U
template <class R, int N>
__device__ __forceinline__ Quat<R> or_block(const Mat<R, N>& u, const Mat<R, N>& st, int i, int j) {
  return block_to_quat2(row_dot_c<R, N>(u, i, st, i), row_dot_c<R, N>(u, i, st, j), row_dot_c<R, N>(u, j, st, i),
                        row_dot_c<R, N>(u, j, st, j));
}

// ---------------------------------------------------------------------------
// One chessboard pass over matrices (Nc >= 2, full or two-row storage):
// staple (Eq. 9) -> W = U Sigma^+ -> SU(2) subgroups in lexicographic order
// (Eq. 15), heatbath (Eqs. 12-14) or overrelaxation (Eq. 17) -> store.
// One thread per link of the pass.
// ---------------------------------------------------------------------------
// COH: the links of direction mu on the other parity may have been written by
// another block of the same launch (wavefront launches): they are read through L2.
template <class R, int N, int S, int MODE, bool ROWS2, bool REUNIT, bool COH = false>
__device__ __forceinline__ void pass_body(const PassParams& p, int par, int64_t h) {
  const Geom& g = p.g;
  const int mu = p.mu, opp = par ^ 1;
  const Site s = decode_half(g, h, par);
  const uint32_t lex = uint32_t(s.lex);
  const int cmu = coord_of(s, mu);
  const uint32_t lex_pmu = fwd(g, lex, cmu, mu);


  constexpr int BL = COH ? kLoadCg : kLoadNc;  // U_mu of the other parity
  Mat<R, N> st;
  mat_zero(st);
  // SU(3) heatbath: the loop over directions is kept rolled, one copy of the
  // staple code beside the heatbath's own (instruction fetch; 48^3 x 96: 0.771 ->
  // 0.722 ms); overrelaxation is faster unrolled (0.514 against 0.528 ms), and so
  // is the SU(4) heatbath (32^4 sweep 10.9 against 11.7 ms rolled)
#pragma unroll((MODE == kHeatbathMode && N == 3) ? 1 : 4)
  for (int nu = 0; nu < 4; ++nu) {
    if (nu == mu) continue;
    const int cnu = s.c[nu];
    const uint32_t lex_pnu = fwd(g, lex, cnu, nu);
    const uint32_t lex_mnu = bwd(g, lex, cnu, nu);
    const uint32_t lex_mnu_pmu = fwd(g, lex_mnu, cmu, mu);
    staple_forward<R, N, S, ROWS2, BL>(st, block_ptr(p, nu, par), h, block_ptr(p, mu, opp), lex_pnu >> 1,
                                       block_ptr(p, nu, opp), lex_pmu >> 1, g.Vh);
    staple_backward<R, N, S, ROWS2, BL>(st, block_ptr(p, nu, opp), lex_mnu >> 1, block_ptr(p, mu, opp),
                                        lex_mnu >> 1, block_ptr(p, nu, par), lex_mnu_pmu >> 1, g.Vh);
  }

  char* ublk = p.links + (2 * mu + par) * p.block_bytes;
  Mat<R, N> u = load_mat<R, N, S, kLoadPlain>(ublk, g.Vh, h);
  // W = U St^+: the heatbath forms it once and carries it along with U; the
  // overrelaxation takes each subgroup's 2x2 block of it from the current U
  // (or_block: 36 instead of about 41 complex products for SU(3); measured
  // faster for overrelaxation only, 48^3 x 96: 0.479 -> 0.474 ms)
  Mat<R, N> w;
  if constexpr (MODE == kHeatbathMode) w = mul_nd(u, st);

  uint32_t step = 0;
  if constexpr (MODE == kHeatbathMode) step = *p.hb_step + p.step_offset;
  const uint32_t glex = global_lex(p, lex);
  const uint32_t link_id = uint32_t(mu) * p.v_global + glex;
  const R alpha_coef = R(p.alpha_coef);

  int sub = 0;
#pragma unroll
  for (int i = 0; i < N - 1; ++i) {
#pragma unroll
    for (int j = i + 1; j < N; ++j) {
      if constexpr (MODE == kHeatbathMode) {
        const bool last = (i == N - 2) && (j == N - 1);
        const Quat<R> v = block_to_quat(w.e[i][i], w.e[i][j], w.e[j][i], w.e[j][j]);
        const R k = d_sqrt(fma(v.a0, v.a0, fma(v.a1, v.a1, fma(v.a2, v.a2, v.a3 * v.a3))));
        if (k > R(1e-15) && d_isfinite(k)) {
          const R inv = R(1) / k;
          const Quat<R> vd = {v.a0 * inv, -v.a1 * inv, -v.a2 * inv, -v.a3 * inv};  // vhat^+
          Quat<R> b;
          const bool apply = heatbath_su2<R>(alpha_coef * k, p.key, link_id, step, uint32_t(sub), b);
          const Quat<R> a = qmul(b, vd);
          if (apply) {
            apply_rows(u, i, j, a);
            if (!last) apply_rows(w, i, j, a);
          }
        }
      } else {
        // v2 = 2v: |v2|^2 = 4 k^2, compared with 4 (1e-15)^2
        const Quat<R> v2 = or_block<R, N>(u, st, i, j);
        const R n3 = fma(v2.a1, v2.a1, fma(v2.a2, v2.a2, v2.a3 * v2.a3));
        const R k2 = fma(v2.a0, v2.a0, n3);
        if (k2 > R(4e-30) && d_isfinite(k2)) apply_rows(u, i, j, or_element(v2, n3, k2));
      }
      ++sub;
    }
  }
  if constexpr (REUNIT) {
    if (reunit_selected(p, glex >> 1)) {
      Mat<double, N> d = mat_cast_int<R, double, N>(u);
      reunit_d<N>(d);
      u = mat_cast_int<double, R, N>(d);
    }
  }
  store_mat<R, N, S>(ublk, g.Vh, h, u);
}

// VAR bit 0: at most 128 threads per block and registers for occ_blocks() blocks per SM;
// VAR bit 1: two-row staple products (SU(3) two-row storage only).
// REUNIT: the FP64 re-unitarization of selected links is compiled in (passes that
// re-unitarize use this instantiation; the others carry no FP64 code).
template <class R, int N, int S, int MODE, int VAR, bool REUNIT>
__global__ void __launch_bounds__(kMaxBlockThreads) update_pass_mat(const PassParams p) {
  const int64_t h = p.h_begin + int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (h >= p.h_end) return;
  pass_body<R, N, S, MODE, (VAR & 2) != 0, REUNIT>(p, p.parity, h);
}

template <class R, int N, int S, int MODE, int VAR, bool REUNIT>
__global__ void __launch_bounds__(128, (occ_blocks<N, VAR, MODE>())) update_pass_mat_occ(const PassParams p) {
  const int64_t h = p.h_begin + int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (h >= p.h_end) return;
  pass_body<R, N, S, MODE, (VAR & 2) != 0, REUNIT>(p, p.parity, h);
}

// ---------------------------------------------------------------------------
// Row-parallel pass for SU(Nc), Nc = 4 and 6 (no fused re-unitarization):
// Nc threads of a warp share one link.  Thread r owns row r of the staple and
// of U, the neighbour links of each staple term are staged row by row in
// shared memory, and for the SU(2) subgroup updates (Eq. 15) thread c owns
// column c of U and W, so every lane works on every subgroup.  The heatbath
// draw runs Nc attempts at once, one per lane; the first accepted attempt in
// attempt order is taken (warp ballot), so the random stream and the result are
// those of the one-attempt-at-a-time sampler.  Lanes beyond the last whole
// group of a warp run a copy of a real link and never store.
// ---------------------------------------------------------------------------
template <class R, int N>
struct Group {
  // rows per lane: SU(6) FP32 lanes own two rows (and two columns), so that every
  // operand read from shared memory feeds two complex multiply-adds
  static constexpr int RB = (N == 6 && sizeof(R) == 4) ? 2 : 1;
  static constexpr int LPL = N / RB;          // lanes per link
  static constexpr int LPW = 32 / LPL;        // links per warp
  static constexpr int WARPS = 4;             // warps per block (128 threads)
  static constexpr int LPB = WARPS * LPW;     // links per block
  static constexpr int CPR = 2 * N * int(sizeof(R)) / 16;  // 16-byte components per row
};

template <class R, int N>
__host__ __device__ constexpr bool has_group() {
  return (N == 4 || N == 6) && (2 * N * int(sizeof(R))) % 16 == 0;
}

// Default choice between the row-parallel and the one-thread-per-link pass
// (measured on 24^4: row-parallel is faster for Nc = 6, slower for Nc = 4 whose
// matrices fit in registers); kernel variant bit 4 takes the other one.
template <class R, int N>
__host__ __device__ constexpr bool group_by_default() {
  return N == 6;
}

template <class R, int N>
__host__ __device__ inline bool use_group(int variant) {
  return has_group<R, N>() && (group_by_default<R, N>() != ((variant & 4) != 0));
}

// row r of a full-storage link
template <class R, int N>
__device__ __forceinline__ void load_row(const char* blk, int64_t Vh, int64_t h, int r, Cpx<R> (&row)[N]) {
  using V = typename Vec16<R>::T;
  constexpr int per16 = 16 / int(sizeof(R));
  R buf[2 * N];
#pragma unroll
  for (int c = 0; c < Group<R, N>::CPR; ++c) {
    const V* p = reinterpret_cast<const V*>(blk + (int64_t(r * Group<R, N>::CPR + c) * Vh + h) * 16);
    unpack(__ldg(p), &buf[c * per16]);
  }
#pragma unroll
  for (int k = 0; k < N; ++k) row[k] = {buf[2 * k], buf[2 * k + 1]};
}

template <class R, int N>
__device__ __forceinline__ void load_row_rw(const char* blk, int64_t Vh, int64_t h, int r, Cpx<R> (&row)[N]) {
  using V = typename Vec16<R>::T;
  constexpr int per16 = 16 / int(sizeof(R));
  R buf[2 * N];
#pragma unroll
  for (int c = 0; c < Group<R, N>::CPR; ++c) {
    const V* p = reinterpret_cast<const V*>(blk + (int64_t(r * Group<R, N>::CPR + c) * Vh + h) * 16);
    unpack(*p, &buf[c * per16]);
  }
#pragma unroll
  for (int k = 0; k < N; ++k) row[k] = {buf[2 * k], buf[2 * k + 1]};
}

template <class R, int N>
__device__ __forceinline__ void store_row(char* blk, int64_t Vh, int64_t h, int r, const Cpx<R> (&row)[N]) {
  using V = typename Vec16<R>::T;
  constexpr int per16 = 16 / int(sizeof(R));
  R buf[2 * N];
#pragma unroll
  for (int k = 0; k < N; ++k) {
    buf[2 * k] = row[k].re;
    buf[2 * k + 1] = row[k].im;
  }
#pragma unroll
  for (int c = 0; c < Group<R, N>::CPR; ++c) {
    V* p = reinterpret_cast<V*>(blk + (int64_t(r * Group<R, N>::CPR + c) * Vh + h) * 16);
    *p = pack4(&buf[c * per16]);
  }
}

template <class R, int N>
__device__ __forceinline__ void smem_put_row(Cpx<R> (*m)[N], int r, const Cpx<R> (&row)[N]) {
#pragma unroll
  for (int k = 0; k < N; ++k) m[r][k] = row[k];
}

// heatbath element of one subgroup drawn by the LANES lanes of a link at once:
// lane q of the link tries attempts round * LANES * PER + q * PER + t, t < PER,
// stopping at its first accepted one, and the link takes the first accepted
// attempt in attempt order, so the draw is that of one attempt at a time.  Not
// inlined: one copy serves the Nc(Nc-1)/2 subgroups (instruction fetch)
template <class R, int LANES, int PER>
__device__ __noinline__ bool heatbath_su2_group(R alpha, bool skip, uint2 key, uint32_t link, uint32_t step,
                                                   uint32_t sub, int q, int base, Quat<R>& b) {
  const bool kp = alpha >= R(1.5);
  const R inv2a = R(1) / (R(2) * alpha);
  const R e = -d_expm1(R(-2) * alpha);
  bool found = skip;
  bool got = false;
  R b0 = R(1);
  for (int round = 0; round * LANES * PER < kHeatbathAttempts; ++round) {
    bool acc = false;
    R x = R(1);
#pragma unroll
    for (int t = 0; t < PER; ++t) {
      const int att = (round * LANES + q) * PER + t;
      if (!found && !acc && att < kHeatbathAttempts) {
        const uint4 u = philox4x32_10(make_uint4(link, step, (sub << 16) | uint32_t(att), kTagHeatbath), key);
        const R r0 = u01<R>(u.x), r1 = u01<R>(u.y), r2 = u01<R>(u.z), r3 = u01<R>(u.w);
        if (kp) {
          const R c = d_cospi(R(2) * r1);
          const R delta = -(d_log(r0) + c * c * d_log(r2)) * inv2a;
          acc = r3 * r3 <= R(1) - delta;
          x = R(1) - R(2) * delta;
        } else {
          x = alpha > R(0) ? R(1) + d_log1p(-r0 * e) / alpha : R(1) - R(2) * r0;
          acc = r1 * r1 <= R(1) - x * x;
        }
      }
    }
    const unsigned bal = __ballot_sync(0xffffffffu, acc);
    const unsigned mine = (base < 32 ? (bal >> base) : 0u) & ((1u << LANES) - 1u);
    const int first = mine ? __ffs(mine) - 1 : 0;
    const R xb = __shfl_sync(0xffffffffu, x, (base + first) & 31);
    if (!found && mine) {
      b0 = xb;
      found = true;
      got = true;
    }
    if (!__any_sync(0xffffffffu, !found)) break;
  }
  if (!got) return false;
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

// ---------------------------------------------------------------------------
// Block-wide staging of the row-parallel pass.  The LPB links of a block sit at
// LPB consecutive half-sites, and so do their neighbours of each role in a
// staple term (up to the lattice's periodic wrap).  The block loads the three
// neighbour links of a term for all its links together, consecutive threads
// taking consecutive 16-byte components of one component array (runs of LPB x
// 16 bytes instead of a warp load spread over Nc component arrays), straight
// into shared memory (cp.async); the lanes then read their rows there.  A link
// has a slot of an odd number of 16-byte quads, so that eight consecutive
// slots start in eight different bank quads.  The update's own links are read
// and written the same way.
// ---------------------------------------------------------------------------
template <class R, int N>
struct GroupTile {
  static constexpr int LPB = Group<R, N>::LPB;
  static constexpr int C16 = N * Group<R, N>::CPR;         // 16-byte components of a link
  static constexpr int kQuads = (C16 & 1) == 0 ? C16 + 1 : C16;
  static constexpr int kSlotBytes = kQuads * 16;
  static constexpr int kSlots = LPB + 1;                   // + one for lanes past a warp's last whole link
  static constexpr int kBytes = 3 * kSlots * kSlotBytes;
};

template <class R, int N>
__device__ __forceinline__ Cpx<R> (*tile_mat(char* tile, int q, int slot))[N] {
  return reinterpret_cast<Cpx<R>(*)[N]>(tile + (q * GroupTile<R, N>::kSlots + slot) * GroupTile<R, N>::kSlotBytes);
}

// Load NQ links (roles q < NQ, at half-sites hidx[q][j] of block pointers b[q])
// of every link j of the block into the tile; cached in L2 only (cp.async.cg),
// so it also serves links this kernel writes afterwards.  Thread t takes link
// j = t % LPB and components t / LPB, + G, + 2G, ... (G threads per link), so
// that consecutive threads read consecutive components of one array.  Ends with
// the block synchronised.
template <class R, int N, int NQ>
__device__ __forceinline__ void group_stage(char* tile, const uint32_t (*hidx)[GroupTile<R, N>::LPB], const char* b0,
                                            const char* b1, const char* b2, int64_t Vh) {
  using T = GroupTile<R, N>;
  constexpr int G = 128 / T::LPB;
  constexpr int PER = (T::C16 + G - 1) / G;
  const int j = int(threadIdx.x) % T::LPB, g = int(threadIdx.x) / T::LPB;
  if (g < G) {
    const int64_t cstep = int64_t(G) * Vh * 16;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const char* blk = q == 0 ? b0 : (q == 1 ? b1 : b2);
      const char* src = blk + (int64_t(g) * Vh + hidx[q][j]) * 16;
      const uint32_t dst = uint32_t(__cvta_generic_to_shared(tile + (q * T::kSlots + j) * T::kSlotBytes + g * 16));
#pragma unroll
      for (int m = 0; m < PER; ++m) {
        if (PER * G == T::C16 || g + m * G < T::C16)
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + uint32_t(m * G * 16)),
                       "l"(src + m * cstep)
                       : "memory");
      }
    }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
}

template <class R, int N, int MODE>
__device__ __forceinline__ void group_pass_body(const PassParams& p, int64_t first_link, int64_t h_end, char* tile,
                                                uint32_t (*hidx)[GroupTile<R, N>::LPB]) {
  using T = GroupTile<R, N>;
  using G = Group<R, N>;
  constexpr int RB = G::RB, LPL = G::LPL;
  const Geom& g = p.g;
  const int mu = p.mu, par = p.parity, opp = par ^ 1;
  // lane -> (link j of the block, lane q of the link: rows and columns q RB .. q RB + RB - 1);
  // lanes past a warp's last whole link use the spare slot, run a copy of a real
  // link and never store
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gi = lane / LPL;
  const int q = lane - gi * LPL;
  const int base = gi * LPL;
  const bool whole = gi < G::LPW;
  const int j = warp * G::LPW + gi;
  const int slot = whole ? j : T::LPB;
  const int64_t link = first_link + j;
  const bool active = whole && link < h_end;
  const int64_t h = link < h_end ? link : h_end - 1;
  const int n_act = int(h_end - first_link < T::LPB ? h_end - first_link : T::LPB);

  const Site s = decode_half(g, h, par);
  const uint32_t lex = uint32_t(s.lex);
  const int cmu = coord_of(s, mu);
  const uint32_t lex_pmu = fwd(g, lex, cmu, mu);
  const bool writer = whole && q == 0;

  Cpx<R> st[RB][N];
#pragma unroll
  for (int t = 0; t < RB; ++t)
#pragma unroll
    for (int k = 0; k < N; ++k) st[t][k] = {R(0), R(0)};
  // one copy of the two staple terms' code, not four (instruction fetch; measured
  // at 24^4 for SU(6): sweep 17.37 -> 17.20 ms, the same links)
#pragma unroll 1
  for (int nu = 0; nu < 4; ++nu) {
    if (nu == mu) continue;
    const int cnu = s.c[nu];
    const uint32_t lex_pnu = fwd(g, lex, cnu, nu);
    const uint32_t lex_mnu = bwd(g, lex, cnu, nu);
    const uint32_t lex_mnu_pmu = fwd(g, lex_mnu, cmu, mu);
    {  // U_nu(x) U_mu(x+nu) U_nu(x+mu)^+ : rows q RB + t of (A B) C^+
      if (writer) {
        hidx[0][j] = uint32_t(h);
        hidx[1][j] = lex_pnu >> 1;
        hidx[2][j] = lex_pmu >> 1;
      }
      __syncthreads();
      group_stage<R, N, 3>(tile, hidx, block_ptr(p, nu, par), block_ptr(p, mu, opp), block_ptr(p, nu, opp), g.Vh);
      const Cpx<R>(*A)[N] = tile_mat<R, N>(tile, 0, slot);
      const Cpx<R>(*B)[N] = tile_mat<R, N>(tile, 1, slot);
      const Cpx<R>(*C)[N] = tile_mat<R, N>(tile, 2, slot);
      Cpx<R> ar[RB][N], ab[RB][N];
#pragma unroll
      for (int t = 0; t < RB; ++t)
#pragma unroll
        for (int k = 0; k < N; ++k) ar[t][k] = A[q * RB + t][k];
#pragma unroll
      for (int jj = 0; jj < N; ++jj) {
        {
          const Cpx<R> b = B[0][jj];
#pragma unroll
          for (int t = 0; t < RB; ++t) ab[t][jj] = cmul(ar[t][0], b);
        }
#pragma unroll
        for (int k = 1; k < N; ++k) {
          const Cpx<R> b = B[k][jj];
#pragma unroll
          for (int t = 0; t < RB; ++t) cfma(ab[t][jj], ar[t][k], b);
        }
      }
#pragma unroll
      for (int jj = 0; jj < N; ++jj) {
        Cpx<R> x[RB];
        {
          const Cpx<R> c = C[jj][0];
#pragma unroll
          for (int t = 0; t < RB; ++t) x[t] = cmulc(ab[t][0], c);
        }
#pragma unroll
        for (int k = 1; k < N; ++k) {
          const Cpx<R> c = C[jj][k];
#pragma unroll
          for (int t = 0; t < RB; ++t) cfmac(x[t], ab[t][k], c);
        }
#pragma unroll
        for (int t = 0; t < RB; ++t) {
          st[t][jj].re += x[t].re;
          st[t][jj].im += x[t].im;
        }
      }
      __syncthreads();
    }
    {  // U_nu(x-nu)^+ U_mu(x-nu) U_nu(x-nu+mu) : rows q RB + t of A^+ (B C)
      if (writer) {
        hidx[0][j] = lex_mnu >> 1;
        hidx[1][j] = lex_mnu >> 1;
        hidx[2][j] = lex_mnu_pmu >> 1;
      }
      __syncthreads();
      group_stage<R, N, 3>(tile, hidx, block_ptr(p, nu, opp), block_ptr(p, mu, opp), block_ptr(p, nu, par), g.Vh);
      const Cpx<R>(*A)[N] = tile_mat<R, N>(tile, 0, slot);
      Cpx<R>(*B)[N] = tile_mat<R, N>(tile, 1, slot);
      const Cpx<R>(*C)[N] = tile_mat<R, N>(tile, 2, slot);
      Cpx<R> br[RB][N], bc[RB][N];
#pragma unroll
      for (int t = 0; t < RB; ++t)
#pragma unroll
        for (int k = 0; k < N; ++k) br[t][k] = B[q * RB + t][k];
#pragma unroll
      for (int jj = 0; jj < N; ++jj) {
        {
          const Cpx<R> c = C[0][jj];
#pragma unroll
          for (int t = 0; t < RB; ++t) bc[t][jj] = cmul(br[t][0], c);
        }
#pragma unroll
        for (int k = 1; k < N; ++k) {
          const Cpx<R> c = C[k][jj];
#pragma unroll
          for (int t = 0; t < RB; ++t) cfma(bc[t][jj], br[t][k], c);
        }
      }
      // rows of B C replace the lane's rows of B, which only this lane reads
#pragma unroll
      for (int t = 0; t < RB; ++t)
#pragma unroll
        for (int jj = 0; jj < N; ++jj) B[q * RB + t][jj] = bc[t][jj];
      __syncwarp();
      Cpx<R> ac[RB][N];  // column q RB + t of A
#pragma unroll
      for (int t = 0; t < RB; ++t)
#pragma unroll
        for (int k = 0; k < N; ++k) ac[t][k] = A[k][q * RB + t];
#pragma unroll
      for (int jj = 0; jj < N; ++jj) {
        Cpx<R> x[RB];
        {
          const Cpx<R> v = B[0][jj];
#pragma unroll
          for (int t = 0; t < RB; ++t) x[t] = ccmul(ac[t][0], v);
        }
#pragma unroll
        for (int k = 1; k < N; ++k) {
          const Cpx<R> v = B[k][jj];
#pragma unroll
          for (int t = 0; t < RB; ++t) ccfma(x[t], ac[t][k], v);
        }
#pragma unroll
        for (int t = 0; t < RB; ++t) {
          st[t][jj].re += x[t].re;
          st[t][jj].im += x[t].im;
        }
      }
      __syncthreads();
    }
  }

  // the links being updated, U_mu(x) of this parity
  char* ublk = p.links + (2 * mu + par) * p.block_bytes;
  if (writer) hidx[0][j] = uint32_t(h);
  __syncthreads();
  group_stage<R, N, 1>(tile, hidx, ublk, ublk, ublk, g.Vh);
  Cpx<R>(*U)[N] = tile_mat<R, N>(tile, 0, slot);
  Cpx<R>(*S)[N] = tile_mat<R, N>(tile, 1, slot);
  Cpx<R>(*Wm)[N] = tile_mat<R, N>(tile, 2, slot);
  // W = U Sigma^+ (rows q RB + t), then columns of U and W for the subgroup updates
#pragma unroll
  for (int t = 0; t < RB; ++t)
#pragma unroll
    for (int k = 0; k < N; ++k) S[q * RB + t][k] = st[t][k];
  __syncwarp();
  {
    Cpx<R> ur[RB][N], w[RB][N];
#pragma unroll
    for (int t = 0; t < RB; ++t)
#pragma unroll
      for (int k = 0; k < N; ++k) ur[t][k] = U[q * RB + t][k];
#pragma unroll
    for (int jj = 0; jj < N; ++jj) {
      {
        const Cpx<R> sv = S[jj][0];
#pragma unroll
        for (int t = 0; t < RB; ++t) w[t][jj] = cmulc(ur[t][0], sv);
      }
#pragma unroll
      for (int k = 1; k < N; ++k) {
        const Cpx<R> sv = S[jj][k];
#pragma unroll
        for (int t = 0; t < RB; ++t) cfmac(w[t][jj], ur[t][k], sv);
      }
    }
#pragma unroll
    for (int t = 0; t < RB; ++t)
#pragma unroll
      for (int k = 0; k < N; ++k) Wm[q * RB + t][k] = w[t][k];
  }
  __syncwarp();
  Cpx<R> uc[RB][N], wc[RB][N];  // columns q RB + t
#pragma unroll
  for (int t = 0; t < RB; ++t)
#pragma unroll
    for (int i = 0; i < N; ++i) {
      uc[t][i] = U[i][q * RB + t];
      wc[t][i] = Wm[i][q * RB + t];
    }
  __syncwarp();

  uint32_t step = 0;
  if constexpr (MODE == kHeatbathMode) step = *p.hb_step + p.step_offset;
  const uint32_t glex = global_lex(p, lex);
  const uint32_t link_id = uint32_t(mu) * p.v_global + glex;
  const R alpha_coef = R(p.alpha_coef);
  int sub = 0;
#pragma unroll
  for (int i = 0; i < N - 1; ++i) {
#pragma unroll
    for (int jn = i + 1; jn < N; ++jn) {
      const bool last = (i == N - 2) && (jn == N - 1);
      // column c sits in lane base + c / RB, register set c % RB
      const int li = (base + i / RB) & 31, lj = (base + jn / RB) & 31;
      const Cpx<R> wii = {__shfl_sync(0xffffffffu, wc[i % RB][i].re, li), __shfl_sync(0xffffffffu, wc[i % RB][i].im, li)};
      const Cpx<R> wji = {__shfl_sync(0xffffffffu, wc[i % RB][jn].re, li), __shfl_sync(0xffffffffu, wc[i % RB][jn].im, li)};
      const Cpx<R> wij = {__shfl_sync(0xffffffffu, wc[jn % RB][i].re, lj), __shfl_sync(0xffffffffu, wc[jn % RB][i].im, lj)};
      const Cpx<R> wjj = {__shfl_sync(0xffffffffu, wc[jn % RB][jn].re, lj), __shfl_sync(0xffffffffu, wc[jn % RB][jn].im, lj)};
      Quat<R> a;
      bool apply;
      if constexpr (MODE == kHeatbathMode) {
        const Quat<R> v = block_to_quat(wii, wij, wji, wjj);
        const R k = d_sqrt(fma(v.a0, v.a0, fma(v.a1, v.a1, fma(v.a2, v.a2, v.a3 * v.a3))));
        const bool ok = active && k > R(1e-15) && d_isfinite(k);
        const R inv = ok ? R(1) / k : R(0);
        const Quat<R> vd = {v.a0 * inv, -v.a1 * inv, -v.a2 * inv, -v.a3 * inv};
        Quat<R> b;
        const bool drawn = heatbath_su2_group<R, LPL, RB>(ok ? alpha_coef * k : R(1), !ok, p.key, link_id, step,
                                                          uint32_t(sub), q, base, b);
        apply = ok && drawn;
        a = qmul(b, vd);
      } else {
        // v2 = 2v, as in the one-thread-per-link pass
        const Quat<R> v2 = block_to_quat2(wii, wij, wji, wjj);
        const R n3 = fma(v2.a1, v2.a1, fma(v2.a2, v2.a2, v2.a3 * v2.a3));
        const R k2 = fma(v2.a0, v2.a0, n3);
        apply = active && k2 > R(4e-30) && d_isfinite(k2);
        a = or_element(v2, n3, apply ? k2 : R(1));
      }
      if (apply) {
        const Cpx<R> A00 = {a.a0, a.a3}, A01 = {a.a2, a.a1}, A10 = {-a.a2, a.a1}, A11 = {a.a0, -a.a3};
#pragma unroll
        for (int t = 0; t < RB; ++t) {
          Cpx<R> ni = cmul(A00, uc[t][i]), nj = cmul(A10, uc[t][i]);
          cfma(ni, A01, uc[t][jn]);
          cfma(nj, A11, uc[t][jn]);
          uc[t][i] = ni;
          uc[t][jn] = nj;
          if (!last) {
            Cpx<R> mi = cmul(A00, wc[t][i]), mj = cmul(A10, wc[t][i]);
            cfma(mi, A01, wc[t][jn]);
            cfma(mj, A11, wc[t][jn]);
            wc[t][i] = mi;
            wc[t][jn] = mj;
          }
        }
      }
      ++sub;
    }
  }
  // back to rows in the tile, then the block stores its links' components
#pragma unroll
  for (int t = 0; t < RB; ++t)
#pragma unroll
    for (int i = 0; i < N; ++i) U[i][q * RB + t] = uc[t][i];
  __syncthreads();
  {
    constexpr int G = 128 / T::LPB;
    constexpr int PER = (T::C16 + G - 1) / G;
    using V = typename Vec16<R>::T;
    const int jl = int(threadIdx.x) % T::LPB, gl = int(threadIdx.x) / T::LPB;
    if (gl < G && jl < n_act) {
      char* dst = ublk + (int64_t(gl) * g.Vh + hidx[0][jl]) * 16;
      const char* src = tile + jl * T::kSlotBytes + gl * 16;
      const int64_t cstep = int64_t(G) * g.Vh * 16;
#pragma unroll
      for (int m = 0; m < PER; ++m)
        if (PER * G == T::C16 || gl + m * G < T::C16)
          *reinterpret_cast<V*>(dst + m * cstep) = *reinterpret_cast<const V*>(src + m * G * 16);
    }
  }
}

template <class R, int N, int MODE>
// 5 resident blocks per SM: measured fastest for SU(6) FP32 (unbounded: 4 blocks,
// 6 blocks: more spills); heatbath 6% and overrelaxation 2% faster than unbounded
__global__ void __launch_bounds__(128, 5) update_pass_group(const PassParams p) {
  __shared__ __align__(16) char tile[GroupTile<R, N>::kBytes];
  __shared__ uint32_t hidx[3][GroupTile<R, N>::LPB];
  group_pass_body<R, N, MODE>(p, p.h_begin + int64_t(blockIdx.x) * Group<R, N>::LPB, p.h_end, tile, hidx);
}

// FP64 passes of Nc >= 5 are built without the fused re-unitarization
// (reunit_mode 1, 2): they would double the largest units' build time.
template <class R, int N>
constexpr bool has_fused_reunit() {
  return !(std::is_same<R, double>::value && N >= 5);
}

// kernel variants are built for the SU(3) FP32 update passes only
template <class R, int N, int S>
constexpr bool has_variants() {
  return std::is_same<R, float>::value && N == 3;
}

// the register-bounded per-link pass (variant bit 1) is also built for SU(4) FP32
template <class R, int N>
constexpr bool has_occ_bound() {
  return std::is_same<R, float>::value && N == 4;
}

// ---------------------------------------------------------------------------
// One chessboard pass for SU(2) stored as quaternions (Eq. 6): the same steps
// with the staple kept in the real span of SU(2).
// ---------------------------------------------------------------------------
template <class R, int MODE, bool REUNIT, bool COH = false>
__device__ __forceinline__ void quat_pass_body(const PassParams& p, int par, int64_t h) {
  constexpr int BL = COH ? kLoadCg : kLoadNc;  // U_mu of the other parity
  const Geom& g = p.g;
  const int mu = p.mu, opp = par ^ 1;
  const Site s = decode_half(g, h, par);
  const uint32_t lex = uint32_t(s.lex);
  const int cmu = coord_of(s, mu);
  const uint32_t lex_pmu = fwd(g, lex, cmu, mu);

  Quat<R> st = {R(0), R(0), R(0), R(0)};
#pragma unroll
  for (int nu = 0; nu < 4; ++nu) {
    if (nu == mu) continue;
    const int cnu = s.c[nu];
    const uint32_t lex_pnu = fwd(g, lex, cnu, nu);
    const uint32_t lex_mnu = bwd(g, lex, cnu, nu);
    const uint32_t lex_mnu_pmu = fwd(g, lex_mnu, cmu, mu);
    {
      const Quat<R> a = load_quat<R>(block_ptr(p, nu, par), g.Vh, h);
      const Quat<R> b = load_quat<R, BL>(block_ptr(p, mu, opp), g.Vh, lex_pnu >> 1);
      const Quat<R> c = load_quat<R>(block_ptr(p, nu, opp), g.Vh, lex_pmu >> 1);
      st = qadd(st, qmul(qmul(a, b), qdag(c)));
    }
    {
      const Quat<R> a = load_quat<R>(block_ptr(p, nu, opp), g.Vh, lex_mnu >> 1);
      const Quat<R> b = load_quat<R, BL>(block_ptr(p, mu, opp), g.Vh, lex_mnu >> 1);
      const Quat<R> c = load_quat<R>(block_ptr(p, nu, par), g.Vh, lex_mnu_pmu >> 1);
      st = qadd(st, qmul(qmul(qdag(a), b), c));
    }
  }
  char* ublk = p.links + (2 * mu + par) * p.block_bytes;
  Quat<R> u = load_quat<R, kLoadPlain>(ublk, g.Vh, h);
  const Quat<R> w = qmul(u, qdag(st));
  if constexpr (MODE == kHeatbathMode) {
    const R k = d_sqrt(fma(w.a0, w.a0, fma(w.a1, w.a1, fma(w.a2, w.a2, w.a3 * w.a3))));
    if (k > R(1e-15) && d_isfinite(k)) {
      const R inv = R(1) / k;
      const Quat<R> vd = {w.a0 * inv, -w.a1 * inv, -w.a2 * inv, -w.a3 * inv};
      const uint32_t step = *p.hb_step + p.step_offset;
      const uint32_t link_id = uint32_t(mu) * p.v_global + global_lex(p, lex);
      Quat<R> b;
      if (heatbath_su2<R>(R(p.alpha_coef) * k, p.key, link_id, step, 0u, b)) u = qmul(qmul(b, vd), u);
    }
  } else {
    const R n3 = fma(w.a1, w.a1, fma(w.a2, w.a2, w.a3 * w.a3));
    const R k2 = fma(w.a0, w.a0, n3);
    if (k2 > R(1e-30) && d_isfinite(k2)) u = qmul(or_element(w, n3, k2), u);
  }
  if constexpr (REUNIT) {
    if (reunit_selected(p, global_lex(p, lex) >> 1)) {
      const double a0 = u.a0, a1 = u.a1, a2 = u.a2, a3 = u.a3;
      const double inv = rsqrt_near_one(fma(a1, a1, fma(a2, a2, fma(a3, a3, a0 * a0))));
      u = Quat<R>{R(a0 * inv), R(a1 * inv), R(a2 * inv), R(a3 * inv)};
    }
  }
  store_quat<R>(ublk, g.Vh, h, u);
}

template <class R, int MODE, bool REUNIT>
__global__ void __launch_bounds__(kMaxBlockThreads) update_pass_quat(const PassParams p) {
  const int64_t h = p.h_begin + int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (h >= p.h_end) return;
  quat_pass_body<R, MODE, REUNIT>(p, p.parity, h);
}

// ---------------------------------------------------------------------------
// Both parities of one direction in one launch (the even and odd pass of a
// step, Sec. 3), as a wavefront over t-slices.
//
// One block per unit of (parity, t-slice, chunk of blockDim.x links); a block
// takes its unit from a ticket counter when it starts.  The staple (Eq. 9) of an
// odd link on slice t reads the even links of the same direction on slices t-1,
// t, t+1, so an odd unit first waits until those three even slices are
// finished; even units wait for nothing.  Even slices run `lag` slices ahead of
// the odd ones, and odd slice 0, which needs the last even slice, comes last.
// Every wait is on units with smaller tickets, all held by blocks that have
// started, so the launch progresses however many blocks are resident.  Each
// link sees the same neighbour values as in two separate passes (all even
// links, then all odd links), so the results are bitwise those of the
// two-launch schedule; the links a slice's even and odd
// units share are still in L2 when the odd unit reads them.
// ---------------------------------------------------------------------------
struct WaveParams {
  uint32_t* sync;       // [0] wait timeouts, [1] ticket, [2 + t] finished even units of slice t
  uint32_t chunks;      // chunks per (parity, slice) = ceil(half_slice / blockDim.x)
  uint32_t half_slice;  // sites of one parity on one t-slice, Nx Ny Nz / 2
  uint32_t nt;
  uint32_t lag;   // 1 <= lag <= nt - 1
  uint32_t skip;  // units left out at the start (fault injection for tests; 0 otherwise)
};

constexpr uint64_t kWaveWaitNs = 2000000000ull;  // give up a wait after 2 s
constexpr uint32_t kWaveWaitPolls = 1u << 24;   // or after this many polls

// Unit j (0 <= j < 2 nt) of the issue order: E0 .. E(lag), then E(k), O(k - lag)
// for k = lag+1 .. nt-1, then O(nt - lag) .. O(nt - 1), then O(0).
__host__ __device__ __forceinline__ void wave_unit(uint32_t j, uint32_t nt, uint32_t lag, int& par, uint32_t& t) {
  if (j <= lag) {
    par = 0;
    t = j;
  } else if (j + lag + 2 <= 2 * nt) {
    const bool even = ((j - lag - 1) & 1u) == 0u;
    par = even ? 0 : 1;
    t = even ? (j + lag + 1) / 2 : (j - lag) / 2;
  } else {
    par = 1;
    t = j == 2 * nt - 1 ? 0u : j + 1 - nt;
  }
}

__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t* a) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
  return v;
}

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Thread 0: wait until the even slices t-1, t, t+1 are finished.  The wait is
// bounded; one that gives up is counted in sync[0] and the unit goes ahead.
__device__ __forceinline__ void wave_wait_even(const WaveParams& w, uint32_t t) {
  const uint32_t ts[3] = {t == 0 ? w.nt - 1 : t - 1, t, t + 1 == w.nt ? 0u : t + 1};
  uint64_t t0 = 0;
  uint32_t polls = 0;
  for (int q = 0; q < 3; ++q) {
    const uint32_t* cnt = w.sync + kWaveSyncWords + ts[q];
    while (ld_acquire_gpu(cnt) < w.chunks) {
      const uint64_t now = global_timer_ns();
      if (polls == 0) t0 = now;
      if (++polls > kWaveWaitPolls || now - t0 > kWaveWaitNs) {
        atomicAdd(w.sync, 1u);
        return;
      }
      __nanosleep(256);
    }
  }
  __threadfence();
}

// QUAT: the body is the quaternion SU(2) pass, else the matrix pass.  (The body is
// called directly, not through a lambda: a lambda holding a reference to the
// kernel parameters would copy them to local memory.)
template <class R, int N, int S, int MODE, bool ROWS2, bool REUNIT, bool QUAT>
__device__ __forceinline__ void wavefront(const PassParams& p, const WaveParams& w) {
  __shared__ uint32_t s_ticket;
  if (threadIdx.x == 0) s_ticket = atomicAdd(w.sync + 1, 1u);
  __syncthreads();
  const uint32_t ticket = s_ticket + w.skip;
  const bool valid = ticket < 2u * w.nt * w.chunks;  // false only if the counter was disturbed
  const uint32_t j = ticket / w.chunks, c = ticket - j * w.chunks;
  int par = 0;
  uint32_t t = 0;
  if (valid) wave_unit(j, w.nt, w.lag, par, t);
  if (par == 1) {
    if (threadIdx.x == 0) wave_wait_even(w, t);
    __syncthreads();
  }
  const uint32_t i = c * blockDim.x + threadIdx.x;
  if (valid && i < w.half_slice) {
    const int64_t h = int64_t(t) * w.half_slice + i;
    if constexpr (QUAT)
      quat_pass_body<R, MODE, REUNIT, true>(p, par, h);
    else
      pass_body<R, N, S, MODE, ROWS2, REUNIT, true>(p, par, h);
  }
  if (valid && par == 0) {
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();  // the block's link stores before the count that publishes them
      atomicAdd(w.sync + kWaveSyncWords + t, 1u);
    }
  }
}

template <class R, int N, int S, int MODE, int VAR, bool REUNIT>
__global__ void __launch_bounds__(kMaxBlockThreads) update_pair_mat(const PassParams p, const WaveParams w) {
  wavefront<R, N, S, MODE, (VAR & 2) != 0, REUNIT, false>(p, w);
}

template <class R, int N, int S, int MODE, int VAR, bool REUNIT>
__global__ void __launch_bounds__(128, kOccBlocks) update_pair_mat_occ(const PassParams p, const WaveParams w) {
  wavefront<R, N, S, MODE, (VAR & 2) != 0, REUNIT, false>(p, w);
}

template <class R, int MODE, bool REUNIT>
__global__ void __launch_bounds__(kMaxBlockThreads) update_pair_quat(const PassParams p, const WaveParams w) {
  wavefront<R, 2, kQuat, MODE, false, REUNIT, true>(p, w);
}

// ---------------------------------------------------------------------------
// Overrelaxation pass with two links per thread in packed FP32 (variant bit 16,
// SU(3) FP32 storage).  Lane 0 of every F2 value belongs to half-site h0, lane 1
// to h1 = h0 + blockDim.x; the staple, W = U Sigma^+ and the subgroup updates
// are the float templates run with R = F2, so every link gets bitwise the
// result of the one-link kernel in half the FP32 instructions (the pass is
// bound by instruction issue).  Square roots and divisions are per lane.
// ---------------------------------------------------------------------------
template <int N, int S, int KL>
__device__ __forceinline__ Mat<F2, N> load_mat2(const char* blk, int64_t Vh, int64_t h0, int64_t h1) {
  constexpr int NR = Layout<float, N, S>::nreals;
  float r0[NR], r1[NR];
  load_reals<float, NR, KL>(blk, Vh, h0, r0);
  load_reals<float, NR, KL>(blk, Vh, h1, r1);
  Mat<F2, N> m;
  constexpr int rows = S == kTwoRow ? 2 : N;
#pragma unroll
  for (int i = 0; i < rows; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j)
      m.e[i][j] = {f2_pack(r0[2 * (N * i + j)], r1[2 * (N * i + j)]),
                   f2_pack(r0[2 * (N * i + j) + 1], r1[2 * (N * i + j) + 1])};
  if constexpr (S == kTwoRow) su3_third_row(m);
  return m;
}

template <int N, int S>
__device__ __forceinline__ void store_mat2(char* blk, int64_t Vh, int64_t h0, int64_t h1, bool store1,
                                           const Mat<F2, N>& m) {
  Mat<float, N> a, b;
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) {
      f2_unpack(m.e[i][j].re, a.e[i][j].re, b.e[i][j].re);
      f2_unpack(m.e[i][j].im, a.e[i][j].im, b.e[i][j].im);
    }
  store_mat<float, N, S>(blk, Vh, h0, a);
  if (store1) store_mat<float, N, S>(blk, Vh, h1, b);
}

template <int N>
__device__ __forceinline__ Mat<double, N> lane_to_double(const Mat<F2, N>& m, int lane) {
  Mat<double, N> d;
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) {
      float r0, r1, i0, i1;
      f2_unpack(m.e[i][j].re, r0, r1);
      f2_unpack(m.e[i][j].im, i0, i1);
      d.e[i][j] = {double(lane ? r1 : r0), double(lane ? i1 : i0)};
    }
  return d;
}

template <int N, int S, bool REUNIT>
__device__ __forceinline__ void or_pass_body2(const PassParams& p, int par, int64_t h0, int64_t h1, bool act1) {
  const Geom& g = p.g;
  const int mu = p.mu, opp = par ^ 1;
  const Site s0 = decode_half(g, h0, par), s1 = decode_half(g, h1, par);
  const uint32_t lex0 = uint32_t(s0.lex), lex1 = uint32_t(s1.lex);
  const int cmu0 = coord_of(s0, mu), cmu1 = coord_of(s1, mu);
  const uint32_t pmu0 = fwd(g, lex0, cmu0, mu), pmu1 = fwd(g, lex1, cmu1, mu);

  Mat<F2, N> st;
  mat_zero(st);
#pragma unroll
  for (int nu = 0; nu < 4; ++nu) {
    if (nu == mu) continue;
    const uint32_t pnu0 = fwd(g, lex0, s0.c[nu], nu), pnu1 = fwd(g, lex1, s1.c[nu], nu);
    const uint32_t mnu0 = bwd(g, lex0, s0.c[nu], nu), mnu1 = bwd(g, lex1, s1.c[nu], nu);
    const uint32_t mnpm0 = fwd(g, mnu0, cmu0, mu), mnpm1 = fwd(g, mnu1, cmu1, mu);
    {  // U_nu(x) U_mu(x+nu) U_nu(x+mu)^+
      const Mat<F2, N> a = load_mat2<N, S, kLoadNc>(block_ptr(p, nu, par), g.Vh, h0, h1);
      const Mat<F2, N> b = load_mat2<N, S, kLoadNc>(block_ptr(p, mu, opp), g.Vh, pnu0 >> 1, pnu1 >> 1);
      const Mat<F2, N> t = mul_nn(a, b);
      const Mat<F2, N> c = load_mat2<N, S, kLoadNc>(block_ptr(p, nu, opp), g.Vh, pmu0 >> 1, pmu1 >> 1);
      acc_nd(st, t, c);
    }
    {  // U_nu(x-nu)^+ U_mu(x-nu) U_nu(x-nu+mu)
      const Mat<F2, N> a = load_mat2<N, S, kLoadNc>(block_ptr(p, nu, opp), g.Vh, mnu0 >> 1, mnu1 >> 1);
      const Mat<F2, N> b = load_mat2<N, S, kLoadNc>(block_ptr(p, mu, opp), g.Vh, mnu0 >> 1, mnu1 >> 1);
      const Mat<F2, N> t = mul_dn(a, b);
      const Mat<F2, N> c = load_mat2<N, S, kLoadNc>(block_ptr(p, nu, par), g.Vh, mnpm0 >> 1, mnpm1 >> 1);
      acc_nn(st, t, c);
    }
  }

  char* ublk = p.links + (2 * mu + par) * p.block_bytes;
  Mat<F2, N> u = load_mat2<N, S, kLoadPlain>(ublk, g.Vh, h0, h1);

#pragma unroll
  for (int i = 0; i < N - 1; ++i) {
#pragma unroll
    for (int j = i + 1; j < N; ++j) {
      // or_block and or_element of each lane, operation by operation (v2 = 2v)
      const Quat<F2> v2 = or_block<F2, N>(u, st, i, j);
      const F2 n3 = fma(v2.a1, v2.a1, fma(v2.a2, v2.a2, v2.a3 * v2.a3));
      float k0, k1;
      f2_unpack(fma(v2.a0, v2.a0, n3), k0, k1);
      const bool ok0 = k0 > 4e-30f && isfinite(k0), ok1 = k1 > 4e-30f && isfinite(k1);
      const F2 inv = f2_pack(ok0 ? 1.0f / k0 : 0.0f, ok1 ? 1.0f / k1 : 0.0f);
      const F2 c = -(v2.a0 + v2.a0) * inv;
      Quat<F2> a = {fma(v2.a0, v2.a0, -n3) * inv, c * v2.a1, c * v2.a2, c * v2.a3};
      if (!(ok0 && ok1)) {
        // a skipped subgroup of one lane: the identity there (applies exactly)
        float x0, x1;
        f2_unpack(a.a0, x0, x1);
        a.a0 = f2_pack(ok0 ? x0 : 1.0f, ok1 ? x1 : 1.0f);
        f2_unpack(a.a1, x0, x1);
        a.a1 = f2_pack(ok0 ? x0 : 0.0f, ok1 ? x1 : 0.0f);
        f2_unpack(a.a2, x0, x1);
        a.a2 = f2_pack(ok0 ? x0 : 0.0f, ok1 ? x1 : 0.0f);
        f2_unpack(a.a3, x0, x1);
        a.a3 = f2_pack(ok0 ? x0 : 0.0f, ok1 ? x1 : 0.0f);
      }
      apply_rows(u, i, j, a);
    }
  }
  if constexpr (REUNIT) {
    Mat<float, N> f[2];
#pragma unroll
    for (int lane = 0; lane < 2; ++lane) {
      Mat<double, N> d = lane_to_double<N>(u, lane);
      if (reunit_selected(p, global_lex(p, lane ? lex1 : lex0) >> 1)) reunit_d<N>(d);
      f[lane] = mat_cast<double, float, N>(d);
    }
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
      for (int b = 0; b < N; ++b)
        u.e[a][b] = {f2_pack(f[0].e[a][b].re, f[1].e[a][b].re), f2_pack(f[0].e[a][b].im, f[1].e[a][b].im)};
  }
  store_mat2<N, S>(ublk, g.Vh, h0, h1, act1, u);
}

template <int N, int S, bool REUNIT>
__global__ void __launch_bounds__(128) update_or_pass2(const PassParams p) {
  const int64_t h0 = p.h_begin + int64_t(blockIdx.x) * (2 * blockDim.x) + threadIdx.x;
  if (h0 >= p.h_end) return;
  int64_t h1 = h0 + blockDim.x;
  const bool act1 = h1 < p.h_end;
  if (!act1) h1 = h0;  // the ragged tail: lane 1 repeats lane 0 and is not stored
  or_pass_body2<N, S, REUNIT>(p, p.parity, h0, h1, act1);
}

struct LinkParams {
  char* links;
  int64_t block_bytes;
  Geom g;
  uint2 key;
  int hot;
  uint32_t lex_offset, v_global;  // a slab's place in the whole lattice (as in PassParams)
};

template <class R, int N, int S>
__global__ void __launch_bounds__(256) reunit_kernel(const LinkParams p) {
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= 8 * p.g.Vh) return;
  const int b = int(idx / p.g.Vh);
  const int64_t h = idx - int64_t(b) * p.g.Vh;
  char* blk = p.links + b * p.block_bytes;
  if constexpr (S == kQuat) {
    const Quat<R> q = load_quat<R, kLoadPlain>(blk, p.g.Vh, h);
    const double a0 = q.a0, a1 = q.a1, a2 = q.a2, a3 = q.a3;
    const double inv = rsqrt_near_one(fma(a1, a1, fma(a2, a2, fma(a3, a3, a0 * a0))));
    store_quat<R>(blk, p.g.Vh, h, Quat<R>{R(a0 * inv), R(a1 * inv), R(a2 * inv), R(a3 * inv)});
  } else {
    Mat<double, N> m = mat_cast_int<R, double, N>(load_mat<R, N, S, kLoadPlain>(blk, p.g.Vh, h));
    reunit_d<N>(m);
    store_mat<R, N, S>(blk, p.g.Vh, h, mat_cast_int<double, R, N>(m));
  }
}

// Cold start: identity.  Hot start: complex Gaussians (Box-Muller on Philox
// counter (mu*V + lex, 0, call, 2)), row by row, then FP64 re-unitarization
// (Gram-Schmidt + determinant phase): a Haar-random SU(Nc) matrix.
template <class R, int N, int S>
__global__ void __launch_bounds__(256) init_kernel(const LinkParams p) {
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= 8 * p.g.Vh) return;
  const int b = int(idx / p.g.Vh);
  const int64_t h = idx - int64_t(b) * p.g.Vh;
  const int mu = b >> 1, par = b & 1;
  char* blk = p.links + b * p.block_bytes;
  Mat<double, N> m;
  if (!p.hot) {
    mat_identity(m);
  } else {
    const Site s = decode_half(p.g, h, par);
    uint32_t glex = uint32_t(s.lex) + p.lex_offset;
    if (glex >= p.v_global) glex -= p.v_global;
    const uint32_t link_id = uint32_t(mu) * p.v_global + glex;
    constexpr int kNormals = 2 * N * N;
    double gauss[kNormals + 3];
#pragma unroll
    for (int call = 0; 4 * call < kNormals; ++call) {
      const uint4 u = philox4x32_10(make_uint4(link_id, 0u, uint32_t(call), kTagInit), p.key);
      const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
      for (int pair = 0; pair < 2; ++pair) {
        const double rad = sqrt(-2.0 * log(u01<double>(w[2 * pair])));
        double sn, cs;
        sincospi(2.0 * u01<double>(w[2 * pair + 1]), &sn, &cs);
        if (4 * call + 2 * pair < kNormals) gauss[4 * call + 2 * pair] = rad * cs;
        if (4 * call + 2 * pair + 1 < kNormals) gauss[4 * call + 2 * pair + 1] = rad * sn;
      }
    }
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
      for (int j = 0; j < N; ++j) m.e[i][j] = {gauss[2 * (N * i + j)], gauss[2 * (N * i + j) + 1]};
    reunit_d<N>(m);
  }
  store_mat<R, N, S>(blk, p.g.Vh, h, mat_cast<double, R, N>(m));
}

// ---------------------------------------------------------------------------
// Deterministic FP64 reductions: per-thread sums -> warp shuffles -> block ->
// one partial per block; the last block to finish adds the partials in a
// fixed order (lane l sums partials l, l + 32, ..., then a warp shuffle tree)
// and writes the scaled result, then re-arms the counter.
// ---------------------------------------------------------------------------
struct ReduceParams {
  double* partials;      // [gridDim.x * K]
  unsigned* counter;     // zero before the launch, zero after
  double* out;           // result slot base
  const uint32_t* slot;  // optional: results go to out[((*slot % cap) * stride + offset) * K + k]
  int cap;
  int stride, offset;    // row stride and column of a table of lattices (1, 0 for one lattice)
  double scale;
};

template <int K>
__device__ __forceinline__ void reduce_finish(double (&v)[K], const ReduceParams& rp) {
  __shared__ double sh[kMaxBlockThreads / 32][K];
  __shared__ bool am_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    if (lane == 0) sh[warp][k] = v[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double s = 0.0;
      for (int w = 0; w < nwarps; ++w) s += sh[w][k];
      rp.partials[blockIdx.x * K + k] = s;
    }
    __threadfence();
    const unsigned done = atomicAdd(rp.counter, 1u);
    am_last = (done == gridDim.x - 1);
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double s = 0.0;
      for (int b = lane; b < int(gridDim.x); b += 32) s += __ldcg(&rp.partials[b * K + k]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (lane == 0) {
        const int idx = rp.slot ? int(*rp.slot % uint32_t(rp.cap)) : 0;
        rp.out[(int64_t(idx) * rp.stride + rp.offset) * K + k] = s * rp.scale;
      }
    }
    if (lane == 0) *rp.counter = 0u;
  }
}

struct ObsParams {
  const char* links;
  int64_t block_bytes;
  Geom g;
  int64_t h_begin, h_end;  // half-sites measured (per parity); a slab's interior slices
};

__device__ __forceinline__ const char* obs_block(const ObsParams& p, int d, int par) {
  return p.links + (2 * d + par) * p.block_bytes;
}

// Entry e = k Nc + j of a full-storage link at half-site h of a block.
template <class R, int N>
__device__ __forceinline__ Cpx<R> load_entry(const char* blk, int64_t Vh, int64_t h, int e) {
  if constexpr (sizeof(R) == 8) {  // one complex double per 16-byte component
    const double2 v = __ldg(reinterpret_cast<const double2*>(blk + (int64_t(e) * Vh + h) * 16));
    return {v.x, v.y};
  } else {
    constexpr int n16 = Layout<R, N, kFull>::n16;
    const int cc = e >> 1;
    const char* q = cc < n16 ? blk + (int64_t(cc) * Vh + h) * 16 + (e & 1) * 8 : blk + int64_t(n16) * Vh * 16 + h * 8;
    const float2 v = __ldg(reinterpret_cast<const float2*>(q));
    return {v.x, v.y};
  }
}

// Re Tr((A B)(C D)^+) as retr_nd(mul_nn(A, B), mul_nn(C, D)) computes it, the
// same operations in the same order, row by row: a row of A and of C at a time,
// the entries of B and D read as they are used (from L1), so that no whole
// Nc x Nc product is held (for Nc >= 5 the whole products do not fit in
// registers and went to local memory).
template <class R, int N>
__device__ __forceinline__ R retr_products_by_rows(const char* a, int64_t ha, const char* b, int64_t hb, const char* c,
                                                   int64_t hc, const char* d, int64_t hd, int64_t Vh) {
  R s = R(0);
#pragma unroll 1
  for (int i = 0; i < N; ++i) {
    Cpx<R> ar[N], cr[N], t1[N], t2[N];
#pragma unroll
    for (int k = 0; k < N; ++k) {
      ar[k] = load_entry<R, N>(a, Vh, ha, i * N + k);
      cr[k] = load_entry<R, N>(c, Vh, hc, i * N + k);
    }
#pragma unroll
    for (int j = 0; j < N; ++j) {
      t1[j] = cmul(ar[0], load_entry<R, N>(b, Vh, hb, j));
      t2[j] = cmul(cr[0], load_entry<R, N>(d, Vh, hd, j));
#pragma unroll
      for (int k = 1; k < N; ++k) {
        cfma(t1[j], ar[k], load_entry<R, N>(b, Vh, hb, k * N + j));
        cfma(t2[j], cr[k], load_entry<R, N>(d, Vh, hd, k * N + j));
      }
    }
#pragma unroll
    for (int j = 0; j < N; ++j) {
      s = fma(t1[j].re, t2[j].re, s);
      s = fma(t1[j].im, t2[j].im, s);
    }
  }
  return s;
}

// Re Tr(X Y^+) of two SU(3) matrices given by rows 0 and 1 (row 2 of each is
// conj(row0 x row1)).  With d_ab = sum_j X_aj conj(Y_bj), rows 0 and 1 give
// Re(d00 + d11), and row 2 gives Re conj(d00 d11 - d01 d10) by the identity
// (a x b).(c x d) = (a.c)(b.d) - (a.d)(b.c) for the cross products of rows.
template <class R>
__device__ __forceinline__ R retr_nd_two_row(const Cpx<R> (&x)[2][3], const Cpx<R> (&y)[2][3]) {
  Cpx<R> d[2][2];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      d[a][b] = cmulc(x[a][0], y[b][0]);
#pragma unroll
      for (int j = 1; j < 3; ++j) cfmac(d[a][b], x[a][j], y[b][j]);
    }
  R t = fma(d[0][0].re, d[1][1].re, -(d[0][0].im * d[1][1].im));
  t = fma(-d[0][1].re, d[1][0].re, t);
  t = fma(d[0][1].im, d[1][0].im, t);
  return d[0][0].re + d[1][1].re + t;
}

// Rows 0 and 1 of A B
template <class R>
__device__ __forceinline__ void mul_nn_two_rows(const Mat<R, 3>& a, const Mat<R, 3>& b, Cpx<R> (&c)[2][3]) {
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Cpx<R> s = cmul(a.e[i][0], b.e[0][j]);
      cfma(s, a.e[i][1], b.e[1][j]);
      cfma(s, a.e[i][2], b.e[2][j]);
      c[i][j] = s;
    }
}

// Sum over the six plaquettes P_{mu nu}(x) = U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+
// (Eq. 4) of one site (half-site h of parity par), ReTr in the storage
// precision, each added in FP64.  SU(3) two-row links: each ReTr from rows 0 and
// 1 of the two products (retr_nd_two_row).
template <class R, int N, int S>
__device__ __forceinline__ double site_plaquette(const ObsParams& p, int par, int64_t h) {
  const Geom& g = p.g;
  const Site s = decode_half(g, h, par);
  const uint32_t lex = uint32_t(s.lex);
  double acc = 0.0;
  if constexpr (S == kTwoRow) {
#pragma unroll
    for (int mu = 0; mu < 3; ++mu) {
      const int64_t xpmu = fwd(g, lex, s.c[mu], mu) >> 1;
      const Mat<R, 3> umx = load_mat<R, 3, S>(obs_block(p, mu, par), g.Vh, h);
#pragma unroll
      for (int nu = mu + 1; nu < 4; ++nu) {
        const int64_t xpnu = fwd(g, lex, s.c[nu], nu) >> 1;
        Cpx<R> t1[2][3], t2[2][3];
        mul_nn_two_rows(umx, load_mat<R, 3, S>(obs_block(p, nu, par ^ 1), g.Vh, xpmu), t1);
        mul_nn_two_rows(load_mat<R, 3, S>(obs_block(p, nu, par), g.Vh, h),
                        load_mat<R, 3, S>(obs_block(p, mu, par ^ 1), g.Vh, xpnu), t2);
        acc += double(retr_nd_two_row(t1, t2));
      }
    }
    return acc;
  }
#pragma unroll
  for (int mu = 0; mu < 3; ++mu) {
    const int64_t xpmu = fwd(g, lex, s.c[mu], mu) >> 1;
    if constexpr (S == kQuat) {
      const Quat<R> umx = load_quat<R>(obs_block(p, mu, par), g.Vh, h);
#pragma unroll
      for (int nu = mu + 1; nu < 4; ++nu) {
        const int64_t xpnu = fwd(g, lex, s.c[nu], nu) >> 1;
        const Quat<R> unx = load_quat<R>(obs_block(p, nu, par), g.Vh, h);
        const Quat<R> t1 = qmul(umx, load_quat<R>(obs_block(p, nu, par ^ 1), g.Vh, xpmu));
        const Quat<R> t2 = qmul(unx, load_quat<R>(obs_block(p, mu, par ^ 1), g.Vh, xpnu));
        acc += double(R(2) * (t1.a0 * t2.a0 + t1.a1 * t2.a1 + t1.a2 * t2.a2 + t1.a3 * t2.a3));
      }
    } else if constexpr (N >= 5) {
#pragma unroll 1
      for (int nu = mu + 1; nu < 4; ++nu) {
        const int64_t xpnu = fwd(g, lex, s.c[nu], nu) >> 1;
        acc += double(retr_products_by_rows<R, N>(obs_block(p, mu, par), h, obs_block(p, nu, par ^ 1), xpmu,
                                                  obs_block(p, nu, par), h, obs_block(p, mu, par ^ 1), xpnu, g.Vh));
      }
    } else {
      const Mat<R, N> umx = load_mat<R, N, S>(obs_block(p, mu, par), g.Vh, h);
#pragma unroll
      for (int nu = mu + 1; nu < 4; ++nu) {
        const int64_t xpnu = fwd(g, lex, s.c[nu], nu) >> 1;
        const Mat<R, N> t1 = mul_nn(umx, load_mat<R, N, S>(obs_block(p, nu, par ^ 1), g.Vh, xpmu));
        const Mat<R, N> t2 = mul_nn(load_mat<R, N, S>(obs_block(p, nu, par), g.Vh, h),
                                    load_mat<R, N, S>(obs_block(p, mu, par ^ 1), g.Vh, xpnu));
        acc += double(retr_nd(t1, t2));
      }
    }
  }
  return acc;
}

// Tr of the ordered product of U_t over t at spatial site xs (products in the
// storage precision, trace returned in FP64).
template <class R, int N, int S>
__device__ __forceinline__ void site_polyakov(const ObsParams& p, int64_t xs, double& re, double& im) {
  const Geom& g = p.g;
  const int64_t nsp = int64_t(g.nx) * g.ny * g.nz;
  const int x = int(xs % g.nx);
  const int y = int((xs / g.nx) % g.ny);
  const int z = int(xs / (int64_t(g.nx) * g.ny));
  const int sp = (x + y + z) & 1;
  re = 0.0;
  im = 0.0;
  if constexpr (S == kQuat) {
    Quat<R> P = load_quat<R>(obs_block(p, 3, sp), g.Vh, xs >> 1);
    for (int t = 1; t < g.nt; ++t) {
      const int64_t lex = xs + int64_t(t) * nsp;
      P = qmul(P, load_quat<R>(obs_block(p, 3, (sp + t) & 1), g.Vh, lex >> 1));
    }
    re = double(R(2) * P.a0);  // Tr of [[a0 + i a3, .], [., a0 - i a3]] is real
  } else {
    Mat<R, N> P = load_mat<R, N, S>(obs_block(p, 3, sp), g.Vh, xs >> 1);
    for (int t = 1; t < g.nt; ++t) {
      const int64_t lex = xs + int64_t(t) * nsp;
      P = mul_nn(P, load_mat<R, N, S>(obs_block(p, 3, (sp + t) & 1), g.Vh, lex >> 1));
    }
#pragma unroll
    for (int d = 0; d < N; ++d) {
      re += double(P.e[d][d].re);
      im += double(P.e[d][d].im);
    }
  }
}

// <P> of one lattice: grid-stride over sites, deterministic FP64 reduction.
// Nc <= 4: idx < V visits half-site idx / 2 of parity idx % 2, both parities
// of a half-site in turn.  A link is read as its own site's link and as a
// forward neighbour of the other parity at nearby half-site indices (within
// Nx Ny Nz / 2), so the second read finds it in L2; in parity-block order the
// two reads are half the lattice apart and each link comes from DRAM twice.
// Nc >= 5 keeps parity-block order, whose loop keeps SU(6) FP32 from spilling
// (its plaquette is arithmetic-bound).  (A loop over a sub-range here costs
// SU(6) its register allocation too: a kernel of its own does the slabs.)
template <class R, int N, int S>
__global__ void __launch_bounds__(256) plaquette_kernel(const ObsParams p, const ReduceParams rp) {
  double acc[1] = {0.0};
  for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < p.g.V;
       idx += int64_t(gridDim.x) * blockDim.x) {
    if constexpr (N <= 4) {
      acc[0] += site_plaquette<R, N, S>(p, int(idx & 1), idx >> 1);
    } else {
      const int par = idx >= p.g.Vh ? 1 : 0;
      acc[0] += site_plaquette<R, N, S>(p, par, idx - par * p.g.Vh);
    }
  }
  reduce_finish<1>(acc, rp);
}

// A slab's interior: half-sites [h_begin, h_end) of each parity.
template <class R, int N, int S>
__global__ void __launch_bounds__(256) plaquette_slab_kernel(const ObsParams p, const ReduceParams rp) {
  double acc[1] = {0.0};
  const int64_t cnt = p.h_end - p.h_begin;
  for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < 2 * cnt;
       idx += int64_t(gridDim.x) * blockDim.x) {
    const int par = idx >= cnt ? 1 : 0;
    acc[0] += site_plaquette<R, N, S>(p, par, p.h_begin + idx - par * cnt);
  }
  reduce_finish<1>(acc, rp);
}

// Polyakov loop of one lattice: grid-stride over spatial sites, FP64 (re, im).
template <class R, int N, int S>
__global__ void __launch_bounds__(256) polyakov_kernel(const ObsParams p, const ReduceParams rp) {
  const int64_t nsp = int64_t(p.g.nx) * p.g.ny * p.g.nz;
  double acc[2] = {0.0, 0.0};
  for (int64_t xs = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; xs < nsp;
       xs += int64_t(gridDim.x) * blockDim.x) {
    double re, im;
    site_polyakov<R, N, S>(p, xs, re, im);
    acc[0] += re;
    acc[1] += im;
  }
  reduce_finish<2>(acc, rp);
}

// ---------------------------------------------------------------------------
// Health of the stored links: per link the largest entry of |U U^+ - 1| and
// |det U - 1| in FP64 (of the stored values, the rebuilt row included), and
// whether any entry is not finite.  out[0], out[1]: the maxima as the bit
// patterns of non-negative doubles (ordered like the values, so an integer
// atomicMax takes the maximum); out[2]: the count of non-finite links.
// ---------------------------------------------------------------------------
template <class R, int N, int S>
__global__ void __launch_bounds__(256) check_links_kernel(const ObsParams p, unsigned long long* out) {
  double dev = 0.0, ddet = 0.0;
  unsigned long long bad = 0;
  for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < 8 * p.g.Vh;
       idx += int64_t(gridDim.x) * blockDim.x) {
    const int b = int(idx / p.g.Vh);
    const int64_t h = idx - int64_t(b) * p.g.Vh;
    const Mat<double, N> m = mat_cast<R, double, N>(load_mat<R, N, S>(p.links + b * p.block_bytes, p.g.Vh, h));
    bool finite = true;
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
      for (int j = 0; j < N; ++j) finite = finite && isfinite(m.e[i][j].re) && isfinite(m.e[i][j].im);
    if (!finite) {
      ++bad;
      continue;
    }
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
      for (int j = 0; j < N; ++j) {
        // (U U^+)_ij = sum_k U_ik conj(U_jk)
        Cpx<double> x = {0.0, 0.0};
#pragma unroll
        for (int k = 0; k < N; ++k) cfmac(x, m.e[i][k], m.e[j][k]);
        if (i == j) x.re -= 1.0;
        dev = fmax(dev, sqrt(x.re * x.re + x.im * x.im));
      }
    const Cpx<double> d = det_lu<N>(m);
    ddet = fmax(ddet, sqrt((d.re - 1.0) * (d.re - 1.0) + d.im * d.im));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    dev = fmax(dev, __shfl_down_sync(0xffffffffu, dev, o));
    ddet = fmax(ddet, __shfl_down_sync(0xffffffffu, ddet, o));
    bad += __shfl_down_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out, static_cast<unsigned long long>(__double_as_longlong(dev)));
    atomicMax(out + 1, static_cast<unsigned long long>(__double_as_longlong(ddet)));
    if (bad) atomicAdd(out + 2, bad);
  }
}

// ---------------------------------------------------------------------------
// Polyakov loop of a lattice cut into t-slabs: each slab multiplies U_t over its
// interior slices, in t order, at every spatial site; then the slabs' partial
// products are multiplied in slab order and traced (storage precision products,
// FP64 trace and sum, as for one lattice).
// ---------------------------------------------------------------------------
template <class R, int N, int S>
using PolyPart = typename std::conditional<S == kQuat, Quat<R>, Mat<R, N>>::type;

template <class R, int N, int S>
__global__ void __launch_bounds__(128) polyakov_partial_kernel(const ObsParams p, int t_begin, int t_end, void* out) {
  const Geom& g = p.g;
  const int64_t nsp = int64_t(g.nx) * g.ny * g.nz;
  const int64_t xs = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (xs >= nsp) return;
  const int x = int(xs % g.nx);
  const int y = int((xs / g.nx) % g.ny);
  const int z = int(xs / (int64_t(g.nx) * g.ny));
  const int sp = (x + y + z) & 1;
  PolyPart<R, N, S>* o = static_cast<PolyPart<R, N, S>*>(out);
  if constexpr (S == kQuat) {
    Quat<R> P = load_quat<R>(obs_block(p, 3, (sp + t_begin) & 1), g.Vh, (xs + int64_t(t_begin) * nsp) >> 1);
    for (int t = t_begin + 1; t < t_end; ++t)
      P = qmul(P, load_quat<R>(obs_block(p, 3, (sp + t) & 1), g.Vh, (xs + int64_t(t) * nsp) >> 1));
    o[xs] = P;
  } else {
    Mat<R, N> P = load_mat<R, N, S>(obs_block(p, 3, (sp + t_begin) & 1), g.Vh, (xs + int64_t(t_begin) * nsp) >> 1);
    for (int t = t_begin + 1; t < t_end; ++t)
      P = mul_nn(P, load_mat<R, N, S>(obs_block(p, 3, (sp + t) & 1), g.Vh, (xs + int64_t(t) * nsp) >> 1));
    o[xs] = P;
  }
}

template <class R, int N, int S>
__global__ void __launch_bounds__(128) polyakov_combine_kernel(const void* const* parts, int n, int64_t nsp,
                                                               const ReduceParams rp) {
  double acc[2] = {0.0, 0.0};
  for (int64_t xs = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; xs < nsp; xs += int64_t(gridDim.x) * blockDim.x) {
    PolyPart<R, N, S> P = static_cast<const PolyPart<R, N, S>*>(parts[0])[xs];
    for (int k = 1; k < n; ++k) {
      const PolyPart<R, N, S> Q = static_cast<const PolyPart<R, N, S>*>(parts[k])[xs];
      if constexpr (S == kQuat)
        P = qmul(P, Q);
      else
        P = mul_nn(P, Q);
    }
    if constexpr (S == kQuat) {
      acc[0] += double(R(2) * P.a0);
    } else {
#pragma unroll
      for (int d = 0; d < N; ++d) {
        acc[0] += double(P.e[d][d].re);
        acc[1] += double(P.e[d][d].im);
      }
    }
  }
  reduce_finish<2>(acc, rp);
}

// ---------------------------------------------------------------------------
// Batched kernels: many independent lattices ("chains") of one (Nc, storage,
// precision) in one launch.  Block b belongs to chain c with
// start[c] <= b < start[c+1]; thread 0 finds c and stages the chain's
// parameters in shared memory for the block.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int find_chain(const uint32_t* start, int n, uint32_t b) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (start[mid] <= b)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

template <class R, int N, int S, int MODE, int VAR, bool REUNIT>
__device__ __forceinline__ void batch_pass_body(const BatchParams& bp, int mu, int parity, uint32_t step_offset,
                                                uint32_t rmod, uint32_t rrem) {
  __shared__ PassParams sp;
  __shared__ uint32_t first;
  if (threadIdx.x == 0) {
    const int c = find_chain(bp.start, bp.n, blockIdx.x);
    const ChainDesc& d = bp.chains[c];
    first = bp.start[c];
    sp.links = d.links;
    sp.block_bytes = d.block_bytes;
    sp.g = d.g;
    sp.mu = mu;
    sp.parity = parity;
    sp.alpha_coef = d.alpha_coef;
    sp.key = d.key;
    sp.hb_step = d.hb_step;
    sp.step_offset = step_offset;
    sp.reunit_mod = rmod;
    sp.reunit_rem = rrem;
    sp.h_begin = 0;
    sp.h_end = d.g.Vh;
    sp.lex_offset = 0u;
    sp.v_global = uint32_t(d.g.V);
  }
  __syncthreads();
  const PassParams p = sp;  // a private copy: the body need not re-read shared memory
  const int64_t h = int64_t(blockIdx.x - first) * blockDim.x + threadIdx.x;
  if (h >= p.g.Vh) return;
  if constexpr (S == kQuat)
    quat_pass_body<R, MODE, REUNIT>(p, p.parity, h);
  else
    pass_body<R, N, S, MODE, (VAR & 2) != 0, REUNIT>(p, p.parity, h);
}

template <class R, int N, int S, int MODE, int VAR, bool REUNIT>
__global__ void __launch_bounds__(kMaxBlockThreads)
    update_pass_batch(const BatchParams bp, int mu, int parity, uint32_t step_offset, uint32_t rmod, uint32_t rrem) {
  batch_pass_body<R, N, S, MODE, VAR, REUNIT>(bp, mu, parity, step_offset, rmod, rrem);
}

template <class R, int N, int S, int MODE, int VAR, bool REUNIT>
__global__ void __launch_bounds__(128, kOccBlocks)
    update_pass_batch_occ(const BatchParams bp, int mu, int parity, uint32_t step_offset, uint32_t rmod,
                          uint32_t rrem) {
  batch_pass_body<R, N, S, MODE, VAR, REUNIT>(bp, mu, parity, step_offset, rmod, rrem);
}

template <class R, int N, int MODE>
__global__ void __launch_bounds__(128)
    update_pass_batch_group(const BatchParams bp, int mu, int parity, uint32_t step_offset) {
  __shared__ PassParams sp;
  __shared__ uint32_t first;
  __shared__ __align__(16) char tile[GroupTile<R, N>::kBytes];
  __shared__ uint32_t hidx[3][GroupTile<R, N>::LPB];
  if (threadIdx.x == 0) {
    const int c = find_chain(bp.start, bp.n, blockIdx.x);
    const ChainDesc& d = bp.chains[c];
    first = bp.start[c];
    sp.links = d.links;
    sp.block_bytes = d.block_bytes;
    sp.g = d.g;
    sp.mu = mu;
    sp.parity = parity;
    sp.alpha_coef = d.alpha_coef;
    sp.key = d.key;
    sp.hb_step = d.hb_step;
    sp.step_offset = step_offset;
    sp.reunit_mod = 0u;
    sp.reunit_rem = 0u;
    sp.h_begin = 0;
    sp.h_end = d.g.Vh;
    sp.lex_offset = 0u;
    sp.v_global = uint32_t(d.g.V);
  }
  __syncthreads();
  const PassParams p = sp;  // a private copy: the body's barriers would force re-reads of shared memory
  group_pass_body<R, N, MODE>(p, int64_t(blockIdx.x - first) * Group<R, N>::LPB, p.g.Vh, tile, hidx);
}

// stage the chain's observable parameters of this block in shared memory
__device__ __forceinline__ void batch_obs_chain(const BatchParams& bp, ObsParams& sp, uint32_t& first) {
  if (threadIdx.x == 0) {
    const int c = find_chain(bp.start, bp.n, blockIdx.x);
    const ChainDesc& d = bp.chains[c];
    first = bp.start[c];
    sp.links = d.links;
    sp.block_bytes = d.block_bytes;
    sp.g = d.g;
    sp.h_begin = 0;
    sp.h_end = d.g.Vh;
  }
  __syncthreads();
}

template <class R, int N, int S>
__global__ void __launch_bounds__(128) reunit_batch(const BatchParams bp) {
  __shared__ ObsParams sp;
  __shared__ uint32_t first;
  batch_obs_chain(bp, sp, first);
  const int64_t idx = int64_t(blockIdx.x - first) * blockDim.x + threadIdx.x;
  if (idx >= 8 * sp.g.Vh) return;
  const int b = int(idx / sp.g.Vh);
  const int64_t h = idx - int64_t(b) * sp.g.Vh;
  char* blk = const_cast<char*>(sp.links) + b * sp.block_bytes;
  if constexpr (S == kQuat) {
    const Quat<R> q = load_quat<R, kLoadPlain>(blk, sp.g.Vh, h);
    const double a0 = q.a0, a1 = q.a1, a2 = q.a2, a3 = q.a3;
    const double inv = rsqrt_near_one(fma(a1, a1, fma(a2, a2, fma(a3, a3, a0 * a0))));
    store_quat<R>(blk, sp.g.Vh, h, Quat<R>{R(a0 * inv), R(a1 * inv), R(a2 * inv), R(a3 * inv)});
  } else {
    Mat<double, N> m = mat_cast_int<R, double, N>(load_mat<R, N, S, kLoadPlain>(blk, sp.g.Vh, h));
    reunit_d<N>(m);
    store_mat<R, N, S>(blk, sp.g.Vh, h, mat_cast_int<double, R, N>(m));
  }
}

// sum of v over the block into thread 0 (warp shuffles, then shared memory)
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K]) {
  __shared__ double sh[kMaxBlockThreads / 32][K];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    if (lane == 0) sh[warp][k] = v[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double s = 0.0;
      for (int w = 0; w < nwarps; ++w) s += sh[w][k];
      v[k] = s;
    }
  }
}

// per-block partial <P> sums, one block per 256 sites of a chain
template <class R, int N, int S>
__global__ void __launch_bounds__(256) plaquette_batch(const BatchParams bp, double* partials) {
  __shared__ ObsParams sp;
  __shared__ uint32_t first;
  batch_obs_chain(bp, sp, first);
  const int64_t idx = int64_t(blockIdx.x - first) * blockDim.x + threadIdx.x;
  const int par = idx >= sp.g.Vh ? 1 : 0;
  double v[1] = {idx < sp.g.V ? site_plaquette<R, N, S>(sp, par, idx - par * sp.g.Vh) : 0.0};
  block_sum<1>(v);
  if (threadIdx.x == 0) partials[blockIdx.x] = v[0];
}

// per-block partial Polyakov sums, one block per 128 spatial sites of a chain
template <class R, int N, int S>
__global__ void __launch_bounds__(128) polyakov_batch(const BatchParams bp, double* partials) {
  __shared__ ObsParams sp;
  __shared__ uint32_t first;
  batch_obs_chain(bp, sp, first);
  const int64_t xs = int64_t(blockIdx.x - first) * blockDim.x + threadIdx.x;
  double v[2] = {0.0, 0.0};
  if (xs < int64_t(sp.g.nx) * sp.g.ny * sp.g.nz) site_polyakov<R, N, S>(sp, xs, v[0], v[1]);
  block_sum<2>(v);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = v[0];
    partials[2 * blockIdx.x + 1] = v[1];
  }
}

// One warp per chain adds the chain's block partials in a fixed order and
// writes out[(slot % cap) * stride + offset + c] (K values per chain).
template <int K>
__global__ void __launch_bounds__(32) batch_finish(const BatchParams bp, const double* partials, int which,
                                                   double* out, const uint32_t* slot, int cap, int offset,
                                                   int stride) {
  const int c = blockIdx.x;
  const int lane = threadIdx.x;
  const uint32_t b0 = bp.start[c], b1 = bp.start[c + 1];
  const ChainDesc& d = bp.chains[c];
  const double scale = which == 0 ? d.plaq_scale : d.poly_scale;
  const int row = slot ? int(*slot % uint32_t(cap)) : 0;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double s = 0.0;
    for (uint32_t b = b0 + lane; b < b1; b += 32) s += partials[b * K + k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) out[(int64_t(row) * stride + offset + c) * K + k] = s * scale;
  }
}


// ---------------------------------------------------------------------------
// Canonical FP64 <-> storage conversion of links [first, first + count),
// canonical link index l = mu * V + lex.  A block converts LPB consecutive links
// through shared memory, so the canonical side (which may be host memory mapped
// into the device address space) is read and written as contiguous 16-byte
// vectors.
// ---------------------------------------------------------------------------
template <int N>
__host__ __device__ constexpr int conv_links_per_block() {
  return N <= 4 ? 128 : (N == 5 ? 64 : 32);
}

__device__ __forceinline__ int link_parity(const Geom& g, int64_t lex) {
  const int x = int(lex % g.nx), y = int((lex / g.nx) % g.ny);
  const int z = int((lex / (int64_t(g.nx) * g.ny)) % g.nz), t = int(lex / (int64_t(g.nx) * g.ny * g.nz));
  return (x + y + z + t) & 1;
}

template <class R, int N, int S>
__global__ void __launch_bounds__(128) export_kernel(const ObsParams p, double* dst, int64_t first, int64_t count) {
  constexpr int D = 2 * N * N;
  constexpr int LPB = conv_links_per_block<N>();
  __shared__ __align__(16) double sm[LPB * D];
  const int64_t rel0 = int64_t(blockIdx.x) * LPB;
  const int nl = int((count - rel0) < LPB ? (count - rel0) : LPB);
  for (int i = threadIdx.x; i < nl; i += blockDim.x) {
    const int64_t l = first + rel0 + i;
    const int mu = int(l / p.g.V);
    const int64_t lex = l - int64_t(mu) * p.g.V;
    const Mat<R, N> m = load_mat<R, N, S>(obs_block(p, mu, link_parity(p.g, lex)), p.g.Vh, lex >> 1);
    double* o = sm + i * D;
    if constexpr (S == kTwoRow) {
      Mat<double, 3> d = mat_cast<R, double, 3>(m);  // third row rebuilt in FP64
      su3_third_row(d);
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          o[2 * (3 * a + b)] = d.e[a][b].re;
          o[2 * (3 * a + b) + 1] = d.e[a][b].im;
        }
    } else {
#pragma unroll
      for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = 0; b < N; ++b) {
          o[2 * (N * a + b)] = double(m.e[a][b].re);
          o[2 * (N * a + b) + 1] = double(m.e[a][b].im);
        }
    }
  }
  __syncthreads();
  double2* out = reinterpret_cast<double2*>(dst + rel0 * D);
  const double2* in = reinterpret_cast<const double2*>(sm);
  for (int j = threadIdx.x; j < nl * D / 2; j += blockDim.x) out[j] = in[j];
}

template <class R, int N, int S>
__global__ void __launch_bounds__(128) import_kernel(const ObsParams p, const double* src, int64_t first, int64_t count) {
  constexpr int D = 2 * N * N;
  constexpr int LPB = conv_links_per_block<N>();
  __shared__ __align__(16) double sm[LPB * D];
  const int64_t rel0 = int64_t(blockIdx.x) * LPB;
  const int nl = int((count - rel0) < LPB ? (count - rel0) : LPB);
  const double2* in = reinterpret_cast<const double2*>(src + rel0 * D);
  double2* st = reinterpret_cast<double2*>(sm);
  for (int j = threadIdx.x; j < nl * D / 2; j += blockDim.x) st[j] = in[j];
  __syncthreads();
  for (int i = threadIdx.x; i < nl; i += blockDim.x) {
    const int64_t l = first + rel0 + i;
    const int mu = int(l / p.g.V);
    const int64_t lex = l - int64_t(mu) * p.g.V;
    const double* s = sm + i * D;
    Mat<R, N> m;
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
      for (int b = 0; b < N; ++b) m.e[a][b] = {R(s[2 * (N * a + b)]), R(s[2 * (N * a + b) + 1])};
    store_mat<R, N, S>(const_cast<char*>(obs_block(p, mu, link_parity(p.g, lex))), p.g.Vh, lex >> 1, m);
  }
}

// The compact host format: the stored rows (rows 0 .. NR / (2 Nc) - 1) of every
// link as (re, im) pairs in canonical link order, in the storage precision.  For
// quaternion storage that is row 0 = (a0 + i a3, a2 + i a1).  Staged through
// shared memory so that host memory is read and written in 8-byte words.
template <class R, int N, int S>
__device__ __forceinline__ void stored_to_rows(const R (&r)[Layout<R, N, S>::nreals], R* o) {
  constexpr int NR = Layout<R, N, S>::nreals;
  if constexpr (S == kQuat) {
    o[0] = r[0];
    o[1] = r[3];
    o[2] = r[2];
    o[3] = r[1];
  } else {
#pragma unroll
    for (int k = 0; k < NR; ++k) o[k] = r[k];
  }
}

template <class R, int N, int S>
__device__ __forceinline__ void rows_to_stored(const R* o, R (&r)[Layout<R, N, S>::nreals]) {
  constexpr int NR = Layout<R, N, S>::nreals;
  if constexpr (S == kQuat) {
    r[0] = o[0];
    r[3] = o[1];
    r[2] = o[2];
    r[1] = o[3];
  } else {
#pragma unroll
    for (int k = 0; k < NR; ++k) r[k] = o[k];
  }
}

// links per block of the compact conversion kernels: up to 512, within 48 KB of
// shared memory (a multiple of 16 links: block offsets stay 16-byte aligned)
template <class R, int N, int S>
__host__ __device__ constexpr int compact_links_per_block() {
  return (48 * 1024 / Layout<R, N, S>::bytes) >= 512 ? 512 : ((48 * 1024 / Layout<R, N, S>::bytes) / 16) * 16;
}

// n bytes (a multiple of 8) between 16-byte aligned addresses: 16-byte words,
// then one 8-byte word if left
__device__ __forceinline__ void copy_words(void* dst, const void* src, int n) {
  uint4* d = static_cast<uint4*>(dst);
  const uint4* s = static_cast<const uint4*>(src);
  const int w16 = n / 16;
  for (int j = threadIdx.x; j < w16; j += blockDim.x) d[j] = s[j];
  if ((n & 15) && threadIdx.x == 0)
    reinterpret_cast<unsigned long long*>(d + w16)[0] = reinterpret_cast<const unsigned long long*>(s + w16)[0];
}

template <class R, int N, int S>
__global__ void __launch_bounds__(256) export_stored_kernel(const ObsParams p, R* dst, int64_t first, int64_t count) {
  constexpr int NR = Layout<R, N, S>::nreals;
  constexpr int LPB = compact_links_per_block<R, N, S>();
  __shared__ __align__(16) R sm[LPB * NR];
  const int64_t rel0 = int64_t(blockIdx.x) * LPB;
  const int nl = int((count - rel0) < LPB ? (count - rel0) : LPB);
  for (int i = threadIdx.x; i < nl; i += blockDim.x) {
    const int64_t l = first + rel0 + i;
    const int mu = int(l / p.g.V);
    const int64_t lex = l - int64_t(mu) * p.g.V;
    R r[NR];
    load_reals<R, NR, kLoadNc>(obs_block(p, mu, link_parity(p.g, lex)), p.g.Vh, lex >> 1, r);
    stored_to_rows<R, N, S>(r, sm + i * NR);
  }
  __syncthreads();
  copy_words(dst + rel0 * NR, sm, nl * NR * int(sizeof(R)));
}

template <class R, int N, int S>
__global__ void __launch_bounds__(256) import_stored_kernel(const ObsParams p, const R* src, int64_t first,
                                                            int64_t count) {
  constexpr int NR = Layout<R, N, S>::nreals;
  constexpr int LPB = compact_links_per_block<R, N, S>();
  __shared__ __align__(16) R sm[LPB * NR];
  const int64_t rel0 = int64_t(blockIdx.x) * LPB;
  const int nl = int((count - rel0) < LPB ? (count - rel0) : LPB);
  copy_words(sm, src + rel0 * NR, nl * NR * int(sizeof(R)));
  __syncthreads();
  for (int i = threadIdx.x; i < nl; i += blockDim.x) {
    const int64_t l = first + rel0 + i;
    const int mu = int(l / p.g.V);
    const int64_t lex = l - int64_t(mu) * p.g.V;
    R r[NR];
    rows_to_stored<R, N, S>(sm + i * NR, r);
    store_reals<R, NR>(const_cast<char*>(obs_block(p, mu, link_parity(p.g, lex))), p.g.Vh, lex >> 1, r);
  }
}

// ---------------------------------------------------------------------------
// Host launchers and the operation table
// ---------------------------------------------------------------------------
inline PassParams make_pass_params(const Ctx& c, int mu, int parity, uint32_t step_offset, uint32_t reunit_mod,
                                   uint32_t reunit_rem) {
  PassParams p;
  p.links = c.links;
  p.block_bytes = c.block_bytes;
  p.g = c.g;
  p.mu = mu;
  p.parity = parity;
  p.alpha_coef = 2.0 * c.beta / c.nc;
  p.key = make_uint2(uint32_t(c.seed & 0xffffffffu), uint32_t(c.seed >> 32));
  p.hb_step = &c.state->hb_step;
  p.step_offset = step_offset;
  p.reunit_mod = reunit_mod;
  p.reunit_rem = reunit_rem;
  p.h_begin = c.h_begin;
  p.h_end = c.h_end;
  p.lex_offset = c.lex_offset;
  p.v_global = c.v_global;
  return p;
}

template <class R, int N, int S>
cudaError_t launch_pass(const Ctx& c, int mode, int mu, int parity, uint32_t step_offset, uint32_t reunit_mod,
                        uint32_t reunit_rem) {
  const PassParams p = make_pass_params(c, mu, parity, step_offset, reunit_mod, reunit_rem);
  const int bt = c.block_threads;
  const int64_t n_links = c.h_end - c.h_begin;
  const unsigned grid = unsigned((n_links + bt - 1) / bt);
  const bool ru = reunit_mod != 0u;
  if constexpr (has_group<R, N>()) {
    if (!ru && use_group<R, N>(c.variant)) {
      const unsigned gg = unsigned((n_links + Group<R, N>::LPB - 1) / Group<R, N>::LPB);
      if (mode == kHeatbathMode)
        update_pass_group<R, N, kHeatbathMode><<<gg, 128, 0, c.stream>>>(p);
      else
        update_pass_group<R, N, kOverrelaxMode><<<gg, 128, 0, c.stream>>>(p);
      return cudaGetLastError();
    }
  }
  if constexpr (!has_fused_reunit<R, N>()) {
    if (ru) return cudaErrorNotSupported;
    if (mode == kHeatbathMode)
      update_pass_mat<R, N, S, kHeatbathMode, 0, false><<<grid, bt, 0, c.stream>>>(p);
    else
      update_pass_mat<R, N, S, kOverrelaxMode, 0, false><<<grid, bt, 0, c.stream>>>(p);
  } else if constexpr (S == kQuat) {
#define SUN_LAUNCH_QUAT(RU)                                                             \
  if (mode == kHeatbathMode)                                                            \
    update_pass_quat<R, kHeatbathMode, RU><<<grid, bt, 0, c.stream>>>(p);               \
  else                                                                                  \
    update_pass_quat<R, kOverrelaxMode, RU><<<grid, bt, 0, c.stream>>>(p);
    if (ru) {
      SUN_LAUNCH_QUAT(true)
    } else {
      SUN_LAUNCH_QUAT(false)
    }
#undef SUN_LAUNCH_QUAT
  } else if constexpr (has_variants<R, N, S>()) {
    if ((c.variant & 16) && mode == kOverrelaxMode) {
      // two links per thread in packed FP32
      const unsigned g2 = unsigned((n_links + 255) / 256);
      if (ru)
        update_or_pass2<N, S, true><<<g2, 128, 0, c.stream>>>(p);
      else
        update_or_pass2<N, S, false><<<g2, 128, 0, c.stream>>>(p);
      return cudaGetLastError();
    }
    const int v = c.variant & 3;
    const unsigned bt1 = (v & 1) ? 128u : unsigned(bt);
    const unsigned g1 = unsigned((n_links + bt1 - 1) / bt1);
#define SUN_LAUNCH_VAR(K, V)                                                            \
  if (mode == kHeatbathMode) {                                                          \
    if (ru)                                                                             \
      K<R, N, S, kHeatbathMode, V, true><<<g1, bt1, 0, c.stream>>>(p);                  \
    else                                                                                \
      K<R, N, S, kHeatbathMode, V, false><<<g1, bt1, 0, c.stream>>>(p);                 \
  } else {                                                                              \
    if (ru)                                                                             \
      K<R, N, S, kOverrelaxMode, V, true><<<g1, bt1, 0, c.stream>>>(p);                 \
    else                                                                                \
      K<R, N, S, kOverrelaxMode, V, false><<<g1, bt1, 0, c.stream>>>(p);                \
  }
    switch (v) {
      case 1: SUN_LAUNCH_VAR(update_pass_mat_occ, 1) break;
      case 2: SUN_LAUNCH_VAR(update_pass_mat, 2) break;
      case 3: SUN_LAUNCH_VAR(update_pass_mat_occ, 3) break;
      default: SUN_LAUNCH_VAR(update_pass_mat, 0) break;
    }
#undef SUN_LAUNCH_VAR
  } else {
    if constexpr (has_occ_bound<R, N>()) {
      if (c.variant & 1) {
        const unsigned g1 = unsigned((n_links + 127) / 128);
        if (mode == kHeatbathMode) {
          if (ru)
            update_pass_mat_occ<R, N, S, kHeatbathMode, 1, true><<<g1, 128, 0, c.stream>>>(p);
          else
            update_pass_mat_occ<R, N, S, kHeatbathMode, 1, false><<<g1, 128, 0, c.stream>>>(p);
        } else {
          if (ru)
            update_pass_mat_occ<R, N, S, kOverrelaxMode, 1, true><<<g1, 128, 0, c.stream>>>(p);
          else
            update_pass_mat_occ<R, N, S, kOverrelaxMode, 1, false><<<g1, 128, 0, c.stream>>>(p);
        }
        return cudaGetLastError();
      }
    }
    if (mode == kHeatbathMode) {
      if (ru)
        update_pass_mat<R, N, S, kHeatbathMode, 0, true><<<grid, bt, 0, c.stream>>>(p);
      else
        update_pass_mat<R, N, S, kHeatbathMode, 0, false><<<grid, bt, 0, c.stream>>>(p);
    } else {
      if (ru)
        update_pass_mat<R, N, S, kOverrelaxMode, 0, true><<<grid, bt, 0, c.stream>>>(p);
      else
        update_pass_mat<R, N, S, kOverrelaxMode, 0, false><<<grid, bt, 0, c.stream>>>(p);
    }
  }
  return cudaGetLastError();
}

// A wavefront launch: the ticket and the slice counters are cleared first, then
// one block per unit; blocks take their unit from the ticket counter in the
// order they start.
template <class K>
cudaError_t launch_wave(K kernel, int bt, const Ctx& c, const PassParams& p, const WaveParams& w) {
  const cudaError_t e = cudaMemsetAsync(w.sync + 1, 0, (kWaveSyncWords - 1 + size_t(w.nt)) * sizeof(uint32_t), c.stream);
  if (e != cudaSuccess) return e;
  const unsigned grid = 2u * w.nt * w.chunks - w.skip;
  kernel<<<grid, bt, 0, c.stream>>>(p, w);
  return cudaGetLastError();
}

template <class R, int N, int S, int VAR>
cudaError_t launch_pair_mat(const Ctx& c, int mode, bool ru, int bt, const PassParams& p, const WaveParams& w) {
  const bool hb = mode == kHeatbathMode;
  if constexpr (!has_fused_reunit<R, N>()) {
    if (ru) return cudaErrorNotSupported;
    return hb ? launch_wave(update_pair_mat<R, N, S, kHeatbathMode, VAR, false>, bt, c, p, w)
              : launch_wave(update_pair_mat<R, N, S, kOverrelaxMode, VAR, false>, bt, c, p, w);
  } else if constexpr ((VAR & 1) != 0) {
    if (hb)
      return ru ? launch_wave(update_pair_mat_occ<R, N, S, kHeatbathMode, VAR, true>, bt, c, p, w)
                : launch_wave(update_pair_mat_occ<R, N, S, kHeatbathMode, VAR, false>, bt, c, p, w);
    return ru ? launch_wave(update_pair_mat_occ<R, N, S, kOverrelaxMode, VAR, true>, bt, c, p, w)
              : launch_wave(update_pair_mat_occ<R, N, S, kOverrelaxMode, VAR, false>, bt, c, p, w);
  } else {
    if (hb)
      return ru ? launch_wave(update_pair_mat<R, N, S, kHeatbathMode, VAR, true>, bt, c, p, w)
                : launch_wave(update_pair_mat<R, N, S, kHeatbathMode, VAR, false>, bt, c, p, w);
    return ru ? launch_wave(update_pair_mat<R, N, S, kOverrelaxMode, VAR, true>, bt, c, p, w)
              : launch_wave(update_pair_mat<R, N, S, kOverrelaxMode, VAR, false>, bt, c, p, w);
  }
}

// The even and the odd pass of direction mu.  Kernels without a wavefront form
// (the row-parallel kernel, the two-row staple and packed variants) run as the two passes.
template <class R, int N, int S>
cudaError_t launch_pair(const Ctx& c, int mode, int mu, uint32_t step_offset, uint32_t reunit_mod,
                        uint32_t reunit_rem) {
  const bool ru = reunit_mod != 0u;
  bool two = !c.wave || c.h_begin != 0 || c.h_end != c.g.Vh;  // a slab: its own pass ranges
  if constexpr (has_group<R, N>()) two = two || (!ru && use_group<R, N>(c.variant));
  if constexpr (has_variants<R, N, S>()) two = two || (c.variant & 18) != 0;
  if (two) {
    const cudaError_t e = launch_pass<R, N, S>(c, mode, mu, 0, step_offset, reunit_mod, reunit_rem);
    if (e != cudaSuccess) return e;
    return launch_pass<R, N, S>(c, mode, mu, 1, step_offset, reunit_mod, reunit_rem);
  }
  const PassParams p = make_pass_params(c, mu, 0, step_offset, reunit_mod, reunit_rem);
  bool occ = false;
  if constexpr (has_variants<R, N, S>()) occ = (c.variant & 1) != 0;
  const int bt = occ ? 128 : c.block_threads;
  WaveParams w;
  w.sync = c.wave;
  w.half_slice = uint32_t(int64_t(c.g.nx) * c.g.ny * c.g.nz / 2);
  w.nt = uint32_t(c.g.nt);
  w.chunks = (w.half_slice + uint32_t(bt) - 1) / uint32_t(bt);
  w.lag = uint32_t(c.wave_lag < 1 ? 1 : (c.wave_lag > c.g.nt - 1 ? c.g.nt - 1 : c.wave_lag));
  w.skip = c.wave_skip < 2u * w.nt * w.chunks ? c.wave_skip : 0u;
  if constexpr (S == kQuat) {
    if (mode == kHeatbathMode)
      return ru ? launch_wave(update_pair_quat<R, kHeatbathMode, true>, bt, c, p, w)
                : launch_wave(update_pair_quat<R, kHeatbathMode, false>, bt, c, p, w);
    return ru ? launch_wave(update_pair_quat<R, kOverrelaxMode, true>, bt, c, p, w)
              : launch_wave(update_pair_quat<R, kOverrelaxMode, false>, bt, c, p, w);
  } else if constexpr (has_variants<R, N, S>()) {
    if (occ) return launch_pair_mat<R, N, S, 1>(c, mode, ru, bt, p, w);
    return launch_pair_mat<R, N, S, 0>(c, mode, ru, bt, p, w);
  } else {
    return launch_pair_mat<R, N, S, 0>(c, mode, ru, bt, p, w);
  }
}

inline LinkParams make_link_params(const Ctx& c, int hot) {
  LinkParams p;
  p.links = c.links;
  p.block_bytes = c.block_bytes;
  p.g = c.g;
  p.key = make_uint2(uint32_t(c.seed & 0xffffffffu), uint32_t(c.seed >> 32));
  p.hot = hot;
  p.lex_offset = c.lex_offset;
  p.v_global = c.v_global;
  return p;
}

template <class R, int N, int S>
cudaError_t launch_init(const Ctx& c, int hot) {
  const int64_t n = 8 * c.g.Vh;
  init_kernel<R, N, S><<<unsigned((n + 127) / 128), 128, 0, c.stream>>>(make_link_params(c, hot));
  return cudaGetLastError();
}

template <class R, int N, int S>
cudaError_t launch_reunit(const Ctx& c) {
  const int64_t n = 8 * c.g.Vh;
  reunit_kernel<R, N, S><<<unsigned((n + 127) / 128), 128, 0, c.stream>>>(make_link_params(c, 0));
  return cudaGetLastError();
}

inline ObsParams make_obs_params(const Ctx& c) {
  ObsParams p;
  p.links = c.links;
  p.block_bytes = c.block_bytes;
  p.g = c.g;
  p.h_begin = c.h_begin;
  p.h_end = c.h_end;
  return p;
}

inline unsigned reduce_grid(const Ctx& c, int64_t items, int bt) {
  int64_t want = (items + bt - 1) / bt;
  int64_t cap = int64_t(c.reduce_blocks);
  return unsigned(want < cap ? (want < 1 ? 1 : want) : cap);
}

template <class R, int N, int S>
cudaError_t launch_plaquette(const Ctx& c, double* out, const uint32_t* slot, int cap) {
  ReduceParams rp;
  rp.partials = c.partials;
  rp.counter = &c.state->plaq_counter;
  rp.out = out;
  rp.slot = slot;
  rp.cap = cap;
  rp.stride = c.obs_stride;
  rp.offset = c.obs_offset;
  rp.scale = 1.0 / (6.0 * double(c.v_global) * N);
  const int bt = 256;
  if (c.h_begin == 0 && c.h_end == c.g.Vh)
    plaquette_kernel<R, N, S><<<reduce_grid(c, c.g.V, bt), bt, 0, c.stream>>>(make_obs_params(c), rp);
  else
    plaquette_slab_kernel<R, N, S><<<reduce_grid(c, 2 * (c.h_end - c.h_begin), bt), bt, 0, c.stream>>>(
        make_obs_params(c), rp);
  return cudaGetLastError();
}

template <class R, int N, int S>
cudaError_t launch_polyakov(const Ctx& c, double* out, const uint32_t* slot, int cap) {
  ReduceParams rp;
  rp.partials = c.partials + 2 * kMaxReduceBlocks;
  rp.counter = &c.state->poly_counter;
  rp.out = out;
  rp.slot = slot;
  rp.cap = cap;
  rp.stride = c.obs_stride;
  rp.offset = c.obs_offset;
  const int64_t nsp = int64_t(c.g.nx) * c.g.ny * c.g.nz;
  rp.scale = 1.0 / (double(N) * double(nsp));
  const int bt = 128;
  polyakov_kernel<R, N, S><<<reduce_grid(c, nsp, bt), bt, 0, c.stream>>>(make_obs_params(c), rp);
  return cudaGetLastError();
}

// a slab's partial Polyakov products over its interior slices [h_begin, h_end) / (Vs / 2)
template <class R, int N, int S>
cudaError_t launch_polyakov_partial(const Ctx& c, void* out) {
  const int64_t nsp = int64_t(c.g.nx) * c.g.ny * c.g.nz;
  const int64_t half_slice = nsp / 2;
  polyakov_partial_kernel<R, N, S><<<unsigned((nsp + 127) / 128), 128, 0, c.stream>>>(
      make_obs_params(c), int(c.h_begin / half_slice), int(c.h_end / half_slice), out);
  return cudaGetLastError();
}

// the slabs' partial products (device array of n pointers) -> Polyakov loop
template <class R, int N, int S>
cudaError_t launch_polyakov_combine(const Ctx& c, const void* const* parts, int n, double* out, const uint32_t* slot,
                                    int cap) {
  ReduceParams rp;
  rp.partials = c.partials + 2 * kMaxReduceBlocks;
  rp.counter = &c.state->poly_counter;
  rp.out = out;
  rp.slot = slot;
  rp.cap = cap;
  rp.stride = c.obs_stride;
  rp.offset = c.obs_offset;
  const int64_t nsp = int64_t(c.g.nx) * c.g.ny * c.g.nz;
  rp.scale = 1.0 / (double(N) * double(nsp));
  polyakov_combine_kernel<R, N, S><<<reduce_grid(c, nsp, 128), 128, 0, c.stream>>>(parts, n, nsp, rp);
  return cudaGetLastError();
}

template <class R, int N, int S>
cudaError_t launch_check_links(const Ctx& c, unsigned long long* out) {
  cudaError_t e = cudaMemsetAsync(out, 0, 3 * sizeof(unsigned long long), c.stream);
  if (e != cudaSuccess) return e;
  check_links_kernel<R, N, S><<<reduce_grid(c, 8 * c.g.Vh, 256), 256, 0, c.stream>>>(make_obs_params(c), out);
  return cudaGetLastError();
}

template <class R, int N, int S>
cudaError_t launch_export(const Ctx& c, double* dst, int64_t first, int64_t count) {
  if (count <= 0) return cudaSuccess;
  constexpr int LPB = conv_links_per_block<N>();
  export_kernel<R, N, S><<<unsigned((count + LPB - 1) / LPB), 128, 0, c.stream>>>(make_obs_params(c), dst, first, count);
  return cudaGetLastError();
}

template <class R, int N, int S>
cudaError_t launch_export_stored(const Ctx& c, void* dst, int64_t first, int64_t count) {
  if (count <= 0) return cudaSuccess;
  constexpr int LPB = compact_links_per_block<R, N, S>();
  export_stored_kernel<R, N, S><<<unsigned((count + LPB - 1) / LPB), 256, 0, c.stream>>>(
      make_obs_params(c), static_cast<R*>(dst), first, count);
  return cudaGetLastError();
}

template <class R, int N, int S>
cudaError_t launch_import_stored(const Ctx& c, const void* src, int64_t first, int64_t count) {
  if (count <= 0) return cudaSuccess;
  constexpr int LPB = compact_links_per_block<R, N, S>();
  import_stored_kernel<R, N, S><<<unsigned((count + LPB - 1) / LPB), 256, 0, c.stream>>>(
      make_obs_params(c), static_cast<const R*>(src), first, count);
  return cudaGetLastError();
}

template <class R, int N, int S>
cudaError_t launch_import(const Ctx& c, const double* src, int64_t first, int64_t count) {
  if (count <= 0) return cudaSuccess;
  constexpr int LPB = conv_links_per_block<N>();
  import_kernel<R, N, S><<<unsigned((count + LPB - 1) / LPB), 128, 0, c.stream>>>(make_obs_params(c), src, first, count);
  return cudaGetLastError();
}

template <class R, int N, int S>
cudaError_t launch_batch_pass(const BatchCtx& b, int mode, int mu, int parity, uint32_t so, uint32_t rmod,
                              uint32_t rrem) {
  if (b.n == 0) return cudaSuccess;
  const BatchParams bp{b.chains, b.pass_start, b.n};
  const bool ru = rmod != 0u;
  if constexpr (has_group<R, N>()) {
    if (!ru && use_group<R, N>(b.variant)) {
      // the pass table of a group batch counts blocks of Group::LPB links
      const BatchParams gp{b.chains, b.group_start, b.n};
      if (mode == kHeatbathMode)
        update_pass_batch_group<R, N, kHeatbathMode><<<b.group_blocks, 128, 0, b.stream>>>(gp, mu, parity, so);
      else
        update_pass_batch_group<R, N, kOverrelaxMode><<<b.group_blocks, 128, 0, b.stream>>>(gp, mu, parity, so);
      return cudaGetLastError();
    }
  }
  const unsigned g1 = b.pass_blocks, bt = unsigned(b.pass_threads);
#define SUN_LAUNCH_BATCH(K, V)                                                              \
  if (mode == kHeatbathMode) {                                                              \
    if (ru)                                                                                 \
      K<R, N, S, kHeatbathMode, V, true><<<g1, bt, 0, b.stream>>>(bp, mu, parity, so, rmod, rrem);   \
    else                                                                                    \
      K<R, N, S, kHeatbathMode, V, false><<<g1, bt, 0, b.stream>>>(bp, mu, parity, so, rmod, rrem);  \
  } else {                                                                                  \
    if (ru)                                                                                 \
      K<R, N, S, kOverrelaxMode, V, true><<<g1, bt, 0, b.stream>>>(bp, mu, parity, so, rmod, rrem);  \
    else                                                                                    \
      K<R, N, S, kOverrelaxMode, V, false><<<g1, bt, 0, b.stream>>>(bp, mu, parity, so, rmod, rrem); \
  }
  if constexpr (has_variants<R, N, S>()) {
    if (b.variant & 1) {
      SUN_LAUNCH_BATCH(update_pass_batch_occ, 1)
    } else {
      SUN_LAUNCH_BATCH(update_pass_batch, 0)
    }
  } else {
    SUN_LAUNCH_BATCH(update_pass_batch, 0)
  }
#undef SUN_LAUNCH_BATCH
  return cudaGetLastError();
}

template <class R, int N, int S>
cudaError_t launch_batch_reunit(const BatchCtx& b) {
  if (b.n == 0) return cudaSuccess;
  reunit_batch<R, N, S><<<b.reunit_blocks, 128, 0, b.stream>>>(BatchParams{b.chains, b.reunit_start, b.n});
  return cudaGetLastError();
}

template <class R, int N, int S>
cudaError_t launch_batch_plaquette(const BatchCtx& b, double* out, const uint32_t* slot, int cap, int offset,
                                   int stride) {
  if (b.n == 0) return cudaSuccess;
  const BatchParams bp{b.chains, b.plaq_start, b.n};
  plaquette_batch<R, N, S><<<b.plaq_blocks, 256, 0, b.stream>>>(bp, b.partials);
  batch_finish<1><<<unsigned(b.n), 32, 0, b.stream>>>(bp, b.partials, 0, out, slot, cap, offset, stride);
  return cudaGetLastError();
}

template <class R, int N, int S>
cudaError_t launch_batch_polyakov(const BatchCtx& b, double* out, const uint32_t* slot, int cap, int offset,
                                  int stride) {
  if (b.n == 0) return cudaSuccess;
  const BatchParams bp{b.chains, b.poly_start, b.n};
  polyakov_batch<R, N, S><<<b.poly_blocks, 128, 0, b.stream>>>(bp, b.partials);
  batch_finish<2><<<unsigned(b.n), 32, 0, b.stream>>>(bp, b.partials, 1, out, slot, cap, offset, stride);
  return cudaGetLastError();
}

// Batched kernels are built for FP32 and for Nc <= 3 (serving runs FP32; FP64
// batches of large Nc cost build time without a use).
template <class R, int N, int S>
constexpr bool has_batch() {
  return std::is_same<R, float>::value || N <= 3;
}

template <class R, int N, int S>
const Ops* ops_instance() {
  static const Ops ops = {
      N,
      Layout<R, N, S>::nreals,
      int(sizeof(R)) * 8,
      Layout<R, N, S>::bytes,
      has_fused_reunit<R, N>() ? 1 : 0,
      has_group<R, N>() && S == kFull ? Group<R, N>::LPB : 0,
      &launch_pass<R, N, S>,
      &launch_pair<R, N, S>,
      &launch_init<R, N, S>,
      &launch_reunit<R, N, S>,
      &launch_plaquette<R, N, S>,
      &launch_polyakov<R, N, S>,
      &launch_polyakov_partial<R, N, S>,
      &launch_polyakov_combine<R, N, S>,
      sizeof(PolyPart<R, N, S>),
      &launch_check_links<R, N, S>,
      &launch_export<R, N, S>,
      &launch_import<R, N, S>,
      &launch_export_stored<R, N, S>,
      &launch_import_stored<R, N, S>,
      has_batch<R, N, S>() ? &launch_batch_pass<R, N, S> : nullptr,
      has_batch<R, N, S>() ? &launch_batch_reunit<R, N, S> : nullptr,
      has_batch<R, N, S>() ? &launch_batch_plaquette<R, N, S> : nullptr,
      has_batch<R, N, S>() ? &launch_batch_polyakov<R, N, S> : nullptr,
  };
  return &ops;
}

}  // namespace sun
