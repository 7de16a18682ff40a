/*
 * sun_oracle.c -- plain FP64 CPU oracle of the SU(Nc) checkerboard link sweep
 * (Cardoso & Bicudo, arXiv:1112.4533, Secs. 2-3).
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, the smoke check and the benchmark's
 * CPU-baseline leg; never by the product path.  Written for a reader checking it
 * against the paper: dense complex matrices, SU(2) elements as literal 2x2
 * matrices a0*1 + i a.sigma (Eq. 6), no fusion, no blocking.  Where the paper
 * is silent the reading taken is stated next to the code:
 *
 *   R1  weight of one link: exp((beta/Nc) ReTr(U Sigma^+)), Sigma = Eq. 9 with mu
 *       the link's own direction and the sum over the three nu != mu.
 *   R2  heatbath of one SU(2) subgroup: alpha = (2 beta / Nc) k (Eqs. 10-13 give
 *       beta*k for Nc=2); b0 drawn with Kennedy-Pendleton for alpha >= 1.5 and
 *       Creutz below; at most 64 attempts, after which the subgroup is left as
 *       it is; the new subgroup element is A = b vhat^+ (Eq. 14 with the drawn
 *       element on the left).
 *   R3  overrelaxation of one SU(2) subgroup: A = (vhat^+)^2 (Eq. 17 in the
 *       orientation of R1).
 *   R4  subgroups in lexicographic order (0,1),(0,2),..,(Nc-2,Nc-1) (Eq. 15).
 *   R5  checkerboard: for mu = 0..3, even sites then odd sites (Sec. 3).
 *   R6  random numbers: Philox4x32-10, key = seed, counter = (mu*V + lex,
 *       heatbath step, (subgroup << 16) | attempt, 1); the direction on S^2
 *       uses attempt slot 64; hot start uses counter (mu*V + lex, 0, call, 2).
 *       Uniforms are (floor(u/2^9) + 1/2) 2^-23, exact in float and double.
 *   R7  a subgroup whose projected strength k is <= 1e-15 or not finite is
 *       skipped.
 *   R8  reunitarization (Sec. 2, last paragraph): Nc=2 normalise row 0 and
 *       rebuild row 1; Nc=3 Gram-Schmidt rows 0,1 and row 2 = conj(row0 x row1);
 *       Nc>3 Gram-Schmidt all rows then multiply the last row by conj(det).
 *   R9  hot start: Gram-Schmidt (R8) of a matrix of independent complex
 *       Gaussians (Box-Muller), i.e. a Haar-random SU(Nc) matrix.
 *   R10 plaquette normalised as sum_x sum_{mu<nu} ReTr P / (6 V Nc); Polyakov
 *       loop sum_xvec Tr prod_{t=0}^{Nt-1} U_3(xvec,t) / (Nc Nx Ny Nz).
 *   R11 re-unitarization placement: after the heatbath and overrelaxation steps
 *       of a sweep (Secs. 2-3); or each link right after its update in the
 *       sweep's last step; or spread over the steps, links grouped in runs of 32
 *       consecutive even/odd site indices (lex >> 1) and run r re-unitarized
 *       right after its update in step r mod (number of steps).  In every
 *       schedule each link is re-unitarized once per sweep.
 *
 * Floating point: compile with -ffp-contract=off and without -ffast-math.
 */
#include "sun_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define HB_MAX_ATTEMPTS 64
#define ALPHA_SWITCH 1.5
#define K_MIN 1e-15
#define TAG_HEATBATH 1u
#define TAG_INIT 2u

int orc_version(void) { return 1; }

int orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

int orc_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10: ten rounds of the Philox S-box; the key is bumped by the   */
/* Weyl constants between rounds (Salmon et al., SC'11, Sec. 5).             */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += W0;
      k1 += W1;
    }
    uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

double orc_uniform(uint32_t u) { return ((double)(u >> 9) + 0.5) * 0x1p-23; }

static void draw4(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, double r[4]) {
  uint32_t ctr[4] = {c0, c1, c2, c3};
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  uint32_t out[4];
  orc_philox4x32_10(ctr, key, out);
  for (int i = 0; i < 4; ++i) r[i] = orc_uniform(out[i]);
}

/* ------------------------------------------------------------------------ */
/* Lattice geometry (Sec. 2): 4D hypercubic, periodic.                       */
/* ------------------------------------------------------------------------ */
static int64_t volume(const int d[4]) { return (int64_t)d[0] * d[1] * d[2] * d[3]; }

static void coords(const int d[4], int64_t lex, int x[4]) {
  for (int m = 0; m < 4; ++m) {
    x[m] = (int)(lex % d[m]);
    lex /= d[m];
  }
}

static int64_t lex_of(const int d[4], const int x[4]) {
  return x[0] + (int64_t)d[0] * (x[1] + (int64_t)d[1] * (x[2] + (int64_t)d[2] * x[3]));
}

/* site reached from lex by one step of sign (+1/-1) in direction dir */
static int64_t hop(const int d[4], int64_t lex, int dir, int sign) {
  int x[4];
  coords(d, lex, x);
  x[dir] = (x[dir] + sign + d[dir]) % d[dir];
  return lex_of(d, x);
}

static int parity_of(const int d[4], int64_t lex) {
  int x[4];
  coords(d, lex, x);
  return (x[0] + x[1] + x[2] + x[3]) & 1;
}

static const cplx* link_c(const double* U, int nc, int64_t V, int mu, int64_t lex) {
  return (const cplx*)U + ((int64_t)mu * V + lex) * nc * nc;
}
static cplx* link_m(double* U, int nc, int64_t V, int mu, int64_t lex) {
  return (cplx*)U + ((int64_t)mu * V + lex) * nc * nc;
}

/* ------------------------------------------------------------------------ */
/* Dense complex matrices, row-major nc x nc.                                */
/* ------------------------------------------------------------------------ */
static void mat_mul(int n, const cplx* A, const cplx* B, cplx* C) { /* C = A B */
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      cplx s = 0;
      for (int k = 0; k < n; ++k) s += A[i * n + k] * B[k * n + j];
      C[i * n + j] = s;
    }
}

static void mat_dag(int n, const cplx* A, cplx* B) { /* B = A^+ */
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) B[i * n + j] = conj(A[j * n + i]);
}

static void mat_copy(int n, const cplx* A, cplx* B) { memcpy(B, A, sizeof(cplx) * n * n); }

static double re_trace(int n, const cplx* A) {
  double s = 0;
  for (int i = 0; i < n; ++i) s += creal(A[i * n + i]);
  return s;
}

/* determinant by Gaussian elimination with partial pivoting */
static cplx mat_det(int n, const cplx* A) {
  cplx M[ORC_NC_MAX * ORC_NC_MAX];
  mat_copy(n, A, M);
  cplx det = 1;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (cabs(M[r * n + c]) > cabs(M[piv * n + c])) piv = r;
    if (M[piv * n + c] == 0) return 0;
    if (piv != c) {
      for (int k = 0; k < n; ++k) {
        cplx t = M[c * n + k];
        M[c * n + k] = M[piv * n + k];
        M[piv * n + k] = t;
      }
      det = -det;
    }
    det *= M[c * n + c];
    for (int r = c + 1; r < n; ++r) {
      cplx f = M[r * n + c] / M[c * n + c];
      for (int k = c; k < n; ++k) M[r * n + k] -= f * M[c * n + k];
    }
  }
  return det;
}

/* ------------------------------------------------------------------------ */
/* SU(2) elements as 2x2 matrices a0*1 + i(a1 s1 + a2 s2 + a3 s3) (Eq. 6).   */
/* ------------------------------------------------------------------------ */
static void su2_from_quaternion(const double a[4], cplx M[4]) {
  /* Pauli matrices */
  const cplx s1[4] = {0, 1, 1, 0};
  const cplx s2[4] = {0, -I, I, 0};
  const cplx s3[4] = {1, 0, 0, -1};
  for (int e = 0; e < 4; ++e)
    M[e] = a[0] * (e == 0 || e == 3 ? 1.0 : 0.0) + I * (a[1] * s1[e] + a[2] * s2[e] + a[3] * s3[e]);
}

/* orthogonal projection of a 2x2 complex block onto the real span of SU(2):
 * v0 = 1/2 ReTr(w), vk = 1/2 ReTr((i s_k)^+ w)                              */
static void su2_project(const cplx w[4], double v[4]) {
  const cplx s1[4] = {0, 1, 1, 0};
  const cplx s2[4] = {0, -I, I, 0};
  const cplx s3[4] = {1, 0, 0, -1};
  const cplx* s[3] = {s1, s2, s3};
  v[0] = 0.5 * creal(w[0] + w[3]);
  for (int k = 0; k < 3; ++k) {
    cplx g[4], gd[4], p[4];
    for (int e = 0; e < 4; ++e) g[e] = I * s[k][e];
    mat_dag(2, g, gd);
    mat_mul(2, gd, w, p);
    v[k + 1] = 0.5 * creal(p[0] + p[3]);
  }
}

/* ------------------------------------------------------------------------ */
/* SU(2) heatbath element (Eqs. 12-13): b0 with density sqrt(1-b0^2)e^{alpha */
/* b0}, b-vector uniform on the sphere of radius sqrt(1-b0^2).               */
/* Returns attempts used (1..64) or 0 when the cap was reached (b = 1).      */
/* ------------------------------------------------------------------------ */
int orc_su2_heatbath(double alpha, uint64_t seed, uint32_t link_id, uint32_t hb_step,
                     int subgroup, double b[4]) {
  double b0 = 1.0;
  int used = 0;
  for (int attempt = 0; attempt < HB_MAX_ATTEMPTS; ++attempt) {
    double r[4];
    draw4(seed, link_id, hb_step, ((uint32_t)subgroup << 16) | (uint32_t)attempt, TAG_HEATBATH, r);
    if (alpha >= ALPHA_SWITCH) {
      /* Kennedy-Pendleton: delta = (1-b0)/2 proposed from Gamma(3/2, rate 2 alpha)
       * (an exponential plus half a squared normal), accepted with sqrt(1-delta). */
      double c = cos(2.0 * M_PI * r[1]);
      double delta = -(log(r[0]) + c * c * log(r[2])) / (2.0 * alpha);
      if (r[3] * r[3] <= 1.0 - delta) {
        b0 = 1.0 - 2.0 * delta;
        used = attempt + 1;
        break;
      }
    } else {
      /* Creutz: b0 from e^{alpha b0} on [-1,1] by inversion, accepted with sqrt(1-b0^2). */
      double e = -expm1(-2.0 * alpha); /* 1 - e^{-2 alpha} */
      /* at alpha = 0 (beta = 0) the inversion is 0/0: take its limit 1 - 2 r */
      double x = alpha > 0.0 ? 1.0 + log1p(-r[0] * e) / alpha : 1.0 - 2.0 * r[0];
      if (r[1] * r[1] <= 1.0 - x * x) {
        b0 = x;
        used = attempt + 1;
        break;
      }
    }
  }
  if (!used) {
    b[0] = 1; b[1] = b[2] = b[3] = 0;
    return 0;
  }
  double r[4];
  draw4(seed, link_id, hb_step, ((uint32_t)subgroup << 16) | (uint32_t)HB_MAX_ATTEMPTS, TAG_HEATBATH, r);
  double cos_theta = 2.0 * r[0] - 1.0;
  double sin_theta = sqrt(1.0 - cos_theta * cos_theta);
  double phi = 2.0 * M_PI * r[1];
  double rho = sqrt(fmax(0.0, 1.0 - b0 * b0));
  b[0] = b0;
  b[1] = rho * sin_theta * cos(phi);
  b[2] = rho * sin_theta * sin(phi);
  b[3] = rho * cos_theta;
  return used;
}

/* ------------------------------------------------------------------------ */
/* Staple, Eq. 9: sum over nu != mu of                                       */
/*   U_nu(x) U_mu(x+nu) U_nu(x+mu)^+ + U_nu(x-nu)^+ U_mu(x-nu) U_nu(x-nu+mu)  */
/* ------------------------------------------------------------------------ */
void orc_staple(const double* U, int nc, const int dims[4], int mu, int64_t lex, double* Sout) {
  int64_t V = volume(dims);
  cplx* S = (cplx*)Sout;
  cplx T1[ORC_NC_MAX * ORC_NC_MAX], T2[ORC_NC_MAX * ORC_NC_MAX], D[ORC_NC_MAX * ORC_NC_MAX];
  for (int e = 0; e < nc * nc; ++e) S[e] = 0;
  for (int nu = 0; nu < 4; ++nu) {
    if (nu == mu) continue;
    int64_t xpmu = hop(dims, lex, mu, +1);
    int64_t xpnu = hop(dims, lex, nu, +1);
    int64_t xmnu = hop(dims, lex, nu, -1);
    int64_t xmnupmu = hop(dims, xmnu, mu, +1);
    /* forward: U_nu(x) U_mu(x+nu) U_nu(x+mu)^+ */
    mat_mul(nc, link_c(U, nc, V, nu, lex), link_c(U, nc, V, mu, xpnu), T1);
    mat_dag(nc, link_c(U, nc, V, nu, xpmu), D);
    mat_mul(nc, T1, D, T2);
    for (int e = 0; e < nc * nc; ++e) S[e] += T2[e];
    /* backward: U_nu(x-nu)^+ U_mu(x-nu) U_nu(x-nu+mu) */
    mat_dag(nc, link_c(U, nc, V, nu, xmnu), D);
    mat_mul(nc, D, link_c(U, nc, V, mu, xmnu), T1);
    mat_mul(nc, T1, link_c(U, nc, V, nu, xmnupmu), T2);
    for (int e = 0; e < nc * nc; ++e) S[e] += T2[e];
  }
}

/* ------------------------------------------------------------------------ */
/* One link update (Sec. 2): W = U Sigma^+; for each SU(2) subgroup (i,j)   */
/* in lexicographic order, project the (i,j) block of W, draw (heatbath) or  */
/* reflect (overrelaxation) the subgroup element A, then U <- A U, W <- A W  */
/* on rows i and j (Eq. 15).  Returns the number of subgroups whose heatbath */
/* reached the attempt cap.                                                 */
/* ------------------------------------------------------------------------ */
int orc_update_link(double* Ulink, const double* Sigma, int nc, double beta, int mode,
                    uint64_t seed, uint32_t link_id, uint32_t hb_step) {
  cplx* U = (cplx*)Ulink;
  const cplx* S = (const cplx*)Sigma;
  cplx Sd[ORC_NC_MAX * ORC_NC_MAX], W[ORC_NC_MAX * ORC_NC_MAX];
  mat_dag(nc, S, Sd);
  mat_mul(nc, U, Sd, W);
  int capped = 0;
  int subgroup = 0;
  for (int i = 0; i < nc - 1; ++i) {
    for (int j = i + 1; j < nc; ++j, ++subgroup) {
      cplx w[4] = {W[i * nc + i], W[i * nc + j], W[j * nc + i], W[j * nc + j]};
      double v[4];
      su2_project(w, v);
      double k = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2] + v[3] * v[3]);
      if (!(k > K_MIN) || !isfinite(k)) continue;
      double vhat[4] = {v[0] / k, v[1] / k, v[2] / k, v[3] / k};
      cplx Vh[4], Vhd[4], A[4];
      su2_from_quaternion(vhat, Vh);
      mat_dag(2, Vh, Vhd);
      if (mode == ORC_HEATBATH) {
        double alpha = 2.0 * beta * k / nc;
        double b[4];
        cplx B[4];
        if (orc_su2_heatbath(alpha, seed, link_id, hb_step, subgroup, b) == 0) {
          ++capped;
          continue;
        }
        su2_from_quaternion(b, B);
        mat_mul(2, B, Vhd, A); /* A = b vhat^+ */
      } else {
        mat_mul(2, Vhd, Vhd, A); /* A = (vhat^+)^2 */
      }
      /* left-multiply rows i, j of U and of W by the embedded A */
      for (int c = 0; c < nc; ++c) {
        cplx ui = U[i * nc + c], uj = U[j * nc + c];
        U[i * nc + c] = A[0] * ui + A[1] * uj;
        U[j * nc + c] = A[2] * ui + A[3] * uj;
        cplx wi = W[i * nc + c], wj = W[j * nc + c];
        W[i * nc + c] = A[0] * wi + A[1] * wj;
        W[j * nc + c] = A[2] * wi + A[3] * wj;
      }
    }
  }
  return capped;
}

/* ------------------------------------------------------------------------ */
/* Re-unitarization (Sec. 2, R8).                                            */
/* ------------------------------------------------------------------------ */
static void normalise_row(int n, cplx* row) {
  double s = 0;
  for (int c = 0; c < n; ++c) s += creal(row[c] * conj(row[c]));
  double inv = 1.0 / sqrt(s);
  for (int c = 0; c < n; ++c) row[c] *= inv;
}

void orc_reunit_link(double* Ulink, int nc) {
  cplx* U = (cplx*)Ulink;
  if (nc == 2) {
    normalise_row(2, U);
    U[2] = -conj(U[1]);
    U[3] = conj(U[0]);
    return;
  }
  int gs_rows = (nc == 3) ? 2 : nc;
  for (int r = 0; r < gs_rows; ++r) {
    for (int s = 0; s < r; ++s) {
      cplx p = 0; /* <row s, row r> */
      for (int c = 0; c < nc; ++c) p += conj(U[s * nc + c]) * U[r * nc + c];
      for (int c = 0; c < nc; ++c) U[r * nc + c] -= p * U[s * nc + c];
    }
    normalise_row(nc, U + r * nc);
  }
  if (nc == 3) {
    const cplx* a = U;
    const cplx* b = U + 3;
    U[6] = conj(a[1] * b[2] - a[2] * b[1]);
    U[7] = conj(a[2] * b[0] - a[0] * b[2]);
    U[8] = conj(a[0] * b[1] - a[1] * b[0]);
  } else {
    cplx d = mat_det(nc, U);
    cplx phase = conj(d) / cabs(d);
    for (int c = 0; c < nc; ++c) U[(nc - 1) * nc + c] *= phase;
  }
}

/* Hot start (R9): complex Gaussians from Box-Muller pairs, row by row,
 * then Gram-Schmidt + determinant phase. */
void orc_random_sun(double* Ulink, int nc, uint64_t seed, uint32_t link_id) {
  cplx* U = (cplx*)Ulink;
  int n_normals = 2 * nc * nc;
  double g[2 * ORC_NC_MAX * ORC_NC_MAX + 4];
  for (int call = 0; 4 * call < n_normals; ++call) {
    double r[4];
    draw4(seed, link_id, 0u, (uint32_t)call, TAG_INIT, r);
    for (int pair = 0; pair < 2; ++pair) {
      double rad = sqrt(-2.0 * log(r[2 * pair]));
      double ang = 2.0 * M_PI * r[2 * pair + 1];
      g[4 * call + 2 * pair] = rad * cos(ang);
      g[4 * call + 2 * pair + 1] = rad * sin(ang);
    }
  }
  for (int e = 0; e < nc * nc; ++e) U[e] = g[2 * e] + I * g[2 * e + 1];
  orc_reunit_link(Ulink, nc);
}

/* ------------------------------------------------------------------------ */
/* Lattice-wide operations                                                   */
/* ------------------------------------------------------------------------ */
void orc_init(double* U, int nc, const int dims[4], int hot, uint64_t seed) {
  int64_t V = volume(dims);
  int64_t nlinks = 4 * V;
#pragma omp parallel for schedule(static)
  for (int64_t l = 0; l < nlinks; ++l) {
    cplx* u = (cplx*)U + l * nc * nc;
    if (hot) {
      orc_random_sun((double*)u, nc, seed, (uint32_t)l);
    } else {
      for (int r = 0; r < nc; ++r)
        for (int c = 0; c < nc; ++c) u[r * nc + c] = (r == c) ? 1.0 : 0.0;
    }
  }
}

/* One checkerboard pass (Sec. 3): every link U_mu(x) with parity(x) == parity
 * and t in [t_begin, t_end) is updated.  Links of one pass never share a
 * staple, so the order (reverse = 1 walks it backwards) does not matter.
 * Returns the number of subgroup heatbaths that reached the attempt cap. */
int64_t orc_pass(double* U, int nc, const int dims[4], double beta, int mode, int mu,
                 int parity, uint32_t hb_step, uint64_t seed, int t_begin, int t_end,
                 int reverse, int reunit_mod, int reunit_rem) {
  int64_t V = volume(dims);
  int64_t per_t = (int64_t)dims[0] * dims[1] * dims[2];
  if (t_begin < 0) t_begin = 0;
  if (t_end > dims[3] || t_end < 0) t_end = dims[3];
  int64_t first = per_t * t_begin, count = per_t * (t_end - t_begin);
  int64_t capped = 0;
#pragma omp parallel for schedule(static) reduction(+ : capped)
  for (int64_t n = 0; n < count; ++n) {
    int64_t lex = reverse ? first + count - 1 - n : first + n;
    if (parity_of(dims, lex) != parity) continue;
    cplx S[ORC_NC_MAX * ORC_NC_MAX];
    orc_staple(U, nc, dims, mu, lex, (double*)S);
    capped += orc_update_link((double*)link_m(U, nc, V, mu, lex), (const double*)S, nc, beta,
                              mode, seed, (uint32_t)((int64_t)mu * V + lex), hb_step);
    if (reunit_mod > 0 && ((lex >> 1) >> 5) % reunit_mod == reunit_rem)
      orc_reunit_link((double*)link_m(U, nc, V, mu, lex), nc);
  }
  return capped;
}

void orc_reunitarize(double* U, int nc, const int dims[4]) {
  int64_t nlinks = 4 * volume(dims);
#pragma omp parallel for schedule(static)
  for (int64_t l = 0; l < nlinks; ++l) orc_reunit_link(U + 2 * l * nc * nc, nc);
}

/* One sweep: n_hb heatbath steps (heatbath step counter hb_step0, hb_step0+1, ...),
 * then n_or overrelaxation steps, each step = 4 directions x (even, odd); then
 * re-unitarization as R11 (reunit = 0 none, 1 after the sweep, 2 in the last
 * step, 3 spread over the steps). */
void orc_sweep(double* U, int nc, const int dims[4], double beta, int n_hb, int n_or,
               int reunit, uint64_t seed, uint32_t hb_step0) {
  int n_steps = n_hb + n_or;
  for (int s = 0; s < n_steps; ++s) {
    int heatbath = s < n_hb;
    int mod = 0, rem = 0;
    if (reunit == 2 && s == n_steps - 1) mod = 1;
    if (reunit == 3) {
      mod = n_steps;
      rem = s;
    }
    for (int mu = 0; mu < 4; ++mu)
      for (int p = 0; p < 2; ++p)
        orc_pass(U, nc, dims, beta, heatbath ? ORC_HEATBATH : ORC_OVERRELAX, mu, p,
                 heatbath ? hb_step0 + (uint32_t)s : 0u, seed, 0, dims[3], 0, mod, rem);
  }
  if (reunit == 1 || (reunit >= 2 && n_steps == 0)) orc_reunitarize(U, nc, dims);
}

/* Plaquette average, Eq. 4 with the normalisation of R10.  Partial sums per
 * time slice are added in slice order, so the result does not depend on the
 * number of threads. */
double orc_plaquette(const double* U, int nc, const int dims[4]) {
  int64_t V = volume(dims);
  int64_t per_t = (int64_t)dims[0] * dims[1] * dims[2];
  double* part = (double*)calloc((size_t)dims[3], sizeof(double));
#pragma omp parallel for schedule(static)
  for (int t = 0; t < dims[3]; ++t) {
    double s = 0;
    for (int64_t i = 0; i < per_t; ++i) {
      int64_t lex = (int64_t)t * per_t + i;
      for (int mu = 0; mu < 4; ++mu)
        for (int nu = mu + 1; nu < 4; ++nu) {
          cplx A[ORC_NC_MAX * ORC_NC_MAX], B[ORC_NC_MAX * ORC_NC_MAX], D[ORC_NC_MAX * ORC_NC_MAX];
          /* P = U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+ */
          mat_mul(nc, link_c(U, nc, V, mu, lex), link_c(U, nc, V, nu, hop(dims, lex, mu, +1)), A);
          mat_dag(nc, link_c(U, nc, V, mu, hop(dims, lex, nu, +1)), D);
          mat_mul(nc, A, D, B);
          mat_dag(nc, link_c(U, nc, V, nu, lex), D);
          mat_mul(nc, B, D, A);
          s += re_trace(nc, A);
        }
    }
    part[t] = s;
  }
  double total = 0;
  for (int t = 0; t < dims[3]; ++t) total += part[t];
  free(part);
  return total / (6.0 * (double)V * nc);
}

/* Polyakov loop (R10): ordered product of the temporal links along t. */
void orc_polyakov(const double* U, int nc, const int dims[4], double* re, double* im) {
  int64_t V = volume(dims);
  int64_t per_t = (int64_t)dims[0] * dims[1] * dims[2];
  double* part_re = (double*)calloc((size_t)dims[2], sizeof(double));
  double* part_im = (double*)calloc((size_t)dims[2], sizeof(double));
  int64_t per_z = (int64_t)dims[0] * dims[1];
#pragma omp parallel for schedule(static)
  for (int z = 0; z < dims[2]; ++z) {
    cplx sum = 0;
    for (int64_t i = 0; i < per_z; ++i) {
      int64_t xs = (int64_t)z * per_z + i; /* spatial lex */
      cplx P[ORC_NC_MAX * ORC_NC_MAX], T[ORC_NC_MAX * ORC_NC_MAX];
      mat_copy(nc, link_c(U, nc, V, 3, xs), P);
      for (int t = 1; t < dims[3]; ++t) {
        mat_mul(nc, P, link_c(U, nc, V, 3, xs + (int64_t)t * per_t), T);
        mat_copy(nc, T, P);
      }
      for (int d = 0; d < nc; ++d) sum += P[d * nc + d];
    }
    part_re[z] = creal(sum);
    part_im[z] = cimag(sum);
  }
  double sr = 0, si = 0;
  for (int z = 0; z < dims[2]; ++z) {
    sr += part_re[z];
    si += part_im[z];
  }
  free(part_re);
  free(part_im);
  *re = sr / ((double)nc * per_t);
  *im = si / ((double)nc * per_t);
}
