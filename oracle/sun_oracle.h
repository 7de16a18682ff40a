/*
 * sun_oracle.h -- plain FP64 CPU oracle for the SU(Nc) pure-gauge link sweep of
 * Cardoso & Bicudo, "Generating SU(Nc) pure gauge lattice QCD configurations on
 * GPUs with CUDA" (arXiv:1112.4533).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or calls
 * this library: only the test-suite, the smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no code, header, table or constant generator
 * with the CUDA library; the two meet only through the canonical link order
 * below and the published definition of Philox4x32-10.
 *
 * Link storage (canonical order, also the host interchange format of the CUDA
 * library): a flat array of doubles
 *     U[ ((mu*V + lex)*nc + row)*nc + col ][re, im]
 * with V = Nx*Ny*Nz*Nt, lex = x + Nx*(y + Ny*(z + Nz*t)), mu = 0..3 = x,y,z,t.
 * Periodic boundaries in all four directions (Sec. 2).  Every extent must be
 * even and >= 2 so that the even/odd colouring of the checkerboard is
 * consistent across the boundary.
 *
 * Functions marked "parity unpinned" in sun_oracle.c have no pin independent of
 * the oracle itself; all others are pinned by tests/test_oracle_*.py.
 */
#ifndef SUN_ORACLE_H
#define SUN_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_NC_MAX 8

/* update modes */
#define ORC_HEATBATH 0
#define ORC_OVERRELAX 1

int orc_version(void);
int orc_set_threads(int n);     /* OpenMP threads used by lattice-wide loops; returns the count in effect */
int orc_get_threads(void);

/* Philox4x32-10 of Salmon, Moraes, Dror & Shaw (SC'11). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* uniform in (0,1): (floor(u / 2^9) + 1/2) * 2^-23 -- exact in float and double */
double orc_uniform(uint32_t u);

/* Lattice-wide operations (U in canonical order, dims = {Nx,Ny,Nz,Nt}). */
void orc_init(double* U, int nc, const int dims[4], int hot, uint64_t seed);
/* reunit_mod > 0: after its update, link U_mu(x) is re-unitarized when
 * ((lex >> 1) >> 5) % reunit_mod == reunit_rem (runs of 32 consecutive even/odd
 * site indices); reunit_mod = 1, reunit_rem = 0 selects every link */
int64_t orc_pass(double* U, int nc, const int dims[4], double beta, int mode, int mu,
                 int parity, uint32_t hb_step, uint64_t seed, int t_begin, int t_end,
                 int reverse, int reunit_mod, int reunit_rem);
/* reunit: 0 none, 1 every link after the sweep (Sec. 2/3 placement), 2 each link
 * right after its update in the sweep's last step, 3 each run r of 32 links right
 * after its update in step r mod (n_hb + n_or) */
void orc_sweep(double* U, int nc, const int dims[4], double beta, int n_hb, int n_or,
               int reunit, uint64_t seed, uint32_t hb_step0);
void orc_reunitarize(double* U, int nc, const int dims[4]);
double orc_plaquette(const double* U, int nc, const int dims[4]);
void orc_polyakov(const double* U, int nc, const int dims[4], double* re, double* im);

/* Single-link pieces, exposed for pins and sampled parity checks. */
void orc_staple(const double* U, int nc, const int dims[4], int mu, int64_t lex, double* S);
int orc_update_link(double* Ulink, const double* S, int nc, double beta, int mode,
                    uint64_t seed, uint32_t link_id, uint32_t hb_step);
int orc_su2_heatbath(double alpha, uint64_t seed, uint32_t link_id, uint32_t hb_step,
                     int subgroup, double b[4]);
void orc_reunit_link(double* Ulink, int nc);
void orc_random_sun(double* Ulink, int nc, uint64_t seed, uint32_t link_id);

#ifdef __cplusplus
}
#endif
#endif
