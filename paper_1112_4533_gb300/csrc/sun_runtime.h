// sun_runtime.h -- host/device types shared by the kernels and the C-ABI runtime.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace sun {

// Division of n < 2^31 by a fixed divisor d < 2^31 with one multiply-high, add
// and shift: q = (umulhi(n, m) + n) >> s with s = ceil(log2 d) and
// m = floor(2^32 (2^s - d) / d) + 1 (Granlund & Montgomery, "Division by
// invariant integers using multiplication", PLDI 1994, Sec. 4).
struct FastDiv {
  uint32_t d, m, s;
};

inline FastDiv make_fastdiv(uint32_t d) {
  FastDiv f;
  f.d = d;
  uint32_t s = 0;
  while ((uint64_t(1) << s) < d) ++s;
  f.s = s;
  f.m = uint32_t((((uint64_t(1) << 32) * ((uint64_t(1) << s) - d)) / d) + 1);
  return f;
}

// Lattice geometry: periodic Nx x Ny x Nz x Nt, even extents, even/odd site order.
// Site indices fit in 32 bits (V <= 2^30).
struct Geom {
  int nx, ny, nz, nt;
  int nxh;            // nx / 2
  int64_t V, Vh;      // sites, sites per parity
  int64_t stride[4];  // lex strides of x, y, z, t
  FastDiv div_nxh, div_ny, div_nz, div_nx;
};

// Device-resident mutable state of one lattice.
struct DevState {
  uint32_t hb_step;       // heatbath step counter (Philox counter word 1)
  uint32_t slot;          // observable-history slot of the current sweep
  unsigned plaq_counter;  // blocks finished, plaquette reduction
  unsigned poly_counter;  // blocks finished, Polyakov reduction
};

constexpr int kMaxReduceBlocks = 1024;

// Words of a lattice's wavefront synchronisation area before the per-t-slice
// counters: wait timeouts, ticket.
constexpr int kWaveSyncWords = 2;

// Everything a launcher needs to enqueue work on one lattice.
struct Ctx {
  char* links;          // 8 blocks (direction, parity)
  int64_t block_bytes;  // Vh * link bytes
  Geom g;
  double beta;
  uint64_t seed;
  int nc;
  DevState* state;
  double* partials;  // 4 * kMaxReduceBlocks doubles
  cudaStream_t stream;
  int block_threads;
  int reduce_blocks;
  int obs_stride, obs_offset;  // observable output: row stride and column (1, 0 for one lattice)
  int variant;  // update-pass kernel variant (1: 5 blocks/SM register bound, 2: two-row staple, 4: swap row-parallel / per-link
                // kernel for Nc 4, 6, 8: even and odd pass of a direction in one wavefront launch,
                // 16: two links per thread in packed FP32 for SU(3) FP32 overrelaxation)
  uint32_t* wave;  // kWaveSyncWords + Nt words of wavefront synchronisation
  int wave_lag;    // t-slices the even units of a wavefront run ahead of the odd ones
  uint32_t wave_skip;  // fault injection: leading units every wavefront launch leaves out (0 normally)
  // A slab of a lattice cut into t-slabs (otherwise the whole lattice: [0, Vh),
  // 0, V): passes and the plaquette cover half-sites [h_begin, h_end) of each
  // parity, and local site lex is site (lex + lex_offset) mod v_global of the
  // whole lattice (random numbers, re-unitarization runs, hot start).
  int64_t h_begin, h_end;
  uint32_t lex_offset, v_global;
};

// One chain (lattice) of a batch, as the batched kernels read it.
struct ChainDesc {
  char* links;
  int64_t block_bytes;
  Geom g;
  double alpha_coef;   // 2 beta / Nc
  uint2 key;           // Philox key (seed)
  uint32_t* hb_step;   // the chain's device heatbath step counter
  double plaq_scale;   // 1 / (6 V Nc)
  double poly_scale;   // 1 / (Nc Nx Ny Nz)
};

// Kernel-side view of a batch for one kernel kind: block b belongs to chain c
// with start[c] <= b < start[c+1].
struct BatchParams {
  const ChainDesc* chains;
  const uint32_t* start;
  int n;
};

// Everything a batched launcher needs (device tables of one group of chains).
struct BatchCtx {
  const ChainDesc* chains;
  int n;
  const uint32_t* pass_start;
  const uint32_t* reunit_start;
  const uint32_t* plaq_start;
  const uint32_t* poly_start;
  const uint32_t* group_start;  // pass table in blocks of group_links_per_block links (row-parallel kernel)
  uint32_t pass_blocks, reunit_blocks, plaq_blocks, poly_blocks, group_blocks;
  int pass_threads;  // block size the pass table was built for
  int variant;
  double* partials;  // >= max(plaq_blocks, 2 * poly_blocks) doubles
  cudaStream_t stream;
};

// The operations of one (Nc, storage, precision) combination.
struct Ops {
  int nc, storage, precision, link_bytes;
  int fused_reunit;  // reunit_mode 1 and 2 built
  int group_links_per_block;  // > 0: passes without re-unitarization use the row-parallel kernel
  cudaError_t (*pass)(const Ctx&, int mode, int mu, int parity, uint32_t step_offset, uint32_t reunit_mod,
                      uint32_t reunit_rem);
  // both parities of direction mu in one wavefront launch (same results as the two passes)
  cudaError_t (*pass_pair)(const Ctx&, int mode, int mu, uint32_t step_offset, uint32_t reunit_mod,
                           uint32_t reunit_rem);
  cudaError_t (*init)(const Ctx&, int hot);
  cudaError_t (*reunit)(const Ctx&);
  cudaError_t (*plaquette)(const Ctx&, double* out, const uint32_t* slot, int cap);
  cudaError_t (*polyakov)(const Ctx&, double* out, const uint32_t* slot, int cap);
  // t-slabs: per-spatial-site products over a slab's interior slices, and their
  // ordered product and trace over n slabs (the Polyakov loop of the whole lattice)
  cudaError_t (*polyakov_partial)(const Ctx&, void* out);
  cudaError_t (*polyakov_combine)(const Ctx&, const void* const* parts, int n, double* out, const uint32_t* slot,
                                  int cap);
  size_t polyakov_partial_bytes;  // per spatial site
  // max |U U^+ - 1|, max |det U - 1| (as double bit patterns) and the non-finite count into out[0..2]
  cudaError_t (*check_links)(const Ctx&, unsigned long long* out);
  cudaError_t (*export_links)(const Ctx&, double* dst, int64_t first, int64_t count);
  cudaError_t (*import_links)(const Ctx&, const double* src, int64_t first, int64_t count);
  // the compact host format: stored rows in the storage precision, canonical order
  cudaError_t (*export_stored)(const Ctx&, void* dst, int64_t first, int64_t count);
  cudaError_t (*import_stored)(const Ctx&, const void* src, int64_t first, int64_t count);
  cudaError_t (*batch_pass)(const BatchCtx&, int mode, int mu, int parity, uint32_t step_offset, uint32_t reunit_mod,
                            uint32_t reunit_rem);
  cudaError_t (*batch_reunit)(const BatchCtx&);
  // per-chain results to out[((*slot % cap) * stride + offset + c) * K + k]
  cudaError_t (*batch_plaquette)(const BatchCtx&, double* out, const uint32_t* slot, int cap, int offset, int stride);
  cudaError_t (*batch_polyakov)(const BatchCtx&, double* out, const uint32_t* slot, int cap, int offset, int stride);
};

const Ops* ops_su2(int storage, int precision);
const Ops* ops_su3(int storage, int precision);
const Ops* ops_su3_two_row(int precision);
const Ops* ops_su3_full(int precision);
const Ops* ops_su4(int storage, int precision);
const Ops* ops_su5(int storage, int precision);
const Ops* ops_su6(int storage, int precision);
const Ops* ops_su4_f32();
const Ops* ops_su4_f64();
const Ops* ops_su5_f32();
const Ops* ops_su5_f64();
const Ops* ops_su6_f32();
const Ops* ops_su6_f64();

// sets the calling thread's sun_last_error() message
void set_last_error_message(const char* msg);

}  // namespace sun
