// sun_runtime.h -- host/device types shared by the kernels and the C-ABI runtime.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace sun {

// Lattice geometry: periodic Nx x Ny x Nz x Nt, even extents, even/odd site order.
struct Geom {
  int nx, ny, nz, nt;
  int nxh;            // nx / 2
  int64_t V, Vh;      // sites, sites per parity
  int64_t stride[4];  // lex strides of x, y, z, t
};

// Device-resident mutable state of one lattice.
struct DevState {
  uint32_t hb_step;       // heatbath step counter (Philox counter word 1)
  uint32_t slot;          // observable-history slot of the current sweep
  unsigned plaq_counter;  // blocks finished, plaquette reduction
  unsigned poly_counter;  // blocks finished, Polyakov reduction
};

constexpr int kMaxReduceBlocks = 1024;

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
};

// The operations of one (Nc, storage, precision) combination.
struct Ops {
  int nc, storage, precision, link_bytes;
  cudaError_t (*pass)(const Ctx&, int mode, int mu, int parity, uint32_t step_offset);
  cudaError_t (*init)(const Ctx&, int hot);
  cudaError_t (*reunit)(const Ctx&);
  cudaError_t (*plaquette)(const Ctx&, double* out, const uint32_t* slot, int cap);
  cudaError_t (*polyakov)(const Ctx&, double* out, const uint32_t* slot, int cap);
  cudaError_t (*export_links)(const Ctx&, double* dst, int64_t first, int64_t count);
  cudaError_t (*import_links)(const Ctx&, const double* src, int64_t first, int64_t count);
};

const Ops* ops_su2(int storage, int precision);
const Ops* ops_su3(int storage, int precision);
const Ops* ops_su4(int storage, int precision);
const Ops* ops_su5(int storage, int precision);
const Ops* ops_su6(int storage, int precision);

}  // namespace sun
