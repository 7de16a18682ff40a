// api_internal.h -- what the translation units of the C ABI share: error
// reporting, the device-memory plan of a lattice, the lattice handle itself and
// the helpers that enqueue its work.  Not part of the public interface.
#pragma once

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "sun.h"
#include "sun_runtime.h"

namespace sun_api {

// records the message for sun_last_error() of the calling thread and returns s
sun_status fail(sun_status s, const char* fmt, ...);

#define SUN_CUDA(call)                                                                             \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess)                                                                         \
      return ::sun_api::fail(SUN_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                             __FILE__, __LINE__);                                                  \
  } while (0)

#define SUN_TRY(expr)               \
  do {                              \
    sun_status s_ = (expr);         \
    if (s_ != SUN_OK) return s_;    \
  } while (0)

constexpr size_t kAlign = 256;
constexpr size_t kStagingCap = size_t(16) << 20;  // import/export chunk buffer
constexpr int kDefaultWaveLag = 3;  // t-slices even units of a wavefront launch run ahead
constexpr int kHistCap = 1024;                    // sweeps per observable-history chunk

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

inline const sun::Ops* find_ops(int nc, int storage, int precision) {
  switch (nc) {
    case 2: return sun::ops_su2(storage, precision);
    case 3: return sun::ops_su3(storage, precision);
    case 4: return sun::ops_su4(storage, precision);
    case 5: return sun::ops_su5(storage, precision);
    case 6: return sun::ops_su6(storage, precision);
    default: return nullptr;
  }
}

inline int default_storage(int nc) { return nc == 2 ? 4 : (nc == 3 ? 12 : 2 * nc * nc); }

inline sun_status check_dims(const int* dims) {
  if (!dims) return fail(SUN_ERR_ARG, "dims is NULL");
  int64_t V = 1;
  for (int m = 0; m < 4; ++m) {
    if (dims[m] < 2 || (dims[m] & 1))
      return fail(SUN_ERR_ARG, "lattice extent dims[%d] = %d must be even and >= 2", m, dims[m]);
    V *= dims[m];
    if (V > (int64_t(1) << 30)) break;
  }
  if (4 * V >= (int64_t(1) << 32)) return fail(SUN_ERR_ARG, "4 * volume must be < 2^32");
  return SUN_OK;
}

struct Plan {
  size_t links_off, state_off, wave_off, partials_off, results_off, hist_off, staging_off, total;
  size_t links_bytes, staging_bytes;
  int64_t staging_links;
};

inline Plan make_plan(int nc, const int* dims, int link_bytes) {
  Plan p;
  const int64_t V = int64_t(dims[0]) * dims[1] * dims[2] * dims[3];
  const size_t canon_link = size_t(2) * nc * nc * sizeof(double);
  p.links_bytes = size_t(4 * V) * size_t(link_bytes);
  int64_t sl = int64_t(kStagingCap / canon_link);
  if (sl < 1) sl = 1;
  if (sl > 4 * V) sl = 4 * V;
  p.staging_links = sl;
  p.staging_bytes = size_t(sl) * canon_link;
  size_t off = 0;
  p.links_off = off;
  off = align_up(off + p.links_bytes, kAlign);
  p.state_off = off;
  off = align_up(off + sizeof(sun::DevState), kAlign);
  p.wave_off = off;
  off = align_up(off + (sun::kWaveSyncWords + size_t(dims[3])) * sizeof(uint32_t), kAlign);
  p.partials_off = off;
  off = align_up(off + 4 * sun::kMaxReduceBlocks * sizeof(double), kAlign);
  p.results_off = off;
  off = align_up(off + 8 * sizeof(double), kAlign);
  p.hist_off = off;
  off = align_up(off + 3 * kHistCap * sizeof(double), kAlign);
  p.staging_off = off;
  off = align_up(off + p.staging_bytes, kAlign);
  p.total = off;
  return p;
}

struct GraphKey {
  int n_hb, n_or, reunit, plaq, poly;
  int sweeps = 1;  // sweeps captured in the graph
  bool operator<(const GraphKey& o) const {
    return std::tie(n_hb, n_or, reunit, plaq, poly, sweeps) <
           std::tie(o.n_hb, o.n_or, o.reunit, o.plaq, o.poly, o.sweeps);
  }
};

}  // namespace sun_api

// the opaque lattice handle of include/sun.h
struct sun_lattice {
  int nc = 0, precision = 0, storage = 0;
  int dims[4] = {0, 0, 0, 0};
  double beta = 0.0;
  uint64_t seed = 0;
  int reunit_every = 1, reunit_mode = 0, block_threads = 128, use_graphs = 1, graph_sweeps = 1;
  int device = 0;
  uint64_t sweeps_done = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaStream_t capture_stream = nullptr;
  char* base = nullptr;
  bool own_mem = false;
  sun_api::Plan plan{};
  const sun::Ops* ops = nullptr;
  sun::Ctx ctx{};
  double* results = nullptr;
  double* hist = nullptr;
  double* staging = nullptr;
  double host_results[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // pageable: creating a lattice pins nothing
  std::map<sun_api::GraphKey, cudaGraphExec_t> graphs;
};

namespace sun_api {

sun_status set_device(const sun_lattice* L);
void drop_graphs(sun_lattice* L);
sun::Ctx ctx_on(const sun_lattice* L, cudaStream_t s);
sun_status check_launch(cudaError_t e, const char* what);
sun_status enqueue_step(const sun::Ops* ops, const sun::Ctx& c, int mode, uint32_t step_offset, uint32_t mod,
                        uint32_t rem);
sun_status enqueue_sweep(sun_lattice* L, cudaStream_t s, int n_hb, int n_or, bool reunit, bool plaq, bool poly,
                         bool hist_mode);
bool reunit_due(const sun_lattice* L, uint64_t sweep_index);
sun_status get_graph(sun_lattice* L, const GraphKey& key, cudaGraphExec_t* out);
sun_status check_wave_timeouts(sun_lattice* L);
// advance a lattice's heatbath step counter and history slot on stream s
sun_status launch_bump(sun::DevState* st, uint32_t hb_steps, uint32_t slots, cudaStream_t s);

// A slab of a lattice cut into t-slabs: its interior t-slices [1, 1 + thickness)
// are slices [t_start, t_start + thickness) of the whole lattice (nt_global slices).
struct SlabSpec {
  int t_start, thickness, nt_global;
};

// sun_lattice_create, with a slab's place in the whole lattice when slab != NULL
sun_status create_lattice(sun_lattice** out, int nc, const int dims[4], double beta, int hot_start, uint64_t seed,
                          const sun_options* opt_in, const SlabSpec* slab);

}  // namespace sun_api
