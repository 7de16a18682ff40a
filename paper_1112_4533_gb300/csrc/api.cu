// api.cu -- C ABI of the SU(Nc) link-sweep library (declared in include/sun.h).
//
// Owns the lattice handle: device memory layout, the chessboard schedule of
// Sec. 3 of Cardoso & Bicudo (arXiv:1112.4533) -- per step, directions
// mu = 0..3 each as an even then an odd pass --, CUDA-graph capture of one
// sweep, deterministic observable reductions and the canonical FP64
// import/export path.
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

namespace {

thread_local std::string g_last_error;

sun_status fail(sun_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

#define SUN_CUDA(call)                                                                             \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess)                                                                         \
      return fail(SUN_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                  __LINE__);                                                                       \
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

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

const sun::Ops* find_ops(int nc, int storage, int precision) {
  switch (nc) {
    case 2: return sun::ops_su2(storage, precision);
    case 3: return sun::ops_su3(storage, precision);
    case 4: return sun::ops_su4(storage, precision);
    case 5: return sun::ops_su5(storage, precision);
    case 6: return sun::ops_su6(storage, precision);
    default: return nullptr;
  }
}

int default_storage(int nc) { return nc == 2 ? 4 : (nc == 3 ? 12 : 2 * nc * nc); }

sun_status check_dims(const int* dims) {
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

Plan make_plan(int nc, const int* dims, int link_bytes) {
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

__global__ void bump_kernel(sun::DevState* st, uint32_t hb_steps, uint32_t slots) {
  st->hb_step += hb_steps;
  st->slot += slots;
}

struct GraphKey {
  int n_hb, n_or, reunit, plaq, poly;
  int sweeps = 1;  // sweeps captured in the graph
  bool operator<(const GraphKey& o) const {
    return std::tie(n_hb, n_or, reunit, plaq, poly, sweeps) <
           std::tie(o.n_hb, o.n_or, o.reunit, o.plaq, o.poly, o.sweeps);
  }
};

}  // namespace

namespace sun {
void set_last_error_message(const char* msg) { g_last_error = msg ? msg : ""; }
}  // namespace sun

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
  Plan plan{};
  const sun::Ops* ops = nullptr;
  sun::Ctx ctx{};
  double* results = nullptr;
  double* hist = nullptr;
  double* staging = nullptr;
  double host_results[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // pageable: creating a lattice pins nothing
  std::map<GraphKey, cudaGraphExec_t> graphs;
};

namespace {

sun_status set_device(const sun_lattice* L) {
  SUN_CUDA(cudaSetDevice(L->device));
  return SUN_OK;
}

void drop_graphs(sun_lattice* L) {
  for (auto& kv : L->graphs) cudaGraphExecDestroy(kv.second);
  L->graphs.clear();
}

sun::Ctx ctx_on(const sun_lattice* L, cudaStream_t s) {
  sun::Ctx c = L->ctx;
  c.stream = s;
  c.beta = L->beta;
  return c;
}

sun_status check_launch(cudaError_t e, const char* what) {
  if (e != cudaSuccess) return fail(SUN_ERR_CUDA, "launch of %s failed: %s", what, cudaGetErrorString(e));
  return SUN_OK;
}

// The eight passes of one step (mu = 0..3 x even, odd) on the lattice of c;
// with variant bit 8 each direction's pair is one wavefront launch.
sun_status enqueue_step(const sun::Ops* ops, const sun::Ctx& c, int mode, uint32_t step_offset, uint32_t mod,
                        uint32_t rem) {
  const char* what = mode == SUN_HEATBATH ? "heatbath pass" : "overrelaxation pass";
  for (int mu = 0; mu < 4; ++mu) {
    if ((c.variant & 8) && ops->pass_pair) {
      SUN_TRY(check_launch(ops->pass_pair(c, mode, mu, step_offset, mod, rem), what));
    } else {
      for (int p = 0; p < 2; ++p) SUN_TRY(check_launch(ops->pass(c, mode, mu, p, step_offset, mod, rem), what));
    }
  }
  return SUN_OK;
}

// Enqueue one sweep on stream s.  hist_mode: observables go to the history slot
// held in device state, which is advanced at the end of the sweep.
sun_status enqueue_sweep(sun_lattice* L, cudaStream_t s, int n_hb, int n_or, bool reunit, bool plaq,
                         bool poly, bool hist_mode) {
  const sun::Ctx c = ctx_on(L, s);
  const int n_steps = n_hb + n_or;
  // reunit_mode 1: every link of the last step re-unitarized in the update kernel;
  // reunit_mode 2: runs of 32 links spread over the steps (run r in step r mod n_steps)
  const bool fused = reunit && L->reunit_mode != 0 && n_steps > 0;
  for (int step = 0; step < n_steps; ++step) {
    const bool hb = step < n_hb;
    uint32_t mod = 0, rem = 0;
    if (fused && L->reunit_mode == 1 && step == n_steps - 1) mod = 1;
    if (fused && L->reunit_mode == 2) {
      mod = uint32_t(n_steps);
      rem = uint32_t(step);
    }
    SUN_TRY(enqueue_step(L->ops, c, hb ? SUN_HEATBATH : SUN_OVERRELAX, hb ? uint32_t(step) : 0u, mod, rem));
  }
  if (reunit && !fused) SUN_TRY(check_launch(L->ops->reunit(c), "reunitarization"));
  const uint32_t* slot = hist_mode ? &L->ctx.state->slot : nullptr;
  if (plaq) SUN_TRY(check_launch(L->ops->plaquette(c, hist_mode ? L->hist : L->results, slot, kHistCap), "plaquette"));
  if (poly)
    SUN_TRY(check_launch(L->ops->polyakov(c, hist_mode ? L->hist + kHistCap : L->results + 2, slot, kHistCap),
                         "polyakov"));
  if (n_hb > 0 || hist_mode) {
    bump_kernel<<<1, 1, 0, s>>>(L->ctx.state, uint32_t(n_hb), hist_mode ? 1u : 0u);
    SUN_TRY(check_launch(cudaGetLastError(), "step counter"));
  }
  return SUN_OK;
}

bool reunit_due(const sun_lattice* L, uint64_t sweep_index) {
  return L->reunit_every > 0 && ((sweep_index + 1) % uint64_t(L->reunit_every)) == 0;
}

sun_status get_graph(sun_lattice* L, const GraphKey& key, cudaGraphExec_t* out) {
  auto it = L->graphs.find(key);
  if (it != L->graphs.end()) {
    *out = it->second;
    return SUN_OK;
  }
  SUN_CUDA(cudaStreamBeginCapture(L->capture_stream, cudaStreamCaptureModeThreadLocal));
  sun_status st = SUN_OK;
  for (int k = 0; k < key.sweeps && st == SUN_OK; ++k)
    st = enqueue_sweep(L, L->capture_stream, key.n_hb, key.n_or, key.reunit != 0, key.plaq != 0, key.poly != 0, true);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(L->capture_stream, &g);
  if (st != SUN_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return fail(SUN_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(SUN_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
  L->graphs[key] = exec;
  *out = exec;
  return SUN_OK;
}

// Waits of wavefront launches that gave up (sync word 0, counted on the device):
// report and clear them.  Call after the lattice's stream has synchronised.
sun_status check_wave_timeouts(sun_lattice* L) {
  if (!(L->ctx.variant & 8) || !L->ops->pass_pair) return SUN_OK;
  uint32_t n = 0;
  SUN_CUDA(cudaMemcpyAsync(&n, L->ctx.wave, sizeof(uint32_t), cudaMemcpyDeviceToHost, L->stream));
  SUN_CUDA(cudaStreamSynchronize(L->stream));
  if (n == 0) return SUN_OK;
  SUN_CUDA(cudaMemsetAsync(L->ctx.wave, 0, sizeof(uint32_t), L->stream));
  SUN_CUDA(cudaStreamSynchronize(L->stream));
  return fail(SUN_ERR_TIMEOUT, "%u wavefront waits gave up after 2 s; the links updated since are not valid", n);
}

sun_status read_results(sun_lattice* L, int count) {
  SUN_CUDA(cudaMemcpyAsync(L->host_results, L->results, count * sizeof(double), cudaMemcpyDeviceToHost, L->stream));
  SUN_CUDA(cudaStreamSynchronize(L->stream));
  return SUN_OK;
}

}  // namespace

extern "C" {

int sun_abi_version(void) { return SUN_ABI_VERSION; }

void sun_options_init(sun_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->precision = 32;
  opt->storage = 0;
  opt->reunit_every = 1;
  opt->block_threads = 0;
  opt->stream = nullptr;
  opt->device_buf = nullptr;
  opt->device_buf_bytes = 0;
  opt->use_graphs = 1;
  opt->graph_sweeps = 0;
  opt->variant = 0;
  opt->reunit_mode = 0;
  opt->wave_lag = 0;
  opt->wave_skip_units = 0;
}

const char* sun_status_string(sun_status s) {
  switch (s) {
    case SUN_OK: return "ok";
    case SUN_ERR_ARG: return "invalid argument";
    case SUN_ERR_OOM: return "out of device memory";
    case SUN_ERR_CUDA: return "CUDA error";
    case SUN_ERR_TIMEOUT: return "device wait timed out";
    case SUN_ERR_UNSUPPORTED: return "unsupported combination";
    case SUN_ERR_STATE: return "invalid state";
  }
  return "unknown status";
}

const char* sun_last_error(void) { return g_last_error.c_str(); }

static sun_status resolve(int nc, const int* dims, const sun_options* opt_in, sun_options* opt, const sun::Ops** ops) {
  if (opt_in)
    *opt = *opt_in;
  else
    sun_options_init(opt);
  if (nc < 2) return fail(SUN_ERR_ARG, "nc = %d must be >= 2", nc);
  SUN_TRY(check_dims(dims));
  if (opt->precision != 32 && opt->precision != 64)
    return fail(SUN_ERR_ARG, "precision = %d must be 32 or 64", opt->precision);
  if (opt->storage == 0) opt->storage = default_storage(nc);
  if (opt->reunit_every < 0) return fail(SUN_ERR_ARG, "reunit_every must be >= 0");
  if (opt->block_threads == 0) opt->block_threads = 128;
  if (opt->variant < 0 || opt->variant > 31) return fail(SUN_ERR_ARG, "variant = %d must be in 0..31", opt->variant);
  if (opt->wave_lag < 0) return fail(SUN_ERR_ARG, "wave_lag = %d must be >= 0", opt->wave_lag);
  if (opt->wave_lag == 0) opt->wave_lag = kDefaultWaveLag;
  if (opt->wave_skip_units < 0) return fail(SUN_ERR_ARG, "wave_skip_units must be >= 0");
  if (opt->graph_sweeps < 0 || opt->graph_sweeps > 64) return fail(SUN_ERR_ARG, "graph_sweeps must be in 0..64");
  if (opt->graph_sweeps == 0) opt->graph_sweeps = 1;
  if (opt->reunit_mode < 0 || opt->reunit_mode > 2)
    return fail(SUN_ERR_ARG, "reunit_mode = %d must be 0, 1 or 2", opt->reunit_mode);
  if (opt->block_threads < 32 || opt->block_threads > 256 || (opt->block_threads & 31))
    return fail(SUN_ERR_ARG, "block_threads = %d must be a multiple of 32 in [32, 256]", opt->block_threads);
  *ops = find_ops(nc, opt->storage, opt->precision);
  if (!*ops)
    return fail(SUN_ERR_UNSUPPORTED, "no kernels for nc = %d, storage = %d, precision = %d (built: nc 2..6)", nc,
                opt->storage, opt->precision);
  if (opt->reunit_mode != 0 && !(*ops)->fused_reunit)
    return fail(SUN_ERR_UNSUPPORTED, "reunit_mode %d is not built for nc = %d at precision %d", opt->reunit_mode, nc,
                opt->precision);
  return SUN_OK;
}

size_t sun_footprint_bytes(int nc, const int dims[4], const sun_options* opt_in) {
  sun_options opt;
  const sun::Ops* ops = nullptr;
  if (resolve(nc, dims, opt_in, &opt, &ops) != SUN_OK) return 0;
  return make_plan(nc, dims, ops->link_bytes).total;
}

}  // extern "C"

namespace {
// A slab of a lattice cut into t-slabs: its interior t-slices [1, 1 + thickness)
// are slices [t_start, t_start + thickness) of the whole lattice (nt_global slices).
struct SlabSpec {
  int t_start, thickness, nt_global;
};
}  // namespace

static sun_status create_lattice(sun_lattice** out, int nc, const int dims[4], double beta, int hot_start,
                                 uint64_t seed, const sun_options* opt_in, const SlabSpec* slab) {
  if (!out) return fail(SUN_ERR_ARG, "out is NULL");
  *out = nullptr;
  sun_options opt;
  const sun::Ops* ops = nullptr;
  SUN_TRY(resolve(nc, dims, opt_in, &opt, &ops));
  if (!(beta >= 0.0)) return fail(SUN_ERR_ARG, "beta must be >= 0");

  sun_lattice* L = new sun_lattice();
  L->nc = nc;
  L->precision = opt.precision;
  L->storage = opt.storage;
  for (int m = 0; m < 4; ++m) L->dims[m] = dims[m];
  L->beta = beta;
  L->seed = seed;
  L->reunit_every = opt.reunit_every;
  L->reunit_mode = opt.reunit_mode;
  L->block_threads = opt.block_threads;
  L->use_graphs = opt.use_graphs;
  L->graph_sweeps = opt.graph_sweeps;
  L->ops = ops;
  L->plan = make_plan(nc, dims, ops->link_bytes);

  auto cleanup = [&](sun_status s) {
    sun_lattice_destroy(L);
    return s;
  };
  if (cudaGetDevice(&L->device) != cudaSuccess) return cleanup(fail(SUN_ERR_CUDA, "no CUDA device"));
  if (opt.device_buf) {
    if (reinterpret_cast<uintptr_t>(opt.device_buf) % kAlign)
      return cleanup(fail(SUN_ERR_ARG, "device_buf must be %zu-byte aligned", kAlign));
    if (opt.device_buf_bytes < L->plan.total)
      return cleanup(fail(SUN_ERR_OOM, "device_buf holds %zu bytes, lattice needs %zu", opt.device_buf_bytes,
                          L->plan.total));
    L->base = static_cast<char*>(opt.device_buf);
    L->own_mem = false;
  } else {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, L->plan.total);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return cleanup(fail(SUN_ERR_OOM, "cudaMalloc(%zu) failed: %s", L->plan.total, cudaGetErrorString(e)));
    }
    L->base = static_cast<char*>(p);
    L->own_mem = true;
  }
  if (opt.stream) {
    L->stream = static_cast<cudaStream_t>(opt.stream);
    L->own_stream = false;
  } else {
    if (cudaStreamCreateWithFlags(&L->stream, cudaStreamNonBlocking) != cudaSuccess)
      return cleanup(fail(SUN_ERR_CUDA, "stream creation failed"));
    L->own_stream = true;
  }
  if (cudaStreamCreateWithFlags(&L->capture_stream, cudaStreamNonBlocking) != cudaSuccess)
    return cleanup(fail(SUN_ERR_CUDA, "capture stream creation failed"));

  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, L->device);
  sun::Geom g;
  g.nx = dims[0];
  g.ny = dims[1];
  g.nz = dims[2];
  g.nt = dims[3];
  g.nxh = dims[0] / 2;
  g.V = int64_t(dims[0]) * dims[1] * dims[2] * dims[3];
  g.Vh = g.V / 2;
  g.stride[0] = 1;
  g.stride[1] = dims[0];
  g.stride[2] = int64_t(dims[0]) * dims[1];
  g.stride[3] = int64_t(dims[0]) * dims[1] * dims[2];
  g.div_nxh = sun::make_fastdiv(uint32_t(g.nxh));
  g.div_ny = sun::make_fastdiv(uint32_t(g.ny));
  g.div_nz = sun::make_fastdiv(uint32_t(g.nz));
  g.div_nx = sun::make_fastdiv(uint32_t(g.nx));

  sun::Ctx& c = L->ctx;
  c.links = L->base + L->plan.links_off;
  c.block_bytes = g.Vh * ops->link_bytes;
  c.g = g;
  c.beta = beta;
  c.seed = seed;
  c.nc = nc;
  c.state = reinterpret_cast<sun::DevState*>(L->base + L->plan.state_off);
  c.partials = reinterpret_cast<double*>(L->base + L->plan.partials_off);
  c.stream = L->stream;
  c.block_threads = L->block_threads;
  c.variant = opt.variant;
  c.wave = reinterpret_cast<uint32_t*>(L->base + L->plan.wave_off);
  c.wave_lag = opt.wave_lag;
  c.wave_skip = uint32_t(opt.wave_skip_units);
  c.h_begin = 0;
  c.h_end = g.Vh;
  c.lex_offset = 0u;
  c.v_global = uint32_t(g.V);
  if (slab) {
    const int64_t vs = int64_t(dims[0]) * dims[1] * dims[2];
    c.h_begin = vs / 2;
    c.h_end = vs / 2 * (1 + slab->thickness);
    c.lex_offset = uint32_t(int64_t((slab->t_start - 1 + slab->nt_global) % slab->nt_global) * vs);
    c.v_global = uint32_t(vs * slab->nt_global);
  }
  c.obs_stride = 1;
  c.obs_offset = 0;
  int rb = 2 * (sms > 0 ? sms : 132);
  c.reduce_blocks = rb > sun::kMaxReduceBlocks ? sun::kMaxReduceBlocks : rb;
  L->results = reinterpret_cast<double*>(L->base + L->plan.results_off);
  L->hist = reinterpret_cast<double*>(L->base + L->plan.hist_off);
  L->staging = reinterpret_cast<double*>(L->base + L->plan.staging_off);

  if (cudaMemsetAsync(c.state, 0, sizeof(sun::DevState), L->stream) != cudaSuccess ||
      cudaMemsetAsync(c.wave, 0, (sun::kWaveSyncWords + size_t(dims[3])) * sizeof(uint32_t), L->stream) != cudaSuccess)
    return cleanup(fail(SUN_ERR_CUDA, "state reset failed"));
  sun_status st = check_launch(ops->init(ctx_on(L, L->stream), hot_start ? 1 : 0), "init");
  if (st != SUN_OK) return cleanup(st);
  *out = L;
  return SUN_OK;
}

extern "C" {

sun_status sun_lattice_create(sun_lattice** out, int nc, const int dims[4], double beta, int hot_start,
                              uint64_t seed, const sun_options* opt_in) {
  return create_lattice(out, nc, dims, beta, hot_start, seed, opt_in, nullptr);
}

void sun_lattice_destroy(sun_lattice* L) {
  if (!L) return;
  cudaSetDevice(L->device);
  if (L->stream) cudaStreamSynchronize(L->stream);
  drop_graphs(L);
  if (L->capture_stream) cudaStreamDestroy(L->capture_stream);
  if (L->own_stream && L->stream) cudaStreamDestroy(L->stream);
  if (L->own_mem && L->base) cudaFree(L->base);
  delete L;
}

sun_status sun_update_pass(sun_lattice* L, int mode, int mu, int parity) {
  if (!L) return fail(SUN_ERR_ARG, "lattice is NULL");
  if (mode != SUN_HEATBATH && mode != SUN_OVERRELAX) return fail(SUN_ERR_ARG, "mode must be 0 or 1");
  if (mu < 0 || mu > 3) return fail(SUN_ERR_ARG, "mu must be in 0..3");
  if (parity != 0 && parity != 1) return fail(SUN_ERR_ARG, "parity must be 0 or 1");
  SUN_TRY(set_device(L));
  return check_launch(L->ops->pass(ctx_on(L, L->stream), mode, mu, parity, 0u, 0u, 0u), "update pass");
}

sun_status sun_sweep(sun_lattice* L, int n_hb, int n_or) {
  if (!L) return fail(SUN_ERR_ARG, "lattice is NULL");
  if (n_hb < 0 || n_or < 0) return fail(SUN_ERR_ARG, "step counts must be >= 0");
  SUN_TRY(set_device(L));
  SUN_TRY(enqueue_sweep(L, L->stream, n_hb, n_or, reunit_due(L, L->sweeps_done), false, false, false));
  L->sweeps_done++;
  return SUN_OK;
}

sun_status sun_run(sun_lattice* L, int n_sweeps, int n_hb, int n_or, double* plaq_hist, double* poly_hist) {
  if (!L) return fail(SUN_ERR_ARG, "lattice is NULL");
  if (n_sweeps < 0 || n_hb < 0 || n_or < 0) return fail(SUN_ERR_ARG, "counts must be >= 0");
  SUN_TRY(set_device(L));
  const bool plaq = plaq_hist != nullptr, poly = poly_hist != nullptr;
  for (int done = 0; done < n_sweeps;) {
    const int chunk = (n_sweeps - done) < kHistCap ? (n_sweeps - done) : kHistCap;
    SUN_CUDA(cudaMemsetAsync(&L->ctx.state->slot, 0, sizeof(uint32_t), L->stream));
    for (int k = 0; k < chunk;) {
      const bool reunit = reunit_due(L, L->sweeps_done);
      // graph_sweeps sweeps per graph launch where every sweep re-unitarizes alike
      const int per = (L->reunit_every <= 1 && chunk - k >= L->graph_sweeps) ? L->graph_sweeps : 1;
      if (L->use_graphs) {
        cudaGraphExec_t exec = nullptr;
        GraphKey key{n_hb, n_or, reunit ? 1 : 0, plaq ? 1 : 0, poly ? 1 : 0};
        key.sweeps = per;
        SUN_TRY(get_graph(L, key, &exec));
        SUN_CUDA(cudaGraphLaunch(exec, L->stream));
      } else {
        for (int q = 0; q < per; ++q) SUN_TRY(enqueue_sweep(L, L->stream, n_hb, n_or, reunit, plaq, poly, true));
      }
      L->sweeps_done += uint64_t(per);
      k += per;
    }
    if (plaq)
      SUN_CUDA(cudaMemcpyAsync(plaq_hist + done, L->hist, chunk * sizeof(double), cudaMemcpyDeviceToHost, L->stream));
    if (poly)
      SUN_CUDA(cudaMemcpyAsync(poly_hist + 2 * done, L->hist + kHistCap, 2 * chunk * sizeof(double),
                               cudaMemcpyDeviceToHost, L->stream));
    done += chunk;
  }
  SUN_CUDA(cudaStreamSynchronize(L->stream));
  return check_wave_timeouts(L);
}

sun_status sun_reunitarize(sun_lattice* L) {
  if (!L) return fail(SUN_ERR_ARG, "lattice is NULL");
  SUN_TRY(set_device(L));
  return check_launch(L->ops->reunit(ctx_on(L, L->stream)), "reunitarization");
}

sun_status sun_plaquette(sun_lattice* L, double* out) {
  if (!L || !out) return fail(SUN_ERR_ARG, "NULL argument");
  SUN_TRY(set_device(L));
  SUN_TRY(check_launch(L->ops->plaquette(ctx_on(L, L->stream), L->results, nullptr, 1), "plaquette"));
  SUN_TRY(read_results(L, 1));
  *out = L->host_results[0];
  return SUN_OK;
}

sun_status sun_polyakov_loop(sun_lattice* L, double* re, double* im) {
  if (!L || !re || !im) return fail(SUN_ERR_ARG, "NULL argument");
  SUN_TRY(set_device(L));
  SUN_TRY(check_launch(L->ops->polyakov(ctx_on(L, L->stream), L->results + 2, nullptr, 1), "polyakov"));
  SUN_TRY(read_results(L, 4));
  *re = L->host_results[2];
  *im = L->host_results[3];
  return SUN_OK;
}

static size_t canonical_doubles(const sun_lattice* L) { return size_t(8) * L->nc * L->nc * size_t(L->ctx.g.V); }

// Device address of page-locked host memory (mapped into the device address
// space), or NULL for pageable memory.  Conversion kernels then read or write
// the host buffer directly; otherwise they go through the staging buffer.
static double* mapped_host(const void* host) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type == cudaMemoryTypeHost && a.devicePointer) return static_cast<double*>(a.devicePointer);
  return nullptr;
}

sun_status sun_export_links(sun_lattice* L, double* host, size_t n) {
  if (!L || !host) return fail(SUN_ERR_ARG, "NULL argument");
  if (n != canonical_doubles(L)) return fail(SUN_ERR_ARG, "host buffer holds %zu doubles, need %zu", n, canonical_doubles(L));
  if (reinterpret_cast<uintptr_t>(host) % 16) return fail(SUN_ERR_ARG, "host buffer must be 16-byte aligned");
  SUN_TRY(set_device(L));
  const sun::Ctx c = ctx_on(L, L->stream);
  const int64_t total = 4 * L->ctx.g.V, per = 2 * L->nc * L->nc;
  if (double* dev = mapped_host(host)) {
    SUN_TRY(check_launch(L->ops->export_links(c, dev, 0, total), "export"));
  } else {
    for (int64_t first = 0; first < total; first += L->plan.staging_links) {
      const int64_t cnt = (total - first) < L->plan.staging_links ? (total - first) : L->plan.staging_links;
      SUN_TRY(check_launch(L->ops->export_links(c, L->staging, first, cnt), "export"));
      SUN_CUDA(cudaMemcpyAsync(host + first * per, L->staging, size_t(cnt * per) * sizeof(double),
                               cudaMemcpyDeviceToHost, L->stream));
    }
  }
  SUN_CUDA(cudaStreamSynchronize(L->stream));
  return SUN_OK;
}

sun_status sun_import_links(sun_lattice* L, const double* host, size_t n) {
  if (!L || !host) return fail(SUN_ERR_ARG, "NULL argument");
  if (n != canonical_doubles(L)) return fail(SUN_ERR_ARG, "host buffer holds %zu doubles, need %zu", n, canonical_doubles(L));
  if (reinterpret_cast<uintptr_t>(host) % 16) return fail(SUN_ERR_ARG, "host buffer must be 16-byte aligned");
  SUN_TRY(set_device(L));
  const sun::Ctx c = ctx_on(L, L->stream);
  const int64_t total = 4 * L->ctx.g.V, per = 2 * L->nc * L->nc;
  if (const double* dev = mapped_host(host)) {
    SUN_TRY(check_launch(L->ops->import_links(c, dev, 0, total), "import"));
  } else {
    for (int64_t first = 0; first < total; first += L->plan.staging_links) {
      const int64_t cnt = (total - first) < L->plan.staging_links ? (total - first) : L->plan.staging_links;
      SUN_CUDA(cudaMemcpyAsync(L->staging, host + first * per, size_t(cnt * per) * sizeof(double),
                               cudaMemcpyHostToDevice, L->stream));
      SUN_TRY(check_launch(L->ops->import_links(c, L->staging, first, cnt), "import"));
    }
  }
  SUN_CUDA(cudaStreamSynchronize(L->stream));
  return SUN_OK;
}

sun_status sun_check_links(sun_lattice* L, double* max_unitarity_dev, double* max_det_dev, uint64_t* nonfinite) {
  if (!L || !max_unitarity_dev || !max_det_dev || !nonfinite) return fail(SUN_ERR_ARG, "NULL argument");
  SUN_TRY(set_device(L));
  // results[4..6] hold the kernel's three words
  unsigned long long* out = reinterpret_cast<unsigned long long*>(L->results + 4);
  SUN_TRY(check_launch(L->ops->check_links(ctx_on(L, L->stream), out), "link check"));
  SUN_CUDA(cudaMemcpyAsync(L->host_results + 4, out, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                           L->stream));
  SUN_CUDA(cudaStreamSynchronize(L->stream));
  unsigned long long w[3];
  std::memcpy(w, L->host_results + 4, sizeof(w));
  std::memcpy(max_unitarity_dev, &w[0], sizeof(double));
  std::memcpy(max_det_dev, &w[1], sizeof(double));
  *nonfinite = w[2];
  return SUN_OK;
}

// The compact host format (stored rows in the storage precision): 4V x link_bytes.
static sun_status copy_stored(sun_lattice* L, void* host, size_t bytes, bool to_host) {
  if (!L || !host) return fail(SUN_ERR_ARG, "NULL argument");
  if (bytes != L->plan.links_bytes)
    return fail(SUN_ERR_ARG, "host buffer holds %zu bytes, need %zu", bytes, L->plan.links_bytes);
  if (reinterpret_cast<uintptr_t>(host) % 16) return fail(SUN_ERR_ARG, "host buffer must be 16-byte aligned");
  SUN_TRY(set_device(L));
  const sun::Ctx c = ctx_on(L, L->stream);
  const int64_t total = 4 * L->ctx.g.V, lb = L->ops->link_bytes;
  char* h = static_cast<char*>(host);
  if (double* dev = mapped_host(host)) {
    SUN_TRY(check_launch(to_host ? L->ops->export_stored(c, dev, 0, total) : L->ops->import_stored(c, dev, 0, total),
                         to_host ? "export" : "import"));
  } else {
    for (int64_t first = 0; first < total; first += L->plan.staging_links) {
      const int64_t cnt = std::min<int64_t>(total - first, L->plan.staging_links);
      if (to_host) {
        SUN_TRY(check_launch(L->ops->export_stored(c, L->staging, first, cnt), "export"));
        SUN_CUDA(cudaMemcpyAsync(h + first * lb, L->staging, size_t(cnt * lb), cudaMemcpyDeviceToHost, L->stream));
      } else {
        SUN_CUDA(cudaMemcpyAsync(L->staging, h + first * lb, size_t(cnt * lb), cudaMemcpyHostToDevice, L->stream));
        SUN_TRY(check_launch(L->ops->import_stored(c, L->staging, first, cnt), "import"));
      }
    }
  }
  SUN_CUDA(cudaStreamSynchronize(L->stream));
  return SUN_OK;
}

sun_status sun_export_stored(sun_lattice* L, void* host, size_t bytes) { return copy_stored(L, host, bytes, true); }

sun_status sun_import_stored(sun_lattice* L, const void* host, size_t bytes) {
  return copy_stored(L, const_cast<void*>(host), bytes, false);
}

sun_status sun_get_heatbath_step(sun_lattice* L, uint64_t* step) {
  if (!L || !step) return fail(SUN_ERR_ARG, "NULL argument");
  SUN_TRY(set_device(L));
  uint32_t v = 0;
  SUN_CUDA(cudaMemcpyAsync(L->host_results, &L->ctx.state->hb_step, sizeof(uint32_t), cudaMemcpyDeviceToHost, L->stream));
  SUN_CUDA(cudaStreamSynchronize(L->stream));
  std::memcpy(&v, L->host_results, sizeof(v));
  *step = v;
  return SUN_OK;
}

sun_status sun_set_heatbath_step(sun_lattice* L, uint64_t step) {
  if (!L) return fail(SUN_ERR_ARG, "lattice is NULL");
  if (step > 0xffffffffull) return fail(SUN_ERR_ARG, "heatbath step counter is 32-bit");
  SUN_TRY(set_device(L));
  const uint32_t v = uint32_t(step);
  SUN_CUDA(cudaStreamSynchronize(L->stream));
  std::memcpy(L->host_results, &v, sizeof(v));
  SUN_CUDA(cudaMemcpyAsync(&L->ctx.state->hb_step, L->host_results, sizeof(uint32_t), cudaMemcpyHostToDevice, L->stream));
  SUN_CUDA(cudaStreamSynchronize(L->stream));
  return SUN_OK;
}

sun_status sun_set_beta(sun_lattice* L, double beta) {
  if (!L) return fail(SUN_ERR_ARG, "lattice is NULL");
  if (!(beta >= 0.0)) return fail(SUN_ERR_ARG, "beta must be >= 0");
  if (beta != L->beta) {
    SUN_TRY(set_device(L));
    SUN_CUDA(cudaStreamSynchronize(L->stream));
    drop_graphs(L);
    L->beta = beta;
  }
  return SUN_OK;
}

sun_status sun_synchronize(sun_lattice* L) {
  if (!L) return fail(SUN_ERR_ARG, "lattice is NULL");
  SUN_TRY(set_device(L));
  SUN_CUDA(cudaStreamSynchronize(L->stream));
  return check_wave_timeouts(L);
}

// ---------------------------------------------------------------------------
// Configuration files
// ---------------------------------------------------------------------------
static_assert(sizeof(sun_config_header) == 120, "configuration header layout");
static const char kConfigMagic[8] = {'S', 'U', 'N', 'C', 'F', 'G', '0', '1'};

static uint64_t fnv1a_words(uint64_t h, const void* data, size_t bytes) {
  const unsigned char* p = static_cast<const unsigned char*>(data);
  for (size_t i = 0; i + 8 <= bytes; i += 8) {
    uint64_t w = 0;
    for (int b = 7; b >= 0; --b) w = (w << 8) | p[i + size_t(b)];  // little-endian word
    h ^= w;
    h *= 1099511628211ull;
  }
  return h;
}
static const uint64_t kFnvBasis = 14695981039346656037ull;

static int stored_rows(int nc, int storage) { return storage / (2 * nc); }

namespace {
struct File {
  FILE* f = nullptr;
  ~File() {
    if (f) fclose(f);
  }
};
}  // namespace

sun_status sun_read_config_header(const char* path, int verify, sun_config_header* out) {
  if (!path || !out) return fail(SUN_ERR_ARG, "NULL argument");
  File F;
  F.f = fopen(path, "rb");
  if (!F.f) return fail(SUN_ERR_ARG, "cannot open %s", path);
  char magic[8];
  sun_config_header h;
  if (fread(magic, 1, 8, F.f) != 8 || std::memcmp(magic, kConfigMagic, 8) != 0)
    return fail(SUN_ERR_ARG, "%s is not a configuration file (magic)", path);
  if (fread(&h, sizeof(h), 1, F.f) != 1) return fail(SUN_ERR_ARG, "%s: truncated header", path);
  if (h.version != 1) return fail(SUN_ERR_ARG, "%s: unknown version %u", path, h.version);
  if (h.nc < 2 || (h.precision != 32 && h.precision != 64) || h.storage < 2 * h.nc ||
      h.storage % (2 * h.nc) != 0 || stored_rows(h.nc, h.storage) > h.nc)
    return fail(SUN_ERR_ARG, "%s: inconsistent header", path);
  SUN_TRY(check_dims(h.dims));
  const uint64_t V = uint64_t(h.dims[0]) * h.dims[1] * h.dims[2] * h.dims[3];
  const uint64_t want = 4 * V * uint64_t(stored_rows(h.nc, h.storage)) * uint64_t(h.nc) * 2 * uint64_t(h.precision / 8);
  if (h.payload_bytes != want) return fail(SUN_ERR_ARG, "%s: payload size does not match the header", path);
  if (verify) {
    std::vector<unsigned char> buf(size_t(8) << 20);
    uint64_t sum = kFnvBasis, got = 0;
    for (;;) {
      const size_t n = fread(buf.data(), 1, buf.size(), F.f);
      if (n == 0) break;
      if (n % 8 != 0 && got + n != h.payload_bytes) return fail(SUN_ERR_ARG, "%s: short read", path);
      sum = fnv1a_words(sum, buf.data(), n);
      got += n;
    }
    if (got != h.payload_bytes) return fail(SUN_ERR_ARG, "%s: payload is %llu bytes, header says %llu", path,
                                            (unsigned long long)got, (unsigned long long)h.payload_bytes);
    if (sum != h.checksum) return fail(SUN_ERR_ARG, "%s: checksum mismatch", path);
  }
  *out = h;
  return SUN_OK;
}

sun_status sun_save_config(sun_lattice* L, const char* path) {
  if (!L || !path) return fail(SUN_ERR_ARG, "NULL argument");
  SUN_TRY(set_device(L));
  uint64_t step = 0;
  SUN_TRY(sun_get_heatbath_step(L, &step));
  sun_config_header h;
  std::memset(&h, 0, sizeof(h));
  h.version = 1;
  h.nc = L->nc;
  h.precision = L->precision;
  h.storage = L->storage;
  for (int m = 0; m < 4; ++m) h.dims[m] = L->dims[m];
  h.beta = L->beta;
  h.seed = L->seed;
  h.heatbath_step = step;
  h.sweeps_done = L->sweeps_done;
  const int64_t total = 4 * L->ctx.g.V;
  // rows storage / (2 Nc) of Nc complex values in the storage precision = the stored link bytes
  h.payload_bytes = uint64_t(total) * uint64_t(L->ops->link_bytes);
  File F;
  F.f = fopen(path, "wb");
  if (!F.f) return fail(SUN_ERR_ARG, "cannot create %s", path);
  if (fwrite(kConfigMagic, 1, 8, F.f) != 8 || fwrite(&h, sizeof(h), 1, F.f) != 1)
    return fail(SUN_ERR_ARG, "write to %s failed", path);
  const sun::Ctx c = ctx_on(L, L->stream);
  // the payload is the compact format: the stored rows in the storage precision
  const int64_t lb = L->ops->link_bytes;
  std::vector<unsigned char> out(size_t(L->plan.staging_links) * size_t(lb));
  uint64_t sum = kFnvBasis;
  for (int64_t first = 0; first < total; first += L->plan.staging_links) {
    const int64_t cnt = std::min<int64_t>(total - first, L->plan.staging_links);
    SUN_TRY(check_launch(L->ops->export_stored(c, L->staging, first, cnt), "export"));
    SUN_CUDA(cudaMemcpyAsync(out.data(), L->staging, size_t(cnt * lb), cudaMemcpyDeviceToHost, L->stream));
    SUN_CUDA(cudaStreamSynchronize(L->stream));
    const size_t nbytes = size_t(cnt * lb);
    sum = fnv1a_words(sum, out.data(), nbytes);
    if (fwrite(out.data(), 1, nbytes, F.f) != nbytes) return fail(SUN_ERR_ARG, "write to %s failed", path);
  }
  h.checksum = sum;
  if (fseek(F.f, 8, SEEK_SET) != 0 || fwrite(&h, sizeof(h), 1, F.f) != 1)
    return fail(SUN_ERR_ARG, "write to %s failed", path);
  if (fclose(F.f) != 0) {
    F.f = nullptr;
    return fail(SUN_ERR_ARG, "closing %s failed", path);
  }
  F.f = nullptr;
  return SUN_OK;
}

sun_status sun_load_config(sun_lattice* L, const char* path) {
  if (!L || !path) return fail(SUN_ERR_ARG, "NULL argument");
  sun_config_header h;
  SUN_TRY(sun_read_config_header(path, 1, &h));
  if (h.nc != L->nc || h.precision != L->precision || h.storage != L->storage)
    return fail(SUN_ERR_ARG, "%s holds nc %d, precision %d, storage %d; the lattice has %d, %d, %d", path, h.nc,
                h.precision, h.storage, L->nc, L->precision, L->storage);
  for (int m = 0; m < 4; ++m)
    if (h.dims[m] != L->dims[m]) return fail(SUN_ERR_ARG, "%s: lattice extents differ", path);
  if (!(h.beta >= 0.0)) return fail(SUN_ERR_ARG, "%s: beta < 0", path);
  SUN_TRY(set_device(L));
  File F;
  F.f = fopen(path, "rb");
  if (!F.f || fseek(F.f, 128, SEEK_SET) != 0) return fail(SUN_ERR_ARG, "cannot read %s", path);
  const int64_t total = 4 * L->ctx.g.V;
  const sun::Ctx c = ctx_on(L, L->stream);
  const int64_t lb = L->ops->link_bytes;
  std::vector<unsigned char> in(size_t(L->plan.staging_links) * size_t(lb));
  SUN_CUDA(cudaStreamSynchronize(L->stream));
  for (int64_t first = 0; first < total; first += L->plan.staging_links) {
    const int64_t cnt = std::min<int64_t>(total - first, L->plan.staging_links);
    const size_t nbytes = size_t(cnt * lb);
    if (fread(in.data(), 1, nbytes, F.f) != nbytes) return fail(SUN_ERR_ARG, "%s: short read", path);
    SUN_CUDA(cudaMemcpyAsync(L->staging, in.data(), nbytes, cudaMemcpyHostToDevice, L->stream));
    SUN_TRY(check_launch(L->ops->import_stored(c, L->staging, first, cnt), "import"));
    SUN_CUDA(cudaStreamSynchronize(L->stream));  // the host buffer is reused
  }
  // the chain state: graphs captured with the old seed or beta are dropped
  if (h.seed != L->seed || h.beta != L->beta) {
    drop_graphs(L);
    L->seed = h.seed;
    L->ctx.seed = h.seed;
    L->beta = h.beta;
  }
  L->sweeps_done = h.sweeps_done;
  return sun_set_heatbath_step(L, h.heatbath_step);
}

sun_status sun_get_info(const sun_lattice* L, sun_lattice_info* info) {
  if (!L || !info) return fail(SUN_ERR_ARG, "NULL argument");
  std::memset(info, 0, sizeof(*info));
  info->nc = L->nc;
  info->precision = L->precision;
  info->storage = L->storage;
  for (int m = 0; m < 4; ++m) info->dims[m] = L->dims[m];
  info->beta = L->beta;
  info->seed = L->seed;
  info->link_bytes = size_t(L->ops->link_bytes);
  info->links_bytes = L->plan.links_bytes;
  info->footprint = L->plan.total;
  info->links = L->ctx.links;
  info->stream = L->stream;
  return SUN_OK;
}

}  // extern "C"

// ===========================================================================
// Batches of chains
// ===========================================================================
namespace {

__global__ void batch_bump_kernel(sun::ChainDesc* chains, int n, uint32_t hb_steps) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < n) *chains[c].hb_step += hb_steps;
}

__global__ void slot_bump_kernel(uint32_t* slot) { *slot += 1u; }

struct BatchGroup {
  const sun::Ops* ops = nullptr;
  std::vector<sun_lattice*> members;  // chains packed into shared launches, then the large chains
  int n_small = 0;                    // members[0, n_small) are packed; the rest run their own launches
  int offset = 0;  // position of the first member in the create call order of the batch table
  std::vector<int> positions;  // create-call position of each member
  sun::ChainDesc* d_chains = nullptr;  // all members (packed ones first)
  uint32_t* d_start = nullptr;  // pass, reunit, plaquette, Polyakov, row-parallel pass tables, n_small+1 each
  double* d_partials = nullptr;
  int* d_pos = nullptr;
  sun::BatchCtx ctx{};
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
};

}  // namespace

struct sun_batch {
  int n = 0;
  int device = 0;
  std::vector<sun_lattice*> lattices;
  std::vector<BatchGroup> groups;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaStream_t capture_stream = nullptr;
  cudaEvent_t fork = nullptr;
  uint32_t* d_slot = nullptr;
  double* d_hist = nullptr;  // [cap][n] plaquette, then [cap][n][2] Polyakov (group-ordered columns)
  std::vector<double> h_hist;
  int hist_cap = 0;
  int reunit_every = 1, reunit_mode = 0;
  uint64_t sweeps_done = 0;
  int use_graphs = 1;
  int graph_sweeps = 1;  // sweeps per graph launch (from the first lattice's options)
  std::map<GraphKey, cudaGraphExec_t> graphs;
};

namespace {

// batch tables are stream-ordered allocations: creating and destroying a batch
// (as a server does whenever its set of chains changes) never synchronises the device
template <class T>
sun_status dev_alloc(T** p, size_t count, cudaStream_t s) {
  void* q = nullptr;
  if (cudaMallocAsync(&q, count * sizeof(T), s) != cudaSuccess) {
    cudaGetLastError();
    return fail(SUN_ERR_OOM, "cudaMallocAsync of %zu bytes for a batch table failed", count * sizeof(T));
  }
  *p = static_cast<T*>(q);
  return SUN_OK;
}

sun_status enqueue_batch_sweep(sun_batch* B, cudaStream_t s, int n_hb, int n_or, bool reunit, bool plaq, bool poly,
                               bool hist_mode) {
  const int n_steps = n_hb + n_or;
  const bool fused = reunit && B->reunit_mode != 0 && n_steps > 0;
  SUN_CUDA(cudaEventRecord(B->fork, s));
  for (auto& g : B->groups) {
    SUN_CUDA(cudaStreamWaitEvent(g.stream, B->fork, 0));
    sun::BatchCtx c = g.ctx;
    c.stream = g.stream;
    for (int step = 0; step < n_steps; ++step) {
      const bool hb = step < n_hb;
      uint32_t mod = 0, rem = 0;
      if (fused && B->reunit_mode == 1 && step == n_steps - 1) mod = 1;
      if (fused && B->reunit_mode == 2) {
        mod = uint32_t(n_steps);
        rem = uint32_t(step);
      }
      const int mode = hb ? SUN_HEATBATH : SUN_OVERRELAX;
      const uint32_t so = hb ? uint32_t(step) : 0u;
      if (g.n_small > 0)
        for (int mu = 0; mu < 4; ++mu)
          for (int p = 0; p < 2; ++p)
            SUN_TRY(check_launch(g.ops->batch_pass(c, mode, mu, p, so, mod, rem), "batched pass"));
      for (size_t k = size_t(g.n_small); k < g.members.size(); ++k)
        SUN_TRY(enqueue_step(g.ops, ctx_on(g.members[k], g.stream), mode, so, mod, rem));
    }
    const uint32_t* slot = hist_mode ? B->d_slot : nullptr;
    double* hist_p = B->d_hist;
    double* hist_l = B->d_hist + size_t(B->hist_cap) * B->n;
    if (g.n_small > 0) {
      if (reunit && !fused) SUN_TRY(check_launch(g.ops->batch_reunit(c), "batched reunitarization"));
      if (plaq) SUN_TRY(check_launch(g.ops->batch_plaquette(c, hist_p, slot, B->hist_cap, g.offset, B->n),
                                     "batched plaquette"));
      if (poly) SUN_TRY(check_launch(g.ops->batch_polyakov(c, hist_l, slot, B->hist_cap, g.offset, B->n),
                                     "batched polyakov"));
    }
    for (size_t k = size_t(g.n_small); k < g.members.size(); ++k) {
      sun::Ctx lc = ctx_on(g.members[k], g.stream);
      lc.obs_stride = B->n;
      lc.obs_offset = g.offset + int(k);
      if (reunit && !fused) SUN_TRY(check_launch(g.ops->reunit(lc), "reunitarization"));
      if (plaq) SUN_TRY(check_launch(g.ops->plaquette(lc, hist_p, slot, B->hist_cap), "plaquette"));
      if (poly) SUN_TRY(check_launch(g.ops->polyakov(lc, hist_l, slot, B->hist_cap), "polyakov"));
    }
    if (n_hb > 0) {
      const int all = int(g.members.size());
      batch_bump_kernel<<<unsigned((all + 127) / 128), 128, 0, g.stream>>>(g.d_chains, all, uint32_t(n_hb));
      SUN_TRY(check_launch(cudaGetLastError(), "batched step counter"));
    }
    SUN_CUDA(cudaEventRecord(g.done, g.stream));
    SUN_CUDA(cudaStreamWaitEvent(s, g.done, 0));
  }
  if (hist_mode) {
    slot_bump_kernel<<<1, 1, 0, s>>>(B->d_slot);
    SUN_TRY(check_launch(cudaGetLastError(), "history slot"));
  }
  return SUN_OK;
}

sun_status get_batch_graph(sun_batch* B, const GraphKey& key, cudaGraphExec_t* out) {
  auto it = B->graphs.find(key);
  if (it != B->graphs.end()) {
    *out = it->second;
    return SUN_OK;
  }
  SUN_CUDA(cudaStreamBeginCapture(B->capture_stream, cudaStreamCaptureModeThreadLocal));
  sun_status st = SUN_OK;
  for (int k = 0; k < key.sweeps && st == SUN_OK; ++k)
    st = enqueue_batch_sweep(B, B->capture_stream, key.n_hb, key.n_or, key.reunit != 0, key.plaq != 0, key.poly != 0,
                             true);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(B->capture_stream, &g);
  if (st != SUN_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return fail(SUN_ERR_CUDA, "batch graph capture failed: %s", cudaGetErrorString(e));
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(SUN_ERR_CUDA, "batch graph instantiation failed: %s", cudaGetErrorString(e));
  B->graphs[key] = exec;
  *out = exec;
  return SUN_OK;
}

}  // namespace

extern "C" {

sun_status sun_batch_create(sun_batch** out, sun_lattice* const* lattices, int n, void* stream, int use_graphs) {
  if (!out) return fail(SUN_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!lattices || n < 1) return fail(SUN_ERR_ARG, "a batch needs at least one lattice");
  for (int i = 0; i < n; ++i)
    if (!lattices[i]) return fail(SUN_ERR_ARG, "lattice %d is NULL", i);
  const sun_lattice* L0 = lattices[0];
  for (int i = 0; i < n; ++i) {
    const sun_lattice* L = lattices[i];
    if (L->device != L0->device) return fail(SUN_ERR_ARG, "all lattices of a batch must be on one device");
    if (L->reunit_every > 1) return fail(SUN_ERR_ARG, "batched lattices need reunit_every 0 or 1");
    if (L->reunit_every != L0->reunit_every || L->reunit_mode != L0->reunit_mode)
      return fail(SUN_ERR_ARG, "batched lattices must share reunit_every and reunit_mode");
    if (!L->ops->batch_pass)
      return fail(SUN_ERR_UNSUPPORTED, "no batched kernels for nc = %d at precision %d", L->nc, L->precision);
    for (int j = 0; j < i; ++j)
      if (lattices[j] == L) return fail(SUN_ERR_ARG, "lattice %d appears twice", i);
  }
  sun_batch* B = new sun_batch();
  auto cleanup = [&](sun_status st) {
    sun_batch_destroy(B);
    return st;
  };
  B->n = n;
  B->device = L0->device;
  B->lattices.assign(lattices, lattices + n);
  B->reunit_every = L0->reunit_every;
  B->reunit_mode = L0->reunit_mode;
  B->use_graphs = use_graphs;
  B->graph_sweeps = L0->graph_sweeps;
  if (cudaSetDevice(B->device) != cudaSuccess) return cleanup(fail(SUN_ERR_CUDA, "cudaSetDevice failed"));
  if (stream) {
    B->stream = static_cast<cudaStream_t>(stream);
  } else {
    if (cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking) != cudaSuccess)
      return cleanup(fail(SUN_ERR_CUDA, "stream creation failed"));
    B->own_stream = true;
  }

  // groups in order of first appearance; in a group the chains packed into shared
  // launches come first (create-call order), then the Nc >= 4 chains that fill
  // the GPU on their own (at least 4 blocks per SM per pass), which run the
  // single-lattice kernels inside the batch (their packed kernels are slower)
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, B->device);
  if (sms <= 0) sms = 132;
  auto is_large = [&](const sun_lattice* L) {
    if (L->nc < 4) return false;  // Nc <= 3: the packed kernels run as fast as the single-lattice ones
    const int lpb = L->ops->group_links_per_block > 0 && !(L->ctx.variant & 4) && L->nc == 6
                        ? L->ops->group_links_per_block
                        : ((L->ctx.variant & 1) ? 128 : L->block_threads);
    return L->ctx.g.Vh >= int64_t(4) * sms * lpb;
  };
  for (int pass = 0; pass < 2; ++pass)
    for (int i = 0; i < n; ++i) {
      sun_lattice* L = lattices[i];
      if (is_large(L) != (pass == 1)) continue;
      auto it = std::find_if(B->groups.begin(), B->groups.end(), [&](const BatchGroup& g) { return g.ops == L->ops; });
      if (it == B->groups.end()) {
        B->groups.emplace_back();
        it = B->groups.end() - 1;
        it->ops = L->ops;
      }
      it->members.push_back(L);
      it->positions.push_back(i);
      if (pass == 0) it->n_small++;
    }
  // history columns are group-ordered: column offset of each group
  int col = 0;
  for (auto& g : B->groups) {
    g.offset = col;
    col += int(g.members.size());
  }
  for (auto& g : B->groups) {
    const int all = int(g.members.size());
    const int m = g.n_small;  // the tables cover the packed chains
    const sun_lattice* first = g.members[0];
    const int bt = (first->ctx.variant & 1) ? 128 : first->block_threads;
    std::vector<sun::ChainDesc> desc(all);
    std::vector<uint32_t> start(5 * (m + 1), 0);
    uint64_t tot[5] = {0, 0, 0, 0, 0};
    const int glpb = g.ops->group_links_per_block > 0 ? g.ops->group_links_per_block : 1;
    for (int k = 0; k < all; ++k) {
      const sun_lattice* L = g.members[k];
      const sun::Geom& ge = L->ctx.g;
      sun::ChainDesc& d = desc[k];
      d.links = L->ctx.links;
      d.block_bytes = L->ctx.block_bytes;
      d.g = ge;
      d.alpha_coef = 2.0 * L->beta / L->nc;
      d.key = make_uint2(uint32_t(L->seed & 0xffffffffu), uint32_t(L->seed >> 32));
      d.hb_step = &L->ctx.state->hb_step;
      const int64_t nsp = int64_t(ge.nx) * ge.ny * ge.nz;
      d.plaq_scale = 1.0 / (6.0 * double(ge.V) * L->nc);
      d.poly_scale = 1.0 / (double(L->nc) * double(nsp));
      const uint64_t blocks[5] = {uint64_t((ge.Vh + bt - 1) / bt), uint64_t((8 * ge.Vh + 127) / 128),
                                  uint64_t((ge.V + 255) / 256), uint64_t((nsp + 127) / 128),
                                  uint64_t((ge.Vh + glpb - 1) / glpb)};
      if (k >= m) continue;
      for (int q = 0; q < 5; ++q) {
        start[q * (m + 1) + k] = uint32_t(tot[q]);
        tot[q] += blocks[q];
      }
    }
    for (int q = 0; q < 5; ++q) {
      if (tot[q] >= (uint64_t(1) << 31)) return cleanup(fail(SUN_ERR_ARG, "batch too large for one grid"));
      start[q * (m + 1) + m] = uint32_t(tot[q]);
    }
    sun_status st;
    if ((st = dev_alloc(&g.d_chains, size_t(all), B->stream)) != SUN_OK) return cleanup(st);
    if ((st = dev_alloc(&g.d_start, start.size(), B->stream)) != SUN_OK) return cleanup(st);
    const size_t npart = std::max<size_t>({size_t(1), size_t(tot[2]), size_t(2 * tot[3])});
    if ((st = dev_alloc(&g.d_partials, npart, B->stream)) != SUN_OK) return cleanup(st);
    // pageable sources: the copies return once the tables are staged
    if (cudaMemcpyAsync(g.d_chains, desc.data(), all * sizeof(sun::ChainDesc), cudaMemcpyHostToDevice, B->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(g.d_start, start.data(), start.size() * sizeof(uint32_t), cudaMemcpyHostToDevice,
                        B->stream) != cudaSuccess)
      return cleanup(fail(SUN_ERR_CUDA, "upload of a batch table failed"));
    if (cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming) != cudaSuccess)
      return cleanup(fail(SUN_ERR_CUDA, "batch stream creation failed"));
    sun::BatchCtx& c = g.ctx;
    c.chains = g.d_chains;
    c.n = m;
    c.pass_start = g.d_start;
    c.reunit_start = g.d_start + (m + 1);
    c.plaq_start = g.d_start + 2 * (m + 1);
    c.poly_start = g.d_start + 3 * (m + 1);
    c.group_start = g.d_start + 4 * (m + 1);
    c.group_blocks = uint32_t(tot[4]);
    c.pass_blocks = uint32_t(tot[0]);
    c.reunit_blocks = uint32_t(tot[1]);
    c.plaq_blocks = uint32_t(tot[2]);
    c.poly_blocks = uint32_t(tot[3]);
    c.pass_threads = bt;
    c.variant = first->ctx.variant;
    c.partials = g.d_partials;
  }
  if (cudaStreamCreateWithFlags(&B->capture_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming) != cudaSuccess)
    return cleanup(fail(SUN_ERR_CUDA, "batch stream creation failed"));
  B->hist_cap = int(std::max<int64_t>(1, std::min<int64_t>(kHistCap, (int64_t(4) << 20) / (3 * int64_t(n)))));
  sun_status st;
  if ((st = dev_alloc(&B->d_slot, 1, B->stream)) != SUN_OK) return cleanup(st);
  if ((st = dev_alloc(&B->d_hist, size_t(3) * B->hist_cap * n, B->stream)) != SUN_OK) return cleanup(st);
  B->h_hist.assign(size_t(3) * B->hist_cap * n, 0.0);
  *out = B;
  return SUN_OK;
}

void sun_batch_destroy(sun_batch* B) {
  if (!B) return;
  cudaSetDevice(B->device);
  for (auto& kv : B->graphs) cudaGraphExecDestroy(kv.second);
  for (auto& g : B->groups) {
    if (g.stream) {
      // the batch stream frees the tables after the group's last work
      if (g.done && B->stream) {
        cudaEventRecord(g.done, g.stream);
        cudaStreamWaitEvent(B->stream, g.done, 0);
      }
    }
    if (B->stream) {
      if (g.d_chains) cudaFreeAsync(g.d_chains, B->stream);
      if (g.d_start) cudaFreeAsync(g.d_start, B->stream);
      if (g.d_partials) cudaFreeAsync(g.d_partials, B->stream);
    }
    if (g.stream) cudaStreamDestroy(g.stream);
    if (g.done) cudaEventDestroy(g.done);
  }
  if (B->stream) {
    if (B->d_slot) cudaFreeAsync(B->d_slot, B->stream);
    if (B->d_hist) cudaFreeAsync(B->d_hist, B->stream);
  }
  if (B->fork) cudaEventDestroy(B->fork);
  if (B->capture_stream) cudaStreamDestroy(B->capture_stream);
  if (B->stream) cudaStreamSynchronize(B->stream);
  if (B->own_stream && B->stream) cudaStreamDestroy(B->stream);
  delete B;
}

sun_status sun_batch_run(sun_batch* B, int n_sweeps, int n_hb, int n_or, double* plaq, double* poly) {
  if (!B) return fail(SUN_ERR_ARG, "batch is NULL");
  if (n_sweeps < 0 || n_hb < 0 || n_or < 0) return fail(SUN_ERR_ARG, "counts must be >= 0");
  SUN_CUDA(cudaSetDevice(B->device));
  for (sun_lattice* L : B->lattices) SUN_CUDA(cudaStreamSynchronize(L->stream));
  const bool want_p = plaq != nullptr, want_l = poly != nullptr;
  const int n = B->n;
  for (int done = 0; done < n_sweeps;) {
    const int chunk = std::min(n_sweeps - done, B->hist_cap);
    SUN_CUDA(cudaMemsetAsync(B->d_slot, 0, sizeof(uint32_t), B->stream));
    for (int k = 0; k < chunk;) {
      const bool reunit = B->reunit_every == 1;
      const int per = chunk - k >= B->graph_sweeps ? B->graph_sweeps : 1;
      if (B->use_graphs) {
        cudaGraphExec_t exec = nullptr;
        GraphKey key{n_hb, n_or, reunit ? 1 : 0, want_p ? 1 : 0, want_l ? 1 : 0};
        key.sweeps = per;
        SUN_TRY(get_batch_graph(B, key, &exec));
        SUN_CUDA(cudaGraphLaunch(exec, B->stream));
      } else {
        for (int q = 0; q < per; ++q)
          SUN_TRY(enqueue_batch_sweep(B, B->stream, n_hb, n_or, reunit, want_p, want_l, true));
      }
      k += per;
    }
    if (want_p || want_l) {
      SUN_CUDA(cudaMemcpyAsync(B->h_hist.data(), B->d_hist, size_t(3) * B->hist_cap * n * sizeof(double),
                               cudaMemcpyDeviceToHost, B->stream));
      SUN_CUDA(cudaStreamSynchronize(B->stream));
      // group-ordered columns back to create-call order
      for (const auto& g : B->groups)
        for (size_t k = 0; k < g.members.size(); ++k) {
          const int colg = g.offset + int(k), pos = g.positions[k];
          for (int r = 0; r < chunk; ++r) {
            if (want_p) plaq[size_t(done + r) * n + pos] = B->h_hist[size_t(r) * n + colg];
            if (want_l) {
              const double* src = B->h_hist.data() + size_t(B->hist_cap) * n + (size_t(r) * n + colg) * 2;
              poly[(size_t(done + r) * n + pos) * 2] = src[0];
              poly[(size_t(done + r) * n + pos) * 2 + 1] = src[1];
            }
          }
        }
    }
    done += chunk;
  }
  SUN_CUDA(cudaStreamSynchronize(B->stream));
  B->sweeps_done += uint64_t(n_sweeps);
  for (sun_lattice* L : B->lattices) L->sweeps_done += uint64_t(n_sweeps);
  for (const auto& g : B->groups)
    for (size_t k = size_t(g.n_small); k < g.members.size(); ++k) SUN_TRY(check_wave_timeouts(g.members[k]));
  return SUN_OK;
}

}  // extern "C"

// ===========================================================================
// t-slab decomposition (the paper's multi-GPU scheme, Sec. 3)
// ===========================================================================
namespace {

// one contiguous run of 16-byte words from a slab's boundary slice to a
// neighbour's halo slice
struct HaloSeg {
  const uint4* src;
  uint4* dst;
  int64_t words;
};

__global__ void halo_copy_kernel(const HaloSeg* segs) {
  const HaloSeg sg = segs[blockIdx.y];
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < sg.words; i += int64_t(gridDim.x) * blockDim.x)
    sg.dst[i] = sg.src[i];
}

}  // namespace

struct sun_slabs {
  int n = 0, nc = 0, thickness = 0;
  int dims[4] = {0, 0, 0, 0};
  int device = 0;
  std::vector<sun_lattice*> slab;
  std::vector<int> t_start, flip;  // flip: local parity = global parity ^ flip
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaStream_t capture_stream = nullptr;
  HaloSeg* d_segs = nullptr;  // [mu][global parity][segment]
  int segs_per_exchange = 0;
  int64_t seg_words = 0;      // the longest segment
  char* d_parts = nullptr;    // n partial Polyakov products per spatial site
  const void** d_part_ptrs = nullptr;
  int reunit_every = 1, reunit_mode = 0;
  uint64_t sweeps_done = 0;
  std::vector<double> h_plaq, h_poly;
  std::map<GraphKey, cudaGraphExec_t> graphs;
};

namespace {

sun_status slabs_exchange(sun_slabs* S, cudaStream_t s, int mu, int parity) {
  const HaloSeg* segs = S->d_segs + size_t(2 * mu + parity) * size_t(S->segs_per_exchange);
  int64_t bx = (S->seg_words + 255) / 256;
  if (bx > 1024) bx = 1024;
  halo_copy_kernel<<<dim3(unsigned(bx), unsigned(S->segs_per_exchange)), 256, 0, s>>>(segs);
  return check_launch(cudaGetLastError(), "halo exchange");
}

sun_status enqueue_slabs_sweep(sun_slabs* S, cudaStream_t s, int n_hb, int n_or, bool reunit, bool plaq, bool poly,
                               bool hist_mode) {
  const sun::Ops* ops = S->slab[0]->ops;
  const int n_steps = n_hb + n_or;
  const bool fused = reunit && S->reunit_mode != 0 && n_steps > 0;
  for (int step = 0; step < n_steps; ++step) {
    const bool hb = step < n_hb;
    uint32_t mod = 0, rem = 0;
    if (fused && S->reunit_mode == 1 && step == n_steps - 1) mod = 1;
    if (fused && S->reunit_mode == 2) {
      mod = uint32_t(n_steps);
      rem = uint32_t(step);
    }
    for (int mu = 0; mu < 4; ++mu)
      for (int p = 0; p < 2; ++p) {
        // every slab's links of this (direction, parity), then the halo slices
        for (int k = 0; k < S->n; ++k)
          SUN_TRY(check_launch(ops->pass(ctx_on(S->slab[size_t(k)], s), hb ? SUN_HEATBATH : SUN_OVERRELAX, mu,
                                         p ^ S->flip[size_t(k)], hb ? uint32_t(step) : 0u, mod, rem),
                               hb ? "heatbath pass" : "overrelaxation pass"));
        SUN_TRY(slabs_exchange(S, s, mu, p));
      }
  }
  // the separate re-unitarization covers the halo copies too (the same per-link map)
  if (reunit && !fused)
    for (int k = 0; k < S->n; ++k) SUN_TRY(check_launch(ops->reunit(ctx_on(S->slab[size_t(k)], s)), "reunitarization"));
  for (int k = 0; k < S->n; ++k) {
    sun_lattice* L = S->slab[size_t(k)];
    const uint32_t* slot = hist_mode ? &L->ctx.state->slot : nullptr;
    if (plaq)
      SUN_TRY(check_launch(ops->plaquette(ctx_on(L, s), hist_mode ? L->hist : L->results, slot, kHistCap), "plaquette"));
    if (poly)
      SUN_TRY(check_launch(ops->polyakov_partial(ctx_on(L, s), S->d_parts + size_t(k) * size_t(L->ctx.g.nx) *
                                                                              L->ctx.g.ny * L->ctx.g.nz *
                                                                              ops->polyakov_partial_bytes),
                           "polyakov"));
  }
  sun_lattice* L0 = S->slab[0];
  if (poly)
    SUN_TRY(check_launch(ops->polyakov_combine(ctx_on(L0, s), S->d_part_ptrs, S->n,
                                               hist_mode ? L0->hist + kHistCap : L0->results + 2,
                                               hist_mode ? &L0->ctx.state->slot : nullptr, kHistCap),
                         "polyakov"));
  for (int k = 0; k < S->n; ++k)
    if (n_hb > 0 || hist_mode) {
      bump_kernel<<<1, 1, 0, s>>>(S->slab[size_t(k)]->ctx.state, uint32_t(n_hb), hist_mode ? 1u : 0u);
      SUN_TRY(check_launch(cudaGetLastError(), "step counter"));
    }
  return SUN_OK;
}

sun_status get_slabs_graph(sun_slabs* S, const GraphKey& key, cudaGraphExec_t* out) {
  auto it = S->graphs.find(key);
  if (it != S->graphs.end()) {
    *out = it->second;
    return SUN_OK;
  }
  SUN_CUDA(cudaStreamBeginCapture(S->capture_stream, cudaStreamCaptureModeThreadLocal));
  sun_status st = enqueue_slabs_sweep(S, S->capture_stream, key.n_hb, key.n_or, key.reunit != 0, key.plaq != 0,
                                      key.poly != 0, true);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(S->capture_stream, &g);
  if (st != SUN_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return fail(SUN_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(SUN_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
  S->graphs[key] = exec;
  *out = exec;
  return SUN_OK;
}

// all 8 (direction, parity) halo exchanges: after an import
sun_status slabs_refresh_halos(sun_slabs* S) {
  for (int mu = 0; mu < 4; ++mu)
    for (int p = 0; p < 2; ++p) SUN_TRY(slabs_exchange(S, S->stream, mu, p));
  SUN_CUDA(cudaStreamSynchronize(S->stream));
  return SUN_OK;
}

}  // namespace

extern "C" {

sun_status sun_slabs_create(sun_slabs** out, int nc, const int dims[4], int n_slabs, double beta, int hot_start,
                            uint64_t seed, const sun_options* opt_in) {
  if (!out) return fail(SUN_ERR_ARG, "out is NULL");
  *out = nullptr;
  SUN_TRY(check_dims(dims));
  if (n_slabs < 1 || dims[3] % n_slabs != 0 || (dims[3] / n_slabs) % 2 != 0)
    return fail(SUN_ERR_ARG, "n_slabs = %d must divide Nt = %d into slabs of an even number of slices", n_slabs,
                dims[3]);
  sun_options opt;
  if (opt_in)
    opt = *opt_in;
  else
    sun_options_init(&opt);
  if (opt.device_buf) return fail(SUN_ERR_ARG, "slabs allocate their own memory: device_buf must be NULL");
  if (opt.reunit_every > 1) return fail(SUN_ERR_ARG, "slabs support reunit_every 0 or 1");
  sun_slabs* S = new sun_slabs();
  auto cleanup = [&](sun_status st) {
    sun_slabs_destroy(S);
    return st;
  };
  S->n = n_slabs;
  S->nc = nc;
  S->thickness = dims[3] / n_slabs;
  for (int m = 0; m < 4; ++m) S->dims[m] = dims[m];
  S->reunit_every = opt.reunit_every;
  S->reunit_mode = opt.reunit_mode;
  if (cudaGetDevice(&S->device) != cudaSuccess) return cleanup(fail(SUN_ERR_CUDA, "no CUDA device"));
  if (opt.stream) {
    S->stream = static_cast<cudaStream_t>(opt.stream);
  } else {
    if (cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) != cudaSuccess)
      return cleanup(fail(SUN_ERR_CUDA, "stream creation failed"));
    S->own_stream = true;
  }
  if (cudaStreamCreateWithFlags(&S->capture_stream, cudaStreamNonBlocking) != cudaSuccess)
    return cleanup(fail(SUN_ERR_CUDA, "stream creation failed"));
  opt.stream = S->stream;  // every slab enqueues on the slabs' stream
  const int ldims[4] = {dims[0], dims[1], dims[2], S->thickness + 2};
  for (int k = 0; k < n_slabs; ++k) {
    SlabSpec spec{k * S->thickness, S->thickness, dims[3]};
    sun_lattice* L = nullptr;
    sun_status st = create_lattice(&L, nc, ldims, beta, hot_start, seed, &opt, &spec);
    if (st != SUN_OK) return cleanup(st);
    S->slab.push_back(L);
    S->t_start.push_back(spec.t_start);
    S->flip.push_back((1 - spec.t_start) & 1);  // local t = global t - t_start + 1
  }
  // halo segments: after a pass of (mu, global parity p), slab k's last interior
  // slice -> slab k+1's lower halo, and its first interior slice -> slab k-1's
  // upper halo, every 16-byte component array of the block
  const sun_lattice* L0 = S->slab[0];
  const int64_t vs = int64_t(dims[0]) * dims[1] * dims[2];
  const int64_t vh = L0->ctx.g.Vh;
  const int link_bytes = L0->ops->link_bytes;
  const int n16 = link_bytes / 16, tail = link_bytes % 16;  // tail: one 8-byte array or none
  const int comps = n16 + (tail ? 1 : 0);
  S->segs_per_exchange = 2 * n_slabs * comps;
  std::vector<HaloSeg> segs;
  segs.reserve(size_t(8) * S->segs_per_exchange);
  S->seg_words = 0;
  for (int mu = 0; mu < 4; ++mu)
    for (int p = 0; p < 2; ++p)
      for (int k = 0; k < n_slabs; ++k)
        for (int dir = 0; dir < 2; ++dir) {
          const int dst_k = dir == 0 ? (k + 1) % n_slabs : (k + n_slabs - 1) % n_slabs;
          const int t_src = dir == 0 ? S->thickness : 1;      // last / first interior slice
          const int t_dst = dir == 0 ? 0 : S->thickness + 1;  // lower / upper halo of the neighbour
          const sun_lattice* A = S->slab[size_t(k)];
          const sun_lattice* B = S->slab[size_t(dst_k)];
          const char* a = A->ctx.links + (2 * mu + (p ^ S->flip[size_t(k)])) * A->ctx.block_bytes;
          char* b = B->ctx.links + (2 * mu + (p ^ S->flip[size_t(dst_k)])) * B->ctx.block_bytes;
          for (int c = 0; c < comps; ++c) {
            const int64_t w = c < n16 ? 16 : 8;  // bytes per link in this component array
            const int64_t base = c < n16 ? int64_t(c) * vh * 16 : int64_t(n16) * vh * 16;
            HaloSeg sg;
            sg.src = reinterpret_cast<const uint4*>(a + base + int64_t(t_src) * (vs / 2) * w);
            sg.dst = reinterpret_cast<uint4*>(b + base + int64_t(t_dst) * (vs / 2) * w);
            sg.words = (vs / 2) * w / 16;  // all extents even: vs / 2 is even
            S->seg_words = std::max(S->seg_words, sg.words);
            segs.push_back(sg);
          }
        }
  const int64_t nsp = vs;
  const size_t part_bytes = size_t(nsp) * L0->ops->polyakov_partial_bytes;
  std::vector<const void*> ptrs(static_cast<size_t>(n_slabs));
  if (cudaMalloc(&S->d_segs, segs.size() * sizeof(HaloSeg)) != cudaSuccess ||
      cudaMalloc(&S->d_parts, part_bytes * size_t(n_slabs)) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&S->d_part_ptrs), ptrs.size() * sizeof(void*)) != cudaSuccess) {
    cudaGetLastError();
    return cleanup(fail(SUN_ERR_OOM, "slab tables: cudaMalloc failed"));
  }
  for (int k = 0; k < n_slabs; ++k) ptrs[size_t(k)] = S->d_parts + size_t(k) * part_bytes;
  if (cudaMemcpy(S->d_segs, segs.data(), segs.size() * sizeof(HaloSeg), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(S->d_part_ptrs, ptrs.data(), ptrs.size() * sizeof(void*), cudaMemcpyHostToDevice) != cudaSuccess)
    return cleanup(fail(SUN_ERR_CUDA, "upload of the slab tables failed"));
  // the hot start drew every slab's halo links from their global counters already;
  // the exchange makes the halos copies of the owners' links in any case
  sun_status st = slabs_refresh_halos(S);
  if (st != SUN_OK) return cleanup(st);
  *out = S;
  return SUN_OK;
}

void sun_slabs_destroy(sun_slabs* S) {
  if (!S) return;
  cudaSetDevice(S->device);
  if (S->stream) cudaStreamSynchronize(S->stream);
  for (auto& kv : S->graphs) cudaGraphExecDestroy(kv.second);
  for (sun_lattice* L : S->slab) sun_lattice_destroy(L);
  if (S->d_segs) cudaFree(S->d_segs);
  if (S->d_parts) cudaFree(S->d_parts);
  if (S->d_part_ptrs) cudaFree(S->d_part_ptrs);
  if (S->capture_stream) cudaStreamDestroy(S->capture_stream);
  if (S->own_stream && S->stream) cudaStreamDestroy(S->stream);
  delete S;
}

sun_status sun_slabs_run(sun_slabs* S, int n_sweeps, int n_hb, int n_or, double* plaq_hist, double* poly_hist) {
  if (!S) return fail(SUN_ERR_ARG, "slabs is NULL");
  if (n_sweeps < 0 || n_hb < 0 || n_or < 0) return fail(SUN_ERR_ARG, "counts must be >= 0");
  SUN_CUDA(cudaSetDevice(S->device));
  const bool plaq = plaq_hist != nullptr, poly = poly_hist != nullptr;
  const bool graphs = S->slab[0]->use_graphs != 0;
  S->h_plaq.resize(kHistCap);
  S->h_poly.resize(2 * kHistCap);
  for (int done = 0; done < n_sweeps;) {
    const int chunk = std::min(n_sweeps - done, kHistCap);
    for (sun_lattice* L : S->slab) SUN_CUDA(cudaMemsetAsync(&L->ctx.state->slot, 0, sizeof(uint32_t), S->stream));
    for (int k = 0; k < chunk; ++k) {
      const bool reunit = S->reunit_every == 1;
      if (graphs) {
        cudaGraphExec_t exec = nullptr;
        SUN_TRY(get_slabs_graph(S, GraphKey{n_hb, n_or, reunit ? 1 : 0, plaq ? 1 : 0, poly ? 1 : 0}, &exec));
        SUN_CUDA(cudaGraphLaunch(exec, S->stream));
      } else {
        SUN_TRY(enqueue_slabs_sweep(S, S->stream, n_hb, n_or, reunit, plaq, poly, true));
      }
    }
    if (plaq) {
      // each slab holds its interior's share (already divided by 6 V Nc of the whole lattice)
      for (int r = 0; r < chunk; ++r) plaq_hist[done + r] = 0.0;
      for (sun_lattice* L : S->slab) {
        SUN_CUDA(cudaMemcpyAsync(S->h_plaq.data(), L->hist, chunk * sizeof(double), cudaMemcpyDeviceToHost, S->stream));
        SUN_CUDA(cudaStreamSynchronize(S->stream));
        for (int r = 0; r < chunk; ++r) plaq_hist[done + r] += S->h_plaq[size_t(r)];
      }
    }
    if (poly) {
      SUN_CUDA(cudaMemcpyAsync(poly_hist + 2 * done, S->slab[0]->hist + kHistCap, 2 * chunk * sizeof(double),
                               cudaMemcpyDeviceToHost, S->stream));
    }
    done += chunk;
  }
  SUN_CUDA(cudaStreamSynchronize(S->stream));
  S->sweeps_done += uint64_t(n_sweeps);
  for (sun_lattice* L : S->slab) L->sweeps_done += uint64_t(n_sweeps);
  return SUN_OK;
}

// the interior links of every slab <-> the canonical host array of the whole lattice
static sun_status slabs_copy_links(sun_slabs* S, double* host, size_t n, bool to_host) {
  const int nc = S->nc;
  const int64_t per = 2 * int64_t(nc) * nc;
  const int64_t vs = int64_t(S->dims[0]) * S->dims[1] * S->dims[2];
  const int64_t V = vs * S->dims[3];
  if (n != size_t(4 * V * per)) return fail(SUN_ERR_ARG, "host buffer holds %zu doubles, need %lld", n,
                                            (long long)(4 * V * per));
  SUN_CUDA(cudaSetDevice(S->device));
  for (int k = 0; k < S->n; ++k) {
    sun_lattice* L = S->slab[size_t(k)];
    const sun::Ctx c = ctx_on(L, S->stream);
    const int64_t vloc = L->ctx.g.V;
    for (int mu = 0; mu < 4; ++mu) {
      // local slices [1, 1 + thickness) <-> global slices [t_start, t_start + thickness)
      const int64_t lfirst = int64_t(mu) * vloc + vs, gfirst = int64_t(mu) * V + int64_t(S->t_start[size_t(k)]) * vs;
      const int64_t total = int64_t(S->thickness) * vs;
      for (int64_t off = 0; off < total; off += L->plan.staging_links) {
        const int64_t cnt = std::min<int64_t>(total - off, L->plan.staging_links);
        double* h = host + (gfirst + off) * per;
        if (to_host) {
          SUN_TRY(check_launch(L->ops->export_links(c, L->staging, lfirst + off, cnt), "export"));
          SUN_CUDA(cudaMemcpyAsync(h, L->staging, size_t(cnt * per) * sizeof(double), cudaMemcpyDeviceToHost,
                                   S->stream));
        } else {
          SUN_CUDA(cudaMemcpyAsync(L->staging, h, size_t(cnt * per) * sizeof(double), cudaMemcpyHostToDevice,
                                   S->stream));
          SUN_TRY(check_launch(L->ops->import_links(c, L->staging, lfirst + off, cnt), "import"));
        }
        SUN_CUDA(cudaStreamSynchronize(S->stream));  // the staging buffer is reused
      }
    }
  }
  if (!to_host) SUN_TRY(slabs_refresh_halos(S));
  return SUN_OK;
}

sun_status sun_slabs_export_links(sun_slabs* S, double* host, size_t n) {
  if (!S || !host) return fail(SUN_ERR_ARG, "NULL argument");
  return slabs_copy_links(S, host, n, true);
}

sun_status sun_slabs_import_links(sun_slabs* S, const double* host, size_t n) {
  if (!S || !host) return fail(SUN_ERR_ARG, "NULL argument");
  return slabs_copy_links(S, const_cast<double*>(host), n, false);
}

}  // extern "C"
