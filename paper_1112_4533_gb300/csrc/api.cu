// api.cu -- C ABI of the SU(Nc) link-sweep library (declared in include/sun.h):
// the lattice handle.
//
// Owns the lattice handle: device memory layout, the chessboard schedule of
// Sec. 3 of Cardoso & Bicudo (arXiv:1112.4533) -- per step, directions
// mu = 0..3 each as an even then an odd pass --, CUDA-graph capture of one
// sweep, deterministic observable reductions and the canonical FP64
// import/export path.  Batches, t-slabs and configuration files live in
// batch.cu, slabs.cu and config_io.cu.
#include "api_internal.h"

namespace sun_api {

namespace {
thread_local std::string g_last_error;
}  // namespace

sun_status fail(sun_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

const char* last_error() { return g_last_error.c_str(); }
void set_last_error(const char* msg) { g_last_error = msg ? msg : ""; }

namespace {
__global__ void bump_kernel(sun::DevState* st, uint32_t hb_steps, uint32_t slots) {
  st->hb_step += hb_steps;
  st->slot += slots;
}

}  // namespace

sun_status launch_bump(sun::DevState* st, uint32_t hb_steps, uint32_t slots, cudaStream_t s) {
  bump_kernel<<<1, 1, 0, s>>>(st, hb_steps, slots);
  return check_launch(cudaGetLastError(), "step counter");
}

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
  if (n_hb > 0 || hist_mode) SUN_TRY(launch_bump(L->ctx.state, uint32_t(n_hb), hist_mode ? 1u : 0u, s));
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

}  // namespace sun_api

namespace sun {
void set_last_error_message(const char* msg) { sun_api::set_last_error(msg); }
}  // namespace sun

using namespace sun_api;

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

const char* sun_last_error(void) { return last_error(); }

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

sun_status sun_api::create_lattice(sun_lattice** out, int nc, const int dims[4], double beta, int hot_start,
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

sun_status sun_update_pass_reunit(sun_lattice* L, int mode, int mu, int parity) {
  if (!L) return fail(SUN_ERR_ARG, "lattice is NULL");
  if (mode != SUN_HEATBATH && mode != SUN_OVERRELAX) return fail(SUN_ERR_ARG, "mode must be 0 or 1");
  if (mu < 0 || mu > 3) return fail(SUN_ERR_ARG, "mu must be in 0..3");
  if (parity != 0 && parity != 1) return fail(SUN_ERR_ARG, "parity must be 0 or 1");
  if (!L->ops->fused_reunit)
    return fail(SUN_ERR_UNSUPPORTED, "the fused re-unitarization is not built for nc = %d at precision %d", L->nc,
                L->precision);
  SUN_TRY(set_device(L));
  // reunit_mod 1, remainder 0: every run of 32 half-sites, i.e. every updated link
  return check_launch(L->ops->pass(ctx_on(L, L->stream), mode, mu, parity, 0u, 1u, 0u), "update pass");
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
// The address through which a kernel on the current device reads and writes
// host memory in place, or NULL: page-locked memory mapped into the device's
// address space, and, for reads (for_reading), where the device reaches pageable
// memory through the host's page tables
// (cudaDevAttrPageableMemoryAccessUsesHostPageTables, e.g. a Grace host on
// NVLink-C2C), any host memory.  NULL sends the transfer through the staging
// buffer.  Measured on GB300 + Grace, 2-6 GB: pageable imports in place 202 GB/s
// against 101 GB/s staged; exports in place 173 GB/s into pages the host has
// touched, but 3.4 GB/s into fresh ones (each first touch is a fault taken by
// the GPU), so exports to pageable memory stay staged (106 GB/s).
static double* mapped_host(const void* host, bool for_reading) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type == cudaMemoryTypeHost && a.devicePointer) return static_cast<double*>(a.devicePointer);
  if (for_reading && a.type == cudaMemoryTypeUnregistered) {
    int dev = 0, pageable = 0, host_tables = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&host_tables, cudaDevAttrPageableMemoryAccessUsesHostPageTables, dev) ==
            cudaSuccess &&
        pageable && host_tables)
      return static_cast<double*>(const_cast<void*>(host));
    cudaGetLastError();
  }
  return nullptr;
}

sun_status sun_export_links(sun_lattice* L, double* host, size_t n) {
  if (!L || !host) return fail(SUN_ERR_ARG, "NULL argument");
  if (n != canonical_doubles(L))
    return fail(SUN_ERR_ARG, "host buffer holds %zu doubles, need %zu", n, canonical_doubles(L));
  if (reinterpret_cast<uintptr_t>(host) % 16) return fail(SUN_ERR_ARG, "host buffer must be 16-byte aligned");
  SUN_TRY(set_device(L));
  const sun::Ctx c = ctx_on(L, L->stream);
  const int64_t total = 4 * L->ctx.g.V, per = 2 * L->nc * L->nc;
  if (double* dev = mapped_host(host, false)) {
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
  if (n != canonical_doubles(L))
    return fail(SUN_ERR_ARG, "host buffer holds %zu doubles, need %zu", n, canonical_doubles(L));
  if (reinterpret_cast<uintptr_t>(host) % 16) return fail(SUN_ERR_ARG, "host buffer must be 16-byte aligned");
  SUN_TRY(set_device(L));
  const sun::Ctx c = ctx_on(L, L->stream);
  const int64_t total = 4 * L->ctx.g.V, per = 2 * L->nc * L->nc;
  if (const double* dev = mapped_host(host, true)) {
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
  if (double* dev = mapped_host(host, !to_host)) {
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
  SUN_CUDA(cudaMemcpyAsync(L->host_results, &L->ctx.state->hb_step, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                           L->stream));
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
  SUN_CUDA(cudaMemcpyAsync(&L->ctx.state->hb_step, L->host_results, sizeof(uint32_t), cudaMemcpyHostToDevice,
                           L->stream));
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

