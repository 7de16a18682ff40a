// batch.cu -- batches of chains (sun_batch_*): many independent lattices swept
// by shared launches, each evolving exactly as alone.
#include "api_internal.h"

using namespace sun_api;

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
