// slabs.cu -- the t-slab decomposition (sun_slabs_*): the paper's multi-GPU
// scheme (Sec. 3), every slab a lattice with halo slices, halos exchanged after
// every chessboard pass.
#include "api_internal.h"

using namespace sun_api;

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
      SUN_TRY(check_launch(ops->plaquette(ctx_on(L, s), hist_mode ? L->hist : L->results, slot, kHistCap),
                           "plaquette"));
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
    if (n_hb > 0 || hist_mode)
      SUN_TRY(launch_bump(S->slab[size_t(k)]->ctx.state, uint32_t(n_hb), hist_mode ? 1u : 0u, s));
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
