// autotune.cu -- measured choice of the kernel configuration of a lattice or a
// batch (sun_autotune, sun_autotune_batch in include/sun.h).
//
// The paper tunes its kernels by hand for its GPU (Sec. 3: threads per block,
// storage format, read path).  Here the choice is measured on the GPU at hand:
// scratch lattices of the requested shape are swept with each candidate
// configuration and the fastest is kept.  The search goes one option at a time
// -- kernel shape (block size, register bound, per-link or row-parallel
// kernel), then storage format, then the re-unitarization placement, then the
// even/odd wavefront launches -- each stage starting from the best of the
// previous one.  Only the public entry points are used, so the timings include
// exactly what a caller of sun_run / sun_batch_run pays.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "sun.h"
#include "sun_runtime.h"

namespace {

struct Spec {
  int nc;
  int dims[4];
  double beta;
};

// the tuned fields of sun_options, and the winner's time per sweep
struct Tuned {
  int storage, block_threads, variant, reunit_mode, graph_sweeps;
  double ms;
};

std::mutex g_cache_mutex;
std::map<std::string, Tuned> g_cache;
bool g_file_loaded = false;

// Optional persistent cache: the file named by SUN_TUNE_CACHE holds one line per
// result, "key<TAB>storage block_threads variant reunit_mode graph_sweeps ms"; it is read on
// the first lookup and every new result is appended.  Keys include the GPU's name
// and multiprocessor count, so one file can serve several kinds of GPU.
const char* cache_file() {
  const char* f = getenv("SUN_TUNE_CACHE");
  return (f && *f) ? f : nullptr;
}

void load_cache_file() {  // with g_cache_mutex held
  if (g_file_loaded) return;
  g_file_loaded = true;
  const char* path = cache_file();
  if (!path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  char line[2048];
  while (fgets(line, sizeof(line), f)) {
    char* tab = strchr(line, '\t');
    if (!tab) continue;
    *tab = '\0';
    Tuned t;
    if (sscanf(tab + 1, "%d %d %d %d %d %lf", &t.storage, &t.block_threads, &t.variant, &t.reunit_mode,
               &t.graph_sweeps, &t.ms) == 6)
      g_cache[line] = t;
  }
  fclose(f);
}

void append_cache_file(const std::string& key, const Tuned& t) {  // with g_cache_mutex held
  const char* path = cache_file();
  if (!path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s\t%d %d %d %d %d %.6f\n", key.c_str(), t.storage, t.block_threads, t.variant, t.reunit_mode,
          t.graph_sweeps, t.ms);
  fclose(f);
}

sun_status tune_fail(sun_status s, const char* msg) {
  sun::set_last_error_message(msg);
  return s;
}

std::string cache_key(const std::vector<Spec>& specs, int n_hb, int n_or, int flags, const sun_options& base,
                      int device) {
  std::string k;
  char buf[512];
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
    cudaGetLastError();
    std::memset(&prop, 0, sizeof(prop));
  }
  for (char* c = prop.name; *c; ++c)
    if (*c == '\t' || *c == '\n' || *c == '|') *c = '_';
  snprintf(buf, sizeof(buf), "%s/%d|%d|%d|%d|%d|%d|%d|%d|%d|%d|", prop.name, prop.multiProcessorCount, n_hb, n_or,
           flags, base.precision, base.reunit_every, base.use_graphs, (flags & SUN_TUNE_STORAGE) ? -1 : base.storage,
           (flags & SUN_TUNE_REUNIT_MODE) ? -1 : base.reunit_mode, base.wave_lag);
  k += buf;
  for (const Spec& s : specs) {
    snprintf(buf, sizeof(buf), "%d:%d,%d,%d,%d:%.17g;", s.nc, s.dims[0], s.dims[1], s.dims[2], s.dims[3], s.beta);
    k += buf;
  }
  return k;
}

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// Milliseconds per sweep of one configuration, or a negative value if the
// configuration cannot be built (unsupported combination, no memory).
double time_config(const std::vector<Spec>& specs, int n_hb, int n_or, const sun_options& o) {
  std::vector<sun_lattice*> lats;
  auto release = [&]() {
    for (sun_lattice* L : lats) sun_lattice_destroy(L);
    lats.clear();
  };
  for (size_t i = 0; i < specs.size(); ++i) {
    sun_lattice* L = nullptr;
    if (sun_lattice_create(&L, specs[i].nc, specs[i].dims, specs[i].beta, 1, 1 + i, &o) != SUN_OK) {
      release();
      return -1.0;
    }
    lats.push_back(L);
  }
  sun_batch* B = nullptr;
  if (lats.size() > 1 && sun_batch_create(&B, lats.data(), int(lats.size()), nullptr, o.use_graphs) != SUN_OK) {
    release();
    return -1.0;
  }
  auto run = [&](int k) -> bool {
    if (B) return sun_batch_run(B, k, n_hb, n_or, nullptr, nullptr) == SUN_OK;
    return sun_run(lats[0], k, n_hb, n_or, nullptr, nullptr) == SUN_OK;
  };
  double ms = -1.0;
  // warm-up (graph capture, first touch), an estimate, then about 30 ms of sweeps
  if (run(1)) {
    double t0 = now_ms();
    if (run(1)) {
      const double one = now_ms() - t0;
      int k = one > 0.0 ? int(std::ceil(30.0 / one)) : 8;
      k = k < 1 ? 1 : (k > 64 ? 64 : k);
      t0 = now_ms();
      if (run(k)) ms = (now_ms() - t0) / k;
    }
  }
  if (B) sun_batch_destroy(B);
  release();
  return ms;
}

std::vector<int> storages_of(int nc) {
  if (nc == 2) return {4, 8};
  if (nc == 3) return {12, 18};
  return {2 * nc * nc};
}

// A later stage changes the configuration only for a gain above the timing noise.
constexpr double kMinGain = 0.02;

// one stage: try every candidate built from `best` by `apply`, keep the fastest
// (within a stage the fastest wins; against the previous stages' best a
// candidate must be faster by kMinGain)
template <class Apply>
void stage(const std::vector<Spec>& specs, int n_hb, int n_or, int n_cand, Apply apply, sun_options& best,
           double& best_ms) {
  const sun_options start = best;
  const double start_ms = best_ms;
  for (int c = 0; c < n_cand; ++c) {
    sun_options o = start;
    if (!apply(c, o)) continue;
    if (std::memcmp(&o, &start, sizeof(o)) == 0 && start_ms > 0.0) continue;
    const double ms = time_config(specs, n_hb, n_or, o);
    const bool beats_start = start_ms <= 0.0 || ms < (1.0 - kMinGain) * start_ms;
    if (ms > 0.0 && beats_start && (best_ms <= 0.0 || ms < best_ms)) {
      best = o;
      best_ms = ms;
    }
  }
}

sun_status autotune(const std::vector<Spec>& specs, int n_hb, int n_or, int flags, sun_options* opt,
                    double* ms_out) {
  if (!opt) return tune_fail(SUN_ERR_ARG, "opt is NULL");
  if (n_hb < 0 || n_or < 0 || n_hb + n_or == 0) return tune_fail(SUN_ERR_ARG, "a sweep needs at least one step");
  if (flags & ~(SUN_TUNE_STORAGE | SUN_TUNE_REUNIT_MODE | SUN_TUNE_TWO_ROW))
    return tune_fail(SUN_ERR_ARG, "unknown autotune flags");
  if (opt->device_buf) return tune_fail(SUN_ERR_ARG, "autotuning uses scratch lattices: device_buf must be NULL");
  int nc0 = specs[0].nc;
  bool same_nc = true;
  for (const Spec& s : specs) {
    if (s.nc < 2 || s.nc > 6) return tune_fail(SUN_ERR_UNSUPPORTED, "kernels are built for nc 2..6");
    same_nc = same_nc && s.nc == nc0;
  }
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) {
    cudaGetLastError();
    return tune_fail(SUN_ERR_CUDA, "no CUDA device");
  }
  const std::string key = cache_key(specs, n_hb, n_or, flags, *opt, device);
  {
    std::lock_guard<std::mutex> lock(g_cache_mutex);
    load_cache_file();
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
      const Tuned& t = it->second;
      opt->storage = t.storage;
      opt->block_threads = t.block_threads;
      opt->variant = t.variant;
      opt->reunit_mode = t.reunit_mode;
      opt->graph_sweeps = t.graph_sweeps;
      opt->wave_skip_units = 0;
      if (ms_out) *ms_out = t.ms;
      return SUN_OK;
    }
  }

  sun_options best = *opt;
  if (best.storage == 0 && same_nc) best.storage = storages_of(nc0)[0];  // the library default
  best.stream = nullptr;  // scratch lattices run on their own streams
  best.variant = 0;
  best.block_threads = 128;
  best.wave_skip_units = 0;
  best.graph_sweeps = 1;
  double best_ms = -1.0;
  const bool fp32 = best.precision == 32;

  // 1. kernel shape: block size, register bound (SU(3), SU(4) FP32),
  //    row-parallel vs per-link kernel (Nc 4, 6), two-row staple if allowed
  struct Shape {
    int variant, block;
  };
  std::vector<Shape> shapes = {{0, 64}, {0, 128}, {0, 256}};
  // a batch of chains that do not fill the GPU alone runs the packed batch kernels,
  // which have neither the packed-FP32 nor the wavefront form
  bool own_launches = specs.size() == 1;
  for (const Spec& s : specs)
    if (s.nc >= 4 && int64_t(s.dims[0]) * s.dims[1] * s.dims[2] * s.dims[3] >= (int64_t(1) << 18)) own_launches = true;
  if (same_nc && nc0 == 3 && fp32) {
    shapes.push_back({1, 128});
    if (own_launches) shapes.push_back({17, 128});  // packed-FP32 overrelaxation, register-bounded heatbath
    if (flags & SUN_TUNE_TWO_ROW) {
      shapes.push_back({3, 128});
      shapes.push_back({2, 128});
    }
  }
  if (same_nc && (nc0 == 4 || nc0 == 6)) {
    // the row-parallel kernel has a fixed block; the per-link one takes the sizes above
    const int row_parallel = nc0 == 6 ? 0 : 4;  // the bit that selects it
    const int per_link = nc0 == 6 ? 4 : 0;
    for (Shape& s : shapes) s.variant = per_link;
    shapes.push_back({row_parallel, 128});
    // the register-bounded per-link pass (its own launches only: the batch kernels ignore it)
    if (nc0 == 4 && fp32 && own_launches) shapes.push_back({1, 128});
  }
  stage(specs, n_hb, n_or, int(shapes.size()),
        [&](int c, sun_options& o) {
          o.variant = shapes[size_t(c)].variant;
          o.block_threads = shapes[size_t(c)].block;
          return true;
        },
        best, best_ms);
  if (best_ms <= 0.0) return tune_fail(SUN_ERR_UNSUPPORTED, "no candidate configuration could be built and run");

  // 2. storage format
  if ((flags & SUN_TUNE_STORAGE) && same_nc) {
    const std::vector<int> st = storages_of(nc0);
    stage(specs, n_hb, n_or, int(st.size()),
          [&](int c, sun_options& o) {
            o.storage = st[size_t(c)];
            // the two-row staple needs two-row storage
            if (o.storage != 12) o.variant &= ~2;
            return true;
          },
          best, best_ms);
  }

  // 3. re-unitarization placement
  if (flags & SUN_TUNE_REUNIT_MODE)
    stage(specs, n_hb, n_or, 3,
          [&](int c, sun_options& o) {
            o.reunit_mode = c;
            return true;
          },
          best, best_ms);

  // 4. even/odd wavefront launches: only for kernels with that form, and in a
  //    batch only where a chain runs its own launches
  const bool has_wave = own_launches && !(best.variant & 18) && !(same_nc && nc0 == 6 && !(best.variant & 4)) &&
                        !(same_nc && nc0 == 4 && (best.variant & 4));
  if (has_wave)
    stage(specs, n_hb, n_or, 1,
          [&](int, sun_options& o) {
            o.variant |= 8;
            return true;
          },
          best, best_ms);

  // 5. sweeps per graph launch (amortises the launch of short sweeps)
  if (best.use_graphs) {
    const int per[2] = {4, 16};
    stage(specs, n_hb, n_or, 2,
          [&](int c, sun_options& o) {
            o.graph_sweeps = per[c];
            return true;
          },
          best, best_ms);
  }

  {
    std::lock_guard<std::mutex> lock(g_cache_mutex);
    const Tuned t{best.storage, best.block_threads, best.variant, best.reunit_mode, best.graph_sweeps, best_ms};
    g_cache[key] = t;
    append_cache_file(key, t);
  }
  best.stream = opt->stream;
  *opt = best;
  if (ms_out) *ms_out = best_ms;
  return SUN_OK;
}

}  // namespace

extern "C" sun_status sun_autotune(int nc, const int dims[4], double beta, int n_heatbath, int n_overrelax,
                                   int flags, sun_options* opt, double* ms_per_sweep) {
  if (!dims) return tune_fail(SUN_ERR_ARG, "dims is NULL");
  Spec s{nc, {dims[0], dims[1], dims[2], dims[3]}, beta};
  return autotune({s}, n_heatbath, n_overrelax, flags, opt, ms_per_sweep);
}

extern "C" sun_status sun_autotune_batch(int n, const int* nc, const int* dims, const double* beta, int n_heatbath,
                                         int n_overrelax, int flags, sun_options* opt, double* ms_per_sweep) {
  if (n < 1 || !nc || !dims || !beta) return tune_fail(SUN_ERR_ARG, "a batch needs n >= 1 chains");
  std::vector<Spec> specs(static_cast<size_t>(n));
  for (int i = 0; i < n; ++i) {
    const int* d = dims + 4 * i;
    specs[size_t(i)] = Spec{nc[i], {d[0], d[1], d[2], d[3]}, beta[i]};
  }
  return autotune(specs, n_heatbath, n_overrelax, flags, opt, ms_per_sweep);
}
