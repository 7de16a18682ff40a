// config_io.cu -- configuration files (sun_save_config, sun_load_config,
// sun_read_config_header; layout in include/sun.h).  The paper stores the
// generated configurations (Sec. 3); here a file also carries the chain's
// state so that a lattice resumes from it bitwise.
#include "api_internal.h"

using namespace sun_api;

extern "C" {

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

}  // extern "C"
