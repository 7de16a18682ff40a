// noalloc.cu -- plaquette of caller-owned link storage without any allocation.
//
// Some callers cannot allocate device memory when they need an observable:
// code that runs inside a memory arena it does not own (a framework that hands
// out fixed buffers and forbids cudaMalloc after start-up), and latency-critical
// loops where an allocation's implicit synchronisation is not acceptable.
// sun_plaquette_noalloc serves them: it reads links the caller already holds
// (in this library's storage layout) and writes the result to a caller-owned
// device double, with its reduction scratch in a fixed array that lives in the
// library's own device image.
#include <cstring>
#include <mutex>

#include "sun.h"
#include "sun_runtime.h"

namespace {

// Reduction scratch: one FP64 partial per block of 256 sites, then the counter
// words of the last-block reduction.  512 KiB + 256 B per GPU that loads the
// library, held until the process exits.
constexpr int kNoAllocMaxBlocks = 65536;
constexpr int64_t kNoAllocSitesPerBlock = 256;
constexpr int64_t kNoAllocMaxSites = int64_t(kNoAllocMaxBlocks) * kNoAllocSitesPerBlock;  // 16,777,216

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocMaxBlocks + 32];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_addr[kMaxDevices] = {};  // device address of g_noalloc_scratch, per device

sun_status noalloc_fail(sun_status s, const char* msg) {
  sun::set_last_error_message(msg);  // reported by sun_last_error()
  return s;
}

const sun::Ops* noalloc_ops(int nc, int storage, int precision) {
  switch (nc) {
    case 2: return sun::ops_su2(storage, precision);
    case 3: return sun::ops_su3(storage, precision);
    case 4: return sun::ops_su4(storage, precision);
    case 5: return sun::ops_su5(storage, precision);
    case 6: return sun::ops_su6(storage, precision);
    default: return nullptr;
  }
}

}  // namespace

extern "C" sun_status sun_plaquette_noalloc(const void* links, int nc, const int dims[4], int precision,
                                            int storage, double* out, void* stream) {
  if (!links || !out || !dims) return noalloc_fail(SUN_ERR_ARG, "NULL argument");
  int64_t V = 1;
  for (int m = 0; m < 4; ++m) {
    if (dims[m] < 2 || (dims[m] & 1)) return noalloc_fail(SUN_ERR_ARG, "lattice extents must be even and >= 2");
    V *= dims[m];
    if (V > kNoAllocMaxSites) break;
  }
  if (V > kNoAllocMaxSites)
    return noalloc_fail(SUN_ERR_ARG,
                        "lattice too large for sun_plaquette_noalloc: at most 16777216 sites (65536 reduction "
                        "blocks of 256 sites in the fixed scratch); use sun_plaquette");
  if (storage == 0) storage = nc == 2 ? 4 : (nc == 3 ? 12 : 2 * nc * nc);
  const sun::Ops* ops = noalloc_ops(nc, storage, precision);
  if (!ops) return noalloc_fail(SUN_ERR_UNSUPPORTED, "no kernels for this (nc, storage, precision)");

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return noalloc_fail(SUN_ERR_CUDA, "no current CUDA device");
  }
  double* scratch = nullptr;
  {
    // set-up, once per device, with that device current: the host-side name
    // g_noalloc_scratch is not a device address, so look the address up
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return noalloc_fail(SUN_ERR_CUDA, "cudaGetSymbolAddress of the plaquette scratch failed");
      }
      g_scratch_addr[dev] = static_cast<double*>(p);
    }
    scratch = g_scratch_addr[dev];
  }

  sun::Geom g;
  g.nx = dims[0];
  g.ny = dims[1];
  g.nz = dims[2];
  g.nt = dims[3];
  g.nxh = dims[0] / 2;
  g.V = V;
  g.Vh = V / 2;
  g.stride[0] = 1;
  g.stride[1] = dims[0];
  g.stride[2] = int64_t(dims[0]) * dims[1];
  g.stride[3] = int64_t(dims[0]) * dims[1] * dims[2];
  g.div_nxh = sun::make_fastdiv(uint32_t(g.nxh));
  g.div_ny = sun::make_fastdiv(uint32_t(g.ny));
  g.div_nz = sun::make_fastdiv(uint32_t(g.nz));
  g.div_nx = sun::make_fastdiv(uint32_t(g.nx));

  sun::Ctx c;
  std::memset(&c, 0, sizeof(c));
  c.links = const_cast<char*>(static_cast<const char*>(links));
  c.block_bytes = g.Vh * ops->link_bytes;
  c.g = g;
  c.nc = nc;
  c.partials = scratch;
  // the reduction's counter words follow the partials (256-byte aligned)
  c.state = reinterpret_cast<sun::DevState*>(scratch + kNoAllocMaxBlocks);
  c.stream = static_cast<cudaStream_t>(stream);
  c.block_threads = 128;
  c.reduce_blocks = kNoAllocMaxBlocks;  // one block per 256 sites: ceil(V/256) <= 65536
  c.h_begin = 0;  // the whole lattice
  c.h_end = g.Vh;
  c.lex_offset = 0u;
  c.v_global = uint32_t(V);

  // the array keeps the last call's contents: re-arm the completion counter
  if (cudaMemsetAsync(c.state, 0, sizeof(sun::DevState), c.stream) != cudaSuccess) {
    cudaGetLastError();
    return noalloc_fail(SUN_ERR_CUDA, "clearing the reduction counter failed");
  }
  const cudaError_t e = ops->plaquette(c, out, nullptr, 1);
  if (e != cudaSuccess) return noalloc_fail(SUN_ERR_CUDA, cudaGetErrorString(e));
  return SUN_OK;
}
