// selftest.cu -- the integer FP32 <-> FP64 conversions against the hardware's.
//
// The re-unitarization kernels convert links between the FP32 storage and FP64
// with to_f64 / to_f32 (sun_device.cuh): integer operations on the IEEE 754
// encodings in place of GB300's FP64-rate conversion instructions.  This checks
// that they return the hardware's bits: every one of the 2^32 float encodings
// through to_f64, and n seeded double encodings through to_f32, drawn so that
// the exponents around the float's normal range and the rounding ties of the 29
// dropped fraction bits are covered.
#include <cstdint>
#include <cstring>

#include "sun.h"
#include "sun_device.cuh"
#include "sun_runtime.h"

namespace {

// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): one 64-bit output per index
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// out[0] mismatches of to_f64, out[1] of to_f32, out[2] / out[3] the smallest
// mismatching float / double encoding (~0 if none)
__global__ void __launch_bounds__(256) check_f64_kernel(unsigned long long* out) {
  unsigned long long bad = 0;
  const uint64_t n = uint64_t(1) << 32;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += uint64_t(gridDim.x) * blockDim.x) {
    const float f = __uint_as_float(uint32_t(i));
    const double mine = sun::to_f64(f), hw = double(f);
    if (__double_as_longlong(mine) != __double_as_longlong(hw)) {
      ++bad;
      atomicMin(&out[2], (unsigned long long)i);
    }
  }
  if (bad) atomicAdd(&out[0], bad);
}

// the double encoding number i of the seeded set
__device__ __forceinline__ uint64_t double_case(uint64_t seed, uint64_t i) {
  const uint64_t r = splitmix64(seed * 0x100000001B3ull + i);
  const uint64_t r2 = splitmix64(r ^ 0xD1B54A32D192ED03ull);
  const uint64_t sign = r & 0x8000000000000000ull;
  const uint64_t frac = r2 & 0x000FFFFFFFFFFFFFull;
  switch (i & 3u) {
    case 0:  // any encoding
      return r;
    case 1: {  // exponent 880 .. 1167: below, across and above the float's normal range
      const uint64_t e = 880u + (r2 >> 55) % 288u;
      return sign | (e << 52) | frac;
    }
    case 2: {  // the 29 dropped bits at a rounding boundary, exponent in or next to the normal range
      // exactly half an ulp (3 of 8 draws), one bit either side of it, and the extremes
      const uint32_t k = uint32_t(r >> 8) & 7u;
      const uint32_t low = k == 0u ? 0u
                         : k == 1u ? 1u
                         : k == 2u ? 0x0FFFFFFFu
                         : k == 3u ? 0x10000001u
                         : k == 4u ? 0x1FFFFFFFu
                                   : 0x10000000u;
      const uint64_t e = 894u + (r >> 40) % 260u;
      return sign | (e << 52) | (frac & ~uint64_t(0x1FFFFFFFu)) | low;
    }
    default: {  // the largest and smallest float exponents with fractions near all ones / zero
      const uint64_t e = (r >> 20) & 1u ? 1150u : 897u;
      const uint64_t f = (r >> 21) & 1u ? (0x000FFFFFFFFFFFFFull ^ (r2 & 0x3FFFFFFFull)) : (r2 & 0x3FFFFFFFull);
      return sign | (e << 52) | f;
    }
  }
}

__global__ void __launch_bounds__(256) check_f32_kernel(uint64_t n, uint64_t seed, unsigned long long* out) {
  unsigned long long bad = 0;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t bits = double_case(seed, i);
    const double d = __longlong_as_double((long long)bits);
    const float mine = sun::to_f32(d), hw = float(d);
    if (__float_as_uint(mine) != __float_as_uint(hw)) {
      ++bad;
      atomicMin(&out[3], (unsigned long long)bits);
    }
  }
  if (bad) atomicAdd(&out[1], bad);
}

sun_status selftest_fail(sun_status s, const char* msg) {
  sun::set_last_error_message(msg);
  return s;
}

}  // namespace

extern "C" sun_status sun_selftest_conversions(uint64_t n, uint64_t seed, uint64_t result[4]) {
  if (!result) return selftest_fail(SUN_ERR_ARG, "NULL argument");
  int sms = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess) {
    cudaGetLastError();
    return selftest_fail(SUN_ERR_CUDA, "no current CUDA device");
  }
  unsigned long long* out = nullptr;
  if (cudaMalloc(&out, 4 * sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    return selftest_fail(SUN_ERR_CUDA, "cudaMalloc of 32 bytes failed");
  }
  const unsigned long long init[4] = {0ull, 0ull, ~0ull, ~0ull};
  cudaError_t e = cudaMemcpy(out, init, sizeof(init), cudaMemcpyHostToDevice);
  const unsigned grid = unsigned(sms > 0 ? 8 * sms : 1024);
  if (e == cudaSuccess) {
    check_f64_kernel<<<grid, 256>>>(out);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && n > 0) {
    check_f32_kernel<<<grid, 256>>>(n, seed, out);
    e = cudaGetLastError();
  }
  unsigned long long host[4] = {0ull, 0ull, 0ull, 0ull};
  if (e == cudaSuccess) e = cudaMemcpy(host, out, sizeof(host), cudaMemcpyDeviceToHost);
  cudaFree(out);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return selftest_fail(SUN_ERR_CUDA, cudaGetErrorString(e));
  }
  for (int k = 0; k < 4; ++k) result[k] = uint64_t(host[k]);
  return SUN_OK;
}
