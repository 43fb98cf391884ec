// Device helpers shared by the single-LP and batched CUDA paths.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <stdexcept>
#include <string>

namespace gb300lp {

struct CudaError : std::runtime_error {
  cudaError_t code;
  CudaError(cudaError_t c, const char *what, int line)
      : std::runtime_error(std::string(what) + " failed at line " + std::to_string(line) + ": " +
                           cudaGetErrorString(c)),
        code(c) {}
};

struct DeviceOOM : std::runtime_error {
  explicit DeviceOOM(const std::string &w) : std::runtime_error(w) {}
};

#define CK(call)                                               \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) throw ::gb300lp::CudaError(e_, #call, __LINE__); \
  } while (0)

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

// clamp that propagates NaN (comparisons with NaN are false)
__device__ __forceinline__ double clampd(double v, double lo, double hi) {
  return v < lo ? lo : (v > hi ? hi : v);
}

// sum_i (v^+ lo - v^- hi) term with 0 * inf := 0
__device__ __forceinline__ double support_term(double v, double lo, double hi) {
  return v > 0.0 ? v * lo : (v < 0.0 ? v * hi : 0.0);
}

}  // namespace gb300lp
