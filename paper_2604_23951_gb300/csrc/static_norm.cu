// lp_power_norm_static: the power-iteration estimate of ||A||_2 that
// lp_solve uses for its step size, run entirely in a fixed, file-scope
// device buffer so that the call allocates no memory at all.
//
// Some callers cannot allocate device memory at the point where they need
// the estimate: a process that reserved all of the GPU's memory up front for
// its own pool, a latency-critical path where a cudaMalloc (which may
// synchronize the device or fail under fragmentation) is not allowed, or a
// host thread that must not call into an allocator it does not own.  They
// pass the matrix and its transpose already on the device and receive the
// estimate; the work vectors and partial sums live in g_norm_scratch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "layout.h"
#include "lp_internal.h"

namespace gb300lp {
void set_last_error(const std::string &m);
}

namespace {

// 2^20 doubles (8 MiB); every GPU that loads the library holds it until exit
constexpr long long kScratchDoubles = 1LL << 20;
constexpr int kSnBlock = 256;
constexpr int kSnMaxBlocks = 1024;  // partial-sum slots at the front of the array

static __device__ __align__(256) double g_norm_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
// per device: the context the address was looked up in, and the address
struct ScratchAddr {
  void *ctx = nullptr;
  double *ptr = nullptr;
};
ScratchAddr g_scratch[kMaxDevices];

// the calling thread's current CUDA context (through the driver entry point,
// so the library needs no link against the driver library), or nullptr when
// it cannot be queried
void *current_context() {
  using CtxGetCurrent = int (*)(void **);
  static CtxGetCurrent fn = []() -> CtxGetCurrent {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<CtxGetCurrent>(f);
  }();
  void *ctx = nullptr;
  if (!fn || fn(&ctx) != 0) return nullptr;
  return ctx;
}

// out[r] = sum_k val[k] * vec[col[k]] (one warp per row); with `partials`,
// each CTA also stores its sum of out[r]^2 in partials[blockIdx.x]
__global__ void k_sn_spmv(int rows, const int *__restrict__ rp, const int *__restrict__ ci,
                          const double *__restrict__ va, const double *__restrict__ vec,
                          double *__restrict__ out, double *partials) {
  __shared__ double red[kSnBlock / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double acc = 0.0;
  for (int r = blockIdx.x * (kSnBlock / 32) + warp; r < rows; r += gridDim.x * (kSnBlock / 32)) {
    double s = 0.0;
    for (int k = rp[r] + lane; k < rp[r + 1]; k += 32) s += va[k] * vec[ci[k]];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      out[r] = s;
      acc += s * s;
    }
  }
  if (partials) {
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < kSnBlock / 32; ++w) t += red[w];
      partials[blockIdx.x] = t;
    }
  }
}

// fixed-order sum of `nparts` partials, evaluated identically by every CTA
__device__ double sn_sum(const double *partials, int nparts) {
  __shared__ double red[kSnBlock / 32];
  __shared__ double total;
  double s = 0.0;
  for (int b = threadIdx.x; b < nparts; b += kSnBlock) s += partials[b];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kSnBlock / 32; ++w) t += red[w];
    total = t;
  }
  __syncthreads();
  return total;
}

// v = w / ||w||; a zero w continues from the fallback start vector
__global__ void k_sn_normalize(int n, const double *__restrict__ w, double *__restrict__ v,
                               const double *partials, int nparts) {
  const double nw = sqrt(sn_sum(partials, nparts));
  const double inv_sqrt_n = 1.0 / sqrt((double)n);
  for (int j = blockIdx.x * kSnBlock + threadIdx.x; j < n; j += gridDim.x * kSnBlock)
    v[j] = nw > 0.0 ? w[j] / nw : gb300lp::power_start(j, inv_sqrt_n);
}

__global__ void k_sn_fill(int n, double *v, double val) {
  for (int j = blockIdx.x * kSnBlock + threadIdx.x; j < n; j += gridDim.x * kSnBlock) v[j] = val;
}

__global__ void k_sn_final(const double *partials, int nparts, double *result) {
  const double s = sn_sum(partials, nparts);
  if (threadIdx.x == 0) *result = sqrt(s);
}

// The device address of g_norm_scratch for the current device.  It is
// looked up (cudaGetSymbolAddress, with that device current) on the first
// call per device and again whenever the device's current context has
// changed since (after a cudaDeviceReset the module, and so the array, is
// loaded afresh in a new context and the old address is stale).  If the
// context cannot be queried, it is looked up on every call.
double *scratch_for_device(int dev, std::string &err) {
  if (dev < 0 || dev >= kMaxDevices) {
    err = "device index out of range";
    return nullptr;
  }
  void *ctx = current_context();
  std::lock_guard<std::mutex> lk(g_mu);
  ScratchAddr &a = g_scratch[dev];
  if (!a.ptr || !ctx || a.ctx != ctx) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_norm_scratch);
    if (e != cudaSuccess) {
      err = std::string("cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
      return nullptr;
    }
    a.ptr = static_cast<double *>(p);
    // the lookup may have created the primary context: record the one in use
    a.ctx = ctx ? current_context() : nullptr;
  }
  return a.ptr;
}

}  // namespace

extern "C" int lp_power_norm_static(int32_t m, int32_t n, const int32_t *a_row_ptr,
                                    const int32_t *a_col_idx, const double *a_val,
                                    const int32_t *at_row_ptr, const int32_t *at_col_idx,
                                    const double *at_val, int32_t iters, void *stream,
                                    double *norm_out) {
  using gb300lp::set_last_error;
  if (!norm_out) {
    set_last_error("norm_out is NULL");
    return LP_ERR_INVALID;
  }
  if (m < 0 || n < 0 || iters < 0) {
    set_last_error("negative size or iteration count");
    return LP_ERR_INVALID;
  }
  const long long need = (long long)kSnMaxBlocks + 1 + 2LL * n + (long long)m;
  if (need > kScratchDoubles) {
    set_last_error("problem too large for the static scratch: need m + 2 n <= " +
                   std::to_string(kScratchDoubles - kSnMaxBlocks - 1) + ", got m + 2 n = " +
                   std::to_string(2LL * n + m));
    return LP_ERR_INVALID;
  }
  if (m == 0 || n == 0) {
    *norm_out = 0.0;
    return LP_OK;
  }
  if (!a_row_ptr || !a_col_idx || !a_val || !at_row_ptr || !at_col_idx || !at_val) {
    set_last_error("matrix pointer is NULL");
    return LP_ERR_INVALID;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_last_error(std::string("cudaGetDevice failed: ") + cudaGetErrorString(e));
    return LP_ERR_CUDA;
  }
  std::string err;
  double *base = scratch_for_device(dev, err);
  if (!base) {
    set_last_error(err);
    return LP_ERR_CUDA;
  }
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    set_last_error(std::string("cudaDeviceGetAttribute failed: ") + cudaGetErrorString(e));
    return LP_ERR_CUDA;
  }
  // layout: [partials (kSnMaxBlocks) | result (1) | v (n) | w (n) | u (m)]
  double *partials = base;
  double *result = base + kSnMaxBlocks;
  double *v = result + 1;
  double *w = v + n;
  double *u = w + n;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  auto rows_grid = [&](int rows) {
    long long g = ((long long)rows + kSnBlock / 32 - 1) / (kSnBlock / 32);
    return (int)std::max<long long>(1, std::min<long long>(g, std::min(kSnMaxBlocks, 4 * sms)));
  };
  const int gT = rows_grid(n), gA = rows_grid(m);
  const int gv = (int)std::max(1, std::min((n + kSnBlock - 1) / kSnBlock, 8 * sms));
  // every region read below is written earlier in this call (the array keeps
  // the previous call's contents)
  k_sn_fill<<<gv, kSnBlock, 0, s>>>(n, v, 1.0 / std::sqrt((double)n));
  for (int it = 0; it < iters; ++it) {
    k_sn_spmv<<<gA, kSnBlock, 0, s>>>(m, a_row_ptr, a_col_idx, a_val, v, u, nullptr);
    k_sn_spmv<<<gT, kSnBlock, 0, s>>>(n, at_row_ptr, at_col_idx, at_val, u, w, partials);
    k_sn_normalize<<<gv, kSnBlock, 0, s>>>(n, w, v, partials, gT);
  }
  k_sn_spmv<<<gA, kSnBlock, 0, s>>>(m, a_row_ptr, a_col_idx, a_val, v, u, partials);
  k_sn_final<<<1, kSnBlock, 0, s>>>(partials, gA, result);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(norm_out, result, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_last_error(std::string("CUDA error: ") + cudaGetErrorString(e));
    return LP_ERR_CUDA;
  }
  return LP_OK;
}
