// Masked MSE loss with its scratch in a file-scope device array, for callers
// that must not allocate device memory (see xmgn_mse_loss_static in
// include/xmgn.h).
//
// The regular loss inside xmgn_forward keeps its per-block partial sums in the
// caller's workspace.  This variant keeps them in `g_loss_partials` below, a
// fixed 16 KB array that every device loading the library holds until the
// process exits.  Host code cannot pass the array's name to a kernel (on the
// host it only names a host-side shadow), so its device address is looked up
// once per device with cudaGetSymbolAddress and cached.
#include <mutex>

#include "model.cuh"

namespace xmgn {
namespace {

constexpr int kStaticThreads = 256;
constexpr int kRowsPerThread = 4;
constexpr int64_t kRowsPerBlock = int64_t(kStaticThreads) * kRowsPerThread;  // 1024 rows
constexpr int kMaxPartials = 4096;  // one partial per block -> at most 4,194,304 rows
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float g_loss_partials[kMaxPartials];

std::mutex g_setup_mu;
float* g_partials_addr[kMaxDevices] = {nullptr};

// Device address of g_loss_partials on the current device (set up on first use).
xmgn_status partials_address(float** out) {
  int dev = 0;
  XMGN_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(XMGN_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> g(g_setup_mu);
  if (!g_partials_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_loss_partials);
    if (e != cudaSuccess || !p)
      return fail(XMGN_ERR_CUDA, "cudaGetSymbolAddress(loss scratch) failed: %s", cudaGetErrorString(e));
    g_partials_addr[dev] = static_cast<float*>(p);
  }
  *out = g_partials_addr[dev];
  return XMGN_OK;
}

// Block b writes the sum over its 1024 rows of the squared error of inner rows.
__global__ void __launch_bounds__(kStaticThreads) static_loss_partial_kernel(
    const float* __restrict__ y, int64_t n, int out, const float* __restrict__ t,
    const int32_t* __restrict__ gid, const uint8_t* __restrict__ hop, float* __restrict__ partials) {
  __shared__ float red[kStaticThreads];
  float s = 0.f;
  const int64_t base = int64_t(blockIdx.x) * kRowsPerBlock;
  for (int k = 0; k < kRowsPerThread; ++k) {
    const int64_t i = base + int64_t(k) * kStaticThreads + threadIdx.x;
    if (i >= n || (hop && hop[i] != 0)) continue;
    const int64_t g = gid ? int64_t(gid[i]) : i;
    for (int c = 0; c < out; ++c) {
      const float d = y[i * out + c] - t[g * out + c];
      s += d * d;
    }
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = kStaticThreads / 2; o; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

// One block adds partials[0..nb) in a fixed order and scales.
__global__ void __launch_bounds__(kStaticThreads) static_loss_final_kernel(const float* __restrict__ partials, int nb,
                                                                         float scale, float* __restrict__ loss) {
  __shared__ float red[kStaticThreads];
  float s = 0.f;
  for (int b = threadIdx.x; b < nb; b += kStaticThreads) s += partials[b];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = kStaticThreads / 2; o; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = red[0] * scale;
}

}  // namespace
}  // namespace xmgn

using namespace xmgn;

extern "C" xmgn_status xmgn_mse_loss_static(const float* y, int64_t n, int32_t out, const float* targets,
                                            const int32_t* gid, const uint8_t* hop, int64_t n_norm,
                                            float* loss, xmgn_stream stream) {
  if (!y || !targets || !loss) return fail(XMGN_ERR_ARG, "y, targets and loss are required");
  if (n < 1 || out < 1 || out > 16 || n_norm < 1) return fail(XMGN_ERR_ARG, "bad sizes (n=%lld out=%d n_norm=%lld)",
                                                              (long long)n, out, (long long)n_norm);
  const int64_t nb = (n + kRowsPerBlock - 1) / kRowsPerBlock;
  if (nb > kMaxPartials)
    return fail(XMGN_ERR_WORKSPACE,
                "xmgn_mse_loss_static handles at most %lld rows (its fixed scratch holds %d partial sums); got %lld",
                (long long)(int64_t(kMaxPartials) * kRowsPerBlock), kMaxPartials, (long long)n);
  float* partials = nullptr;
  XMGN_TRY(partials_address(&partials));
  cudaStream_t s = (cudaStream_t)stream;
  // every partial read below is written by this call first: nothing to clear
  static_loss_partial_kernel<<<unsigned(nb), kStaticThreads, 0, s>>>(y, n, out, targets, gid, hop, partials);
  XMGN_LAUNCH_CHECK();
  static_loss_final_kernel<<<1, kStaticThreads, 0, s>>>(partials, int(nb), 1.f / (float(out) * float(n_norm)), loss);
  XMGN_LAUNCH_CHECK();
  return XMGN_OK;
}
