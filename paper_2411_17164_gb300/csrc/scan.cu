// Exclusive prefix sums (int32/int64 -> int64) used to turn per-row counts into
// CSR offsets.  Three-phase: per-block scan, recursive scan of block totals,
// add-back.  Deterministic (integer arithmetic).
#include "common.cuh"

namespace xmgn {

namespace {
constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

template <class T>
__global__ void scan_tile_kernel(const T* __restrict__ in, int64_t* __restrict__ out, int64_t n,
                                 int64_t* __restrict__ tile_sums, int write_total) {
  __shared__ int64_t warp_tot[kScanThreads / 32];
  const int64_t base = int64_t(blockIdx.x) * kScanTile;
  int64_t v[kScanItems];
  int64_t run = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    int64_t idx = base + int64_t(threadIdx.x) * kScanItems + i;
    v[i] = idx < n ? int64_t(in[idx]) : 0;
    run += v[i];
  }
  // inclusive warp scan of per-thread totals
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int64_t x = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[wid] = x;
  __syncthreads();
  int64_t warp_off = 0;
  for (int w = 0; w < wid; ++w) warp_off += warp_tot[w];
  int64_t excl = warp_off + x - run;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    int64_t idx = base + int64_t(threadIdx.x) * kScanItems + i;
    if (idx < n) out[idx] = excl;
    excl += v[i];
  }
  if (threadIdx.x == kScanThreads - 1) {
    if (tile_sums) tile_sums[blockIdx.x] = excl;
    if (write_total) out[n] = excl;
  }
}

__global__ void scan_add_kernel(int64_t* __restrict__ out, int64_t n,
                                const int64_t* __restrict__ offs, int64_t ntiles) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x)
    out[i] += offs[i / kScanTile];
  if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = offs[ntiles];
}

template <class T>
xmgn_status scan_impl(const T* in, int64_t* out, int64_t n, int64_t* tmp, cudaStream_t s) {
  if (n <= 0) {
    XMGN_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
    return XMGN_OK;
  }
  int64_t nt = (n + kScanTile - 1) / kScanTile;
  if (nt == 1) {
    scan_tile_kernel<T><<<1, kScanThreads, 0, s>>>(in, out, n, nullptr, 1);
    XMGN_LAUNCH_CHECK();
    return XMGN_OK;
  }
  int64_t* sums = tmp;
  int64_t* offs = tmp + nt;
  scan_tile_kernel<T><<<unsigned(nt), kScanThreads, 0, s>>>(in, out, n, sums, 0);
  XMGN_LAUNCH_CHECK();
  XMGN_TRY(scan_impl<int64_t>(sums, offs, nt, tmp + 2 * nt + 1, s));
  scan_add_kernel<<<grid_for(n, 256), 256, 0, s>>>(out, n, offs, nt);
  XMGN_LAUNCH_CHECK();
  return XMGN_OK;
}
}  // namespace

size_t scan_tmp_elems(int64_t n) {
  int64_t nt = (n + kScanTile - 1) / kScanTile;
  if (nt <= 1) return 1;
  return size_t(2 * nt + 1) + scan_tmp_elems(nt);
}

xmgn_status exclusive_scan_i32(const int32_t* in, int64_t* out, int64_t n, int64_t* tmp,
                               cudaStream_t s) {
  return scan_impl<int32_t>(in, out, n, tmp, s);
}
xmgn_status exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* tmp,
                               cudaStream_t s) {
  return scan_impl<int64_t>(in, out, n, tmp, s);
}

}  // namespace xmgn
