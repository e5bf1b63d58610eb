// Tensor-core (tcgen05) building blocks of the BF16 path that are not fused
// MLPs: weight-image packing, a row-tiled GEMM  D = A B  (node projections,
// dh += S W^T) and the reduction-over-rows GEMM  G = X^T Y  (node-level weight
// gradients).  One CTA of 128 threads per SM, persistent over 128-row tiles,
// operands staged in 128-byte-swizzled shared memory, accumulators in TMEM.
#pragma once

#include <vector>

#include "model.cuh"
#include "tc.cuh"

namespace xmgn {

using bf16 = __nv_bfloat16;

// A packed weight image: the shared-memory image of a K-major B operand
// (R rows = output features, C columns = input features, bf16, swizzled).
struct Img {
  size_t off = 0;    // byte offset inside the image buffer
  uint32_t R = 0, C = 0;
  uint32_t bytes() const { return R * C * 2u; }
};

// A packing job: rows [r0, r0+nr) of image `img` from W (row-major
// [in][out], ld): element (r, c) = W[(wk0 + c) * ld + wn0 + (r - r0)] for
// c < kvalid and r - r0 < nvalid, else 0.  With lo the image holds the
// rounding residual bf16(W - bf16(W)), so that W_hi + W_lo represents W to
// about 16 significant bits.
struct PackJob {
  uint8_t* dst;
  const float* W;
  int64_t ld, wk0, wn0;
  uint32_t R, C, r0, nr, nvalid, kvalid;
  int lo;
};
constexpr int kPackBatch = 24;  // images per launch
PackJob pack_job(uint8_t* base, const Img& img, uint32_t r0, uint32_t nr, uint32_t nvalid, uint32_t kvalid,
                 const float* W, int64_t ld, int64_t wk0, int64_t wn0, bool lo = false);
// Packs all jobs, kPackBatch images per launch.
xmgn_status pack_images(const std::vector<PackJob>& jobs, cudaStream_t s);

// A row source of the tensor-core kernels: up to two bf16 segments of
// contiguous rows, each `w` columns (multiple of 64) wide.
struct Bf16Rows {
  const bf16* p0 = nullptr;
  int64_t ld0 = 0;
  int w0 = 0;
  const bf16* p1 = nullptr;
  int64_t ld1 = 0;
  int w1 = 0;
  __host__ __device__ int K() const { return w0 + w1; }
};

// D[M, N] (=|+=) A[M, K] * B  where B is the image `img` used K-major
// (img.R = N, img.C = K) or, if b_mn, MN-major (img.R = K, img.C = N).
// With D null the product is rounded to bf16 and written to D16 instead.
xmgn_status tc_gemm(const Bf16Rows& A, int64_t M, const uint8_t* img_base, const Img& img, bool b_mn,
                    int N, float* D, int64_t ldd, bool accumulate, cudaStream_t s, bf16* D16 = nullptr);

// G = X^T Y summed over M rows; X has K1 columns (128 or 256), Y has N
// columns (64..256).  Result element (k, n), for k < kvalid and n < nvalid,
// lands in out[((n / nsplit) * K1 + k) * nsplit + n % nsplit] (written, not
// added).  `part` needs tc_gemm_tn_part_elems floats.
size_t tc_gemm_tn_part_elems(int K1, int N);
xmgn_status tc_gemm_tn(const Bf16Rows& X, const bf16* Y, int64_t ldy, int N, int64_t M, float* out,
                       int kvalid, int nvalid, int nsplit, float* part, cudaStream_t s);

int tc_grid(int64_t tiles);

// Opts a kernel into the largest dynamic shared memory the device allows
// next to the kernel's static shared memory.
template <class K>
xmgn_status allow_max_smem(K kernel) {
  int dev = 0, optin = 0;
  XMGN_CUDA(cudaGetDevice(&dev));
  XMGN_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  cudaFuncAttributes fa;
  XMGN_CUDA(cudaFuncGetAttributes(&fa, kernel));
  XMGN_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin - int(fa.sharedSizeBytes)));
  return XMGN_OK;
}

}  // namespace xmgn
