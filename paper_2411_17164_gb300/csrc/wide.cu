// Tensor-core GEMMs of the wide BF16 path (hidden width > 128, the paper's
// production width 512): at those widths one 128-row tile's accumulator fills
// TMEM and a weight matrix no longer fits in shared memory, so the fused
// one-CTA-per-tile kernels do not apply.  The wide path keeps the layer
// structure of the FP32 plain path (gathered rows, LayerNorm and segmented-sum
// kernels, fp32 activations) and runs its three GEMM shapes as plain library
// GEMMs on the tensor cores: operands rounded to bf16 (the gathered rows
// materialised once per product), fp32 accumulation, then an elementwise
// epilogue (bias, SiLU, residual accumulation, SiLU') in fp32.
#include <cublas_v2.h>

#include <mutex>

#include "model.cuh"

namespace xmgn {

namespace {

// One warp per row (grid-stride over rows), lanes across the columns: no
// index division, coalesced loads and stores.
__device__ __forceinline__ int64_t warp_id() { return (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; }
__device__ __forceinline__ int64_t warp_count() { return (int64_t(gridDim.x) * blockDim.x) >> 5; }

__device__ __forceinline__ uint2 bf16x4(float4 v) {
  __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
  return make_uint2(*reinterpret_cast<uint32_t*>(&a), *reinterpret_cast<uint32_t*>(&b));
}

// out[r, :] = bf16 of row r of the segmented source A, leading dimension ldo;
// segments whose width, leading dimension and offsets are multiples of 4 move
// four values per lane (16-byte loads, 8-byte stores).
__global__ void gather_bf16_kernel(RowSrc A, int64_t M, bf16* __restrict__ out, int64_t ldo) {
  const int lane = threadIdx.x & 31;
  for (int64_t r = warp_id(); r < M; r += warp_count()) {
    int k0 = 0;
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      if (s < A.nseg) {
        const RowSeg& g = A.s[s];
        const float* src = g.p + (g.idx ? int64_t(g.idx[r]) : r) * g.ld;
        bf16* dst = out + r * ldo + k0;
        const bool vec = ((g.width | g.ld | k0 | ldo) & 3) == 0 && (reinterpret_cast<uintptr_t>(g.p) & 15) == 0;
        if (vec) {
          for (int k = 4 * lane; k < g.width; k += 128)
            *reinterpret_cast<uint2*>(dst + k) = bf16x4(*reinterpret_cast<const float4*>(src + k));
        } else {
          for (int k = lane; k < g.width; k += 32) dst[k] = __float2bfloat16_rn(src[k]);
        }
        k0 += g.width;
      }
    }
  }
}

// out[r, c] = bf16(X[r * ld + c]) for a dense fp32 matrix [M, N].
__global__ void dense_bf16_kernel(const float* __restrict__ X, int64_t M, int N, int64_t ld, bf16* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  for (int64_t r = warp_id(); r < M; r += warp_count())
    for (int c = lane; c < N; c += 32) out[r * N + c] = __float2bfloat16_rn(X[r * ld + c]);
}

__device__ __forceinline__ float silu(float z) { return z / (1.f + expf(-z)); }
__device__ __forceinline__ float silu_grad(float z) {
  const float s = 1.f / (1.f + expf(-z));
  return s * (1.f + z * (1.f - s));
}

__device__ __forceinline__ float epi_one(float z, int epi, float* pre_el, float aux_el, float* dst) {
  if (epi == EPI_SILU) {
    if (pre_el) *pre_el = z;
    return silu(z);
  }
  if (epi == EPI_ACCUM) return *dst + z;
  if (epi == EPI_SILU_GRAD) return z * silu_grad(aux_el);
  return z;
}

// C = epi(acc (+ bias)), acc dense [M, N] fp32; four columns per lane when
// N and ldc are multiples of 4 (16-byte accesses).
__global__ void epilogue_kernel(const float* __restrict__ acc, int64_t M, int N, const float* __restrict__ bias,
                                float* __restrict__ C, int64_t ldc, int epi, float* __restrict__ pre,
                                const float* __restrict__ aux) {
  const int lane = threadIdx.x & 31;
  const bool vec = ((N | ldc) & 3) == 0;
  for (int64_t r = warp_id(); r < M; r += warp_count()) {
    if (vec) {
      for (int c = 4 * lane; c < N; c += 128) {
        float4 z = *reinterpret_cast<const float4*>(acc + r * N + c);
        if (bias) {
          const float4 b = *reinterpret_cast<const float4*>(bias + c);
          z.x += b.x, z.y += b.y, z.z += b.z, z.w += b.w;
        }
        float* dst = C + r * ldc + c;
        float* pe = pre ? pre + r * ldc + c : nullptr;
        float4 ax = make_float4(0.f, 0.f, 0.f, 0.f);
        if (epi == EPI_SILU_GRAD) ax = *reinterpret_cast<const float4*>(aux + r * ldc + c);
        float4 o;
        o.x = epi_one(z.x, epi, pe ? pe : nullptr, ax.x, dst);
        o.y = epi_one(z.y, epi, pe ? pe + 1 : nullptr, ax.y, dst + 1);
        o.z = epi_one(z.z, epi, pe ? pe + 2 : nullptr, ax.z, dst + 2);
        o.w = epi_one(z.w, epi, pe ? pe + 3 : nullptr, ax.w, dst + 3);
        *reinterpret_cast<float4*>(dst) = o;
      }
    } else {
      for (int c = lane; c < N; c += 32) {
        float* dst = C + r * ldc + c;
        *dst = epi_one(acc[r * N + c] + (bias ? bias[c] : 0.f), epi, pre ? pre + r * ldc + c : nullptr,
                       epi == EPI_SILU_GRAD ? aux[r * ldc + c] : 0.f, dst);
      }
    }
  }
}

// Split epilogue: columns [q*W, (q+1)*W) of acc [M, nseg*W] go to out[q]
// (store or accumulate), four columns per lane.
__global__ void split_epilogue_kernel(const float* __restrict__ acc, int64_t M, int W, WideOut o) {
  const int lane = threadIdx.x & 31;
  const int N = o.n * W;
  for (int64_t r = warp_id(); r < M; r += warp_count()) {
    for (int c = 4 * lane; c < N; c += 128) {
      const int q = c / W, cc = c - q * W;
      float4 z = *reinterpret_cast<const float4*>(acc + r * N + c);
      float4* d = reinterpret_cast<float4*>(o.C[q] + r * o.ldc[q] + cc);
      if (o.accum[q]) {
        const float4 p = *d;
        z.x += p.x, z.y += p.y, z.z += p.z, z.w += p.w;
      }
      *d = z;
    }
  }
}

struct Blas {
  std::mutex mu;
  cublasHandle_t h[64] = {};
};

Blas& blas() {
  static Blas b;
  return b;
}

xmgn_status handle(cudaStream_t s, cublasHandle_t* out) {
  int dev = 0;
  XMGN_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(XMGN_ERR_CUDA, "device id %d", dev);
  Blas& b = blas();
  std::lock_guard<std::mutex> g(b.mu);
  if (!b.h[dev]) {
    if (cublasCreate(&b.h[dev]) != CUBLAS_STATUS_SUCCESS) return fail(XMGN_ERR_CUDA, "cublasCreate failed");
  }
  if (cublasSetStream(b.h[dev], s) != CUBLAS_STATUS_SUCCESS) return fail(XMGN_ERR_CUDA, "cublasSetStream failed");
  *out = b.h[dev];
  return XMGN_OK;
}

unsigned blocks(int64_t rows) { return grid_for(rows * 32, 256, int64_t(num_sms()) * 16); }  // a warp per row

// Column-major C[m, n] = op(A) op(B), bf16 operands, fp32 accumulate and output.
xmgn_status gemm_ex(cudaStream_t s, cublasOperation_t ta, cublasOperation_t tb, int m, int n, int k, const bf16* A,
                    int lda, const bf16* B, int ldb, float* C, int ldc) {
  cublasHandle_t h;
  XMGN_TRY(handle(s, &h));
  const float one = 1.f, zero = 0.f;
  const cublasStatus_t st = cublasGemmEx(h, ta, tb, m, n, k, &one, A, CUDA_R_16BF, lda, B, CUDA_R_16BF, ldb, &zero,
                                         C, CUDA_R_32F, ldc, CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT);
  if (st != CUBLAS_STATUS_SUCCESS) return fail(XMGN_ERR_CUDA, "cublasGemmEx failed (%d)", int(st));
  return XMGN_OK;
}

}  // namespace

size_t wide_scratch_bytes(int64_t R, int H) {
  // gathered A (up to R x 3H bf16), second operand (R x H bf16 or the weight), fp32 accumulator R x 3H
  const size_t a = size_t(R) * 3 * H * 2, b = size_t(R) * 3 * H * 2, c = size_t(R) * 3 * H * 4;
  return a + b + c + 3 * 256;
}

WideScratch wide_scratch(void* p, int64_t R, int H) {
  char* q = static_cast<char*>(p);
  WideScratch w;
  w.a = reinterpret_cast<bf16*>(q);
  q += (size_t(R) * 3 * H * 2 + 255) & ~size_t(255);
  w.b = reinterpret_cast<bf16*>(q);
  q += (size_t(R) * 3 * H * 2 + 255) & ~size_t(255);
  w.acc = reinterpret_cast<float*>(q);
  return w;
}

xmgn_status gemm_nn_tc(const WideScratch& w, const RowSrc& A, int64_t M, const float* B, int N, const float* bias,
                       float* C, int64_t ldc, int epi, float* pre, const float* aux, cudaStream_t s) {
  if (M <= 0) return XMGN_OK;
  const int K = A.K;
  gather_bf16_kernel<<<blocks(M), 256, 0, s>>>(A, M, w.a, K);
  XMGN_LAUNCH_CHECK();
  dense_bf16_kernel<<<blocks(K), 256, 0, s>>>(B, K, N, N, w.b);
  XMGN_LAUNCH_CHECK();
  // row-major acc[M, N] = A[M, K] B[K, N]  <=>  column-major acc^T = B^T A^T
  XMGN_TRY(gemm_ex(s, CUBLAS_OP_N, CUBLAS_OP_N, N, int(M), K, w.b, N, w.a, K, w.acc, N));
  epilogue_kernel<<<blocks(M), 256, 0, s>>>(w.acc, M, N, bias, C, ldc, epi, pre, aux);
  XMGN_LAUNCH_CHECK();
  return XMGN_OK;
}

xmgn_status gemm_nt_tc(const WideScratch& w, const RowSrc& A, int64_t M, const float* B, int N, float* C, int64_t ldc,
                       int epi, const float* aux, cudaStream_t s) {
  if (M <= 0) return XMGN_OK;
  const int K = A.K;
  gather_bf16_kernel<<<blocks(M), 256, 0, s>>>(A, M, w.a, K);
  XMGN_LAUNCH_CHECK();
  dense_bf16_kernel<<<blocks(N), 256, 0, s>>>(B, N, K, K, w.b);
  XMGN_LAUNCH_CHECK();
  // row-major acc[M, N] = A[M, K] B[N, K]^T  <=>  column-major acc^T = B A^T (B^T stored, transposed)
  XMGN_TRY(gemm_ex(s, CUBLAS_OP_T, CUBLAS_OP_N, N, int(M), K, w.b, K, w.a, K, w.acc, N));
  epilogue_kernel<<<blocks(M), 256, 0, s>>>(w.acc, M, N, nullptr, C, ldc, epi, nullptr, aux);
  XMGN_LAUNCH_CHECK();
  return XMGN_OK;
}

xmgn_status gemm_nt_split_tc(const WideScratch& w, const RowSrc& A, int64_t M, const float* B, const WideOut& o,
                             cudaStream_t s) {
  if (M <= 0) return XMGN_OK;
  const int K = A.K, N = o.n * o.W;
  if (o.W % 4) return fail(XMGN_ERR_ARG, "split epilogue needs a width that is a multiple of 4");
  gather_bf16_kernel<<<blocks(M), 256, 0, s>>>(A, M, w.a, K);
  XMGN_LAUNCH_CHECK();
  dense_bf16_kernel<<<blocks(N), 256, 0, s>>>(B, N, K, K, w.b);
  XMGN_LAUNCH_CHECK();
  XMGN_TRY(gemm_ex(s, CUBLAS_OP_T, CUBLAS_OP_N, N, int(M), K, w.b, K, w.a, K, w.acc, N));
  split_epilogue_kernel<<<blocks(M), 256, 0, s>>>(w.acc, M, o.W, o);
  XMGN_LAUNCH_CHECK();
  return XMGN_OK;
}

xmgn_status gemm_tn_tc(const WideScratch& w, const RowSrc& A, int64_t M, const float* B, int64_t ldb, int N, float* G,
                       cudaStream_t s) {
  const int K1 = A.K;
  if (M <= 0) {
    XMGN_CUDA(cudaMemsetAsync(G, 0, sizeof(float) * size_t(K1) * N, s));
    return XMGN_OK;
  }
  gather_bf16_kernel<<<blocks(M), 256, 0, s>>>(A, M, w.a, K1);
  XMGN_LAUNCH_CHECK();
  dense_bf16_kernel<<<blocks(M), 256, 0, s>>>(B, M, N, ldb, w.b);
  XMGN_LAUNCH_CHECK();
  // row-major G[K1, N] = A[M, K1]^T B[M, N]  <=>  column-major G^T = B^T A (A^T stored, transposed)
  return gemm_ex(s, CUBLAS_OP_N, CUBLAS_OP_T, N, K1, int(M), w.b, N, w.a, K1, G, N);
}

}  // namespace xmgn
