// Tensor-core products of the wide BF16 path (hidden width > 128, the paper's
// production width 512): at those widths one 128-row tile's accumulator fills
// TMEM and a weight matrix no longer fits in shared memory, so the fused
// one-CTA-per-tile kernels do not apply.  The wide path keeps the layer
// structure of the FP32 plain path (gathered rows, LayerNorm and segmented-sum
// kernels, fp32 activations) and runs its products on this project's
// tcgen05 GEMMs (wgemm.cu: TMA-fed, warp-specialised, TMEM accumulators) with
// bf16 operands and fp32 accumulation.  The operands are bf16 copies in
// scratch, each made once and reused by every product that reads it (the
// gathered MLP input by X W1 and by the gradient Xᵀ dZ1); every copy of width
// w is stored with leading dimension pad8(w) (zeros in the padding), the
// 16-byte row pitch that TMA needs.  The elementwise work after a product runs
// in fp32: the bias + SiLU epilogue writes A1 straight in bf16 for the next
// product, the SiLU' kernel writes dZ1 in bf16 together with the partial
// column sums of its fp32 values (the first bias gradient), and the products
// that feed fp32 gradients (dZ1 W1ᵀ blocks) store into or add to their
// outputs from the GEMM itself.
#include "model.cuh"
#include "wgemm.cuh"

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
    for (int k = k0 + lane; k < ldo; k += 32) out[r * ldo + k] = __float2bfloat16_rn(0.f);  // row padding
  }
}

// SiLU and its derivative with the fast exponential and division (their
// error is far below the bf16 rounding the results go through; a huge
// denominator gives 0, the correct limit).
__device__ __forceinline__ float silu(float z) { return __fdividef(z, 1.f + __expf(-z)); }
__device__ __forceinline__ float silu_grad(float z) {
  const float s = __fdividef(1.f, 1.f + __expf(-z));
  return s * (1.f + z * (1.f - s));
}

__device__ __forceinline__ float epi_one(float z, int epi, float* pre_el, float aux_el, const float* dst) {
  if (epi == EPI_SILU) {
    if (pre_el) *pre_el = z;
    return silu(z);
  }
  if (epi == EPI_ACCUM) return *dst + z;
  if (epi == EPI_SILU_GRAD) return z * silu_grad(aux_el);
  return z;
}

// C = epi(acc (+ bias)), acc dense [M, N] fp32; C (fp32, ld ldc) and C16
// (bf16, ld N) are each optional; pre and aux share C's leading dimension.
// Four columns per lane when N and ldc are multiples of 4 (16-byte accesses).
__global__ void epilogue_kernel(const float* __restrict__ acc, int64_t M, int N, const float* __restrict__ bias,
                                float* __restrict__ C, int64_t ldc, int epi, float* __restrict__ pre,
                                const float* __restrict__ aux, bf16* __restrict__ C16) {
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
        const int64_t at = r * ldc + c;
        float* pe = pre ? pre + at : nullptr;
        const float* dst = C ? C + at : nullptr;
        float4 ax = make_float4(0.f, 0.f, 0.f, 0.f);
        if (epi == EPI_SILU_GRAD) ax = *reinterpret_cast<const float4*>(aux + at);
        float4 o;
        o.x = epi_one(z.x, epi, pe, ax.x, dst);
        o.y = epi_one(z.y, epi, pe ? pe + 1 : nullptr, ax.y, dst ? dst + 1 : nullptr);
        o.z = epi_one(z.z, epi, pe ? pe + 2 : nullptr, ax.z, dst ? dst + 2 : nullptr);
        o.w = epi_one(z.w, epi, pe ? pe + 3 : nullptr, ax.w, dst ? dst + 3 : nullptr);
        if (C) *reinterpret_cast<float4*>(C + at) = o;
        if (C16) *reinterpret_cast<uint2*>(C16 + r * N + c) = bf16x4(o);
      }
    } else {
      for (int c = lane; c < N; c += 32) {
        const int64_t at = r * ldc + c;
        const float o = epi_one(acc[r * N + c] + (bias ? bias[c] : 0.f), epi, pre ? pre + at : nullptr,
                                epi == EPI_SILU_GRAD ? aux[at] : 0.f, C ? C + at : nullptr);
        if (C) C[at] = o;
        if (C16) C16[r * N + c] = __float2bfloat16_rn(o);
      }
    }
  }
}

// SiLU' epilogue fused with the column sums of its output (the first
// layer's bias gradient): the rows in contiguous chunks of rpc, a block per
// chunk and a warp per row within it.  dZ1 = acc * silu'(Z1) is written in
// bf16 only; each lane sums its four columns per 128, and the eight warps'
// sums are added in order into the block's partial row.  N % 4 == 0, N <= 512.
__global__ void __launch_bounds__(256) silu_grad_colsum_kernel(const float* __restrict__ acc, int64_t M, int N,
                                                               const float* __restrict__ Z1, bf16* __restrict__ C16,
                                                               int64_t rpc, float* __restrict__ part) {
  __shared__ float red[8][512];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  float cs[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) cs[k] = 0.f;
  const int64_t r0 = int64_t(blockIdx.x) * rpc, r1 = min(M, r0 + rpc);
  for (int64_t r = r0 + wib; r < r1; r += 8) {
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int c = 4 * lane + 128 * t;
      if (c < N) {
        const float4 z = *reinterpret_cast<const float4*>(acc + r * N + c);
        const float4 ax = *reinterpret_cast<const float4*>(Z1 + r * N + c);
        float4 o;
        o.x = z.x * silu_grad(ax.x);
        o.y = z.y * silu_grad(ax.y);
        o.z = z.z * silu_grad(ax.z);
        o.w = z.w * silu_grad(ax.w);
        *reinterpret_cast<uint2*>(C16 + r * N + c) = bf16x4(o);
        cs[4 * t] += o.x, cs[4 * t + 1] += o.y, cs[4 * t + 2] += o.z, cs[4 * t + 3] += o.w;
      }
    }
  }
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int c = 4 * lane + 128 * t;
    if (c < N) {
#pragma unroll
      for (int k = 0; k < 4; ++k) red[wib][c + k] = cs[4 * t + k];
    }
  }
  __syncthreads();
  for (int c = threadIdx.x; c < N; c += blockDim.x) {
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += red[w][c];
    part[int64_t(blockIdx.x) * N + c] = t;
  }
}

unsigned blocks(int64_t rows) { return grid_for(rows * 32, 256, int64_t(num_sms()) * 16); }  // a warp per row

}  // namespace

namespace {
size_t slot(int64_t rows, int cols, size_t elem) { return (size_t(rows) * size_t(cols) * elem + 255) & ~size_t(255); }
}  // namespace

int pad8(int w) { return (w + 7) & ~7; }

size_t wide_scratch_bytes(int64_t R, int H, int Kmax, int out) {
  const int Ho = H > out ? H : pad8(out), Kp = pad8(Kmax);
  return slot(R, Kp, 2) + slot(R, H, 2) + slot(R, Ho, 2) + slot(R, H, 2) + slot(Kp, H, 2) + slot(H, Ho, 2) +
         slot(R, Ho, 4) + slot(wg_part_elems(), 1, 4) + 256;
}

WideScratch wide_scratch(void* p, int64_t R, int H, int Kmax, int out) {
  const int Ho = H > out ? H : pad8(out);
  Kmax = pad8(Kmax);
  char* q = static_cast<char*>(p);
  q = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(q) + 255) & ~uintptr_t(255));
  WideScratch w;
  w.x = reinterpret_cast<bf16*>(q);
  q += slot(R, Kmax, 2);
  w.a1 = reinterpret_cast<bf16*>(q);
  q += slot(R, H, 2);
  w.dz2 = reinterpret_cast<bf16*>(q);
  q += slot(R, Ho, 2);
  w.dz1 = reinterpret_cast<bf16*>(q);
  q += slot(R, H, 2);
  w.w1 = reinterpret_cast<bf16*>(q);
  q += slot(Kmax, H, 2);
  w.w2 = reinterpret_cast<bf16*>(q);
  q += slot(H, Ho, 2);
  w.acc = reinterpret_cast<float*>(q);
  q += slot(R, Ho, 4);
  w.part = reinterpret_cast<float*>(q);
  return w;
}

xmgn_status wide_gather(const RowSrc& A, int64_t M, bf16* out, cudaStream_t s) {
  if (M <= 0) return XMGN_OK;
  gather_bf16_kernel<<<blocks(M), 256, 0, s>>>(A, M, out, pad8(A.K));
  XMGN_LAUNCH_CHECK();
  return XMGN_OK;
}

xmgn_status wide_round(const float* X, int64_t M, int N, int64_t ld, bf16* out, cudaStream_t s) {
  return wide_gather(rows1(X, ld, N), M, out, s);
}

xmgn_status wide_nn(const bf16* A, int64_t M, int K, const bf16* B, int N, float* acc, cudaStream_t s) {
  return wg_gemm(WG_NN, A, pad8(K), B, pad8(N), M, N, K, acc, N, false, s);
}

xmgn_status wide_nn_silu(const bf16* A, int64_t M, int K, const bf16* B, int N, const float* bias, bf16* a1,
                         cudaStream_t s, float* pre) {
  return wg_gemm_silu(A, pad8(K), B, pad8(N), M, N, K, bias, a1, pad8(N), s, pre, N);
}

xmgn_status wide_nt(const bf16* A, int64_t M, int K, const bf16* B, int N, float* acc, cudaStream_t s) {
  return wg_gemm(WG_NT, A, pad8(K), B, pad8(K), M, N, K, acc, N, false, s);
}

xmgn_status wide_tn(const bf16* A, int64_t M, int K1, const bf16* B, int N, float* G, float* part, cudaStream_t s) {
  return wg_gemm_tn(A, pad8(K1), B, pad8(N), M, K1, N, G, part, s);
}

xmgn_status wide_epilogue(const float* acc, int64_t M, int N, const float* bias, float* C, int64_t ldc, int epi,
                          float* pre, const float* aux, bf16* C16, cudaStream_t s) {
  if (M <= 0) return XMGN_OK;
  epilogue_kernel<<<blocks(M), 256, 0, s>>>(acc, M, N, bias, C, ldc, epi, pre, aux, C16);
  XMGN_LAUNCH_CHECK();
  return XMGN_OK;
}

xmgn_status wide_silu_grad_colsum(const float* acc, int64_t M, int N, const float* Z1, bf16* C16, float* db,
                                  float* part, cudaStream_t s) {
  if (N % 4 || N > 512) return fail(XMGN_ERR_UNSUPPORTED, "fused SiLU' column sums need N %% 4 == 0, N <= 512");
  const int nb = colsum_chunk_count(M);
  int64_t rpc = (M + nb - 1) / nb;
  if (rpc < 1) rpc = 1;
  silu_grad_colsum_kernel<<<nb, 256, 0, s>>>(acc, M, N, Z1, C16, rpc, part);
  XMGN_LAUNCH_CHECK();
  return sum_parts_f32(part, nb, N, db, s);
}

xmgn_status wide_nt_into(const bf16* A, int64_t M, int K, const bf16* B, int N, float* C, int64_t ldc, bool accum,
                         cudaStream_t s) {
  return wg_gemm(WG_NT, A, pad8(K), B, pad8(K), M, N, K, C, ldc, accum, s);
}

}  // namespace xmgn
