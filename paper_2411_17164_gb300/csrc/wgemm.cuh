// Hand-written tcgen05 GEMMs of the wide BF16 path (see wgemm.cu).
#pragma once

#include <cuda.h>

#include "common.cuh"

namespace xmgn {

// Tensor map of an fp32 [rows, cols] array with leading dimension ld (a
// multiple of 4, 16-byte aligned base) for epilogue stores and reduce-adds:
// boxes of 32 columns x 128 rows in the 128-byte swizzle (a staged box is
// row r's 128 bytes with 16-byte chunk q at position q ^ (r mod 8)).
xmgn_status f32_map(CUtensorMap* m, float* p, int64_t rows, int64_t cols, int64_t ld);

enum WgMode : int { WG_NN = 0, WG_NT = 1, WG_TN = 2 };

// D[M, N] (=|+=) A[M, K] B, with B [K, N] (WG_NN) or [N, K] (WG_NT); bf16
// operands, leading dimensions lda, ldb multiples of 8, 16-byte aligned
// bases; fp32 D with leading dimension ldd; N <= 512.
xmgn_status wg_gemm(int mode, const __nv_bfloat16* A, int64_t lda, const __nv_bfloat16* B, int64_t ldb, int64_t M,
                    int N, int K, float* D, int64_t ldd, bool accum, cudaStream_t s);
// As WG_NN with the first MLP layer's epilogue in the GEMM: c16 = bf16(SiLU(A B
// + bias)) (bias [N]; c16 leading dimension ld16, a multiple of 8); with pre
// (fp32, leading dimension ldp, a multiple of 4) the pre-activation A B + bias
// is stored too, else the fp32 product is never stored.
xmgn_status wg_gemm_silu(const __nv_bfloat16* A, int64_t lda, const __nv_bfloat16* B, int64_t ldb, int64_t M, int N,
                         int K, const float* bias, __nv_bfloat16* c16, int64_t ld16, cudaStream_t s,
                         float* pre = nullptr, int64_t ldp = 0);
// G[K1, N] = A[M, K1]^T B[M, N] (written, dense), summed over the M rows by
// row-range splits whose partial tiles (part: wg_part_elems floats) are then
// added in split order.
xmgn_status wg_gemm_tn(const __nv_bfloat16* A, int64_t lda, const __nv_bfloat16* B, int64_t ldb, int64_t M, int K1,
                       int N, float* G, float* part, cudaStream_t s);
int64_t wg_part_elems();

}  // namespace xmgn
