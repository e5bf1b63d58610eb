// Parameter plan, graph view and the SIMT building blocks shared by the FP32
// and BF16 model paths.
#pragma once

#include <vector>

#include <cuda_bf16.h>

#include "common.cuh"

namespace xmgn {

constexpr float kLnEps = 1e-5f;
constexpr int kInEdge = 4;

// Offsets (in floats) of one MLP inside the packed parameter vector.
struct MlpOff {
  int64_t W1, b1, W2, b2, g, be;  // g/be = -1 when the MLP has no LayerNorm
  int in, hid, out;
  bool ln;
};

struct ParamPlan {
  MlpOff ne, ee, dec;
  std::vector<MlpOff> edge, node;
  int64_t total = 0;
  int H = 0, L = 0, in_node = 0, out = 0;
  int fourier = 0, in_enc = 0;  // Fourier frequencies; node-encoder inputs = in_node + 6 * fourier
};

inline MlpOff plan_mlp(int64_t& o, int in, int hid, int out, bool ln) {
  MlpOff m;
  m.in = in;
  m.hid = hid;
  m.out = out;
  m.ln = ln;
  m.W1 = o; o += int64_t(in) * hid;
  m.b1 = o; o += hid;
  m.W2 = o; o += int64_t(hid) * out;
  m.b2 = o; o += out;
  if (ln) {
    m.g = o; o += out;
    m.be = o; o += out;
  } else {
    m.g = m.be = -1;
  }
  return m;
}

inline ParamPlan make_plan(const xmgn_model_desc& d) {
  ParamPlan p;
  p.H = d.H;
  p.L = d.L;
  p.in_node = d.in_node;
  p.out = d.out;
  p.fourier = d.fourier;
  p.in_enc = d.in_node + 6 * d.fourier;
  int64_t o = 0;
  p.ne = plan_mlp(o, p.in_enc, d.H, d.H, true);
  p.ee = plan_mlp(o, kInEdge, d.H, d.H, true);
  for (int l = 0; l < d.L; ++l) {
    p.edge.push_back(plan_mlp(o, 3 * d.H, d.H, d.H, true));
    p.node.push_back(plan_mlp(o, 2 * d.H, d.H, d.H, true));
  }
  p.dec = plan_mlp(o, d.H, d.H, d.out, false);
  p.total = o;
  return p;
}

// ---------------------------------------------------------------- SIMT blocks
// Row source: row r of the virtual matrix is the concatenation of up to three
// segments; segment s contributes `width` floats from p + (idx ? idx[r] : r)*ld.
struct RowSeg {
  const float* p = nullptr;
  int64_t ld = 0;
  const int32_t* idx = nullptr;
  int width = 0;
};
struct RowSrc {
  RowSeg s[3];
  int nseg = 0;
  int K = 0;
};
inline RowSrc rows1(const float* p, int64_t ld, int w, const int32_t* idx = nullptr) {
  RowSrc r;
  r.s[0] = {p, ld, idx, w};
  r.nseg = 1;
  r.K = w;
  return r;
}
inline void rows_add(RowSrc& r, const float* p, int64_t ld, int w, const int32_t* idx = nullptr) {
  r.s[r.nseg++] = {p, ld, idx, w};
  r.K += w;
}

enum Epi : int {
  EPI_STORE = 0,      // C = acc + bias
  EPI_SILU = 1,       // C = silu(acc + bias); pre (optional) = acc + bias
  EPI_ACCUM = 2,      // C += acc + bias
  EPI_SILU_GRAD = 3,  // C = acc * silu'(aux)
};

// C[M,N] = A[M,K] * B[K,N]   (B row-major [K][N], e.g. a weight W[in][out])
xmgn_status gemm_nn_f32(const RowSrc& A, int64_t M, const float* B, int N, const float* bias,
                        float* C, int64_t ldc, int epi, float* pre, const float* aux,
                        cudaStream_t s);
// C[M,N] = A[M,K] * B^T      (B row-major [N][K]; dX = dZ W^T with W[in][out], N=in, K=out)
xmgn_status gemm_nt_f32(const RowSrc& A, int64_t M, const float* B, int N, float* C, int64_t ldc,
                        int epi, const float* aux, cudaStream_t s);
// G[K1,N] = A^T B over M rows, written (not added) into G (row-major, ld N);
// deterministic two-level reduction through `part` scratch.
size_t gemm_tn_part_elems(int64_t M, int K1, int N);
xmgn_status gemm_tn_f32(const RowSrc& A, int64_t M, const float* B, int64_t ldb, int N, float* G,
                        float* part, cudaStream_t s);
// Column sums in two levels: colsum_chunk_count(M) row chunks, each written as
// one partial row, then out[c] = the sum of the nb partial rows (fixed order).
int colsum_chunk_count(int64_t M);
xmgn_status sum_parts_f32(const float* part, int nb, int len, float* out, cudaStream_t s);
// g[N] = column sums of X[M,N] (ld), deterministic.
size_t colsum_part_elems(int64_t M, int N);
xmgn_status colsum_f32(const float* X, int64_t M, int N, int64_t ld, float* g, float* part,
                       cudaStream_t s);

// Y = LN(Z + bias) * gamma + beta (rows of N features; bias optional, added
// to every row).  If resid_out: resid_out = resid_in + Y (resid_in may alias
// resid_out).  Y may be null when only the residual output is wanted.
xmgn_status layernorm_fwd_f32(const float* Z, int64_t M, int N, const float* gamma,
                              const float* beta, float* Y, const float* resid_in,
                              float* resid_out, cudaStream_t s, const float* bias = nullptr);
// Edge form of layernorm_fwd_f32 fused with the receiver sums of eq. (2): the
// M = row_ptr[n] rows are edges in CSR order; resid_out = resid_in + Y for
// every row and agg[i] = the sum of Y over node i's rows in row order; Y
// itself is not stored.
xmgn_status layernorm_fwd_agg_f32(const float* Z, const float* bias, const int64_t* row_ptr, int64_t n, int N,
                                  const float* gamma, const float* beta, const float* resid_in, float* resid_out,
                                  float* agg, cudaStream_t s);
// LayerNorm backward at the input Z + bias (bias optional).
// dY(r) = dY1[r] + (dY2 ? dY2[idx2[r]] : 0); dZ = LN'(Z + bias)^T dY; dgamma,
// dbeta written (deterministic for a given device).
size_t ln_bwd_part_elems(int N);
xmgn_status layernorm_bwd_f32(const float* Z, int64_t M, int N, const float* gamma,
                              const float* dY1, const float* dY2, const int32_t* idx2, float* dZ,
                              float* dgamma, float* dbeta, float* part, cudaStream_t s,
                              const float* bias = nullptr);

// out[i] (+)= sum_{e in row i} v[e]            (receiver segments, CSR order)
xmgn_status seg_sum_rows_f32(const float* v, int64_t ldv, const int64_t* row_ptr, int64_t n, int H,
                             float* out, int64_t ldo, bool accumulate, cudaStream_t s);
// out[j] (+)= sum_{t in csc row j} v[perm[t]]  (sender segments)
xmgn_status seg_sum_cols_f32(const float* v, int64_t ldv, const int64_t* row_ptr,
                             const int32_t* perm, int64_t n, int H, float* out, int64_t ldo,
                             bool accumulate, cudaStream_t s);

// f[e] = (x_s - x_r, |x_s - x_r|) with x = xyz[gid[.]]
// Node-encoder input rows [n, in_node + 6*fourier] (inputs gathered by gid,
// then the Fourier features of the coordinates).
xmgn_status node_features(const float* node_in, int in_node, const float* xyz, const int32_t* gid, int64_t n,
                          int fourier, float* out, cudaStream_t s);
xmgn_status edge_features(const float* xyz, const int32_t* gid, const int32_t* recv,
                          const int32_t* col, int64_t E, float* f, cudaStream_t s);
// Masked MSE: loss (device scalar, written), dy[n,out] (nullable) =
// 2 (y - t[gid]) / (out * n_norm) on inner rows, 0 elsewhere; scatters inner
// rows of y into y_global[gid] (nullable).
size_t loss_part_elems(int64_t n);
xmgn_status mse_loss(const float* y, int64_t n, int out, const float* targets, const int32_t* gid,
                     const uint8_t* hop, int64_t n_norm, float* loss, float* dy, float* y_global,
                     float* part, cudaStream_t s);
// dst[i] += src[i] with Neumaier compensation in comp (comp nullable -> plain add)
xmgn_status accumulate_grad(float* dst, float* comp, const float* src, int64_t n, cudaStream_t s);

// ---------------------------------------------------------------- wide BF16 products
// The wide path (hidden width other than 128) runs its products on the tensor
// cores (this project's tcgen05 GEMMs, wgemm.cu) with bf16 operands and fp32
// accumulation and output.  Operands are bf16 copies kept in scratch and
// reused across the products of one MLP: the gathered input X (for X W1 and
// for Xᵀ dZ1), the SiLU output A1 (written in bf16 by the first epilogue), dZ2
// and dZ1 (each rounded once), and the two weight images.  A bf16 copy of
// width w is stored with leading dimension pad8(w), zero-padded.
using bf16 = __nv_bfloat16;
struct WideScratch {
  bf16* x;     // gathered MLP input, R x Kmax
  bf16* a1;    // first layer's SiLU output, R x H
  bf16* dz2;   // gradient at the second layer's output, R x max(H, out)
  bf16* dz1;   // gradient at the first layer's output, R x H
  bf16* w1;    // first-layer weight image [in][H], in <= Kmax
  bf16* w2;    // second-layer weight image [H][out]
  float* acc;  // a product before its epilogue, R x max(H, out)
  float* part; // partial tiles of the row-reduction products (wg_part_elems)
};
int pad8(int w);
size_t wide_scratch_bytes(int64_t R, int H, int Kmax, int out);
WideScratch wide_scratch(void* p, int64_t R, int H, int Kmax, int out);
// out[M, A.K] = bf16 of the rows of A (leading dimension pad8(A.K), zero
// padding); wide_round: the same for a dense [M, N] fp32 matrix with leading
// dimension ld (out: leading dimension pad8(N)).
xmgn_status wide_gather(const RowSrc& A, int64_t M, bf16* out, cudaStream_t s);
xmgn_status wide_round(const float* X, int64_t M, int N, int64_t ld, bf16* out, cudaStream_t s);
// acc[M,N] = A[M,K] B[K,N]            (B row-major [K][N], e.g. a weight W[in][out])
xmgn_status wide_nn(const bf16* A, int64_t M, int K, const bf16* B, int N, float* acc, cudaStream_t s);
// a1[M,N] = bf16(SiLU(A[M,K] B[K,N] + bias)): a first MLP layer with its
// epilogue inside the product; pre [M,N] (fp32, nullable) receives A B + bias
xmgn_status wide_nn_silu(const bf16* A, int64_t M, int K, const bf16* B, int N, const float* bias, bf16* a1,
                         cudaStream_t s, float* pre = nullptr);
// acc[M,N] = A[M,K] B[N,K]^T          (dX = dZ Wᵀ with W[in][out], N = in, K = out)
xmgn_status wide_nt(const bf16* A, int64_t M, int K, const bf16* B, int N, float* acc, cudaStream_t s);
// G[K1,N] = A[M,K1]^T B[M,N], written (zero when M = 0); part: partial tiles
xmgn_status wide_tn(const bf16* A, int64_t M, int K1, const bf16* B, int N, float* G, float* part, cudaStream_t s);
// C = epi(acc + bias) with the Epi codes above, acc dense [M,N].  C (fp32,
// leading dimension ldc, shared by pre and aux) and C16 (bf16, dense) are
// each optional.
xmgn_status wide_epilogue(const float* acc, int64_t M, int N, const float* bias, float* C, int64_t ldc, int epi,
                          float* pre, const float* aux, bf16* C16, cudaStream_t s);
// dZ1 = acc * silu'(Z1) (acc, Z1 dense [M,N]) written in bf16 to C16, and
// db = its column sums, exact fp32 values summed in a fixed order through
// part (colsum_part_elems(M, N) floats).  N % 4 == 0, N <= 512.
xmgn_status wide_silu_grad_colsum(const float* acc, int64_t M, int N, const float* Z1, bf16* C16, float* db,
                                  float* part, cudaStream_t s);
// C[M,N] = A[M,K] B[N,K]^T, or C += that product (accum), written by the GEMM
// itself into C (leading dimension ldc).
xmgn_status wide_nt_into(const bf16* A, int64_t M, int K, const bf16* B, int N, float* C, int64_t ldc, bool accum,
                         cudaStream_t s);
// Outputs of the dZ1 W1ᵀ product split by the row blocks of W1 = [W_0; W_1;
// ...] (W rows each): block q's product is stored into C[q] or added there.
struct WideOut {
  int n = 0, W = 0;
  float* C[3] = {};
  int64_t ldc[3] = {};
  int accum[3] = {};
};

}  // namespace xmgn
