// FP32 "plain" form of the model: eqs. (1)-(4) evaluated literally, layer by
// layer, with CUDA-core fp32 GEMMs over gathered rows (the edge MLP input
// [h_i, h_j, e_ij] is never materialised, rows are gathered inside the GEMM),
// LayerNorm kernels (the edge one also forms the receiver sums of eq. (2)),
// and CSR/CSC segmented sums in the backward.  Per-layer checkpoints hold
// h^l, e^l and a^l; the backward recomputes each MLP's activations.
//
// The same code is the wide BF16 path (hidden widths other than 128): with
// Gemm::tc set, every product runs on the tensor cores with bf16 operands
// (wide.cu); activations, LayerNorm, sums and gradients stay fp32.
#include "model.cuh"
#include "paths.cuh"

namespace xmgn {

namespace {

struct F32Ckpt {
  float* h;    // (L+1) x n x H
  float* e;    // L x E x H
  float* agg;  // L x n x H
  float* y;    // n x out
};

// Which products: fp32 on the CUDA cores, or (tc) bf16 on the tensor cores
// with the operand copies in w.
struct Gemm {
  bool tc = false;
  WideScratch w{};
};

struct F32Ws {
  float* nfeat;  // node-encoder inputs when Fourier features are appended
  float *feat, *Z1, *A1, *Z2, *dZ2, *dZ1, *elast;
  float *dy, *dh, *dagg, *de, *dhr, *dhs, *grad;
  float *tnpart, *cspart, *lnpart, *losspart;
  void* wide;  // tensor-core GEMM scratch (wide BF16 path only)
};

void f32_ckpt_layout(Arena& A, const ParamPlan& p, int64_t n, int64_t E, F32Ckpt& c) {
  const int H = p.H;
  c.h = A.take<float>(size_t(p.L + 1) * n * H);
  c.e = A.take<float>(size_t(p.L) * E * H);
  c.agg = A.take<float>(size_t(p.L) * n * H);
  c.y = A.take<float>(size_t(n) * p.out);
}

// Widest MLP input: the edge MLP's [h_i, h_j, e_ij] or an encoder's.
int wide_kmax(const ParamPlan& p) {
  int k = 3 * p.H;
  if (p.in_enc > k) k = p.in_enc;
  if (kInEdge > k) k = kInEdge;
  return k;
}

void f32_ws_layout(Arena& A, const ParamPlan& p, int64_t n, int64_t E, F32Ws& w, bool tc = false) {
  const int H = p.H;
  const int64_t R = n > E ? n : E;
  w.nfeat = p.fourier ? A.take<float>(size_t(n) * p.in_enc) : nullptr;
  w.feat = A.take<float>(size_t(E) * kInEdge);
  w.Z1 = A.take<float>(size_t(R) * H);
  w.A1 = A.take<float>(size_t(R) * H);
  w.Z2 = A.take<float>(size_t(R) * H);
  w.dZ2 = A.take<float>(size_t(R) * H);
  w.dZ1 = A.take<float>(size_t(R) * H);
  w.elast = A.take<float>(size_t(E) * H);
  w.dy = A.take<float>(size_t(n) * p.out);
  w.dh = A.take<float>(size_t(n) * H);
  w.dagg = A.take<float>(size_t(n) * H);
  w.de = A.take<float>(size_t(E) * H);
  w.dhr = A.take<float>(size_t(E) * H);
  w.dhs = A.take<float>(size_t(E) * H);
  w.grad = A.take<float>(size_t(p.total));
  size_t tn = gemm_tn_part_elems(R, 3 * H, H);
  w.tnpart = A.take<float>(tn);
  w.cspart = A.take<float>(colsum_part_elems(R, H));
  w.lnpart = A.take<float>(ln_bwd_part_elems(H));
  w.losspart = A.take<float>(loss_part_elems(n));
  w.wide = tc ? A.take<char>(wide_scratch_bytes(R, H, wide_kmax(p), p.out)) : nullptr;
}

// Wide path forward of Y = MLP(X): the gathered input and A1 stay in bf16
// scratch; with a LayerNorm, the second layer's bias is added inside the
// LayerNorm kernel, so Z2 is never stored.
// Receiver sums fused into an edge MLP's LayerNorm (eq. (2)): when `out` is
// set, the LayerNorm output is summed per receiver into out instead of stored.
struct Agg {
  const int64_t* row_ptr = nullptr;
  int64_t n = 0;
  float* out = nullptr;
};

xmgn_status mlp_fwd_wide(const WideScratch& x, const MlpOff& o, const float* P, const RowSrc& X, int64_t M,
                         float* Y, const float* resid_in, float* resid_out, cudaStream_t s, const Agg& agg) {
  const int K = X.K, H = o.hid;
  XMGN_TRY(wide_round(P + o.W1, K, H, H, x.w1, s));
  XMGN_TRY(wide_round(P + o.W2, H, o.out, o.out, x.w2, s));
  XMGN_TRY(wide_gather(X, M, x.x, s));
  // bias + SiLU inside the product: A1 leaves the GEMM in bf16, no fp32 product round trip
  XMGN_TRY(wide_nn_silu(x.x, M, K, x.w1, H, P + o.b1, x.a1, s));
  XMGN_TRY(wide_nn(x.a1, M, H, x.w2, o.out, x.acc, s));
  if (!o.ln) return wide_epilogue(x.acc, M, o.out, P + o.b2, Y, o.out, EPI_STORE, nullptr, nullptr, nullptr, s);
  if (agg.out)
    return layernorm_fwd_agg_f32(x.acc, P + o.b2, agg.row_ptr, agg.n, o.out, P + o.g, P + o.be, resid_in, resid_out,
                                 agg.out, s);
  return layernorm_fwd_f32(x.acc, M, o.out, P + o.g, P + o.be, Y, resid_in, resid_out, s, P + o.b2);
}

xmgn_status mlp_fwd(const Gemm& gm, const MlpOff& o, const float* P, const RowSrc& X, int64_t M, float* A1,
                    float* Z2, float* Y, const float* resid_in, float* resid_out, cudaStream_t s,
                    const Agg& agg = Agg{}) {
  if (gm.tc) return mlp_fwd_wide(gm.w, o, P, X, M, Y, resid_in, resid_out, s, agg);
  XMGN_TRY(gemm_nn_f32(X, M, P + o.W1, o.hid, P + o.b1, A1, o.hid, EPI_SILU, nullptr, nullptr, s));
  if (!o.ln) {
    return gemm_nn_f32(rows1(A1, o.hid, o.hid), M, P + o.W2, o.out, P + o.b2, Y, o.out, EPI_STORE, nullptr,
                       nullptr, s);
  }
  XMGN_TRY(gemm_nn_f32(rows1(A1, o.hid, o.hid), M, P + o.W2, o.out, P + o.b2, Z2, o.out, EPI_STORE, nullptr,
                       nullptr, s));
  if (agg.out)
    return layernorm_fwd_agg_f32(Z2, nullptr, agg.row_ptr, agg.n, o.out, P + o.g, P + o.be, resid_in, resid_out,
                                 agg.out, s);
  return layernorm_fwd_f32(Z2, M, o.out, P + o.g, P + o.be, Y, resid_in, resid_out, s);
}

// Wide path backward of Y = MLP(X) (activations recomputed): every operand is
// rounded to bf16 once and reused, X by the recompute and by Xᵀ dZ1.  Leaves
// dZ1 in x.dz1 (bf16; its fp32 values only feed the fused bias-gradient sums)
// and the first-layer weight image in x.w1, for the caller's dZ1 W1ᵀ product.
xmgn_status mlp_bwd_wide(const WideScratch& x, const MlpOff& o, const float* P, const RowSrc& X, int64_t M,
                         const float* dY1, const float* dY2, const int32_t* idx2, float* g, F32Ws& w,
                         cudaStream_t s) {
  const int K = X.K, H = o.hid;
  XMGN_TRY(wide_round(P + o.W1, K, H, H, x.w1, s));
  XMGN_TRY(wide_round(P + o.W2, H, o.out, o.out, x.w2, s));
  XMGN_TRY(wide_gather(X, M, x.x, s));
  XMGN_TRY(wide_nn_silu(x.x, M, K, x.w1, H, P + o.b1, x.a1, s, w.Z1));  // A1 and the pre-activation Z1
  const float* dZ2 = dY1;
  if (o.ln) {
    XMGN_TRY(wide_nn(x.a1, M, H, x.w2, o.out, x.acc, s));
    XMGN_TRY(layernorm_bwd_f32(x.acc, M, o.out, P + o.g, dY1, dY2, idx2, w.dZ2, g + o.g, g + o.be, w.lnpart, s,
                               P + o.b2));
    dZ2 = w.dZ2;
  }
  XMGN_TRY(wide_round(dZ2, M, o.out, o.out, x.dz2, s));
  XMGN_TRY(wide_tn(x.a1, M, H, x.dz2, o.out, g + o.W2, x.part, s));
  XMGN_TRY(colsum_f32(dZ2, M, o.out, o.out, g + o.b2, w.cspart, s));
  XMGN_TRY(wide_nt(x.dz2, M, o.out, x.w2, H, x.acc, s));
  XMGN_TRY(wide_silu_grad_colsum(x.acc, M, H, w.Z1, x.dz1, g + o.b1, w.cspart, s));
  return wide_tn(x.x, M, K, x.dz1, H, g + o.W1, x.part, s);
}

// Backward of Y = MLP(X) given dY = dY1 + dY2[idx2]; writes every gradient of
// the MLP into g and leaves dZ1 (gradient at the first layer's output) in w.dZ1.
xmgn_status mlp_bwd(const Gemm& gm, const MlpOff& o, const float* P, const RowSrc& X, int64_t M, const float* dY1,
                    const float* dY2, const int32_t* idx2, float* g, F32Ws& w, cudaStream_t s) {
  if (gm.tc) return mlp_bwd_wide(gm.w, o, P, X, M, dY1, dY2, idx2, g, w, s);
  const int H = o.hid;
  XMGN_TRY(gemm_nn_f32(X, M, P + o.W1, H, P + o.b1, w.A1, H, EPI_SILU, w.Z1, nullptr, s));
  const float* dZ2 = dY1;
  if (o.ln) {
    XMGN_TRY(gemm_nn_f32(rows1(w.A1, H, H), M, P + o.W2, o.out, P + o.b2, w.Z2, o.out, EPI_STORE, nullptr, nullptr,
                         s));
    XMGN_TRY(layernorm_bwd_f32(w.Z2, M, o.out, P + o.g, dY1, dY2, idx2, w.dZ2, g + o.g, g + o.be,
                               w.lnpart, s));
    dZ2 = w.dZ2;
  }
  XMGN_TRY(gemm_tn_f32(rows1(w.A1, H, H), M, dZ2, o.out, o.out, g + o.W2, w.tnpart, s));
  XMGN_TRY(colsum_f32(dZ2, M, o.out, o.out, g + o.b2, w.cspart, s));
  XMGN_TRY(gemm_nt_f32(rows1(dZ2, o.out, o.out), M, P + o.W2, H, w.dZ1, H, EPI_SILU_GRAD, w.Z1, s));
  XMGN_TRY(gemm_tn_f32(X, M, w.dZ1, H, H, g + o.W1, w.tnpart, s));
  XMGN_TRY(colsum_f32(w.dZ1, M, H, H, g + o.b1, w.cspart, s));
  return XMGN_OK;
}

// Wide path: dZ1 W_qᵀ for each row block W_q of the first-layer weight image
// that mlp_bwd_wide left in x.w1, each GEMM writing (or adding to) its output
// directly.
xmgn_status dz1_w1t_wide(const WideScratch& x, int64_t M, int H, const WideOut& o, cudaStream_t s) {
  for (int q = 0; q < o.n; ++q)
    XMGN_TRY(wide_nt_into(x.dz1, M, H, x.w1 + int64_t(q) * o.W * H, o.W, o.C[q], o.ldc[q], o.accum[q] != 0, s));
  return XMGN_OK;
}

}  // namespace

void f32_sizes(const ParamPlan& p, int64_t n, int64_t E, size_t* ws, size_t* ckpt, bool tc) {
  Arena a, b;
  a.dry = b.dry = true;
  F32Ws w;
  F32Ckpt c;
  f32_ws_layout(a, p, n, E, w, tc);
  f32_ckpt_layout(b, p, n, E, c);
  *ws = a.used + 256;
  *ckpt = b.used + 256;
}

xmgn_status f32_forward(const ParamPlan& p, const float* P, const xmgn_graph& g,
                        const float* node_in, const float* xyz, const float* targets, float* y,
                        float* loss, void* ckpt, size_t ckpt_bytes, void* ws, size_t ws_bytes,
                        cudaStream_t s, bool tc) {
  const int64_t n = g.n_nodes, E = g.n_edges;
  const int H = p.H;
  Arena A{static_cast<char*>(ws), ws_bytes};
  Arena C{static_cast<char*>(ckpt), ckpt_bytes};
  F32Ws w;
  F32Ckpt c;
  f32_ws_layout(A, p, n, E, w, tc);
  f32_ckpt_layout(C, p, n, E, c);
  if (!A.ok() || !C.ok()) return fail(XMGN_ERR_WORKSPACE, "fp32 forward: ws/ckpt too small");
  Gemm gm;
  gm.tc = tc;
  if (tc) gm.w = wide_scratch(w.wide, n > E ? n : E, H, wide_kmax(p), p.out);

  XMGN_TRY(edge_features(xyz, g.gid, g.recv, g.col, E, w.feat, s));
  if (p.fourier) XMGN_TRY(node_features(node_in, p.in_node, xyz, g.gid, n, p.fourier, w.nfeat, s));
  const RowSrc nrows = p.fourier ? rows1(w.nfeat, p.in_enc, p.in_enc) : rows1(node_in, p.in_node, p.in_node, g.gid);
  XMGN_TRY(mlp_fwd(gm, p.ne, P, nrows, n, w.A1, w.Z2, c.h, nullptr, nullptr, s));
  float* e0 = p.L > 0 ? c.e : w.elast;
  XMGN_TRY(mlp_fwd(gm, p.ee, P, rows1(w.feat, kInEdge, kInEdge), E, w.A1, w.Z2, e0, nullptr, nullptr, s));
  for (int l = 0; l < p.L; ++l) {
    float* hl = c.h + size_t(l) * n * H;
    float* hn = c.h + size_t(l + 1) * n * H;
    float* el = c.e + size_t(l) * E * H;
    float* en = (l + 1 < p.L) ? c.e + size_t(l + 1) * E * H : w.elast;
    float* agg = c.agg + size_t(l) * n * H;
    RowSrc X = rows1(hl, H, H, g.recv);                          // eq. (1): [h_i, h_j, e_ij]
    rows_add(X, hl, H, H, g.col);
    rows_add(X, el, H, H);
    Agg ag;                                                       // eq. (2), fused
    ag.row_ptr = g.row_ptr, ag.n = n, ag.out = agg;
    XMGN_TRY(mlp_fwd(gm, p.edge[l], P, X, E, w.A1, w.Z2, nullptr, el, en, s, ag));
    RowSrc Xn = rows1(hl, H, H);                                  // eq. (3): [h_i, a_i]
    rows_add(Xn, agg, H, H);
    XMGN_TRY(mlp_fwd(gm, p.node[l], P, Xn, n, w.A1, w.Z2, nullptr, hl, hn, s));
  }
  const float* hL = c.h + size_t(p.L) * n * H;
  XMGN_TRY(mlp_fwd(gm, p.dec, P, rows1(hL, H, H), n, w.A1, w.Z2, c.y, nullptr, nullptr, s));
  if (targets || y)
    XMGN_TRY(mse_loss(c.y, n, p.out, targets, g.gid, g.hop, g.n_norm, targets ? loss : nullptr,
                      nullptr, y, w.losspart, s));
  return XMGN_OK;
}

xmgn_status f32_backward(const ParamPlan& p, const float* P, const xmgn_graph& g,
                         const float* node_in, const float* xyz, const float* targets,
                         const void* ckpt, size_t ckpt_bytes, float* dparams, float* dcomp,
                         void* ws, size_t ws_bytes, cudaStream_t s, bool tc) {
  const int64_t n = g.n_nodes, E = g.n_edges;
  const int H = p.H;
  Arena A{static_cast<char*>(ws), ws_bytes};
  Arena C{static_cast<char*>(const_cast<void*>(ckpt)), ckpt_bytes};
  F32Ws w;
  F32Ckpt c;
  f32_ws_layout(A, p, n, E, w, tc);
  f32_ckpt_layout(C, p, n, E, c);
  if (!A.ok() || !C.ok()) return fail(XMGN_ERR_WORKSPACE, "fp32 backward: ws/ckpt too small");
  Gemm gm;
  gm.tc = tc;
  if (tc) gm.w = wide_scratch(w.wide, n > E ? n : E, H, wide_kmax(p), p.out);
  float* G = w.grad;
  XMGN_CUDA(cudaMemsetAsync(G, 0, sizeof(float) * size_t(p.total), s));

  XMGN_TRY(mse_loss(c.y, n, p.out, targets, g.gid, g.hop, g.n_norm, nullptr, w.dy, nullptr,
                    w.losspart, s));
  const float* hL = c.h + size_t(p.L) * n * H;
  XMGN_TRY(mlp_bwd(gm, p.dec, P, rows1(hL, H, H), n, w.dy, nullptr, nullptr, G, w, s));
  if (gm.tc) {
    WideOut o;
    o.n = 1;
    o.W = H;
    o.C[0] = w.dh, o.ldc[0] = H, o.accum[0] = 0;
    XMGN_TRY(dz1_w1t_wide(gm.w, n, H, o, s));
  } else {
    XMGN_TRY(gemm_nt_f32(rows1(w.dZ1, H, H), n, P + p.dec.W1, H, w.dh, H, EPI_STORE, nullptr, s));
  }
  XMGN_CUDA(cudaMemsetAsync(w.de, 0, sizeof(float) * size_t(E) * H, s));
  for (int l = p.L - 1; l >= 0; --l) {
    const float* hl = c.h + size_t(l) * n * H;
    const float* el = c.e + size_t(l) * E * H;
    const float* agg = c.agg + size_t(l) * n * H;
    const MlpOff& on = p.node[l];
    const MlpOff& oe = p.edge[l];
    // node update: h' = h + MLP_n([h, a])
    RowSrc Xn = rows1(hl, H, H);
    rows_add(Xn, agg, H, H);
    XMGN_TRY(mlp_bwd(gm, on, P, Xn, n, w.dh, nullptr, nullptr, G, w, s));
    if (gm.tc) {  // dZ1 [W1_h; W1_a]^T: dh += first block, da = second
      WideOut o;
      o.n = 2;
      o.W = H;
      o.C[0] = w.dh, o.ldc[0] = H, o.accum[0] = 1;
      o.C[1] = w.dagg, o.ldc[1] = H, o.accum[1] = 0;
      XMGN_TRY(dz1_w1t_wide(gm.w, n, H, o, s));
    } else {
      XMGN_TRY(gemm_nt_f32(rows1(w.dZ1, H, H), n, P + on.W1 + int64_t(H) * H, H, w.dagg, H, EPI_STORE, nullptr, s));
      XMGN_TRY(gemm_nt_f32(rows1(w.dZ1, H, H), n, P + on.W1, H, w.dh, H, EPI_ACCUM, nullptr, s));
    }
    // edge update: e' = e + m, a_i = sum m_ij  ->  dm = de' + da[recv]
    RowSrc X = rows1(hl, H, H, g.recv);
    rows_add(X, hl, H, H, g.col);
    rows_add(X, el, H, H);
    XMGN_TRY(mlp_bwd(gm, oe, P, X, E, w.de, w.dagg, g.recv, G, w, s));
    if (gm.tc) {  // dZ1 [W1_r; W1_s; W1_e]^T, one product per block
      WideOut o;
      o.n = 3;
      o.W = H;
      o.C[0] = w.dhr, o.ldc[0] = H, o.accum[0] = 0;
      o.C[1] = w.dhs, o.ldc[1] = H, o.accum[1] = 0;
      o.C[2] = w.de, o.ldc[2] = H, o.accum[2] = 1;
      XMGN_TRY(dz1_w1t_wide(gm.w, E, H, o, s));
    } else {
      XMGN_TRY(gemm_nt_f32(rows1(w.dZ1, H, H), E, P + oe.W1, H, w.dhr, H, EPI_STORE, nullptr, s));
      XMGN_TRY(gemm_nt_f32(rows1(w.dZ1, H, H), E, P + oe.W1 + int64_t(H) * H, H, w.dhs, H, EPI_STORE, nullptr, s));
      XMGN_TRY(gemm_nt_f32(rows1(w.dZ1, H, H), E, P + oe.W1 + 2 * int64_t(H) * H, H, w.de, H, EPI_ACCUM, nullptr,
                           s));
    }
    XMGN_TRY(seg_sum_rows_f32(w.dhr, H, g.row_ptr, n, H, w.dh, H, true, s));
    XMGN_TRY(seg_sum_cols_f32(w.dhs, H, g.row_ptr, g.csc_perm, n, H, w.dh, H, true, s));
  }
  XMGN_TRY(edge_features(xyz, g.gid, g.recv, g.col, E, w.feat, s));
  XMGN_TRY(mlp_bwd(gm, p.ee, P, rows1(w.feat, kInEdge, kInEdge), E, w.de, nullptr, nullptr, G, w, s));
  if (p.fourier) XMGN_TRY(node_features(node_in, p.in_node, xyz, g.gid, n, p.fourier, w.nfeat, s));
  const RowSrc nrows = p.fourier ? rows1(w.nfeat, p.in_enc, p.in_enc) : rows1(node_in, p.in_node, p.in_node, g.gid);
  XMGN_TRY(mlp_bwd(gm, p.ne, P, nrows, n, w.dh, nullptr, nullptr, G, w, s));
  return accumulate_grad(dparams, dcomp, G, p.total, s);
}

}  // namespace xmgn
