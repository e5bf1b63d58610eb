// Fused two-layer MLP kernels on tcgen05 (BF16 operands, FP32 accumulators in
// TMEM).  One CTA of 512 threads per SM, persistent over 128-row tiles; a thread
// owns one 32-column slice of one tile row in every epilogue.
#pragma once

#include "tc_gemm.cuh"

namespace xmgn {

enum MlpMode : int {
  M_EDGE = 0,  // processor edge MLP, eq. (1): rows = edges, A = e_ij, first layer completed by P_r[i] + P_s[j]
  M_NODE = 1,  // processor node MLP, eq. (3): rows = nodes, A = [h_i, a_i]
  M_DEC = 2,   // decoder: rows = nodes, A = h_i, no LayerNorm, `out` outputs
  M_NENC = 3,  // node encoder: A = node inputs (fp32, gathered by global id)
  M_EENC = 4,  // edge encoder: A = (x_j - x_i, |x_j - x_i|) built in the kernel
};

struct MlpImgs {
  const uint8_t* w1;    // K-major image of GEMM1's B operand (R = H, C = K1), bf16(W1)
  const uint8_t* w2;    // K-major image of GEMM2's B operand (R = N2, C = H), bf16(W2)
  const uint8_t* w1lo;  // bf16(W1 - bf16(W1)) (all modes but the node MLP)
  const uint8_t* w2lo;  // bf16(W2 - bf16(W2))
  uint32_t w1_bytes, w2_bytes;
};

struct MlpParams {
  const float *b1, *b2, *gamma, *beta;
};

struct FwdArgs {
  int64_t rows;
  int H;
  // A sources
  const bf16* a0;  // EDGE: e16; NODE, DEC: h16
  const bf16* a1;  // NODE: a16
  const float* fin;  // NENC: node inputs [n_global, fin_w]; EENC: xyz [n_global, 3]
  int fin_w;
  const float* xyz;  // NENC: coordinates [n_global, 3] for the Fourier features
  int fourier;       // NENC: Fourier frequencies appended after the fin_w inputs
  const bf16* feat8; // EENC: edge inputs [rows, 8] bf16 (x_j - x_i, |x_j - x_i|, zeros) from edge_inputs_bf16
  const int32_t* gid;
  const int32_t* recv;
  const int32_t* col;
  const bf16* P;  // EDGE: [n, 2H] node projections, bf16 (receiver block, sender block)
  MlpImgs w;
  MlpParams p;
  // outputs
  bf16* o16;        // EDGE: e16 next (null: not stored); NODE: h16 next; NENC: h16; EENC: e16
  bf16* agg16;      // EDGE: a_i = sum_j m_ij for receivers whose edges lie in one 128-edge tile
  float* agg_part;  // EDGE: [tiles][2][H] fp32 partial sums of receivers crossing a tile boundary
  float* o32;       // NODE: h32 next; NENC: h32; DEC: y
  const float* r32; // NODE: h32 (residual input)
  int out_w;        // DEC: outputs
  int order;        // EDGE: tile order over the CTAs (0 round-robin, 1 contiguous runs; set by the launcher)
  uint32_t* err;
};

struct BwdArgs {
  int64_t rows;
  int H;
  const bf16* a0;
  const bf16* a1;
  const float* fin;
  int fin_w;
  const float* xyz;  // NENC: as in FwdArgs
  int fourier;
  const bf16* feat8; // EENC: as in FwdArgs
  const int32_t* gid;
  const int32_t* recv;
  const int32_t* col;
  const bf16* P;  // EDGE: as in FwdArgs
  MlpImgs w;
  MlpParams p;
  // incoming gradient dY = dY1[row] + dY2[idx2[row]]; each given either as
  // fp32 (dY*) or bf16 (dY*h), the other pointer null
  const float* dY1;  // NODE: dh; DEC: dy [rows, out]; NENC: dh
  const bf16* dY1h;  // EDGE, EENC: de (edge-state gradient, bf16; null = 0)
  const float* dY2;
  const bf16* dY2h;  // EDGE: d a (aggregated-message gradient, bf16)
  const int32_t* idx2;
  // outputs
  float* dX0;   // NODE: dh_out (= dY1 + dX_h); DEC: dh
  bf16* dX0h;   // EDGE: de_out (= dY1 + dX_e, may alias dY1h)
  bf16* dX1h;   // NODE: d a
  bf16* A1g;    // NODE, NENC, DEC: SiLU activations (for X^T dY products)
  bf16* dZ2g;   // NODE, NENC: LayerNorm input gradient; DEC: dy (64 cols, zero padded)
  bf16* dZ1g;   // all: gradient at the first layer output
  bf16* X16g;   // NENC: bf16 node inputs (128 cols, zero padded)
  float* wpart; // EDGE, EENC: [cta][2][128][H] partial dW1, dW2 from TMEM
  float* cpart; // [cta][4][H] partial column sums: db1, db2, dgamma, dbeta
  uint32_t* spill;  // EDGE, two-group kernel: [cta][2][128][H/2] fp16 pairs of SiLU'(Z1) (edge_bwd_spill_words)
  int out_w;
  int order;    // EDGE: tile order over the CTAs, as in FwdArgs
  uint32_t* err;
};

xmgn_status mlp_fwd_tc(int mode, const FwdArgs& a, cudaStream_t s);
xmgn_status mlp_bwd_tc(int mode, const BwdArgs& a, cudaStream_t s);
int mlp_grid(int64_t rows);
// Edge-encoder inputs of every edge (Sec. II-E: x_j - x_i and its norm, j the
// sender, i the receiver, coordinates by global id) in fp32, rounded to bf16
// into out [E, 8] (the last four entries zero): the operand rows of the edge
// encoder's first layer.
xmgn_status edge_inputs_bf16(const float* xyz, const int32_t* gid, const int32_t* recv, const int32_t* col,
                             int64_t E, bf16* out, cudaStream_t s);
// 32-bit words of the SiLU' scratch slots of the two-group edge backward kernel.
int64_t edge_bwd_spill_words();

}  // namespace xmgn
