// BF16 tensor-core path of the model (tcgen05, FP32 accumulation).
//
// Per processor layer l (eqs. 1-4), forward:
//   P = h16 [W1_r | W1_s]                 node projections (tc_gemm, bf16 output)
//   edge kernel: m = MLP_e completed as e W1_e + P_r[i] + P_s[j];  e' = e + m
//   aggregation a_i = sum_j m_ij (fp32, CSR order) -> bf16, fused into the edge
//     kernel's epilogue (agg_fixup_kernel completes runs crossing 128-edge tiles)
//   node kernel: h' = h + MLP_n([h, a])
// The first Linear of the edge MLP is split by input block: the receiver and
// sender blocks are applied once per node instead of once per edge.  This is
// the same linear map ([h_i, h_j, e] W1 = h_i W1_r + h_j W1_s + e W1_e), so
// results agree with eq. (1) up to rounding; the edge kernel's tensor work
// drops from K = 3H to K = H per edge.  In the backward pass the same split
// gives d h_i = (sum_{j} dZ1_ij) W1_r^T and d W1_r = sum_i h_i^T (sum_j dZ1_ij),
// i.e. per-node sums of dZ1 over receiver (CSR) and sender (CSC) segments
// followed by node-level products.
#include "mlp_tc.cuh"
#include "paths.cuh"
#include "tune.cuh"

namespace xmgn {

namespace {

// Packed weight images (bf16, swizzled); *l = low part bf16(W - bf16(W)).
struct LayerImgs {
  Img ew1e, ew1el, ew2, ew2l, ewrs, nw1, nw1l, nw2, nw2l;
};
struct ImgPlan {
  Img new1, new1l, new2, new2l, eew1, eew1l, eew2, eew2l, dw1, dw1l, dw2, dw2l;
  std::vector<LayerImgs> layer;
  size_t total = 0;
};

ImgPlan make_imgs(const ParamPlan& p) {
  ImgPlan ip;
  const uint32_t H = p.H;
  size_t o = 0;
  auto mk = [&](uint32_t R, uint32_t C) {
    Img im;
    im.off = o;
    im.R = R;
    im.C = C;
    o += (size_t(R) * C * 2 + 1023) & ~size_t(1023);
    return im;
  };
  ip.new1 = mk(H, 64);
  ip.new1l = mk(H, 64);
  ip.new2 = mk(H, H);
  ip.new2l = mk(H, H);
  ip.eew1 = mk(H, 64);
  ip.eew1l = mk(H, 64);
  ip.eew2 = mk(H, H);
  ip.eew2l = mk(H, H);
  ip.dw1 = mk(H, H);
  ip.dw1l = mk(H, H);
  ip.dw2 = mk(16, H);
  ip.dw2l = mk(16, H);
  for (int l = 0; l < p.L; ++l) {
    LayerImgs li;
    li.ew1e = mk(H, H);
    li.ew1el = mk(H, H);
    li.ew2 = mk(H, H);
    li.ew2l = mk(H, H);
    li.ewrs = mk(2 * H, H);
    li.nw1 = mk(H, 2 * H);
    li.nw1l = mk(H, 2 * H);
    li.nw2 = mk(H, H);
    li.nw2l = mk(H, H);
    ip.layer.push_back(li);
  }
  ip.total = o;
  return ip;
}

struct BCkpt {
  uint8_t* img;
  float* h32;  // (L+1) x n x H
  bf16* h16;   // (L+1) x n x H
  bf16* e16;   // L x E x H
  bf16* a16;   // L x n x H
  bf16* P16;   // L x n x 2H node projections h [W1_r | W1_s] of each layer (none with offload: recomputed)
  float* y;    // n x out
  bf16* feat8; // E x 8 edge-encoder inputs (bf16), made by the forward, read again by the backward
};

struct BWs {
  float *losspart, *grad, *dy32, *dh, *wpart, *cpart, *tnpart;
  bf16* P;          // node projections, rounded to bf16 like any GEMM output under AMP
  bf16 *dagg, *de;  // gradients of a (node level) and of the edge state, bf16
  float* agg_part;  // [edge tiles][2][H]: partial sums of receivers that cross a tile boundary
  bf16 *A1g, *dZ2g, *dZ1g, *S16, *X16;
  float* colp;  // [seg_sums blocks][2][H]: column partials of the receiver sums and of indeg * da
  float* tsum;  // [L][H]: sum over nodes of indeg(i) * da_i, per layer
  float* vbeta; // [L][H]: db1_l W1_e,l^T, per layer
  uint32_t* spill;  // SiLU' scratch slots of the two-group edge backward kernel (L2-resident)
};

// With offload the device keeps kRing edge-state slots (a ring) and every
// layer's e^l lives in host memory between the two passes.
constexpr int kRing = 3;
void ckpt_layout(Arena& A, const ParamPlan& p, const ImgPlan& ip, int64_t n, int64_t E, BCkpt& c,
                 bool offload = false) {
  const int H = p.H;
  c.img = A.take<uint8_t>(ip.total);
  c.h32 = A.take<float>(size_t(p.L + 1) * n * H);
  c.h16 = A.take<bf16>(size_t(p.L + 1) * n * H);
  c.e16 = A.take<bf16>(size_t(offload ? (p.L < kRing ? p.L : kRing) : p.L) * E * H);
  c.a16 = A.take<bf16>(size_t(p.L) * n * H);
  c.P16 = offload ? nullptr : A.take<bf16>(size_t(p.L) * n * 2 * H);
  c.y = A.take<float>(size_t(n) * p.out);
  c.feat8 = A.take<bf16>(size_t(E) * 8);
}

unsigned seg_grid_max(int64_t n) { return grid_for(n * 32, 256, int64_t(num_sms()) * 16); }

void ws_layout(Arena& A, const ParamPlan& p, int64_t n, int64_t E, BWs& w) {
  const int H = p.H;
  const int64_t R = n > E ? n : E;
  const int g = num_sms();
  w.P = A.take<bf16>(size_t(n) * 2 * H);
  w.agg_part = A.take<float>(size_t((E + 127) / 128) * 2 * H);
  w.losspart = A.take<float>(loss_part_elems(n));
  w.grad = A.take<float>(size_t(p.total));
  w.dy32 = A.take<float>(size_t(n) * p.out);
  w.dh = A.take<float>(size_t(n) * H);
  w.dagg = A.take<bf16>(size_t(n) * H);
  w.de = A.take<bf16>(size_t(E) * H);
  w.wpart = A.take<float>(size_t(g) * 2 * 128 * H);
  w.cpart = A.take<float>(size_t(g) * 4 * H);
  w.tnpart = A.take<float>(tc_gemm_tn_part_elems(256, 256));
  w.A1g = A.take<bf16>(size_t(n) * H);
  w.dZ2g = A.take<bf16>(size_t(n) * H);
  w.dZ1g = A.take<bf16>(size_t(R) * H);
  w.S16 = A.take<bf16>(size_t(n) * 2 * H);
  w.X16 = A.take<bf16>(size_t(n) * 128);
  w.colp = A.take<float>(size_t(seg_grid_max(n)) * 2 * H);
  w.tsum = A.take<float>(size_t(p.L) * H);
  w.vbeta = A.take<float>(size_t(p.L) * H);
  w.spill = A.take<uint32_t>(size_t(edge_bwd_spill_words()));
}

__device__ __forceinline__ void acc_bf16x4(float4& s, uint2 u) {
  float2 a = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&u.x));
  float2 b = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&u.y));
  s.x += a.x;
  s.y += a.y;
  s.z += b.x;
  s.w += b.y;
}

// Completes the aggregation (eq. 2) that the edge kernel fuses into its
// epilogue: receivers without edges get a_i = 0, and a receiver whose edge
// run [rp[i], rp[i+1]) crosses 128-edge tile boundaries gets the tail partial
// of its first tile plus the head partials of the following tiles, in tile
// order (each partial an fp32 sum in CSR order).  Receivers whose run lies in
// one tile were written by the edge kernel and are skipped.
__global__ void agg_fixup_kernel(const float* __restrict__ part, const int64_t* __restrict__ rp, int64_t n,
                                 bf16* __restrict__ a16) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t i0 = warp * 32; i0 < n; i0 += nw * 32) {
    // lane l looks at node i0 + l; the warp then serves the nodes that need it
    const int64_t i = i0 + lane;
    int64_t e0 = 0, e1 = 0;
    bool todo = false;
    if (i < n) {
      e0 = rp[i];
      e1 = rp[i + 1];
      todo = e1 == e0 || (e0 >> 7) != ((e1 - 1) >> 7);
    }
    uint32_t pending = __ballot_sync(0xffffffffu, todo);
    while (pending) {
      const int src = __ffs(pending) - 1;
      pending &= pending - 1;
      const int64_t j = i0 + src;
      const int64_t f0 = __shfl_sync(0xffffffffu, e0, src), f1 = __shfl_sync(0xffffffffu, e1, src);
      float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
      if (f1 > f0) {
        const int64_t t0 = f0 >> 7, t1 = (f1 - 1) >> 7;
        s = reinterpret_cast<const float4*>(part + (t0 * 2 + 1) * 128)[lane];
        for (int64_t t = t0 + 1; t <= t1; ++t) {
          const float4 h = reinterpret_cast<const float4*>(part + t * 2 * 128)[lane];
          s.x += h.x;
          s.y += h.y;
          s.z += h.z;
          s.w += h.w;
        }
      }
      uint2 o;
      o.x = tc::pack_bf16(s.x, s.y);
      o.y = tc::pack_bf16(s.z, s.w);
      reinterpret_cast<uint2*>(a16 + j * 128)[lane] = o;
    }
  }
}

// C consecutive bf16 values (C = 4 or 8) added into a[0..C).
template <int C>
__device__ __forceinline__ void acc_bf16(float (&a)[C], const bf16* p) {
  if constexpr (C == 4) {
    float4 t = make_float4(a[0], a[1], a[2], a[3]);
    acc_bf16x4(t, *reinterpret_cast<const uint2*>(p));
    a[0] = t.x, a[1] = t.y, a[2] = t.z, a[3] = t.w;
  } else {
    const uint4 u = *reinterpret_cast<const uint4*>(p);
    float4 t = make_float4(a[0], a[1], a[2], a[3]), v = make_float4(a[4], a[5], a[6], a[7]);
    acc_bf16x4(t, make_uint2(u.x, u.y));
    acc_bf16x4(v, make_uint2(u.z, u.w));
    a[0] = t.x, a[1] = t.y, a[2] = t.z, a[3] = t.w, a[4] = v.x, a[5] = v.y, a[6] = v.z, a[7] = v.w;
  }
}

// S[i] = [ sum over edges received by i of dZ1 , sum over edges sent by i of dZ1 ],
// each node handled by a group of LPN lanes (32: a warp, 16: a half-warp),
// lane l of the group owning features C*l .. C*l + C - 1.  Also two column
// sums, as per-block partials colp[block] (fp32, fixed order: nodes in group
// order, then the groups of the block in index order):
//   colp[block][0:H]  = sum over the block's nodes of S_r[i] before rounding,
//                       i.e. of dZ1 over the block's edges: the edge MLP's db1;
//   colp[block][H:2H] = sum of indeg(i) da[i]: the receiver part of the
//                       column sum of dm = de + da[recv] (its dbeta).
// With these the edge backward kernel needs no column reductions for db1 or
// dbeta (the de part of dbeta follows from db1, see edge_beta_kernel).
template <int LPN>
__global__ void __launch_bounds__(256) seg_sums_kernel(const bf16* __restrict__ dz1, const int64_t* __restrict__ rp,
                                                       const int32_t* __restrict__ perm, int64_t n,
                                                       const bf16* __restrict__ da, bf16* __restrict__ S,
                                                       float* __restrict__ colp) {
  constexpr int C = 128 / LPN, NG = 8 * (32 / LPN);  // features per lane, node groups per block
  __shared__ float red[2][NG][128];
  const int lane = threadIdx.x & 31;
  const int hl = lane % LPN, gi = threadIdx.x / LPN;  // lane in the group, group in the block
  const int64_t grp = int64_t(blockIdx.x) * NG + gi;
  const int64_t ngrp = int64_t(gridDim.x) * NG;
  const int c0 = C * hl;
  float cr[C], cd[C];
#pragma unroll
  for (int j = 0; j < C; ++j) cr[j] = cd[j] = 0.f;
  for (int64_t i = grp; i < n; i += ngrp) {
    float r[C], sv[C], d[C];
#pragma unroll
    for (int j = 0; j < C; ++j) r[j] = sv[j] = d[j] = 0.f;
    const int64_t e0 = rp[i], e1 = rp[i + 1];
    if (da) acc_bf16<C>(d, da + i * 128 + c0);
    for (int64_t e = e0; e < e1; ++e) acc_bf16<C>(r, dz1 + e * 128 + c0);
    for (int64_t t = e0; t < e1; ++t) acc_bf16<C>(sv, dz1 + int64_t(perm[t]) * 128 + c0);
    uint32_t o[C];
#pragma unroll
    for (int j = 0; j < C / 2; ++j) {
      o[j] = tc::pack_bf16(r[2 * j], r[2 * j + 1]);
      o[C / 2 + j] = tc::pack_bf16(sv[2 * j], sv[2 * j + 1]);
    }
    if constexpr (C == 4) {
      *reinterpret_cast<uint2*>(S + i * 256 + c0) = make_uint2(o[0], o[1]);
      *reinterpret_cast<uint2*>(S + i * 256 + 128 + c0) = make_uint2(o[2], o[3]);
    } else {
      *reinterpret_cast<uint4*>(S + i * 256 + c0) = make_uint4(o[0], o[1], o[2], o[3]);
      *reinterpret_cast<uint4*>(S + i * 256 + 128 + c0) = make_uint4(o[4], o[5], o[6], o[7]);
    }
    const float k = float(e1 - e0);
#pragma unroll
    for (int j = 0; j < C; ++j) {
      cr[j] += r[j];
      cd[j] += k * d[j];
    }
  }
#pragma unroll
  for (int j = 0; j < C; ++j) {
    red[0][gi][c0 + j] = cr[j];
    red[1][gi][c0 + j] = cd[j];
  }
  __syncthreads();
  const int q = threadIdx.x >> 7, c = threadIdx.x & 127;
  float t = 0.f;
#pragma unroll
  for (int g = 0; g < NG; ++g) t += red[q][g][c];
  colp[(int64_t(blockIdx.x) * 2 + q) * 128 + c] = t;
}

// Launch shape of seg_sums_kernel for tuner candidate `choice`: {32, 16}
// lanes per node x {16, 8} blocks per SM.
struct SegShape {
  int lpn;
  unsigned grid;
};
SegShape seg_shape(int64_t n, int choice) {
  const int lpn = choice >= 2 ? 16 : 32;
  const int64_t per_sm = (choice & 1) ? 8 : 16;
  return {lpn, grid_for(n * lpn, 256, int64_t(num_sms()) * per_sm)};
}

// dbeta of every layer's edge MLP.  dbeta_l = sum over edges of dm = D_l +
// T_l, where T_l = sum_i indeg(i) da_l[i] and D_l is the column sum of the
// gradient de_l arriving at layer l's edge output.  That gradient is the
// residual pass-through plus the MLP input term, de_{l-1} = de_l + dZ1_l
// W1_e,l^T (the edge-state block of W1), so D_{L-1} = 0 and D_{l-1} = D_l +
// v_l with v_l = db1_l W1_e,l^T.  edge_beta_mv_kernel forms every v_l (block
// l; warp w takes the outputs k = w (mod 8), each a coalesced dot product
// with a fixed shuffle tree); edge_beta_kernel then walks the layers from the
// top.  Layer l's offsets are the layer-0 offsets plus l * stride.
__global__ void __launch_bounds__(256) edge_beta_mv_kernel(const float* __restrict__ P, int64_t w1e0, int64_t b10,
                                                           int64_t stride, const float* __restrict__ G,
                                                           float* __restrict__ v) {
  __shared__ float db1[128];
  const int l = blockIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t o = int64_t(l) * stride;
  if (threadIdx.x < 128) db1[threadIdx.x] = G[b10 + o + threadIdx.x];
  __syncthreads();
  const float4 d = reinterpret_cast<const float4*>(db1)[lane];
  for (int k = w; k < 128; k += 8) {  // input feature k of the edge-state block: row 2H + k of W1
    const float4 q = reinterpret_cast<const float4*>(P + w1e0 + o + int64_t(k) * 128)[lane];
    float s = (d.x * q.x + d.y * q.y) + (d.z * q.z + d.w * q.w);
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
    if (lane == 0) v[int64_t(l) * 128 + k] = s;
  }
}

__global__ void edge_beta_kernel(int L, int64_t be0, int64_t stride, const float* __restrict__ tsum,
                                 const float* __restrict__ v, float* __restrict__ G) {
  const int k = threadIdx.x;
  float D = 0.f;
  for (int l = L - 1; l >= 0; --l) {
    G[be0 + int64_t(l) * stride + k] = D + tsum[int64_t(l) * 128 + k];
    D += v[int64_t(l) * 128 + k];
  }
}

// Sums of per-CTA partials, out[i] = sum over parts p of part[p*stride + off
// + i] for i < count, up to kRedJobs outputs per launch (blockIdx.y = job).
// A block owns 32 consecutive outputs; warp w sums the parts p = w (mod 8) in
// four interleaved running sums (p = w + 8m by m mod 4), and the sums are
// combined in a fixed tree: deterministic.
constexpr int kRedJobs = 8;
struct RedJob {
  const float* part;
  int nparts;
  int64_t stride, off, count;
  float* out;
};
struct RedBatch {
  int n;
  RedJob j[kRedJobs];
};

__global__ void __launch_bounds__(256) reduce_parts_kernel(RedBatch b) {
  __shared__ float red[8][32];
  const RedJob& J = b.j[blockIdx.y];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int64_t i0 = int64_t(blockIdx.x) * 32; i0 < J.count; i0 += int64_t(gridDim.x) * 32) {
    const int64_t i = i0 + lane;
    float s = 0.f;
    if (i < J.count) {  // parts w, w+8, ... in four interleaved running sums (independent loads in flight)
      const float* q = J.part + J.off + i;
      float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
      int p = w;
      for (; p + 24 < J.nparts; p += 32) {
        s0 += q[int64_t(p) * J.stride];
        s1 += q[int64_t(p + 8) * J.stride];
        s2 += q[int64_t(p + 16) * J.stride];
        s3 += q[int64_t(p + 24) * J.stride];
      }
      for (; p < J.nparts; p += 8) s0 += q[int64_t(p) * J.stride];
      s = (s0 + s1) + (s2 + s3);
    }
    red[w][lane] = s;
    __syncthreads();
    if (w == 0 && i < J.count)
      J.out[i] = ((red[0][lane] + red[1][lane]) + (red[2][lane] + red[3][lane])) +
                 ((red[4][lane] + red[5][lane]) + (red[6][lane] + red[7][lane]));
    __syncthreads();
  }
}

xmgn_status reduce_batch(const std::vector<RedJob>& jobs, cudaStream_t s) {
  for (size_t b0 = 0; b0 < jobs.size(); b0 += kRedJobs) {
    RedBatch b;
    b.n = int(jobs.size() - b0 < size_t(kRedJobs) ? jobs.size() - b0 : size_t(kRedJobs));
    int64_t most = 1;
    for (int i = 0; i < b.n; ++i) {
      b.j[i] = jobs[b0 + i];
      if (b.j[i].count > most) most = b.j[i].count;
    }
    const int64_t gx = (most + 31) / 32 < 1024 ? (most + 31) / 32 : 1024;
    reduce_parts_kernel<<<dim3(unsigned(gx), unsigned(b.n)), 256, 0, s>>>(b);
    XMGN_LAUNCH_CHECK();
  }
  return XMGN_OK;
}

// bias / gamma / beta gradients from the per-CTA column partials
void col_jobs(std::vector<RedJob>& j, const float* cpart, int nparts, int H, const MlpOff& o, float* G) {
  j.push_back({cpart, nparts, 4 * int64_t(H), 0, o.hid, G + o.b1});
  j.push_back({cpart, nparts, 4 * int64_t(H), H, o.out, G + o.b2});
  if (o.ln) {
    j.push_back({cpart, nparts, 4 * int64_t(H), 2 * int64_t(H), o.out, G + o.g});
    j.push_back({cpart, nparts, 4 * int64_t(H), 3 * int64_t(H), o.out, G + o.be});
  }
}

xmgn_status reduce_cols(const float* cpart, int nparts, int H, const MlpOff& o, float* G, cudaStream_t s) {
  std::vector<RedJob> j;
  col_jobs(j, cpart, nparts, H, o, G);
  return reduce_batch(j, s);
}

MlpImgs imgs_of(const uint8_t* base, const Img& a, const Img& b, const Img* al = nullptr,
                const Img* bl = nullptr) {
  MlpImgs m;
  m.w1 = base + a.off;
  m.w2 = base + b.off;
  m.w1lo = al ? base + al->off : nullptr;
  m.w2lo = bl ? base + bl->off : nullptr;
  m.w1_bytes = a.bytes();
  m.w2_bytes = b.bytes();
  return m;
}

MlpParams params_of(const float* P, const MlpOff& o) {
  MlpParams m;
  m.b1 = P + o.b1;
  m.b2 = P + o.b2;
  m.gamma = o.ln ? P + o.g : nullptr;
  m.beta = o.ln ? P + o.be : nullptr;
  return m;
}

xmgn_status pack_all(const ParamPlan& p, const ImgPlan& ip, const float* P, uint8_t* img, cudaStream_t s) {
  const uint32_t H = p.H;
  std::vector<PackJob> j;
  j.reserve(12 + 10 * p.L);
  for (int lo = 0; lo < 2; ++lo) {
    j.push_back(pack_job(img, lo ? ip.new1l : ip.new1, 0, H, H, p.in_enc, P + p.ne.W1, H, 0, 0, lo));
    j.push_back(pack_job(img, lo ? ip.new2l : ip.new2, 0, H, H, H, P + p.ne.W2, H, 0, 0, lo));
    j.push_back(pack_job(img, lo ? ip.eew1l : ip.eew1, 0, H, H, kInEdge, P + p.ee.W1, H, 0, 0, lo));
    j.push_back(pack_job(img, lo ? ip.eew2l : ip.eew2, 0, H, H, H, P + p.ee.W2, H, 0, 0, lo));
    j.push_back(pack_job(img, lo ? ip.dw1l : ip.dw1, 0, H, H, H, P + p.dec.W1, H, 0, 0, lo));
    j.push_back(pack_job(img, lo ? ip.dw2l : ip.dw2, 0, 16, p.out, H, P + p.dec.W2, p.out, 0, 0, lo));
  }
  for (int l = 0; l < p.L; ++l) {
    const LayerImgs& li = ip.layer[l];
    const MlpOff& e = p.edge[l];
    const MlpOff& nd = p.node[l];
    for (int lo = 0; lo < 2; ++lo) {
      j.push_back(pack_job(img, lo ? li.ew1el : li.ew1e, 0, H, H, H, P + e.W1, H, 2 * H, 0, lo));
      j.push_back(pack_job(img, lo ? li.ew2l : li.ew2, 0, H, H, H, P + e.W2, H, 0, 0, lo));
    }
    j.push_back(pack_job(img, li.ewrs, 0, H, H, H, P + e.W1, H, 0, 0));  // receiver block
    j.push_back(pack_job(img, li.ewrs, H, H, H, H, P + e.W1, H, H, 0));  // sender block
    for (int lo = 0; lo < 2; ++lo) {
      j.push_back(pack_job(img, lo ? li.nw1l : li.nw1, 0, H, H, 2 * H, P + nd.W1, H, 0, 0, lo));
      j.push_back(pack_job(img, lo ? li.nw2l : li.nw2, 0, H, H, H, P + nd.W2, H, 0, 0, lo));
    }
  }
  return pack_images(j, s);
}

Bf16Rows rows_of(const bf16* p, int w, const bf16* p1 = nullptr, int w1 = 0) {
  Bf16Rows r;
  r.p0 = p;
  r.ld0 = w;
  r.w0 = w;
  r.p1 = p1;
  r.ld1 = w1;
  r.w1 = w1;
  return r;
}

}  // namespace

bool bf16_supported(const ParamPlan& p) { return p.H == 128 && p.in_enc <= 32 && p.out <= 16; }

void bf16_sizes(const ParamPlan& p, int64_t n, int64_t E, size_t* ws, size_t* ckpt, bool offload, size_t* host) {
  Arena a, b;
  a.dry = b.dry = true;
  BWs w;
  BCkpt c;
  ImgPlan ip = make_imgs(p);
  ws_layout(a, p, n, E, w);
  ckpt_layout(b, p, ip, n, E, c, offload);
  *ws = a.used + 256;
  *ckpt = b.used + 256;
  if (host) *host = offload ? size_t(p.L) * size_t(E) * size_t(p.H) * sizeof(bf16) : 0;
}

namespace {
// Copy stream and events of the checkpoint offload, one set per device.
struct OffloadCtx {
  cudaStream_t copy = nullptr;
  cudaEvent_t used[kRing], moved[kRing], sync[2];
};

xmgn_status offload_ctx(OffloadCtx** out) {
  static OffloadCtx ctx[64];
  static bool made[64] = {};
  int dev = 0;
  XMGN_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(XMGN_ERR_UNSUPPORTED, "device index %d", dev);
  OffloadCtx& c = ctx[dev];
  if (!made[dev]) {
    XMGN_CUDA(cudaStreamCreateWithFlags(&c.copy, cudaStreamNonBlocking));
    for (int i = 0; i < kRing; ++i) {
      XMGN_CUDA(cudaEventCreateWithFlags(&c.used[i], cudaEventDisableTiming));
      XMGN_CUDA(cudaEventCreateWithFlags(&c.moved[i], cudaEventDisableTiming));
    }
    for (int i = 0; i < 2; ++i) XMGN_CUDA(cudaEventCreateWithFlags(&c.sync[i], cudaEventDisableTiming));
    made[dev] = true;
  }
  *out = &c;
  return XMGN_OK;
}
}  // namespace

xmgn_status bf16_forward(const ParamPlan& p, const float* P, const xmgn_graph& g, const float* node_in,
                         const float* xyz, const float* targets, float* y, float* loss, void* ckpt,
                         size_t ckpt_bytes, void* ws, size_t ws_bytes, cudaStream_t s, void* host_e16) {
  const int64_t n = g.n_nodes, E = g.n_edges;
  const int H = p.H;
  const ImgPlan ip = make_imgs(p);
  Arena A{static_cast<char*>(ws), ws_bytes};
  Arena C{static_cast<char*>(ckpt), ckpt_bytes};
  BWs w;
  BCkpt c;
  const bool off = host_e16 != nullptr && p.L > 1 && E > 0;
  ws_layout(A, p, n, E, w);
  ckpt_layout(C, p, ip, n, E, c, host_e16 != nullptr);
  if (!A.ok() || !C.ok()) return fail(XMGN_ERR_WORKSPACE, "bf16 forward: ws/ckpt too small");
  const size_t layer_elems = size_t(E) * H;
  // e^l: its own checkpoint slot, or ring slot l % kRing whose content is
  // copied to host memory once layer l's edge kernel has read it
  auto e_at = [&](int l) { return c.e16 + (host_e16 ? size_t(l % kRing) : size_t(l)) * layer_elems; };
  OffloadCtx* oc = nullptr;
  if (off) XMGN_TRY(offload_ctx(&oc));
  uint32_t* err = device_error_word();
  XMGN_TRY(pack_all(p, ip, P, c.img, s));

  FwdArgs f{};
  f.H = H;
  f.err = err;
  f.gid = g.gid;
  f.recv = g.recv;
  f.col = g.col;
  // node encoder
  f.rows = n;
  f.fin = node_in;
  f.fin_w = p.in_node;
  f.xyz = xyz;
  f.fourier = p.fourier;
  f.w = imgs_of(c.img, ip.new1, ip.new2, &ip.new1l, &ip.new2l);
  f.p = params_of(P, p.ne);
  f.o32 = c.h32;
  f.o16 = c.h16;
  XMGN_TRY(mlp_fwd_tc(M_NENC, f, s));
  // edge encoder: its inputs once as bf16 rows (also for the backward), then the MLP
  XMGN_TRY(edge_inputs_bf16(xyz, g.gid, g.recv, g.col, E, c.feat8, s));
  f.rows = E;
  f.fin = xyz;
  f.feat8 = c.feat8;
  f.w = imgs_of(c.img, ip.eew1, ip.eew2, &ip.eew1l, &ip.eew2l);
  f.p = params_of(P, p.ee);
  f.o32 = nullptr;
  f.o16 = e_at(0);
  XMGN_TRY(mlp_fwd_tc(M_EENC, f, s));
  for (int l = 0; l < p.L; ++l) {
    const LayerImgs& li = ip.layer[l];
    const bf16* h16 = c.h16 + size_t(l) * n * H;
    const float* h32 = c.h32 + size_t(l) * n * H;
    const bf16* e16 = e_at(l);
    bf16* e16n = (l + 1 < p.L) ? e_at(l + 1) : nullptr;  // no layer reads e^L
    if (off && l + 1 >= kRing)  // e^{l+1} overwrites e^{l+1-kRing}: its copy to host must be done
      XMGN_CUDA(cudaStreamWaitEvent(s, oc->moved[(l + 1) % kRing], 0));
    bf16* a16 = c.a16 + size_t(l) * n * H;
    bf16* Pl = c.P16 ? c.P16 + size_t(l) * n * 2 * H : w.P;  // kept for the backward
    XMGN_TRY(tc_gemm(rows_of(h16, H), n, c.img, li.ewrs, false, 2 * H, nullptr, 2 * H, false, s, Pl));
    FwdArgs fe = f;
    fe.rows = E;
    fe.a0 = e16;
    fe.P = Pl;
    fe.w = imgs_of(c.img, li.ew1e, li.ew2, &li.ew1el, &li.ew2l);
    fe.p = params_of(P, p.edge[l]);
    fe.o16 = e16n;
    fe.agg16 = a16;
    fe.agg_part = w.agg_part;
    XMGN_TRY(mlp_fwd_tc(M_EDGE, fe, s));
    if (off) {  // e^l is read: copy it out on the copy stream
      XMGN_CUDA(cudaEventRecord(oc->used[l % kRing], s));
      XMGN_CUDA(cudaStreamWaitEvent(oc->copy, oc->used[l % kRing], 0));
      XMGN_CUDA(cudaMemcpyAsync(static_cast<bf16*>(host_e16) + size_t(l) * layer_elems, e16,
                                layer_elems * sizeof(bf16), cudaMemcpyDeviceToHost, oc->copy));
      XMGN_CUDA(cudaEventRecord(oc->moved[l % kRing], oc->copy));
    }
    agg_fixup_kernel<<<grid_for(n, 256, int64_t(num_sms()) * 16), 256, 0, s>>>(w.agg_part, g.row_ptr, n, a16);
    XMGN_LAUNCH_CHECK();
    FwdArgs fn = f;
    fn.rows = n;
    fn.a0 = h16;
    fn.a1 = a16;
    fn.r32 = h32;
    fn.w = imgs_of(c.img, li.nw1, li.nw2, &li.nw1l, &li.nw2l);
    fn.p = params_of(P, p.node[l]);
    fn.o32 = c.h32 + size_t(l + 1) * n * H;
    fn.o16 = c.h16 + size_t(l + 1) * n * H;
    XMGN_TRY(mlp_fwd_tc(M_NODE, fn, s));
  }
  FwdArgs fd = f;
  fd.rows = n;
  fd.a0 = c.h16 + size_t(p.L) * n * H;
  fd.w = imgs_of(c.img, ip.dw1, ip.dw2, &ip.dw1l, &ip.dw2l);
  fd.p = params_of(P, p.dec);
  fd.o32 = c.y;
  fd.out_w = p.out;
  XMGN_TRY(mlp_fwd_tc(M_DEC, fd, s));
  if (targets || y)
    XMGN_TRY(mse_loss(c.y, n, p.out, targets, g.gid, g.hop, g.n_norm, targets ? loss : nullptr, nullptr, y,
                      w.losspart, s));
  if (off) {  // the stream's work ends after the last copy
    XMGN_CUDA(cudaEventRecord(oc->sync[0], oc->copy));
    XMGN_CUDA(cudaStreamWaitEvent(s, oc->sync[0], 0));
  }
  return XMGN_OK;
}

xmgn_status bf16_backward(const ParamPlan& p, const float* P, const xmgn_graph& g, const float* node_in,
                          const float* xyz, const float* targets, const void* ckpt, size_t ckpt_bytes,
                          float* dparams, float* dcomp, void* ws, size_t ws_bytes, cudaStream_t s,
                          const void* host_e16) {
  const int64_t n = g.n_nodes, E = g.n_edges;
  const int H = p.H;
  const ImgPlan ip = make_imgs(p);
  Arena A{static_cast<char*>(ws), ws_bytes};
  Arena C{static_cast<char*>(const_cast<void*>(ckpt)), ckpt_bytes};
  BWs w;
  BCkpt c;
  const bool off = host_e16 != nullptr && p.L > 1 && E > 0;
  ws_layout(A, p, n, E, w);
  ckpt_layout(C, p, ip, n, E, c, host_e16 != nullptr);
  if (!A.ok() || !C.ok()) return fail(XMGN_ERR_WORKSPACE, "bf16 backward: ws/ckpt too small");
  const size_t layer_elems = size_t(E) * H;
  auto e_at = [&](int l) { return c.e16 + (host_e16 ? size_t(l % kRing) : size_t(l)) * layer_elems; };
  OffloadCtx* oc = nullptr;
  bool slot_used[kRing] = {};  // ring slot read by a layer of this call
  // e^l from host memory into its ring slot once the layer that last read the slot is done
  auto fetch = [&](int l) -> xmgn_status {
    if (slot_used[l % kRing]) XMGN_CUDA(cudaStreamWaitEvent(oc->copy, oc->used[l % kRing], 0));
    XMGN_CUDA(cudaMemcpyAsync(e_at(l), static_cast<const bf16*>(host_e16) + size_t(l) * layer_elems,
                              layer_elems * sizeof(bf16), cudaMemcpyHostToDevice, oc->copy));
    XMGN_CUDA(cudaEventRecord(oc->moved[l % kRing], oc->copy));
    return XMGN_OK;
  };
  if (off) {
    XMGN_TRY(offload_ctx(&oc));
    XMGN_CUDA(cudaEventRecord(oc->sync[0], s));  // the copy stream starts after the work before this call
    XMGN_CUDA(cudaStreamWaitEvent(oc->copy, oc->sync[0], 0));
    XMGN_TRY(fetch(p.L - 1));
  }
  uint32_t* err = device_error_word();
  float* G = w.grad;
  XMGN_CUDA(cudaMemsetAsync(G, 0, sizeof(float) * size_t(p.total), s));
  XMGN_TRY(mse_loss(c.y, n, p.out, targets, g.gid, g.hop, g.n_norm, nullptr, w.dy32, nullptr, w.losspart, s));

  BwdArgs b{};
  b.H = H;
  b.err = err;
  b.gid = g.gid;
  b.recv = g.recv;
  b.col = g.col;
  b.A1g = w.A1g;
  b.dZ2g = w.dZ2g;
  b.dZ1g = w.dZ1g;
  b.X16g = w.X16;
  b.wpart = w.wpart;
  b.cpart = w.cpart;
  b.spill = w.spill;
  const int gn = mlp_grid(n), ge = mlp_grid(E);
  const bf16* hL = c.h16 + size_t(p.L) * n * H;

  // decoder: y = W2 SiLU(W1 h + b1) + b2
  BwdArgs bd = b;
  bd.rows = n;
  bd.a0 = hL;
  bd.w = imgs_of(c.img, ip.dw1, ip.dw2, &ip.dw1l, &ip.dw2l);
  bd.p = params_of(P, p.dec);
  bd.dY1 = w.dy32;
  bd.dX0 = w.dh;
  bd.out_w = p.out;
  XMGN_TRY(mlp_bwd_tc(M_DEC, bd, s));
  XMGN_TRY(reduce_cols(w.cpart, gn, H, p.dec, G, s));
  XMGN_TRY(tc_gemm_tn(rows_of(hL, H), w.dZ1g, H, H, n, G + p.dec.W1, H, H, H, w.tnpart, s));
  XMGN_TRY(tc_gemm_tn(rows_of(w.A1g, H), w.dZ2g, 64, 64, n, G + p.dec.W2, H, p.out, p.out, w.tnpart, s));

  for (int l = p.L - 1; l >= 0; --l) {
    const LayerImgs& li = ip.layer[l];
    const bf16* h16 = c.h16 + size_t(l) * n * H;
    const bf16* a16 = c.a16 + size_t(l) * n * H;
    const bf16* e16 = e_at(l);
    if (off && l >= 1) XMGN_TRY(fetch(l - 1));  // prefetch the next layer's edge states
    const MlpOff& on = p.node[l];
    const MlpOff& oe = p.edge[l];
    // node update h' = h + MLP_n([h, a])
    BwdArgs bn = b;
    bn.rows = n;
    bn.a0 = h16;
    bn.a1 = a16;
    bn.w = imgs_of(c.img, li.nw1, li.nw2);
    bn.p = params_of(P, on);
    bn.dY1 = w.dh;
    bn.dX0 = w.dh;
    bn.dX1h = w.dagg;
    XMGN_TRY(mlp_bwd_tc(M_NODE, bn, s));
    XMGN_TRY(reduce_cols(w.cpart, gn, H, on, G, s));
    XMGN_TRY(tc_gemm_tn(rows_of(h16, H, a16, H), w.dZ1g, H, H, n, G + on.W1, 2 * H, H, H, w.tnpart, s));
    XMGN_TRY(tc_gemm_tn(rows_of(w.A1g, H), w.dZ2g, H, H, n, G + on.W2, H, H, H, w.tnpart, s));
    // edge update e' = e + m, a_i = sum_j m_ij (node projections checkpointed, or recomputed with offload)
    const bf16* Pl = w.P;
    if (c.P16)
      Pl = c.P16 + size_t(l) * n * 2 * H;
    else
      XMGN_TRY(tc_gemm(rows_of(h16, H), n, c.img, li.ewrs, false, 2 * H, nullptr, 2 * H, false, s, w.P));
    BwdArgs be = b;
    be.rows = E;
    be.a0 = e16;
    be.P = Pl;
    be.w = imgs_of(c.img, li.ew1e, li.ew2, &li.ew1el, &li.ew2l);
    be.p = params_of(P, oe);
    be.dY1h = l + 1 < p.L ? w.de : nullptr;  // nothing reads the top layer's edge output
    be.dY2h = w.dagg;
    be.idx2 = g.recv;
    be.dX0h = w.de;
    if (off) XMGN_CUDA(cudaStreamWaitEvent(s, oc->moved[l % kRing], 0));
    XMGN_TRY(mlp_bwd_tc(M_EDGE, be, s));
    if (off) {
      XMGN_CUDA(cudaEventRecord(oc->used[l % kRing], s));
      slot_used[l % kRing] = true;
    }
    const SegShape ss = seg_shape(n, tune_choice(TUNE_SEG_SUMS, n));
    const unsigned sg = ss.grid;
    tune_begin(TUNE_SEG_SUMS, s);
    if (ss.lpn == 32)
      seg_sums_kernel<32><<<sg, 256, 0, s>>>(w.dZ1g, g.row_ptr, g.csc_perm, n, w.dagg, w.S16, w.colp);
    else
      seg_sums_kernel<16><<<sg, 256, 0, s>>>(w.dZ1g, g.row_ptr, g.csc_perm, n, w.dagg, w.S16, w.colp);
    XMGN_LAUNCH_CHECK();
    tune_end(TUNE_SEG_SUMS, s);
    {  // dW1_e, dW2, db2, dgamma (per-CTA partials of the edge kernel), db1 and T_l (seg_sums partials)
      const int64_t cs = 4 * int64_t(H), ps = 2 * int64_t(H);
      std::vector<RedJob> j = {{w.colp, int(sg), ps, 0, H, G + oe.b1},
                               {w.colp, int(sg), ps, H, H, w.tsum + int64_t(l) * H}};
      if (E > 0) {  // without edges the edge kernel left no partials (those gradients stay zero)
        j.push_back({w.wpart, ge, 2 * 128 * int64_t(H), 0, int64_t(H) * H, G + oe.W1 + 2 * int64_t(H) * H});
        j.push_back({w.wpart, ge, 2 * 128 * int64_t(H), 128 * int64_t(H), int64_t(H) * H, G + oe.W2});
        j.push_back({w.cpart, ge, cs, H, H, G + oe.b2});
        j.push_back({w.cpart, ge, cs, 2 * int64_t(H), H, G + oe.g});
      }
      XMGN_TRY(reduce_batch(j, s));
    }
    XMGN_TRY(tc_gemm(rows_of(w.S16, 2 * H), n, c.img, li.ewrs, true, H, w.dh, H, true, s));
    XMGN_TRY(tc_gemm_tn(rows_of(h16, H), w.S16, 2 * H, 2 * H, n, G + oe.W1, H, 2 * H, H, w.tnpart, s));
  }
  {  // dbeta of the edge MLPs from db1 and T_l (the edge kernel does not sum it)
    const int64_t stride = p.L > 1 ? p.edge[1].W1 - p.edge[0].W1 : 0;
    for (int l = 0; l < p.L; ++l)
      if (p.edge[l].W1 != p.edge[0].W1 + l * stride || p.edge[l].b1 != p.edge[0].b1 + l * stride ||
          p.edge[l].be != p.edge[0].be + l * stride)
        return fail(XMGN_ERR_ARG, "edge MLP parameters are not laid out with a fixed stride per layer");
    edge_beta_mv_kernel<<<p.L, 256, 0, s>>>(P, p.edge[0].W1 + 2 * int64_t(H) * H, p.edge[0].b1, stride, G,
                                            w.vbeta);
    XMGN_LAUNCH_CHECK();
    edge_beta_kernel<<<1, 128, 0, s>>>(p.L, p.edge[0].be, stride, w.tsum, w.vbeta, G);
    XMGN_LAUNCH_CHECK();
  }
  // edge encoder
  BwdArgs bee = b;
  bee.rows = E;
  bee.fin = xyz;
  bee.feat8 = c.feat8;
  bee.w = imgs_of(c.img, ip.eew1, ip.eew2, &ip.eew1l, &ip.eew2l);
  bee.p = params_of(P, p.ee);
  bee.dY1h = w.de;
  bee.dZ1g = nullptr;  // its weight gradients are summed in TMEM: no node-level product reads dZ1
  XMGN_TRY(mlp_bwd_tc(M_EENC, bee, s));
  if (E > 0) {
    std::vector<RedJob> j = {{w.wpart, ge, 2 * 128 * int64_t(H), 0, int64_t(kInEdge) * H, G + p.ee.W1},
                             {w.wpart, ge, 2 * 128 * int64_t(H), 128 * int64_t(H), int64_t(H) * H, G + p.ee.W2}};
    col_jobs(j, w.cpart, ge, H, p.ee, G);
    XMGN_TRY(reduce_batch(j, s));
  }
  // node encoder
  BwdArgs bne = b;
  bne.rows = n;
  bne.fin = node_in;
  bne.fin_w = p.in_node;
  bne.xyz = xyz;
  bne.fourier = p.fourier;
  bne.w = imgs_of(c.img, ip.new1, ip.new2, &ip.new1l, &ip.new2l);
  bne.p = params_of(P, p.ne);
  bne.dY1 = w.dh;
  XMGN_TRY(mlp_bwd_tc(M_NENC, bne, s));
  XMGN_TRY(reduce_cols(w.cpart, gn, H, p.ne, G, s));
  XMGN_TRY(tc_gemm_tn(rows_of(w.X16, 128), w.dZ1g, H, H, n, G + p.ne.W1, p.in_enc, H, H, w.tnpart, s));
  XMGN_TRY(tc_gemm_tn(rows_of(w.A1g, H), w.dZ2g, H, H, n, G + p.ne.W2, H, H, H, w.tnpart, s));
  if (off) {  // join the copy stream
    XMGN_CUDA(cudaEventRecord(oc->sync[1], oc->copy));
    XMGN_CUDA(cudaStreamWaitEvent(s, oc->sync[1], 0));
  }
  return accumulate_grad(dparams, dcomp, G, p.total, s);
}

}  // namespace xmgn
