// Fused two-layer MLP kernels on tcgen05 (see mlp_tc.cuh).
//
// Forward, per 128-row tile:
//   GEMM1  Z1 = X W1            (TMEM cols [0, H))
//   epi1   A1 = SiLU(Z1 + b1 [+ P_r[i] + P_s[j]])  -> bf16 tile in smem
//   GEMM2  Z2 = A1 W2           (TMEM cols [H, 2H))
//   epi2   LayerNorm(Z2 + b2) (+ residual) -> outputs
// Backward, per tile (activations recomputed from the checkpointed inputs):
//   GEMM1, epi1 (Z1 + b1 + gathers written back to TMEM, A1 to smem)
//   GEMM2, epi2  LayerNorm backward -> dZ2 (smem)
//   GEMM3  dA1 = dZ2 W2^T  [+ dW2 += A1^T dZ2 in TMEM]
//   epi3   dZ1 = dA1 * SiLU'(Z1) -> smem (reusing the A1 tile)
//   GEMM4  dX = dZ1 W1^T   [+ dW1 += X^T dZ1 in TMEM]
//   epi4   input gradients (+ residual pass-through)
// W^T products read the forward weight images as MN-major operands, and
// X^T dY products read the activation tiles as MN-major operands, so every
// operand is staged in shared memory exactly once per tile.
// Column sums (bias, gamma, beta gradients) are reduced across the 32 rows of
// a warp with a shuffle transpose and accumulated per lane in registers, in a
// fixed order, so results are deterministic.
#include "mlp_tc.cuh"

namespace xmgn {

using namespace tc;

namespace {

constexpr int kH = 128;
constexpr int kThreads = 128;

__device__ __forceinline__ float silu_f(float z) { return z / (1.f + __expf(-z)); }
__device__ __forceinline__ float silu_grad_f(float z) {
  const float s = 1.f / (1.f + __expf(-z));
  return s * (1.f + z * (1.f - s));
}

// Sum over the 32 lanes of each of the 32 values; lane j returns column j.
__device__ __forceinline__ float col_reduce32(float (&v)[32]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < o; ++i) {
      const float send = up ? v[i] : v[i + o];
      const float keep = up ? v[i + o] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  return v[0];
}

__device__ __forceinline__ void st_tile32(uint8_t* tile, uint32_t R, int r, int c, const float (&v)[32]) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    uint4 u;
    u.x = pack_bf16(v[8 * q + 0], v[8 * q + 1]);
    u.y = pack_bf16(v[8 * q + 2], v[8 * q + 3]);
    u.z = pack_bf16(v[8 * q + 4], v[8 * q + 5]);
    u.w = pack_bf16(v[8 * q + 6], v[8 * q + 7]);
    *reinterpret_cast<uint4*>(tile + sw_chunk(R, r, c / 8 + q)) = u;
  }
}

__device__ __forceinline__ void unpack8(uint4 u, float* f) {
  const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float2 t = __bfloat1622float2(h[i]);
    f[2 * i] = t.x;
    f[2 * i + 1] = t.y;
  }
}

__device__ __forceinline__ void ld_tile32(const uint8_t* tile, uint32_t R, int r, int c, float (&v)[32]) {
#pragma unroll
  for (int q = 0; q < 4; ++q)
    unpack8(*reinterpret_cast<const uint4*>(tile + sw_chunk(R, r, c / 8 + q)), v + 8 * q);
}

__device__ __forceinline__ void st_g16(bf16* dst, const float (&v)[32]) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    uint4 u;
    u.x = pack_bf16(v[8 * q + 0], v[8 * q + 1]);
    u.y = pack_bf16(v[8 * q + 2], v[8 * q + 3]);
    u.z = pack_bf16(v[8 * q + 4], v[8 * q + 5]);
    u.w = pack_bf16(v[8 * q + 6], v[8 * q + 7]);
    reinterpret_cast<uint4*>(dst)[q] = u;
  }
}

__device__ __forceinline__ void st_g32(float* dst, const float (&v)[32]) {
#pragma unroll
  for (int q = 0; q < 8; ++q)
    reinterpret_cast<float4*>(dst)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}

__device__ __forceinline__ void add_g32(float (&v)[32], const float* src) {
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    float4 t = reinterpret_cast<const float4*>(src)[q];
    v[4 * q] += t.x;
    v[4 * q + 1] += t.y;
    v[4 * q + 2] += t.z;
    v[4 * q + 3] += t.w;
  }
}

template <int MODE>
struct Shape {
  static constexpr int XC = MODE == M_NODE ? 2 * kH : (MODE == M_NENC ? 64 : (MODE == M_EENC ? 128 : kH));
  static constexpr int K1S = (MODE == M_NENC || MODE == M_EENC) ? 1 : XC / 16;
  static constexpr int N2 = MODE == M_DEC ? 16 : kH;
  static constexpr int DZC = MODE == M_DEC ? 64 : kH;  // columns of the dZ2 tile
};

__host__ __device__ __forceinline__ uint32_t align1k(uint32_t x) { return (x + 1023u) & ~1023u; }

// Stages the A tile (rows r0..r0+127) of the given mode into `xa`.
template <int MODE, class Args>
__device__ __forceinline__ void load_a_tile(uint8_t* xa, const Args& a, int64_t r0, int tid, bf16* x16g) {
  using S = Shape<MODE>;
  if (MODE == M_EDGE || MODE == M_DEC || MODE == M_NODE) {
    constexpr int cpr = S::XC / 8;
    for (int q = tid; q < 128 * cpr; q += kThreads) {
      const int r = q / cpr, j = q % cpr;
      const int64_t row = r0 + r;
      const bool ok = row < a.rows;
      const int64_t rr = ok ? row : 0;
      const bf16* src = (MODE == M_NODE && j >= kH / 8) ? a.a1 + rr * kH + (j * 8 - kH) : a.a0 + rr * kH + j * 8;
      cp_async16(xa + sw_chunk(128, r, j), src, ok ? 16u : 0u);
    }
    cp_async_commit();
    cp_async_wait<0>();
  } else {
    // one thread per row builds the (few) input features in fp32, stores bf16
    const int r = tid;
    const int64_t row = r0 + r;
    float f[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) f[j] = 0.f;
    if (row < a.rows) {
      if (MODE == M_NENC) {
        const int64_t g = a.gid ? int64_t(a.gid[row]) : row;
        for (int j = 0; j < a.fin_w; ++j) f[j] = a.fin[g * a.fin_w + j];
      } else {
        int64_t i = a.recv[row], jn = a.col[row];
        if (a.gid) {
          i = a.gid[i];
          jn = a.gid[jn];
        }
        const float dx = a.fin[3 * jn] - a.fin[3 * i];
        const float dy = a.fin[3 * jn + 1] - a.fin[3 * i + 1];
        const float dz = a.fin[3 * jn + 2] - a.fin[3 * i + 2];
        f[0] = dx;
        f[1] = dy;
        f[2] = dz;
        f[3] = sqrtf(dx * dx + dy * dy + dz * dz);
      }
    }
    st_tile32(xa, 128, r, 0, f);
    float z[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) z[j] = 0.f;
    st_tile32(xa, 128, r, 32, z);
    if (S::XC == 128) {
      st_tile32(xa, 128, r, 64, z);
      st_tile32(xa, 128, r, 96, z);
    }
    if (x16g && row < a.rows) {
      st_g16(x16g + row * 128, f);
      st_g16(x16g + row * 128 + 32, z);
      st_g16(x16g + row * 128 + 64, z);
      st_g16(x16g + row * 128 + 96, z);
    }
  }
}

struct Smem {
  uint8_t *w1, *w2, *xa, *a1, *dz2;
};

template <int MODE>
__device__ __forceinline__ Smem carve(uint8_t* base, uint32_t w1b, uint32_t w2b, bool bwd) {
  using S = Shape<MODE>;
  Smem s;
  uint32_t o = 0;
  s.w1 = base + o;
  o += align1k(w1b);
  s.w2 = base + o;
  o += align1k(w2b);
  s.xa = base + o;
  o += align1k(128u * S::XC * 2u);
  s.a1 = base + o;
  o += 128u * kH * 2u;
  s.dz2 = bwd ? base + o : nullptr;
  return s;
}

template <int MODE>
uint32_t smem_bytes(uint32_t w1b, uint32_t w2b, bool bwd) {
  using S = Shape<MODE>;
  uint32_t o = align1k(w1b) + align1k(w2b) + align1k(128u * S::XC * 2u) + 128u * kH * 2u;
  if (bwd) o += 128u * S::DZC * 2u;
  return o + 1024u;
}

__device__ __forceinline__ bool setup(uint64_t* wbar, uint64_t* mbar, uint32_t* tbase, uint32_t ncols,
                                      const MlpImgs& w, uint8_t* w1, uint8_t* w2, uint32_t* err) {
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(wbar, 1);
    mbar_init(mbar, 1);
    fence_barrier_init();
  }
  if ((tid >> 5) == 0) {
    tmem_alloc(tbase, ncols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (tid == 0) {
    mbar_arrive_expect_tx(wbar, w.w1_bytes + w.w2_bytes);
    for (uint32_t o = 0; o < w.w1_bytes; o += 16384u)
      bulk_g2s(w1 + o, w.w1 + o, min(16384u, w.w1_bytes - o), wbar);
    for (uint32_t o = 0; o < w.w2_bytes; o += 16384u)
      bulk_g2s(w2 + o, w.w2 + o, min(16384u, w.w2_bytes - o), wbar);
  }
  return mbar_wait(wbar, 0, err);
}

// ============================================================ forward
template <int MODE>
__global__ void __launch_bounds__(kThreads, 1) mlp_fwd_kernel(FwdArgs a) {
  using S = Shape<MODE>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ uint64_t wbar, mbar;
  __shared__ uint32_t tbase;
  const Smem sm = carve<MODE>(base, a.w.w1_bytes, a.w.w2_bytes, false);
  const int tid = threadIdx.x, warp = tid >> 5;
  bool ok = setup(&wbar, &mbar, &tbase, 256, a.w, sm.w1, sm.w2, a.err);
  const uint32_t tm = tbase;
  const uint32_t lane_base = uint32_t(warp * 32) << 16;
  const int64_t tiles = (a.rows + 127) / 128;
  uint32_t ph = 0;
  for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    if (__syncthreads_or(!ok)) break;
    const int64_t r0 = t * 128;
    load_a_tile<MODE>(sm.xa, a, r0, tid, nullptr);
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t xs = smem_u32(sm.xa), ws = smem_u32(sm.w1);
      const uint32_t id = idesc_bf16(128, kH, false, false);
#pragma unroll 1
      for (int k = 0; k < S::K1S; ++k) mma_bf16(tm, kmajor_desc(xs, 128, k), kmajor_desc(ws, kH, k), id, k > 0);
      mma_commit(&mbar);
    }
    ok = mbar_wait(&mbar, ph, a.err);
    ph ^= 1;
    if (__syncthreads_or(!ok)) break;
    tc_fence_after();
    const int64_t row = r0 + tid;
    const bool valid = row < a.rows;
    int64_t rcv = 0, snd = 0;
    if (MODE == M_EDGE && valid) {
      rcv = a.recv[row];
      snd = a.col[row];
    }
    float v[32];
#pragma unroll 1
    for (int c = 0; c < kH; c += 32) {
      tmem_ld32(tm + lane_base + c, v);
      add_g32(v, a.p.b1 + c);
      if (MODE == M_EDGE && valid) {
        add_g32(v, a.P + rcv * 2 * kH + c);
        add_g32(v, a.P + snd * 2 * kH + kH + c);
      }
#pragma unroll
      for (int j = 0; j < 32; ++j) v[j] = silu_f(v[j]);
      st_tile32(sm.a1, 128, tid, c, v);
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t as = smem_u32(sm.a1), ws = smem_u32(sm.w2);
      const uint32_t id = idesc_bf16(128, S::N2, false, false);
#pragma unroll 1
      for (int k = 0; k < kH / 16; ++k)
        mma_bf16(tm + kH, kmajor_desc(as, 128, k), kmajor_desc(ws, S::N2, k), id, k > 0);
      mma_commit(&mbar);
    }
    ok = mbar_wait(&mbar, ph, a.err);
    ph ^= 1;
    if (__syncthreads_or(!ok)) break;
    tc_fence_after();
    if (MODE == M_DEC) {
      tmem_ld32(tm + lane_base + kH, v);
      if (valid)
        for (int o = 0; o < a.out_w; ++o) a.o32[row * a.out_w + o] = v[o] + a.p.b2[o];
    } else {
      float s = 0.f;
#pragma unroll 1
      for (int c = 0; c < kH; c += 32) {
        tmem_ld32(tm + lane_base + kH + c, v);
        add_g32(v, a.p.b2 + c);
#pragma unroll
        for (int j = 0; j < 32; ++j) s += v[j];
      }
      const float mu = s * (1.f / kH);
      float q = 0.f;
#pragma unroll 1
      for (int c = 0; c < kH; c += 32) {
        tmem_ld32(tm + lane_base + kH + c, v);
        add_g32(v, a.p.b2 + c);
#pragma unroll
        for (int j = 0; j < 32; ++j) q += (v[j] - mu) * (v[j] - mu);
      }
      const float rstd = rsqrtf(q * (1.f / kH) + kLnEps);
#pragma unroll 1
      for (int c = 0; c < kH; c += 32) {
        tmem_ld32(tm + lane_base + kH + c, v);
        add_g32(v, a.p.b2 + c);
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = (v[j] - mu) * rstd * a.p.gamma[c + j] + a.p.beta[c + j];
        if (!valid) continue;
        if (MODE == M_EDGE) {
          st_g32(a.o32 + row * kH + c, v);  // message m_ij (eq. 1)
          float e[32];
          ld_tile32(sm.xa, 128, tid, c, e);
#pragma unroll
          for (int j = 0; j < 32; ++j) e[j] += v[j];
          st_g16(a.o16 + row * kH + c, e);
        } else if (MODE == M_NODE) {
          add_g32(v, a.r32 + row * kH + c);
          st_g32(a.o32 + row * kH + c, v);
          st_g16(a.o16 + row * kH + c, v);
        } else if (MODE == M_NENC) {
          st_g32(a.o32 + row * kH + c, v);
          st_g16(a.o16 + row * kH + c, v);
        } else {
          st_g16(a.o16 + row * kH + c, v);
        }
      }
    }
    tc_fence_before();
    __syncthreads();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tm, 256);
}

// ============================================================ backward
template <int MODE>
__global__ void __launch_bounds__(kThreads, 1) mlp_bwd_kernel(BwdArgs a) {
  using S = Shape<MODE>;
  constexpr bool TMW = MODE == M_EDGE || MODE == M_EENC;
  constexpr bool HAS_DX = MODE == M_EDGE || MODE == M_NODE || MODE == M_DEC;
  constexpr bool LN = MODE != M_DEC;
  constexpr int NX = MODE == M_NODE ? 2 * kH : kH;
  constexpr uint32_t tZ1 = 0, tZ2 = kH, tDX = 0, tW1 = 256, tW2 = 384;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ uint64_t wbar, mbar;
  __shared__ uint32_t tbase;
  const Smem sm = carve<MODE>(base, a.w.w1_bytes, a.w.w2_bytes, true);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  bool ok = setup(&wbar, &mbar, &tbase, 512, a.w, sm.w1, sm.w2, a.err);
  const uint32_t tm = tbase;
  const uint32_t lane_base = uint32_t(warp * 32) << 16;
  const int64_t tiles = (a.rows + 127) / 128;
  float cacc[4][kH / 32];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int j = 0; j < kH / 32; ++j) cacc[q][j] = 0.f;
  uint32_t ph = 0;
  bool first = true;
  for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    if (__syncthreads_or(!ok)) break;
    const int64_t r0 = t * 128;
    load_a_tile<MODE>(sm.xa, a, r0, tid, MODE == M_NENC ? a.X16g : nullptr);
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    // ---- GEMM1
    if (tid == 0) {
      tc_fence_after();
      const uint32_t xs = smem_u32(sm.xa), ws = smem_u32(sm.w1);
      const uint32_t id = idesc_bf16(128, kH, false, false);
#pragma unroll 1
      for (int k = 0; k < S::K1S; ++k) mma_bf16(tm + tZ1, kmajor_desc(xs, 128, k), kmajor_desc(ws, kH, k), id, k > 0);
      mma_commit(&mbar);
    }
    ok = mbar_wait(&mbar, ph, a.err);
    ph ^= 1;
    if (__syncthreads_or(!ok)) break;
    tc_fence_after();
    const int64_t row = r0 + tid;
    const bool valid = row < a.rows;
    int64_t rcv = 0, snd = 0;
    if (MODE == M_EDGE && valid) {
      rcv = a.recv[row];
      snd = a.col[row];
    }
    float v[32];
    // ---- epi1: full pre-activation back to TMEM, SiLU to smem
#pragma unroll 1
    for (int c = 0; c < kH; c += 32) {
      tmem_ld32(tm + lane_base + tZ1 + c, v);
      add_g32(v, a.p.b1 + c);
      if (MODE == M_EDGE && valid) {
        add_g32(v, a.P + rcv * 2 * kH + c);
        add_g32(v, a.P + snd * 2 * kH + kH + c);
      }
      tmem_st32(tm + lane_base + tZ1 + c, v);
#pragma unroll
      for (int j = 0; j < 32; ++j) v[j] = silu_f(v[j]);
      st_tile32(sm.a1, 128, tid, c, v);
      if (!TMW && valid) st_g16(a.A1g + row * kH + c, v);
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    // ---- GEMM2 (not needed without LayerNorm)
    if (LN) {
      if (tid == 0) {
        tc_fence_after();
        const uint32_t as = smem_u32(sm.a1), ws = smem_u32(sm.w2);
        const uint32_t id = idesc_bf16(128, kH, false, false);
#pragma unroll 1
        for (int k = 0; k < kH / 16; ++k) mma_bf16(tm + tZ2, kmajor_desc(as, 128, k), kmajor_desc(ws, kH, k), id, k > 0);
        mma_commit(&mbar);
      }
      ok = mbar_wait(&mbar, ph, a.err);
      ph ^= 1;
      if (__syncthreads_or(!ok)) break;
      tc_fence_after();
    }
    // ---- epi2: LayerNorm backward -> dZ2
    if (!LN) {
      for (int j = 0; j < 32; ++j) v[j] = (valid && j < a.out_w) ? a.dY1[row * a.out_w + j] : 0.f;
      st_tile32(sm.dz2, 128, tid, 0, v);
      if (valid) st_g16(a.dZ2g + row * 64, v);
      float z[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) z[j] = 0.f;
      st_tile32(sm.dz2, 128, tid, 32, z);
      if (valid) st_g16(a.dZ2g + row * 64 + 32, z);
      cacc[1][0] += col_reduce32(v);
    } else {
      const float* dy2 = nullptr;
      if (a.dY2 && valid) dy2 = a.dY2 + (a.idx2 ? int64_t(a.idx2[row]) : row) * kH;
      const float* dy1 = (a.dY1 && valid) ? a.dY1 + row * kH : nullptr;
      float s = 0.f;
#pragma unroll 1
      for (int c = 0; c < kH; c += 32) {
        tmem_ld32(tm + lane_base + tZ2 + c, v);
        add_g32(v, a.p.b2 + c);
#pragma unroll
        for (int j = 0; j < 32; ++j) s += v[j];
      }
      const float mu = s * (1.f / kH);
      float q = 0.f;
#pragma unroll 1
      for (int c = 0; c < kH; c += 32) {
        tmem_ld32(tm + lane_base + tZ2 + c, v);
        add_g32(v, a.p.b2 + c);
#pragma unroll
        for (int j = 0; j < 32; ++j) q += (v[j] - mu) * (v[j] - mu);
      }
      const float rstd = rsqrtf(q * (1.f / kH) + kLnEps);
      float sg = 0.f, sgx = 0.f;
#pragma unroll 1
      for (int c = 0; c < kH; c += 32) {
        float dm[32], t2[32];
        tmem_ld32(tm + lane_base + tZ2 + c, v);
        add_g32(v, a.p.b2 + c);
#pragma unroll
        for (int j = 0; j < 32; ++j) dm[j] = 0.f;
        if (dy1) add_g32(dm, dy1 + c);
        if (dy2) add_g32(dm, dy2 + c);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const float xh = (v[j] - mu) * rstd;
          const float g = dm[j] * a.p.gamma[c + j];
          sg += g;
          sgx += g * xh;
          t2[j] = dm[j] * xh;
        }
        const float rb = col_reduce32(dm);
        const float rg = col_reduce32(t2);
        cacc[3][c / 32] += rb;
        cacc[2][c / 32] += rg;
      }
      const float mg = sg * (1.f / kH), mgx = sgx * (1.f / kH);
#pragma unroll 1
      for (int c = 0; c < kH; c += 32) {
        float dm[32];
        tmem_ld32(tm + lane_base + tZ2 + c, v);
        add_g32(v, a.p.b2 + c);
#pragma unroll
        for (int j = 0; j < 32; ++j) dm[j] = 0.f;
        if (dy1) add_g32(dm, dy1 + c);
        if (dy2) add_g32(dm, dy2 + c);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const float xh = (v[j] - mu) * rstd;
          v[j] = rstd * (dm[j] * a.p.gamma[c + j] - mg - xh * mgx);
        }
        st_tile32(sm.dz2, 128, tid, c, v);
        if (!TMW && valid) st_g16(a.dZ2g + row * kH + c, v);
        cacc[1][c / 32] += col_reduce32(v);
      }
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    // ---- GEMM3: dA1 = dZ2 W2^T  [+ dW2 += A1^T dZ2]
    if (tid == 0) {
      tc_fence_after();
      const uint32_t ds = smem_u32(sm.dz2), ws = smem_u32(sm.w2), as = smem_u32(sm.a1);
      const uint32_t id = idesc_bf16(128, kH, false, true);
#pragma unroll 1
      for (int k = 0; k < S::N2 / 16; ++k)
        mma_bf16(tm + tZ2, kmajor_desc(ds, 128, k), mnmajor_desc(ws, S::N2, k), id, k > 0);
      if (TMW) {
        const uint32_t idw = idesc_bf16(128, kH, true, true);
#pragma unroll 1
        for (int k = 0; k < 8; ++k)
          mma_bf16(tm + tW2, mnmajor_desc(as, 128, k), mnmajor_desc(ds, 128, k), idw, (first && k == 0) ? 0u : 1u);
      }
      mma_commit(&mbar);
    }
    ok = mbar_wait(&mbar, ph, a.err);
    ph ^= 1;
    if (__syncthreads_or(!ok)) break;
    tc_fence_after();
    // ---- epi3: dZ1 = dA1 * SiLU'(Z1)
#pragma unroll 1
    for (int c = 0; c < kH; c += 32) {
      float z[32];
      tmem_ld32(tm + lane_base + tZ2 + c, v);
      tmem_ld32(tm + lane_base + tZ1 + c, z);
#pragma unroll
      for (int j = 0; j < 32; ++j) v[j] *= silu_grad_f(z[j]);
      if (!valid) {
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = 0.f;
      }
      st_tile32(sm.a1, 128, tid, c, v);
      if (valid) st_g16(a.dZ1g + row * kH + c, v);
      cacc[0][c / 32] += col_reduce32(v);
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    // ---- GEMM4: dX = dZ1 W1^T  [+ dW1 += X^T dZ1]
    if (HAS_DX || TMW) {
      if (tid == 0) {
        tc_fence_after();
        const uint32_t ds = smem_u32(sm.a1), ws = smem_u32(sm.w1), xs = smem_u32(sm.xa);
        if (HAS_DX) {
          const uint32_t id = idesc_bf16(128, NX, false, true);
#pragma unroll 1
          for (int k = 0; k < kH / 16; ++k) mma_bf16(tm + tDX, kmajor_desc(ds, 128, k), mnmajor_desc(ws, kH, k), id, k > 0);
        }
        if (TMW) {
          const uint32_t idw = idesc_bf16(128, kH, true, true);
#pragma unroll 1
          for (int k = 0; k < 8; ++k)
            mma_bf16(tm + tW1, mnmajor_desc(xs, 128, k), mnmajor_desc(ds, 128, k), idw, (first && k == 0) ? 0u : 1u);
        }
        mma_commit(&mbar);
      }
      ok = mbar_wait(&mbar, ph, a.err);
      ph ^= 1;
      if (__syncthreads_or(!ok)) break;
      tc_fence_after();
    }
    // ---- epi4: input gradients
    if (HAS_DX) {
#pragma unroll 1
      for (int c = 0; c < NX; c += 32) {
        tmem_ld32(tm + lane_base + tDX + c, v);
        if (!valid) continue;
        if (MODE == M_EDGE) {
          if (a.dY1) add_g32(v, a.dY1 + row * kH + c);
          st_g32(a.dX0 + row * kH + c, v);
        } else if (MODE == M_NODE) {
          if (c < kH) {
            add_g32(v, a.dY1 + row * kH + c);
            st_g32(a.dX0 + row * kH + c, v);
          } else {
            st_g32(a.dX1 + row * kH + (c - kH), v);
          }
        } else {
          st_g32(a.dX0 + row * kH + c, v);
        }
      }
    }
    first = false;
    tc_fence_before();
    __syncthreads();
  }
  // ---- partial outputs of this CTA
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (TMW) {
#pragma unroll 1
    for (int m = 0; m < 2; ++m) {
      float* P = a.wpart + ((int64_t(blockIdx.x) * 2 + m) * 128 + tid) * kH;
#pragma unroll 1
      for (int c = 0; c < kH; c += 32) {
        float w[32];
        tmem_ld32(tm + lane_base + (m == 0 ? tW1 : tW2) + c, w);
        if (first || !ok) {
#pragma unroll
          for (int j = 0; j < 32; ++j) w[j] = 0.f;
        }
        st_g32(P + c, w);
      }
    }
  }
  float* red = reinterpret_cast<float*>(sm.xa);  // [4 warps][4][kH]
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int j = 0; j < kH / 32; ++j) red[(warp * 4 + q) * kH + 32 * j + lane] = cacc[q][j];
  __syncthreads();
  for (int q = 0; q < 4; ++q) {
    float s = 0.f;
    for (int w = 0; w < 4; ++w) s += red[(w * 4 + q) * kH + tid];
    a.cpart[(int64_t(blockIdx.x) * 4 + q) * kH + tid] = s;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tm, 512);
}

template <class K>
xmgn_status set_smem(K kernel) {
  return allow_max_smem(kernel);
}

template <int MODE>
xmgn_status launch_fwd(const FwdArgs& a, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    XMGN_TRY(set_smem(mlp_fwd_kernel<MODE>));
    attr = true;
  }
  const uint32_t sm = smem_bytes<MODE>(a.w.w1_bytes, a.w.w2_bytes, false);
  mlp_fwd_kernel<MODE><<<mlp_grid(a.rows), kThreads, sm, s>>>(a);
  XMGN_LAUNCH_CHECK();
  return XMGN_OK;
}

template <int MODE>
xmgn_status launch_bwd(const BwdArgs& a, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    XMGN_TRY(set_smem(mlp_bwd_kernel<MODE>));
    attr = true;
  }
  const uint32_t sm = smem_bytes<MODE>(a.w.w1_bytes, a.w.w2_bytes, true);
  if (sm > 227u * 1024u) return fail(XMGN_ERR_UNSUPPORTED, "bwd smem %u", sm);
  mlp_bwd_kernel<MODE><<<mlp_grid(a.rows), kThreads, sm, s>>>(a);
  XMGN_LAUNCH_CHECK();
  return XMGN_OK;
}

}  // namespace

int mlp_grid(int64_t rows) { return tc_grid((rows + 127) / 128); }

xmgn_status mlp_fwd_tc(int mode, const FwdArgs& a, cudaStream_t s) {
  if (a.H != kH) return fail(XMGN_ERR_UNSUPPORTED, "bf16 MLP kernels are built for H=%d", kH);
  if (a.rows <= 0) return XMGN_OK;
  switch (mode) {
    case M_EDGE: return launch_fwd<M_EDGE>(a, s);
    case M_NODE: return launch_fwd<M_NODE>(a, s);
    case M_DEC: return launch_fwd<M_DEC>(a, s);
    case M_NENC: return launch_fwd<M_NENC>(a, s);
    case M_EENC: return launch_fwd<M_EENC>(a, s);
  }
  return fail(XMGN_ERR_ARG, "bad mode");
}

xmgn_status mlp_bwd_tc(int mode, const BwdArgs& a, cudaStream_t s) {
  if (a.H != kH) return fail(XMGN_ERR_UNSUPPORTED, "bf16 MLP kernels are built for H=%d", kH);
  if (a.rows <= 0) return XMGN_OK;
  switch (mode) {
    case M_EDGE: return launch_bwd<M_EDGE>(a, s);
    case M_NODE: return launch_bwd<M_NODE>(a, s);
    case M_DEC: return launch_bwd<M_DEC>(a, s);
    case M_NENC: return launch_bwd<M_NENC>(a, s);
    case M_EENC: return launch_bwd<M_EENC>(a, s);
  }
  return fail(XMGN_ERR_ARG, "bad mode");
}

}  // namespace xmgn
