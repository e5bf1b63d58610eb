// Fused two-layer MLP kernels on tcgen05 (see mlp_tc.cuh).
//
// Forward, per 128-row tile:
//   GEMM1  Z1 = X W1            (TMEM cols [0, H))
//   epi1   A1 = SiLU(Z1 + b1 [+ P_r[i] + P_s[j]])  -> bf16 tile in smem
//   GEMM2  Z2 = A1 W2           (TMEM cols [H, 2H))
//   epi2   LayerNorm(Z2 + b2) (+ residual) -> outputs
// Backward, per tile (activations recomputed from the checkpointed inputs):
//   GEMM1, epi1 (A1 to smem; SiLU'(Z1) back to TMEM)
//   GEMM2, epi2  LayerNorm backward -> dZ2 (smem)
//   GEMM3  dA1 = dZ2 W2^T  [+ dW2 += A1^T dZ2 in TMEM]
//   epi3   dZ1 = dA1 * SiLU'(Z1) -> smem (reusing the A1 tile)
//   GEMM4  dX = dZ1 W1^T   [+ dW1 += X^T dZ1 in TMEM]
//   epi4   input gradients (+ residual pass-through)
// mlp_fwd_kernel serves the encoders and the decoder, mlp_bwd_kernel those
// and the node MLP; the node update forward has node_fwd_kernel (operands in
// TMEM), the edge update edge_fwd_kernel (two 8-warp groups, A1 kept in TMEM,
// the messages summed per receiver in the epilogue, eq. 2) and
// edge_bwd_kernel (same phases as above, its own shared-memory plan).
// W^T products read the forward weight images as MN-major operands, and
// X^T dY products read the activation tiles as MN-major operands, so every
// operand is staged in shared memory exactly once per tile.
//
// Weight precision: in the forward-direction products (GEMM1, GEMM2, also when
// recomputed in the backward) a weight matrix W is applied as W_hi + W_lo,
// both bf16 (W_hi = bf16(W), W_lo = bf16(W - W_hi)), i.e. two MMAs into the
// same fp32 accumulator; activations stay single bf16.  The backward W^T
// products use W_hi only.  (Rounding the weights of the forward products was
// the largest error term at 15 layers.)  The backward of the node and edge
// MLPs recomputes with W_hi only (no shared memory left for the low parts).
//
// Threads: 16 warps.  Warp w reads TMEM lanes 32*(w%4).. (tile rows) and owns
// the 32 columns 32*(w/4).. of every H-wide accumulator, so each thread holds
// one 32-column slice of one row.  Per-row LayerNorm statistics are combined
// over the four column slices through shared memory in a fixed order.  Column
// sums (bias, gamma, beta gradients) are reduced across the 32 rows of a warp
// with a shuffle transpose and accumulated per lane, again in a fixed order,
// so every result is deterministic.
#include <cuda.h>

#include "mlp_tc.cuh"
#include "tune.cuh"

namespace xmgn {

using namespace tc;

namespace {

constexpr int kH = 128;
constexpr int kThreads = 512;

// SiLU with the fast exponential and fast division intrinsics (a huge
// denominator gives 0, the correct limit).
__device__ __forceinline__ float silu_f(float z) { return __fdividef(z, 1.f + __expf(-z)); }

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

// Row-slice global accesses use 256-bit per-thread loads and stores (every
// slice is 64- or 128-byte aligned): half the memory instructions of 128-bit
// accesses, and each thread touches whole 32-byte sectors.
__device__ __forceinline__ void ld8(const float* p, float* v) {
  asm volatile("ld.global.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
               : "l"(p));
}
__device__ __forceinline__ void st8(float* p, const float* v) {
  asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(v[0]), "f"(v[1]), "f"(v[2]),
               "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
               : "memory");
}
__device__ __forceinline__ void st8u(void* p, const uint32_t* u) {
  asm volatile("st.global.v8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "r"(u[0]), "r"(u[1]), "r"(u[2]),
               "r"(u[3]), "r"(u[4]), "r"(u[5]), "r"(u[6]), "r"(u[7])
               : "memory");
}

__device__ __forceinline__ void st_g16(bf16* dst, const float (&v)[32]) {
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    uint32_t u[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) u[i] = pack_bf16(v[16 * q + 2 * i], v[16 * q + 2 * i + 1]);
    st8u(dst + 16 * q, u);
  }
}

__device__ __forceinline__ void st_g32(float* dst, const float (&v)[32]) {
#pragma unroll
  for (int q = 0; q < 4; ++q) st8(dst + 8 * q, v + 8 * q);
}

__device__ __forceinline__ void ld_g32(float (&v)[32], const float* src) {
#pragma unroll
  for (int q = 0; q < 4; ++q) ld8(src + 8 * q, v + 8 * q);
}

__device__ __forceinline__ void add_g32(float (&v)[32], const float* src) {
  float t[32];
  ld_g32(t, src);
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] += t[j];
}

// v += 32 bf16 values at src (64 bytes, two 256-bit loads)
__device__ __forceinline__ void add_g16(float (&v)[32], const bf16* src) {
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    uint32_t u[8];
    asm volatile("ld.global.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7])
                 : "l"(src + 16 * q));
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u[i]));
      v[16 * q + 2 * i] += f.x;
      v[16 * q + 2 * i + 1] += f.y;
    }
  }
}

// 32 bf16 values at src, packed in pairs (two 256-bit loads).
__device__ __forceinline__ void ld_raw16(uint32_t (&u)[16], const bf16* src) {
#pragma unroll
  for (int q = 0; q < 2; ++q)
    asm volatile("ld.global.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(u[8 * q]), "=r"(u[8 * q + 1]), "=r"(u[8 * q + 2]), "=r"(u[8 * q + 3]), "=r"(u[8 * q + 4]),
                   "=r"(u[8 * q + 5]), "=r"(u[8 * q + 6]), "=r"(u[8 * q + 7])
                 : "l"(src + 16 * q));
}
// Element j of 32 packed bf16 values (exact widening).
__device__ __forceinline__ float bf16_at(const uint32_t (&u)[16], int j) {
  return __uint_as_float((j & 1) ? (u[j >> 1] & 0xffff0000u) : (u[j >> 1] << 16));
}

// v = 32 bf16 values at src
__device__ __forceinline__ void ld_g16(float (&v)[32], const bf16* src) {
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = 0.f;
  add_g16(v, src);
}

// Copies rows [r0, min(r0+128, rows)) of a swizzled 128 x 128 bf16 tile to
// row-major global memory: consecutive threads move consecutive 16-byte
// chunks of a row, so each warp writes two full rows per instruction.
__device__ __forceinline__ void copy_tile_out(const uint8_t* tile, bf16* dst, int64_t r0, int64_t rows, int tid,
                                              int nthr = kThreads) {
  for (int q = tid; q < 128 * 16; q += nthr) {
    const int r = q >> 4, j = q & 15;
    if (r0 + r < rows)
      *reinterpret_cast<uint4*>(dst + (r0 + r) * kH + 8 * j) = *reinterpret_cast<const uint4*>(tile + sw_chunk(128, r, j));
  }
}

// Tile k of this CTA's share of `tiles` 128-row tiles of a persistent launch:
// dealt round-robin (order 0: tiles b, b + G, b + 2G, ...) or as one
// contiguous run (order 1: tiles b*per .. b*per + per - 1, per = ceil(tiles /
// G)).  Returns `tiles` past the end of the share.
__device__ __forceinline__ int64_t cta_tile(int order, int64_t k, int64_t tiles) {
  const int64_t b = blockIdx.x, G = gridDim.x;
  if (order == 0) {
    const int64_t t = b + k * G;
    return t < tiles ? t : tiles;
  }
  const int64_t per = (tiles + G - 1) / G;
  const int64_t t = b * per + k;
  return (k < per && t < tiles) ? t : tiles;
}

// Aggregation (eq. 2) of one 128-edge tile whose messages m_ij sit, rounded to
// bf16, in the swizzled tile `mt`.  Edges are sorted by receiver, so every
// receiver owns a contiguous run of rows; the tile holds nseg runs, run q
// starting at row first[q], and srecv[k] is row k's receiver.  Eight lanes
// sum run q, q + nthr/8, ... in row order in fp32, lane l of the eight owning
// features 8l..8l+7 and 64+8l..64+8l+7 (so that the eight lanes of a run read
// eight different 16-byte slots of a row).  A run that lies wholly in the
// tile is the complete sum and is written, rounded to bf16, to agg16; the run
// that began in an earlier tile (head) and the run that goes on into the next
// tile (tail) are written in fp32 to part[t][0] and part[t][1] for
// agg_fixup_kernel (a run spanning the whole tile counts as the head).
__device__ __forceinline__ void aggregate_tile(const uint8_t* mt, const int32_t* srecv, const uint8_t* first,
                                               int nseg, int64_t rows, int64_t t, uint32_t ht, bf16* agg16,
                                               float* part, int tid, int nthr) {
  const int64_t r0 = t * 128;
  const int nrows = rows - r0 < 128 ? int(rows - r0) : 128;
  const int ql = tid & 7;
#pragma unroll 1
  for (int q = tid >> 3; q < nseg; q += nthr / 8) {
    const int b = first[q];
    const int e = q + 1 < nseg ? int(first[q + 1]) : nrows;
    float lo[8], hi[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) lo[j] = hi[j] = 0.f;
#pragma unroll 4
    for (int k = b; k < e; ++k) {
      float x[8], y[8];
      unpack8(*reinterpret_cast<const uint4*>(mt + sw_chunk(128, k, ql)), x);
      unpack8(*reinterpret_cast<const uint4*>(mt + sw_chunk(128, k, 8 + ql)), y);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        lo[j] += x[j];
        hi[j] += y[j];
      }
    }
    const bool head = q == 0 && (ht & 1u), tail = !head && q == nseg - 1 && (ht & 2u);
    if (head || tail) {
      float* d = part + (t * 2 + (head ? 0 : 1)) * kH + 8 * ql;
      reinterpret_cast<float4*>(d)[0] = make_float4(lo[0], lo[1], lo[2], lo[3]);
      reinterpret_cast<float4*>(d)[1] = make_float4(lo[4], lo[5], lo[6], lo[7]);
      reinterpret_cast<float4*>(d + 64)[0] = make_float4(hi[0], hi[1], hi[2], hi[3]);
      reinterpret_cast<float4*>(d + 64)[1] = make_float4(hi[4], hi[5], hi[6], hi[7]);
    } else {
      bf16* d = agg16 + int64_t(srecv[b]) * kH + 8 * ql;
      *reinterpret_cast<uint4*>(d) = make_uint4(pack_bf16(lo[0], lo[1]), pack_bf16(lo[2], lo[3]),
                                                pack_bf16(lo[4], lo[5]), pack_bf16(lo[6], lo[7]));
      *reinterpret_cast<uint4*>(d + 64) = make_uint4(pack_bf16(hi[0], hi[1]), pack_bf16(hi[2], hi[3]),
                                                     pack_bf16(hi[4], hi[5]), pack_bf16(hi[6], hi[7]));
    }
  }
}

// Element j of a 16-byte-aligned shared-memory vector; with j a compile-time
// constant after unrolling, four consecutive j share one 16-byte load.
__device__ __forceinline__ float cst(const float* p, int j) {
  const float4 t = reinterpret_cast<const float4*>(p)[j >> 2];
  return (j & 3) == 0 ? t.x : (j & 3) == 1 ? t.y : (j & 3) == 2 ? t.z : t.w;
}

template <int MODE>
struct Shape {
  static constexpr int XC = MODE == M_NODE ? 2 * kH : (MODE == M_NENC ? 64 : (MODE == M_EENC ? 128 : kH));
  static constexpr int K1S = MODE == M_NENC ? 2 : (MODE == M_EENC ? 1 : XC / 16);  // NENC: <= 32 inputs
  static constexpr int N2 = MODE == M_DEC ? 16 : kH;
  static constexpr bool ASYNC_A = MODE == M_DEC || MODE == M_NODE || MODE == M_EENC;  // operand tile staged with cp.async
  static constexpr bool TMW = MODE == M_EENC;  // weight gradients kept in TMEM
  static constexpr bool SPLIT = MODE != M_NODE;  // hi + lo weights in the generic kernels' forward products
  // forward: two ping-pong buffers serve as operand tile and A1 tile
  static constexpr bool PINGPONG = MODE == M_DEC;
};

__host__ __device__ __forceinline__ uint32_t align1k(uint32_t x) { return (x + 1023u) & ~1023u; }

// Issues cp.async copies of the A tile (rows r0..r0+127) of a bf16-row mode.
// The edge encoder's rows are 8 bf16 (one 16-byte chunk: four inputs and
// zeros); its first product reads 16 columns, so the second chunk is zeroed.
template <int MODE, class Args>
__device__ __forceinline__ void issue_a_tile(uint8_t* xa, const Args& a, int64_t r0, int tid) {
  using S = Shape<MODE>;
  if constexpr (MODE == M_EENC) {
    if (tid < 128) {
      const int64_t row = r0 + tid;
      const bool ok = row < a.rows;
      cp_async16(xa + sw_chunk(128, tid, 0), a.feat8 + (ok ? row : 0) * 8, ok ? 16u : 0u);
      *reinterpret_cast<uint4*>(xa + sw_chunk(128, tid, 1)) = make_uint4(0u, 0u, 0u, 0u);
    }
    return;
  }
  constexpr int cpr = S::XC / 8;
  for (int q = tid; q < 128 * cpr; q += kThreads) {
    const int r = q / cpr, j = q % cpr;
    const int64_t row = r0 + r;
    const bool ok = row < a.rows;
    const int64_t rr = ok ? row : 0;
    const bf16* src = (MODE == M_NODE && j >= kH / 8) ? a.a1 + rr * kH + (j * 8 - kH) : a.a0 + rr * kH + j * 8;
    cp_async16(xa + sw_chunk(128, r, j), src, ok ? 16u : 0u);
  }
}

// Builds the A tile of the encoder modes (few fp32 features per row).
template <int MODE, class Args>
__device__ __forceinline__ void build_feature_tile(uint8_t* xa, const Args& a, int64_t r0, int tid, bf16* x16g) {
  using S = Shape<MODE>;
  if (tid >= 128) return;
  const int r = tid;
  const int64_t row = r0 + r;
  float f[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) f[j] = 0.f;
  if (row < a.rows) {
    if (MODE == M_NENC) {
      const int64_t g = a.gid ? int64_t(a.gid[row]) : row;
      for (int j = 0; j < a.fin_w; ++j) f[j] = a.fin[g * a.fin_w + j];
      // Fourier features of the coordinates: sin, cos of 2^(q+1) pi x_c
      for (int q = 0; q < a.fourier; ++q) {
        const float fr = float(2 << q);
        for (int c = 0; c < 3; ++c) {
          float sv, cv;
          sincospif(fr * a.xyz[3 * g + c], &sv, &cv);
          f[a.fin_w + 6 * q + c] = sv;
          f[a.fin_w + 6 * q + 3 + c] = cv;
        }
      }
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

// Shared-memory plan.  Forward: w1[hi,lo], w2[hi,lo], then either two
// ping-pong buffers B0/B1 (operand tile of tile i in B[i&1], its A1 tile in
// the other, the next operand tile prefetched into that one once GEMM2 is
// done) or separate xa and a1.  Backward: w1[hi,lo], w2[hi,lo], xa, a1; the
// dZ2 tile reuses xa (modes with TMEM weight gradients; xa is reloaded for
// X^T dZ1) or a1 (the others, where A1 is dead after GEMM2); dZ1 reuses a1.
struct Smem {
  uint8_t *w1h, *w1l, *w2h, *w2l, *buf[2], *a1, *dz2;
  float* cst;  // b1, b2, gamma, beta (4 x kH)
  float* red;  // 4 x 4 x kH row-statistics / column-sum scratch
};

template <int MODE>
__host__ __device__ __forceinline__ uint32_t carve_bytes(const MlpImgs& w, bool bwd, Smem* s, uint8_t* base) {
  using S = Shape<MODE>;
  uint32_t o = 0;
  auto at = [&](uint32_t bytes) {
    uint8_t* p = base ? base + o : nullptr;
    o += align1k(bytes);
    return p;
  };
  Smem m;
  m.w1h = at(w.w1_bytes);
  m.w1l = S::SPLIT ? at(w.w1_bytes) : nullptr;
  m.w2h = at(w.w2_bytes);
  m.w2l = S::SPLIT ? at(w.w2_bytes) : nullptr;
  const uint32_t xbytes = 128u * S::XC * 2u;
  if (!bwd && S::PINGPONG) {
    m.buf[0] = at(xbytes);
    m.buf[1] = at(xbytes);
    m.a1 = nullptr;
  } else {
    m.buf[0] = m.buf[1] = at(xbytes);
    m.a1 = at(128u * kH * 2u);
  }
  m.dz2 = bwd ? (S::TMW ? m.buf[0] : m.a1) : nullptr;
  m.cst = reinterpret_cast<float*>(at(4u * kH * 4u));
  m.red = reinterpret_cast<float*>(at(4u * 4u * kH * 4u));
  if (s) *s = m;
  return o;
}

template <int MODE>
uint32_t smem_bytes(const MlpImgs& w, bool bwd) {
  return carve_bytes<MODE>(w, bwd, nullptr, nullptr) + 1024u;
}

template <int MODE>
__device__ __forceinline__ bool setup(uint64_t* wbar, uint64_t* mbar, uint32_t* tbase, uint32_t ncols,
                                      const MlpImgs& w, const MlpParams& p, int n2, const Smem& sm,
                                      uint32_t* err) {
  using S = Shape<MODE>;
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
  if (tid < kH) {
    sm.cst[tid] = p.b1[tid];
    sm.cst[kH + tid] = tid < n2 ? p.b2[tid] : 0.f;
    sm.cst[2 * kH + tid] = p.gamma ? p.gamma[tid] : 0.f;
    sm.cst[3 * kH + tid] = p.beta ? p.beta[tid] : 0.f;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const bool lo = sm.w1l != nullptr;  // the backward of the edge and node MLPs recomputes with W_hi only
  if (tid == 0) {
    const uint32_t total = (lo ? 2u : 1u) * (w.w1_bytes + w.w2_bytes);
    mbar_arrive_expect_tx(wbar, total);
    auto copy = [&](uint8_t* dst, const uint8_t* src, uint32_t bytes) {
      for (uint32_t o = 0; o < bytes; o += 16384u) bulk_g2s(dst + o, src + o, min(16384u, bytes - o), wbar);
    };
    copy(sm.w1h, w.w1, w.w1_bytes);
    copy(sm.w2h, w.w2, w.w2_bytes);
    if (lo) {
      copy(sm.w1l, w.w1lo, w.w1_bytes);
      copy(sm.w2l, w.w2lo, w.w2_bytes);
    }
  }
  return mbar_wait(wbar, 0, err);
}

// GEMM1 / GEMM2 of the forward direction: X W_hi [+ X W_lo].
template <int MODE>
__device__ __forceinline__ void fwd_gemm(uint32_t d, uint32_t xs, uint32_t R_b, uint32_t wh, uint32_t wl, int ksteps,
                                         int N) {
  using S = Shape<MODE>;
  const uint32_t id = idesc_bf16(128, N, false, false);
#pragma unroll 1
  for (int k = 0; k < ksteps; ++k) mma_bf16(d, kmajor_desc(xs, 128, k), kmajor_desc(wh, R_b, k), id, k > 0);
  if (S::SPLIT) {
#pragma unroll 1
    for (int k = 0; k < ksteps; ++k) mma_bf16(d, kmajor_desc(xs, 128, k), kmajor_desc(wl, R_b, k), id, 1u);
  }
}

// The four warps that hold the column slices of the same 32 rows (lane
// quadrant r / 32 of a 16-warp CTA) meet at named barrier 1 + r / 32: row
// statistics need no CTA-wide barrier.
__device__ __forceinline__ void quadrant_sync(int r) { asm volatile("bar.sync %0, 128;" ::"r"(1 + (r >> 5)) : "memory"); }

// Sum over the four column slices of row r (fixed order).
__device__ __forceinline__ float row_total(float* red, int slot, int cq, int r, float part) {
  red[(slot * 4 + cq) * kH + r] = part;
  quadrant_sync(r);
  const float* p = red + slot * 4 * kH + r;
  return (p[0] + p[kH]) + (p[2 * kH] + p[3 * kH]);
}

// Two row sums (slots a and b) behind one barrier.
__device__ __forceinline__ float2 row_total2(float* red, int a, int b, int cq, int r, float pa, float pb) {
  red[(a * 4 + cq) * kH + r] = pa;
  red[(b * 4 + cq) * kH + r] = pb;
  quadrant_sync(r);
  const float* p = red + a * 4 * kH + r;
  const float* q = red + b * 4 * kH + r;
  return make_float2((p[0] + p[kH]) + (p[2 * kH] + p[3 * kH]), (q[0] + q[kH]) + (q[2 * kH] + q[3 * kH]));
}

// Tensor map of a row-major [rows, 128] bf16 array in boxes of 64 columns x
// 128 rows with the 128-byte swizzle of the MMA operand tiles.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
xmgn_status rows_map(CUtensorMap* m, const void* base, int64_t rows) {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    XMGN_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !p) return fail(XMGN_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
    fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  if (!base || rows < 1 || rows >= (int64_t(1) << 31) || (reinterpret_cast<uintptr_t>(base) & 15u))
    return fail(XMGN_ERR_ARG, "tensor map: bad base or row count");
  const cuuint64_t dims[2] = {cuuint64_t(kH), cuuint64_t(rows)};
  const cuuint64_t strides[1] = {cuuint64_t(kH) * 2u};
  const cuuint32_t box[2] = {64u, 128u};
  const cuuint32_t es[2] = {1u, 1u};
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(XMGN_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", int(r));
  return XMGN_OK;
}

// ============================================================ forward
template <int MODE>
__global__ void __launch_bounds__(kThreads, 1) mlp_fwd_kernel(FwdArgs a) {
  static_assert(MODE != M_EDGE && MODE != M_NODE, "the edge and node updates have their own forward kernels");
  using S = Shape<MODE>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ uint64_t wbar, mbar;
  __shared__ uint32_t tbase;
  Smem sm;
  carve_bytes<MODE>(a.w, false, &sm, base);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int sp = warp & 3, cq = warp >> 2;
  const int r = sp * 32 + lane;  // tile row (TMEM lane) of this thread
  const int c0 = cq * 32;        // first of the 32 columns of this thread
  bool ok = setup<MODE>(&wbar, &mbar, &tbase, 256, a.w, a.p, MODE == M_DEC ? a.out_w : kH, sm, a.err);
  const uint32_t tm = tbase;
  const uint32_t lane_base = uint32_t(sp * 32) << 16;
  const int64_t tiles = (a.rows + 127) / 128;
  const float* b1 = sm.cst;
  const float* b2 = sm.cst + kH;
  const float* gam = sm.cst + 2 * kH;
  const float* bet = sm.cst + 3 * kH;
  uint32_t ph = 0;
  int i = 0;
  for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x, ++i) {
    if (__syncthreads_or(!ok)) break;
    const int64_t r0 = t * 128;
    uint8_t* xa = sm.buf[i & 1];
    uint8_t* a1 = S::PINGPONG ? sm.buf[(i + 1) & 1] : sm.a1;
    if (S::ASYNC_A) {
      if (i == 0) {
        issue_a_tile<MODE>(xa, a, r0, tid);
        cp_async_commit();
      }
      cp_async_wait<0>();  // this tile (issued here or prefetched during the previous one)
    } else {
      build_feature_tile<MODE>(xa, a, r0, tid, nullptr);
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      fwd_gemm<MODE>(tm, smem_u32(xa), kH, smem_u32(sm.w1h), S::SPLIT ? smem_u32(sm.w1l) : 0u, S::K1S, kH);
      mma_commit(&mbar);
    }
    const int64_t row = r0 + r;
    const bool valid = row < a.rows;
    float v[32];
    ok = mbar_wait(&mbar, ph, a.err);
    ph ^= 1;
    if (__syncthreads_or(!ok)) break;
    tc_fence_after();
    if (S::ASYNC_A && !S::PINGPONG && t + gridDim.x < tiles) {  // GEMM1 consumed the operand tile
      issue_a_tile<MODE>(xa, a, (t + gridDim.x) * 128, tid);
      cp_async_commit();
    }
    tmem_ld32(tm + lane_base + c0, v);
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      v[j] = silu_f(v[j] + cst(b1 + c0, j));
    }
    st_tile32(a1, 128, r, c0, v);
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      fwd_gemm<MODE>(tm + kH, smem_u32(a1), S::N2, smem_u32(sm.w2h), S::SPLIT ? smem_u32(sm.w2l) : 0u, kH / 16,
                     S::N2);
      mma_commit(&mbar);
    }
    ok = mbar_wait(&mbar, ph, a.err);
    ph ^= 1;
    if (__syncthreads_or(!ok)) break;
    tc_fence_after();
    if (S::PINGPONG && t + gridDim.x < tiles) {  // A1 is consumed: prefetch the next operand tile into it
      issue_a_tile<MODE>(a1, a, (t + gridDim.x) * 128, tid);
      cp_async_commit();
    }
    if (MODE == M_DEC) {
      if (cq == 0) {
        tmem_ld32(tm + lane_base + kH, v);
        if (valid)
          for (int o = 0; o < a.out_w; ++o) a.o32[row * a.out_w + o] = v[o] + b2[o];
      }
    } else {
      tmem_ld32(tm + lane_base + kH + c0, v);
      float s = 0.f;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        v[j] += cst(b2 + c0, j);
        s += v[j];
      }
      const float mu = row_total(sm.red, 0, cq, r, s) * (1.f / kH);
      float q = 0.f;
#pragma unroll
      for (int j = 0; j < 32; ++j) q += (v[j] - mu) * (v[j] - mu);
      const float rstd = rsqrtf(row_total(sm.red, 1, cq, r, q) * (1.f / kH) + kLnEps);
#pragma unroll
      for (int j = 0; j < 32; ++j) v[j] = (v[j] - mu) * rstd * cst(gam + c0, j) + cst(bet + c0, j);
      if (valid) {
        if (MODE == M_NENC) st_g32(a.o32 + row * kH + c0, v);
        st_g16(a.o16 + row * kH + c0, v);
      }
    }
    tc_fence_before();
  }
  cp_async_wait<0>();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tm, 256);
}

// ============================================================ edge forward, two groups
// The edge update runs as two independent groups of 8 warps in one CTA, each
// streaming its own 128-edge tiles through the same phases (load e, GEMM1,
// SiLU, GEMM2, LayerNorm, e' = e + m, aggregation), so that one group's
// memory and tensor latencies overlap the other group's arithmetic.  The
// groups share the weight images (W1_e and W2, hi + lo) in shared memory and
// split TMEM by columns: group g owns [256g, 256g + 256), Z1 in the first 128
// (overwritten by the packed bf16 A1 once every Z1 value of the tile has been
// read; GEMM2 takes A1 from TMEM) and Z2 in the last 128.  Warp w of group g
// reads TMEM lanes 32*(w%4).. and owns columns 64*((w/4)%2).. in two 32-wide
// chunks; LayerNorm row statistics combine the two column halves in fixed
// order through shared memory.  Group barriers are named barriers 1 + g.
struct EdgeFwdSmem {
  uint8_t *w1h, *w1l, *w2h, *w2l, *x[2];  // x[g]: group g's edge-state / output / message tile
  float* cst;
  float* red;  // [g][slot 2][half 2][128]
};

__host__ __device__ __forceinline__ uint32_t carve_edge_fwd(const MlpImgs& w, EdgeFwdSmem* s, uint8_t* base) {
  uint32_t o = 0;
  auto at = [&](uint32_t bytes) {
    uint8_t* p = base ? base + o : nullptr;
    o += align1k(bytes);
    return p;
  };
  EdgeFwdSmem m;
  m.w1h = at(w.w1_bytes);
  m.w1l = at(w.w1_bytes);
  m.w2h = at(w.w2_bytes);
  m.w2l = at(w.w2_bytes);
  m.x[0] = at(128u * kH * 2u);
  m.x[1] = at(128u * kH * 2u);
  m.cst = reinterpret_cast<float*>(at(4u * kH * 4u));
  m.red = reinterpret_cast<float*>(at(2u * 2u * 2u * 128u * 4u));
  if (s) *s = m;
  return o;
}

__device__ __forceinline__ void group_sync(int g) { asm volatile("bar.sync %0, 256;" ::"r"(1 + g) : "memory"); }
// AND of `p` over the 256 threads of group g (also a group barrier).
__device__ __forceinline__ bool group_all(int g, bool p) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred q, o;\n\tsetp.ne.u32 q, %1, 0;\n\tbar.red.and.pred o, %2, 256, q;\n\tselp.u32 %0, 1, 0, o;\n\t}"
      : "=r"(r)
      : "r"(p ? 1u : 0u), "r"(1 + g)
      : "memory");
  return r != 0;
}

__global__ void __launch_bounds__(kThreads, 1) edge_fwd_kernel(FwdArgs a, const __grid_constant__ CUtensorMap me) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ uint64_t wbar, mb[2], eb[2];
  __shared__ uint32_t tbase;
  __shared__ uint32_t seg_start[2][4], seg_ht[2];
  __shared__ int32_t seg_recv[2][128];
  __shared__ uint8_t seg_first[2][128];  // first row of each receiver run of the group's tile, in run order
  EdgeFwdSmem sm;
  carve_edge_fwd(a.w, &sm, base);
  Smem ss{};
  ss.w1h = sm.w1h;
  ss.w1l = sm.w1l;
  ss.w2h = sm.w2h;
  ss.w2l = sm.w2l;
  ss.cst = sm.cst;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = warp >> 3, gt = tid & 255;
  const int sp = warp & 3, ch = (warp >> 2) & 1;
  const int r = sp * 32 + lane;
  if (tid == 0) {  // setup() initialises mb[0] and fences these
    mbar_init(&mb[1], 1);
    mbar_init(&eb[0], 1);
    mbar_init(&eb[1], 1);
  }
  bool ok = setup<M_EDGE>(&wbar, &mb[0], &tbase, 512, a.w, a.p, kH, ss, a.err);
  const uint32_t T = tbase + 256u * g;  // this group's TMEM columns
  const uint32_t lane_base = uint32_t(sp * 32) << 16;
  const int64_t tiles = (a.rows + 127) / 128;
  const int64_t G = gridDim.x;
  uint8_t* const X = sm.x[g];
  float* const red = sm.red + g * (2 * 2 * 128);
  uint32_t* const sstart = seg_start[g];
  int32_t* const srecv = seg_recv[g];
  uint8_t* const sfirst = seg_first[g];
  const float* b1 = sm.cst;
  const float* b2 = sm.cst + kH;
  const float* gam = sm.cst + 2 * kH;
  const float* bet = sm.cst + 3 * kH;
  const uint32_t id_x = idesc_bf16(128, kH, false, false);
  uint32_t ph = 0, eph = 0;
  bool gok = group_all(g, ok);
  for (int64_t k = 0; gok; ++k) {
    const int64_t t = cta_tile(a.order, 2 * k + g, tiles);  // the CTA's tiles alternate between its groups
    if (t >= tiles) break;
    const int64_t r0 = t * 128;
    const int nrows = a.rows - r0 < 128 ? int(a.rows - r0) : 128;
    // ---- GEMM1: Z1 = e (W1_hi + W1_lo), the edge-state tile by TMA (rows past the end read as 0)
    bool lok = true;
    if (gt == 0) {
      mbar_arrive_expect_tx(&eb[g], 128u * kH * 2u);
      tma_load_2d(X, &me, 0, int(r0), &eb[g]);
      tma_load_2d(X + 128u * kH, &me, 64, int(r0), &eb[g]);
      const int64_t tn2 = cta_tile(a.order, 2 * k + 2 + g, tiles);  // the group's next edge-state tile, into L2
      if (tn2 < tiles) {
        tma_prefetch_2d(&me, 0, int(tn2 * 128));
        tma_prefetch_2d(&me, 64, int(tn2 * 128));
      }
      lok = mbar_wait(&eb[g], eph, a.err);
      tc_fence_after();
      if (lok) fwd_gemm<M_EDGE>(T, smem_u32(X), kH, smem_u32(sm.w1h), smem_u32(sm.w1l), kH / 16, kH);
      mma_commit(&mb[g]);
    }
    const int64_t row = r0 + r;
    const bool valid = r < nrows;
    const int64_t rcv = valid ? int64_t(a.recv[row]) : 0, snd = valid ? int64_t(a.col[row]) : 0;
    uint32_t pr[16], ps[16];  // 32 bf16 node projections each, packed
    const int cA = 64 * ch;   // first of this thread's 64 columns
    if (valid) {
      ld_raw16(pr, a.P + rcv * 2 * kH + cA);
      ld_raw16(ps, a.P + snd * 2 * kH + kH + cA);
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j) pr[j] = ps[j] = 0u;
    }
    // every thread observes the edge-state tile's arrival itself (it reads the tile for e' = e + m)
    gok = group_all(g, mbar_wait(&mb[g], ph, a.err) && lok && mbar_wait(&eb[g], eph, a.err));
    ph ^= 1;
    eph ^= 1;
    if (!gok) break;
    tc_fence_after();
    // ---- epi1: A1 = SiLU(Z1 + b1 + P_r + P_s), packed bf16, into TMEM over Z1
    uint32_t ap[2][16];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int cc = cA + 32 * c;
      float v[32];
      tmem_ld32(T + lane_base + cc, v);
      if (c == 1 && valid) {  // the second chunk's node projections
        ld_raw16(pr, a.P + rcv * 2 * kH + cc);
        ld_raw16(ps, a.P + snd * 2 * kH + kH + cc);
      }
#pragma unroll
      for (int j = 0; j < 32; ++j) v[j] = silu_f(v[j] + cst(b1 + cc, j) + bf16_at(pr, j) + bf16_at(ps, j));
#pragma unroll
      for (int i = 0; i < 16; ++i) ap[c][i] = pack_bf16(v[2 * i], v[2 * i + 1]);
    }
    tc_fence_before();
    group_sync(g);  // every Z1 value of the tile has been read
    tc_fence_after();
    tmem_st16(T + lane_base + cA / 2, ap[0]);
    tmem_st16(T + lane_base + cA / 2 + 16, ap[1]);
    tc_fence_before();
    group_sync(g);
    // ---- GEMM2: Z2 = A1 (W2_hi + W2_lo), A1 from TMEM
    if (gt == 0) {
      tc_fence_after();
      const uint32_t wh = smem_u32(sm.w2h), wl = smem_u32(sm.w2l);
#pragma unroll 1
      for (int kk = 0; kk < kH / 16; ++kk) mma_bf16_ts(T + kH, T + 8 * kk, kmajor_desc(wh, kH, kk), id_x, kk > 0);
#pragma unroll 1
      for (int kk = 0; kk < kH / 16; ++kk) mma_bf16_ts(T + kH, T + 8 * kk, kmajor_desc(wl, kH, kk), id_x, 1u);
      mma_commit(&mb[g]);
    }
    {  // the group's next tile's node projections, for its epi1, towards L2 (one line per block and row)
      const int64_t tn2 = cta_tile(a.order, 2 * k + 2 + g, tiles);
      const int64_t rn = tn2 * 128 + r;
      if (tn2 < tiles && rn < a.rows) {
        prefetch_l2(a.P + int64_t(a.recv[rn]) * 2 * kH + cA);
        prefetch_l2(a.P + int64_t(a.col[rn]) * 2 * kH + kH + cA);
      }
    }
    if (ch == 0) {  // receiver runs of this tile, while GEMM2 runs
      const int32_t rc = valid ? int32_t(rcv) : -1;
      const int32_t rp = (valid && r > 0) ? a.recv[row - 1] : -1;
      const uint32_t m = __ballot_sync(0xffffffffu, valid && (r == 0 || rc != rp));
      if (lane == 0) sstart[sp] = m;
      srecv[r] = rc;
      if (gt == 0) {
        const bool head = r0 > 0 && a.recv[r0 - 1] == rc;
        const bool tail = r0 + 128 < a.rows && a.recv[r0 + 128] == a.recv[r0 + 127];
        seg_ht[g] = (head ? 1u : 0u) | (tail ? 2u : 0u);
      }
    }
    gok = group_all(g, mbar_wait(&mb[g], ph, a.err));
    ph ^= 1;
    if (!gok) break;
    tc_fence_after();
    if (ch == 0 && ((sstart[sp] >> lane) & 1u)) {  // run order of the runs' first rows
      int idx = __popc(sstart[sp] & ((1u << lane) - 1u));
      for (int w = 0; w < sp; ++w) idx += __popc(sstart[w]);
      sfirst[idx] = uint8_t(r);
    }
    // ---- epi2: LayerNorm statistics over the two column halves of each row
    float sum = 0.f;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int cc = cA + 32 * c;
      float v[32];
      tmem_ld32(T + lane_base + kH + cc, v);
#pragma unroll
      for (int j = 0; j < 32; ++j) sum += v[j] + cst(b2 + cc, j);
    }
    red[(0 * 2 + ch) * 128 + r] = sum;
    group_sync(g);
    const float mu = (red[0 * 128 + r] + red[1 * 128 + r]) * (1.f / kH);
    float qs = 0.f;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int cc = cA + 32 * c;
      float v[32];
      tmem_ld32(T + lane_base + kH + cc, v);
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const float d = v[j] + cst(b2 + cc, j) - mu;
        qs += d * d;
      }
    }
    red[(1 * 2 + ch) * 128 + r] = qs;
    group_sync(g);
    const float rstd = rsqrtf((red[2 * 128 + r] + red[3 * 128 + r]) * (1.f / kH) + kLnEps);
    // messages m_ij = LN(Z2 + b2) (eq. 1): e' = e + m goes straight to global
    // memory (this thread's 32 columns of the row are 64 contiguous bytes),
    // m replaces e in the staged tile, to be summed per receiver (eq. 2)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int cc = cA + 32 * c;
      float v[32];
      tmem_ld32(T + lane_base + kH + cc, v);
#pragma unroll
      for (int j = 0; j < 32; ++j) v[j] = (v[j] + cst(b2 + cc, j) - mu) * rstd * cst(gam + cc, j) + cst(bet + cc, j);
      if (a.o16) {
        float e[32];
        ld_tile32(X, 128, r, cc, e);
#pragma unroll
        for (int j = 0; j < 32; ++j) e[j] += v[j];
        if (valid) st_g16(a.o16 + row * kH + cc, e);
      }
      st_tile32(X, 128, r, cc, v);
    }
    tc_fence_before();
    group_sync(g);
    aggregate_tile(X, srecv, sfirst, __popc(sstart[0]) + __popc(sstart[1]) + __popc(sstart[2]) + __popc(sstart[3]),
                   a.rows, t, seg_ht[g], a.agg16, a.agg_part, gt, 256);
    fence_proxy_async();
    group_sync(g);  // the tile buffer is free for the next load (by the async proxy)
  }
  cp_async_wait<0>();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tbase, 512);
}

// ============================================================ node forward
// The node update (eq. 3 + residual) with W = W_hi + W_lo in both products.
// The operand tile X = [h_i, a_i] (K = 2H) and A1 live in TMEM as packed
// bf16 pairs (the A operand of GEMM1 and GEMM2), which leaves shared memory
// to the four weight images (W1 hi and lo 64 KB each, W2 hi and lo 32 KB
// each).  TMEM columns: Z1 [0, H), Z2 [H, 2H), X [2H, 3H), A1 [3H, 3H + H/2).
// Warp w fills TMEM lanes 32*(w%4).. of X with the 64 operand columns
// 64*(w/4).. of its rows (columns 0..H-1 from h, H..2H-1 from a); the next
// tile's slice is loaded into registers while GEMM1 runs and stored once
// GEMM1, the last reader of X, is complete.
__host__ __device__ __forceinline__ uint32_t carve_node_fwd(const MlpImgs& w, Smem* s, uint8_t* base) {
  uint32_t o = 0;
  auto at = [&](uint32_t bytes) {
    uint8_t* p = base ? base + o : nullptr;
    o += align1k(bytes);
    return p;
  };
  Smem m{};
  m.w1h = at(w.w1_bytes);
  m.w1l = at(w.w1_bytes);
  m.w2h = at(w.w2_bytes);
  m.w2l = at(w.w2_bytes);
  m.cst = reinterpret_cast<float*>(at(4u * kH * 4u));
  m.red = reinterpret_cast<float*>(at(4u * 4u * kH * 4u));
  if (s) *s = m;
  return o;
}

__global__ void __launch_bounds__(kThreads, 1) node_fwd_kernel(FwdArgs a) {
  constexpr uint32_t tZ1 = 0, tZ2 = kH, tX = 2 * kH, tA = 3 * kH;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ uint64_t wbar, mbar;
  __shared__ uint32_t tbase;
  Smem sm;
  carve_node_fwd(a.w, &sm, base);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int sp = warp & 3, cq = warp >> 2;
  const int r = sp * 32 + lane;
  const int c0 = cq * 32;
  bool ok = setup<M_NODE>(&wbar, &mbar, &tbase, 512, a.w, a.p, kH, sm, a.err);
  const uint32_t tm = tbase;
  const uint32_t lane_base = uint32_t(sp * 32) << 16;
  const int64_t tiles = (a.rows + 127) / 128;
  const float* b1 = sm.cst;
  const float* b2 = sm.cst + kH;
  const float* gam = sm.cst + 2 * kH;
  const float* bet = sm.cst + 3 * kH;
  const uint32_t id = idesc_bf16(128, kH, false, false);
  const bf16* xsrc = cq < 2 ? a.a0 + 64 * cq : a.a1 + 64 * (cq - 2);
  uint32_t xa[16], xb[16];  // 64 operand values of row r (packed pairs)
  auto load_x = [&](int64_t t) {
    const int64_t row = t * 128 + r;
    if (t < tiles && row < a.rows) {
      ld_raw16(xa, xsrc + row * kH);
      ld_raw16(xb, xsrc + row * kH + 32);
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j) xa[j] = xb[j] = 0u;
    }
  };
  auto store_x = [&]() {
    tmem_st16(tm + lane_base + tX + 32 * cq, xa);
    tmem_st16(tm + lane_base + tX + 32 * cq + 16, xb);
  };
  if (ok && blockIdx.x < tiles) {
    load_x(blockIdx.x);
    store_x();
  }
  uint32_t ph = 0;
  for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    tc_fence_before();
    if (__syncthreads_or(!ok)) break;
    const int64_t r0 = t * 128;
    // ---- GEMM1: Z1 = X (W1_hi + W1_lo), X from TMEM
    if (tid == 0) {
      tc_fence_after();
      const uint32_t wh = smem_u32(sm.w1h), wl = smem_u32(sm.w1l);
#pragma unroll 1
      for (int kk = 0; kk < 2 * kH / 16; ++kk) mma_bf16_ts(tm + tZ1, tm + tX + 8 * kk, kmajor_desc(wh, kH, kk), id, kk > 0);
#pragma unroll 1
      for (int kk = 0; kk < 2 * kH / 16; ++kk) mma_bf16_ts(tm + tZ1, tm + tX + 8 * kk, kmajor_desc(wl, kH, kk), id, 1u);
      mma_commit(&mbar);
    }
    const int64_t row = r0 + r;
    const bool valid = row < a.rows;
    // towards L2: this tile's residual row slice (read in epi2) and the operand slice two tiles ahead
    if (valid) prefetch_l2(a.r32 + row * kH + c0);
    {
      const int64_t t2 = t + 2 * int64_t(gridDim.x), row2 = t2 * 128 + r;
      if (t2 < tiles && row2 < a.rows) prefetch_l2(xsrc + row2 * kH);
    }
    load_x(t + gridDim.x);  // the next tile's operand slice, while GEMM1 runs
    ok = mbar_wait(&mbar, ph, a.err);
    ph ^= 1;
    if (__syncthreads_or(!ok)) break;
    tc_fence_after();
    store_x();  // GEMM1 is complete: X takes the next tile
    // ---- epi1: A1 = SiLU(Z1 + b1), packed bf16, into TMEM
    {
      float v[32];
      uint32_t ap[16];
      tmem_ld32(tm + lane_base + tZ1 + c0, v);
#pragma unroll
      for (int j = 0; j < 16; ++j)
        ap[j] = pack_bf16(silu_f(v[2 * j] + cst(b1 + c0, 2 * j)), silu_f(v[2 * j + 1] + cst(b1 + c0, 2 * j + 1)));
      tmem_st16(tm + lane_base + tA + 16 * cq, ap);
    }
    tc_fence_before();
    __syncthreads();
    // ---- GEMM2: Z2 = A1 (W2_hi + W2_lo), A1 from TMEM
    if (tid == 0) {
      tc_fence_after();
      const uint32_t wh = smem_u32(sm.w2h), wl = smem_u32(sm.w2l);
#pragma unroll 1
      for (int kk = 0; kk < kH / 16; ++kk) mma_bf16_ts(tm + tZ2, tm + tA + 8 * kk, kmajor_desc(wh, kH, kk), id, kk > 0);
#pragma unroll 1
      for (int kk = 0; kk < kH / 16; ++kk) mma_bf16_ts(tm + tZ2, tm + tA + 8 * kk, kmajor_desc(wl, kH, kk), id, 1u);
      mma_commit(&mbar);
    }
    float v[32], g0[32];
    if (valid) ld_g32(g0, a.r32 + row * kH + c0);  // the residual h_i
    ok = mbar_wait(&mbar, ph, a.err);
    ph ^= 1;
    if (__syncthreads_or(!ok)) break;
    tc_fence_after();
    // ---- epi2: h_i + LayerNorm(Z2 + b2), fp32 and bf16
    tmem_ld32(tm + lane_base + tZ2 + c0, v);
    float sum = 0.f;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      v[j] += cst(b2 + c0, j);
      sum += v[j];
    }
    const float mu = row_total(sm.red, 0, cq, r, sum) * (1.f / kH);
    float q = 0.f;
#pragma unroll
    for (int j = 0; j < 32; ++j) q += (v[j] - mu) * (v[j] - mu);
    const float rstd = rsqrtf(row_total(sm.red, 1, cq, r, q) * (1.f / kH) + kLnEps);
    if (valid) {
#pragma unroll
      for (int j = 0; j < 32; ++j) v[j] = g0[j] + ((v[j] - mu) * rstd * cst(gam + c0, j) + cst(bet + c0, j));
      st_g32(a.o32 + row * kH + c0, v);
      st_g16(a.o16 + row * kH + c0, v);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tm, 512);
}

// ============================================================ backward
template <int MODE>
__global__ void __launch_bounds__(kThreads, 1) mlp_bwd_kernel(BwdArgs a) {
  static_assert(MODE != M_EDGE, "the edge update has its own backward kernel (edge_bwd_kernel)");
  using S = Shape<MODE>;
  constexpr bool TMW = S::TMW;
  constexpr bool HAS_DX = MODE == M_NODE || MODE == M_DEC;
  constexpr bool LN = MODE != M_DEC;
  constexpr int NX = MODE == M_NODE ? 2 * kH : kH;
  constexpr uint32_t tZ1 = 0, tZ2 = kH, tDX = 0, tW1 = 256, tW2 = 384;
  constexpr uint32_t tRes = 256;  // NODE: the incoming gradient of the tile (no TMEM weight gradients there)
  static_assert(MODE != M_NODE || !TMW, "the residual columns are the weight-gradient columns");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ uint64_t wbar, mbar;
  __shared__ uint32_t tbase;
  Smem sm;
  carve_bytes<MODE>(a.w, true, &sm, base);
  uint8_t* const xa = sm.buf[0];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int sp = warp & 3, cq = warp >> 2;
  const int r = sp * 32 + lane;
  const int c0 = cq * 32;
  bool ok = setup<MODE>(&wbar, &mbar, &tbase, 512, a.w, a.p, MODE == M_DEC ? a.out_w : kH, sm, a.err);
  const uint32_t tm = tbase;
  const uint32_t lane_base = uint32_t(sp * 32) << 16;
  const int64_t tiles = (a.rows + 127) / 128;
  const float* b1 = sm.cst;
  const float* b2 = sm.cst + kH;
  const float* gam = sm.cst + 2 * kH;
  float cacc[4] = {0.f, 0.f, 0.f, 0.f};  // this lane's column 32*cq + lane: db1, db2, dgamma, dbeta
  uint32_t ph = 0;
  bool first = true;
  for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    if (__syncthreads_or(!ok)) break;
    const int64_t r0 = t * 128;
    if (MODE == M_NODE && a.dY1 && r0 + r < a.rows)  // this tile's incoming gradient slice towards L2
      prefetch_l2(a.dY1 + (r0 + r) * kH + c0);
    if (MODE == M_EENC) {  // this tile's gradient rows and the next tile's staged inputs towards L2
      if (a.dY1h && r0 + r < a.rows && (cq & 1) == 0) prefetch_l2(a.dY1h + (r0 + r) * kH + c0);
      const int64_t rn = (t + gridDim.x) * 128 + 8 * tid;
      if (a.feat8 && tid < 16 && rn < a.rows) prefetch_l2(a.feat8 + rn * 8);
    }
    if (S::ASYNC_A) {
      if (first) {
        issue_a_tile<MODE>(xa, a, r0, tid);
        cp_async_commit();
      }
      cp_async_wait<0>();  // this tile (issued here or prefetched during the previous one)
    } else {
      build_feature_tile<MODE>(xa, a, r0, tid, MODE == M_NENC ? a.X16g : nullptr);
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    // ---- GEMM1
    if (tid == 0) {
      tc_fence_after();
      fwd_gemm<MODE>(tm + tZ1, smem_u32(xa), kH, smem_u32(sm.w1h), S::SPLIT ? smem_u32(sm.w1l) : 0u, S::K1S, kH);
      mma_commit(&mbar);
    }
    const int64_t row = r0 + r;
    const bool valid = row < a.rows;
    float v[32], g0[32], g1[32];
    ok = mbar_wait(&mbar, ph, a.err);
    ph ^= 1;
    if (__syncthreads_or(!ok)) break;
    tc_fence_after();
    if (S::ASYNC_A && !TMW && t + gridDim.x < tiles) {  // GEMM1 consumed the operand tile: prefetch the next
      issue_a_tile<MODE>(xa, a, (t + gridDim.x) * 128, tid);
      cp_async_commit();
    }
    // ---- epi1: full pre-activation back to TMEM, SiLU to smem
    tmem_ld32(tm + lane_base + tZ1 + c0, v);
#pragma unroll
    for (int j = 0; j < 32; ++j) {  // A1 = SiLU(Z1); SiLU'(Z1) = s + A1 (1 - s) back to TMEM
      const float z = v[j] + cst(b1 + c0, j);
      const float sg = __fdividef(1.f, 1.f + __expf(-z));
      v[j] = z * sg;
      g1[j] = sg + v[j] * (1.f - sg);
    }
    tmem_st32(tm + lane_base + tZ1 + c0, g1);
    st_tile32(sm.a1, 128, r, c0, v);
    if (!TMW && valid) st_g16(a.A1g + row * kH + c0, v);
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    // ---- GEMM2 (not needed without LayerNorm)
    if (LN) {
      if (tid == 0) {
        tc_fence_after();
        fwd_gemm<MODE>(tm + tZ2, smem_u32(sm.a1), kH, smem_u32(sm.w2h), S::SPLIT ? smem_u32(sm.w2l) : 0u, kH / 16,
                       kH);
        mma_commit(&mbar);
      }
      // incoming gradient of this slice while the MMA runs
#pragma unroll
      for (int j = 0; j < 32; ++j) g0[j] = 0.f;
      if (valid) {
        const int64_t r2 = a.idx2 ? int64_t(a.idx2[row]) : row;
        if (a.dY1) add_g32(g0, a.dY1 + row * kH + c0);
        if (a.dY1h) add_g16(g0, a.dY1h + row * kH + c0);
        if (a.dY2) add_g32(g0, a.dY2 + r2 * kH + c0);
        if (a.dY2h) add_g16(g0, a.dY2h + r2 * kH + c0);
      }
      // the node update's residual passes the same gradient on: it waits in
      // TMEM columns the node MLP leaves free (no weight gradients there)
      if (MODE == M_NODE) tmem_st32(tm + lane_base + tRes + c0, g0);
      ok = mbar_wait(&mbar, ph, a.err);
      ph ^= 1;
      if (__syncthreads_or(!ok)) break;
      tc_fence_after();
    }
    // ---- epi2: LayerNorm backward -> dZ2
    if (!LN) {
      if (cq < 2) {
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = (cq == 0 && valid && j < a.out_w) ? a.dY1[row * a.out_w + j] : 0.f;
        st_tile32(sm.dz2, 128, r, c0, v);
        if (valid) st_g16(a.dZ2g + row * 64 + c0, v);
        const float cs = col_reduce32(v);
        if (cq == 0) cacc[1] += cs;
      }
    } else {
      tmem_ld32(tm + lane_base + tZ2 + c0, v);
      float s = 0.f;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        v[j] += cst(b2 + c0, j);
        s += v[j];
      }
      const float mu = row_total(sm.red, 0, cq, r, s) * (1.f / kH);
      float q = 0.f;
#pragma unroll
      for (int j = 0; j < 32; ++j) q += (v[j] - mu) * (v[j] - mu);
      const float rstd = rsqrtf(row_total(sm.red, 1, cq, r, q) * (1.f / kH) + kLnEps);
      float sg = 0.f, sgx = 0.f;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        v[j] = (v[j] - mu) * rstd;  // x_hat
        const float gg = g0[j] * cst(gam + c0, j);
        sg += gg;
        sgx += gg * v[j];
        g1[j] = g0[j] * v[j];
      }
      const float2 mm = row_total2(sm.red, 2, 3, cq, r, sg, sgx);
      const float mg = mm.x * (1.f / kH), mgx = mm.y * (1.f / kH);
      cacc[2] += col_reduce32(g1);  // dgamma
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        g1[j] = rstd * (g0[j] * cst(gam + c0, j) - mg - v[j] * mgx);  // dZ2
      }
      cacc[3] += col_reduce32(g0);  // dbeta
      st_tile32(sm.dz2, 128, r, c0, g1);
      if (!TMW && valid) st_g16(a.dZ2g + row * kH + c0, g1);
      cacc[1] += col_reduce32(g1);  // db2
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    // ---- GEMM3: dA1 = dZ2 W2^T  [+ dW2 += A1^T dZ2]
    if (tid == 0) {
      tc_fence_after();
      const uint32_t ds = smem_u32(sm.dz2), ws = smem_u32(sm.w2h), as = smem_u32(sm.a1);
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
    // ---- epi3: dZ1 = dA1 * SiLU'(Z1); with TMEM weight gradients the
    //      operand tile is restored into xa (it held dZ2) for X^T dZ1
    if (TMW) {
      if (S::ASYNC_A) {
        issue_a_tile<MODE>(xa, a, r0, tid);
        cp_async_commit();
      } else {
        build_feature_tile<MODE>(xa, a, r0, tid, nullptr);
      }
    }
    {
      float z[32];
      tmem_ld32(tm + lane_base + tZ2 + c0, v);
      tmem_ld32(tm + lane_base + tZ1 + c0, z);
#pragma unroll
      for (int j = 0; j < 32; ++j) v[j] = valid ? v[j] * z[j] : 0.f;  // z holds SiLU'(Z1)
      st_tile32(sm.a1, 128, r, c0, v);
      cacc[0] += col_reduce32(v);
    }
    if (TMW && S::ASYNC_A) cp_async_wait<0>();
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    // ---- GEMM4: dX = dZ1 W1^T  [+ dW1 += X^T dZ1]
    if ((HAS_DX || TMW) && tid == 0) {
      tc_fence_after();
      const uint32_t ds = smem_u32(sm.a1), ws = smem_u32(sm.w1h), xs = smem_u32(xa);
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
    // dZ1 leaves through its smem tile, row-contiguously (GEMM4 reads the same
    // tile); the edge encoder's weight gradients stay in TMEM and nothing reads its dZ1
    if (a.dZ1g) copy_tile_out(sm.a1, a.dZ1g, r0, a.rows, tid);
    if (HAS_DX || TMW) {
      // residual pass-through of this slice (the node update's incoming gradient, kept in TMEM)
      if (MODE == M_NODE) tmem_ld32(tm + lane_base + tRes + c0, g0);
      ok = mbar_wait(&mbar, ph, a.err);
      ph ^= 1;
      if (__syncthreads_or(!ok)) break;
      tc_fence_after();
    }
    // with TMEM weight gradients the operand tile is consumed only now
    if (S::ASYNC_A && TMW && t + gridDim.x < tiles) {
      issue_a_tile<MODE>(xa, a, (t + gridDim.x) * 128, tid);
      cp_async_commit();
    }
    // ---- epi4: input gradients
    if (HAS_DX) {
      tmem_ld32(tm + lane_base + tDX + c0, v);
      if (valid) {
        if (MODE != M_DEC) {
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] += g0[j];
        }
        if (a.dX0h) st_g16(a.dX0h + row * kH + c0, v);
        else st_g32(a.dX0 + row * kH + c0, v);
      }
      if (MODE == M_NODE) {
        tmem_ld32(tm + lane_base + tDX + kH + c0, v);
        if (valid) st_g16(a.dX1h + row * kH + c0, v);
      }
    }
    first = false;
    tc_fence_before();
  }
  cp_async_wait<0>();
  // ---- partial outputs of this CTA
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (TMW) {
#pragma unroll 1
    for (int m = 0; m < 2; ++m) {
      float w[32];
      tmem_ld32(tm + lane_base + (m == 0 ? tW1 : tW2) + c0, w);
      if (first || !ok) {
#pragma unroll
        for (int j = 0; j < 32; ++j) w[j] = 0.f;
      }
      st_g32(a.wpart + ((int64_t(blockIdx.x) * 2 + m) * 128 + r) * kH + c0, w);
    }
  }
  float* red = sm.red;  // [sp][q][kH]
#pragma unroll
  for (int q = 0; q < 4; ++q) red[(sp * 4 + q) * kH + c0 + lane] = cacc[q];
  __syncthreads();
  if (tid < kH) {
    for (int q = 0; q < 4; ++q) {
      const float s = (red[(0 * 4 + q) * kH + tid] + red[(1 * 4 + q) * kH + tid]) +
                      (red[(2 * 4 + q) * kH + tid] + red[(3 * 4 + q) * kH + tid]);
      a.cpart[(int64_t(blockIdx.x) * 4 + q) * kH + tid] = s;
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tm, 512);
}

// ============================================================ edge backward
// Shared-memory plan of the edge backward kernel: W1_e and W2 (bf16, the
// recompute uses W_hi only), the edge-state tile e (GEMM1 operand and the X
// of dW1 = e^T dZ1, kept for the whole tile), A1 (then dZ1), dZ2, and the
// incoming edge-state gradient tile de, which is read once, coalesced, and
// overwritten in place by the outgoing gradient before it is copied out.
struct EdgeBwdSmem {
  uint8_t *w1, *w2, *xe, *a1, *dz2, *de;
  float* cst;
  float* red;
};

__host__ __device__ __forceinline__ uint32_t carve_edge_bwd(const MlpImgs& w, EdgeBwdSmem* s, uint8_t* base) {
  uint32_t o = 0;
  auto at = [&](uint32_t bytes) {
    uint8_t* p = base ? base + o : nullptr;
    o += align1k(bytes);
    return p;
  };
  EdgeBwdSmem m;
  m.w1 = at(w.w1_bytes);
  m.w2 = at(w.w2_bytes);
  m.xe = at(128u * kH * 2u);
  m.a1 = at(128u * kH * 2u);
  m.dz2 = at(128u * kH * 2u);
  m.de = at(128u * kH * 2u);
  m.cst = reinterpret_cast<float*>(at(4u * kH * 4u));
  m.red = reinterpret_cast<float*>(at(4u * 4u * kH * 4u));
  if (s) *s = m;
  return o;
}

// cp.async of rows r0..r0+127 of a row-major [rows, 128] bf16 array into a
// swizzled tile (rows past the end, or a null source, read as zeros).
__device__ __forceinline__ void issue_rows16(uint8_t* tile, const bf16* src, int64_t rows, int64_t r0, int tid) {
  for (int q = tid; q < 128 * 16; q += kThreads) {
    const int r = q >> 4, j = q & 15;
    if (!src) {  // no source: plain zero stores, no copy is issued
      *reinterpret_cast<uint4*>(tile + sw_chunk(128, r, j)) = make_uint4(0u, 0u, 0u, 0u);
      continue;
    }
    const bool ok = r0 + r < rows;
    cp_async16(tile + sw_chunk(128, r, j), ok ? src + (r0 + r) * kH + 8 * j : src, ok ? 16u : 0u);
  }
}

// cp.async of the node-projection rows P[idx[k]] (the 128 columns from `off`
// on) of one 128-edge tile into a swizzled tile; idx[k] < 0 reads zeros.
__device__ __forceinline__ void issue_gather16(uint8_t* tile, const bf16* P, const int32_t* idx, int off, int tid) {
  for (int q = tid; q < 128 * 16; q += kThreads) {
    const int r = q >> 4, j = q & 15;
    const int32_t n = idx[r];
    cp_async16(tile + sw_chunk(128, r, j), n >= 0 ? P + int64_t(n) * 2 * kH + off + 8 * j : P, n >= 0 ? 16u : 0u);
  }
}

// Tensor maps of the edge backward's row arrays ([rows, 128] bf16, boxes of
// 64 columns x 128 rows in the 128-byte swizzle of the operand tiles): the
// edge states e, the incoming edge-state gradient de, and the two outputs dZ1
// and de_out.
struct EdgeBwdMaps {
  CUtensorMap e, de, dz1, deo;
};

// Backward of the edge update (eq. 1 + residual) with recompute, per 128-edge
// tile:  Z1 = e W1_e + P_r[i] + P_s[j] + b1, A1 = SiLU(Z1), Z2 = A1 W2 + b2
// (GEMM1, GEMM2), dm = de + da[i] (the message feeds e' = e + m and a_i),
// dZ2 = LN backward (dm), dA1 = dZ2 W2^T and dW2 += A1^T dZ2 (GEMM3),
// dZ1 = dA1 SiLU'(Z1), de_out = de + dZ1 W1_e^T and dW1_e += e^T dZ1 (GEMM4).
// Tiles move by TMA (thread 32 issues every tensor copy): the edge-state and
// incoming-gradient tiles arrive straight in their swizzled layout, dZ1 (for
// the node-level receiver/sender sums) and de_out leave from their tiles.
// The gathered node projections of the next tile are staged with cp.async
// while the current tile finishes: P_r rows into the dZ2 tile once GEMM3 has
// consumed it, P_s rows into the A1/dZ1 tile once GEMM4 and the dZ1 store
// have read it.  The next edge-state tile follows GEMM4, the next gradient
// tile the store of de_out.
__global__ void __launch_bounds__(kThreads, 1) edge_bwd_kernel(BwdArgs a, const __grid_constant__ EdgeBwdMaps mp) {
  constexpr uint32_t tZ1 = 0, tZ2 = kH, tDX = 0, tW1 = 256, tW2 = 384;
  constexpr uint32_t kTileBytes = 128u * kH * 2u;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ uint64_t wbar, mbar, ebar, dbar;
  __shared__ uint32_t tbase;
  __shared__ int32_t nidx[2][128];  // receiver and sender of each row of the next tile (-1: none)
  EdgeBwdSmem sm;
  carve_edge_bwd(a.w, &sm, base);
  Smem ss{};
  ss.w1h = sm.w1;
  ss.w2h = sm.w2;
  ss.cst = sm.cst;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int sp = warp & 3, cq = warp >> 2;
  const int r = sp * 32 + lane;
  const int c0 = cq * 32;
  const bool tma_thread = tid == 32;
  const bool has_de = a.dY1h != nullptr;  // the top layer has no incoming edge-state gradient
  if (tid == 0) {
    mbar_init(&ebar, 1);  // setup() fences the initialisations
    mbar_init(&dbar, 1);
  }
  bool ok = setup<M_EDGE>(&wbar, &mbar, &tbase, 512, a.w, a.p, kH, ss, a.err);
  const uint32_t tm = tbase;
  const uint32_t lane_base = uint32_t(sp * 32) << 16;
  const int64_t tiles = (a.rows + 127) / 128;
  const float* b1 = sm.cst;
  const float* b2 = sm.cst + kH;
  const float* gam = sm.cst + 2 * kH;
  // this lane's column 32*cq + lane of db2 and dgamma (slots 1 and 2 of the partials; db1 and
  // dbeta, slots 0 and 3, are left zero: they follow from node-level sums of dZ1 and da)
  float cacc[4] = {0.f, 0.f, 0.f, 0.f};
  uint32_t ph = 0, eph = 0, dph = 0;
  bool first = true;
  const uint32_t id_f = idesc_bf16(128, kH, false, false);  // X W (W image K-major)
  const uint32_t id_t = idesc_bf16(128, kH, false, true);   // dY W^T (same image MN-major)
  const uint32_t id_w = idesc_bf16(128, kH, true, true);    // X^T dY
  // the next tile's receivers (threads 0..127) and senders (128..255)
  auto load_idx = [&](int64_t tn) {
    if (tid < 256) {
      const int k = tid & 127;
      const int64_t rr = tn * 128 + k;
      nidx[tid >> 7][k] = (tn < tiles && rr < a.rows) ? (tid < 128 ? a.recv[rr] : a.col[rr]) : -1;
    }
  };
  auto tma_rows = [&](uint8_t* tile, const CUtensorMap* map, int64_t r0, uint64_t* bar) {
    mbar_arrive_expect_tx(bar, kTileBytes);
    tma_load_2d(tile, map, 0, int(r0), bar);
    tma_load_2d(tile + kTileBytes / 2, map, 64, int(r0), bar);
  };
  const int64_t t0 = cta_tile(a.order, 0, tiles);
  if (t0 < tiles) {  // first tile: P_r, edge states, P_s, incoming gradients
    load_idx(t0);
    __syncthreads();
    issue_gather16(sm.dz2, a.P, nidx[0], 0, tid);
    cp_async_commit();
    if (tma_thread) {
      tma_rows(sm.xe, &mp.e, t0 * 128, &ebar);
      if (has_de) tma_rows(sm.de, &mp.de, t0 * 128, &dbar);
    }
    issue_gather16(sm.a1, a.P, nidx[1], kH, tid);
    cp_async_commit();
  }
  for (int64_t k = 0;; ++k) {
    const int64_t t = cta_tile(a.order, k, tiles);
    if (t >= tiles) break;
    if (__syncthreads_or(!ok)) break;
    const int64_t r0 = t * 128;
    const int64_t tn = cta_tile(a.order, k + 1, tiles);
    if (tma_thread && k > 0 && has_de) {  // the previous tile's de_out store has left the gradient tile
      bulk_wait_read0();
      tma_rows(sm.de, &mp.de, r0, &dbar);
    }
    // ---- GEMM1: Z1 = e W1_e (the edge-state tile arrives by TMA)
    if (tid == 0) {
      ok = mbar_wait(&ebar, eph, a.err);
      tc_fence_after();
      const uint32_t xs = smem_u32(sm.xe), ws = smem_u32(sm.w1);
      if (ok) {
#pragma unroll 1
        for (int kk = 0; kk < kH / 16; ++kk)
          mma_bf16(tm + tZ1, kmajor_desc(xs, 128, kk), kmajor_desc(ws, kH, kk), id_f, kk > 0);
      }
      mma_commit(&mbar);
    }
    eph ^= 1;
    const int64_t row = r0 + r;
    const bool valid = row < a.rows;
    float v[32], g0[32], g1[32];
    const int64_t rcv = valid ? int64_t(a.recv[row]) : 0;
    load_idx(tn);
    cp_async_wait<0>();  // P_r and P_s rows
    ok = mbar_wait(&mbar, ph, a.err) && ok;
    ph ^= 1;
    if (__syncthreads_or(!ok)) break;
    tc_fence_after();
    // ---- epi1: A1 = SiLU(Z1) to smem (over the staged P_s rows, element by element);
    //      SiLU'(Z1) = s + A1 (1 - s), s = sigmoid(Z1), back to TMEM
    ld_tile32(sm.dz2, 128, r, c0, g0);
    ld_tile32(sm.a1, 128, r, c0, g1);
    tmem_ld32(tm + lane_base + tZ1 + c0, v);
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const float z = v[j] + cst(b1 + c0, j) + g0[j] + g1[j];
      const float sg = __fdividef(1.f, 1.f + __expf(-z));
      v[j] = z * sg;
      g1[j] = sg + v[j] * (1.f - sg);
    }
    tmem_st32(tm + lane_base + tZ1 + c0, g1);
    st_tile32(sm.a1, 128, r, c0, v);
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    // ---- GEMM2: Z2 = A1 W2
    if (tid == 0) {
      tc_fence_after();
      const uint32_t as = smem_u32(sm.a1), ws = smem_u32(sm.w2);
#pragma unroll 1
      for (int kk = 0; kk < kH / 16; ++kk) mma_bf16(tm + tZ2, kmajor_desc(as, 128, kk), kmajor_desc(ws, kH, kk), id_f, kk > 0);
      mma_commit(&mbar);
    }
    // incoming gradient dm = de + da[receiver] while the MMA runs
#pragma unroll
    for (int j = 0; j < 32; ++j) g0[j] = 0.f;
    if (valid && a.dY2h) add_g16(g0, a.dY2h + rcv * kH + c0);
    bool dok = true;
    if (has_de) {
      dok = mbar_wait(&dbar, dph, a.err);  // the gradient tile
      dph ^= 1;
    }
    ok = mbar_wait(&mbar, ph, a.err) && dok;
    ph ^= 1;
    if (__syncthreads_or(!ok)) break;
    tc_fence_after();
    if (has_de) {
      float d[32];
      ld_tile32(sm.de, 128, r, c0, d);
#pragma unroll
      for (int j = 0; j < 32; ++j) g0[j] += d[j];
    }
    // ---- epi2: LayerNorm backward -> dZ2
    tmem_ld32(tm + lane_base + tZ2 + c0, v);
    {
      float s = 0.f;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        v[j] += cst(b2 + c0, j);
        s += v[j];
      }
      const float mu = row_total(sm.red, 0, cq, r, s) * (1.f / kH);
      float q = 0.f;
#pragma unroll
      for (int j = 0; j < 32; ++j) q += (v[j] - mu) * (v[j] - mu);
      const float rstd = rsqrtf(row_total(sm.red, 1, cq, r, q) * (1.f / kH) + kLnEps);
      float sg = 0.f, sgx = 0.f;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        v[j] = (v[j] - mu) * rstd;  // x_hat
        const float gg = g0[j] * cst(gam + c0, j);
        sg += gg;
        sgx += gg * v[j];
        g1[j] = g0[j] * v[j];
      }
      const float2 mm = row_total2(sm.red, 2, 3, cq, r, sg, sgx);
      const float mg = mm.x * (1.f / kH), mgx = mm.y * (1.f / kH);
      cacc[2] += col_reduce32(g1);  // dgamma
#pragma unroll
      for (int j = 0; j < 32; ++j) g1[j] = rstd * (g0[j] * cst(gam + c0, j) - mg - v[j] * mgx);  // dZ2
      st_tile32(sm.dz2, 128, r, c0, g1);
      cacc[1] += col_reduce32(g1);  // db2
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    // ---- GEMM3: dA1 = dZ2 W2^T,  dW2 += A1^T dZ2
    if (tid == 0) {
      tc_fence_after();
      const uint32_t ds = smem_u32(sm.dz2), ws = smem_u32(sm.w2), as = smem_u32(sm.a1);
#pragma unroll 1
      for (int kk = 0; kk < kH / 16; ++kk)
        mma_bf16(tm + tZ2, kmajor_desc(ds, 128, kk), mnmajor_desc(ws, kH, kk), id_t, kk > 0);
#pragma unroll 1
      for (int kk = 0; kk < 8; ++kk)
        mma_bf16(tm + tW2, mnmajor_desc(as, 128, kk), mnmajor_desc(ds, 128, kk), id_w, (first && kk == 0) ? 0u : 1u);
      mma_commit(&mbar);
    }
    ok = mbar_wait(&mbar, ph, a.err);
    ph ^= 1;
    if (__syncthreads_or(!ok)) break;
    tc_fence_after();
    if (tn < tiles) {  // dZ2 is consumed: stage the next tile's P_r rows in its place
      issue_gather16(sm.dz2, a.P, nidx[0], 0, tid);
      cp_async_commit();
    }
    // the next tile's aggregated-message gradient rows, for its epi2, towards L2
    if (a.dY2h && nidx[0][r] >= 0) prefetch_l2(a.dY2h + int64_t(nidx[0][r]) * kH + c0);
    // ---- epi3: dZ1 = dA1 SiLU'(Z1) (A1 is consumed: dZ1 takes its tile)
    {
      float z[32];
      tmem_ld32(tm + lane_base + tZ2 + c0, v);
      tmem_ld32(tm + lane_base + tZ1 + c0, z);
#pragma unroll
      for (int j = 0; j < 32; ++j) v[j] = valid ? v[j] * z[j] : 0.f;  // z holds SiLU'(Z1)
      st_tile32(sm.a1, 128, r, c0, v);
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    // ---- GEMM4: dX = dZ1 W1_e^T,  dW1_e += e^T dZ1; dZ1 leaves by TMA meanwhile
    if (tid == 0) {
      tc_fence_after();
      const uint32_t ds = smem_u32(sm.a1), ws = smem_u32(sm.w1), xs = smem_u32(sm.xe);
#pragma unroll 1
      for (int kk = 0; kk < kH / 16; ++kk)
        mma_bf16(tm + tDX, kmajor_desc(ds, 128, kk), mnmajor_desc(ws, kH, kk), id_t, kk > 0);
#pragma unroll 1
      for (int kk = 0; kk < 8; ++kk)
        mma_bf16(tm + tW1, mnmajor_desc(xs, 128, kk), mnmajor_desc(ds, 128, kk), id_w, (first && kk == 0) ? 0u : 1u);
      mma_commit(&mbar);
    }
    if (tma_thread) {
      tma_store_2d(&mp.dz1, 0, int(r0), sm.a1);
      tma_store_2d(&mp.dz1, 64, int(r0), sm.a1 + kTileBytes / 2);
      bulk_commit();
    }
    ok = mbar_wait(&mbar, ph, a.err);
    ph ^= 1;
    if (tma_thread) {
      bulk_wait_read0();  // the dZ1 tile is read: P_s rows may replace it
      if (tn < tiles) tma_rows(sm.xe, &mp.e, tn * 128, &ebar);  // e is consumed by GEMM4
    }
    if (__syncthreads_or(!ok)) break;
    tc_fence_after();
    if (tn < tiles) {
      issue_gather16(sm.a1, a.P, nidx[1], kH, tid);
      cp_async_commit();
    }
    // ---- epi4: de_out = de + dX, out by TMA; then the next gradient tile
    {
      float d[32];
      tmem_ld32(tm + lane_base + tDX + c0, v);
      if (has_de) {
        ld_tile32(sm.de, 128, r, c0, d);
#pragma unroll
        for (int j = 0; j < 32; ++j) d[j] += v[j];
        st_tile32(sm.de, 128, r, c0, d);
      } else {
        st_tile32(sm.de, 128, r, c0, v);
      }
    }
    fence_proxy_async();
    __syncthreads();
    if (tma_thread) {  // the next gradient tile follows at the top of the next tile
      tma_store_2d(&mp.deo, 0, int(r0), sm.de);
      tma_store_2d(&mp.deo, 64, int(r0), sm.de + kTileBytes / 2);
      bulk_commit();
    }
    first = false;
    tc_fence_before();
  }
  cp_async_wait<0>();
  if (tma_thread) bulk_wait0();
  // ---- partial outputs of this CTA
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
#pragma unroll 1
  for (int m = 0; m < 2; ++m) {
    float w[32];
    tmem_ld32(tm + lane_base + (m == 0 ? tW1 : tW2) + c0, w);
    if (first || !ok) {
#pragma unroll
      for (int j = 0; j < 32; ++j) w[j] = 0.f;
    }
    st_g32(a.wpart + ((int64_t(blockIdx.x) * 2 + m) * 128 + r) * kH + c0, w);
  }
  float* red = sm.red;  // [sp][q][kH]
#pragma unroll
  for (int q = 0; q < 4; ++q) red[(sp * 4 + q) * kH + c0 + lane] = cacc[q];
  __syncthreads();
  if (tid < kH) {
    for (int q = 0; q < 4; ++q) {
      const float s = (red[(0 * 4 + q) * kH + tid] + red[(1 * 4 + q) * kH + tid]) +
                      (red[(2 * 4 + q) * kH + tid] + red[(3 * 4 + q) * kH + tid]);
      a.cpart[(int64_t(blockIdx.x) * 4 + q) * kH + tid] = s;
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tm, 512);
}

// ============================================================ edge backward, 32 warps
// The edge backward of edge_bwd_kernel (same phases, TMA tile movement,
// cp.async node-row staging and shared-memory plan) with twice the warps:
// 1024 threads, warp w reads TMEM lanes 32*(w%4).. and owns the 16 columns
// 16*(w/4).. of every accumulator, so each thread carries half the state of
// the 16-warp kernel and each scheduler has eight warps to switch between.
// Row statistics meet at named barriers of the eight warps of a lane
// quadrant.
constexpr int kT32 = 1024;

__device__ __forceinline__ void st_tile16(uint8_t* tile, uint32_t R, int r, int c, const float (&v)[16]) {
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    uint4 u;
    u.x = pack_bf16(v[8 * q + 0], v[8 * q + 1]);
    u.y = pack_bf16(v[8 * q + 2], v[8 * q + 3]);
    u.z = pack_bf16(v[8 * q + 4], v[8 * q + 5]);
    u.w = pack_bf16(v[8 * q + 6], v[8 * q + 7]);
    *reinterpret_cast<uint4*>(tile + sw_chunk(R, r, c / 8 + q)) = u;
  }
}
__device__ __forceinline__ void ld_tile16(const uint8_t* tile, uint32_t R, int r, int c, float (&v)[16]) {
#pragma unroll
  for (int q = 0; q < 2; ++q) unpack8(*reinterpret_cast<const uint4*>(tile + sw_chunk(R, r, c / 8 + q)), v + 8 * q);
}
// v += 16 bf16 values at src (32 bytes, one 256-bit load)
__device__ __forceinline__ void add_g16x16(float (&v)[16], const bf16* src) {
  uint32_t u[8];
  asm volatile("ld.global.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7])
               : "l"(src));
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u[i]));
    v[2 * i] += f.x;
    v[2 * i + 1] += f.y;
  }
}
__device__ __forceinline__ void tmem_st16f(uint32_t taddr, const float (&v)[16]) {
  uint32_t u[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) u[i] = __float_as_uint(v[i]);
  tmem_st16(taddr, u);
}
// Sum over the 32 lanes of each of the 16 values; lane l returns column l % 16.
__device__ __forceinline__ float col_reduce16(float (&v)[16]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], 16);
#pragma unroll
  for (int o = 8; o >= 1; o >>= 1) {
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
// Row totals over the eight 16-column slices of row r (fixed order), at the
// named barrier of the eight warps of r's lane quadrant.
__device__ __forceinline__ void octet_sync(int r) { asm volatile("bar.sync %0, 256;" ::"r"(1 + (r >> 5)) : "memory"); }
__device__ __forceinline__ float sum8(const float* p) {
  return ((p[0] + p[kH]) + (p[2 * kH] + p[3 * kH])) + ((p[4 * kH] + p[5 * kH]) + (p[6 * kH] + p[7 * kH]));
}
__device__ __forceinline__ float row_total8(float* red, int slot, int cq, int r, float part) {
  red[(slot * 8 + cq) * kH + r] = part;
  octet_sync(r);
  return sum8(red + slot * 8 * kH + r);
}
__device__ __forceinline__ float2 row_total8x2(float* red, int a, int b, int cq, int r, float pa, float pb) {
  red[(a * 8 + cq) * kH + r] = pa;
  red[(b * 8 + cq) * kH + r] = pb;
  octet_sync(r);
  return make_float2(sum8(red + a * 8 * kH + r), sum8(red + b * 8 * kH + r));
}
__device__ __forceinline__ void issue_gather16n(uint8_t* tile, const bf16* P, const int32_t* idx, int off, int tid) {
  for (int q = tid; q < 128 * 16; q += kT32) {
    const int r = q >> 4, j = q & 15;
    const int32_t n = idx[r];
    cp_async16(tile + sw_chunk(128, r, j), n >= 0 ? P + int64_t(n) * 2 * kH + off + 8 * j : P, n >= 0 ? 16u : 0u);
  }
}

__host__ __device__ __forceinline__ uint32_t carve_edge_bwd32(const MlpImgs& w, EdgeBwdSmem* s, uint8_t* base) {
  uint32_t o = 0;
  auto at = [&](uint32_t bytes) {
    uint8_t* p = base ? base + o : nullptr;
    o += align1k(bytes);
    return p;
  };
  EdgeBwdSmem m;
  m.w1 = at(w.w1_bytes);
  m.w2 = at(w.w2_bytes);
  m.xe = at(128u * kH * 2u);
  m.a1 = at(128u * kH * 2u);
  m.dz2 = at(128u * kH * 2u);
  m.de = at(128u * kH * 2u);
  m.cst = reinterpret_cast<float*>(at(4u * kH * 4u));
  m.red = reinterpret_cast<float*>(at(4u * 8u * kH * 4u));
  if (s) *s = m;
  return o;
}

__global__ void __launch_bounds__(kT32, 1) edge_bwd32_kernel(BwdArgs a, const __grid_constant__ EdgeBwdMaps mp) {
  constexpr uint32_t tZ1 = 0, tZ2 = kH, tDX = 0, tW1 = 256, tW2 = 384;
  constexpr uint32_t kTileBytes = 128u * kH * 2u;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ uint64_t wbar, mbar, ebar, dbar;
  __shared__ uint32_t tbase;
  __shared__ int32_t nidx[2][128];  // receiver and sender of each row of the next tile (-1: none)
  EdgeBwdSmem sm;
  carve_edge_bwd32(a.w, &sm, base);
  Smem ss{};
  ss.w1h = sm.w1;
  ss.w2h = sm.w2;
  ss.cst = sm.cst;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int sp = warp & 3, cq = warp >> 2;
  const int r = sp * 32 + lane;
  const int c0 = cq * 16;
  const bool tma_thread = tid == 32;
  const bool has_de = a.dY1h != nullptr;
  if (tid == 0) {
    mbar_init(&ebar, 1);  // setup() fences the initialisations
    mbar_init(&dbar, 1);
  }
  bool ok = setup<M_EDGE>(&wbar, &mbar, &tbase, 512, a.w, a.p, kH, ss, a.err);
  const uint32_t tm = tbase;
  const uint32_t lane_base = uint32_t(sp * 32) << 16;
  const int64_t tiles = (a.rows + 127) / 128;
  const float* b1 = sm.cst;
  const float* b2 = sm.cst + kH;
  const float* gam = sm.cst + 2 * kH;
  float cacc[2] = {0.f, 0.f};  // db2 and dgamma of column 16*cq + lane % 16
  uint32_t ph = 0, eph = 0, dph = 0;
  bool first = true;
  const uint32_t id_f = idesc_bf16(128, kH, false, false);
  const uint32_t id_t = idesc_bf16(128, kH, false, true);
  const uint32_t id_w = idesc_bf16(128, kH, true, true);
  auto load_idx = [&](int64_t tn) {
    if (tid < 256) {
      const int k = tid & 127;
      const int64_t rr = tn * 128 + k;
      nidx[tid >> 7][k] = (tn < tiles && rr < a.rows) ? (tid < 128 ? a.recv[rr] : a.col[rr]) : -1;
    }
  };
  auto tma_rows = [&](uint8_t* tile, const CUtensorMap* map, int64_t r0, uint64_t* bar) {
    mbar_arrive_expect_tx(bar, kTileBytes);
    tma_load_2d(tile, map, 0, int(r0), bar);
    tma_load_2d(tile + kTileBytes / 2, map, 64, int(r0), bar);
  };
  const int64_t t0 = cta_tile(a.order, 0, tiles);
  if (t0 < tiles) {
    load_idx(t0);
    __syncthreads();
    issue_gather16n(sm.dz2, a.P, nidx[0], 0, tid);
    cp_async_commit();
    if (tma_thread) {
      tma_rows(sm.xe, &mp.e, t0 * 128, &ebar);
      if (has_de) tma_rows(sm.de, &mp.de, t0 * 128, &dbar);
    }
    issue_gather16n(sm.a1, a.P, nidx[1], kH, tid);
    cp_async_commit();
  }
  for (int64_t k = 0;; ++k) {
    const int64_t t = cta_tile(a.order, k, tiles);
    if (t >= tiles) break;
    if (__syncthreads_or(!ok)) break;
    const int64_t r0 = t * 128;
    const int64_t tn = cta_tile(a.order, k + 1, tiles);
    if (tma_thread && k > 0 && has_de) {
      bulk_wait_read0();
      tma_rows(sm.de, &mp.de, r0, &dbar);
    }
    // ---- GEMM1: Z1 = e W1_e
    if (tid == 0) {
      ok = mbar_wait(&ebar, eph, a.err);
      tc_fence_after();
      const uint32_t xs = smem_u32(sm.xe), ws = smem_u32(sm.w1);
      if (ok) {
#pragma unroll 1
        for (int kk = 0; kk < kH / 16; ++kk)
          mma_bf16(tm + tZ1, kmajor_desc(xs, 128, kk), kmajor_desc(ws, kH, kk), id_f, kk > 0);
      }
      mma_commit(&mbar);
    }
    eph ^= 1;
    const int64_t row = r0 + r;
    const bool valid = row < a.rows;
    float v[16], g0[16], g1[16];
    const int64_t rcv = valid ? int64_t(a.recv[row]) : 0;
    load_idx(tn);
    cp_async_wait<0>();
    ok = mbar_wait(&mbar, ph, a.err) && ok;
    ph ^= 1;
    if (__syncthreads_or(!ok)) break;
    tc_fence_after();
    // ---- epi1
    ld_tile16(sm.dz2, 128, r, c0, g0);
    ld_tile16(sm.a1, 128, r, c0, g1);
    tmem_ld16(tm + lane_base + tZ1 + c0, v);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const float z = v[j] + cst(b1 + c0, j) + g0[j] + g1[j];
      const float sg = __fdividef(1.f, 1.f + __expf(-z));
      v[j] = z * sg;
      g1[j] = sg + v[j] * (1.f - sg);
    }
    tmem_st16f(tm + lane_base + tZ1 + c0, g1);
    st_tile16(sm.a1, 128, r, c0, v);
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    // ---- GEMM2: Z2 = A1 W2
    if (tid == 0) {
      tc_fence_after();
      const uint32_t as = smem_u32(sm.a1), ws = smem_u32(sm.w2);
#pragma unroll 1
      for (int kk = 0; kk < kH / 16; ++kk) mma_bf16(tm + tZ2, kmajor_desc(as, 128, kk), kmajor_desc(ws, kH, kk), id_f, kk > 0);
      mma_commit(&mbar);
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) g0[j] = 0.f;
    if (valid && a.dY2h) add_g16x16(g0, a.dY2h + rcv * kH + c0);
    bool dok = true;
    if (has_de) {
      dok = mbar_wait(&dbar, dph, a.err);
      dph ^= 1;
    }
    ok = mbar_wait(&mbar, ph, a.err) && dok;
    ph ^= 1;
    if (__syncthreads_or(!ok)) break;
    tc_fence_after();
    if (has_de) {
      float d[16];
      ld_tile16(sm.de, 128, r, c0, d);
#pragma unroll
      for (int j = 0; j < 16; ++j) g0[j] += d[j];
    }
    // ---- epi2: LayerNorm backward -> dZ2
    tmem_ld16(tm + lane_base + tZ2 + c0, v);
    {
      float s = 0.f;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        v[j] += cst(b2 + c0, j);
        s += v[j];
      }
      const float mu = row_total8(sm.red, 0, cq, r, s) * (1.f / kH);
      float q = 0.f;
#pragma unroll
      for (int j = 0; j < 16; ++j) q += (v[j] - mu) * (v[j] - mu);
      const float rstd = rsqrtf(row_total8(sm.red, 1, cq, r, q) * (1.f / kH) + kLnEps);
      float sg = 0.f, sgx = 0.f;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        v[j] = (v[j] - mu) * rstd;  // x_hat
        const float gg = g0[j] * cst(gam + c0, j);
        sg += gg;
        sgx += gg * v[j];
        g1[j] = g0[j] * v[j];
      }
      const float2 mm = row_total8x2(sm.red, 2, 3, cq, r, sg, sgx);
      const float mg = mm.x * (1.f / kH), mgx = mm.y * (1.f / kH);
      cacc[1] += col_reduce16(g1);  // dgamma
#pragma unroll
      for (int j = 0; j < 16; ++j) g1[j] = rstd * (g0[j] * cst(gam + c0, j) - mg - v[j] * mgx);  // dZ2
      st_tile16(sm.dz2, 128, r, c0, g1);
      cacc[0] += col_reduce16(g1);  // db2
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    // ---- GEMM3: dA1 = dZ2 W2^T,  dW2 += A1^T dZ2
    if (tid == 0) {
      tc_fence_after();
      const uint32_t ds = smem_u32(sm.dz2), ws = smem_u32(sm.w2), as = smem_u32(sm.a1);
#pragma unroll 1
      for (int kk = 0; kk < kH / 16; ++kk)
        mma_bf16(tm + tZ2, kmajor_desc(ds, 128, kk), mnmajor_desc(ws, kH, kk), id_t, kk > 0);
#pragma unroll 1
      for (int kk = 0; kk < 8; ++kk)
        mma_bf16(tm + tW2, mnmajor_desc(as, 128, kk), mnmajor_desc(ds, 128, kk), id_w, (first && kk == 0) ? 0u : 1u);
      mma_commit(&mbar);
    }
    ok = mbar_wait(&mbar, ph, a.err);
    ph ^= 1;
    if (__syncthreads_or(!ok)) break;
    tc_fence_after();
    if (tn < tiles) {
      issue_gather16n(sm.dz2, a.P, nidx[0], 0, tid);
      cp_async_commit();
    }
    if (a.dY2h && nidx[0][r] >= 0 && (cq & 3) == 0) prefetch_l2(a.dY2h + int64_t(nidx[0][r]) * kH + c0);  // c0 = 0, 64: both lines
    // ---- epi3: dZ1 = dA1 SiLU'(Z1)
    {
      float z[16];
      tmem_ld16(tm + lane_base + tZ2 + c0, v);
      tmem_ld16(tm + lane_base + tZ1 + c0, z);
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = valid ? v[j] * z[j] : 0.f;
      st_tile16(sm.a1, 128, r, c0, v);
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    // ---- GEMM4: dX = dZ1 W1_e^T,  dW1_e += e^T dZ1; dZ1 leaves by TMA meanwhile
    if (tid == 0) {
      tc_fence_after();
      const uint32_t ds = smem_u32(sm.a1), ws = smem_u32(sm.w1), xs = smem_u32(sm.xe);
#pragma unroll 1
      for (int kk = 0; kk < kH / 16; ++kk)
        mma_bf16(tm + tDX, kmajor_desc(ds, 128, kk), mnmajor_desc(ws, kH, kk), id_t, kk > 0);
#pragma unroll 1
      for (int kk = 0; kk < 8; ++kk)
        mma_bf16(tm + tW1, mnmajor_desc(xs, 128, kk), mnmajor_desc(ds, 128, kk), id_w, (first && kk == 0) ? 0u : 1u);
      mma_commit(&mbar);
    }
    if (tma_thread) {
      tma_store_2d(&mp.dz1, 0, int(r0), sm.a1);
      tma_store_2d(&mp.dz1, 64, int(r0), sm.a1 + kTileBytes / 2);
      bulk_commit();
    }
    ok = mbar_wait(&mbar, ph, a.err);
    ph ^= 1;
    if (tma_thread) {
      bulk_wait_read0();
      if (tn < tiles) tma_rows(sm.xe, &mp.e, tn * 128, &ebar);
    }
    if (__syncthreads_or(!ok)) break;
    tc_fence_after();
    if (tn < tiles) {
      issue_gather16n(sm.a1, a.P, nidx[1], kH, tid);
      cp_async_commit();
    }
    // ---- epi4: de_out = de + dX, out by TMA
    {
      float d[16];
      tmem_ld16(tm + lane_base + tDX + c0, v);
      if (has_de) {
        ld_tile16(sm.de, 128, r, c0, d);
#pragma unroll
        for (int j = 0; j < 16; ++j) d[j] += v[j];
        st_tile16(sm.de, 128, r, c0, d);
      } else {
        st_tile16(sm.de, 128, r, c0, v);
      }
    }
    fence_proxy_async();
    __syncthreads();
    if (tma_thread) {
      tma_store_2d(&mp.deo, 0, int(r0), sm.de);
      tma_store_2d(&mp.deo, 64, int(r0), sm.de + kTileBytes / 2);
      bulk_commit();
    }
    first = false;
    tc_fence_before();
  }
  cp_async_wait<0>();
  if (tma_thread) bulk_wait0();
  // ---- partial outputs of this CTA
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
#pragma unroll 1
  for (int m = 0; m < 2; ++m) {
    float w[16];
    tmem_ld16(tm + lane_base + (m == 0 ? tW1 : tW2) + c0, w);
    if (first || !ok) {
#pragma unroll
      for (int j = 0; j < 16; ++j) w[j] = 0.f;
    }
    float* dst = a.wpart + ((int64_t(blockIdx.x) * 2 + m) * 128 + r) * kH + c0;
#pragma unroll
    for (int j = 0; j < 16; j += 4) *reinterpret_cast<float4*>(dst + j) = make_float4(w[j], w[j + 1], w[j + 2], w[j + 3]);
  }
  float* red = sm.red;  // [sp][db2, dgamma][kH]
  if (lane < 16) {
    red[(sp * 2 + 0) * kH + c0 + lane] = cacc[0];
    red[(sp * 2 + 1) * kH + c0 + lane] = cacc[1];
  }
  __syncthreads();
  if (tid < kH) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const float s = (red[(0 * 2 + q) * kH + tid] + red[(1 * 2 + q) * kH + tid]) +
                      (red[(2 * 2 + q) * kH + tid] + red[(3 * 2 + q) * kH + tid]);
      a.cpart[(int64_t(blockIdx.x) * 4 + 1 + q) * kH + tid] = (first || !ok) ? 0.f : s;
    }
    a.cpart[(int64_t(blockIdx.x) * 4 + 0) * kH + tid] = 0.f;
    a.cpart[(int64_t(blockIdx.x) * 4 + 3) * kH + tid] = 0.f;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tm, 512);
}

// ============================================================ edge backward, two groups
// The same per-tile phases as edge_bwd_kernel, run by two independent groups
// of 8 warps that each keep one 128-edge tile in flight, so that one group's
// products, barriers and memory latencies overlap the other group's
// arithmetic.  What makes two tiles fit:
//  * TMEM: a group needs only one 128-column accumulator region, reused by
//    Z1, Z2, dA1 and dX in turn (each product starts after the epilogue that
//    reads the previous one), because SiLU'(Z1) -- needed again after GEMM3 --
//    leaves TMEM: it is written as fp16 to a per-(CTA, group) scratch slot of
//    32 KB (9.7 MB for the whole grid, so it stays in L2) and read back by the
//    same thread.  Columns: group 0 [0, 128), group 1 [128, 256), dW1_e
//    [256, 384), dW2 [384, 512), the weight gradients shared by both groups.
//  * Shared memory: per group two 128 x 128 bf16 tiles, T1 (edge states for
//    GEMM1, then dZ2, then the edge states again, reloaded -- from L2 in
//    practice -- for dW1 = e^T dZ1) and T2 (A1, then dZ1), next to the shared
//    W1_e and W2 images: 192 KB.
//  * Determinism: both groups accumulate into the same dW1 / dW2, so their
//    weight-gradient products are issued in CTA tile order: a group issues
//    its tile j's dW2 (dW1) products only after tile j-1's were issued (a
//    token in shared memory, passed with tcgen05 fences around the thread
//    synchronisation), whichever group that was.
// Group g takes the CTA's tiles j = g, g + 2, ...; warp w of group g reads TMEM
// lanes 32*(w%4).. and owns the 64 columns 64*((w/4)%2).. of every
// accumulator, in two 32-column chunks.
struct EdgeBwd2Smem {
  uint8_t *w1, *w2, *t1[2], *t2[2];
  float* cst;
  float* red;  // row statistics [g][slot 4][half 2][128]; at the end column partials [g][sp 4][2][128]
};

__host__ __device__ __forceinline__ uint32_t carve_edge_bwd2(const MlpImgs& w, EdgeBwd2Smem* s, uint8_t* base) {
  uint32_t o = 0;
  auto at = [&](uint32_t bytes) {
    uint8_t* p = base ? base + o : nullptr;
    o += align1k(bytes);
    return p;
  };
  EdgeBwd2Smem m;
  m.w1 = at(w.w1_bytes);
  m.w2 = at(w.w2_bytes);
  for (int g = 0; g < 2; ++g) {
    m.t1[g] = at(128u * kH * 2u);
    m.t2[g] = at(128u * kH * 2u);
  }
  m.cst = reinterpret_cast<float*>(at(4u * kH * 4u));
  m.red = reinterpret_cast<float*>(at(2u * 4u * 2u * 128u * 4u));
  if (s) *s = m;
  return o;
}

__device__ __forceinline__ uint32_t pack_f16(float a, float b) {
  __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}
__device__ __forceinline__ float f16_at(const uint32_t (&u)[16], int j) {
  const __half2 h = *reinterpret_cast<const __half2*>(&u[j >> 1]);
  return (j & 1) ? __high2float(h) : __low2float(h);
}

// Waits (bounded, about one second) until the token reaches `want`.
__device__ __forceinline__ bool token_wait(volatile int32_t* tok, int32_t want, uint32_t* err) {
  if (*tok == want) return true;
  const uint64_t t0 = globaltimer();
  while (*tok != want) {
    if (globaltimer() - t0 > 1000000000ull) {
      dev_flag(err, DEV_ERR_TIMEOUT);
      return false;
    }
    __nanosleep(64);
  }
  return true;
}

__global__ void __launch_bounds__(kThreads, 1) edge_bwd2_kernel(BwdArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ uint64_t wbar, mb[2];
  __shared__ uint32_t tbase;
  __shared__ int32_t tok[2];  // CTA tiles whose dW2 (0) / dW1_e (1) products have been issued
  __shared__ int32_t bad;     // a group gave up (error flagged): the partials are left zero
  EdgeBwd2Smem sm;
  carve_edge_bwd2(a.w, &sm, base);
  Smem ss{};
  ss.w1h = sm.w1;
  ss.w2h = sm.w2;
  ss.cst = sm.cst;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = warp >> 3, gt = tid & 255;
  const int sp = warp & 3, ch = (warp >> 2) & 1;
  const int r = sp * 32 + lane;
  if (tid == 0) {
    mbar_init(&mb[1], 1);  // setup() initialises mb[0] and fences both
    tok[0] = tok[1] = 0;
    bad = 0;
  }
  bool ok = setup<M_EDGE>(&wbar, &mb[0], &tbase, 512, a.w, a.p, kH, ss, a.err);
  const uint32_t R = tbase + 128u * g;  // this group's accumulator region
  const uint32_t tW1 = tbase + 256u, tW2 = tbase + 384u;
  const uint32_t lane_base = uint32_t(sp * 32) << 16;
  const int64_t tiles = (a.rows + 127) / 128;
  uint8_t* const T1 = sm.t1[g];
  uint8_t* const T2 = sm.t2[g];
  float* const red = sm.red + g * (4 * 2 * 128);
  uint32_t* const spill = a.spill + ((int64_t(blockIdx.x) * 2 + g) * 128 + r) * (kH / 2);
  const float* b1 = sm.cst;
  const float* b2 = sm.cst + kH;
  const float* gam = sm.cst + 2 * kH;
  const uint32_t id_f = idesc_bf16(128, kH, false, false);  // X W (W image K-major)
  const uint32_t id_t = idesc_bf16(128, kH, false, true);   // dY W^T (same image MN-major)
  const uint32_t id_w = idesc_bf16(128, kH, true, true);    // X^T dY
  const int cA = 64 * ch;
  float cacc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};  // [chunk][db2, dgamma] of column cA + 32 chunk + lane
  uint32_t ph = 0;
  bool gok = group_all(g, ok);
  auto load_e = [&](int64_t r0, int nrows) {
    for (int q = gt; q < 128 * 16; q += 256) {
      const int rr = q >> 4, jj = q & 15;
      const bool in = rr < nrows;
      cp_async16(T1 + sw_chunk(128, rr, jj), a.a0 + (in ? (r0 + rr) * kH + 8 * jj : 0), in ? 16u : 0u);
    }
    cp_async_commit();
  };
  for (int64_t k = 0; gok; ++k) {
    const int64_t j = 2 * k + g;  // the CTA's tiles alternate between its groups
    const int64_t t = cta_tile(a.order, j, tiles);
    if (t >= tiles) break;
    const int64_t r0 = t * 128;
    const int nrows = a.rows - r0 < 128 ? int(a.rows - r0) : 128;
    load_e(r0, nrows);
    const int64_t row = r0 + r;
    const bool valid = r < nrows;
    const int64_t rcv = valid ? int64_t(a.recv[row]) : 0, snd = valid ? int64_t(a.col[row]) : 0;
    cp_async_wait<0>();
    fence_proxy_async();
    tc_fence_before();
    group_sync(g);
    // ---- GEMM1: Z1 = e W1_e
    if (gt == 0) {
      tc_fence_after();
      const uint32_t xs = smem_u32(T1), ws = smem_u32(sm.w1);
#pragma unroll 1
      for (int kk = 0; kk < kH / 16; ++kk) mma_bf16(R, kmajor_desc(xs, 128, kk), kmajor_desc(ws, kH, kk), id_f, kk > 0);
      mma_commit(&mb[g]);
    }
    uint32_t pr[16], ps[16];  // 32 bf16 node projections each, packed
    if (valid) {
      ld_raw16(pr, a.P + rcv * 2 * kH + cA);
      ld_raw16(ps, a.P + snd * 2 * kH + kH + cA);
    } else {
#pragma unroll
      for (int q = 0; q < 16; ++q) pr[q] = ps[q] = 0u;
    }
    gok = group_all(g, mbar_wait(&mb[g], ph, a.err));
    ph ^= 1;
    if (!gok) break;
    tc_fence_after();
    // ---- epi1: A1 = SiLU(Z1 + b1 + P_r + P_s) to T2; SiLU'(Z1) = s + A1 (1 - s) to the spill slot
#pragma unroll 1
    for (int c = 0; c < 2; ++c) {
      const int cc = cA + 32 * c;
      float v[32], d[32];
      tmem_ld32(R + lane_base + cc, v);
      if (c == 1 && valid) {
        ld_raw16(pr, a.P + rcv * 2 * kH + cc);
        ld_raw16(ps, a.P + snd * 2 * kH + kH + cc);
      }
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const float z = v[q] + cst(b1 + cc, q) + bf16_at(pr, q) + bf16_at(ps, q);
        const float sg = __fdividef(1.f, 1.f + __expf(-z));
        v[q] = z * sg;
        d[q] = sg + v[q] * (1.f - sg);
      }
      st_tile32(T2, 128, r, cc, v);
      uint32_t h[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) h[q] = pack_f16(d[2 * q], d[2 * q + 1]);
      st8u(spill + cc / 2, h);
      st8u(spill + cc / 2 + 8, h + 8);
    }
    fence_proxy_async();
    tc_fence_before();
    group_sync(g);
    // ---- GEMM2: Z2 = A1 W2 (every Z1 value has been read)
    if (gt == 0) {
      tc_fence_after();
      const uint32_t as = smem_u32(T2), ws = smem_u32(sm.w2);
#pragma unroll 1
      for (int kk = 0; kk < kH / 16; ++kk) mma_bf16(R, kmajor_desc(as, 128, kk), kmajor_desc(ws, kH, kk), id_f, kk > 0);
      mma_commit(&mb[g]);
    }
    gok = group_all(g, mbar_wait(&mb[g], ph, a.err));
    ph ^= 1;
    if (!gok) break;
    tc_fence_after();
    // ---- epi2: LayerNorm backward of dm = de + da[receiver] -> dZ2 (into T1; GEMM1 has read e)
    float mu, rstd;
    {
      float s = 0.f;
#pragma unroll 1
      for (int c = 0; c < 2; ++c) {
        const int cc = cA + 32 * c;
        float v[32];
        tmem_ld32(R + lane_base + cc, v);
#pragma unroll
        for (int q = 0; q < 32; ++q) s += v[q] + cst(b2 + cc, q);
      }
      red[(0 * 2 + ch) * 128 + r] = s;
      group_sync(g);
      mu = (red[0 * 128 + r] + red[1 * 128 + r]) * (1.f / kH);
      float qs = 0.f;
#pragma unroll 1
      for (int c = 0; c < 2; ++c) {
        const int cc = cA + 32 * c;
        float v[32];
        tmem_ld32(R + lane_base + cc, v);
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          const float dd = v[q] + cst(b2 + cc, q) - mu;
          qs += dd * dd;
        }
      }
      red[(1 * 2 + ch) * 128 + r] = qs;
      group_sync(g);
      rstd = rsqrtf((red[2 * 128 + r] + red[3 * 128 + r]) * (1.f / kH) + kLnEps);
    }
    auto load_dm = [&](float (&d)[32], int cc) {
#pragma unroll
      for (int q = 0; q < 32; ++q) d[q] = 0.f;
      if (valid) {
        if (a.dY1h) add_g16(d, a.dY1h + row * kH + cc);
        if (a.dY2h) add_g16(d, a.dY2h + rcv * kH + cc);
      }
    };
    float sg = 0.f, sgx = 0.f;
#pragma unroll 1
    for (int c = 0; c < 2; ++c) {
      const int cc = cA + 32 * c;
      float v[32], d[32];
      load_dm(d, cc);
      tmem_ld32(R + lane_base + cc, v);
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const float xh = (v[q] + cst(b2 + cc, q) - mu) * rstd;
        const float gg = d[q] * cst(gam + cc, q);
        sg += gg;
        sgx += gg * xh;
        v[q] = d[q] * xh;
      }
      cacc[c][1] += col_reduce32(v);  // dgamma
    }
    red[(2 * 2 + ch) * 128 + r] = sg;
    red[(3 * 2 + ch) * 128 + r] = sgx;
    group_sync(g);
    const float mg = (red[4 * 128 + r] + red[5 * 128 + r]) * (1.f / kH);
    const float mgx = (red[6 * 128 + r] + red[7 * 128 + r]) * (1.f / kH);
#pragma unroll 1
    for (int c = 0; c < 2; ++c) {
      const int cc = cA + 32 * c;
      float v[32], d[32];
      load_dm(d, cc);
      tmem_ld32(R + lane_base + cc, v);
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const float xh = (v[q] + cst(b2 + cc, q) - mu) * rstd;
        v[q] = rstd * (d[q] * cst(gam + cc, q) - mg - xh * mgx);  // dZ2
      }
      st_tile32(T1, 128, r, cc, v);
      cacc[c][0] += col_reduce32(v);  // db2
    }
    fence_proxy_async();
    tc_fence_before();
    group_sync(g);
    // ---- GEMM3: dA1 = dZ2 W2^T (Z2 has been read);  dW2 += A1^T dZ2 in CTA tile order
    bool lok = true;
    if (gt == 0) {
      tc_fence_after();
      const uint32_t ds = smem_u32(T1), ws = smem_u32(sm.w2), as = smem_u32(T2);
#pragma unroll 1
      for (int kk = 0; kk < kH / 16; ++kk) mma_bf16(R, kmajor_desc(ds, 128, kk), mnmajor_desc(ws, kH, kk), id_t, kk > 0);
      lok = token_wait(&tok[0], int32_t(j), a.err);
      if (lok) {
        tc_fence_after();
#pragma unroll 1
        for (int kk = 0; kk < 8; ++kk)
          mma_bf16(tW2, mnmajor_desc(as, 128, kk), mnmajor_desc(ds, 128, kk), id_w, (j == 0 && kk == 0) ? 0u : 1u);
      }
      mma_commit(&mb[g]);
      if (lok) {
        tc_fence_before();
        __threadfence_block();
        *reinterpret_cast<volatile int32_t*>(&tok[0]) = int32_t(j + 1);
      }
    }
    gok = group_all(g, mbar_wait(&mb[g], ph, a.err) && lok);
    ph ^= 1;
    if (!gok) break;
    tc_fence_after();
    load_e(r0, nrows);  // dZ2 is consumed: the edge states again, for dW1 = e^T dZ1
    // ---- epi3: dZ1 = dA1 SiLU'(Z1) into T2 (A1 is consumed)
#pragma unroll 1
    for (int c = 0; c < 2; ++c) {
      const int cc = cA + 32 * c;
      float v[32];
      uint32_t h[16];
#pragma unroll
      for (int q = 0; q < 2; ++q)
        asm volatile("ld.global.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(h[8 * q]), "=r"(h[8 * q + 1]), "=r"(h[8 * q + 2]), "=r"(h[8 * q + 3]), "=r"(h[8 * q + 4]),
                       "=r"(h[8 * q + 5]), "=r"(h[8 * q + 6]), "=r"(h[8 * q + 7])
                     : "l"(spill + cc / 2 + 8 * q));
      tmem_ld32(R + lane_base + cc, v);
#pragma unroll
      for (int q = 0; q < 32; ++q) v[q] = valid ? v[q] * f16_at(h, q) : 0.f;
      st_tile32(T2, 128, r, cc, v);
    }
    cp_async_wait<0>();
    fence_proxy_async();
    tc_fence_before();
    group_sync(g);
    // ---- GEMM4: dX = dZ1 W1_e^T (dA1 has been read);  dW1_e += e^T dZ1 in CTA tile order
    if (gt == 0) {
      tc_fence_after();
      const uint32_t ds = smem_u32(T2), ws = smem_u32(sm.w1), xs = smem_u32(T1);
#pragma unroll 1
      for (int kk = 0; kk < kH / 16; ++kk) mma_bf16(R, kmajor_desc(ds, 128, kk), mnmajor_desc(ws, kH, kk), id_t, kk > 0);
      lok = token_wait(&tok[1], int32_t(j), a.err);
      if (lok) {
        tc_fence_after();
#pragma unroll 1
        for (int kk = 0; kk < 8; ++kk)
          mma_bf16(tW1, mnmajor_desc(xs, 128, kk), mnmajor_desc(ds, 128, kk), id_w, (j == 0 && kk == 0) ? 0u : 1u);
      }
      mma_commit(&mb[g]);
      if (lok) {
        tc_fence_before();
        __threadfence_block();
        *reinterpret_cast<volatile int32_t*>(&tok[1]) = int32_t(j + 1);
      }
    }
    // dZ1 to global memory for the node-level receiver / sender sums, while the products run
    copy_tile_out(T2, a.dZ1g, r0, a.rows, gt, 256);
    gok = group_all(g, mbar_wait(&mb[g], ph, a.err) && lok);
    ph ^= 1;
    if (!gok) break;
    tc_fence_after();
    // ---- epi4: de_out = de + dX (may overwrite de in place: each thread rereads its own slice first)
#pragma unroll 1
    for (int c = 0; c < 2; ++c) {
      const int cc = cA + 32 * c;
      float v[32];
      tmem_ld32(R + lane_base + cc, v);
      if (valid) {
        if (a.dY1h) add_g16(v, a.dY1h + row * kH + cc);
        st_g16(a.dX0h + row * kH + cc, v);
      }
    }
    tc_fence_before();
    group_sync(g);  // the accumulator region and both tiles are free for the next tile
  }
  if (!gok && gt == 0) bad = 1;
  cp_async_wait<0>();
  // ---- partial outputs of this CTA
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const bool none = bad != 0 || cta_tile(a.order, 0, tiles) >= tiles;
  {
    const int cq = warp >> 2;  // 16 warps: lane quadrant sp, column quarter cq
#pragma unroll 1
    for (int m = 0; m < 2; ++m) {
      float w[32];
      tmem_ld32(tbase + lane_base + (m == 0 ? 256u : 384u) + 32 * cq, w);
      if (none) {
#pragma unroll
        for (int q = 0; q < 32; ++q) w[q] = 0.f;
      }
      st_g32(a.wpart + ((int64_t(blockIdx.x) * 2 + m) * 128 + r) * kH + 32 * cq, w);
    }
  }
  // column partials: [g][sp][db2, dgamma][128], summed in fixed order
  float* cr = sm.red;
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    cr[((g * 4 + sp) * 2 + 0) * 128 + cA + 32 * c + lane] = cacc[c][0];
    cr[((g * 4 + sp) * 2 + 1) * 128 + cA + 32 * c + lane] = cacc[c][1];
  }
  __syncthreads();
  if (tid < kH) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      float s = 0.f;
#pragma unroll
      for (int gg = 0; gg < 2; ++gg)
        s += (cr[((gg * 4 + 0) * 2 + q) * 128 + tid] + cr[((gg * 4 + 1) * 2 + q) * 128 + tid]) +
             (cr[((gg * 4 + 2) * 2 + q) * 128 + tid] + cr[((gg * 4 + 3) * 2 + q) * 128 + tid]);
      a.cpart[(int64_t(blockIdx.x) * 4 + 1 + q) * kH + tid] = none ? 0.f : s;
    }
    a.cpart[(int64_t(blockIdx.x) * 4 + 0) * kH + tid] = 0.f;
    a.cpart[(int64_t(blockIdx.x) * 4 + 3) * kH + tid] = 0.f;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tbase, 512);
}

template <int MODE>
xmgn_status check_smem(uint32_t bytes) {
  int dev = 0, optin = 0;
  XMGN_CUDA(cudaGetDevice(&dev));
  XMGN_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (bytes + 64 > uint32_t(optin)) return fail(XMGN_ERR_UNSUPPORTED, "MLP kernel mode %d needs %u B smem", MODE, bytes);
  return XMGN_OK;
}

template <int MODE>
xmgn_status launch_fwd(const FwdArgs& a, cudaStream_t s) {
  if (!a.w.w1lo || !a.w.w2lo) return fail(XMGN_ERR_ARG, "missing low weight images");
  const int probe = MODE == M_EDGE ? PROBE_EDGE_FWD : (MODE == M_NODE ? PROBE_NODE_FWD : -1);
  static bool attr = false;
  if constexpr (MODE == M_EDGE) {
    if (!attr) {
      XMGN_TRY(allow_max_smem(edge_fwd_kernel));
      attr = true;
    }
    const uint32_t sm = carve_edge_fwd(a.w, nullptr, nullptr) + 1024u;
    XMGN_TRY(check_smem<MODE>(sm));
    FwdArgs b = a;
    b.order = tune_choice(TUNE_EDGE_FWD_ORDER, a.rows);
    CUtensorMap me;
    XMGN_TRY(rows_map(&me, a.a0, a.rows));
    probe_begin(probe, s);
    tune_begin(TUNE_EDGE_FWD_ORDER, s);
    edge_fwd_kernel<<<mlp_grid(a.rows), kThreads, sm, s>>>(b, me);
    tune_end(TUNE_EDGE_FWD_ORDER, s);
  } else if constexpr (MODE == M_NODE) {
    if (!attr) {
      XMGN_TRY(allow_max_smem(node_fwd_kernel));
      attr = true;
    }
    const uint32_t sm = carve_node_fwd(a.w, nullptr, nullptr) + 1024u;
    XMGN_TRY(check_smem<MODE>(sm));
    probe_begin(probe, s);
    node_fwd_kernel<<<mlp_grid(a.rows), kThreads, sm, s>>>(a);
  } else {
    if (!attr) {
      XMGN_TRY(allow_max_smem(mlp_fwd_kernel<MODE>));
      attr = true;
    }
    const uint32_t sm = smem_bytes<MODE>(a.w, false);
    XMGN_TRY(check_smem<MODE>(sm));
    probe_begin(probe, s);
    mlp_fwd_kernel<MODE><<<mlp_grid(a.rows), kThreads, sm, s>>>(a);
  }
  probe_end(probe, s);
  XMGN_LAUNCH_CHECK();
  return XMGN_OK;
}

template <int MODE>
xmgn_status launch_bwd(const BwdArgs& a, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    if constexpr (MODE == M_EDGE) {
      XMGN_TRY(allow_max_smem(edge_bwd_kernel));
      XMGN_TRY(allow_max_smem(edge_bwd2_kernel));
      XMGN_TRY(allow_max_smem(edge_bwd32_kernel));
    } else {
      XMGN_TRY(allow_max_smem(mlp_bwd_kernel<MODE>));
    }
    attr = true;
  }
  if (MODE != M_EDGE && Shape<MODE>::SPLIT && (!a.w.w1lo || !a.w.w2lo))
    return fail(XMGN_ERR_ARG, "missing low weight images");
  const int variant = MODE == M_EDGE ? tune_choice(TUNE_EDGE_BWD_TILES, a.rows) : 0;
  const bool tiles2 = variant == 1;  // two tiles in flight
  const bool warps32 = variant == 2; // one tile, 32 warps
  if (MODE == M_EDGE && tiles2 && !a.spill) return fail(XMGN_ERR_ARG, "edge backward: missing SiLU' scratch");
  const uint32_t sm = MODE != M_EDGE ? smem_bytes<MODE>(a.w, true)
                                     : (tiles2 ? carve_edge_bwd2(a.w, nullptr, nullptr)
                                               : warps32 ? carve_edge_bwd32(a.w, nullptr, nullptr)
                                                         : carve_edge_bwd(a.w, nullptr, nullptr)) + 1024u;
  XMGN_TRY(check_smem<MODE>(sm));
  const int probe = MODE == M_EDGE ? PROBE_EDGE_BWD : (MODE == M_NODE ? PROBE_NODE_BWD : -1);
  probe_begin(probe, s);
  if constexpr (MODE == M_EDGE) {
    BwdArgs b = a;
    b.order = tune_choice(TUNE_EDGE_BWD_ORDER, a.rows);
    tune_begin(TUNE_EDGE_BWD_ORDER, s);
    tune_begin(TUNE_EDGE_BWD_TILES, s);
    if (tiles2) {
      edge_bwd2_kernel<<<mlp_grid(a.rows), kThreads, sm, s>>>(b);
    } else {
      EdgeBwdMaps mp;
      XMGN_TRY(rows_map(&mp.e, a.a0, a.rows));
      XMGN_TRY(rows_map(&mp.de, a.dY1h ? a.dY1h : a.a0, a.rows));
      XMGN_TRY(rows_map(&mp.dz1, a.dZ1g, a.rows));
      XMGN_TRY(rows_map(&mp.deo, a.dX0h, a.rows));
      if (warps32)
        edge_bwd32_kernel<<<mlp_grid(a.rows), kT32, sm, s>>>(b, mp);
      else
        edge_bwd_kernel<<<mlp_grid(a.rows), kThreads, sm, s>>>(b, mp);
    }
    tune_end(TUNE_EDGE_BWD_TILES, s);
    tune_end(TUNE_EDGE_BWD_ORDER, s);
  } else {
    mlp_bwd_kernel<MODE><<<mlp_grid(a.rows), kThreads, sm, s>>>(a);
  }
  probe_end(probe, s);
  XMGN_LAUNCH_CHECK();
  return XMGN_OK;
}

}  // namespace

int mlp_grid(int64_t rows) { return tc_grid((rows + 127) / 128); }

int64_t edge_bwd_spill_words() { return int64_t(num_sms()) * 2 * 128 * (kH / 2); }

namespace {
__global__ void edge_inputs_bf16_kernel(const float* __restrict__ xyz, const int32_t* __restrict__ gid,
                                        const int32_t* __restrict__ recv, const int32_t* __restrict__ col, int64_t E,
                                        bf16* __restrict__ out) {
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < E; e += int64_t(gridDim.x) * blockDim.x) {
    int64_t i = recv[e], j = col[e];
    if (gid) {
      i = gid[i];
      j = gid[j];
    }
    const float dx = xyz[3 * j] - xyz[3 * i];
    const float dy = xyz[3 * j + 1] - xyz[3 * i + 1];
    const float dz = xyz[3 * j + 2] - xyz[3 * i + 2];
    uint4 u;
    u.x = pack_bf16(dx, dy);
    u.y = pack_bf16(dz, sqrtf(dx * dx + dy * dy + dz * dz));
    u.z = u.w = 0u;
    reinterpret_cast<uint4*>(out)[e] = u;
  }
}
}  // namespace

xmgn_status edge_inputs_bf16(const float* xyz, const int32_t* gid, const int32_t* recv, const int32_t* col,
                             int64_t E, bf16* out, cudaStream_t s) {
  if (E <= 0) return XMGN_OK;
  edge_inputs_bf16_kernel<<<grid_for(E, 256, int64_t(num_sms()) * 16), 256, 0, s>>>(xyz, gid, recv, col, E, out);
  XMGN_LAUNCH_CHECK();
  return XMGN_OK;
}

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
