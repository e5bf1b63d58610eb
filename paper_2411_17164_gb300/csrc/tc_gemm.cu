// Weight packing, row-tiled tensor-core GEMM and the reduction-over-rows
// tensor-core GEMM (see tc_gemm.cuh).
//
// Both GEMM kernels run 16 warps per CTA, one CTA per SM, persistent over
// 128-row tiles, and stage operand tiles with cp.async into two buffers so
// that the next tile loads while the current one multiplies.
#include "tc_gemm.cuh"
#include "tune.cuh"
#include "wgemm.cuh"

namespace xmgn {

using namespace tc;

namespace {

struct PackBatch {
  int n;
  PackJob j[kPackBatch];
};

// One image per blockIdx.y; element (r, c) of rows [r0, r0+nr) of the image.
__global__ void pack_kernel(PackBatch b) {
  const PackJob& J = b.j[blockIdx.y];
  const int64_t total = int64_t(J.nr) * J.C;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
       i += int64_t(gridDim.x) * blockDim.x) {
    const uint32_t rr = uint32_t(i / J.C), c = uint32_t(i % J.C);
    float v = 0.f;
    if (rr < J.nvalid && c < J.kvalid) v = J.W[(J.wk0 + c) * J.ld + J.wn0 + rr];
    const bf16 hi = __float2bfloat16_rn(v);
    *reinterpret_cast<bf16*>(J.dst + sw_off(J.R, J.r0 + rr, c)) =
        J.lo ? __float2bfloat16_rn(v - __bfloat162float(hi)) : hi;
  }
}

constexpr int kThreads = 512;

// Issues cp.async copies of rows [r0, r0+128) of a two-segment bf16 source
// into a swizzled 128-row tile (rows beyond M are zero-filled) and commits
// them as one group.
__device__ __forceinline__ void issue_rows(uint8_t* tile, const Bf16Rows& A, int64_t r0, int64_t M, int tid) {
  const int cpr = A.K() / 8;  // 16-byte chunks per row
  for (int q = tid; q < 128 * cpr; q += kThreads) {
    const int r = q / cpr, j = q % cpr;
    const int64_t row = r0 + r;
    const bool ok = row < M;
    const int col = j * 8;
    const bf16* src = col < A.w0 ? A.p0 + (ok ? row : 0) * A.ld0 + col
                                 : A.p1 + (ok ? row : 0) * A.ld1 + (col - A.w0);
    cp_async16(tile + sw_chunk(128, r, j), src, ok ? 16u : 0u);
  }
  cp_async_commit();
}

__device__ __forceinline__ void st8(float* p, const float* v) {
  asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(v[0]), "f"(v[1]), "f"(v[2]),
               "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
               : "memory");
}
__device__ __forceinline__ void ld8(const float* p, float* v) {
  asm volatile("ld.global.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
               : "l"(p));
}

struct GemmArgs {
  Bf16Rows A;
  int64_t M;
  const uint8_t* img;
  uint32_t img_bytes, R;
  int N, K;
  int b_mn;
  float* D;
  bf16* D16;
  int64_t ldd;
  int accumulate;
  int staged;  // fp32 output staged through the A buffer and stored (or added) by TMA (N <= 128, K >= 2N)
  uint32_t* err;
};

// D[M, N] (=|+=) A[M, K] * B (fp32 D, or bf16 D16).  Thread (warp w, lane l) owns tile row
// 32*(w%4) + l and the 32-column slices 32*(w/4) + 128*s of the accumulator.
__global__ void __launch_bounds__(kThreads, 1) tc_gemm_kernel(GemmArgs a, const __grid_constant__ CUtensorMap td) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ uint64_t wbar, mbar;
  __shared__ uint32_t tbase;
  const uint32_t abytes = 128u * uint32_t(a.K) * 2u;
  uint8_t* wimg = smem;
  uint8_t* xbuf[2];
  xbuf[0] = smem + ((a.img_bytes + 1023) & ~1023u);
  xbuf[1] = xbuf[0] + abytes;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int sp = warp & 3, cq = warp >> 2;
  if (tid == 0) {
    mbar_init(&wbar, 1);
    mbar_init(&mbar, 1);
    fence_barrier_init();
  }
  if (warp == 0) {
    tmem_alloc(&tbase, 256);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tm = tbase;
  if (tid == 0) {
    mbar_arrive_expect_tx(&wbar, a.img_bytes);
    for (uint32_t o = 0; o < a.img_bytes; o += 32768u) {
      uint32_t n = a.img_bytes - o < 32768u ? a.img_bytes - o : 32768u;
      bulk_g2s(wimg + o, a.img + o, n, &wbar);
    }
  }
  const int64_t tiles = (a.M + 127) / 128;
  if (blockIdx.x < tiles) issue_rows(xbuf[0], a.A, int64_t(blockIdx.x) * 128, a.M, tid);
  bool ok = mbar_wait(&wbar, 0, a.err);
  uint32_t ph = 0;
  const uint32_t idesc = idesc_bf16(128, a.N, false, a.b_mn != 0);
  const uint32_t lane_base = uint32_t(sp * 32) << 16;
  int i = 0;
  for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x, ++i) {
    // the previous tile's output stores have read its buffer, which the prefetch below refills
    if (a.staged && tid == 0) bulk_wait_read0();
    if (__syncthreads_or(!ok)) break;
    uint8_t* xa = xbuf[i & 1];
    const int64_t r0 = t * 128;
    if (t + gridDim.x < tiles) {  // prefetch the next tile, wait for this one
      issue_rows(xbuf[(i + 1) & 1], a.A, (t + gridDim.x) * 128, a.M, tid);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t xs = smem_u32(xa), ws = smem_u32(wimg);
      for (int k = 0; k < a.K / 16; ++k) {
        uint64_t bd = a.b_mn ? mnmajor_desc(ws, a.R, k) : kmajor_desc(ws, a.R, k);
        mma_bf16(tm, kmajor_desc(xs, 128, k), bd, idesc, k > 0);
      }
      mma_commit(&mbar);
    }
    ok = mbar_wait(&mbar, ph, a.err);
    ph ^= 1;
    if (__syncthreads_or(!ok)) break;
    tc_fence_after();
    const int r = sp * 32 + lane;
    const int64_t row = r0 + r;
    float v[32];
    if (a.D16) {
      // bf16 output, staged through this tile's A buffer (consumed by the MMA)
      // 128 columns at a time and copied out as whole row segments
      for (int c1 = 0; c1 < a.N; c1 += 128) {
        if (c1 + cq * 32 < a.N) {
          tmem_ld32(tm + lane_base + c1 + cq * 32, v);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            uint4 u;
            u.x = pack_bf16(v[8 * q + 0], v[8 * q + 1]);
            u.y = pack_bf16(v[8 * q + 2], v[8 * q + 3]);
            u.z = pack_bf16(v[8 * q + 4], v[8 * q + 5]);
            u.w = pack_bf16(v[8 * q + 6], v[8 * q + 7]);
            *reinterpret_cast<uint4*>(xa + sw_chunk(128, r, cq * 4 + q)) = u;
          }
        }
        __syncthreads();
        const int cw = a.N - c1 < 128 ? (a.N - c1) / 8 : 16;  // 16-byte chunks per row in this pass
        for (int q = tid; q < 128 * 16; q += kThreads) {
          const int rr = q >> 4, j = q & 15;
          if (j < cw && r0 + rr < a.M)
            *reinterpret_cast<uint4*>(a.D16 + (r0 + rr) * a.ldd + c1 + 8 * j) =
                *reinterpret_cast<const uint4*>(xa + sw_chunk(128, rr, j));
        }
        __syncthreads();
      }
    } else if (a.staged) {
      // fp32 output (N <= 128; the A buffer, consumed by the MMA, holds
      // 128 x K bf16 >= 128 x N fp32): 32-column boxes of 128 rows in the
      // 128-byte swizzle, stored or added into D by TMA (rows past M are
      // dropped by the copy), so no thread waits on a read of D
      if (cq * 32 < a.N) {
        tmem_ld32(tm + lane_base + cq * 32, v);
        uint8_t* const box = xa + cq * (128 * 128);
#pragma unroll
        for (int q = 0; q < 8; ++q)
          *reinterpret_cast<float4*>(box + r * 128 + ((q ^ (r & 7)) << 4)) =
              make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
      }
      fence_proxy_async();
      __syncthreads();
      if (tid == 0) {
        for (int b = 0; b < a.N / 32; ++b) {
          if (a.accumulate)
            tma_reduce_add_2d(&td, 32 * b, int(r0), xa + b * (128 * 128));
          else
            tma_store_2d(&td, 32 * b, int(r0), xa + b * (128 * 128));
        }
        bulk_commit();
      }
    } else {
      for (int c = cq * 32; c < a.N; c += 128) {
        tmem_ld32(tm + lane_base + c, v);
        if (row < a.M) {
          float* d = a.D + row * a.ldd + c;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            if (a.accumulate) {
              float p[8];
              ld8(d + 8 * q, p);
#pragma unroll
              for (int j = 0; j < 8; ++j) v[8 * q + j] += p[j];
            }
            st8(d + 8 * q, v + 8 * q);
          }
        }
      }
    }
    tc_fence_before();
  }
  cp_async_wait<0>();
  if (a.staged && tid == 0) bulk_wait0();  // every output copy is complete
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tm, 256);
}

// ---- G = X^T Y over rows.
struct TnArgs {
  Bf16Rows X;
  const bf16* Y;
  int64_t ldy;
  int N;
  int64_t M;
  int64_t tiles_per_cta;
  float* part;  // [cta][K1][N]
  uint32_t* err;
};

__global__ void __launch_bounds__(kThreads, 1) tc_gemm_tn_kernel(TnArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ uint64_t mbar;
  __shared__ uint32_t tbase;
  const int K1 = a.X.K();
  const uint32_t stage = 128u * uint32_t(K1 + a.N) * 2u;  // X tile then Y tile
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int sp = warp & 3, cq = warp >> 2;
  if (tid == 0) {
    mbar_init(&mbar, 1);
    fence_barrier_init();
  }
  if (warp == 0) {
    tmem_alloc(&tbase, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tm = tbase;
  const int64_t tiles = (a.M + 127) / 128;
  const int64_t t0 = int64_t(blockIdx.x) * a.tiles_per_cta;
  const int64_t t1 = min(tiles, t0 + a.tiles_per_cta);
  const uint32_t idesc = idesc_bf16(128, a.N, true, true);
  Bf16Rows Yr;
  Yr.p0 = a.Y;
  Yr.ld0 = a.ldy;
  Yr.w0 = a.N;
  auto issue = [&](int64_t t, int b) {
    uint8_t* st = smem + uint32_t(b) * stage;
    issue_rows(st, a.X, t * 128, a.M, tid);
    issue_rows(st + 128u * uint32_t(K1) * 2u, Yr, t * 128, a.M, tid);
  };
  if (t0 < t1) issue(t0, 0);
  uint32_t ph = 0;
  bool ok = true, any = false;
  for (int64_t t = t0; t < t1; ++t) {
    const int b = int((t - t0) & 1);
    if (t + 1 < t1) {
      // the other buffer was read by the previous tile's MMAs, which completed
      issue(t + 1, b ^ 1);
      cp_async_wait<2>();
    } else {
      cp_async_wait<0>();
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t xs = smem_u32(smem + uint32_t(b) * stage);
      const uint32_t ys = xs + 128u * uint32_t(K1) * 2u;
      for (int mb = 0; mb < K1 / 128; ++mb)
        for (int k = 0; k < 8; ++k)
          mma_bf16(tm + uint32_t(mb * a.N), mnmajor_desc(xs + uint32_t(mb) * 32768u, 128, k),
                   mnmajor_desc(ys, 128, k), idesc, (t > t0 || k > 0) ? 1u : 0u);
      mma_commit(&mbar);
    }
    ok = mbar_wait(&mbar, ph, a.err);
    ph ^= 1;
    any = true;
    if (__syncthreads_or(!ok)) break;
  }
  cp_async_wait<0>();
  tc_fence_after();
  float* P = a.part + int64_t(blockIdx.x) * K1 * a.N;
  const uint32_t lane_base = uint32_t(sp * 32) << 16;
  float v[32];
  for (int mb = 0; mb < K1 / 128; ++mb) {
    const int k = mb * 128 + sp * 32 + lane;
    for (int c = cq * 32; c < a.N; c += 128) {
      if (ok && any) {
        tmem_ld32(tm + lane_base + uint32_t(mb * a.N + c), v);
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = 0.f;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) st8(P + int64_t(k) * a.N + c + 8 * q, v + 8 * q);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tm, 512);
}

// Sums the per-CTA partials: a block owns 32 consecutive outputs, warp w sums
// the parts p = w (mod 8) in increasing order, the eight warp sums combine in
// a fixed tree (deterministic).
__global__ void __launch_bounds__(256) tn_reduce_kernel(const float* __restrict__ part, int nparts, int K1, int N,
                                                        int kvalid, int nvalid, int nsplit,
                                                        float* __restrict__ out) {
  __shared__ float red[8][32];
  const int64_t len = int64_t(K1) * N;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t i = int64_t(blockIdx.x) * 32 + lane;
  float s = 0.f;
  if (i < len)
    for (int p = w; p < nparts; p += 8) s += part[int64_t(p) * len + i];
  red[w][lane] = s;
  __syncthreads();
  if (w != 0 || i >= len) return;
  const int k = int(i / N), n = int(i % N);
  if (k >= kvalid || n >= nvalid) return;
  out[(int64_t(n / nsplit) * K1 + k) * nsplit + n % nsplit] =
      ((red[0][lane] + red[1][lane]) + (red[2][lane] + red[3][lane])) +
      ((red[4][lane] + red[5][lane]) + (red[6][lane] + red[7][lane]));
}

}  // namespace

int tc_grid(int64_t tiles) {
  int64_t g = num_sms();
  if (tiles < g) g = tiles;
  return int(g < 1 ? 1 : g);
}

PackJob pack_job(uint8_t* base, const Img& img, uint32_t r0, uint32_t nr, uint32_t nvalid, uint32_t kvalid,
                 const float* W, int64_t ld, int64_t wk0, int64_t wn0, bool lo) {
  PackJob j;
  j.dst = base + img.off;
  j.W = W;
  j.ld = ld;
  j.wk0 = wk0;
  j.wn0 = wn0;
  j.R = img.R;
  j.C = img.C;
  j.r0 = r0;
  j.nr = nr;
  j.nvalid = nvalid;
  j.kvalid = kvalid;
  j.lo = lo ? 1 : 0;
  return j;
}

xmgn_status pack_images(const std::vector<PackJob>& jobs, cudaStream_t s) {
  for (size_t b0 = 0; b0 < jobs.size(); b0 += kPackBatch) {
    PackBatch b;
    b.n = int(jobs.size() - b0 < size_t(kPackBatch) ? jobs.size() - b0 : size_t(kPackBatch));
    int64_t most = 1;
    for (int i = 0; i < b.n; ++i) {
      b.j[i] = jobs[b0 + i];
      const int64_t e = int64_t(b.j[i].nr) * b.j[i].C;
      if (e > most) most = e;
    }
    const int64_t gx = (most + 255) / 256 < 128 ? (most + 255) / 256 : 128;
    pack_kernel<<<dim3(unsigned(gx), unsigned(b.n)), 256, 0, s>>>(b);
    XMGN_LAUNCH_CHECK();
  }
  return XMGN_OK;
}

xmgn_status tc_gemm(const Bf16Rows& A, int64_t M, const uint8_t* img_base, const Img& img, bool b_mn,
                    int N, float* D, int64_t ldd, bool accumulate, cudaStream_t s, bf16* D16) {
  if (M <= 0) return XMGN_OK;
  if (N % 32 || N > 256 || A.K() % 64 || A.K() > 256) return fail(XMGN_ERR_UNSUPPORTED, "tc_gemm shape");
  if (!D == !D16 || (D16 && accumulate)) return fail(XMGN_ERR_ARG, "tc_gemm: one of D, D16; D16 is written");
  if (D16 && (ldd % 8 || reinterpret_cast<uintptr_t>(D16) % 16))
    return fail(XMGN_ERR_ARG, "tc_gemm: bf16 output rows must be 16-byte aligned");
  GemmArgs a;
  a.A = A;
  a.M = M;
  a.img = img_base + img.off;
  a.img_bytes = img.bytes();
  a.R = img.R;
  a.N = N;
  a.K = A.K();
  a.b_mn = b_mn ? 1 : 0;
  a.D = D;
  a.D16 = D16;
  a.ldd = ldd;
  a.accumulate = accumulate ? 1 : 0;
  a.staged = (!D16 && N <= 128 && a.K >= 2 * N && ldd % 4 == 0 &&
              reinterpret_cast<uintptr_t>(D) % 16 == 0) ? 1 : 0;
  a.err = device_error_word();
  CUtensorMap td;
  memset(&td, 0, sizeof(td));
  if (a.staged) XMGN_TRY(f32_map(&td, D, M, N, ldd));
  const size_t smem = 1024 + ((a.img_bytes + 1023) & ~1023u) + 2 * size_t(128) * a.K * 2;
  static bool attr = false;
  if (!attr) {
    XMGN_TRY(allow_max_smem(tc_gemm_kernel));
    attr = true;
  }
  tc_gemm_kernel<<<tc_grid((M + 127) / 128), kThreads, smem, s>>>(a, td);
  XMGN_LAUNCH_CHECK();
  return XMGN_OK;
}

size_t tc_gemm_tn_part_elems(int K1, int N) { return size_t(num_sms()) * size_t(K1) * size_t(N); }

xmgn_status tc_gemm_tn(const Bf16Rows& X, const bf16* Y, int64_t ldy, int N, int64_t M, float* out,
                       int kvalid, int nvalid, int nsplit, float* part, cudaStream_t s) {
  const int K1 = X.K();
  if ((K1 != 128 && K1 != 256) || N % 64 || N > 256 || (K1 / 128) * N > 512)
    return fail(XMGN_ERR_UNSUPPORTED, "tc_gemm_tn shape K1=%d N=%d", K1, N);
  const int64_t tiles = (M + 127) / 128;
  // one CTA per SM, or (tuned) one per two SMs: half the partials to reduce
  const int full = tc_grid(tiles);
  const int grid = tune_choice(TUNE_TN_GRID, M) == 1 && full > 1 ? (full + 1) / 2 : full;
  TnArgs a;
  a.X = X;
  a.Y = Y;
  a.ldy = ldy;
  a.N = N;
  a.M = M;
  a.tiles_per_cta = (tiles + grid - 1) / grid;
  a.part = part;
  a.err = device_error_word();
  const size_t smem = 1024 + 2 * size_t(128) * (K1 + N) * 2;
  static bool attr = false;
  if (!attr) {
    XMGN_TRY(allow_max_smem(tc_gemm_tn_kernel));
    attr = true;
  }
  tune_begin(TUNE_TN_GRID, s);
  tc_gemm_tn_kernel<<<grid, kThreads, smem, s>>>(a);
  XMGN_LAUNCH_CHECK();
  tn_reduce_kernel<<<unsigned((int64_t(K1) * N + 31) / 32), 256, 0, s>>>(part, grid, K1, N, kvalid, nvalid, nsplit,
                                                                         out);
  XMGN_LAUNCH_CHECK();
  tune_end(TUNE_TN_GRID, s);
  return XMGN_OK;
}

}  // namespace xmgn
