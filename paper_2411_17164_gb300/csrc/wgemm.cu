// Tensor-core GEMMs of the wide BF16 path (hidden widths other than 128, the
// paper's production width 512), hand-written for tcgen05:
//
//   NN  D[M, N] (=|+=) A[M, K] B[K, N]        B row-major, N contiguous (MN-major operand)
//   NT  D[M, N] (=|+=) A[M, K] B[N, K]^T      B row-major, K contiguous (K-major operand)
//   TN  G[K1, N] = sum over rows m of A[m, :]^T B[m, :]   (the weight gradients; the rows
//       are the reduction, split over CTAs, partials summed in a fixed order)
//
// Operands are bf16 row-major arrays whose leading dimensions are multiples of
// 8 elements (16 bytes, the TMA stride rule); results are fp32.  Shapes need
// no padding in memory beyond that: TMA reads zeros past the last row and
// column, so K, N and M are arbitrary.
//
// One persistent CTA per SM of 192 threads: warp 0 moves 64-deep slices of A
// and B into a ring of four shared-memory stages with TMA (128-byte swizzle,
// the layout tcgen05.mma reads), warp 1 issues the MMAs (one thread) into one
// of two TMEM accumulators of 128 x BN fp32, warps 2-5 read the finished
// accumulator (lane quadrant w % 4) and store it, so that one output tile's
// stores overlap the next tile's products.  The epilogue writes each 128 x 32
// fp32 chunk of the accumulator into one of two 16 KB shared-memory staging
// buffers (128-byte swizzle, conflict-free) and one thread sends it out with a
// TMA tensor store (a TMA reduce-add for the accumulating form), so global
// memory sees whole 128-byte row segments.  The first-layer form
// (wg_gemm_silu) applies bias and SiLU in the epilogue and stores bf16 blocks
// of 64 columns (optionally also the fp32 pre-activation), so the fp32
// product never goes to memory.  Every wait is bounded: a wait that gives up
// flags the device error word and the roles wind down.
#include <cuda.h>

#include "model.cuh"
#include "tc_gemm.cuh"
#include "wgemm.cuh"

namespace xmgn {

using namespace tc;

namespace {

constexpr int kBM = 128, kBK = 64, kStages = 4, kWgThreads = 192;
constexpr uint32_t kAStage = kBM * kBK * 2;  // 16 KB
constexpr uint32_t kStage = kBM * 32 * 4;    // an output staging buffer: 128 rows x 32 fp32, 16 KB

struct WgArgs {
  int mode;             // WG_NN, WG_NT, WG_TN
  int64_t M;            // NN/NT: output rows; TN: reduction rows
  int N;                // output columns
  int K;                // NN/NT: reduction depth; TN: output rows K1
  int BN;               // output tile width: 64, 128 or 256
  int tiles_m, tiles_n; // output tiles (TN: of K1 x N)
  int splits;           // TN: row-range splits
  int64_t kb_split;     // TN: 64-row blocks per split
  float* D;             // NN/NT output
  int64_t ldd;
  int accum;            // NN/NT: add into D
  float* part;          // TN: [split][tile][128][BN] partial sums
  int silu;             // NN with the first MLP layer's epilogue: SiLU(product + bias) stored in bf16
  int pre;              // with silu: the pre-activation product + bias also stored (fp32, map tp)
  const float* bias;    // [N], with silu
  uint32_t* err;
};

// SiLU with the fast exponential and division (its output is rounded to bf16)
__device__ __forceinline__ float silu_fast(float z) { return __fdividef(z, 1.f + __expf(-z)); }

// Bounded wait that also gives up at once when another role already has.
__device__ __forceinline__ bool wg_wait(uint64_t* bar, uint32_t parity, uint32_t* err, volatile int* quit) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*quit) return false;
    if (globaltimer() - t0 > 1000000000ull) {
      dev_flag(err, DEV_ERR_TIMEOUT);
      *quit = 1;
      return false;
    }
  }
}

// Output tile t of the launch: (tile row, tile column, split).
__device__ __forceinline__ void tile_of(const WgArgs& a, int64_t t, int& tm, int& tn, int& sp) {
  tn = int(t % a.tiles_n);
  const int64_t q = t / a.tiles_n;
  tm = int(q % a.tiles_m);
  sp = int(q / a.tiles_m);
}

// 64-deep K slices of tile t: NN/NT the reduction depth, TN the rows of the split.
__device__ __forceinline__ int64_t kblocks(const WgArgs& a, int sp, int64_t& kb0) {
  if (a.mode != WG_TN) {
    kb0 = 0;
    return (a.K + kBK - 1) / kBK;
  }
  const int64_t nb = (a.M + kBK - 1) / kBK;
  kb0 = int64_t(sp) * a.kb_split;
  const int64_t e = kb0 + a.kb_split < nb ? kb0 + a.kb_split : nb;
  return e > kb0 ? e - kb0 : 0;
}

__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }
// AND of p over the 128 epilogue threads (also a barrier among them), so that
// they leave the tile loop together.
__device__ __forceinline__ bool epi_all(bool p) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred q, o;\n\tsetp.ne.u32 q, %1, 0;\n\tbar.red.and.pred o, 1, 128, q;\n\tselp.u32 %0, 1, 0, o;\n\t}"
      : "=r"(r)
      : "r"(p ? 1u : 0u)
      : "memory");
  return r != 0;
}

__global__ void __launch_bounds__(kWgThreads, 1) wg_kernel(WgArgs a, const __grid_constant__ CUtensorMap ta,
                                                             const __grid_constant__ CUtensorMap tb,
                                                             const __grid_constant__ CUtensorMap td,
                                                             const __grid_constant__ CUtensorMap tp) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ uint64_t full[kStages], empty[kStages], accf[2], acce[2];
  __shared__ uint32_t tbase;
  __shared__ volatile int quit;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int BN = a.BN;
  const uint32_t bstage = uint32_t(BN) * kBK * 2u;
  const uint32_t stage = kAStage + bstage;
  const int64_t tiles = int64_t(a.tiles_m) * a.tiles_n * a.splits;
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&accf[i], 1);
      mbar_init(&acce[i], 128);
    }
    quit = 0;
    fence_barrier_init();
  }
  if (warp == 1) {
    tmem_alloc(&tbase, uint32_t(2 * BN) < 32u ? 32u : uint32_t(2 * BN));
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tacc = tbase;
  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      for (int s = 0; s < kStages; ++s) mbar_arrive(&empty[s]);  // every stage starts free
      uint32_t it = 0;
      for (int64_t t = blockIdx.x; t < tiles && !quit; t += gridDim.x) {
        int tm, tn, sp;
        tile_of(a, t, tm, tn, sp);
        int64_t kb0;
        const int64_t nk = kblocks(a, sp, kb0);
        for (int64_t kb = 0; kb < nk; ++kb, ++it) {
          const int s = int(it % kStages);
          if (!wg_wait(&empty[s], (it / kStages) & 1u, a.err, &quit)) break;
          uint8_t* sa = base + s * stage;
          uint8_t* sb = sa + kAStage;
          mbar_arrive_expect_tx(&full[s], stage);
          const int k0 = int((kb0 + kb) * kBK);
          if (a.mode == WG_TN) {
            // A^T slice: 64 rows of A x 128 of its K1 columns, as two 64-column blocks
            tma_load_2d(sa, &ta, tm * kBM, k0, &full[s]);
            tma_load_2d(sa + kAStage / 2, &ta, tm * kBM + 64, k0, &full[s]);
          } else {
            tma_load_2d(sa, &ta, k0, tm * kBM, &full[s]);  // 128 rows x 64 K
          }
          if (a.mode == WG_NT) {
            tma_load_2d(sb, &tb, k0, tn * BN, &full[s]);  // BN rows x 64 K
          } else {
            for (int j = 0; j < BN / 64; ++j)  // 64 K rows x BN columns, 64-column blocks
              tma_load_2d(sb + j * (kBK * 128), &tb, tn * BN + 64 * j, k0, &full[s]);
          }
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const bool a_mn = a.mode == WG_TN, b_mn = a.mode != WG_NT;
      const uint32_t idesc = idesc_bf16(kBM, BN, a_mn, b_mn);
      uint32_t it = 0, i = 0;
      for (int64_t t = blockIdx.x; t < tiles && !quit; t += gridDim.x, ++i) {
        int tm, tn, sp;
        tile_of(a, t, tm, tn, sp);
        int64_t kb0;
        const int64_t nk = kblocks(a, sp, kb0);
        const uint32_t acc = i & 1u;
        // the epilogue has emptied this accumulator (its 128 arrivals complete one phase per use;
        // the first use of each accumulator finds it free)
        if (i >= 2 && !wg_wait(&acce[acc], ((i >> 1) - 1) & 1u, a.err, &quit)) break;
        tc_fence_after();
        const uint32_t d = tacc + acc * uint32_t(BN);
        bool any = false;
        for (int64_t kb = 0; kb < nk; ++kb, ++it) {
          const int s = int(it % kStages);
          if (!wg_wait(&full[s], (it / kStages) & 1u, a.err, &quit)) break;
          tc_fence_after();
          const uint32_t sa = smem_u32(base + s * stage), sb = sa + kAStage;
#pragma unroll
          for (int k = 0; k < kBK / 16; ++k) {
            const uint64_t da = a_mn ? mnmajor_desc(sa, 64, k) : kmajor_desc(sa, kBM, k);
            const uint64_t db = b_mn ? mnmajor_desc(sb, 64, k) : kmajor_desc(sb, BN, k);
            mma_bf16(d, da, db, idesc, any ? 1u : 0u);
            any = true;
          }
          mma_commit(&empty[s]);  // the stage is free once these products have read it
        }
        mma_commit(&accf[acc]);
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue (warps 2..5)
    const int q = warp & 3;  // TMEM lane quadrant of this warp
    const int r = 32 * q + lane;
    const uint32_t lane_base = uint32_t(32 * q) << 16;
    const bool leader = tid == 64;
    uint8_t* const stg = base + kStages * stage;  // two staging buffers
    uint32_t i = 0, nchunk = 0;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x, ++i) {
      int tm, tn, sp;
      tile_of(a, t, tm, tn, sp);
      int64_t kb0;
      const int64_t nk = kblocks(a, sp, kb0);
      const uint32_t acc = i & 1u;
      if (!epi_all(wg_wait(&accf[acc], (i >> 1) & 1u, a.err, &quit))) break;
      tc_fence_after();
      const uint32_t d = tacc + acc * uint32_t(BN) + lane_base;
      // output coordinates of the tile: NN/NT the rows and columns of D, TN the
      // tile's rows in the partial array (one 128 x BN block per split and tile)
      const int y0 = a.mode == WG_TN ? int(((int64_t(sp) * a.tiles_m + tm) * a.tiles_n + tn) * kBM) : tm * kBM;
      const int x0 = a.mode == WG_TN ? 0 : tn * BN;
      if (a.silu) {  // 64-column blocks: A1 = bf16(SiLU(product + b1)), one TMA store each
        for (int c = 0; c < BN; c += 64, ++nchunk) {
          uint32_t h[32];
#pragma unroll 1
          for (int half = 0; half < 2; ++half) {
            float v[32];
            tmem_ld32(d + c + 32 * half, v);
            const int col = x0 + c + 32 * half;
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] += col + j < a.N ? a.bias[col + j] : 0.f;
            if (a.pre) {  // the pre-activation, 32 fp32 columns, through a staging buffer
              uint8_t* const pb = stg + (nchunk & 1u) * kStage;
              ++nchunk;
              if (leader) bulk_wait_read1();
              epi_sync();
#pragma unroll
              for (int j = 0; j < 8; ++j)
                *reinterpret_cast<float4*>(pb + r * 128 + ((j ^ (r & 7)) << 4)) =
                    make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
              fence_proxy_async();
              epi_sync();
              if (leader) {
                tma_store_2d(&tp, col, y0, pb);
                bulk_commit();
              }
            }
#pragma unroll
            for (int j = 0; j < 32; j += 2) h[16 * half + j / 2] = pack_bf16(silu_fast(v[j]), silu_fast(v[j + 1]));
          }
          uint8_t* const buf = stg + (nchunk & 1u) * kStage;
          if (leader) bulk_wait_read1();  // the store that last used this buffer has read it
          epi_sync();
#pragma unroll
          for (int j = 0; j < 8; ++j)
            *reinterpret_cast<uint4*>(buf + r * 128 + ((j ^ (r & 7)) << 4)) =
                make_uint4(h[4 * j], h[4 * j + 1], h[4 * j + 2], h[4 * j + 3]);
          fence_proxy_async();
          epi_sync();
          if (leader) {
            tma_store_2d(&td, x0 + c, y0, buf);
            bulk_commit();
          }
        }
        tc_fence_before();
        mbar_arrive(&acce[acc]);
        continue;
      }
      for (int c = 0; c < BN; c += 32, ++nchunk) {
        float v[32];
        tmem_ld32(d + c, v);
        if (nk == 0) {
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] = 0.f;
        }
        uint8_t* const buf = stg + (nchunk & 1u) * kStage;
        if (leader) bulk_wait_read1();  // the store that last used this buffer has read it
        epi_sync();
#pragma unroll
        for (int j = 0; j < 8; ++j)
          *reinterpret_cast<float4*>(buf + r * 128 + ((j ^ (r & 7)) << 4)) =
              make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
        fence_proxy_async();
        epi_sync();
        if (leader) {
          if (a.accum)
            tma_reduce_add_2d(&td, x0 + c, y0, buf);
          else
            tma_store_2d(&td, x0 + c, y0, buf);
          bulk_commit();
        }
      }
      tc_fence_before();
      mbar_arrive(&acce[acc]);
    }
  }
  if (tid == 64) bulk_wait0();  // every output store is complete
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tacc, uint32_t(2 * BN) < 32u ? 32u : uint32_t(2 * BN));
}

// G[K1, N] = sum over splits of the partial tiles, in split order.
__global__ void __launch_bounds__(256) wg_reduce_kernel(const float* __restrict__ part, int splits, int tiles_m,
                                                        int tiles_n, int BN, int K1, int N, float* __restrict__ G) {
  const int64_t total = int64_t(K1) * N;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const int k = int(e / N), n = int(e % N);
    const int tm = k / kBM, tn = n / BN;
    const int64_t off = (int64_t(tm) * tiles_n + tn) * (int64_t(kBM) * BN) + int64_t(k % kBM) * BN + n % BN;
    const int64_t stride = int64_t(tiles_m) * tiles_n * kBM * BN;
    float s = 0.f;
    for (int sp = 0; sp < splits; ++sp) s += part[sp * stride + off];
    G[e] = s;
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// Tensor map of a row-major bf16 [rows, cols] array with leading dimension ld
// (a multiple of 8), boxes of 64 columns x box_rows rows, 128-byte swizzle.
xmgn_status bf16_map(CUtensorMap* m, const bf16* p, int64_t rows, int64_t cols, int64_t ld, uint32_t box_rows) {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    XMGN_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !f) return fail(XMGN_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
    fn = reinterpret_cast<EncodeTiledFn>(f);
  }
  if (!p || rows < 1 || cols < 1 || cols > ld || (ld & 7) || (reinterpret_cast<uintptr_t>(p) & 15) ||
      rows >= (int64_t(1) << 31))
    return fail(XMGN_ERR_ARG, "wide GEMM operand: bad pointer, shape or leading dimension (%lld x %lld, ld %lld)",
                (long long)rows, (long long)cols, (long long)ld);
  const cuuint64_t dims[2] = {cuuint64_t(cols), cuuint64_t(rows)};
  const cuuint64_t strides[1] = {cuuint64_t(ld) * 2u};
  const cuuint32_t box[2] = {64u, box_rows};
  const cuuint32_t es[2] = {1u, 1u};
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16*>(p), dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(XMGN_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", int(r));
  return XMGN_OK;
}

}  // namespace

xmgn_status f32_map(CUtensorMap* m, float* p, int64_t rows, int64_t cols, int64_t ld) {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    XMGN_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !f) return fail(XMGN_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
    fn = reinterpret_cast<EncodeTiledFn>(f);
  }
  if (!p || rows < 1 || cols < 1 || cols > ld || (ld & 3) || (reinterpret_cast<uintptr_t>(p) & 15) ||
      rows >= (int64_t(1) << 31))
    return fail(XMGN_ERR_ARG, "GEMM fp32 output: bad pointer, shape or leading dimension (%lld x %lld, ld %lld)",
                (long long)rows, (long long)cols, (long long)ld);
  const cuuint64_t dims[2] = {cuuint64_t(cols), cuuint64_t(rows)};
  const cuuint64_t strides[1] = {cuuint64_t(ld) * 4u};
  const cuuint32_t box[2] = {32u, uint32_t(kBM)};
  const cuuint32_t es[2] = {1u, 1u};
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, p, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(XMGN_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", int(r));
  return XMGN_OK;
}

namespace {

int tile_width(int N) { return N > 128 ? 256 : (N > 64 ? 128 : 64); }

uint32_t smem_of(int BN) { return kStages * (kAStage + uint32_t(BN) * kBK * 2u) + 2u * kStage + 1024u; }

xmgn_status launch(WgArgs& a, const CUtensorMap& ta, const CUtensorMap& tb, const CUtensorMap& td, cudaStream_t s,
                   const CUtensorMap* tp = nullptr) {
  static bool attr = false;
  if (!attr) {
    XMGN_CUDA(cudaFuncSetAttribute(wg_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem_of(256))));
    attr = true;
  }
  a.err = device_error_word();
  const int64_t tiles = int64_t(a.tiles_m) * a.tiles_n * a.splits;
  const int grid = int(tiles < num_sms() ? tiles : num_sms());
  const uint32_t smem = smem_of(a.BN);
  probe_begin(PROBE_WIDE_GEMM, s);
  CUtensorMap none;
  memset(&none, 0, sizeof(none));
  wg_kernel<<<grid, kWgThreads, smem, s>>>(a, ta, tb, td, tp ? *tp : none);
  probe_end(PROBE_WIDE_GEMM, s);
  XMGN_LAUNCH_CHECK();
  return XMGN_OK;
}

}  // namespace

int64_t wg_part_elems() { return int64_t(2) * num_sms() * kBM * 256; }

xmgn_status wg_gemm(int mode, const bf16* A, int64_t lda, const bf16* B, int64_t ldb, int64_t M, int N, int K,
                    float* D, int64_t ldd, bool accum, cudaStream_t s) {
  if (mode != WG_NN && mode != WG_NT) return fail(XMGN_ERR_ARG, "wg_gemm: mode");
  if (M <= 0 || N <= 0 || K <= 0) return XMGN_OK;
  if (N > 512 || !D || ldd < N) return fail(XMGN_ERR_ARG, "wg_gemm: N %d (at most 512) or ldd", N);
  WgArgs a{};
  a.mode = mode;
  a.M = M;
  a.N = N;
  a.K = K;
  a.BN = tile_width(N);
  a.tiles_m = int((M + kBM - 1) / kBM);
  a.tiles_n = (N + a.BN - 1) / a.BN;
  a.splits = 1;
  a.D = D;
  a.ldd = ldd;
  a.accum = accum ? 1 : 0;
  CUtensorMap ta, tb, td;
  XMGN_TRY(bf16_map(&ta, A, M, K, lda, kBM));
  if (mode == WG_NT)
    XMGN_TRY(bf16_map(&tb, B, N, K, ldb, uint32_t(a.BN)));  // B [N, K]
  else
    XMGN_TRY(bf16_map(&tb, B, K, N, ldb, kBK));  // B [K, N]
  XMGN_TRY(f32_map(&td, D, M, N, ldd));
  return launch(a, ta, tb, td, s);
}

xmgn_status wg_gemm_silu(const bf16* A, int64_t lda, const bf16* B, int64_t ldb, int64_t M, int N, int K,
                         const float* bias, bf16* c16, int64_t ld16, cudaStream_t s, float* pre, int64_t ldp) {
  if (M <= 0 || N <= 0 || K <= 0) return XMGN_OK;
  if (N > 512 || !bias || !c16 || ld16 < N) return fail(XMGN_ERR_ARG, "wg_gemm_silu: N %d or output", N);
  WgArgs a{};
  a.mode = WG_NN;
  a.M = M;
  a.N = N;
  a.K = K;
  a.BN = tile_width(N);
  a.tiles_m = int((M + kBM - 1) / kBM);
  a.tiles_n = (N + a.BN - 1) / a.BN;
  a.splits = 1;
  a.silu = 1;
  a.bias = bias;
  CUtensorMap ta, tb, td;
  XMGN_TRY(bf16_map(&ta, A, M, K, lda, kBM));
  XMGN_TRY(bf16_map(&tb, B, K, N, ldb, kBK));
  XMGN_TRY(bf16_map(&td, c16, M, N, ld16, kBM));  // 64 bf16 columns x 128 rows per store
  if (!pre) return launch(a, ta, tb, td, s);
  CUtensorMap tp;
  XMGN_TRY(f32_map(&tp, pre, M, N, ldp));  // 32 fp32 columns x 128 rows per store
  a.pre = 1;
  return launch(a, ta, tb, td, s, &tp);
}

xmgn_status wg_gemm_tn(const bf16* A, int64_t lda, const bf16* B, int64_t ldb, int64_t M, int K1, int N, float* G,
                       float* part, cudaStream_t s) {
  if (K1 <= 0 || N <= 0) return XMGN_OK;
  if (M <= 0) {
    XMGN_CUDA(cudaMemsetAsync(G, 0, sizeof(float) * size_t(K1) * N, s));
    return XMGN_OK;
  }
  if (N > 512 || K1 > 4096) return fail(XMGN_ERR_ARG, "wg_gemm_tn: K1 %d or N %d too large", K1, N);
  WgArgs a{};
  a.mode = WG_TN;
  a.M = M;
  a.N = N;
  a.K = K1;
  a.BN = tile_width(N);
  a.tiles_m = (K1 + kBM - 1) / kBM;
  a.tiles_n = (N + a.BN - 1) / a.BN;
  const int64_t nb = (M + kBK - 1) / kBK;
  const int64_t tiles = int64_t(a.tiles_m) * a.tiles_n;
  // about two partial tiles per SM, bounded by the partial buffer, no empty split
  const int64_t cap = wg_part_elems() / (int64_t(kBM) * a.BN) / tiles;
  int64_t splits = (2 * int64_t(num_sms()) + tiles - 1) / tiles;
  if (splits > cap) splits = cap;
  if (splits > nb) splits = nb;
  if (splits < 1) return fail(XMGN_ERR_ARG, "wg_gemm_tn: partial buffer too small for %d x %d", K1, N);
  a.kb_split = (nb + splits - 1) / splits;
  a.splits = int((nb + a.kb_split - 1) / a.kb_split);
  a.part = part;
  CUtensorMap ta, tb, td;
  XMGN_TRY(bf16_map(&ta, A, M, K1, lda, kBK));  // 64 rows x 64 of K1
  XMGN_TRY(bf16_map(&tb, B, M, N, ldb, kBK));   // 64 rows x 64 of N
  XMGN_TRY(f32_map(&td, part, int64_t(a.splits) * tiles * kBM, a.BN, a.BN));  // [split][tile] blocks of 128 x BN
  XMGN_TRY(launch(a, ta, tb, td, s));
  const int64_t total = int64_t(K1) * N;
  wg_reduce_kernel<<<grid_for(total, 256, int64_t(num_sms()) * 8), 256, 0, s>>>(part, a.splits, a.tiles_m, a.tiles_n,
                                                                               a.BN, K1, N, G);
  XMGN_LAUNCH_CHECK();
  return XMGN_OK;
}

}  // namespace xmgn
