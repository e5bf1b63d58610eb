// SIMT (CUDA-core, fp32) building blocks: tiled GEMMs over gathered row
// sources, LayerNorm forward/backward, segmented sums over CSR/CSC, edge
// features, masked MSE.  All reductions use fixed work assignment and fixed
// summation order, so results are bit-reproducible.
#include <math.h>

#include <initializer_list>

#include "model.cuh"

namespace xmgn {

namespace {
constexpr int BT = 64;   // output tile edge
constexpr int BK = 16;   // reduction step
constexpr int kLnBlocksMax = 1024;  // LayerNorm-backward blocks, each writing one partial of dgamma, dbeta

__device__ __forceinline__ float src_get(const RowSrc& A, int64_t r, int k) {
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    if (s < A.nseg) {
      const RowSeg& g = A.s[s];
      if (k < g.width) {
        int64_t row = g.idx ? int64_t(g.idx[r]) : r;
        return g.p[row * g.ld + k];
      }
      k -= g.width;
    }
  }
  return 0.f;
}

// sum_{p < n} x[p * stride] as eight independent partial sums (p mod 8)
// combined in a fixed order: deterministic, and eight loads in flight.
__device__ __forceinline__ float sum_strided(const float* __restrict__ x, int n, int64_t stride) {
  float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  int p = 0;
  for (; p + 8 <= n; p += 8)
#pragma unroll
    for (int q = 0; q < 8; ++q) s[q] += x[int64_t(p + q) * stride];
  for (int q = 0; p < n; ++p, ++q) s[q] += x[int64_t(p) * stride];
  return ((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7]));
}

__device__ __forceinline__ float silu_f(float z) { return z / (1.f + __expf(-z)); }
__device__ __forceinline__ float silu_grad_f(float z) {
  float s = 1.f / (1.f + __expf(-z));
  return s * (1.f + z * (1.f - s));
}

template <bool NT>
__global__ void __launch_bounds__(256) gemm_nnt_kernel(RowSrc A, int64_t M, const float* __restrict__ B,
                                                       int N, const float* __restrict__ bias,
                                                       float* __restrict__ C, int64_t ldc, int epi,
                                                       float* __restrict__ pre,
                                                       const float* __restrict__ aux) {
  __shared__ float As[BK][BT + 4];
  __shared__ float Bs[BK][BT + 4];
  const int K = A.K;
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  const int64_t m0 = int64_t(blockIdx.x) * BT;
  const int n0 = blockIdx.y * BT;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int idx = t + 256 * i;
      int mm = idx >> 4, kk = idx & 15;
      int64_t m = m0 + mm;
      int k = k0 + kk;
      As[kk][mm] = (m < M && k < K) ? src_get(A, m, k) : 0.f;
      int nn = idx & 63, kb = idx >> 6;
      int n = n0 + nn, kq = k0 + kb;
      float bv = 0.f;
      if (n < N && kq < K) bv = NT ? B[int64_t(n) * K + kq] : B[int64_t(kq) * N + n];
      Bs[kb][nn] = bv;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int64_t m = m0 + ty * 4 + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int n = n0 + tx * 4 + j;
      if (n >= N) continue;
      float v = acc[i][j] + (bias ? bias[n] : 0.f);
      float* c = C + m * ldc + n;
      switch (epi) {
        case EPI_STORE: *c = v; break;
        case EPI_SILU:
          if (pre) pre[m * ldc + n] = v;
          *c = silu_f(v);
          break;
        case EPI_ACCUM: *c += v; break;
        case EPI_SILU_GRAD: *c = acc[i][j] * silu_grad_f(aux[m * ldc + n]); break;
      }
    }
  }
}

__global__ void __launch_bounds__(256) gemm_tn_kernel(RowSrc A, int64_t M, const float* __restrict__ B,
                                                      int64_t ldb, int N, int64_t rows_per_chunk,
                                                      float* __restrict__ part) {
  __shared__ float As[BK][BT + 4];
  __shared__ float Bs[BK][BT + 4];
  const int K1 = A.K;
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  const int ntn = (N + BT - 1) / BT;
  const int k10 = (blockIdx.x / ntn) * BT;
  const int n0 = (blockIdx.x % ntn) * BT;
  const int64_t r_begin = int64_t(blockIdx.y) * rows_per_chunk;
  const int64_t r_end = min(M, r_begin + rows_per_chunk);
  float acc[4][4] = {};
  for (int64_t r0 = r_begin; r0 < r_end; r0 += BK) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int idx = t + 256 * i;
      int rr = idx >> 6, cc = idx & 63;
      int64_t r = r0 + rr;
      int k1 = k10 + cc, n = n0 + cc;
      bool rv = r < r_end;
      As[rr][cc] = (rv && k1 < K1) ? src_get(A, r, k1) : 0.f;
      Bs[rr][cc] = (rv && n < N) ? B[r * ldb + n] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int rr = 0; rr < BK; ++rr) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[rr][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[rr][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  float* P = part + int64_t(blockIdx.y) * K1 * N;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int k1 = k10 + ty * 4 + i;
    if (k1 >= K1) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int n = n0 + tx * 4 + j;
      if (n < N) P[int64_t(k1) * N + n] = acc[i][j];
    }
  }
}

__global__ void reduce_chunks_kernel(const float* __restrict__ part, int nchunk, int64_t len,
                                     float* __restrict__ out) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < len;
       i += int64_t(gridDim.x) * blockDim.x) {
    out[i] = sum_strided(part + i, nchunk, len);
  }
}

int tn_chunks(int64_t M) {
  int64_t c = (M + 4095) / 4096;
  if (c > 128) c = 128;
  if (c < 1) c = 1;
  return int(c);
}

// Column sums of one chunk of rows (eight loads in flight per thread).
__global__ void colsum_kernel(const float* __restrict__ X, int64_t M, int N, int64_t ld,
                              int64_t rows_per_chunk, float* __restrict__ part) {
  const int64_t r0 = int64_t(blockIdx.x) * rows_per_chunk;
  const int64_t r1 = min(M, r0 + rows_per_chunk);
  for (int n = threadIdx.x; n < N; n += blockDim.x)
    part[int64_t(blockIdx.x) * N + n] = r1 > r0 ? sum_strided(X + r0 * ld + n, int(r1 - r0), ld) : 0.f;
}

// Row chunks of the column sums: enough blocks to fill the GPU.
int colsum_chunks(int64_t M) {
  int64_t c = (M + 255) / 256;
  const int64_t cap = int64_t(num_sms()) * 8;
  if (c > cap) c = cap;
  if (c < 1) c = 1;
  return int(c);
}

constexpr int kMaxVpl = 16;  // features per lane (N <= 512)

__global__ void ln_fwd_kernel(const float* __restrict__ Z, const float* __restrict__ bias, int64_t M, int N,
                              const float* __restrict__ gamma, const float* __restrict__ beta,
                              float* __restrict__ Y, const float* resid_in, float* resid_out) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  const int vpl = N >> 5;
  for (int64_t r = warp; r < M; r += nw) {
    float v[kMaxVpl];
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kMaxVpl; ++j)
      if (j < vpl) {
        v[j] = Z[r * N + lane + 32 * j];
        if (bias) v[j] += bias[lane + 32 * j];
        s += v[j];
      }
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const float mu = s / N;
    float q = 0.f;
#pragma unroll
    for (int j = 0; j < kMaxVpl; ++j)
      if (j < vpl) {
        float d = v[j] - mu;
        q += d * d;
      }
    for (int o = 16; o; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    const float rstd = rsqrtf(q / N + kLnEps);
#pragma unroll
    for (int j = 0; j < kMaxVpl; ++j)
      if (j < vpl) {
        int c = lane + 32 * j;
        float y = (v[j] - mu) * rstd * gamma[c] + beta[c];
        if (Y) Y[r * N + c] = y;
        if (resid_out) resid_out[r * N + c] = resid_in[r * N + c] + y;
      }
  }
}

// LayerNorm backward, a warp per row.  The dgamma/dbeta contributions are
// accumulated per warp in shared memory (each lane owns its columns, so the
// updates need no atomics), combined over the block's eight warps in fixed
// order, and written as one partial row pair per block.
__global__ void __launch_bounds__(256, 3)
    ln_bwd_kernel(const float* __restrict__ Z, const float* __restrict__ bias, int64_t M, int N,
                  const float* __restrict__ gamma, const float* __restrict__ dY1, const float* __restrict__ dY2,
                  const int32_t* __restrict__ idx2, float* __restrict__ dZ, float* __restrict__ part) {
  extern __shared__ float ln_acc[];  // [8 warps][dgamma N | dbeta N]
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  float* acc = ln_acc + wib * 2 * N;
  for (int c = lane; c < 2 * N; c += 32) acc[c] = 0.f;
  __syncwarp();
  const int vpl = N >> 5;
  for (int64_t r = int64_t(blockIdx.x) * 8 + wib; r < M; r += int64_t(gridDim.x) * 8) {
    float v[kMaxVpl], dy[kMaxVpl];
    float s = 0.f;
    const int64_t r2 = dY2 ? (idx2 ? int64_t(idx2[r]) : r) : 0;
#pragma unroll
    for (int j = 0; j < kMaxVpl; ++j)
      if (j < vpl) {
        int c = lane + 32 * j;
        v[j] = Z[r * N + c];
        if (bias) v[j] += bias[c];
        dy[j] = dY1[r * N + c] + (dY2 ? dY2[r2 * N + c] : 0.f);
        s += v[j];
      }
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const float mu = s / N;
    float q = 0.f;
#pragma unroll
    for (int j = 0; j < kMaxVpl; ++j)
      if (j < vpl) {
        float d = v[j] - mu;
        q += d * d;
      }
    for (int o = 16; o; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    const float rstd = rsqrtf(q / N + kLnEps);
    float sg = 0.f, sgx = 0.f;
#pragma unroll
    for (int j = 0; j < kMaxVpl; ++j)
      if (j < vpl) {
        int c = lane + 32 * j;
        float xh = (v[j] - mu) * rstd;
        float g = dy[j] * gamma[c];
        v[j] = xh;
        sg += g;
        sgx += g * xh;
        acc[c] += dy[j] * xh;
        acc[N + c] += dy[j];
      }
    for (int o = 16; o; o >>= 1) {
      sg += __shfl_xor_sync(0xffffffffu, sg, o);
      sgx += __shfl_xor_sync(0xffffffffu, sgx, o);
    }
    sg /= N;
    sgx /= N;
#pragma unroll
    for (int j = 0; j < kMaxVpl; ++j)
      if (j < vpl) {
        int c = lane + 32 * j;
        dZ[r * N + c] = rstd * (dy[j] * gamma[c] - sg - v[j] * sgx);
      }
  }
  __syncthreads();
  float* P = part + int64_t(blockIdx.x) * 2 * N;
  for (int c = threadIdx.x; c < 2 * N; c += blockDim.x) {
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += ln_acc[w * 2 * N + c];
    P[c] = t;
  }
}

// out[c] = sum over b < nb of part[b * len + c], for c < len; columns at or
// past `split` go to out2[c - split] instead.  A block per 32 columns: warp w
// sums a contiguous run of the partials for its lane's column, and the eight
// warp sums are added in order (deterministic, and with 8 x 32 independent
// load streams per block where one thread per column would wait on one).
__global__ void __launch_bounds__(256) sum_parts_kernel(const float* __restrict__ part, int nb, int len,
                                                        float* __restrict__ out, int split, float* __restrict__ out2) {
  __shared__ float red[8][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int c = blockIdx.x * 32 + lane;
  const int per = (nb + 7) / 8, b0 = wib * per, b1 = min(nb, b0 + per);
  red[wib][lane] = (c < len && b1 > b0) ? sum_strided(part + int64_t(b0) * len + c, b1 - b0, len) : 0.f;
  __syncthreads();
  if (wib == 0 && c < len) {
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += red[w][lane];
    if (c < split) out[c] = t; else out2[c - split] = t;
  }
}

// Edge LayerNorm forward fused with the receiver sums of eq. (2): a warp per
// receiver node i walks its edge rows e in [rp[i], rp[i+1]) in order,
// y_e = LN(Z_e + bias) gamma + beta, resid_out_e = resid_in_e + y_e, and
// agg_i = the sum of y_e in edge order (the order of seg_rows_kernel).
__global__ void ln_fwd_agg_kernel(const float* __restrict__ Z, const float* __restrict__ bias,
                                  const int64_t* __restrict__ rp, int64_t n, int N, const float* __restrict__ gamma,
                                  const float* __restrict__ beta, const float* resid_in, float* resid_out,
                                  float* __restrict__ agg) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  const int vpl = N >> 5;
  for (int64_t i = warp; i < n; i += nw) {
    float a[kMaxVpl];
#pragma unroll
    for (int j = 0; j < kMaxVpl; ++j) a[j] = 0.f;
    const int64_t e1 = rp[i + 1];
    for (int64_t r = rp[i]; r < e1; ++r) {
      float v[kMaxVpl];
      float s = 0.f;
#pragma unroll
      for (int j = 0; j < kMaxVpl; ++j)
        if (j < vpl) {
          v[j] = Z[r * N + lane + 32 * j];
          if (bias) v[j] += bias[lane + 32 * j];
          s += v[j];
        }
      for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      const float mu = s / N;
      float q = 0.f;
#pragma unroll
      for (int j = 0; j < kMaxVpl; ++j)
        if (j < vpl) {
          float d = v[j] - mu;
          q += d * d;
        }
      for (int o = 16; o; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
      const float rstd = rsqrtf(q / N + kLnEps);
#pragma unroll
      for (int j = 0; j < kMaxVpl; ++j)
        if (j < vpl) {
          int c = lane + 32 * j;
          float y = (v[j] - mu) * rstd * gamma[c] + beta[c];
          resid_out[r * N + c] = resid_in[r * N + c] + y;
          a[j] += y;
        }
    }
#pragma unroll
    for (int j = 0; j < kMaxVpl; ++j)
      if (j < vpl) agg[i * N + lane + 32 * j] = a[j];
  }
}

// ---- vectorised LayerNorm rows for N = 128 V4 (V4 = 1, 2, 4): lane l owns
// the columns 128 t + 4 l .. 128 t + 4 l + 3 (t < V4), moved as float4; the
// row streams of a warp's next row are requested into L2 while it works on
// the current one, so a warp keeps two rows of loads in flight without
// holding the next row in registers.  Same formulas as the kernels above;
// only the order of the per-row sums differs.
__device__ __forceinline__ void pf_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
  for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

template <int V4>
__device__ __forceinline__ void pf_row(const float* row, int lane) {
#pragma unroll
  for (int t = 0; t < V4; ++t) pf_l2(row + 128 * t + 4 * lane);
}

// LayerNorm statistics of one row held as float4 per lane: mean and 1/std
template <int V4>
__device__ __forceinline__ void row_stats(const float4 (&v)[V4], float& mu, float& rstd) {
  constexpr int N = 128 * V4;
  float s = 0.f;
#pragma unroll
  for (int t = 0; t < V4; ++t) s += (v[t].x + v[t].y) + (v[t].z + v[t].w);
  mu = warp_sum(s) / N;
  float q = 0.f;
#pragma unroll
  for (int t = 0; t < V4; ++t) {
    const float a = v[t].x - mu, b = v[t].y - mu, c = v[t].z - mu, d = v[t].w - mu;
    q += (a * a + b * b) + (c * c + d * d);
  }
  rstd = rsqrtf(warp_sum(q) / N + kLnEps);
}

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float4 add4(float4 a, float4 b) { return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w); }
// column values of a parameter vector (scalar loads: parameter blocks need not be 16-byte aligned)
__device__ __forceinline__ float4 par4(const float* p, int c) { return make_float4(p[c], p[c + 1], p[c + 2], p[c + 3]); }

template <int V4>
__global__ void __launch_bounds__(256) ln_fwd_v4_kernel(const float* __restrict__ Z, const float* __restrict__ bias,
                                                        int64_t M, const float* __restrict__ gamma,
                                                        const float* __restrict__ beta, float* __restrict__ Y,
                                                        const float* resid_in, float* resid_out) {
  constexpr int N = 128 * V4;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t r = warp; r < M; r += nw) {
    if (r + nw < M) {
      pf_row<V4>(Z + (r + nw) * N, lane);
      if (resid_in) pf_row<V4>(resid_in + (r + nw) * N, lane);
    }
    float4 v[V4], ri[V4];
#pragma unroll
    for (int t = 0; t < V4; ++t) {
      const int c = 128 * t + 4 * lane;
      v[t] = ld4(Z + r * N + c);
      if (resid_out) ri[t] = ld4(resid_in + r * N + c);
      if (bias) v[t] = add4(v[t], par4(bias, c));
    }
    float mu, rstd;
    row_stats<V4>(v, mu, rstd);
#pragma unroll
    for (int t = 0; t < V4; ++t) {
      const int c = 128 * t + 4 * lane;
      const float4 g = par4(gamma, c), b = par4(beta, c);
      const float4 y = make_float4((v[t].x - mu) * rstd * g.x + b.x, (v[t].y - mu) * rstd * g.y + b.y,
                                   (v[t].z - mu) * rstd * g.z + b.z, (v[t].w - mu) * rstd * g.w + b.w);
      if (Y) st4(Y + r * N + c, y);
      if (resid_out) st4(resid_out + r * N + c, add4(ri[t], y));
    }
  }
}

template <int V4>
__global__ void __launch_bounds__(256) ln_fwd_agg_v4_kernel(const float* __restrict__ Z, const float* __restrict__ bias,
                                                            const int64_t* __restrict__ rp, int64_t n,
                                                            const float* __restrict__ gamma,
                                                            const float* __restrict__ beta, const float* resid_in,
                                                            float* resid_out, float* __restrict__ agg) {
  constexpr int N = 128 * V4;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t i = warp; i < n; i += nw) {
    float4 a[V4];
#pragma unroll
    for (int t = 0; t < V4; ++t) a[t] = make_float4(0.f, 0.f, 0.f, 0.f);
    const int64_t e1 = rp[i + 1];
    for (int64_t r = rp[i]; r < e1; ++r) {
      if (r + 1 < e1) {  // the node's next edge row
        pf_row<V4>(Z + (r + 1) * N, lane);
        pf_row<V4>(resid_in + (r + 1) * N, lane);
      }
      float4 v[V4], ri[V4];
#pragma unroll
      for (int t = 0; t < V4; ++t) {
        const int c = 128 * t + 4 * lane;
        v[t] = ld4(Z + r * N + c);
        ri[t] = ld4(resid_in + r * N + c);
        if (bias) v[t] = add4(v[t], par4(bias, c));
      }
      float mu, rstd;
      row_stats<V4>(v, mu, rstd);
#pragma unroll
      for (int t = 0; t < V4; ++t) {
        const int c = 128 * t + 4 * lane;
        const float4 g = par4(gamma, c), b = par4(beta, c);
        const float4 y = make_float4((v[t].x - mu) * rstd * g.x + b.x, (v[t].y - mu) * rstd * g.y + b.y,
                                     (v[t].z - mu) * rstd * g.z + b.z, (v[t].w - mu) * rstd * g.w + b.w);
        st4(resid_out + r * N + c, add4(ri[t], y));
        a[t] = add4(a[t], y);
      }
    }
#pragma unroll
    for (int t = 0; t < V4; ++t) st4(agg + i * N + 128 * t + 4 * lane, a[t]);
  }
}

template <int V4>
__global__ void __launch_bounds__(256, 3)
    ln_bwd_v4_kernel(const float* __restrict__ Z, const float* __restrict__ bias, int64_t M,
                     const float* __restrict__ gamma, const float* __restrict__ dY1, const float* __restrict__ dY2,
                     const int32_t* __restrict__ idx2, float* __restrict__ dZ, float* __restrict__ part) {
  constexpr int N = 128 * V4;
  extern __shared__ float ln_acc[];  // [8 warps][dgamma N | dbeta N]
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  float* acc = ln_acc + wib * 2 * N;
  for (int c = lane; c < 2 * N; c += 32) acc[c] = 0.f;
  __syncwarp();
  const int64_t stride = int64_t(gridDim.x) * 8;
  auto gather_row = [&](int64_t q) -> int64_t { return (dY2 && q < M) ? (idx2 ? int64_t(idx2[q]) : q) : 0; };
  int64_t r = int64_t(blockIdx.x) * 8 + wib;
  int64_t r2 = gather_row(r), r2n = gather_row(r + stride);
  for (; r < M; r += stride) {
    const int64_t rn = r + stride;
    // the gather index two rows ahead (used one row from now, so its load is not waited for here)
    const int64_t r2nn = gather_row(rn + stride);
    if (rn < M) {  // the warp's next row towards L2
      pf_row<V4>(Z + rn * N, lane);
      pf_row<V4>(dY1 + rn * N, lane);
      if (dY2) pf_row<V4>(dY2 + r2n * N, lane);
    }
    float4 v[V4], dy[V4];
#pragma unroll
    for (int t = 0; t < V4; ++t) {
      const int c = 128 * t + 4 * lane;
      v[t] = ld4(Z + r * N + c);
      dy[t] = ld4(dY1 + r * N + c);
      if (dY2) dy[t] = add4(dy[t], ld4(dY2 + r2 * N + c));
      if (bias) v[t] = add4(v[t], par4(bias, c));
    }
    float mu, rstd;
    row_stats<V4>(v, mu, rstd);
    float sg = 0.f, sgx = 0.f;
#pragma unroll
    for (int t = 0; t < V4; ++t) {
      const int c = 128 * t + 4 * lane;
      const float4 g4 = par4(gamma, c);
      v[t] = make_float4((v[t].x - mu) * rstd, (v[t].y - mu) * rstd, (v[t].z - mu) * rstd, (v[t].w - mu) * rstd);
      const float4 g = make_float4(dy[t].x * g4.x, dy[t].y * g4.y, dy[t].z * g4.z, dy[t].w * g4.w);
      sg += (g.x + g.y) + (g.z + g.w);
      sgx += (g.x * v[t].x + g.y * v[t].y) + (g.z * v[t].z + g.w * v[t].w);
      float4 ag = *reinterpret_cast<float4*>(acc + c), ab = *reinterpret_cast<float4*>(acc + N + c);
      ag = make_float4(ag.x + dy[t].x * v[t].x, ag.y + dy[t].y * v[t].y, ag.z + dy[t].z * v[t].z,
                       ag.w + dy[t].w * v[t].w);
      *reinterpret_cast<float4*>(acc + c) = ag;
      *reinterpret_cast<float4*>(acc + N + c) = add4(ab, dy[t]);
    }
    sg = warp_sum(sg) / N;
    sgx = warp_sum(sgx) / N;
#pragma unroll
    for (int t = 0; t < V4; ++t) {
      const int c = 128 * t + 4 * lane;
      const float4 g4 = par4(gamma, c);
      st4(dZ + r * N + c, make_float4(rstd * (dy[t].x * g4.x - sg - v[t].x * sgx),
                                      rstd * (dy[t].y * g4.y - sg - v[t].y * sgx),
                                      rstd * (dy[t].z * g4.z - sg - v[t].z * sgx),
                                      rstd * (dy[t].w * g4.w - sg - v[t].w * sgx)));
    }
    r2 = r2n;
    r2n = r2nn;
  }
  __syncthreads();
  float* P = part + int64_t(blockIdx.x) * 2 * N;
  for (int c = threadIdx.x; c < 2 * N; c += blockDim.x) {
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += ln_acc[w * 2 * N + c];
    P[c] = t;
  }
}

// Receiver / sender sums with four columns per lane (H % 4 == 0, H <= 512,
// 16-byte aligned rows): the node's rows are walked once, each row's lane
// slots loaded together; the sum of each column runs in edge order as in the
// scalar kernels below.
template <bool PERM>
__global__ void seg_sum_v4_kernel(const float* __restrict__ v, int64_t ldv, const int64_t* __restrict__ rp,
                                  const int32_t* __restrict__ perm, int64_t n, int H, float* __restrict__ out,
                                  int64_t ldo, int acc) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t i = warp; i < n; i += nw) {
    const int64_t e0 = rp[i], e1 = rp[i + 1];
    float4 a[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) a[t] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int64_t e = e0; e < e1; ++e) {
      const float* row = v + (PERM ? int64_t(perm[e]) : e) * ldv;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int c = 4 * lane + 128 * t;
        if (c < H) a[t] = add4(a[t], ld4(row + c));
      }
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int c = 4 * lane + 128 * t;
      if (c < H) {
        float* d = out + i * ldo + c;
        st4(d, acc ? add4(ld4(d), a[t]) : a[t]);
      }
    }
  }
}

__global__ void seg_rows_kernel(const float* __restrict__ v, int64_t ldv, const int64_t* __restrict__ rp,
                                int64_t n, int H, float* __restrict__ out, int64_t ldo, int acc) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t i = warp; i < n; i += nw) {
    const int64_t e0 = rp[i], e1 = rp[i + 1];
    for (int c = lane; c < H; c += 32) {
      float s = 0.f;
      for (int64_t e = e0; e < e1; ++e) s += v[e * ldv + c];
      if (acc) out[i * ldo + c] += s; else out[i * ldo + c] = s;
    }
  }
}

__global__ void seg_cols_kernel(const float* __restrict__ v, int64_t ldv, const int64_t* __restrict__ rp,
                                const int32_t* __restrict__ perm, int64_t n, int H,
                                float* __restrict__ out, int64_t ldo, int acc) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t i = warp; i < n; i += nw) {
    const int64_t t0 = rp[i], t1 = rp[i + 1];
    for (int c = lane; c < H; c += 32) {
      float s = 0.f;
      for (int64_t t = t0; t < t1; ++t) s += v[int64_t(perm[t]) * ldv + c];
      if (acc) out[i * ldo + c] += s; else out[i * ldo + c] = s;
    }
  }
}

__global__ void edge_feat_kernel(const float* __restrict__ xyz, const int32_t* __restrict__ gid,
                                 const int32_t* __restrict__ recv, const int32_t* __restrict__ col,
                                 int64_t E, float* __restrict__ f) {
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < E;
       e += int64_t(gridDim.x) * blockDim.x) {
    int64_t r = recv[e], s = col[e];
    if (gid) {
      r = gid[r];
      s = gid[s];
    }
    float dx = xyz[3 * s] - xyz[3 * r];
    float dy = xyz[3 * s + 1] - xyz[3 * r + 1];
    float dz = xyz[3 * s + 2] - xyz[3 * r + 2];
    f[4 * e] = dx;
    f[4 * e + 1] = dy;
    f[4 * e + 2] = dz;
    f[4 * e + 3] = sqrtf(dx * dx + dy * dy + dz * dz);
  }
}

constexpr int kLossBlocks = 256;

__global__ void loss_kernel(const float* __restrict__ y, int64_t n, int out,
                            const float* __restrict__ t, const int32_t* __restrict__ gid,
                            const uint8_t* __restrict__ hop, float scale, float* __restrict__ dy,
                            float* __restrict__ yg, float* __restrict__ part) {
  __shared__ float red[256];
  float s = 0.f;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x) {
    const bool inner = !hop || hop[i] == 0;
    const int64_t g = gid ? int64_t(gid[i]) : i;
    for (int c = 0; c < out; ++c) {
      float yv = y[i * out + c];
      float d = 0.f;
      if (inner) {
        if (t) d = yv - t[g * out + c];
        if (yg) yg[g * out + c] = yv;
      }
      s += d * d;
      if (dy) dy[i * out + c] = 2.f * d * scale;
    }
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void loss_reduce_kernel(const float* __restrict__ part, int nb, float scale, float* loss) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    float s = 0.f;
    for (int b = 0; b < nb; ++b) s += part[b];
    *loss = s * scale;
  }
}

__global__ void accum_kernel(float* __restrict__ dst, float* __restrict__ comp,
                             const float* __restrict__ src, int64_t n) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x) {
    float x = src[i];
    if (!comp) {
      dst[i] += x;
      continue;
    }
    float s = dst[i];
    float t = s + x;
    float c = fabsf(s) >= fabsf(x) ? (s - t) + x : (x - t) + s;
    comp[i] += c;
    dst[i] = t;
  }
}

}  // namespace

xmgn_status gemm_nn_f32(const RowSrc& A, int64_t M, const float* B, int N, const float* bias,
                        float* C, int64_t ldc, int epi, float* pre, const float* aux,
                        cudaStream_t s) {
  if (M <= 0) return XMGN_OK;
  dim3 grid(unsigned((M + BT - 1) / BT), unsigned((N + BT - 1) / BT));
  gemm_nnt_kernel<false><<<grid, 256, 0, s>>>(A, M, B, N, bias, C, ldc, epi, pre, aux);
  XMGN_LAUNCH_CHECK();
  return XMGN_OK;
}

xmgn_status gemm_nt_f32(const RowSrc& A, int64_t M, const float* B, int N, float* C, int64_t ldc,
                        int epi, const float* aux, cudaStream_t s) {
  if (M <= 0) return XMGN_OK;
  dim3 grid(unsigned((M + BT - 1) / BT), unsigned((N + BT - 1) / BT));
  gemm_nnt_kernel<true><<<grid, 256, 0, s>>>(A, M, B, N, nullptr, C, ldc, epi, nullptr, aux);
  XMGN_LAUNCH_CHECK();
  return XMGN_OK;
}

size_t gemm_tn_part_elems(int64_t M, int K1, int N) {
  return size_t(tn_chunks(M)) * size_t(K1) * size_t(N);
}

xmgn_status gemm_tn_f32(const RowSrc& A, int64_t M, const float* B, int64_t ldb, int N, float* G,
                        float* part, cudaStream_t s) {
  const int K1 = A.K;
  const int nc = tn_chunks(M);
  int64_t rpc = (M + nc - 1) / nc;
  rpc = (rpc + BK - 1) / BK * BK;
  if (rpc < BK) rpc = BK;
  const int tiles = ((K1 + BT - 1) / BT) * ((N + BT - 1) / BT);
  gemm_tn_kernel<<<dim3(tiles, nc), 256, 0, s>>>(A, M, B, ldb, N, rpc, part);
  XMGN_LAUNCH_CHECK();
  const int64_t len = int64_t(K1) * N;
  reduce_chunks_kernel<<<grid_for(len, 256), 256, 0, s>>>(part, nc, len, G);
  XMGN_LAUNCH_CHECK();
  return XMGN_OK;
}

size_t colsum_part_elems(int64_t M, int N) { return size_t(colsum_chunks(M)) * size_t(N); }

xmgn_status colsum_f32(const float* X, int64_t M, int N, int64_t ld, float* g, float* part,
                       cudaStream_t s) {
  const int nc = colsum_chunks(M);
  int64_t rpc = (M + nc - 1) / nc;
  if (rpc < 1) rpc = 1;
  colsum_kernel<<<nc, 256, 0, s>>>(X, M, N, ld, rpc, part);
  XMGN_LAUNCH_CHECK();
  sum_parts_kernel<<<(N + 31) / 32, 256, 0, s>>>(part, nc, N, g, N, nullptr);
  XMGN_LAUNCH_CHECK();
  return XMGN_OK;
}

// Whether the vectorised LayerNorm kernels apply: N in {128, 256, 512} and
// every row array (null ones aside) 16-byte aligned.
bool rows_vec4(int N, std::initializer_list<const float*> rows) {
  if (N != 128 && N != 256 && N != 512) return false;
  for (const float* p : rows)
    if (p && (reinterpret_cast<uintptr_t>(p) & 15)) return false;
  return true;
}

xmgn_status layernorm_fwd_f32(const float* Z, int64_t M, int N, const float* gamma,
                              const float* beta, float* Y, const float* resid_in,
                              float* resid_out, cudaStream_t s, const float* bias) {
  if (N % 32 || N > 32 * kMaxVpl) return fail(XMGN_ERR_UNSUPPORTED, "LayerNorm width %d", N);
  if (M <= 0) return XMGN_OK;
  const unsigned grid = grid_for(M * 32, 256, int64_t(num_sms()) * 16);
  if (rows_vec4(N, {Z, Y, resid_in, resid_out})) {
    if (N == 128) ln_fwd_v4_kernel<1><<<grid, 256, 0, s>>>(Z, bias, M, gamma, beta, Y, resid_in, resid_out);
    if (N == 256) ln_fwd_v4_kernel<2><<<grid, 256, 0, s>>>(Z, bias, M, gamma, beta, Y, resid_in, resid_out);
    if (N == 512) ln_fwd_v4_kernel<4><<<grid, 256, 0, s>>>(Z, bias, M, gamma, beta, Y, resid_in, resid_out);
    XMGN_LAUNCH_CHECK();
    return XMGN_OK;
  }
  ln_fwd_kernel<<<grid, 256, 0, s>>>(Z, bias, M, N, gamma, beta, Y, resid_in, resid_out);
  XMGN_LAUNCH_CHECK();
  return XMGN_OK;
}

xmgn_status layernorm_fwd_agg_f32(const float* Z, const float* bias, const int64_t* row_ptr, int64_t n, int N,
                                  const float* gamma, const float* beta, const float* resid_in, float* resid_out,
                                  float* agg, cudaStream_t s) {
  if (N % 32 || N > 32 * kMaxVpl) return fail(XMGN_ERR_UNSUPPORTED, "LayerNorm width %d", N);
  if (n <= 0) return XMGN_OK;
  const unsigned grid = grid_for(n * 32, 256, int64_t(num_sms()) * 16);
  if (rows_vec4(N, {Z, resid_in, resid_out, agg})) {
    if (N == 128) ln_fwd_agg_v4_kernel<1><<<grid, 256, 0, s>>>(Z, bias, row_ptr, n, gamma, beta, resid_in, resid_out, agg);
    if (N == 256) ln_fwd_agg_v4_kernel<2><<<grid, 256, 0, s>>>(Z, bias, row_ptr, n, gamma, beta, resid_in, resid_out, agg);
    if (N == 512) ln_fwd_agg_v4_kernel<4><<<grid, 256, 0, s>>>(Z, bias, row_ptr, n, gamma, beta, resid_in, resid_out, agg);
    XMGN_LAUNCH_CHECK();
    return XMGN_OK;
  }
  ln_fwd_agg_kernel<<<grid, 256, 0, s>>>(Z, bias, row_ptr, n, N, gamma, beta, resid_in, resid_out, agg);
  XMGN_LAUNCH_CHECK();
  return XMGN_OK;
}

int colsum_chunk_count(int64_t M) { return colsum_chunks(M); }

xmgn_status sum_parts_f32(const float* part, int nb, int len, float* out, cudaStream_t s) {
  if (len <= 0) return XMGN_OK;
  sum_parts_kernel<<<(len + 31) / 32, 256, 0, s>>>(part, nb, len, out, len, nullptr);
  XMGN_LAUNCH_CHECK();
  return XMGN_OK;
}

size_t ln_bwd_part_elems(int N) { return size_t(kLnBlocksMax) * 2 * size_t(N); }

xmgn_status layernorm_bwd_f32(const float* Z, int64_t M, int N, const float* gamma,
                              const float* dY1, const float* dY2, const int32_t* idx2, float* dZ,
                              float* dgamma, float* dbeta, float* part, cudaStream_t s, const float* bias) {
  if (N % 32 || N > 32 * kMaxVpl) return fail(XMGN_ERR_UNSUPPORTED, "LayerNorm width %d", N);
  // three blocks of eight warps per SM, at most one row per warp
  int64_t nb = int64_t(num_sms()) * 3;
  if (nb > kLnBlocksMax) nb = kLnBlocksMax;
  if (nb > (M + 7) / 8) nb = (M + 7) / 8;
  if (nb < 1) nb = 1;
  const size_t sh = size_t(8) * 2 * N * sizeof(float);
  if (rows_vec4(N, {Z, dY1, dY2, dZ})) {
    if (N == 128) ln_bwd_v4_kernel<1><<<unsigned(nb), 256, sh, s>>>(Z, bias, M, gamma, dY1, dY2, idx2, dZ, part);
    if (N == 256) ln_bwd_v4_kernel<2><<<unsigned(nb), 256, sh, s>>>(Z, bias, M, gamma, dY1, dY2, idx2, dZ, part);
    if (N == 512) ln_bwd_v4_kernel<4><<<unsigned(nb), 256, sh, s>>>(Z, bias, M, gamma, dY1, dY2, idx2, dZ, part);
  } else {
    ln_bwd_kernel<<<unsigned(nb), 256, sh, s>>>(Z, bias, M, N, gamma, dY1, dY2, idx2, dZ, part);
  }
  XMGN_LAUNCH_CHECK();
  sum_parts_kernel<<<(2 * N + 31) / 32, 256, 0, s>>>(part, int(nb), 2 * N, dgamma, N, dbeta);
  XMGN_LAUNCH_CHECK();
  return XMGN_OK;
}

// Whether the four-columns-per-lane segment sums apply.
bool seg_vec4(const float* v, int64_t ldv, int H, const float* out, int64_t ldo) {
  return H % 4 == 0 && H <= 512 && ldv % 4 == 0 && ldo % 4 == 0 && (reinterpret_cast<uintptr_t>(v) & 15) == 0 &&
         (reinterpret_cast<uintptr_t>(out) & 15) == 0;
}

xmgn_status seg_sum_rows_f32(const float* v, int64_t ldv, const int64_t* row_ptr, int64_t n, int H,
                             float* out, int64_t ldo, bool accumulate, cudaStream_t s) {
  if (n <= 0) return XMGN_OK;
  const unsigned grid = grid_for(n * 32, 256, int64_t(num_sms()) * 16);
  if (seg_vec4(v, ldv, H, out, ldo))
    seg_sum_v4_kernel<false><<<grid, 256, 0, s>>>(v, ldv, row_ptr, nullptr, n, H, out, ldo, accumulate ? 1 : 0);
  else
    seg_rows_kernel<<<grid, 256, 0, s>>>(v, ldv, row_ptr, n, H, out, ldo, accumulate ? 1 : 0);
  XMGN_LAUNCH_CHECK();
  return XMGN_OK;
}

xmgn_status seg_sum_cols_f32(const float* v, int64_t ldv, const int64_t* row_ptr,
                             const int32_t* perm, int64_t n, int H, float* out, int64_t ldo,
                             bool accumulate, cudaStream_t s) {
  if (n <= 0) return XMGN_OK;
  const unsigned grid = grid_for(n * 32, 256, int64_t(num_sms()) * 16);
  if (seg_vec4(v, ldv, H, out, ldo))
    seg_sum_v4_kernel<true><<<grid, 256, 0, s>>>(v, ldv, row_ptr, perm, n, H, out, ldo, accumulate ? 1 : 0);
  else
    seg_cols_kernel<<<grid, 256, 0, s>>>(v, ldv, row_ptr, perm, n, H, out, ldo, accumulate ? 1 : 0);
  XMGN_LAUNCH_CHECK();
  return XMGN_OK;
}

namespace {
// Node-encoder inputs: the node_in row, then for q < F: sin and cos of
// 2^(q+1) pi x_c for the three coordinates (sines first).
__global__ void node_feat_kernel(const float* __restrict__ node_in, int in_node, const float* __restrict__ xyz,
                                 const int32_t* __restrict__ gid, int64_t n, int F, float* __restrict__ out) {
  const int w = in_node + 6 * F;
  for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < n;
       r += int64_t(gridDim.x) * blockDim.x) {
    const int64_t g = gid ? int64_t(gid[r]) : r;
    for (int j = 0; j < in_node; ++j) out[r * w + j] = node_in[g * in_node + j];
    for (int q = 0; q < F; ++q) {
      const float fr = float(2 << q);
      for (int c = 0; c < 3; ++c) {
        float sv, cv;
        sincospif(fr * xyz[3 * g + c], &sv, &cv);
        out[r * w + in_node + 6 * q + c] = sv;
        out[r * w + in_node + 6 * q + 3 + c] = cv;
      }
    }
  }
}
}  // namespace

xmgn_status node_features(const float* node_in, int in_node, const float* xyz, const int32_t* gid, int64_t n,
                          int fourier, float* out, cudaStream_t s) {
  node_feat_kernel<<<grid_for(n, 256), 256, 0, s>>>(node_in, in_node, xyz, gid, n, fourier, out);
  XMGN_LAUNCH_CHECK();
  return XMGN_OK;
}

xmgn_status edge_features(const float* xyz, const int32_t* gid, const int32_t* recv,
                          const int32_t* col, int64_t E, float* f, cudaStream_t s) {
  if (E <= 0) return XMGN_OK;
  edge_feat_kernel<<<grid_for(E, 256), 256, 0, s>>>(xyz, gid, recv, col, E, f);
  XMGN_LAUNCH_CHECK();
  return XMGN_OK;
}

size_t loss_part_elems(int64_t) { return kLossBlocks; }

xmgn_status mse_loss(const float* y, int64_t n, int out, const float* targets, const int32_t* gid,
                     const uint8_t* hop, int64_t n_norm, float* loss, float* dy, float* y_global,
                     float* part, cudaStream_t s) {
  const float scale = 1.f / (float(out) * float(n_norm));
  loss_kernel<<<kLossBlocks, 256, 0, s>>>(y, n, out, targets, gid, hop, scale, dy, y_global, part);
  XMGN_LAUNCH_CHECK();
  if (loss) {
    loss_reduce_kernel<<<1, 32, 0, s>>>(part, kLossBlocks, scale, loss);
    XMGN_LAUNCH_CHECK();
  }
  return XMGN_OK;
}

xmgn_status accumulate_grad(float* dst, float* comp, const float* src, int64_t n, cudaStream_t s) {
  accum_kernel<<<grid_for(n, 256), 256, 0, s>>>(dst, comp, src, n);
  XMGN_LAUNCH_CHECK();
  return XMGN_OK;
}

}  // namespace xmgn
