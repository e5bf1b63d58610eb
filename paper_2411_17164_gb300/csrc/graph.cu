// kNN graph construction (Sec. III-B "K-Nearest Neighbor Connectivity") and
// symmetrisation into receiver-major CSR.
//
// Exactness: coordinates are mapped to the integer lattice q = rint(x*s) with
// s a power of two, so x*s is exact in float32 and rintf gives the same
// round-half-even result as any exact reference; squared distances are int64.
// Candidates are ranked by (d^2, index), so the result is unique and
// independent of thread scheduling.
//
// Search: uniform grid over the lattice bounding box, points counting-sorted
// into cells, then for each point rings of cells at Chebyshev distance
// r = 0, 1, 2, ... are scanned.  Any point outside rings 0..r differs by at
// least r*c + 1 lattice units along some axis (c = cell edge), so the search
// stops once the k-th best d^2 < (r*c + 1)^2.
#include <math.h>

#include "common.cuh"

namespace xmgn {

namespace {
constexpr int kMaxK = 32;

__global__ void quantize_kernel(const float* __restrict__ xyz, int64_t n, float scale,
                                int32_t* __restrict__ q, int32_t* __restrict__ bbox,
                                uint32_t* err) {
  int lo[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, hi[3] = {INT32_MIN, INT32_MIN, INT32_MIN};
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float v = rintf(xyz[3 * i + a] * scale);  // exact product (power-of-two scale)
      int32_t qi = 0;
      if (!(fabsf(v) < 16777216.0f)) {  // also catches NaN / inf
        dev_flag(err, DEV_ERR_RANGE);
      } else {
        qi = int32_t(v);
      }
      q[3 * i + a] = qi;
      lo[a] = min(lo[a], qi);
      hi[a] = max(hi[a], qi);
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    for (int o = 16; o; o >>= 1) {
      lo[a] = min(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
      hi[a] = max(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
    }
  }
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      atomicMin(&bbox[a], lo[a]);
      atomicMax(&bbox[3 + a], hi[a]);
    }
  }
}

__global__ void bbox_init_kernel(int32_t* bbox) {
  if (threadIdx.x < 3) {
    bbox[threadIdx.x] = INT32_MAX;
    bbox[3 + threadIdx.x] = INT32_MIN;
  }
}

struct Grid {
  int32_t lo[3];
  int64_t c;      // cell edge in lattice units
  int64_t g[3];   // cells per axis
};

__device__ __forceinline__ int64_t cell_coord(int32_t q, int32_t lo, int64_t c) {
  return (int64_t(q) - lo) / c;
}

__global__ void cell_count_kernel(const int32_t* __restrict__ q, int64_t n, Grid G,
                                  int64_t* __restrict__ cell_of, int32_t* __restrict__ cnt) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x) {
    int64_t cx = cell_coord(q[3 * i], G.lo[0], G.c);
    int64_t cy = cell_coord(q[3 * i + 1], G.lo[1], G.c);
    int64_t cz = cell_coord(q[3 * i + 2], G.lo[2], G.c);
    int64_t cell = (cz * G.g[1] + cy) * G.g[0] + cx;
    cell_of[i] = cell;
    atomicAdd(&cnt[cell], 1);
  }
}

__global__ void cell_scatter_kernel(const int64_t* __restrict__ cell_of, int64_t n,
                                    const int64_t* __restrict__ start, int32_t* __restrict__ fill,
                                    int32_t* __restrict__ sorted) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x) {
    int64_t c = cell_of[i];
    int32_t off = atomicAdd(&fill[c], 1);
    sorted[start[c] + off] = int32_t(i);
  }
}

__device__ __forceinline__ bool key_less(int64_t d1, int32_t j1, int64_t d2, int32_t j2) {
  return d1 < d2 || (d1 == d2 && j1 < j2);
}

__global__ void knn_search_kernel(const int32_t* __restrict__ q, const int32_t* __restrict__ sorted,
                                  const int64_t* __restrict__ start, int64_t n, int k, Grid G,
                                  int32_t* __restrict__ nbr) {
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int32_t i = sorted[t];
    const int64_t px = q[3 * i], py = q[3 * i + 1], pz = q[3 * i + 2];
    const int64_t cx = (px - G.lo[0]) / G.c, cy = (py - G.lo[1]) / G.c, cz = (pz - G.lo[2]) / G.c;
    int64_t bd[kMaxK];
    int32_t bj[kMaxK];
    int have = 0;
    const int64_t rmax = max(G.g[0], max(G.g[1], G.g[2]));
    for (int64_t r = 0; r <= rmax; ++r) {
      for (int64_t dz = -r; dz <= r; ++dz) {
        int64_t z = cz + dz;
        if (z < 0 || z >= G.g[2]) continue;
        for (int64_t dy = -r; dy <= r; ++dy) {
          int64_t y = cy + dy;
          if (y < 0 || y >= G.g[1]) continue;
          bool face = (dz == -r || dz == r || dy == -r || dy == r);
          int64_t step = face ? 1 : 2 * r;  // interior rows only touch the two x faces
          for (int64_t dx = -r; dx <= r; dx += (step > 0 ? step : 1)) {
            int64_t x = cx + dx;
            if (x < 0 || x >= G.g[0]) continue;
            int64_t cell = (z * G.g[1] + y) * G.g[0] + x;
            for (int64_t s = start[cell], e = start[cell + 1]; s < e; ++s) {
              int32_t j = sorted[s];
              if (j == i) continue;
              int64_t ddx = q[3 * j] - px, ddy = q[3 * j + 1] - py, ddz = q[3 * j + 2] - pz;
              int64_t d = ddx * ddx + ddy * ddy + ddz * ddz;
              if (have == k && !key_less(d, j, bd[k - 1], bj[k - 1])) continue;
              int pos = have < k ? have : k - 1;
              while (pos > 0 && key_less(d, j, bd[pos - 1], bj[pos - 1])) {
                bd[pos] = bd[pos - 1];
                bj[pos] = bj[pos - 1];
                --pos;
              }
              bd[pos] = d;
              bj[pos] = j;
              if (have < k) ++have;
            }
          }
        }
      }
      if (have == k) {
        int64_t lim = r * G.c + 1;
        if (bd[k - 1] < lim * lim) break;
      }
    }
    for (int a = 0; a < k; ++a) nbr[int64_t(i) * k + a] = a < have ? bj[a] : -1;
  }
}

// ---- symmetrisation
__global__ void sym_count_kernel(const int32_t* __restrict__ nbr, int64_t n, int k,
                                 int32_t* __restrict__ cnt, uint32_t* err) {
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n * k;
       t += int64_t(gridDim.x) * blockDim.x) {
    int32_t j = nbr[t];
    if (j < 0 || j >= n) {
      dev_flag(err, DEV_ERR_GRAPH);
      continue;
    }
    atomicAdd(&cnt[j], 1);
  }
}

__global__ void sym_own_kernel(const int32_t* __restrict__ nbr, int64_t n, int k,
                               const int64_t* __restrict__ cstart, int32_t* __restrict__ cand,
                               unsigned long long* __restrict__ fill) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x) {
    for (int a = 0; a < k; ++a) cand[cstart[i] + a] = nbr[i * k + a];
    fill[i] = (unsigned long long)(cstart[i] + k);
  }
}

__global__ void sym_rev_kernel(const int32_t* __restrict__ nbr, int64_t n, int k,
                               int32_t* __restrict__ cand, unsigned long long* __restrict__ fill) {
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n * k;
       t += int64_t(gridDim.x) * blockDim.x) {
    int32_t j = nbr[t];
    if (j < 0 || j >= n) continue;
    unsigned long long pos = atomicAdd(&fill[j], 1ull);
    cand[pos] = int32_t(t / k);
  }
}

__global__ void sym_sort_kernel(int32_t* __restrict__ cand, const int64_t* __restrict__ cstart,
                                int64_t n, int32_t* __restrict__ deg) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x) {
    int32_t* c = cand + cstart[i];
    int64_t m = cstart[i + 1] - cstart[i];
    for (int64_t a = 1; a < m; ++a) {  // insertion sort (rows are short)
      int32_t v = c[a];
      int64_t b = a - 1;
      while (b >= 0 && c[b] > v) {
        c[b + 1] = c[b];
        --b;
      }
      c[b + 1] = v;
    }
    int32_t u = 0;
    for (int64_t a = 0; a < m; ++a)
      if (c[a] != int32_t(i) && (a == 0 || c[a] != c[a - 1])) ++u;
    deg[i] = u;
  }
}

__global__ void sym_emit_kernel(const int32_t* __restrict__ cand, const int64_t* __restrict__ cstart,
                                const int64_t* __restrict__ row_ptr, int64_t n,
                                int32_t* __restrict__ col, int32_t* __restrict__ recv) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x) {
    const int32_t* c = cand + cstart[i];
    int64_t m = cstart[i + 1] - cstart[i];
    int64_t o = row_ptr[i];
    for (int64_t a = 0; a < m; ++a) {
      if (c[a] != int32_t(i) && (a == 0 || c[a] != c[a - 1])) {
        col[o] = c[a];
        if (recv) recv[o] = int32_t(i);
        ++o;
      }
    }
  }
}

__global__ void add_ramp_kernel(int64_t* cs, int64_t n, int k) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i <= n;
       i += int64_t(gridDim.x) * blockDim.x)
    cs[i] += int64_t(k) * i;
}

}  // namespace

xmgn_status quantize_launch(const float* xyz, int64_t n, double scale, int32_t* q, int32_t* bbox,
                            uint32_t* err, cudaStream_t s) {
  bbox_init_kernel<<<1, 32, 0, s>>>(bbox);
  XMGN_LAUNCH_CHECK();
  quantize_kernel<<<grid_for(n, 256), 256, 0, s>>>(xyz, n, float(scale), q, bbox, err);
  XMGN_LAUNCH_CHECK();
  return XMGN_OK;
}

// Edge p = (j <- r) at row j; csc_perm[p] = CSR position of the reverse edge
// (r <- j).  Shared by the kNN builder and the partitioner.
__global__ void csc_perm_kernel(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                const int32_t* __restrict__ recv, const int32_t* __restrict__ key,
                                int64_t n, int64_t e, int32_t* __restrict__ perm, uint32_t* err) {
  for (int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < e;
       p += int64_t(gridDim.x) * blockDim.x) {
    int32_t j = recv[p], r = col[p];
    if (r < 0 || r >= n || j < 0 || j >= n) {
      dev_flag(err, DEV_ERR_GRAPH);
      perm[p] = 0;
      continue;
    }
    // rows are sorted by key[] of their senders (key = identity or global id)
    int32_t want = key ? key[j] : j;
    int64_t lo = row_ptr[r], hi = row_ptr[r + 1];
    while (lo < hi) {
      int64_t mid = (lo + hi) >> 1;
      int32_t v = key ? key[col[mid]] : col[mid];
      if (v < want) lo = mid + 1; else hi = mid;
    }
    if (lo >= row_ptr[r + 1] || col[lo] != j) {
      dev_flag(err, DEV_ERR_GRAPH);
      perm[p] = 0;
      continue;
    }
    perm[p] = int32_t(lo);
  }
}

static xmgn_status knn_layout(int64_t N, int32_t k, Arena& A, int32_t** q, int32_t** bbox,
                              int64_t** cell_of, int32_t** sorted, int32_t** nbr_tmp,
                              int32_t** cnt, int64_t** cstart, int32_t** cand,
                              unsigned long long** fill, int32_t** deg, int64_t** scan_tmp,
                              int64_t max_cells) {
  *q = A.take<int32_t>(size_t(3 * N));
  *bbox = A.take<int32_t>(8);
  *cell_of = A.take<int64_t>(size_t(N));
  *sorted = A.take<int32_t>(size_t(N));
  *nbr_tmp = A.take<int32_t>(size_t(N * k));
  int64_t cnt_n = max_cells > N ? max_cells : N;
  *cnt = A.take<int32_t>(size_t(cnt_n + 1));
  *cstart = A.take<int64_t>(size_t(cnt_n + 1));
  *cand = A.take<int32_t>(size_t(2 * N * k));
  *fill = A.take<unsigned long long>(size_t(N));
  *deg = A.take<int32_t>(size_t(N));
  *scan_tmp = A.take<int64_t>(scan_tmp_elems(cnt_n + 1) + 16);
  return XMGN_OK;
}

static int64_t knn_max_cells(int64_t N) { return 2 * N + 1024; }

xmgn_status build_knn_ws(int64_t N, int32_t k, size_t* ws_bytes) {
  Arena A;
  A.dry = true;
  int32_t *q, *bbox, *sorted, *nbr_tmp, *cnt, *cand, *deg;
  int64_t *cell_of, *cstart, *scan_tmp;
  unsigned long long* fill;
  knn_layout(N, k, A, &q, &bbox, &cell_of, &sorted, &nbr_tmp, &cnt, &cstart, &cand, &fill, &deg,
             &scan_tmp, knn_max_cells(N));
  *ws_bytes = A.used + 256;
  return XMGN_OK;
}

xmgn_status build_knn(const float* xyz, int64_t N, int32_t k, double scale, void* ws,
                      size_t ws_bytes, int32_t* nbr_out, int64_t* row_ptr, int32_t* col,
                      int32_t* recv, int32_t* csc_perm, int64_t E_cap, int64_t* E_out,
                      cudaStream_t s) {
  if (!xyz || !row_ptr || !col || !E_out || !ws) return fail(XMGN_ERR_ARG, "null pointer");
  if (k < 1 || k > kMaxK) return fail(XMGN_ERR_ARG, "k must be in [1, %d]", kMaxK);
  if (N < int64_t(k) + 1) return fail(XMGN_ERR_ARG, "need N >= k+1 (N=%lld, k=%d)", (long long)N, k);
  if (N >= (int64_t(1) << 31)) return fail(XMGN_ERR_ARG, "N must be < 2^31");
  int ex = 0;
  double fr = frexp(scale, &ex);
  if (!(scale > 0) || fr != 0.5) return fail(XMGN_ERR_ARG, "lattice_scale must be a power of two");
  if (csc_perm && !recv) return fail(XMGN_ERR_ARG, "csc_perm requires recv");

  Arena A;
  A.base = static_cast<char*>(ws);
  A.cap = ws_bytes;
  int32_t *q, *bbox, *sorted, *nbr_tmp, *cnt, *cand, *deg;
  int64_t *cell_of, *cstart, *scan_tmp;
  unsigned long long* fill;
  const int64_t max_cells = knn_max_cells(N);
  knn_layout(N, k, A, &q, &bbox, &cell_of, &sorted, &nbr_tmp, &cnt, &cstart, &cand, &fill, &deg,
             &scan_tmp, max_cells);
  if (!A.ok()) return fail(XMGN_ERR_WORKSPACE, "knn workspace too small: need %zu", A.used);
  uint32_t* err = device_error_word();
  int32_t* nbr = nbr_out ? nbr_out : nbr_tmp;

  bbox_init_kernel<<<1, 32, 0, s>>>(bbox);
  XMGN_LAUNCH_CHECK();
  quantize_kernel<<<grid_for(N, 256), 256, 0, s>>>(xyz, N, float(scale), q, bbox, err);
  XMGN_LAUNCH_CHECK();
  int32_t hb[6];
  uint32_t herr = 0;
  XMGN_CUDA(cudaMemcpyAsync(hb, bbox, sizeof(hb), cudaMemcpyDeviceToHost, s));
  XMGN_CUDA(cudaMemcpyAsync(&herr, err, sizeof(herr), cudaMemcpyDeviceToHost, s));
  XMGN_CUDA(cudaStreamSynchronize(s));
  if (herr & DEV_ERR_RANGE) {
    XMGN_CUDA(cudaMemsetAsync(err, 0, sizeof(uint32_t), s));
    return fail(XMGN_ERR_RANGE, "coordinate outside the lattice range (|x*scale| >= 2^24 or not finite)");
  }

  // cell edge: about two cells per point over the bounding volume
  Grid G;
  double vol = 1.0;
  for (int a = 0; a < 3; ++a) {
    G.lo[a] = hb[a];
    vol *= double(int64_t(hb[3 + a]) - hb[a] + 1);
  }
  double c = cbrt(vol / (2.0 * double(N)));
  if (c < 1) c = 1;
  G.c = int64_t(ceil(c));
  for (;;) {
    int64_t tot = 1;
    for (int a = 0; a < 3; ++a) {
      G.g[a] = (int64_t(hb[3 + a]) - hb[a]) / G.c + 1;
      tot *= G.g[a];
    }
    if (tot <= max_cells) break;
    G.c = G.c + G.c / 4 + 1;
  }
  const int64_t ncell = G.g[0] * G.g[1] * G.g[2];

  XMGN_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * size_t(ncell), s));
  cell_count_kernel<<<grid_for(N, 256), 256, 0, s>>>(q, N, G, cell_of, cnt);
  XMGN_LAUNCH_CHECK();
  XMGN_TRY(exclusive_scan_i32(cnt, cstart, ncell, scan_tmp, s));
  XMGN_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * size_t(ncell), s));
  cell_scatter_kernel<<<grid_for(N, 256), 256, 0, s>>>(cell_of, N, cstart, cnt, sorted);
  XMGN_LAUNCH_CHECK();
  knn_search_kernel<<<grid_for(N, 128), 128, 0, s>>>(q, sorted, cstart, N, k, G, nbr);
  XMGN_LAUNCH_CHECK();

  // symmetrise: candidates = own kNN list + every j that lists i
  // candidate count of i = k (own list) + number of j listing i; the scan of
  // the reverse counts is shifted by k*i afterwards
  XMGN_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * size_t(N), s));
  sym_count_kernel<<<grid_for(N * k, 256), 256, 0, s>>>(nbr, N, k, cnt, err);
  XMGN_LAUNCH_CHECK();
  XMGN_TRY(exclusive_scan_i32(cnt, cstart, N, scan_tmp, s));
  // add k*i to the exclusive offsets (own entries come first)
  add_ramp_kernel<<<grid_for(N + 1, 256), 256, 0, s>>>(cstart, N, k);
  XMGN_LAUNCH_CHECK();
  sym_own_kernel<<<grid_for(N, 256), 256, 0, s>>>(nbr, N, k, cstart, cand, fill);
  XMGN_LAUNCH_CHECK();
  sym_rev_kernel<<<grid_for(N * k, 256), 256, 0, s>>>(nbr, N, k, cand, fill);
  XMGN_LAUNCH_CHECK();
  sym_sort_kernel<<<grid_for(N, 128), 128, 0, s>>>(cand, cstart, N, deg);
  XMGN_LAUNCH_CHECK();
  XMGN_TRY(exclusive_scan_i32(deg, row_ptr, N, scan_tmp, s));
  int64_t E = 0;
  XMGN_CUDA(cudaMemcpyAsync(&E, row_ptr + N, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  XMGN_CUDA(cudaStreamSynchronize(s));
  *E_out = E;
  if (E > E_cap) return fail(XMGN_ERR_WORKSPACE, "E=%lld exceeds E_cap=%lld", (long long)E, (long long)E_cap);
  sym_emit_kernel<<<grid_for(N, 128), 128, 0, s>>>(cand, cstart, row_ptr, N, col, recv);
  XMGN_LAUNCH_CHECK();
  if (csc_perm) {
    csc_perm_kernel<<<grid_for(E, 256), 256, 0, s>>>(row_ptr, col, recv, nullptr, N, E, csc_perm, err);
    XMGN_LAUNCH_CHECK();
  }
  return XMGN_OK;
}

}  // namespace xmgn
