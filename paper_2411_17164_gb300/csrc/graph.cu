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

// The k nearest reference points of lattice point i (excluding i itself),
// ranked by (d^2, index), from the cell-sorted reference set; returns how
// many were found (k unless the reference set is smaller).
__device__ __forceinline__ int knn_point(const int32_t* __restrict__ q, const int32_t* __restrict__ sorted,
                                         const int64_t* __restrict__ start, int k, const Grid& G, int32_t i,
                                         int64_t* bd, int32_t* bj) {
  const int64_t px = q[3 * i], py = q[3 * i + 1], pz = q[3 * i + 2];
  const int64_t cx = (px - G.lo[0]) / G.c, cy = (py - G.lo[1]) / G.c, cz = (pz - G.lo[2]) / G.c;
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
  return have;
}

// kNN of every reference point among the reference points (visited in cell
// order); row i of the output is nbr[i*stride + off .. + k), -1 if missing.
__global__ void knn_search_kernel(const int32_t* __restrict__ q, const int32_t* __restrict__ sorted,
                                  const int64_t* __restrict__ start, int64_t n, int k, Grid G,
                                  int32_t* __restrict__ nbr, int64_t stride, int off) {
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int32_t i = sorted[t];
    int64_t bd[kMaxK];
    int32_t bj[kMaxK];
    const int have = knn_point(q, sorted, start, k, G, i, bd, bj);
    for (int a = 0; a < k; ++a) nbr[int64_t(i) * stride + off + a] = a < have ? bj[a] : -1;
  }
}

// kNN among the reference points of the query points q0..q1-1 (not in the
// reference set; they must lie inside the grid).
__global__ void knn_query_kernel(const int32_t* __restrict__ q, const int32_t* __restrict__ sorted,
                                 const int64_t* __restrict__ start, int64_t q0, int64_t q1, int k, Grid G,
                                 int32_t* __restrict__ nbr, int64_t stride, int off) {
  for (int64_t i = q0 + int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < q1;
       i += int64_t(gridDim.x) * blockDim.x) {
    int64_t bd[kMaxK];
    int32_t bj[kMaxK];
    const int have = knn_point(q, sorted, start, k, G, int32_t(i), bd, bj);
    for (int a = 0; a < k; ++a) nbr[i * stride + off + a] = a < have ? bj[a] : -1;
  }
}

// ---- symmetrisation
__global__ void sym_count_kernel(const int32_t* __restrict__ nbr, int64_t n, int k,
                                 int32_t* __restrict__ cnt, uint32_t* err) {
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n * k;
       t += int64_t(gridDim.x) * blockDim.x) {
    int32_t j = nbr[t];
    if (j == -1) continue;  // empty slot
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
      if (c[a] >= 0 && c[a] != int32_t(i) && (a == 0 || c[a] != c[a - 1])) ++u;
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
      if (c[a] >= 0 && c[a] != int32_t(i) && (a == 0 || c[a] != c[a - 1])) {
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

struct KnnWs {
  int32_t *q, *bbox, *sorted, *nbr, *cnt, *cand, *deg;
  int64_t *cell_of, *cstart, *scan_tmp;
  unsigned long long* fill;
};

static int64_t knn_max_cells(int64_t N) { return 2 * N + 1024; }

// Workspace for N points with K directed slots per point.
static void knn_layout(int64_t N, int32_t K, Arena& A, KnnWs& w) {
  const int64_t cnt_n = knn_max_cells(N) > N ? knn_max_cells(N) : N;
  w.q = A.take<int32_t>(size_t(3 * N));
  w.bbox = A.take<int32_t>(8);
  w.cell_of = A.take<int64_t>(size_t(N));
  w.sorted = A.take<int32_t>(size_t(N));
  w.nbr = A.take<int32_t>(size_t(N * K));
  w.cnt = A.take<int32_t>(size_t(cnt_n + 1));
  w.cstart = A.take<int64_t>(size_t(cnt_n + 1));
  w.cand = A.take<int32_t>(size_t(2 * N * K));
  w.fill = A.take<unsigned long long>(size_t(N));
  w.deg = A.take<int32_t>(size_t(N));
  w.scan_tmp = A.take<int64_t>(scan_tmp_elems(cnt_n + 1) + 16);
}

// Lattice coordinates of all N points and their bounding box (host).
static xmgn_status quantize_all(const float* xyz, int64_t N, double scale, KnnWs& w, int32_t hb[6],
                                uint32_t* err, cudaStream_t s) {
  bbox_init_kernel<<<1, 32, 0, s>>>(w.bbox);
  XMGN_LAUNCH_CHECK();
  quantize_kernel<<<grid_for(N, 256), 256, 0, s>>>(xyz, N, float(scale), w.q, w.bbox, err);
  XMGN_LAUNCH_CHECK();
  uint32_t herr = 0;
  XMGN_CUDA(cudaMemcpyAsync(hb, w.bbox, sizeof(int32_t) * 6, cudaMemcpyDeviceToHost, s));
  XMGN_CUDA(cudaMemcpyAsync(&herr, err, sizeof(herr), cudaMemcpyDeviceToHost, s));
  XMGN_CUDA(cudaStreamSynchronize(s));
  if (herr & DEV_ERR_RANGE) {
    XMGN_CUDA(cudaMemsetAsync(err, 0, sizeof(uint32_t), s));
    return fail(XMGN_ERR_RANGE, "coordinate outside the lattice range (|x*scale| >= 2^24 or not finite)");
  }
  return XMGN_OK;
}

// Counting sort of the reference points 0..n_ref-1 into a uniform grid over
// the bounding box hb of all points (about two cells per reference point).
static xmgn_status grid_sort(int64_t n_ref, const int32_t hb[6], int64_t max_cells, KnnWs& w, Grid* Gout,
                             cudaStream_t s) {
  Grid G;
  double vol = 1.0;
  for (int a = 0; a < 3; ++a) {
    G.lo[a] = hb[a];
    vol *= double(int64_t(hb[3 + a]) - hb[a] + 1);
  }
  double c = cbrt(vol / (2.0 * double(n_ref)));
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
  XMGN_CUDA(cudaMemsetAsync(w.cnt, 0, sizeof(int32_t) * size_t(ncell), s));
  cell_count_kernel<<<grid_for(n_ref, 256), 256, 0, s>>>(w.q, n_ref, G, w.cell_of, w.cnt);
  XMGN_LAUNCH_CHECK();
  XMGN_TRY(exclusive_scan_i32(w.cnt, w.cstart, ncell, w.scan_tmp, s));
  XMGN_CUDA(cudaMemsetAsync(w.cnt, 0, sizeof(int32_t) * size_t(ncell), s));
  cell_scatter_kernel<<<grid_for(n_ref, 256), 256, 0, s>>>(w.cell_of, n_ref, w.cstart, w.cnt, w.sorted);
  XMGN_LAUNCH_CHECK();
  *Gout = G;
  return XMGN_OK;
}

// Undirected receiver-major CSR from K directed slots per point (w.nbr,
// -1 = empty): candidates of i = its own slots + every j listing i; the
// candidate offsets are the scan of the reverse counts shifted by K*i.
static xmgn_status symmetrise_slots(int64_t N, int32_t K, KnnWs& w, int64_t* row_ptr, int32_t* col,
                                    int32_t* recv, int32_t* csc_perm, int64_t E_cap, int64_t* E_out,
                                    uint32_t* err, cudaStream_t s) {
  XMGN_CUDA(cudaMemsetAsync(w.cnt, 0, sizeof(int32_t) * size_t(N), s));
  sym_count_kernel<<<grid_for(N * K, 256), 256, 0, s>>>(w.nbr, N, K, w.cnt, err);
  XMGN_LAUNCH_CHECK();
  XMGN_TRY(exclusive_scan_i32(w.cnt, w.cstart, N, w.scan_tmp, s));
  add_ramp_kernel<<<grid_for(N + 1, 256), 256, 0, s>>>(w.cstart, N, K);
  XMGN_LAUNCH_CHECK();
  sym_own_kernel<<<grid_for(N, 256), 256, 0, s>>>(w.nbr, N, K, w.cstart, w.cand, w.fill);
  XMGN_LAUNCH_CHECK();
  sym_rev_kernel<<<grid_for(N * K, 256), 256, 0, s>>>(w.nbr, N, K, w.cand, w.fill);
  XMGN_LAUNCH_CHECK();
  sym_sort_kernel<<<grid_for(N, 128), 128, 0, s>>>(w.cand, w.cstart, N, w.deg);
  XMGN_LAUNCH_CHECK();
  XMGN_TRY(exclusive_scan_i32(w.deg, row_ptr, N, w.scan_tmp, s));
  int64_t E = 0;
  XMGN_CUDA(cudaMemcpyAsync(&E, row_ptr + N, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  XMGN_CUDA(cudaStreamSynchronize(s));
  *E_out = E;
  if (E > E_cap) return fail(XMGN_ERR_WORKSPACE, "E=%lld exceeds E_cap=%lld", (long long)E, (long long)E_cap);
  sym_emit_kernel<<<grid_for(N, 128), 128, 0, s>>>(w.cand, w.cstart, row_ptr, N, col, recv);
  XMGN_LAUNCH_CHECK();
  if (csc_perm) {
    csc_perm_kernel<<<grid_for(E, 256), 256, 0, s>>>(row_ptr, col, recv, nullptr, N, E, csc_perm, err);
    XMGN_LAUNCH_CHECK();
  }
  return XMGN_OK;
}

static xmgn_status check_scale(double scale) {
  int ex = 0;
  double fr = frexp(scale, &ex);
  if (!(scale > 0) || fr != 0.5) return fail(XMGN_ERR_ARG, "lattice_scale must be a power of two");
  return XMGN_OK;
}

xmgn_status build_knn_ws(int64_t N, int32_t k, size_t* ws_bytes) {
  Arena A;
  A.dry = true;
  KnnWs w;
  knn_layout(N, k, A, w);
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
  XMGN_TRY(check_scale(scale));
  if (csc_perm && !recv) return fail(XMGN_ERR_ARG, "csc_perm requires recv");

  Arena A;
  A.base = static_cast<char*>(ws);
  A.cap = ws_bytes;
  KnnWs w;
  knn_layout(N, k, A, w);
  if (!A.ok()) return fail(XMGN_ERR_WORKSPACE, "knn workspace too small: need %zu", A.used);
  uint32_t* err = device_error_word();
  if (nbr_out) w.nbr = nbr_out;
  int32_t hb[6];
  XMGN_TRY(quantize_all(xyz, N, scale, w, hb, err, s));
  Grid G;
  XMGN_TRY(grid_sort(N, hb, knn_max_cells(N), w, &G, s));
  knn_search_kernel<<<grid_for(N, 128), 128, 0, s>>>(w.q, w.sorted, w.cstart, N, k, G, w.nbr, k, 0);
  XMGN_LAUNCH_CHECK();
  return symmetrise_slots(N, k, w, row_ptr, col, recv, csc_perm, E_cap, E_out, err, s);
}

static int32_t multiscale_slots(int32_t n_levels, int32_t k, int32_t k_cross) {
  return n_levels * k + (n_levels > 1 ? k_cross : 0);
}

xmgn_status build_multiscale_ws(int64_t N, int32_t n_levels, int32_t k, int32_t k_cross, size_t* ws_bytes) {
  if (n_levels < 1) return fail(XMGN_ERR_ARG, "need at least one level");
  Arena A;
  A.dry = true;
  KnnWs w;
  knn_layout(N, multiscale_slots(n_levels, k, k_cross), A, w);
  *ws_bytes = A.used + 256;
  return XMGN_OK;
}

xmgn_status build_multiscale(const float* xyz, int64_t N, const int64_t* sizes, int32_t n_levels, int32_t k,
                             int32_t k_cross, double scale, void* ws, size_t ws_bytes, int32_t* nbr_out,
                             int64_t* row_ptr, int32_t* col, int32_t* recv, int32_t* csc_perm, int64_t E_cap,
                             int64_t* E_out, cudaStream_t s) {
  if (!xyz || !sizes || !row_ptr || !col || !E_out || !ws) return fail(XMGN_ERR_ARG, "null pointer");
  if (n_levels < 1 || n_levels > 16) return fail(XMGN_ERR_ARG, "n_levels must be in [1, 16]");
  if (k < 1 || k > kMaxK || k_cross < 1 || k_cross > kMaxK)
    return fail(XMGN_ERR_ARG, "k and k_cross must be in [1, %d]", kMaxK);
  if (N >= (int64_t(1) << 31)) return fail(XMGN_ERR_ARG, "N must be < 2^31");
  for (int l = 0; l < n_levels; ++l) {
    const int64_t lo = l ? sizes[l - 1] : 0;
    if (sizes[l] <= lo) return fail(XMGN_ERR_ARG, "level sizes must increase");
  }
  if (sizes[n_levels - 1] != N) return fail(XMGN_ERR_ARG, "the last level size must be N");
  if (sizes[0] < int64_t(k) + 1) return fail(XMGN_ERR_ARG, "the first level needs more than k points");
  if (n_levels > 1 && sizes[0] < k_cross) return fail(XMGN_ERR_ARG, "the first level needs k_cross points");
  XMGN_TRY(check_scale(scale));
  if (csc_perm && !recv) return fail(XMGN_ERR_ARG, "csc_perm requires recv");

  const int32_t K = multiscale_slots(n_levels, k, k_cross);
  Arena A;
  A.base = static_cast<char*>(ws);
  A.cap = ws_bytes;
  KnnWs w;
  knn_layout(N, K, A, w);
  if (!A.ok()) return fail(XMGN_ERR_WORKSPACE, "multiscale workspace too small: need %zu", A.used);
  uint32_t* err = device_error_word();
  if (nbr_out) w.nbr = nbr_out;
  int32_t hb[6];
  XMGN_TRY(quantize_all(xyz, N, scale, w, hb, err, s));
  XMGN_CUDA(cudaMemsetAsync(w.nbr, 0xff, sizeof(int32_t) * size_t(N) * K, s));  // all slots empty (-1)
  for (int l = 0; l < n_levels; ++l) {
    // kNN within level l (the first sizes[l] points): slots [l*k, l*k + k)
    Grid G;
    XMGN_TRY(grid_sort(sizes[l], hb, knn_max_cells(N), w, &G, s));
    knn_search_kernel<<<grid_for(sizes[l], 128), 128, 0, s>>>(w.q, w.sorted, w.cstart, sizes[l], k, G, w.nbr, K,
                                                               l * k);
    XMGN_LAUNCH_CHECK();
    if (l > 0) {  // points new in level l -> k_cross nearest of level l-1: slots [L*k, L*k + k_cross)
      XMGN_TRY(grid_sort(sizes[l - 1], hb, knn_max_cells(N), w, &G, s));
      knn_query_kernel<<<grid_for(sizes[l] - sizes[l - 1], 128), 128, 0, s>>>(
          w.q, w.sorted, w.cstart, sizes[l - 1], sizes[l], k_cross, G, w.nbr, K, n_levels * k);
      XMGN_LAUNCH_CHECK();
    }
  }
  return symmetrise_slots(N, K, w, row_ptr, col, recv, csc_perm, E_cap, E_out, err, s);
}

}  // namespace xmgn
