// Halo partitioning (Sec. III-A "Graph Partitioning", "Message Passing Across
// Partitions").
//
// Parts: recursive coordinate bisection (the paper uses METIS).  Each level
// sorts packed keys (segment | lattice coordinate on the segment's split axis |
// node id) with a bitonic sort; keys are unique, so the order -- and the split
// -- is fully determined.
//
// Halos: one multi-source BFS per part, all parts advanced together one hop
// per launch; a (part, node) pair is claimed exactly once through a bit in a
// P x N bitmask.  Every reached pair becomes a packed key (part | hop | node);
// sorting those keys yields the batch order directly: part-major, inner
// nodes by id, then halo nodes by (hop, id).
#include <math.h>

#include <vector>

#include "common.cuh"

namespace xmgn {

__global__ void csc_perm_kernel(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                const int32_t* __restrict__ recv, const int32_t* __restrict__ key,
                                int64_t n, int64_t e, int32_t* __restrict__ perm, uint32_t* err);

namespace {

constexpr int kSortTile = 2048;  // keys per shared-memory bitonic tile

__device__ __forceinline__ void cmp_swap(uint64_t& a, uint64_t& b, bool up) {
  if ((a > b) == up) {
    uint64_t t = a;
    a = b;
    b = t;
  }
}

// Sorts each 2048-key tile fully (directions alternate per bitonic rule with
// respect to the global sequence length).
__global__ void bitonic_tile_sort(uint64_t* __restrict__ keys) {
  __shared__ uint64_t s[kSortTile];
  const int64_t base = int64_t(blockIdx.x) * kSortTile;
  for (int i = threadIdx.x; i < kSortTile; i += blockDim.x) s[i] = keys[base + i];
  __syncthreads();
  for (int k = 2; k <= kSortTile; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < kSortTile / 2; t += blockDim.x) {
        int i = 2 * t - (t & (j - 1));
        int l = i + j;
        bool up = ((base + i) & k) == 0;
        cmp_swap(s[i], s[l], up);
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < kSortTile; i += blockDim.x) keys[base + i] = s[i];
}

// Merge steps j < kSortTile of stage k, inside shared memory.
__global__ void bitonic_tile_merge(uint64_t* __restrict__ keys, int64_t k) {
  __shared__ uint64_t s[kSortTile];
  const int64_t base = int64_t(blockIdx.x) * kSortTile;
  for (int i = threadIdx.x; i < kSortTile; i += blockDim.x) s[i] = keys[base + i];
  __syncthreads();
  const bool up = (base & k) == 0;
  for (int j = kSortTile >> 1; j > 0; j >>= 1) {
    for (int t = threadIdx.x; t < kSortTile / 2; t += blockDim.x) {
      int i = 2 * t - (t & (j - 1));
      cmp_swap(s[i], s[i + j], up);
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < kSortTile; i += blockDim.x) keys[base + i] = s[i];
}

__global__ void bitonic_global_step(uint64_t* __restrict__ keys, int64_t m, int64_t k, int64_t j) {
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < m / 2;
       t += int64_t(gridDim.x) * blockDim.x) {
    int64_t i = 2 * t - (t & (j - 1));
    int64_t l = i + j;
    bool up = (i & k) == 0;
    uint64_t a = keys[i], b = keys[l];
    if ((a > b) == up) {
      keys[i] = b;
      keys[l] = a;
    }
  }
}

__global__ void fill_u64(uint64_t* p, int64_t from, int64_t to, uint64_t v) {
  for (int64_t i = from + int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < to;
       i += int64_t(gridDim.x) * blockDim.x)
    p[i] = v;
}

}  // namespace

int64_t pow2_at_least(int64_t n) {
  int64_t m = kSortTile;
  while (m < n) m <<= 1;
  return m;
}

// Sorts keys[0..n) ascending; keys must have room for pow2_at_least(n).
xmgn_status sort_u64(uint64_t* keys, int64_t n, cudaStream_t s) {
  const int64_t m = pow2_at_least(n);
  if (m > n) {
    fill_u64<<<grid_for(m - n, 256), 256, 0, s>>>(keys, n, m, ~uint64_t(0));
    XMGN_LAUNCH_CHECK();
  }
  bitonic_tile_sort<<<unsigned(m / kSortTile), 1024, 0, s>>>(keys);
  XMGN_LAUNCH_CHECK();
  for (int64_t k = 2 * kSortTile; k <= m; k <<= 1) {
    for (int64_t j = k >> 1; j >= kSortTile; j >>= 1) {
      bitonic_global_step<<<grid_for(m / 2, 256), 256, 0, s>>>(keys, m, k, j);
      XMGN_LAUNCH_CHECK();
    }
    bitonic_tile_merge<<<unsigned(m / kSortTile), 1024, 0, s>>>(keys, k);
    XMGN_LAUNCH_CHECK();
  }
  return XMGN_OK;
}

xmgn_status quantize_launch(const float* xyz, int64_t n, double scale, int32_t* q, int32_t* bbox,
                            uint32_t* err, cudaStream_t s);

namespace {

constexpr int kIdBits = 28;       // RCB: node ids < 2^28
constexpr int kCoordBits = 25;    // lattice coordinate + 2^24
constexpr uint64_t kIdMask = (uint64_t(1) << kIdBits) - 1;

__global__ void seg_extent_kernel(const uint64_t* __restrict__ keys, int64_t n,
                                  const int64_t* __restrict__ seg_start, int nseg,
                                  const int32_t* __restrict__ q, int32_t* __restrict__ ext) {
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n;
       t += int64_t(gridDim.x) * blockDim.x) {
    int64_t id = int64_t(keys[t] & kIdMask);
    int lo = 0, hi = nseg;  // segment containing position t
    while (hi - lo > 1) {
      int mid = (lo + hi) >> 1;
      if (seg_start[mid] <= t) lo = mid; else hi = mid;
    }
    for (int a = 0; a < 3; ++a) {
      atomicMin(&ext[6 * lo + a], q[3 * id + a]);
      atomicMax(&ext[6 * lo + 3 + a], q[3 * id + a]);
    }
  }
}

__global__ void ext_init_kernel(int32_t* ext, int nseg) {
  for (int i = threadIdx.x; i < nseg; i += blockDim.x) {
    for (int a = 0; a < 3; ++a) {
      ext[6 * i + a] = INT32_MAX;
      ext[6 * i + 3 + a] = INT32_MIN;
    }
  }
}

__global__ void rcb_key_kernel(uint64_t* __restrict__ keys, int64_t n, const int64_t* __restrict__ seg_start,
                               const int32_t* __restrict__ seg_axis, int nseg, const int32_t* __restrict__ q,
                               int first) {
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n;
       t += int64_t(gridDim.x) * blockDim.x) {
    int64_t id = first ? t : int64_t(keys[t] & kIdMask);
    int lo = 0, hi = nseg;
    while (hi - lo > 1) {
      int mid = (lo + hi) >> 1;
      if (seg_start[mid] <= t) lo = mid; else hi = mid;
    }
    uint64_t c = uint64_t(int64_t(q[3 * id + seg_axis[lo]]) + (int64_t(1) << 24));
    keys[t] = (uint64_t(lo) << (kIdBits + kCoordBits)) | (c << kIdBits) | uint64_t(id);
  }
}

__global__ void rcb_assign_kernel(const uint64_t* __restrict__ keys, int64_t n,
                                  const int64_t* __restrict__ seg_start, const int32_t* __restrict__ seg_part,
                                  int nseg, int32_t* __restrict__ part) {
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n;
       t += int64_t(gridDim.x) * blockDim.x) {
    int lo = 0, hi = nseg;
    while (hi - lo > 1) {
      int mid = (lo + hi) >> 1;
      if (seg_start[mid] <= t) lo = mid; else hi = mid;
    }
    part[keys[t] & kIdMask] = seg_part[lo];
  }
}

// ---- halo BFS
// member key: part (16 bits) | hop (8 bits) | node id (32 bits)
__device__ __forceinline__ uint64_t mkey(uint32_t p, uint32_t hop, uint32_t v) {
  return (uint64_t(p) << 40) | (uint64_t(hop) << 32) | uint64_t(v);
}

__global__ void bfs_seed_kernel(const int32_t* __restrict__ part, int64_t n, int P,
                                uint32_t* __restrict__ bits, int64_t words,
                                uint64_t* __restrict__ members, unsigned long long* __restrict__ count,
                                int64_t cap, uint32_t* err) {
  for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < n;
       v += int64_t(gridDim.x) * blockDim.x) {
    int p = part[v];
    if (p == -1) continue;  // inner in no part (may still be another part's halo)
    if (p < 0 || p >= P) {
      dev_flag(err, DEV_ERR_GRAPH);
      continue;
    }
    atomicOr(&bits[int64_t(p) * words + (v >> 5)], 1u << (v & 31));
    unsigned long long pos = atomicAdd(count, 1ull);
    if (int64_t(pos) < cap) members[pos] = mkey(p, 0, uint32_t(v));
    else dev_flag(err, DEV_ERR_CAP);
  }
}

__global__ void bfs_mark_kernel(unsigned long long* bounds, int h, const unsigned long long* count) {
  if (threadIdx.x == 0 && blockIdx.x == 0) bounds[h] = *count;
}

__global__ void bfs_round_kernel(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                 int64_t n, uint32_t* __restrict__ bits, int64_t words,
                                 uint64_t* __restrict__ members, unsigned long long* __restrict__ count,
                                 const unsigned long long* __restrict__ bounds, int h, int64_t cap,
                                 uint32_t* err) {
  const int64_t lo = int64_t(bounds[h - 1]);
  const int64_t hi = min(int64_t(bounds[h]), cap);
  for (int64_t t = lo + int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < hi;
       t += int64_t(gridDim.x) * blockDim.x) {
    uint64_t key = members[t];
    uint32_t p = uint32_t(key >> 40);
    uint32_t u = uint32_t(key & 0xffffffffu);
    for (int64_t e = row_ptr[u], ee = row_ptr[u + 1]; e < ee; ++e) {
      int32_t w = col[e];
      if (w < 0 || w >= n) {
        dev_flag(err, DEV_ERR_GRAPH);
        continue;
      }
      uint32_t m = 1u << (w & 31);
      uint32_t* word = &bits[int64_t(p) * words + (w >> 5)];
      if (__ldcg(word) & m) continue;
      if (atomicOr(word, m) & m) continue;
      unsigned long long pos = atomicAdd(count, 1ull);
      if (int64_t(pos) < cap) members[pos] = mkey(p, uint32_t(h), uint32_t(w));
      else dev_flag(err, DEV_ERR_CAP);
    }
  }
}

__global__ void batch_nodes_kernel(const uint64_t* __restrict__ members, int64_t nb, int64_t n,
                                   int32_t* __restrict__ map, int32_t* __restrict__ gid,
                                   uint8_t* __restrict__ hop, unsigned long long* __restrict__ pcount,
                                   unsigned long long* __restrict__ icount) {
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < nb;
       t += int64_t(gridDim.x) * blockDim.x) {
    uint64_t key = members[t];
    uint32_t p = uint32_t(key >> 40);
    uint32_t hh = uint32_t((key >> 32) & 0xff);
    uint32_t v = uint32_t(key & 0xffffffffu);
    map[int64_t(p) * n + v] = int32_t(t);
    if (gid) gid[t] = int32_t(v);
    if (hop) hop[t] = uint8_t(hh);
    if (pcount) {
      // members are sorted by partition, so a warp's keys fall into one or
      // two partitions: one atomic per partition and warp, from its lowest lane
      const unsigned am = __activemask();
      const unsigned same = __match_any_sync(am, p);
      const unsigned inner = __ballot_sync(am, hh == 0) & same;
      if ((threadIdx.x & 31) == __ffs(same) - 1) {
        atomicAdd(&pcount[p], (unsigned long long)__popc(same));
        if (inner) atomicAdd(&icount[p], (unsigned long long)__popc(inner));
      }
    }
  }
}

__global__ void batch_deg_kernel(const uint64_t* __restrict__ members, int64_t nb, int64_t n,
                                 const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                 const int32_t* __restrict__ map, int32_t* __restrict__ deg) {
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < nb;
       t += int64_t(gridDim.x) * blockDim.x) {
    uint64_t key = members[t];
    int64_t p = int64_t(key >> 40);
    uint32_t v = uint32_t(key & 0xffffffffu);
    int32_t d = 0;
    for (int64_t e = row_ptr[v], ee = row_ptr[v + 1]; e < ee; ++e)
      d += map[p * n + col[e]] >= 0;
    deg[t] = d;
  }
}

__global__ void batch_edges_kernel(const uint64_t* __restrict__ members, int64_t nb, int64_t n,
                                   const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                   const int32_t* __restrict__ map, const int64_t* __restrict__ brp,
                                   int32_t* __restrict__ bcol, int32_t* __restrict__ brecv) {
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < nb;
       t += int64_t(gridDim.x) * blockDim.x) {
    uint64_t key = members[t];
    int64_t p = int64_t(key >> 40);
    uint32_t v = uint32_t(key & 0xffffffffu);
    int64_t o = brp[t];
    for (int64_t e = row_ptr[v], ee = row_ptr[v + 1]; e < ee; ++e) {
      int32_t b = map[p * n + col[e]];
      if (b >= 0) {
        bcol[o] = b;
        brecv[o] = int32_t(t);
        ++o;
      }
    }
  }
}

struct PartLayout {
  int32_t* q;
  int32_t* bbox;
  uint64_t* keys;      // RCB keys, pow2(N)
  int32_t* part;       // part ids when caller gives no part array
  int32_t* ext;        // 6 per segment
  int64_t* seg_start;  // per segment
  int32_t* seg_axis;
  int32_t* seg_part;
  uint32_t* bits;      // P x words
  uint64_t* members;   // pow2(cap)
  unsigned long long* counters;  // [0] count, [1..L+2] bounds, then P pcount, P icount
  int32_t* map;        // P x N
  int32_t* deg;        // cap
  int64_t* brp;        // cap + 1
  int32_t* gid;        // cap (sizing pass)
  int64_t* scan_tmp;
  int64_t* stamp;      // [8]: what the last sizing pass left in this workspace (see kStampMagic)
  int64_t cap;
};

// Written by a completed sizing pass, checked by the emit pass that resumes
// from it: magic, N, E, P, hops, batch nodes, batch edges, part_in given.
constexpr int64_t kStampMagic = 0x78686c6f73697a65;

int64_t member_cap(int64_t N, int32_t P) {
  int64_t c = int64_t(P) * N;
  int64_t lim = 8 * N + 4096;
  return c < lim ? c : lim;
}

void part_layout(Arena& A, int64_t N, int32_t P, int32_t L, PartLayout& w) {
  const int64_t words = (N + 31) / 32;
  w.cap = member_cap(N, P);
  w.q = A.take<int32_t>(size_t(3 * N));
  w.bbox = A.take<int32_t>(8);
  w.keys = A.take<uint64_t>(size_t(pow2_at_least(N)));
  w.part = A.take<int32_t>(size_t(N));
  w.ext = A.take<int32_t>(size_t(6 * P + 6));
  w.seg_start = A.take<int64_t>(size_t(P + 1));
  w.seg_axis = A.take<int32_t>(size_t(P + 1));
  w.seg_part = A.take<int32_t>(size_t(P + 1));
  w.bits = A.take<uint32_t>(size_t(int64_t(P) * words));
  w.members = A.take<uint64_t>(size_t(pow2_at_least(w.cap)));
  w.counters = A.take<unsigned long long>(size_t(4 + 256 + 2 * P));
  w.map = A.take<int32_t>(size_t(int64_t(P) * N));
  w.deg = A.take<int32_t>(size_t(w.cap));
  w.brp = A.take<int64_t>(size_t(w.cap + 1));
  w.gid = nullptr;
  w.scan_tmp = A.take<int64_t>(scan_tmp_elems(w.cap + 1) + 16);
  w.stamp = A.take<int64_t>(8);
  (void)L;
}

struct Seg {
  int64_t start, end;
  int32_t parts, base;
};

}  // namespace

xmgn_status partition_halo_ws(int64_t N, int64_t E, int32_t P, size_t* ws_bytes) {
  (void)E;
  Arena A;
  A.dry = true;
  PartLayout w;
  part_layout(A, N, P, 0, w);
  *ws_bytes = A.used + 256;
  return XMGN_OK;
}

xmgn_status partition_halo(const int64_t* row_ptr, const int32_t* col, int64_t N, int64_t E,
                           const float* xyz, double scale, int32_t P, int32_t L,
                           const int32_t* part_in, void* ws, size_t ws_bytes, int32_t* part_out,
                           int64_t* node_ptr, int64_t* edge_ptr, int64_t* inner_cnt, int32_t* gid,
                           uint8_t* hop, int64_t* b_row_ptr, int32_t* b_col, int32_t* b_recv,
                           int32_t* b_csc_perm, int64_t cap_nodes, int64_t cap_edges,
                           cudaStream_t s, bool resume) {
  if (!row_ptr || !col || !ws || !node_ptr || !edge_ptr || !inner_cnt)
    return fail(XMGN_ERR_ARG, "null pointer");
  if (P < 1 || P > 65535 || int64_t(P) > N) return fail(XMGN_ERR_ARG, "need 1 <= P <= min(N, 65535)");
  if (L < 0 || L > 255) return fail(XMGN_ERR_ARG, "halo_hops must be in [0, 255]");
  if (N < 1 || N >= (int64_t(1) << kIdBits)) return fail(XMGN_ERR_ARG, "N must be in [1, 2^28)");
  if (!part_in && !xyz) return fail(XMGN_ERR_ARG, "xyz required for RCB");
  const bool emit = gid != nullptr;
  if (emit && (!b_row_ptr || !b_col || !b_recv || !hop))
    return fail(XMGN_ERR_ARG, "emit pass needs gid, hop, b_row_ptr, b_col, b_recv");

  Arena A;
  A.base = static_cast<char*>(ws);
  A.cap = ws_bytes;
  PartLayout w;
  part_layout(A, N, P, L, w);
  if (!A.ok()) return fail(XMGN_ERR_WORKSPACE, "partition workspace too small: need %zu", A.used);
  uint32_t* err = device_error_word();
  int32_t* part = part_out ? part_out : w.part;
  if (resume) {
    if (!emit) return fail(XMGN_ERR_ARG, "the emit pass needs gid, hop, b_row_ptr, b_col, b_recv");
    int64_t st[8];
    XMGN_CUDA(cudaMemcpyAsync(st, w.stamp, sizeof(st), cudaMemcpyDeviceToHost, s));
    XMGN_CUDA(cudaStreamSynchronize(s));
    if (st[0] != kStampMagic || st[1] != N || st[2] != E || st[3] != P || st[4] != L || st[5] != node_ptr[P] ||
        st[6] != edge_ptr[P] || st[7] != (part_in ? 1 : 0))
      return fail(XMGN_ERR_ARG, "partition emit pass: the workspace holds no sizing pass of these inputs");
    const int64_t nb = node_ptr[P], eb = edge_ptr[P];
    if (cap_nodes < nb) return fail(XMGN_ERR_WORKSPACE, "cap_nodes %lld < %lld", (long long)cap_nodes, (long long)nb);
    if (cap_edges < eb) return fail(XMGN_ERR_WORKSPACE, "cap_edges %lld < %lld", (long long)cap_edges, (long long)eb);
    if (nb > 0) {  // ids and hops of the sorted members; the sizing pass left the map and the row pointers
      batch_nodes_kernel<<<grid_for(nb, 256), 256, 0, s>>>(w.members, nb, N, w.map, gid, hop, nullptr, nullptr);
      XMGN_LAUNCH_CHECK();
    }
    XMGN_CUDA(cudaMemcpyAsync(b_row_ptr, w.brp, sizeof(int64_t) * size_t(nb + 1), cudaMemcpyDeviceToDevice, s));
    batch_edges_kernel<<<grid_for(nb, 256), 256, 0, s>>>(w.members, nb, N, row_ptr, col, w.map, b_row_ptr, b_col,
                                                         b_recv);
    XMGN_LAUNCH_CHECK();
    if (b_csc_perm) {
      csc_perm_kernel<<<grid_for(eb, 256), 256, 0, s>>>(b_row_ptr, b_col, b_recv, gid, nb, eb, b_csc_perm, err);
      XMGN_LAUNCH_CHECK();
    }
    XMGN_CUDA(cudaMemsetAsync(w.stamp, 0, sizeof(int64_t) * 8, s));  // one emit per sizing pass
    XMGN_CUDA(cudaStreamSynchronize(s));
    return XMGN_OK;
  }

  // ---------------- parts
  if (part_in) {
    if (part != part_in)
      XMGN_CUDA(cudaMemcpyAsync(part, part_in, sizeof(int32_t) * size_t(N), cudaMemcpyDeviceToDevice, s));
  } else {
    XMGN_TRY(quantize_launch(xyz, N, scale, w.q, w.bbox, err, s));
    uint32_t herr = 0;
    XMGN_CUDA(cudaMemcpyAsync(&herr, err, sizeof(herr), cudaMemcpyDeviceToHost, s));
    XMGN_CUDA(cudaStreamSynchronize(s));
    if (herr & DEV_ERR_RANGE) {
      XMGN_CUDA(cudaMemsetAsync(err, 0, sizeof(uint32_t), s));
      return fail(XMGN_ERR_RANGE, "coordinate outside the lattice range");
    }
    std::vector<Seg> segs{{0, N, P, 0}};
    bool first = true;
    for (;;) {
      bool any = false;
      for (auto& g : segs) any |= g.parts > 1;
      if (!any) break;
      const int nseg = int(segs.size());
      std::vector<int64_t> hstart(nseg);
      for (int i = 0; i < nseg; ++i) hstart[i] = segs[i].start;
      XMGN_CUDA(cudaMemcpyAsync(w.seg_start, hstart.data(), sizeof(int64_t) * nseg, cudaMemcpyHostToDevice, s));
      std::vector<int32_t> axis(nseg, 0);
      if (!first) {
        ext_init_kernel<<<1, 256, 0, s>>>(w.ext, nseg);
        XMGN_LAUNCH_CHECK();
        seg_extent_kernel<<<grid_for(N, 256), 256, 0, s>>>(w.keys, N, w.seg_start, nseg, w.q, w.ext);
        XMGN_LAUNCH_CHECK();
        std::vector<int32_t> hext(6 * nseg);
        XMGN_CUDA(cudaMemcpyAsync(hext.data(), w.ext, sizeof(int32_t) * 6 * nseg, cudaMemcpyDeviceToHost, s));
        XMGN_CUDA(cudaStreamSynchronize(s));
        for (int i = 0; i < nseg; ++i) {
          int64_t best = -1;
          for (int a = 0; a < 3; ++a) {
            int64_t e = int64_t(hext[6 * i + 3 + a]) - hext[6 * i + a];
            if (e > best) { best = e; axis[i] = a; }
          }
        }
      } else {
        int32_t hb[6];
        XMGN_CUDA(cudaMemcpyAsync(hb, w.bbox, sizeof(hb), cudaMemcpyDeviceToHost, s));
        XMGN_CUDA(cudaStreamSynchronize(s));
        int64_t best = -1;
        for (int a = 0; a < 3; ++a) {
          int64_t e = int64_t(hb[3 + a]) - hb[a];
          if (e > best) { best = e; axis[0] = a; }
        }
      }
      XMGN_CUDA(cudaMemcpyAsync(w.seg_axis, axis.data(), sizeof(int32_t) * nseg, cudaMemcpyHostToDevice, s));
      rcb_key_kernel<<<grid_for(N, 256), 256, 0, s>>>(w.keys, N, w.seg_start, w.seg_axis, nseg, w.q, first ? 1 : 0);
      XMGN_LAUNCH_CHECK();
      XMGN_TRY(sort_u64(w.keys, N, s));
      first = false;
      std::vector<Seg> next;
      for (auto& g : segs) {
        if (g.parts == 1) {
          next.push_back(g);
          continue;
        }
        int32_t pl = g.parts / 2;
        int64_t nl = ((g.end - g.start) * pl) / g.parts;
        next.push_back({g.start, g.start + nl, pl, g.base});
        next.push_back({g.start + nl, g.end, g.parts - pl, g.base + pl});
      }
      segs.swap(next);
      // keep host vectors alive until the copies above have been consumed
      XMGN_CUDA(cudaStreamSynchronize(s));
    }
    const int nseg = int(segs.size());
    std::vector<int64_t> hstart(nseg);
    std::vector<int32_t> hpart(nseg);
    for (int i = 0; i < nseg; ++i) {
      hstart[i] = segs[i].start;
      hpart[i] = segs[i].base;
    }
    if (P == 1) {
      XMGN_CUDA(cudaMemsetAsync(part, 0, sizeof(int32_t) * size_t(N), s));
    } else {
      XMGN_CUDA(cudaMemcpyAsync(w.seg_start, hstart.data(), sizeof(int64_t) * nseg, cudaMemcpyHostToDevice, s));
      XMGN_CUDA(cudaMemcpyAsync(w.seg_part, hpart.data(), sizeof(int32_t) * nseg, cudaMemcpyHostToDevice, s));
      rcb_assign_kernel<<<grid_for(N, 256), 256, 0, s>>>(w.keys, N, w.seg_start, w.seg_part, nseg, part);
      XMGN_LAUNCH_CHECK();
    }
    XMGN_CUDA(cudaStreamSynchronize(s));
  }

  // ---------------- halo BFS
  const int64_t words = (N + 31) / 32;
  XMGN_CUDA(cudaMemsetAsync(w.bits, 0, sizeof(uint32_t) * size_t(int64_t(P) * words), s));
  XMGN_CUDA(cudaMemsetAsync(w.counters, 0, sizeof(unsigned long long) * size_t(4 + 256 + 2 * P), s));
  unsigned long long* count = w.counters;
  unsigned long long* bounds = w.counters + 1;  // bounds[h] = members before round h+1
  unsigned long long* pcount = w.counters + 4 + 256;
  unsigned long long* icount = pcount + P;
  const unsigned bfs_grid = unsigned(num_sms()) * 8;
  bfs_seed_kernel<<<grid_for(N, 256), 256, 0, s>>>(part, N, P, w.bits, words, w.members, count, w.cap, err);
  XMGN_LAUNCH_CHECK();
  // bounds[0] = 0 (memset); bounds[1] = after seeding
  bfs_mark_kernel<<<1, 32, 0, s>>>(bounds, 1, count);
  XMGN_LAUNCH_CHECK();
  for (int h = 1; h <= L; ++h) {
    // round h expands members[bounds[h-1] .. bounds[h])
    bfs_round_kernel<<<bfs_grid, 256, 0, s>>>(row_ptr, col, N, w.bits, words, w.members, count, bounds,
                                              h, w.cap, err);
    XMGN_LAUNCH_CHECK();
    bfs_mark_kernel<<<1, 32, 0, s>>>(bounds, h + 1, count);
    XMGN_LAUNCH_CHECK();
  }
  unsigned long long hcount = 0;
  uint32_t herr = 0;
  XMGN_CUDA(cudaMemcpyAsync(&hcount, count, sizeof(hcount), cudaMemcpyDeviceToHost, s));
  XMGN_CUDA(cudaMemcpyAsync(&herr, err, sizeof(herr), cudaMemcpyDeviceToHost, s));
  XMGN_CUDA(cudaStreamSynchronize(s));
  if (herr & (DEV_ERR_CAP | DEV_ERR_GRAPH)) {
    XMGN_CUDA(cudaMemsetAsync(err, 0, sizeof(uint32_t), s));
    if (herr & DEV_ERR_GRAPH) return fail(XMGN_ERR_GRAPH, "part id or sender id out of range");
    return fail(XMGN_ERR_WORKSPACE, "halo members exceed the workspace capacity (%lld)", (long long)w.cap);
  }
  const int64_t nb = int64_t(hcount);
  XMGN_TRY(sort_u64(w.members, nb, s));

  // ---------------- batch nodes and degrees
  XMGN_CUDA(cudaMemsetAsync(w.map, 0xff, sizeof(int32_t) * size_t(int64_t(P) * N), s));
  batch_nodes_kernel<<<grid_for(nb, 256), 256, 0, s>>>(w.members, nb, N, w.map, emit ? gid : nullptr,
                                                       emit ? hop : nullptr, pcount, icount);
  XMGN_LAUNCH_CHECK();
  batch_deg_kernel<<<grid_for(nb, 256), 256, 0, s>>>(w.members, nb, N, row_ptr, col, w.map, w.deg);
  XMGN_LAUNCH_CHECK();
  int64_t* brp = emit ? b_row_ptr : w.brp;
  if (emit && cap_nodes < nb) return fail(XMGN_ERR_WORKSPACE, "cap_nodes %lld < %lld", (long long)cap_nodes, (long long)nb);
  XMGN_TRY(exclusive_scan_i32(w.deg, brp, nb, w.scan_tmp, s));
  std::vector<unsigned long long> hp(2 * size_t(P));
  XMGN_CUDA(cudaMemcpyAsync(hp.data(), pcount, sizeof(unsigned long long) * 2 * size_t(P), cudaMemcpyDeviceToHost, s));
  XMGN_CUDA(cudaStreamSynchronize(s));
  node_ptr[0] = 0;
  for (int p = 0; p < P; ++p) {
    node_ptr[p + 1] = node_ptr[p] + int64_t(hp[p]);
    inner_cnt[p] = int64_t(hp[P + p]);
  }
  for (int p = 0; p <= P; ++p)
    XMGN_CUDA(cudaMemcpyAsync(&edge_ptr[p], brp + node_ptr[p], sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  XMGN_CUDA(cudaStreamSynchronize(s));
  if (!emit) {  // leave the stamp that lets an emit pass resume from this one
    const int64_t st[8] = {kStampMagic, N, E, P, L, node_ptr[P], edge_ptr[P], part_in ? 1 : 0};
    XMGN_CUDA(cudaMemcpyAsync(w.stamp, st, sizeof(st), cudaMemcpyHostToDevice, s));
    XMGN_CUDA(cudaStreamSynchronize(s));
    return XMGN_OK;
  }
  XMGN_CUDA(cudaMemsetAsync(w.stamp, 0, sizeof(int64_t) * 8, s));
  const int64_t eb = edge_ptr[P];
  if (cap_edges < eb) return fail(XMGN_ERR_WORKSPACE, "cap_edges %lld < %lld", (long long)cap_edges, (long long)eb);
  batch_edges_kernel<<<grid_for(nb, 256), 256, 0, s>>>(w.members, nb, N, row_ptr, col, w.map, brp, b_col, b_recv);
  XMGN_LAUNCH_CHECK();
  if (b_csc_perm) {
    csc_perm_kernel<<<grid_for(eb, 256), 256, 0, s>>>(brp, b_col, b_recv, gid, nb, eb, b_csc_perm, err);
    XMGN_LAUNCH_CHECK();
  }
  XMGN_CUDA(cudaStreamSynchronize(s));
  (void)E;
  return XMGN_OK;
}

}  // namespace xmgn
