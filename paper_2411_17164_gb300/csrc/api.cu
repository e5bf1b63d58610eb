// C-ABI entry points of libxmgn (declared in include/xmgn.h): argument
// validation on the host, then dispatch to the graph builders and the FP32 /
// BF16 model paths.
#include <stdarg.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <utility>
#include <vector>

#include "paths.cuh"
#include "tc.cuh"

namespace xmgn {

static thread_local char g_err[1024] = "no error";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

xmgn_status fail(xmgn_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return s;
}

static std::atomic<int64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// ---- kernel timing probes
struct ProbeState {
  std::mutex mu;
  bool on = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> used[PROBE_KINDS], pool;
  cudaEvent_t open[PROBE_KINDS] = {};
};
static ProbeState& probes() {
  static ProbeState p;
  return p;
}

// Inside a stream capture a plain event record only orders the graph; the
// external flag makes it an event-record node that every replay re-records,
// so the probes also time steps replayed from a CUDA graph.
static void record_probe(cudaEvent_t ev, cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &st) == cudaSuccess && st == cudaStreamCaptureStatusActive)
    cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal);
  else
    cudaEventRecord(ev, s);
}

void probe_begin(int kind, cudaStream_t s) {
  ProbeState& P = probes();
  std::lock_guard<std::mutex> g(P.mu);
  if (!P.on || kind < 0 || kind >= PROBE_KINDS) return;
  std::pair<cudaEvent_t, cudaEvent_t> e{nullptr, nullptr};
  if (!P.pool.empty()) {
    e = P.pool.back();
    P.pool.pop_back();
  } else if (cudaEventCreate(&e.first) != cudaSuccess || cudaEventCreate(&e.second) != cudaSuccess) {
    return;
  }
  record_probe(e.first, s);
  P.used[kind].push_back(e);
  P.open[kind] = e.second;
}

void probe_end(int kind, cudaStream_t s) {
  ProbeState& P = probes();
  std::lock_guard<std::mutex> g(P.mu);
  if (!P.on || kind < 0 || kind >= PROBE_KINDS || !P.open[kind]) return;
  record_probe(P.open[kind], s);
  P.open[kind] = nullptr;
}

__device__ uint32_t g_device_error;

uint32_t* device_error_word() {
  static uint32_t* cache[64] = {nullptr};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  if (!cache[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_device_error) != cudaSuccess) return nullptr;
    cache[dev] = static_cast<uint32_t*>(p);
  }
  return cache[dev];
}

namespace {

__global__ void validate_graph_kernel(xmgn_graph g, uint32_t* err) {
  const int64_t n = g.n_nodes, E = g.n_edges;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i <= n || i < E;
       i += int64_t(gridDim.x) * blockDim.x) {
    if (i < n) {
      int64_t a = g.row_ptr[i], b = g.row_ptr[i + 1];
      if (a > b || a < 0 || b > E) dev_flag(err, DEV_ERR_GRAPH);
      if (g.gid && (g.gid[i] < 0 || g.gid[i] >= g.n_global)) dev_flag(err, DEV_ERR_GRAPH);
    }
    if (i == 0 && (g.row_ptr[0] != 0 || g.row_ptr[n] != E)) dev_flag(err, DEV_ERR_GRAPH);
    if (i < E) {
      int32_t c = g.col[i], r = g.recv[i];
      if (c < 0 || c >= n || r < 0 || r >= n) dev_flag(err, DEV_ERR_GRAPH);
      else if (i < g.row_ptr[r] || i >= g.row_ptr[r + 1]) dev_flag(err, DEV_ERR_GRAPH);
      if (g.csc_perm) {
        int32_t q = g.csc_perm[i];
        if (q < 0 || q >= E) dev_flag(err, DEV_ERR_GRAPH);
      }
    }
  }
}

xmgn_status check_desc(const xmgn_model_desc* d) {
  if (!d) return fail(XMGN_ERR_ARG, "null model descriptor");
  if (d->H < 1 || d->L < 1 || d->in_node < 1 || d->out < 1 || d->out > 16 || d->fourier < 0 ||
      d->fourier > 4 || d->in_node + 6 * d->fourier > 32)
    return fail(XMGN_ERR_ARG, "model descriptor out of range (H=%d L=%d in=%d out=%d fourier=%d)", d->H, d->L,
                d->in_node, d->out, d->fourier);
  if (d->dtype == XMGN_FP32) {
    if (d->H % 32 || d->H > 512) return fail(XMGN_ERR_UNSUPPORTED, "fp32 path needs H %% 32 == 0, H <= 512");
  } else if (d->dtype == XMGN_BF16) {
    const ParamPlan p = make_plan(*d);
    if (!bf16_supported(p) && !wide_supported(p))
      return fail(XMGN_ERR_UNSUPPORTED, "bf16 path needs H = 128 (fused kernels) or H %% 32 == 0, H <= 512 (wide path)");
  } else {
    return fail(XMGN_ERR_ARG, "unknown dtype %d", d->dtype);
  }
  return XMGN_OK;
}

xmgn_status check_graph(const xmgn_graph* g) {
  if (!g) return fail(XMGN_ERR_ARG, "null graph");
  if (g->n_nodes < 1 || g->n_edges < 0 || g->n_nodes >= (int64_t(1) << 31))
    return fail(XMGN_ERR_ARG, "graph sizes out of range");
  if (!g->row_ptr || (g->n_edges > 0 && (!g->col || !g->recv || !g->csc_perm)))
    return fail(XMGN_ERR_ARG, "graph arrays row_ptr, col, recv, csc_perm are required (the last three when n_edges > 0)");
  if (g->n_norm < 1) return fail(XMGN_ERR_ARG, "n_norm must be >= 1");
  if (!g->gid && g->n_global != g->n_nodes) return fail(XMGN_ERR_ARG, "n_global must equal n_nodes when gid is NULL");
  if (g->gid && g->n_global < 1) return fail(XMGN_ERR_ARG, "n_global must be >= 1");
  return XMGN_OK;
}

}  // namespace
}  // namespace xmgn

using namespace xmgn;

namespace xmgn {
namespace diag {
// An mbarrier that nothing ever completes: the bounded wait gives up after
// about one second, flags the device error word and the kernel returns.
__global__ void wait_timeout_kernel(uint32_t* err) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_barrier_init();
  }
  __syncthreads();
  tc::mbar_wait(&bar, 0, err);
}
}  // namespace diag
}  // namespace xmgn

extern "C" {

const char* xmgn_last_error(void) { return g_err; }

int32_t xmgn_version(void) { return 10000; }

int64_t xmgn_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

xmgn_status xmgn_probe_enable(int32_t on) {
  ProbeState& P = probes();
  std::lock_guard<std::mutex> g(P.mu);
  P.on = on != 0;
  return XMGN_OK;
}

xmgn_status xmgn_probe_read(int32_t kind, int64_t* launches, double* total_ms, int32_t reset) {
  if (kind < 0 || kind >= PROBE_KINDS || !launches || !total_ms) return fail(XMGN_ERR_ARG, "bad probe query");
  ProbeState& P = probes();
  std::lock_guard<std::mutex> g(P.mu);
  double ms = 0.0;
  for (auto& e : P.used[kind]) {
    XMGN_CUDA(cudaEventSynchronize(e.second));
    float t = 0.f;
    XMGN_CUDA(cudaEventElapsedTime(&t, e.first, e.second));
    ms += t;
  }
  *launches = int64_t(P.used[kind].size());
  *total_ms = ms;
  if (reset) {
    for (auto& e : P.used[kind]) P.pool.push_back(e);
    P.used[kind].clear();
  }
  return XMGN_OK;
}

xmgn_status xmgn_selftest_wait_timeout(xmgn_stream stream) {
  uint32_t* w = device_error_word();
  if (!w) return fail(XMGN_ERR_CUDA, "no device error word (no CUDA device?)");
  xmgn::diag::wait_timeout_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(w);
  XMGN_LAUNCH_CHECK();
  return xmgn_check_device(stream);
}

xmgn_status xmgn_check_device(xmgn_stream stream) {
  uint32_t* w = device_error_word();
  if (!w) return fail(XMGN_ERR_CUDA, "no device error word (no CUDA device?)");
  uint32_t h = 0;
  XMGN_CUDA(cudaMemcpyAsync(&h, w, sizeof(h), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
  XMGN_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  if (h) XMGN_CUDA(cudaMemsetAsync(w, 0, sizeof(uint32_t), (cudaStream_t)stream));
  XMGN_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  if (h & DEV_ERR_TIMEOUT) return fail(XMGN_ERR_TIMEOUT, "a bounded device wait gave up (code 0x%x)", h);
  if (h & DEV_ERR_GRAPH) return fail(XMGN_ERR_GRAPH, "graph id out of range seen on the device (code 0x%x)", h);
  if (h & DEV_ERR_RANGE) return fail(XMGN_ERR_RANGE, "coordinate off the lattice (code 0x%x)", h);
  if (h & DEV_ERR_CAP) return fail(XMGN_ERR_WORKSPACE, "device capacity exceeded (code 0x%x)", h);
  return XMGN_OK;
}

xmgn_status xmgn_validate_graph(const xmgn_graph* g, xmgn_stream stream) {
  XMGN_TRY(check_graph(g));
  uint32_t* w = device_error_word();
  if (!w) return fail(XMGN_ERR_CUDA, "no device error word");
  XMGN_TRY(xmgn_check_device(stream));
  int64_t m = g->n_nodes + 1 > g->n_edges ? g->n_nodes + 1 : g->n_edges;
  validate_graph_kernel<<<grid_for(m, 256), 256, 0, (cudaStream_t)stream>>>(*g, w);
  XMGN_LAUNCH_CHECK();
  return xmgn_check_device(stream);
}

xmgn_status xmgn_build_knn_ws(int64_t N, int32_t k, size_t* ws_bytes) {
  if (!ws_bytes || N < 1 || k < 1) return fail(XMGN_ERR_ARG, "bad arguments");
  return build_knn_ws(N, k, ws_bytes);
}

xmgn_status xmgn_build_knn(const float* xyz, int64_t N, int32_t k, double lattice_scale, void* ws,
                           size_t ws_bytes, int32_t* nbr, int64_t* row_ptr, int32_t* col,
                           int32_t* recv, int32_t* csc_perm, int64_t E_cap, int64_t* E_out,
                           xmgn_stream stream) {
  return build_knn(xyz, N, k, lattice_scale, ws, ws_bytes, nbr, row_ptr, col, recv, csc_perm, E_cap,
                   E_out, (cudaStream_t)stream);
}

xmgn_status xmgn_build_multiscale_ws(int64_t N, int32_t n_levels, int32_t k, int32_t k_cross,
                                     size_t* ws_bytes) {
  if (!ws_bytes || N < 1 || k < 1 || k_cross < 1 || n_levels < 1) return fail(XMGN_ERR_ARG, "bad arguments");
  return build_multiscale_ws(N, n_levels, k, k_cross, ws_bytes);
}

xmgn_status xmgn_build_multiscale(const float* xyz, int64_t N, const int64_t* sizes, int32_t n_levels,
                                  int32_t k, int32_t k_cross, double lattice_scale, void* ws,
                                  size_t ws_bytes, int32_t* nbr, int64_t* row_ptr, int32_t* col,
                                  int32_t* recv, int32_t* csc_perm, int64_t E_cap, int64_t* E_out,
                                  xmgn_stream stream) {
  return build_multiscale(xyz, N, sizes, n_levels, k, k_cross, lattice_scale, ws, ws_bytes, nbr, row_ptr,
                          col, recv, csc_perm, E_cap, E_out, (cudaStream_t)stream);
}

xmgn_status xmgn_partition_halo_ws(int64_t N, int64_t E, int32_t P, size_t* ws_bytes) {
  if (!ws_bytes || N < 1 || P < 1) return fail(XMGN_ERR_ARG, "bad arguments");
  return partition_halo_ws(N, E, P, ws_bytes);
}

xmgn_status xmgn_partition_halo(const int64_t* row_ptr, const int32_t* col, int64_t N, int64_t E,
                                const float* xyz, double lattice_scale, int32_t P,
                                int32_t halo_hops, const int32_t* part_in, void* ws,
                                size_t ws_bytes, int32_t* part, int64_t* node_ptr,
                                int64_t* edge_ptr, int64_t* inner_cnt, int32_t* gid, uint8_t* hop,
                                int64_t* b_row_ptr, int32_t* b_col, int32_t* b_recv,
                                int32_t* b_csc_perm, int64_t cap_nodes, int64_t cap_edges,
                                xmgn_stream stream) {
  if (lattice_scale <= 0) lattice_scale = 2097152.0;
  return partition_halo(row_ptr, col, N, E, xyz, lattice_scale, P, halo_hops, part_in, ws, ws_bytes,
                        part, node_ptr, edge_ptr, inner_cnt, gid, hop, b_row_ptr, b_col, b_recv,
                        b_csc_perm, cap_nodes, cap_edges, (cudaStream_t)stream);
}

xmgn_status xmgn_partition_halo_emit(const int64_t* row_ptr, const int32_t* col, int64_t N, int64_t E,
                                     const float* xyz, double lattice_scale, int32_t P,
                                     int32_t halo_hops, const int32_t* part_in, void* ws,
                                     size_t ws_bytes, int32_t* part, int64_t* node_ptr,
                                     int64_t* edge_ptr, int64_t* inner_cnt, int32_t* gid, uint8_t* hop,
                                     int64_t* b_row_ptr, int32_t* b_col, int32_t* b_recv,
                                     int32_t* b_csc_perm, int64_t cap_nodes, int64_t cap_edges,
                                     xmgn_stream stream) {
  if (lattice_scale <= 0) lattice_scale = 2097152.0;
  return partition_halo(row_ptr, col, N, E, xyz, lattice_scale, P, halo_hops, part_in, ws, ws_bytes,
                        part, node_ptr, edge_ptr, inner_cnt, gid, hop, b_row_ptr, b_col, b_recv,
                        b_csc_perm, cap_nodes, cap_edges, (cudaStream_t)stream, true);
}

int64_t xmgn_param_count(const xmgn_model_desc* desc) {
  if (!desc || desc->H < 1 || desc->L < 0) return -1;
  return make_plan(*desc).total;
}

xmgn_status xmgn_model_ws(const xmgn_model_desc* desc, int64_t n_nodes, int64_t n_edges,
                          size_t* ws_bytes, size_t* ckpt_bytes) {
  XMGN_TRY(check_desc(desc));
  if (!ws_bytes || !ckpt_bytes || n_nodes < 1 || n_edges < 0) return fail(XMGN_ERR_ARG, "bad arguments");
  ParamPlan p = make_plan(*desc);
  if (desc->dtype == XMGN_FP32) f32_sizes(p, n_nodes, n_edges, ws_bytes, ckpt_bytes);
  else if (bf16_supported(p)) bf16_sizes(p, n_nodes, n_edges, ws_bytes, ckpt_bytes);
  else f32_sizes(p, n_nodes, n_edges, ws_bytes, ckpt_bytes, true);
  return XMGN_OK;
}

xmgn_status xmgn_forward(const xmgn_model_desc* desc, const float* params, const xmgn_graph* g,
                         const float* node_in, const float* xyz, const float* targets, float* y,
                         float* loss, void* ckpt, void* ws, size_t ws_bytes, xmgn_stream stream) {
  XMGN_TRY(check_desc(desc));
  XMGN_TRY(check_graph(g));
  if (!params || !node_in || !xyz || !ckpt || !ws) return fail(XMGN_ERR_ARG, "null pointer");
  ParamPlan p = make_plan(*desc);
  size_t need_ws = 0, need_ck = 0;
  XMGN_TRY(xmgn_model_ws(desc, g->n_nodes, g->n_edges, &need_ws, &need_ck));
  if (ws_bytes < need_ws) return fail(XMGN_ERR_WORKSPACE, "ws_bytes %zu < %zu", ws_bytes, need_ws);
  if (desc->dtype == XMGN_FP32 || !bf16_supported(p))
    return f32_forward(p, params, *g, node_in, xyz, targets, y, loss, ckpt, need_ck, ws, ws_bytes,
                       (cudaStream_t)stream, desc->dtype == XMGN_BF16);
  return bf16_forward(p, params, *g, node_in, xyz, targets, y, loss, ckpt, need_ck, ws, ws_bytes,
                      (cudaStream_t)stream);
}

xmgn_status xmgn_backward(const xmgn_model_desc* desc, const float* params, const xmgn_graph* g,
                          const float* node_in, const float* xyz, const float* targets,
                          const void* ckpt, float* dparams, float* dcomp, void* ws,
                          size_t ws_bytes, xmgn_stream stream) {
  XMGN_TRY(check_desc(desc));
  XMGN_TRY(check_graph(g));
  if (!params || !node_in || !xyz || !ckpt || !ws || !dparams || !targets)
    return fail(XMGN_ERR_ARG, "null pointer");
  ParamPlan p = make_plan(*desc);
  size_t need_ws = 0, need_ck = 0;
  XMGN_TRY(xmgn_model_ws(desc, g->n_nodes, g->n_edges, &need_ws, &need_ck));
  if (ws_bytes < need_ws) return fail(XMGN_ERR_WORKSPACE, "ws_bytes %zu < %zu", ws_bytes, need_ws);
  if (desc->dtype == XMGN_FP32 || !bf16_supported(p))
    return f32_backward(p, params, *g, node_in, xyz, targets, ckpt, need_ck, dparams, dcomp, ws,
                        ws_bytes, (cudaStream_t)stream, desc->dtype == XMGN_BF16);
  return bf16_backward(p, params, *g, node_in, xyz, targets, ckpt, need_ck, dparams, dcomp, ws,
                       ws_bytes, (cudaStream_t)stream);
}

xmgn_status xmgn_grad_accumulate(float* dst, float* comp, const float* src, int64_t n, xmgn_stream stream) {
  if (n < 0 || (n > 0 && (!dst || !src))) return fail(XMGN_ERR_ARG, "grad_accumulate: null pointer or n < 0");
  if (n == 0) return XMGN_OK;
  return accumulate_grad(dst, comp, src, n, reinterpret_cast<cudaStream_t>(stream));
}

xmgn_status xmgn_model_ws_offload(const xmgn_model_desc* desc, int64_t n_nodes, int64_t n_edges,
                                  size_t* ws_bytes, size_t* ckpt_bytes, size_t* host_bytes) {
  XMGN_TRY(check_desc(desc));
  if (desc->dtype != XMGN_BF16 || !bf16_supported(make_plan(*desc)))
    return fail(XMGN_ERR_UNSUPPORTED, "checkpoint offload needs the fused bf16 path (H = 128)");
  if (!ws_bytes || !ckpt_bytes || !host_bytes || n_nodes < 1 || n_edges < 0)
    return fail(XMGN_ERR_ARG, "bad arguments");
  bf16_sizes(make_plan(*desc), n_nodes, n_edges, ws_bytes, ckpt_bytes, true, host_bytes);
  return XMGN_OK;
}

static xmgn_status offload_sizes_ok(const xmgn_model_desc* desc, const xmgn_graph* g, size_t ws_bytes,
                                    size_t* ck) {
  size_t ws = 0, host = 0;
  XMGN_TRY(xmgn_model_ws_offload(desc, g->n_nodes, g->n_edges, &ws, ck, &host));
  if (ws_bytes < ws) return fail(XMGN_ERR_WORKSPACE, "ws_bytes %zu < %zu", ws_bytes, ws);
  return XMGN_OK;
}

xmgn_status xmgn_forward_offload(const xmgn_model_desc* desc, const float* params, const xmgn_graph* g,
                                 const float* node_in, const float* xyz, const float* targets, float* y,
                                 float* loss, void* ckpt, void* host_ckpt, void* ws, size_t ws_bytes,
                                 xmgn_stream stream) {
  XMGN_TRY(check_desc(desc));
  XMGN_TRY(check_graph(g));
  if (!params || !node_in || !xyz || !ckpt || !host_ckpt || !ws) return fail(XMGN_ERR_ARG, "null pointer");
  size_t ck = 0;
  XMGN_TRY(offload_sizes_ok(desc, g, ws_bytes, &ck));
  return bf16_forward(make_plan(*desc), params, *g, node_in, xyz, targets, y, loss, ckpt, ck, ws, ws_bytes,
                      (cudaStream_t)stream, host_ckpt);
}

xmgn_status xmgn_backward_offload(const xmgn_model_desc* desc, const float* params, const xmgn_graph* g,
                                  const float* node_in, const float* xyz, const float* targets,
                                  const void* ckpt, const void* host_ckpt, float* dparams, float* dcomp,
                                  void* ws, size_t ws_bytes, xmgn_stream stream) {
  XMGN_TRY(check_desc(desc));
  XMGN_TRY(check_graph(g));
  if (!params || !node_in || !xyz || !ckpt || !host_ckpt || !ws || !dparams || !targets)
    return fail(XMGN_ERR_ARG, "null pointer");
  size_t ck = 0;
  XMGN_TRY(offload_sizes_ok(desc, g, ws_bytes, &ck));
  return bf16_backward(make_plan(*desc), params, *g, node_in, xyz, targets, ckpt, ck, dparams, dcomp, ws,
                       ws_bytes, (cudaStream_t)stream, host_ckpt);
}

}  // extern "C"
