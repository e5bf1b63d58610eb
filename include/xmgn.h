/*
 * xmgn.h -- C-ABI of the GB300-native X-MeshGraphNet message-passing library.
 *
 * The library implements the data-parallel hot path of X-MeshGraphNet
 * (arXiv 2411.17164): kNN graph construction from a point cloud (Sec. III-B),
 * halo partitioning (Sec. III-A "Graph Partitioning"), and the MeshGraphNet
 * encode-process-decode message passing of eqs. (1)-(4), forward and backward
 * (Sec. II-B..II-D, III-D), with per-layer activation checkpointing and
 * gradient aggregation across partitions (Sec. III-A "Gradient Aggregation").
 *
 * Conventions (apply to every entry point):
 *  - Pointers are DEVICE pointers unless a parameter is marked "host".
 *  - The caller owns every buffer; the library never allocates or frees
 *    caller-visible memory.  Scratch space is passed as (ws, ws_bytes) and is
 *    sized by the matching *_ws query.
 *  - Calls are asynchronous on `stream` except where a host-visible result is
 *    returned (documented per call); those synchronise `stream` once.
 *  - Every call returns xmgn_status; no exception crosses the ABI.  On error,
 *    xmgn_last_error() returns a thread-local message.  Invalid arguments are
 *    rejected on the host before any launch.
 *  - Node ids are int32 (N < 2^31), edge offsets int64.  Graphs are
 *    symmetric (every (i <- j) has its (j <- i)), so the sender-major (CSC)
 *    view shares row_ptr with the receiver-major CSR.
 *  - Results are deterministic: no floating-point atomics; repeated calls
 *    and CUDA-graph replays give bit-identical outputs.
 *  - Device-side waits are bounded; a wait that gives up makes the call
 *    report XMGN_ERR_TIMEOUT on the next host check (xmgn_check_device).
 */
#ifndef XMGN_H
#define XMGN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* xmgn_stream; /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
  XMGN_OK = 0,
  XMGN_ERR_ARG = 1,       /* bad argument (null pointer, size, unsupported shape) */
  XMGN_ERR_RANGE = 2,     /* a coordinate lies outside the integer lattice range */
  XMGN_ERR_GRAPH = 3,     /* malformed graph (non-monotone row_ptr, id out of range) */
  XMGN_ERR_WORKSPACE = 4, /* ws / output capacity too small (required size reported) */
  XMGN_ERR_CUDA = 5,      /* a CUDA runtime call failed */
  XMGN_ERR_TIMEOUT = 6,   /* a bounded device-side wait gave up */
  XMGN_ERR_UNSUPPORTED = 7
} xmgn_status;

typedef enum { XMGN_FP32 = 0, XMGN_BF16 = 1 } xmgn_dtype;

/* Thread-local description of the last error (never NULL). */
const char* xmgn_last_error(void);
/* Library version (major*10000 + minor*100 + patch). */
int32_t xmgn_version(void);
/* Diagnostic (no paper counterpart): runs one kernel whose mbarrier wait can
 * never complete.  The bounded wait gives up after about one second, flags
 * the device error word and the kernel returns, so the call synchronises
 * `stream` and returns XMGN_ERR_TIMEOUT with the context still usable.  It
 * shows that a stuck wait ends in an error status, not a hang. */
xmgn_status xmgn_selftest_wait_timeout(xmgn_stream stream);
/* Reads and clears the device error word written by bounded waits and by
 * in-kernel checks of ids; synchronises `stream`. */
xmgn_status xmgn_check_device(xmgn_stream stream);

/* ------------------------------------------------------------------------
 * kNN graph construction (Sec. III-B "K-Nearest Neighbor Connectivity")
 *
 * Each point is connected to its k nearest other points.  Distances are
 * exact: coordinates are mapped to the integer lattice q = rint(x * s)
 * (round half to even, s = lattice_scale, a power of two, default 2^21) and
 * compared by the int64 squared distance; ties go to the smaller index; a
 * point is never its own neighbour; coincident points are allowed.  |q| must
 * stay below 2^24 (|x| < 8 at the default scale), else XMGN_ERR_RANGE.
 *
 * The kNN relation is then symmetrised (edge (i <- j) iff j in kNN(i) or
 * i in kNN(j), no duplicates) and emitted as receiver-major CSR with senders
 * ascending in each row.
 *
 *  xyz       [N,3] float32, row-major.
 *  nbr       [N,k] int32 out, nearest first (nullable).
 *  row_ptr   [N+1] int64 out; col [E] int32 out (senders); recv [E] int32 out
 *            (receiver of each edge, nullable); csc_perm [E] int32 out
 *            (nullable): CSR positions of the edges listed sender-major,
 *            receivers ascending, so that csc_perm[row_ptr[j] .. row_ptr[j+1])
 *            are the edges leaving j.
 *  E_cap     capacity of col/recv/csc_perm; 2*N*k always suffices.
 *  E_out     host out: number of directed edges.  Synchronises `stream`.
 *            If E > E_cap, E_out is set and XMGN_ERR_WORKSPACE returned.
 * ---------------------------------------------------------------------- */
xmgn_status xmgn_build_knn_ws(int64_t N, int32_t k, size_t* ws_bytes /*host*/);
xmgn_status xmgn_build_knn(const float* xyz, int64_t N, int32_t k, double lattice_scale,
                           void* ws, size_t ws_bytes, int32_t* nbr, int64_t* row_ptr,
                           int32_t* col, int32_t* recv, int32_t* csc_perm, int64_t E_cap,
                           int64_t* E_out /*host*/, xmgn_stream stream);

/* ------------------------------------------------------------------------
 * Multi-scale graph (Sec. III-C "Multi-Scale Graph Generation")
 *
 * The points are nested levels: level l is the first sizes[l] points, so
 * each level is a subset of the next finer one.  Edges: the kNN relation of
 * every level among its own points (k neighbours, as in xmgn_build_knn),
 * plus a link from every point that first appears in level l >= 1 to its
 * k_cross nearest points of level l-1 (same exact lattice distances and
 * tie rule); the union is symmetrised and emitted exactly as by
 * xmgn_build_knn.
 *
 *  sizes     host [n_levels] int64, strictly increasing, sizes[n_levels-1] == N,
 *            sizes[0] > k, sizes[0] >= k_cross.  1 <= n_levels <= 16.
 *  nbr       [N, n_levels*k + (n_levels > 1 ? k_cross : 0)] int32 out
 *            (nullable): slots [l*k, l*k+k) hold the level-l neighbours of a
 *            point of level l, the last k_cross slots its coarser-level
 *            links; -1 where a slot does not apply.
 *  E_cap     2*N*(n_levels*k + k_cross) always suffices.
 *  Other arguments and errors as for xmgn_build_knn; synchronises `stream`.
 * ---------------------------------------------------------------------- */
xmgn_status xmgn_build_multiscale_ws(int64_t N, int32_t n_levels, int32_t k, int32_t k_cross,
                                     size_t* ws_bytes /*host*/);
xmgn_status xmgn_build_multiscale(const float* xyz, int64_t N, const int64_t* sizes /*host*/,
                                  int32_t n_levels, int32_t k, int32_t k_cross, double lattice_scale,
                                  void* ws, size_t ws_bytes, int32_t* nbr, int64_t* row_ptr,
                                  int32_t* col, int32_t* recv, int32_t* csc_perm, int64_t E_cap,
                                  int64_t* E_out /*host*/, xmgn_stream stream);

/* ------------------------------------------------------------------------
 * Halo partitioning (Sec. III-A "Graph Partitioning", "Message Passing
 * Across Partitions")
 *
 * Splits the graph into P parts and surrounds each with a halo of
 * `halo_hops` hops (set equal to the number of message-passing layers, so
 * that every inner node's computational graph is complete).  The paper uses
 * METIS; this library uses recursive coordinate bisection: a set of n points
 * destined for P parts is split on the axis of largest lattice extent (x, y,
 * z order on ties) after the floor(n*floor(P/2)/P) smallest points in
 * (coordinate, id) order, which receive part ids [base, base+floor(P/2)).
 * If part_in is given (int32 [N], values in [0,P), or -1 for a node that is
 * inner in no part and can only appear in halos) it is used instead.
 *
 * The P induced subgraphs (inner U halo, every edge with both ends inside)
 * are concatenated into one block-diagonal "batch" graph.  Within part p the
 * nodes are: inner nodes by ascending global id, then halo nodes by (hop,
 * global id).  Each batch row lists its senders in ascending GLOBAL id, so a
 * receiver sums its messages in the same order as in the full graph.
 *
 * Two-call protocol: with gid == NULL only the host arrays node_ptr,
 * edge_ptr, inner_cnt are filled; a second call with capacities
 * cap_nodes >= node_ptr[P], cap_edges >= edge_ptr[P] fills the device arrays.
 * Both calls synchronise `stream`.
 *
 * xmgn_partition_halo_emit: the second call of that protocol without
 * repeating the first's work (partitioning, halo search, sort, degrees): same
 * arguments as xmgn_partition_halo, called right after a gid == NULL call
 * with the same inputs, the same ws (untouched in between) and the host
 * arrays that call filled; gid, hop, b_row_ptr, b_col, b_recv required.  The
 * sizing call leaves a stamp in ws (sizes, hops, part_in given or not); a
 * mismatch is rejected with XMGN_ERR_ARG before any device array is
 * written, and a completed emit clears it.  Synchronises `stream`.
 *
 *  part      [N] int32 out: part id of each node (nullable).
 *  node_ptr  host [P+1] int64 out: batch node range of part p.
 *  edge_ptr  host [P+1] int64 out: batch edge range of part p.
 *  inner_cnt host [P]  int64 out: inner nodes of part p (batch nodes
 *            node_ptr[p] .. node_ptr[p]+inner_cnt[p]-1 are the inner ones).
 *  gid [n] int32 out: global id of each batch node; hop [n] uint8 out
 *  (0 = inner); b_row_ptr [n+1] int64, b_col [e] int32, b_recv [e] int32,
 *  b_csc_perm [e] int32: batch graph in the layout of xmgn_build_knn (the
 *  sender-major order lists receivers by ascending global id).
 * ---------------------------------------------------------------------- */
xmgn_status xmgn_partition_halo_ws(int64_t N, int64_t E, int32_t P, size_t* ws_bytes /*host*/);
xmgn_status xmgn_partition_halo(const int64_t* row_ptr, const int32_t* col, int64_t N, int64_t E,
                                const float* xyz, double lattice_scale, int32_t P,
                                int32_t halo_hops, const int32_t* part_in, void* ws,
                                size_t ws_bytes, int32_t* part, int64_t* node_ptr /*host*/,
                                int64_t* edge_ptr /*host*/, int64_t* inner_cnt /*host*/,
                                int32_t* gid, uint8_t* hop, int64_t* b_row_ptr, int32_t* b_col,
                                int32_t* b_recv, int32_t* b_csc_perm, int64_t cap_nodes,
                                int64_t cap_edges, xmgn_stream stream);
xmgn_status xmgn_partition_halo_emit(const int64_t* row_ptr, const int32_t* col, int64_t N, int64_t E,
                                     const float* xyz, double lattice_scale, int32_t P,
                                     int32_t halo_hops, const int32_t* part_in, void* ws,
                                     size_t ws_bytes, int32_t* part, int64_t* node_ptr /*host*/,
                                     int64_t* edge_ptr /*host*/, int64_t* inner_cnt /*host*/,
                                     int32_t* gid, uint8_t* hop, int64_t* b_row_ptr, int32_t* b_col,
                                     int32_t* b_recv, int32_t* b_csc_perm, int64_t cap_nodes,
                                     int64_t cap_edges, xmgn_stream stream);

/* ------------------------------------------------------------------------
 * Model (Sec. II-B..II-D eqs. 1-4, Sec. III-D; MLP form: Linear, SiLU,
 * Linear, LayerNorm; processor updates are residual; decoder has no LN)
 *
 *   h0 = MLP_ne(node_in)            e0 = MLP_ee([x_j - x_i, |x_j - x_i|])
 *   for l in 0..L-1:
 *     m_ij = MLP_e^l([h_i, h_j, e_ij])   (eq. 1; i receiver, j sender)
 *     e_ij <- e_ij + m_ij
 *     a_i  = sum_j m_ij                  (eq. 2)
 *     h_i  <- h_i + MLP_n^l([h_i, a_i])  (eq. 3)
 *   y = MLP_d(h)
 *   loss = sum over inner nodes and outputs of (y - t)^2 / (out * n_norm)
 *
 * MLP(z) = LN(W2 SiLU(W1 z + b1) + b2); LN per row over the output
 * features, biased variance, eps 1e-5, then gamma, beta.
 *
 * Parameter layout: one float32 vector, MLPs in the order node encoder,
 * edge encoder, for l = 0..L-1 (edge MLP l, node MLP l), decoder.  Each MLP
 * stores W1 [in][H] row-major (z W1), b1 [H], W2 [H][out] row-major, b2 [out]
 * and, unless it is the decoder, gamma [out], beta [out].  Inputs: node
 * encoder in_node, edge encoder 4, edge MLP 3H as [h_i; h_j; e_ij], node MLP
 * 2H as [h_i; a_i], decoder H.  Outputs are H except the decoder (out).
 *
 * dtype XMGN_FP32: every product and state in float32 on CUDA cores; H a
 * multiple of 32, up to 512.
 * dtype XMGN_BF16: MLP products in bf16 x bf16 -> fp32 on the tensor cores;
 * LayerNorm statistics, aggregation sums, loss and parameter-gradient sums in
 * fp32.  H = 128: the fused tcgen05 kernels; edge states e stored bf16, node
 * states h kept in fp32 with a bf16 copy for the products.  Other H (a
 * multiple of 32, up to 512, e.g. the paper's 512): the wide path, every
 * product on this library's tcgen05 GEMM with bf16 copies of the operands
 * (no library GEMM), all states fp32; checkpoint offload
 * is not available there (XMGN_ERR_UNSUPPORTED).  Any other H:
 * XMGN_ERR_UNSUPPORTED.
 * ---------------------------------------------------------------------- */
typedef struct {
  int32_t H;       /* hidden width */
  int32_t L;       /* processor layers */
  int32_t in_node; /* node input features read from node_in */
  int32_t out;     /* outputs per node (<= 16) */
  int32_t dtype;   /* xmgn_dtype */
  int32_t fourier; /* Fourier frequencies F in [0, 4] appended to the node
                      inputs by the node encoder itself (Sec. IV-A/IV-D):
                      for f = 0..F-1, sin then cos of 2^(f+1) pi x_c for the
                      three coordinates c of xyz; the encoder then reads
                      in_node + 6F <= 32 features (the paper: 6 + 18 = 24) */
} xmgn_model_desc;

/* A graph the model runs on: a full graph, or a batch of halo partitions.
 * Inputs (node_in, xyz, targets) and outputs (y) are indexed by GLOBAL id,
 * gid[b] for batch node b (identity if gid == NULL).  A graph may have no
 * edges (then col, recv and csc_perm may be NULL and every message is 0). */
typedef struct {
  int64_t n_nodes;         /* nodes of this graph (batch nodes) */
  int64_t n_edges;         /* directed edges */
  const int64_t* row_ptr;  /* [n_nodes+1] receiver-major CSR (also CSC pointer) */
  const int32_t* col;      /* [n_edges] sender of each edge */
  const int32_t* recv;     /* [n_edges] receiver of each edge */
  const int32_t* csc_perm; /* [n_edges] edges leaving each node, see xmgn_build_knn */
  const int32_t* gid;      /* [n_nodes] global id (NULL = identity) */
  const uint8_t* hop;      /* [n_nodes] 0 = inner (owns its loss and output), NULL = all inner */
  int64_t n_global;        /* rows of node_in / xyz / targets / y */
  int64_t n_norm;          /* loss normaliser (nodes of the whole graph) */
} xmgn_graph;

/* Checks a graph on the device: row_ptr monotone with row_ptr[0] = 0 and
 * row_ptr[n] = E, every col/recv id in [0, n) and recv consistent with
 * row_ptr, csc_perm entries in [0, E), gid in [0, n_global).  Returns
 * XMGN_ERR_GRAPH on violation.  Synchronises `stream`.  (xmgn_forward does
 * not re-validate, so that it stays asynchronous and capturable.) */
xmgn_status xmgn_validate_graph(const xmgn_graph* g, xmgn_stream stream);

int64_t xmgn_param_count(const xmgn_model_desc* desc);
/* Scratch and checkpoint sizes for a graph of n_nodes / n_edges. */
xmgn_status xmgn_model_ws(const xmgn_model_desc* desc, int64_t n_nodes, int64_t n_edges,
                          size_t* ws_bytes /*host*/, size_t* ckpt_bytes /*host*/);

/* Forward pass.  params [P] float32.  node_in [n_global, in_node], xyz
 * [n_global, 3].  targets [n_global, out] (nullable: no loss).  y
 * [n_global, out] out (nullable): rows of inner nodes are written, each by
 * its owning partition.  loss: device float32 scalar out (overwritten;
 * nullable).  ckpt: per-layer checkpoints (h^l, e^l, a^l; on the BF16 path
 * also the node projections h^l [W1_r | W1_s] of each edge MLP) consumed by
 * xmgn_backward; must stay untouched between the two calls. */
xmgn_status xmgn_forward(const xmgn_model_desc* desc, const float* params, const xmgn_graph* g,
                         const float* node_in, const float* xyz, const float* targets, float* y,
                         float* loss, void* ckpt, void* ws, size_t ws_bytes, xmgn_stream stream);

/* Backward pass of the loss of the matching xmgn_forward call (which must
 * have been given targets).  Recomputes each layer's activations from the
 * checkpoints (activation checkpointing, Sec. IV-C) and ADDS the parameter
 * gradient into dparams [P] float32.  If dcomp [P] is non-NULL the addition
 * is Neumaier-compensated with dcomp as the running compensation, so that
 * gradients of many partitions or batches (Sec. III-A "Gradient
 * Aggregation") sum in fixed order with fp32 storage; the caller zeroes
 * dparams and dcomp before the first call and adds dcomp at the end. */
xmgn_status xmgn_backward(const xmgn_model_desc* desc, const float* params, const xmgn_graph* g,
                          const float* node_in, const float* xyz, const float* targets,
                          const void* ckpt, float* dparams, float* dcomp, void* ws,
                          size_t ws_bytes, xmgn_stream stream);

/* Fixed-order, compensated gradient sum (Sec. III-A "Gradient Aggregation":
 * the gradients of all partitions are summed before the update).  Adds
 * src [n] float32 into dst [n] float32 element by element; if comp [n] is
 * non-NULL the addition is Neumaier-compensated exactly as in xmgn_backward
 * (the rounding error of each addition is added into comp, so dst + comp
 * carries the sum to about twice fp32 precision).  Summing the per-rank or
 * per-partition gradients one call at a time in a fixed order gives the same
 * bits on every rank.  dst and src may not overlap; asynchronous on
 * `stream`. */
xmgn_status xmgn_grad_accumulate(float* dst, float* comp, const float* src, int64_t n, xmgn_stream stream);

/* Activation-checkpoint offload (Sec. IV-E: activation checkpointing with
 * offloading).  BF16 path only.  The per-layer edge-state checkpoints e^l,
 * the bulk of the checkpoint memory (L * n_edges * H bf16), are kept in a
 * caller-owned host buffer of host_bytes instead of device memory: the
 * forward copies e^l out on an internal copy stream as soon as layer l has
 * read it, the backward copies it back one layer ahead of its use; the
 * device keeps three edge-state slots and recomputes the node projections
 * instead of keeping them.  host_ckpt must be page-locked (e.g.
 * cudaHostAlloc) so that the copies are asynchronous.  ckpt_bytes is the
 * (smaller) device checkpoint size for these calls; results equal those of
 * xmgn_forward / xmgn_backward bit for bit.  Both calls order all their
 * work, copies included, on `stream` (the copy stream joins it before they
 * return), so they can be captured into a CUDA graph. */
xmgn_status xmgn_model_ws_offload(const xmgn_model_desc* desc, int64_t n_nodes, int64_t n_edges,
                                  size_t* ws_bytes /*host*/, size_t* ckpt_bytes /*host*/,
                                  size_t* host_bytes /*host*/);
xmgn_status xmgn_forward_offload(const xmgn_model_desc* desc, const float* params, const xmgn_graph* g,
                                 const float* node_in, const float* xyz, const float* targets, float* y,
                                 float* loss, void* ckpt, void* host_ckpt, void* ws, size_t ws_bytes,
                                 xmgn_stream stream);
xmgn_status xmgn_backward_offload(const xmgn_model_desc* desc, const float* params, const xmgn_graph* g,
                                  const float* node_in, const float* xyz, const float* targets,
                                  const void* ckpt, const void* host_ckpt, float* dparams, float* dcomp,
                                  void* ws, size_t ws_bytes, xmgn_stream stream);

/* ------------------------------------------------------------------------
 * Masked MSE loss without any allocation (the paper has no counterpart: it
 * is a packaging of the inner-node loss for callers that cannot allocate).
 *
 * Some callers may not allocate device memory at all: code running inside a
 * framework whose allocator already owns the whole device, real-time or
 * embedded hosts whose memory is fixed before the run starts, and callers
 * that are not allowed to synchronise, which cudaMalloc/cudaFree may do.
 * This call computes the same quantity as the loss of xmgn_forward, from a
 * caller-held prediction array, using no caller workspace and calling no
 * cudaMalloc, cudaFree or allocating library routine: its scratch (one
 * partial sum per 1024 rows) lives in a fixed 16 KB device array inside the
 * library, which every GPU that loads the library keeps until the process
 * exits.
 *
 *  y        [n, out] float32 predictions, one row per node of the graph.
 *  targets  [n_global, out] float32, row gid[i] (or i if gid is NULL).
 *  gid      [n] int32 (nullable); hop [n] uint8 (nullable): rows with
 *           hop != 0 are halo rows and do not count.
 *  loss     device float32 scalar out:
 *           sum over counted rows and outputs of (y - t)^2 / (out * n_norm).
 *  Limits: 1 <= n <= 4,194,304 (XMGN_ERR_WORKSPACE beyond, with a message),
 *           1 <= out <= 16.
 *  Asynchronous on `stream`.  The first call on a device looks up the
 *  array's device address (cudaGetSymbolAddress, cached per device), so make
 *  that first call before any stream capture.  All calls share the array and
 *  it keeps the last call's contents; each call writes every partial it reads
 *  before reading it, so nothing needs clearing, but calls that overlap on
 *  the GPU (different streams, or different host threads on one device) race
 *  on it: order them.
 * ---------------------------------------------------------------------- */
xmgn_status xmgn_mse_loss_static(const float* y, int64_t n, int32_t out, const float* targets,
                                 const int32_t* gid, const uint8_t* hop, int64_t n_norm, float* loss,
                                 xmgn_stream stream);

/* ------------------------------------------------------------------------
 * Instrumentation (no counterpart in the paper; used to measure the
 * roofline fraction of the kernels).
 *
 * xmgn_launch_count: number of kernel launches the library has issued since
 *   it was loaded (all threads, all devices).
 * xmgn_probe_enable(on): while on, every launch of the fused edge/node MLP
 *   kernels and of the wide path's GEMM is bracketed by a pair of CUDA events
 *   recorded on the launch stream.  Events are created by the library and
 *   reused.
 * xmgn_probe_read(kind, launches, total_ms, reset): synchronises with the
 *   recorded events of one kernel class and returns how many launches were
 *   bracketed and their summed device time in milliseconds; reset != 0
 *   forgets them.  kind: XMGN_PROBE_*.
 * ---------------------------------------------------------------------- */
typedef enum {
  XMGN_PROBE_EDGE_FWD = 0, /* fused edge-MLP forward (eq. 1, residual)            */
  XMGN_PROBE_EDGE_BWD = 1, /* fused edge-MLP backward (recompute + LN/SiLU bwd)   */
  XMGN_PROBE_NODE_FWD = 2, /* fused node-MLP forward (eq. 3, residual)            */
  XMGN_PROBE_NODE_BWD = 3, /* fused node-MLP backward                             */
  XMGN_PROBE_WIDE_GEMM = 4 /* tcgen05 GEMM of the wide path (hidden width != 128) */
} xmgn_probe_kind;
int64_t xmgn_launch_count(void);
xmgn_status xmgn_probe_enable(int32_t on);
xmgn_status xmgn_probe_read(int32_t kind, int64_t* launches /*host*/, double* total_ms /*host*/,
                            int32_t reset);

/* ------------------------------------------------------------------------
 * Launch-shape autotuner (no paper counterpart: it serves the batched
 * persistent launches, whose best launch shapes depend on the graph).
 *
 * Tunable launch classes (op ids 0 .. xmgn_tune_op_count()-1, names from
 * xmgn_tune_op_name), each with xmgn_tune_candidates(op) launch shapes:
 *   0 edge_fwd_order  fused edge forward: 128-edge tiles dealt to the
 *                     persistent CTAs round-robin (0) or in contiguous runs (1)
 *   1 edge_bwd_order  fused edge backward: the same two orders
 *   2 seg_sums        receiver/sender sums of dZ1: {32, 16} lanes per node
 *                     x {16, 8} blocks per SM (candidates 0..3)
 *   3 tn_grid         node-level X^T dY products: one CTA per SM (0) or one
 *                     per two SMs (1)
 *   4 edge_bwd_tiles  fused edge backward: one 128-edge tile in flight per
 *                     CTA on 16 warps (0), two tiles in flight (1: two groups
 *                     of 8 warps, weight-gradient products in fixed tile
 *                     order), or one tile on 32 warps (2: half the columns per
 *                     thread)
 * A choice is stored per (op, size bucket), the bucket being the bit length
 * of the launch's row count; launches without an entry use candidate 0.
 * Results depend on the choices only through the order of floating-point
 * sums; with fixed choices every call is deterministic.
 *
 * xmgn_autotune: for one op at a time, runs for every candidate one warm-up
 *   forward + backward of the given model and graph, then `iters` rounds of
 *   one timed step per candidate (candidates interleaved, CUDA events around
 *   the whole step, replayed as a CUDA graph captured on a stream the tuner
 *   creates, or launched directly where capture is refused), and stores for
 *   every size bucket the op was launched with the candidate with the least
 *   summed step time -- candidate 0 unless another is faster by more than
 *   0.3 %.  Arguments as for xmgn_forward / xmgn_backward; dparams
 *   [P] receives the gradients of all these steps (scratch); targets are
 *   required.  Synchronises `stream`.  Not to be called while other threads
 *   launch work of this library.  An FP32 model has nothing to tune.
 * xmgn_tune_get / xmgn_tune_set: read / write the choice for an op at a row
 *   count (get returns -1 for an unknown op).
 * xmgn_tune_save / xmgn_tune_load: the table as text ("xmgn-tune 1", then
 *   one "name bucket choice" line per entry); load merges into the table and
 *   rejects unknown names or out-of-range choices without changing it.
 * xmgn_tune_clear: forgets every choice.
 * ---------------------------------------------------------------------- */
int32_t xmgn_tune_op_count(void);
const char* xmgn_tune_op_name(int32_t op);
int32_t xmgn_tune_candidates(int32_t op);
xmgn_status xmgn_autotune(const xmgn_model_desc* desc, const float* params, const xmgn_graph* g,
                          const float* node_in, const float* xyz, const float* targets, void* ckpt, void* ws,
                          size_t ws_bytes, float* dparams, int32_t iters, xmgn_stream stream);
int32_t xmgn_tune_get(int32_t op, int64_t rows);
xmgn_status xmgn_tune_set(int32_t op, int64_t rows, int32_t choice);
xmgn_status xmgn_tune_save(const char* path);
xmgn_status xmgn_tune_load(const char* path);
xmgn_status xmgn_tune_clear(void);

#ifdef __cplusplus
}
#endif
#endif /* XMGN_H */
