// Entry points of the two model paths behind xmgn_forward / xmgn_backward.
#pragma once

#include "model.cuh"

namespace xmgn {

// FP32 plain path (CUDA cores); with tc the wide BF16 path (the same layer
// structure with every product on the tensor cores in bf16).
void f32_sizes(const ParamPlan& p, int64_t n, int64_t E, size_t* ws, size_t* ckpt, bool tc = false);
xmgn_status f32_forward(const ParamPlan& p, const float* P, const xmgn_graph& g,
                        const float* node_in, const float* xyz, const float* targets, float* y,
                        float* loss, void* ckpt, size_t ckpt_bytes, void* ws, size_t ws_bytes,
                        cudaStream_t s, bool tc = false);
xmgn_status f32_backward(const ParamPlan& p, const float* P, const xmgn_graph& g,
                         const float* node_in, const float* xyz, const float* targets,
                         const void* ckpt, size_t ckpt_bytes, float* dparams, float* dcomp,
                         void* ws, size_t ws_bytes, cudaStream_t s, bool tc = false);
// Widths the wide BF16 path takes (those the fused kernels do not).
inline bool wide_supported(const ParamPlan& p) { return p.H % 32 == 0 && p.H <= 512; }

// BF16 tensor-core path (tcgen05).
bool bf16_supported(const ParamPlan& p);
// With offload the edge-state checkpoints live in a host buffer of *host
// bytes (host_e16) and the device keeps a two-slot ring.
void bf16_sizes(const ParamPlan& p, int64_t n, int64_t E, size_t* ws, size_t* ckpt, bool offload = false,
                size_t* host = nullptr);
xmgn_status bf16_forward(const ParamPlan& p, const float* P, const xmgn_graph& g,
                         const float* node_in, const float* xyz, const float* targets, float* y,
                         float* loss, void* ckpt, size_t ckpt_bytes, void* ws, size_t ws_bytes,
                         cudaStream_t s, void* host_e16 = nullptr);
xmgn_status bf16_backward(const ParamPlan& p, const float* P, const xmgn_graph& g,
                          const float* node_in, const float* xyz, const float* targets,
                          const void* ckpt, size_t ckpt_bytes, float* dparams, float* dcomp,
                          void* ws, size_t ws_bytes, cudaStream_t s, const void* host_e16 = nullptr);

// Graph construction and partitioning.
xmgn_status build_knn_ws(int64_t N, int32_t k, size_t* ws_bytes);
xmgn_status build_knn(const float* xyz, int64_t N, int32_t k, double scale, void* ws,
                      size_t ws_bytes, int32_t* nbr_out, int64_t* row_ptr, int32_t* col,
                      int32_t* recv, int32_t* csc_perm, int64_t E_cap, int64_t* E_out,
                      cudaStream_t s);
xmgn_status build_multiscale_ws(int64_t N, int32_t n_levels, int32_t k, int32_t k_cross, size_t* ws_bytes);
xmgn_status build_multiscale(const float* xyz, int64_t N, const int64_t* sizes, int32_t n_levels, int32_t k,
                             int32_t k_cross, double scale, void* ws, size_t ws_bytes, int32_t* nbr_out,
                             int64_t* row_ptr, int32_t* col, int32_t* recv, int32_t* csc_perm, int64_t E_cap,
                             int64_t* E_out, cudaStream_t s);
xmgn_status partition_halo_ws(int64_t N, int64_t E, int32_t P, size_t* ws_bytes);
xmgn_status partition_halo(const int64_t* row_ptr, const int32_t* col, int64_t N, int64_t E,
                           const float* xyz, double scale, int32_t P, int32_t L,
                           const int32_t* part_in, void* ws, size_t ws_bytes, int32_t* part_out,
                           int64_t* node_ptr, int64_t* edge_ptr, int64_t* inner_cnt, int32_t* gid,
                           uint8_t* hop, int64_t* b_row_ptr, int32_t* b_col, int32_t* b_recv,
                           int32_t* b_csc_perm, int64_t cap_nodes, int64_t cap_edges,
                           cudaStream_t s, bool resume = false);

}  // namespace xmgn
