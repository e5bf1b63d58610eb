// Shared host/device utilities of libxmgn (errors, workspace carving, launch
// helpers).  Everything here is internal; the public surface is include/xmgn.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <string>

#include "../../include/xmgn.h"

namespace xmgn {

// ---------------------------------------------------------------- errors
void set_error(const char* fmt, ...);
xmgn_status fail(xmgn_status s, const char* fmt, ...);

#define XMGN_CUDA(call)                                                                  \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return ::xmgn::fail(XMGN_ERR_CUDA, "%s:%d %s: %s", __FILE__, __LINE__, #call,        \
                          cudaGetErrorString(e_));                                       \
  } while (0)

#define XMGN_TRY(expr)                     \
  do {                                     \
    xmgn_status s_ = (expr);               \
    if (s_ != XMGN_OK) return s_;          \
  } while (0)

// Every kernel launch is followed by exactly one XMGN_LAUNCH_CHECK(), which
// also counts the launch (xmgn_launch_count).
#define XMGN_LAUNCH_CHECK()          \
  do {                               \
    ::xmgn::count_launch();          \
    XMGN_CUDA(cudaGetLastError());   \
  } while (0)

void count_launch();

// CUDA-event probes around the launches of one kernel class (xmgn_probe_*).
enum ProbeKind : int {
  PROBE_EDGE_FWD = 0,
  PROBE_EDGE_BWD = 1,
  PROBE_NODE_FWD = 2,
  PROBE_NODE_BWD = 3,
  PROBE_WIDE_GEMM = 4,
  PROBE_KINDS = 5
};
void probe_begin(int kind, cudaStream_t s);
void probe_end(int kind, cudaStream_t s);

// Device error word (one per device, lives in api.cu).  Kernels OR a code
// into it instead of trapping; xmgn_check_device reads and clears it.
enum : uint32_t {
  DEV_ERR_RANGE = 1u,    // coordinate off the lattice
  DEV_ERR_GRAPH = 2u,    // id out of range in a graph array
  DEV_ERR_TIMEOUT = 4u,  // bounded wait gave up
  DEV_ERR_CAP = 8u,      // an output capacity was exceeded
};
uint32_t* device_error_word();  // device address for the current device

// ---------------------------------------------------------------- workspace
// Bump allocator over a caller-provided buffer; all carve-outs 256-B aligned.
struct Arena {
  char* base = nullptr;
  size_t cap = 0;
  size_t used = 0;
  bool dry = false;  // size-only pass
  template <class T>
  T* take(size_t count) {
    size_t off = (used + 255) & ~size_t(255);
    used = off + count * sizeof(T);
    if (dry) return nullptr;
    return reinterpret_cast<T*>(base + off);
  }
  bool ok() const { return dry || used <= cap; }
};

inline int num_sms() {
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!cached[dev]) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = n > 0 ? n : 1;
  }
  return cached[dev];
}

inline unsigned grid_for(int64_t n, int threads, int64_t cap_blocks = 0) {
  int64_t b = (n + threads - 1) / threads;
  if (cap_blocks <= 0) cap_blocks = int64_t(num_sms()) * 32;
  if (b > cap_blocks) b = cap_blocks;
  if (b < 1) b = 1;
  return unsigned(b);
}

// ---------------------------------------------------------------- scans
// Exclusive prefix sum of n int32 (or int64) values into int64 out[0..n]
// (out[n] = total).  Uses `tmp` scratch of scan_tmp_elems(n) int64.
size_t scan_tmp_elems(int64_t n);
xmgn_status exclusive_scan_i32(const int32_t* in, int64_t* out, int64_t n, int64_t* tmp,
                               cudaStream_t s);
xmgn_status exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* tmp,
                               cudaStream_t s);

// ---------------------------------------------------------------- device helpers
__device__ __forceinline__ void dev_flag(uint32_t* err, uint32_t code) {
  if (err) atomicOr(err, code);
}

}  // namespace xmgn
