// Launch-shape autotuner: the tunable launches, their candidate shapes, and
// the table the launch sites read.  A choice is kept per (launch, size
// bucket), the bucket being the bit length of the launch's row count, so one
// table serves graphs of different sizes.  xmgn_autotune (api) fills the
// table by timing every candidate inside real forward + backward steps.
#pragma once

#include "common.cuh"

namespace xmgn {

enum TuneOp : int {
  TUNE_EDGE_FWD_ORDER = 0,  // edge forward: 128-edge tiles dealt to CTAs round-robin (0) or in contiguous runs (1)
  TUNE_EDGE_BWD_ORDER = 1,  // edge backward: the same two tile orders
  TUNE_SEG_SUMS = 2,        // receiver/sender sums of dZ1: {32, 16} lanes per node x {16, 8} blocks per SM
  TUNE_TN_GRID = 3,         // node-level X^T dY products: CTAs = SMs (0) or SMs / 2 (1)
  TUNE_EDGE_BWD_TILES = 4,  // edge backward: one 128-edge tile on 16 warps (0), two tiles in flight (1), one tile on 32 warps (2)
  TUNE_NOPS = 5
};

int tune_ncand(int op);
const char* tune_name(int op);
// The candidate a launch of `op` over `rows` rows uses (0 when untuned).
int tune_choice(int op, int64_t rows);
// Timing hooks around a tunable launch; they record events only while the
// tuner is timing `op`.
void tune_begin(int op, cudaStream_t s);
void tune_end(int op, cudaStream_t s);

// Tuner control (used by xmgn_autotune).
void tune_force(int op, int choice);  // op < 0: no override
void tune_time(int op);               // op < 0: stop timing
xmgn_status tune_elapsed(float* ms, int* launches);  // sum over the recorded launches (after a sync)
void tune_commit(int op, int choice);  // store `choice` for every size bucket `op` was launched with
void tune_forget_seen();

// Table access.
int tune_get(int op, int64_t rows);
void tune_set(int op, int bucket, int choice);
int tune_bucket(int64_t rows);
void tune_clear();
// Visits every entry in (op, bucket) order.
void tune_entries(void (*fn)(int op, int bucket, int choice, void* ctx), void* ctx);

}  // namespace xmgn
