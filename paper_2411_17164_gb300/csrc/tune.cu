// Launch-shape autotuner: table, timing hooks and the xmgn_autotune /
// xmgn_tune_* entry points (see tune.cuh and include/xmgn.h).
//
// xmgn_autotune tunes one launch class at a time: a warm-up forward + backward
// step per candidate (CUDA events around the class's launches show whether the
// model launches it at all), the step captured as a CUDA graph per candidate,
// then `iters` rounds of one timed graph replay per candidate, interleaved; it
// keeps the candidate with the least summed step time, and the default
// (candidate 0) unless another wins by more than 0.3 %.  The other classes
// keep their current choice meanwhile (coordinate descent, one pass).
#include <map>
#include <mutex>
#include <set>
#include <vector>

#include "tune.cuh"

namespace xmgn {

namespace {

constexpr int kNCand[TUNE_NOPS] = {2, 2, 4, 2, 3};
constexpr double kTuneMargin = 0.003;  // 0.3 % of the step
const char* const kName[TUNE_NOPS] = {"edge_fwd_order", "edge_bwd_order", "seg_sums", "tn_grid", "edge_bwd_tiles"};

struct TuneState {
  std::mutex mu;
  std::map<std::pair<int, int>, int> table;  // (op, bucket) -> candidate
  std::set<int> seen[TUNE_NOPS];             // buckets launched since the last tune_forget_seen
  int force_op = -1, force_c = 0;
  int time_op = -1;
  std::vector<cudaEvent_t> ev;  // begin/end pairs of the timed launches
  size_t nev = 0;
};

TuneState& st() {
  static TuneState s;
  return s;
}

}  // namespace

int tune_ncand(int op) { return op >= 0 && op < TUNE_NOPS ? kNCand[op] : 0; }
const char* tune_name(int op) { return op >= 0 && op < TUNE_NOPS ? kName[op] : nullptr; }

int tune_bucket(int64_t rows) {
  int b = 0;
  for (uint64_t r = rows > 0 ? uint64_t(rows) : 0u; r; r >>= 1) ++b;
  return b;
}

int tune_choice(int op, int64_t rows) {
  TuneState& s = st();
  std::lock_guard<std::mutex> g(s.mu);
  const int b = tune_bucket(rows);
  s.seen[op].insert(b);
  if (s.force_op == op) return s.force_c;
  auto it = s.table.find({op, b});
  return it == s.table.end() ? 0 : it->second;
}

int tune_get(int op, int64_t rows) {
  TuneState& s = st();
  std::lock_guard<std::mutex> g(s.mu);
  auto it = s.table.find({op, tune_bucket(rows)});
  return it == s.table.end() ? 0 : it->second;
}

void tune_set(int op, int bucket, int choice) {
  TuneState& s = st();
  std::lock_guard<std::mutex> g(s.mu);
  s.table[{op, bucket}] = choice;
}

void tune_clear() {
  TuneState& s = st();
  std::lock_guard<std::mutex> g(s.mu);
  s.table.clear();
}

void tune_entries(void (*fn)(int, int, int, void*), void* ctx) {
  TuneState& s = st();
  std::vector<std::pair<std::pair<int, int>, int>> copy;
  {
    std::lock_guard<std::mutex> g(s.mu);
    copy.assign(s.table.begin(), s.table.end());
  }
  for (auto& e : copy) fn(e.first.first, e.first.second, e.second, ctx);
}

void tune_begin(int op, cudaStream_t stream) {
  TuneState& s = st();
  std::lock_guard<std::mutex> g(s.mu);
  if (s.time_op != op) return;
  while (s.ev.size() < s.nev + 2) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    s.ev.push_back(e);
  }
  cudaEventRecord(s.ev[s.nev], stream);
}

void tune_end(int op, cudaStream_t stream) {
  TuneState& s = st();
  std::lock_guard<std::mutex> g(s.mu);
  if (s.time_op != op || s.ev.size() < s.nev + 2) return;
  cudaEventRecord(s.ev[s.nev + 1], stream);
  s.nev += 2;
}

void tune_force(int op, int choice) {
  TuneState& s = st();
  std::lock_guard<std::mutex> g(s.mu);
  s.force_op = op;
  s.force_c = choice;
}

void tune_time(int op) {
  TuneState& s = st();
  std::lock_guard<std::mutex> g(s.mu);
  s.time_op = op;
  s.nev = 0;
}

xmgn_status tune_elapsed(float* ms, int* launches) {
  TuneState& s = st();
  std::lock_guard<std::mutex> g(s.mu);
  float total = 0.f;
  for (size_t i = 0; i + 1 < s.nev; i += 2) {
    float t = 0.f;
    XMGN_CUDA(cudaEventElapsedTime(&t, s.ev[i], s.ev[i + 1]));
    total += t;
  }
  *ms = total;
  *launches = int(s.nev / 2);
  return XMGN_OK;
}

void tune_commit(int op, int choice) {
  TuneState& s = st();
  std::lock_guard<std::mutex> g(s.mu);
  for (int b : s.seen[op]) s.table[{op, b}] = choice;
}

void tune_forget_seen() {
  TuneState& s = st();
  std::lock_guard<std::mutex> g(s.mu);
  for (auto& x : s.seen) x.clear();
}

}  // namespace xmgn

using namespace xmgn;

extern "C" {

int32_t xmgn_tune_op_count(void) { return TUNE_NOPS; }

const char* xmgn_tune_op_name(int32_t op) { return tune_name(op); }

int32_t xmgn_tune_candidates(int32_t op) { return tune_ncand(op); }

int32_t xmgn_tune_get(int32_t op, int64_t rows) {
  if (op < 0 || op >= TUNE_NOPS) return -1;
  return tune_get(op, rows);
}

xmgn_status xmgn_tune_set(int32_t op, int64_t rows, int32_t choice) {
  if (op < 0 || op >= TUNE_NOPS || choice < 0 || choice >= tune_ncand(op) || rows < 1)
    return fail(XMGN_ERR_ARG, "xmgn_tune_set: op %d, choice %d, rows %lld", op, choice, (long long)rows);
  tune_set(op, tune_bucket(rows), choice);
  return XMGN_OK;
}

xmgn_status xmgn_tune_clear(void) {
  tune_clear();
  return XMGN_OK;
}

xmgn_status xmgn_tune_save(const char* path) {
  if (!path) return fail(XMGN_ERR_ARG, "xmgn_tune_save: null path");
  FILE* f = fopen(path, "w");
  if (!f) return fail(XMGN_ERR_ARG, "xmgn_tune_save: cannot open %s", path);
  fprintf(f, "xmgn-tune 1\n");
  tune_entries([](int op, int b, int c, void* ctx) { fprintf(static_cast<FILE*>(ctx), "%s %d %d\n", tune_name(op), b, c); },
               f);
  const bool ok = fclose(f) == 0;
  return ok ? XMGN_OK : fail(XMGN_ERR_ARG, "xmgn_tune_save: write failed for %s", path);
}

xmgn_status xmgn_tune_load(const char* path) {
  if (!path) return fail(XMGN_ERR_ARG, "xmgn_tune_load: null path");
  FILE* f = fopen(path, "r");
  if (!f) return fail(XMGN_ERR_ARG, "xmgn_tune_load: cannot open %s", path);
  char name[64];
  int version = 0;
  if (fscanf(f, "xmgn-tune %d", &version) != 1 || version != 1) {
    fclose(f);
    return fail(XMGN_ERR_ARG, "xmgn_tune_load: %s is not a tuning table", path);
  }
  std::vector<std::pair<std::pair<int, int>, int>> rows;
  int b = 0, c = 0;
  while (fscanf(f, "%63s %d %d", name, &b, &c) == 3) {
    int op = -1;
    for (int i = 0; i < TUNE_NOPS; ++i)
      if (std::string(name) == kName[i]) op = i;
    if (op < 0 || c < 0 || c >= kNCand[op] || b < 0 || b > 64) {
      fclose(f);
      return fail(XMGN_ERR_ARG, "xmgn_tune_load: bad entry '%s %d %d' in %s", name, b, c, path);
    }
    rows.push_back({{op, b}, c});
  }
  const bool eof = feof(f) != 0;
  fclose(f);
  if (!eof) return fail(XMGN_ERR_ARG, "xmgn_tune_load: unreadable entry in %s", path);
  for (auto& r : rows) tune_set(r.first.first, r.first.second, r.second);
  return XMGN_OK;
}

xmgn_status xmgn_autotune(const xmgn_model_desc* desc, const float* params, const xmgn_graph* g,
                          const float* node_in, const float* xyz, const float* targets, void* ckpt, void* ws,
                          size_t ws_bytes, float* dparams, int32_t iters, xmgn_stream stream) {
  if (!desc || !targets || !dparams || iters < 1) return fail(XMGN_ERR_ARG, "xmgn_autotune: bad arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  auto step_on = [&](cudaStream_t q) -> xmgn_status {
    XMGN_TRY(xmgn_forward(desc, params, g, node_in, xyz, targets, nullptr, nullptr, ckpt, ws, ws_bytes, q));
    return xmgn_backward(desc, params, g, node_in, xyz, targets, ckpt, dparams, nullptr, ws, ws_bytes, q);
  };
  XMGN_CUDA(cudaStreamSynchronize(s));
  // The timed steps replay a CUDA graph of the step, as a training loop does
  // (back-to-back kernels, no launch gaps), on a stream of the tuner's own
  // (capture needs one other than the legacy default stream); where capture
  // is refused they run as direct launches on the caller's stream.
  cudaStream_t cs = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  xmgn_status rc = XMGN_OK;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&ev[0]) != cudaSuccess ||
      cudaEventCreate(&ev[1]) != cudaSuccess)
    rc = fail(XMGN_ERR_CUDA, "xmgn_autotune: stream or event creation failed");
  auto sync = [&](cudaStream_t q) -> xmgn_status {
    if (cudaStreamSynchronize(q) != cudaSuccess)
      return fail(XMGN_ERR_CUDA, "xmgn_autotune: %s", cudaGetErrorString(cudaGetLastError()));
    return XMGN_OK;
  };
  // the step as a graph; false (and nothing launched) when capture is refused
  auto capture = [&](cudaGraphExec_t* ex) -> bool {
    cudaGraph_t gr = nullptr;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    const xmgn_status r = step_on(cs);
    const cudaError_t e = cudaStreamEndCapture(cs, &gr);
    bool ok = r == XMGN_OK && e == cudaSuccess && gr != nullptr &&
              cudaGraphInstantiate(ex, gr, 0) == cudaSuccess;
    if (gr) cudaGraphDestroy(gr);
    if (!ok) cudaGetLastError();
    return ok;
  };
  bool use_graph = rc == XMGN_OK;
  for (int op = 0; op < TUNE_NOPS && rc == XMGN_OK; ++op) {
    const int nc = kNCand[op];
    std::vector<double> total(nc, 0.0);
    std::vector<cudaGraphExec_t> ex(nc, nullptr);
    tune_forget_seen();
    // one warm-up step per candidate; it also shows whether this model launches the class
    bool launched = true;
    for (int c = 0; c < nc && rc == XMGN_OK && launched; ++c) {
      tune_force(op, c);
      tune_time(op);
      rc = step_on(s);
      if (rc == XMGN_OK) rc = sync(s);
      float ms = 0.f;
      int n = 0;
      if (rc == XMGN_OK) rc = tune_elapsed(&ms, &n);
      tune_time(-1);
      launched = n > 0;
    }
    for (int c = 0; c < nc && rc == XMGN_OK && launched && use_graph; ++c) {
      tune_force(op, c);  // the choice is made while the launches are recorded
      use_graph = capture(&ex[c]);
    }
    // timed rounds, candidates interleaved so that clock drift affects every
    // candidate alike; the whole step is timed, since the way one kernel deals
    // its tiles also changes what the next kernel finds in L2
    cudaStream_t q = use_graph ? cs : s;
    for (int i = 0; i <= iters && rc == XMGN_OK && launched; ++i)  // round 0: warm-up of the graphs
      for (int c = 0; c < nc && rc == XMGN_OK; ++c) {
        tune_force(op, c);
        if (cudaEventRecord(ev[0], q) != cudaSuccess) rc = fail(XMGN_ERR_CUDA, "xmgn_autotune: event record failed");
        if (rc == XMGN_OK) {
          if (use_graph) {
            if (cudaGraphLaunch(ex[c], q) != cudaSuccess) rc = fail(XMGN_ERR_CUDA, "xmgn_autotune: graph launch failed");
          } else {
            rc = step_on(q);
          }
        }
        if (rc == XMGN_OK && cudaEventRecord(ev[1], q) != cudaSuccess)
          rc = fail(XMGN_ERR_CUDA, "xmgn_autotune: event record failed");
        if (rc == XMGN_OK) rc = sync(q);
        float ms = 0.f;
        if (rc == XMGN_OK && cudaEventElapsedTime(&ms, ev[0], ev[1]) != cudaSuccess)
          rc = fail(XMGN_ERR_CUDA, "xmgn_autotune: event timing failed");
        if (i > 0) total[c] += ms;
      }
    for (auto e : ex)
      if (e) cudaGraphExecDestroy(e);
    tune_force(-1, 0);
    if (rc != XMGN_OK || !launched) continue;
    int best = 0;
    for (int c = 1; c < nc; ++c)
      if (total[c] < total[best]) best = c;
    // another candidate replaces the default only when it wins by more than
    // the run-to-run spread of a step
    if (best != 0 && total[best] > total[0] * (1.0 - kTuneMargin)) best = 0;
    tune_commit(op, best);
  }
  for (auto e : ev)
    if (e) cudaEventDestroy(e);
  if (cs) {
    cudaStreamSynchronize(cs);
    cudaStreamDestroy(cs);
  }
  if (rc == XMGN_OK) XMGN_CUDA(cudaStreamSynchronize(s));
  return rc;
}

}  // extern "C"
