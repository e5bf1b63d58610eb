// Launch-shape autotuner: table, timing hooks and the xmgn_autotune /
// xmgn_tune_* entry points (see tune.cuh and include/xmgn.h).
//
// xmgn_autotune tunes one launch class at a time: for each candidate it runs
// a warm-up forward + backward step with that candidate forced, then `iters`
// steps during which CUDA events bracket every launch of the class, and keeps
// the candidate with the least summed device time.  The other classes keep
// their current choice meanwhile (coordinate descent, one pass).
#include <map>
#include <mutex>
#include <set>
#include <vector>

#include "tune.cuh"

namespace xmgn {

namespace {

constexpr int kNCand[TUNE_NOPS] = {2, 2, 4, 2, 3};
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
  auto step = [&]() -> xmgn_status {
    XMGN_TRY(xmgn_forward(desc, params, g, node_in, xyz, targets, nullptr, nullptr, ckpt, ws, ws_bytes, stream));
    return xmgn_backward(desc, params, g, node_in, xyz, targets, ckpt, dparams, nullptr, ws, ws_bytes, stream);
  };
  XMGN_CUDA(cudaStreamSynchronize(s));
  xmgn_status rc = XMGN_OK;
  for (int op = 0; op < TUNE_NOPS && rc == XMGN_OK; ++op) {
    int best = -1;
    float best_ms = 0.f;
    tune_forget_seen();
    for (int c = 0; c < kNCand[op] && rc == XMGN_OK; ++c) {
      tune_force(op, c);
      rc = step();  // warm-up with this candidate
      if (rc != XMGN_OK) break;
      tune_time(op);
      for (int i = 0; i < iters && rc == XMGN_OK; ++i) rc = step();
      if (rc != XMGN_OK) break;
      if (cudaStreamSynchronize(s) != cudaSuccess) {
        rc = fail(XMGN_ERR_CUDA, "xmgn_autotune: %s", cudaGetErrorString(cudaGetLastError()));
        break;
      }
      float ms = 0.f;
      int n = 0;
      rc = tune_elapsed(&ms, &n);
      tune_time(-1);
      if (rc != XMGN_OK || n == 0) break;  // the class is not launched by this model
      if (best < 0 || ms < best_ms) {
        best = c;
        best_ms = ms;
      }
    }
    tune_time(-1);
    tune_force(-1, 0);
    if (rc == XMGN_OK && best >= 0) tune_commit(op, best);
  }
  if (rc == XMGN_OK) XMGN_CUDA(cudaStreamSynchronize(s));
  return rc;
}

}  // extern "C"
