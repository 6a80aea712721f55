// Autotuner of the split-K counts of the FP32 CUDA-core contractions (the
// batching pattern's "tile shapes and split-K chosen by an autotuner").
//
// The FP32 products that run on the CUDA cores split their contraction over
// CTAs and sum the partials in a fixed order: Y = X_(k) W splits the
// columns of the unfolding (`xb32_shape`), the TTM W = X_(k)^T B splits the
// rows when there are few column tiles (`xtb32_shape`).  The fixed
// heuristics target about three CTAs per SM for ONE problem; in a batch,
// where every problem's blocks share one persistent launch, fewer splits
// can be faster.  The tuner keeps a process-wide table from a shape class
// (kind, n_k, output width, column count rounded up to a power of two) to a
// split count.  Both the single-problem calls and the batch planner read
// their split counts through `tune_splits`, so a batch item and its single
// call keep identical summation orders (bitwise-equal results).
//
// Measurements happen only in tucker_tune_batch: it plans and times the
// batch once per candidate scale of the heuristic (2, 1, 1/2, ..., 1/16),
// recording the split count every shape class takes under that scale, and
// stores the fastest candidate's counts.  Planning never measures.
#include <atomic>
#include <cstdio>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "tk_common.cuh"
#include "tk_internal.h"
#include "tk_plan.h"

namespace tk {
namespace {

typedef std::tuple<int, int64_t, int, int64_t> TuneKey;   // kind, n, width, column bucket

std::mutex g_mu;
std::map<TuneKey, int> g_table;
std::atomic<bool> g_on{false};

// a tuning run in progress on this thread: the candidate scale (splits x
// 2^-shift, shift = -1 doubles) and the classes it met
thread_local bool t_active = false;
thread_local int t_shift = 0;
thread_local std::map<TuneKey, int>* t_seen = nullptr;

int64_t bucket(int64_t cols) {
  int64_t b = 1;
  while (b < cols) b <<= 1;
  return b;
}

}  // namespace

int tune_splits(int kind, int64_t n, int width, int64_t cols, int heuristic, int maxs) {
  const TuneKey key(kind, n, width, bucket(cols));
  maxs = std::max(1, maxs);
  if (t_active) {
    int s = t_shift >= 0 ? heuristic >> t_shift : heuristic << (-t_shift);
    s = std::min(std::max(1, s), maxs);
    if (t_seen) t_seen->emplace(key, s);
    return s;
  }
  if (!g_on.load(std::memory_order_relaxed)) return heuristic;
  std::lock_guard<std::mutex> lock(g_mu);
  auto it = g_table.find(key);
  if (it == g_table.end()) return heuristic;
  return std::min(std::max(1, it->second), maxs);
}

}  // namespace tk

using namespace tk;

extern "C" {

tk_status tucker_tune_enable(int on) {
  g_on.store(on != 0);
  return TK_OK;
}

tk_status tucker_tune_clear(void) {
  std::lock_guard<std::mutex> lock(g_mu);
  g_table.clear();
  return TK_OK;
}

tk_status tucker_tune_entries(int* count) {
  if (!count) return TK_EINVAL;
  std::lock_guard<std::mutex> lock(g_mu);
  *count = (int)g_table.size();
  return TK_OK;
}

tk_status tucker_tune_save(const char* path) {
  if (!path) return TK_EINVAL;
  std::lock_guard<std::mutex> lock(g_mu);
  FILE* f = std::fopen(path, "w");
  if (!f) return TK_EINVAL;
  std::fprintf(f, "tucker-tune 1\n");
  for (const auto& e : g_table)
    std::fprintf(f, "%d %lld %d %lld %d\n", std::get<0>(e.first),
                 (long long)std::get<1>(e.first), std::get<2>(e.first),
                 (long long)std::get<3>(e.first), e.second);
  const bool ok = std::fclose(f) == 0;
  return ok ? TK_OK : TK_EINVAL;
}

tk_status tucker_tune_load(const char* path) {
  if (!path) return TK_EINVAL;
  FILE* f = std::fopen(path, "r");
  if (!f) return TK_EINVAL;
  int version = 0;
  if (std::fscanf(f, "tucker-tune %d", &version) != 1 || version != 1) {
    std::fclose(f);
    return TK_EINVAL;
  }
  std::map<TuneKey, int> rows;
  int kind, width, splits;
  long long n, cb;
  int got;
  while ((got = std::fscanf(f, "%d %lld %d %lld %d", &kind, &n, &width, &cb, &splits)) == 5) {
    if (kind < 0 || n < 1 || width < 1 || cb < 1 || splits < 1) {
      std::fclose(f);
      return TK_EINVAL;
    }
    rows[TuneKey(kind, n, width, cb)] = splits;
  }
  const bool clean = got == EOF;
  std::fclose(f);
  if (!clean) return TK_EINVAL;
  std::lock_guard<std::mutex> lock(g_mu);
  for (const auto& e : rows) g_table[e.first] = e.second;
  return TK_OK;
}

tk_status tucker_tune_batch(const tk_item* items, int count, tk_shift rule, void* stream,
                            double* best_ms, double* base_ms, int* best_shift) {
  if (!items || count < 1) return TK_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  static const int kShifts[] = {0, -1, 1, 2, 3, 4};
  double best = -1.0, base = -1.0;
  int best_s = 0;
  std::map<TuneKey, int> best_seen;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  TK_TRY(cudaEventCreate(&e0));
  cudaError_t ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) {
    cudaEventDestroy(e0);
    return from_cuda(ce);
  }
  tk_status res = TK_OK;
  for (int shift : kShifts) {
    std::map<TuneKey, int> seen;
    t_active = true;
    t_shift = shift;
    t_seen = &seen;
    tk_batch b = nullptr;
    tk_status s = tucker_batch_create(items, count, rule, 1, &b);
    t_active = false;
    t_seen = nullptr;
    if (s != TK_OK) {
      res = s;
      break;
    }
    float ms = 0.f;
    for (int w = 0; w < 2 && s == TK_OK; ++w) s = tucker_batch_run(b, stream);
    if (s == TK_OK) s = from_cuda(cudaEventRecord(e0, st));
    for (int r = 0; r < 3 && s == TK_OK; ++r) s = tucker_batch_run(b, stream);
    if (s == TK_OK) s = from_cuda(cudaEventRecord(e1, st));
    if (s == TK_OK) s = tucker_batch_wait(b, nullptr);
    if (s == TK_OK) s = from_cuda(cudaEventElapsedTime(&ms, e0, e1));
    tucker_batch_destroy(b);
    if (s != TK_OK) {
      res = s;
      break;
    }
    const double per = ms / 3.0;
    if (shift == 0) base = per;
    if (best < 0.0 || per < best) {
      best = per;
      best_s = shift;
      best_seen.swap(seen);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (res != TK_OK) return res;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    for (const auto& e : best_seen) g_table[e.first] = e.second;
  }
  if (best_ms) *best_ms = best;
  if (base_ms) *base_ms = base;
  if (best_shift) *best_shift = best_s;
  return TK_OK;
}

}  // extern "C"
