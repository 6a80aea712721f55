// Batched problems: every item of a batch is compiled into its program of
// phases (tk_program.h); the phases of all items that fall in the same
// schedule slot (mode step and sketch / power step t / finish) are merged into
// one launch per (position, step kind, tile class), and the whole run is
// optionally captured into one CUDA graph.
#include <algorithm>
#include <cstring>
#include <vector>

#include "tk_program.h"

namespace tk {

struct Batch {
  int count = 0;
  int dev = 0;
  std::vector<Problem> probs;
  std::vector<LaunchRec> recs;
  unsigned char* ws = nullptr;       // all problems' workspaces
  size_t ws_bytes = 0;
  unsigned char* tables = nullptr;   // job tables
  size_t table_bytes = 0;
  std::vector<size_t> state_off;     // each problem's ItemState (offset in ws)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t last = nullptr;
  bool ran = false;
};

static tk_status enqueue_run(Batch* b, cudaStream_t st, bool profile) {
  for (int i = 0; i < b->count; ++i)
    TK_TRY(cudaMemsetAsync(b->ws + b->state_off[i], 0, sizeof(ItemState), st));
  for (const auto& r : b->recs) TK_TRY(issue(r, st, profile));
  return TK_OK;
}

static void free_batch(Batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->ws) cudaFree(b->ws);
  if (b->tables) cudaFree(b->tables);
  delete b;
}

}  // namespace tk

using namespace tk;

extern "C" {

struct tk_batch_s {
  Batch* b;
};

tk_status tucker_batch_create(const tk_item* items, int count, tk_shift rule, int use_graph,
                              tk_batch* out) {
  if (!items || count < 1 || !out) return TK_EINVAL;
  *out = nullptr;
  if (rule != TK_SHIFT_PAPER && rule != TK_SHIFT_NONE) return TK_EINVAL;
  Batch* b = new Batch;
  b->count = count;
  cudaGetDevice(&b->dev);
  b->probs.resize(count);
  std::vector<size_t> off(count);
  size_t tot = 0;
  for (int i = 0; i < count; ++i) {
    if (items[i].A.dtype != items[0].A.dtype) {
      delete b;
      return TK_EINVAL;
    }
    tk_status s = problem_plan(items[i], rule, &b->probs[i]);
    if (s != TK_OK) {
      delete b;
      return s;
    }
    off[i] = tot;
    tot += al(b->probs[i].ws_bytes);
  }
  b->ws_bytes = tot;
  cudaError_t e = cudaMalloc((void**)&b->ws, std::max<size_t>(tot, 256));
  if (e != cudaSuccess) {
    b->ws = nullptr;
    free_batch(b);
    return from_cuda(e);
  }
  std::vector<int> slots;
  b->state_off.resize(count);
  for (int i = 0; i < count; ++i) {
    problem_build(items[i], b->ws + off[i], &b->probs[i]);
    b->state_off[i] = (size_t)((unsigned char*)b->probs[i].state - b->ws);
    slots.insert(slots.end(), b->probs[i].slot.begin(), b->probs[i].slot.end());
  }
  std::sort(slots.begin(), slots.end());
  slots.erase(std::unique(slots.begin(), slots.end()), slots.end());
  // every problem's phase of one schedule slot -> merged launches (a
  // problem's slots ascend with its phases, so its order is kept)
  std::vector<unsigned char> blob;
  for (int sl : slots) {
    std::vector<const Op*> ops;
    for (int i = 0; i < count; ++i) {
      const Problem& pr = b->probs[i];
      for (size_t ph = 0; ph < pr.prog.size(); ++ph)
        if (pr.slot[ph] == sl)
          for (const Op& o : pr.prog[ph]) ops.push_back(&o);
    }
    merge_ops(ops, blob, b->recs);
  }
  b->table_bytes = blob.size();
  e = cudaMalloc((void**)&b->tables, std::max<size_t>(blob.size(), 256));
  if (e == cudaSuccess) e = cudaMemcpy(b->tables, blob.data(), blob.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    free_batch(b);
    return from_cuda(e);
  }
  resolve(b->recs, b->tables);
  batch_kernels_init();
  if (use_graph) {
    cudaStream_t cs;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      free_batch(b);
      return from_cuda(e);
    }
    tk_status s = TK_OK;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      count_kernels(-(int)b->recs.size());   // counted per run instead
      s = enqueue_run(b, cs, false);
      cudaError_t e2 = cudaStreamEndCapture(cs, &b->graph);
      if (s == TK_OK && e2 != cudaSuccess) s = from_cuda(e2);
      if (s == TK_OK) s = from_cuda(cudaGraphInstantiate(&b->exec, b->graph, 0));
    } else {
      s = from_cuda(e);
    }
    cudaStreamDestroy(cs);
    if (s != TK_OK) {
      free_batch(b);
      return s;
    }
  }
  *out = new tk_batch_s{b};
  return TK_OK;
}

tk_status tucker_batch_run(tk_batch h, void* stream) {
  if (!h || !h->b) return TK_EINVAL;
  Batch* b = h->b;
  cudaStream_t st = (cudaStream_t)stream;
  b->last = st;
  b->ran = true;
  if (b->exec) {
    count_kernels((int)b->recs.size());
    TK_TRY(cudaGraphLaunch(b->exec, st));
    return TK_OK;
  }
  return enqueue_run(b, st, true);
}

tk_status tucker_batch_wait(tk_batch h, int* status) {
  if (!h || !h->b) return TK_EINVAL;
  Batch* b = h->b;
  if (!b->ran) return TK_EINVAL;
  TK_TRY(cudaStreamSynchronize(b->last));
  tk_status first = TK_OK;
  for (int i = 0; i < b->count; ++i) {
    int s = 0;
    TK_TRY(cudaMemcpy(&s, b->ws + b->state_off[i] + offsetof(ItemState, status), sizeof(int),
                      cudaMemcpyDeviceToHost));
    if (status) status[i] = s;
    if (s != 0 && first == TK_OK) first = (tk_status)s;
  }
  return first;
}

tk_status tucker_batch_info(tk_batch h, int64_t* launches, size_t* device_bytes) {
  if (!h || !h->b) return TK_EINVAL;
  if (launches) *launches = (int64_t)h->b->recs.size();
  if (device_bytes) *device_bytes = h->b->ws_bytes + h->b->table_bytes;
  return TK_OK;
}

tk_status tucker_batch_destroy(tk_batch h) {
  if (!h) return TK_EINVAL;
  if (h->b) free_batch(h->b);
  delete h;
  return TK_OK;
}

tk_status tucker_batch_rsthosvd(const tk_item* items, int count, tk_shift rule, void* stream) {
  tk_batch h = nullptr;
  tk_status s = tucker_batch_create(items, count, rule, 0, &h);
  if (s != TK_OK) return s;
  s = tucker_batch_run(h, stream);
  tk_status w = s == TK_OK ? tucker_batch_wait(h, nullptr) : s;
  tucker_batch_destroy(h);
  return w;
}

}  // extern "C"
