// Host-side planning shared by the single-problem entry points and the
// work-list (batched / serving) paths: the per-call plan of Algorithms 2/3
// and the carving of its device workspace.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "tk_internal.h"
#include "tucker.h"

namespace tk {

inline tk_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return TK_OK;
  if (e == cudaErrorMemoryAllocation) return TK_ENOMEM;
  return TK_ECUDA;
}

#define TK_TRY(expr)                              \
  do {                                            \
    cudaError_t e_ = (expr);                      \
    if (e_ != cudaSuccess) return from_cuda(e_);  \
  } while (0)

inline size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

// Bump allocator; with base == nullptr it only measures.
struct Arena {
  unsigned char* base = nullptr;
  size_t off = 0;
  void* take(size_t bytes) {
    const size_t o = offset(bytes);
    return base ? base + o : nullptr;
  }
  size_t offset(size_t bytes) {
    off = al(off);
    const size_t o = off;
    off += al(bytes);
    return o;
  }
};

inline View view_of(const std::vector<int64_t>& dims, int k) {
  View v;
  v.P = 1;
  for (int m = 0; m < k; ++m) v.P *= dims[m];
  v.n = dims[k];
  v.S = 1;
  for (size_t m = k + 1; m < dims.size(); ++m) v.S *= dims[m];
  return v;
}

inline int64_t prod(const std::vector<int64_t>& d) {
  int64_t p = 1;
  for (auto x : d) p *= x;
  return p;
}

inline bool valid_tensor(const tk_tensor* A, bool allow_bf16) {
  if (!A || A->d < 1 || A->d > TK_MAX_D || !A->data) return false;
  if (!(A->dtype == TK_F64 || A->dtype == TK_F32 || (allow_bf16 && A->dtype == TK_BF16)))
    return false;
  int64_t tot = 1;
  for (int k = 0; k < A->d; ++k) {
    if (A->n[k] < 1) return false;
    if (tot > INT64_MAX / A->n[k]) return false;
    tot *= A->n[k];
  }
  return true;
}

inline XType xtype(tk_dtype d) { return d == TK_F64 ? X_F64 : (d == TK_F32 ? X_F32 : X_BF16); }

// ---------------------------------------------------------------------------
// Plan of one tucker_rthosvd / tucker_rsthosvd call.
// ---------------------------------------------------------------------------
struct HosvdPlan {
  int d = 0;
  bool st = true;
  XType xt = X_F32;
  std::vector<int64_t> n;
  std::vector<int> r, s, order, l;
  int q = 0;
  bool bf16 = false;
  tk_shift rule = TK_SHIFT_PAPER;
  int omega = TK_OMEGA_GAUSS;   // test matrix kind (tk_omega)
  // rot (ST-HOSVD, FP32, modes in natural order): every TTM writes its output
  // with the contracted mode moved last, so each step sees its mode first
  // (a mode-major view) and the core comes out in natural order.
  bool rot = false;
  // sizes (bytes)
  size_t gbuf = 0, shadow = 0, wbuf = 0, part = 0, ymat = 0, small = 0, qd = 0;
  size_t kr = 0;   // Khatri-Rao factor scratch
  std::vector<SmallPlan> sp;
  std::vector<std::vector<int64_t>> dims_at;  // tensor dims seen by each step
};

// View of mode k of the current tensor (dims cur, in natural mode order).
// Natural layout: the strided view, ka = 0.  Rotated layout (p.rot): the
// layout is (k, k+1..d, 1..k-1), the view is mode-major and column j of it
// is row j/ka + kb*(j%ka) of Omega_k (the unfolding's own column order).
inline View step_view(const HosvdPlan& p, const std::vector<int64_t>& cur, int k, int64_t* ka,
                      int64_t* kb) {
  if (!p.rot) {
    *ka = 0;
    *kb = 1;
    return view_of(cur, k);
  }
  int64_t a = 1, b = 1;
  for (size_t m = k + 1; m < cur.size(); ++m) a *= cur[m];
  for (int m = 0; m < k; ++m) b *= cur[m];
  *ka = a;
  *kb = b;
  View v;
  v.P = 1;
  v.n = cur[k];
  v.S = a * b;
  return v;
}

struct HosvdWs {
  void* g[2];
  void* shadow;
  void* w;
  void* part;
  double* Y;
  double* Q;
  void* small;
  double* qd;
  double* alpha;
  double* ahist;
  double* shist;
  double* sig;
  int* status;
  float* kr;
};

// full_ok: accept r_k = n_k (the holistic range finder keeps l_k = n_k
// columns when r_k + s_k >= n_k).
tk_status make_plan(const tk_tensor* A, const int* r, const tk_opts* o, bool st, HosvdPlan& p,
                    bool full_ok = false);
// Lays the workspace out from `base` (nullptr: only measures); returns bytes.
// ws (when given) receives workspace_copies(p) entries (one per concurrently
// factored mode; they share the tensor buffers, histories and status).
int workspace_copies(const HosvdPlan& p);
size_t carve(const HosvdPlan& p, unsigned char* base, HosvdWs* ws);

}  // namespace tk
