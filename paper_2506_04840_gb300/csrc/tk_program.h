// Per-problem programs of work-list jobs and their merging into launches.
//
// A problem (one tensor, one Tucker rank) is compiled into a list of phases
// following Algorithm 3 mode by mode:
//   sketch phase      Y = X_(k) Omega_k; Y -> Q (orthonormal basis; with
//                     q = 0 the svd);
//   power phase t     W = X_(k)^T Q; Y = X_(k) W - alpha_{t-1} Q;
//                     [Q, Sigma] = svd(Y); shift update;
//   finish phase      U_k = Q(:, 1:r_k) (FP64 CholeskyQR polish on the FP32
//                     path, copy out), G <- G x_k U_k^T;
// and, if the caller asks for it, an error phase (the expansion chain of
// tucker_error fused with the squared-difference sums).  Jobs inside a phase
// carry a position: a problem's jobs at position p depend on its jobs at
// positions < p of the same phase.  Phases of different problems are
// independent, so any set of problems' phases can be merged into one launch
// per (position, step kind, tile class).
#pragma once

#include <stdint.h>
#include <string.h>

#include <vector>

#include "tk_batch.h"
#include "tk_plan.h"
#include "tucker.h"

namespace tk {

struct Op {
  int pos;            // position inside the phase
  int prof;           // tk_kernel_kind of the profiler
  BatchLaunch key;    // kind, xt, tile, flag, smem (jobs/start unset)
  uint32_t blocks;    // this job's blocks
  double bytes, flops;
  alignas(64) unsigned char job[kJobBytes];
};
typedef std::vector<Op> Phase;

// Small per-problem device state (zeroed before a problem starts).
struct ItemState {
  double alpha[TK_MAX_D];                 // alpha of mode k (alpha_0 = 0)
  double ahist[TK_MAX_D * TK_MAX_Q];
  double shist[TK_MAX_D * TK_MAX_Q];
  double sig[TK_MAX_D * TK_MAX_L];
  int status;
  int pad[3];
};

// A compiled problem: its plan, workspace layout and program.
struct Problem {
  HosvdPlan p;
  HosvdWs w;
  std::vector<Phase> prog;
  // schedule slot of each phase: step m of the mode loop, then 0 = sketch,
  // t = power step t, TK_MAX_Q + 1 = finish; the error phase comes last.
  // Phases of different problems with the same slot do the same kind of work.
  std::vector<int> slot;
  size_t ws_bytes = 0;      // workspace this problem needs (incl. its ItemState)
  ItemState* state = nullptr;   // device, inside the workspace
};

// Validates `it` (ST-HOSVD in natural or descending mode order, plain
// precision) and sizes its workspace.  Returns TK_OK and fills pr->p and pr->ws_bytes.
tk_status problem_plan(const tk_item& it, tk_shift rule, Problem* pr);
// Lays the problem out at `base` (pr->ws_bytes bytes, 256-aligned) and builds
// its program; pr->state points at its ItemState.
tk_status problem_build(const tk_item& it, unsigned char* base, Problem* pr);

// A merged launch: job arrays and block starts at offsets of a table blob.
struct LaunchRec {
  BatchLaunch b;       // jobs/start filled by resolve()
  size_t jobs_off, start_off;
  int prof;
  double bytes, flops;
};

// Appends the launches that run `ops` (any problems' phases) to `out`,
// writing their job tables into `blob`.
void merge_ops(const std::vector<const Op*>& ops, std::vector<unsigned char>& blob,
               std::vector<LaunchRec>& out);
// Points the launches' tables at the device copy of the blob.
void resolve(std::vector<LaunchRec>& recs, const unsigned char* dev_blob);
// Launches one merged launch (profiled when `profile`).
cudaError_t issue(const LaunchRec& r, cudaStream_t st, bool profile);

}  // namespace tk
