// Host-side objects shared by the C ABI and the sweep planners.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/cbc.h"

namespace cbc {

// A TTNS (kind 0) or TTNO (kind 1) in device memory, FP64 / complex128 storage, node
// tensors in the canonical leg order of cbc.h.
struct Net {
  int kind = 0;
  int n = 0;
  int root = 0;
  std::vector<int32_t> parent;
  std::vector<int64_t> phys, bond;
  std::vector<std::vector<int>> children;
  bool cplx = false;
  std::vector<void*> data;
  std::vector<int64_t> numel;
  void* block = nullptr;  // when set, data[i] point into this one allocation
  double log_norm = 0.0;
  // outputs of cbc_apply: relative weight discarded on the edge of node i to its parent
  // (the forward compression on a chain; steps 1 and 2 added on a tree), 0 at the root
  std::vector<double> discarded;
  cudaStream_t stream = nullptr;
  size_t elem_bytes() const { return cplx ? 16 : 8; }
  virtual ~Net();
};

enum { kMethodCBC = 0, kMethodZipUp = 1, kMethodSRC = 2, kMethodDirect = 3 };

struct Options {
  int precision = CBC_PREC_FP64;
  // rank floor: singular values s_j <= eps_rank * s_0 are dropped.  FP64 keeps the
  // oracle's floor; the mixed path's products resolve s only to ~3e-11 s_0, so its floor
  // sits above that (set by parse_options when the caller gives none)
  double eps_rank = 1e-12;
  int slices_fwd = 5;
  int slices_bwd = 4;
  // cbc_apply_batched: most instances per lockstep group
  int max_group = 32;
  // the method the chain sweeps run (Sec. III A, or a comparison method of Sec. III C)
  int method = kMethodCBC;
  // SRC: sketch width s and, per site, the device pointer of its d x s random matrix
  // (FP64 storage of the network's type; the last site's is not used)
  int sketch = 0;
  const void* const* sketch_mats = nullptr;
  // set for instances that run next to others on their own streams (cbc_apply_batched):
  // kernels whose CTAs wait on each other then use cluster launches, which run
  // concurrently with other streams' work, instead of cooperative ones, which do not
  bool concurrent = false;
  // mixed path: the Gram matrices of CholeskyQR2 in FP64 instead of on the tensor cores
  // (set by the planner when the tensor-core Gram met a Cholesky breakdown: a backward
  // factor S too ill conditioned for the slices' precision)
  bool cholqr_f64 = false;
};

int run_cbc(const Net& st, const Net& op, int64_t max_bond, double tol, const Options& o,
            Net* out);

// Truncation rank rule shared by the planners (planner.cu): weights w[0..kmax) of the
// candidate directions of a compression in descending order (w_j = s_j^2 measured on
// the factor), `beyond` the weight outside them (used when tol > 0): keep w_j > floor^2
// w_0 (a prefix), then the smallest k with sum_{j>=k} w_j + beyond <= tol^2 (sum_j w_j +
// beyond), then at most max_bond, at least 1.
int pick_rank(const double* w, int kmax, double beyond, int64_t max_bond, double tol,
              double floor_rel);
// number of leading candidates with w_j > res * w_0 (directions the Gram resolves)
int resolved_prefix(const double* w, int kmax, double res);
// Whether the first-level directions (from a Gram with relative error nu) decide the cut
// at k accurately enough (state error below target), and if not, the first direction of
// the second level (the residual's Gram recomputes directions from there on); -1: no
// second level.  g = min(m, n); w_next estimates the weight of the first direction after
// the kmax candidates; total is the cut's whole weight.
int refine_start(const double* w, int kmax, int g, int k, double w_next, double total,
                 double tol, double nu, double target, double res);
// Directions whose weight is below kResolved * w_0 are not trusted as singular
// directions: the Gram's own rounding (FP64: ~m eps w_0; mixed: ~1e-12 w_0 from the
// operand slices and the double-float reduction) is too close.
constexpr double kResolvedFP64 = 1e-10;
constexpr double kResolvedMixed = 1e-8;
// A tolerance that keeps every candidate while some are unresolved is checked by a second
// level only when at most this many are unresolved (the second level's eigensolver pays
// for each one); larger blocks are kept whole.
constexpr int kMaxSecondLevel = 64;
// candidates of the second level for a first-level cut at k that starts at jlo: the
// directions up to the cut and as many again (at least 16) beyond it, within kmax
int second_level_size(int kmax, int k, int jlo);

// A group (see run_cbc_group) that cannot run in lockstep: shapes differ, a tree, or the
// instances chose different ranks at some cut.  The caller runs the members one by one.
constexpr int kGroupSplit = -77;

// nb instances with identical chain shapes, max_bond and tol, in lockstep: one launch
// per step for the whole group.  Returns CBC_OK, an error, or kGroupSplit.
int run_cbc_group(const std::vector<const Net*>& sts, const std::vector<const Net*>& ops,
                  int64_t max_bond, double tol, const Options& o, const std::vector<Net*>& outs);

// launch statistics (cbc_stats_* in cbc.h)
struct KTimer {
  int cls;
  cudaStream_t s;
  cudaEvent_t e0 = nullptr;
  KTimer(int cls_, cudaStream_t s_, int64_t launches, double flops);
  ~KTimer();
};

void note_launches(int cls, int n);
void note_flops(int cls, double flops);

// stream-ordered device allocation from the library's own pool on the current device
// (freed with cudaFreeAsync); the caller's default pool is never touched
cudaError_t pool_malloc(void** p, size_t bytes, cudaStream_t s);

int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);
int num_sms();

}  // namespace cbc
