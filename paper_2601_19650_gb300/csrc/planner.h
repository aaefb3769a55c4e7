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
  cudaStream_t stream = nullptr;
  size_t elem_bytes() const { return cplx ? 16 : 8; }
  virtual ~Net();
};

struct Options {
  int precision = CBC_PREC_FP64;
  double eps_rank = 1e-6;
  int slices_fwd = 5;
  int slices_bwd = 4;
  // set for instances that run next to others on their own streams (cbc_apply_batched):
  // kernels whose CTAs wait on each other then use cluster launches, which run
  // concurrently with other streams' work, instead of cooperative ones, which do not
  bool concurrent = false;
};

int run_cbc(const Net& st, const Net& op, int64_t max_bond, double tol, const Options& o,
            Net* out);

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

int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);
int num_sms();

}  // namespace cbc
