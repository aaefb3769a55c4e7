// Tensor-train CBC without device allocation (cbc_apply_tt_noalloc in cbc.h).
//
// For callers that may not allocate device memory when they need an application (a
// framework that owns all device memory through its own pool, a real-time host loop
// that forbids allocation after start-up).  The sweeps and kernels are those of
// cbc_apply on a chain in FP64; every intermediate is carved from one file-scope
// __device__ array, and the result goes to a buffer the caller passes in.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "kernels.cuh"
#include "planner.h"

namespace cbc {
namespace {

// The scratch of every call on this device.  In host code the name below is only a
// host-side stand-in: kernels get the device address looked up by scratch_base().
static __device__ __align__(256) unsigned char g_noalloc_scratch[CBC_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
void* g_addr[kMaxDevices] = {};

// device address of the scratch array on the current device, looked up once per device
int scratch_base(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cbc_apply_tt_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices)
    return fail(CBC_ERR_UNSUPPORTED, "cbc_apply_tt_noalloc: device ordinal %d", dev);
  std::lock_guard<std::mutex> lk(g_addr_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cbc_apply_tt_noalloc: cudaGetSymbolAddress");
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return CBC_OK;
}

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

// bump allocator over the scratch array; a dry run only counts
struct Bump {
  char* base;
  size_t cap;
  size_t used = 0, peak = 0;
  bool over = false;
  template <typename T>
  T* get(size_t n) {
    size_t bytes = al256(std::max<size_t>(n * sizeof(T), 256));
    if (!base || used + bytes > cap) {  // dry run, or out of room
      over = over || (used + bytes > cap);
      used += bytes;
      peak = std::max(peak, used);
      return nullptr;
    }
    T* p = reinterpret_cast<T*>(base + used);
    used += bytes;
    peak = std::max(peak, used);
    return p;
  }
};

struct Args {
  int L;
  const int64_t* phys;
  const int64_t* sbond;
  const int64_t* obond;
  const void* const* st;
  const void* const* op;
  int64_t max_bond;
  double tol;
  char* out;
  int64_t out_cap;
  int64_t* out_off;
  int64_t* out_bond;
  double* log_norm;
  cudaStream_t s;
};

#define NA_CK(expr)                                                   \
  do {                                                                \
    cudaError_t e_ = (expr);                                          \
    if (e_ != cudaSuccess) return cuda_fail(e_, "noalloc: " #expr);   \
  } while (0)
#define NA_GET(var, T, n)                                             \
  T* var = b.get<T>(n);                                               \
  if (!dry && !var)                                                   \
    return fail(CBC_ERR_INVALID_ARG,                                  \
                "cbc_apply_tt_noalloc: intermediates need more than the %u-byte scratch", \
                (unsigned)CBC_NOALLOC_SCRATCH_BYTES);

// One pass of the sweeps.  dry = true: no launches, every rank at its upper bound, only
// the scratch high-water mark is computed.
template <typename T>
int sweeps(const Args& a, Bump& b, bool dry) {
  const int L = a.L;
  cudaStream_t s = a.s;
  const double floor_rel = 1e-12;  // cbc_apply's FP64 rank floor on singular values
  auto sb = [&](int i) { return (i < L && i > 0) ? (int)a.sbond[i] : 1; };
  auto ob = [&](int i) { return (i < L && i > 0) ? (int)a.obond[i] : 1; };
  NA_GET(d_int, int, 4);
  NA_GET(d_dbl, double, 4);
  int* status = d_int;
  int* k_dev = d_int + 1;
  double* log_fwd = d_dbl;
  double* log_out = d_dbl + 1;
  double* dscr = d_dbl + 2;
  T one;
  if constexpr (ops<T>::cplx)
    one = zdbl{1.0, 0.0};
  else
    one = 1.0;
  std::vector<T*> env(L, nullptr);
  std::vector<int> chi(L, 1);
  NA_GET(env0, T, 1);
  env[0] = env0;
  if (!dry) {
    NA_CK(cudaMemsetAsync(d_int, 0, 4 * sizeof(int), s));
    NA_CK(cudaMemsetAsync(d_dbl, 0, 4 * sizeof(double), s));
    NA_CK(cudaMemcpyAsync(env0, &one, sizeof(T), cudaMemcpyHostToDevice, s));
  }
  // ---- forward sweep, Eq. (tt_cbc_first_contraction) and the compression after it,
  // with cbc_apply's first-level truncation: every candidate direction of the Gram, the
  // rank rule on the weights measured on M (pick_rank), the first k rows of U^H M (or
  // diag(sqrt(w)) V^H) as the new environment.  A rank that would keep directions below
  // the Gram's resolution needs cbc_apply's second level, which is not built here.
  for (int i = 0; i < L - 1; ++i) {
    const int c = chi[i], bb = ob(i), aa = sb(i), d = (int)a.phys[i], a2 = sb(i + 1), b2 = ob(i + 1);
    const int m = c * d, n = b2 * a2, g = std::min(m, n);
    const bool rows = (m <= n);
    const int kmax = (int)((a.max_bond > 0) ? std::min<int64_t>(a.max_bond, g) : g);
    NA_GET(envn, T, (size_t)kmax * n);  // below this step's temporaries
    const size_t mark = b.used;
    NA_GET(X, T, (size_t)c * bb * d * a2);
    NA_GET(Lp, T, (size_t)m * n);
    NA_GET(K, T, (size_t)g * g);
    NA_GET(lam, double, g);
    NA_GET(U, T, (size_t)g * kmax);
    NA_GET(work, char, eig_workspace_bytes(g, kmax, ops<T>::cplx));
    NA_GET(wv, double, kmax + 2);
    NA_GET(Wc, T, rows ? 1 : (size_t)m * kmax);
    NA_GET(P, T, a.tol > 0.0 ? (size_t)m * n : 1);
    int k = kmax;
    if (!dry) {
      const T* Ti = static_cast<const T*>(a.st[i]);
      const T* Wi = static_cast<const T*>(a.op[i]);
      NA_CK(cudaMemsetAsync(wv, 0, sizeof(double) * (kmax + 2), s));
      NA_CK(gemm_f64<T>(c * bb, d * a2, aa, 1, env[i], View::rowmajor(aa), false, Ti,
                        View::rowmajor(d * a2), false, X, View::rowmajor(d * a2), s));
      View vw;
      vw.rows2(b2, (int64_t)d * b2, 1).cols2(d, (int64_t)d * d * b2, b2);
      View vx;
      vx.rs_in = a2;
      vx.cols2(a2, (int64_t)bb * d * a2, 1);
      View vl;
      vl.rs_in = a2;
      vl.cols2(a2, (int64_t)d * b2 * a2, 1);
      NA_CK(gemm_f64<T>(d * b2, c * a2, bb * d, 1, Wi, vw, false, X, vx, false, Lp, vl, s));
      if (rows)
        NA_CK(gemm_f64<T>(m, m, n, 1, Lp, View::rowmajor(n), false, Lp, View::transposed(n), true,
                          K, View::rowmajor(m), s));
      else
        NA_CK(gemm_f64<T>(n, n, m, 1, Lp, View::transposed(n), true, Lp, View::rowmajor(n), false,
                          K, View::rowmajor(n), s));
      NA_CK(heev_top<T>(K, g, kmax, kmax, 0.0, -1.0, lam, U, k_dev, work, status, num_sms(), s));
      if (rows) {  // U^H M, kmax x n, in the environment buffer
        NA_CK(gemm_f64<T>(kmax, n, m, 1, U, View::transposed(kmax), true, Lp, View::rowmajor(n),
                          false, envn, View::rowmajor(n), s));
        NA_CK(row_norms2<T>(envn, kmax, n, n, 0, wv, s));
      } else {     // M V, m x kmax
        NA_CK(gemm_f64<T>(m, kmax, n, 1, Lp, View::rowmajor(n), false, U, View::rowmajor(kmax),
                          false, Wc, View::rowmajor(kmax), s));
        NA_CK(col_norms2<T>(Wc, m, kmax, kmax, 0, wv, s));
      }
      NA_CK(sum_squares<T>(Lp, (int64_t)m * n, wv + kmax + 1, s));  // the cut's weight
      if (a.tol > 0.0) {  // weight outside the candidates
        if (rows)
          NA_CK(gemm_f64<T>(m, n, kmax, 1, U, View::rowmajor(kmax), false, envn, View::rowmajor(n),
                            false, P, View::rowmajor(n), s));
        else
          NA_CK(gemm_f64<T>(m, n, kmax, 1, Wc, View::rowmajor(kmax), false, U,
                            View::transposed(kmax), true, P, View::rowmajor(n), s));
        NA_CK(diff_sumsq<T>(Lp, (int64_t)m * n, P, nullptr, (int64_t)m * n, wv + kmax, s));
      }
      std::vector<double> hw(kmax + 2, 0.0);
      double w_next = 0.0;
      int hs = 0;
      NA_CK(cudaMemcpyAsync(hw.data(), wv, sizeof(double) * (kmax + 2), cudaMemcpyDeviceToHost, s));
      if (kmax < g)
        NA_CK(cudaMemcpyAsync(&w_next, lam + kmax, sizeof(double), cudaMemcpyDeviceToHost, s));
      NA_CK(cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, s));
      NA_CK(cudaStreamSynchronize(s));
      if (hs != 0) return fail(hs, "cbc_apply_tt_noalloc: device status %d", hs);
      if (hw[kmax + 1] == 0.0)
        return fail(CBC_ERR_NUMERICAL, "cbc_apply_tt_noalloc: O|psi> vanishes");
      for (int j = 0; j < kmax + 2; ++j)
        if (!std::isfinite(hw[j]))
          return fail(CBC_ERR_NUMERICAL, "cbc_apply_tt_noalloc: NaN or Inf in a truncation");
      k = pick_rank(hw.data(), kmax, a.tol > 0.0 ? hw[kmax] : -1.0, a.max_bond, a.tol, floor_rel);
      const double nu = 4.0 * std::sqrt((double)g) * 1.1102230246251565e-16;
      if (refine_start(hw.data(), kmax, g, k, w_next, hw[kmax + 1], a.tol, nu, 1e-11,
                       kResolvedFP64) >= 0)
        return fail(CBC_ERR_UNSUPPORTED,
                    "cbc_apply_tt_noalloc: the cut at site %d falls among directions the "
                    "Gram does not resolve (small singular values close together); cbc_apply "
                    "refines those, this entry point does not", i);
      if (!rows) NA_CK(scaled_adjoint_w<T>(U, kmax, wv, kmax, k, n, envn, 0, s));
      NA_CK(normalize_inplace<T>(envn, (int64_t)k * n, log_fwd, status, dscr, s));
    }
    env[i + 1] = envn;
    chi[i + 1] = k;
    b.used = mark;
  }
  // ---- backward sweep, Eqs. (right_sweep_init_contr), (tt_cbc_qr_decomp),
  // (tt_cbc_final_contraction); two R buffers alternate.  At a site whose S has at
  // least as many rows as columns the new tensor is the identity (every unitary spans
  // the whole row space, the rule cbc_apply follows), so S is only formed at the first
  // site or when it has fewer rows than columns.
  //
  // Every rank is known once the forward sweep has run, so the size of the result is
  // checked here, before the backward sweep launches anything; on failure the stream is
  // drained first, so nothing still runs when the caller sees the error.
  int64_t out_need = 0;
  {
    int cp = 1;
    for (int i = L - 1; i >= 0; --i) {
      const int m = chi[i], n = (int)a.phys[i] * cp;
      const int cn = (m < n) ? m : n;
      out_need += (int64_t)cn * n;
      cp = cn;
    }
  }
  if (!dry && out_need > a.out_cap) {
    cudaStreamSynchronize(s);
    return fail(CBC_ERR_INVALID_ARG,
                "cbc_apply_tt_noalloc: out_capacity %lld elements is too small: the result "
                "needs %lld", (long long)a.out_cap, (long long)out_need);
  }
  size_t rmax = 1;
  for (int i = 0; i < L; ++i) rmax = std::max(rmax, (size_t)chi[i] * ob(i) * sb(i));
  NA_GET(Ra, T, rmax);
  NA_GET(Rb, T, rmax);
  NA_GET(bar, GridBarrier, 1);
  T* R = Ra;
  if (!dry) NA_CK(cudaMemcpyAsync(R, &one, sizeof(T), cudaMemcpyHostToDevice, s));
  int chiR = 1;
  int64_t out_used = 0;
  for (int i = L - 1; i >= 0; --i) {
    const int a_in = sb(i), b_in = ob(i), d = (int)a.phys[i], a_out = sb(i + 1), b_out = ob(i + 1);
    const int cp = chiR, c = chi[i], m = c, n = d * cp;
    const int cn = (m < n) ? m : n;
    const bool formed = (i == 0 || m < n);
    const size_t mark = b.used;
    NA_GET(Y, T, (size_t)a_in * d * cp * b_out);
    NA_GET(Z, T, (size_t)b_in * a_in * d * cp);
    NA_GET(G, T, (size_t)m * m);
    NA_GET(rn, double, m);
    if (!dry) {
      T* node = reinterpret_cast<T*>(a.out) + out_used;
      a.out_off[i] = out_used;
      const T* Ti = static_cast<const T*>(a.st[i]);
      const T* Wi = static_cast<const T*>(a.op[i]);
      NA_CK(gemm_f64<T>(a_in * d, cp * b_out, a_out, 1, Ti, View::rowmajor(a_out), false, R,
                        View::transposed(a_out), false, Y, View::rowmajor(cp * b_out), s));
      View vy;
      vy.rows2(b_out, (int64_t)cp * b_out, 1).cols2(cp, (int64_t)d * cp * b_out, b_out);
      View vz;
      vz.rows2(d, (int64_t)a_in * d * cp, cp).cols2(cp, (int64_t)d * cp, 1);
      NA_CK(gemm_f64<T>(b_in * d, a_in * cp, d * b_out, 1, Wi, View::rowmajor(d * b_out), false, Y,
                        vy, false, Z, vz, s));
      if (formed)
        NA_CK(gemm_f64<T>(m, n, b_in * a_in, 1, env[i], View::rowmajor(b_in * a_in), false, Z,
                          View::rowmajor(n), false, node, View::rowmajor(n), s));
      if (i == 0) {
        NA_CK(normalize_inplace<T>(node, (int64_t)n, log_out, status, dscr, s));
        a.out_bond[0] = 1;
        out_used += n;
        break;
      }
      if (m < n) {
        // unit rows first (same row space, a well-conditioned Gram), as cbc_apply does
        NA_CK(row_norms2<T>(node, m, n, n, 0, rn, s));
        NA_CK(scale_rows<T>(node, m, n, 0, rn, s));
        for (int rep = 0; rep < 2; ++rep) {
          NA_CK(gemm_f64<T>(m, m, n, 1, node, View::rowmajor(n), false, node, View::transposed(n),
                            true, G, View::rowmajor(m), s));
          NA_CK(cholesky_lower<T>(G, m, status, bar, num_sms(), s));
          NA_CK(trsm_lower_left<T>(G, node, m, n, status, bar, num_sms(), s));
        }
      } else {
        NA_CK(fill_identity<T>(node, n, s));
      }
      T* Rn = (R == Ra) ? Rb : Ra;
      NA_CK(gemm_f64<T>(cn, b_in * a_in, n, 1, node, View::rowmajor(n), true, Z,
                        View::transposed(n), false, Rn, View::rowmajor(b_in * a_in), s));
      NA_CK(normalize_inplace<T>(Rn, (int64_t)cn * b_in * a_in, log_out, status, dscr, s));
      R = Rn;
      a.out_bond[i] = cn;
      out_used += (int64_t)cn * n;
    }
    chiR = cn;
    b.used = mark;
    if (i == 0) break;
  }
  if (!dry) {
    int h[2] = {0, 0};
    double ln = 0.0;
    NA_CK(cudaMemcpyAsync(h, status, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    NA_CK(cudaMemcpyAsync(&ln, log_out, sizeof(double), cudaMemcpyDeviceToHost, s));
    NA_CK(cudaStreamSynchronize(s));
    if (h[0] != 0) return fail(h[0], "cbc_apply_tt_noalloc: device status %d", h[0]);
    *a.log_norm = ln;
  }
  return CBC_OK;
}

}  // namespace
}  // namespace cbc

using namespace cbc;

extern "C" int cbc_apply_tt_noalloc(int L, const int64_t* phys_dim, const int64_t* state_bond,
                                    const int64_t* op_bond, int dtype,
                                    const void* const* state_nodes, const void* const* op_nodes,
                                    int64_t max_bond, double tol, void* out_data,
                                    int64_t out_capacity, int64_t* out_offsets,
                                    int64_t* out_bonds, double* log_norm, void* cuda_stream) {
  if (L < 1 || !phys_dim || !state_bond || !op_bond || !state_nodes || !op_nodes || !out_data ||
      !out_offsets || !out_bonds || !log_norm)
    return fail(CBC_ERR_INVALID_ARG, "cbc_apply_tt_noalloc: null argument or L < 1");
  if (dtype != CBC_F64 && dtype != CBC_C128)
    return fail(CBC_ERR_INVALID_ARG, "cbc_apply_tt_noalloc: dtype must be CBC_F64 or CBC_C128");
  if (!(tol == tol)) return fail(CBC_ERR_INVALID_ARG, "cbc_apply_tt_noalloc: tol is NaN");
  for (int i = 0; i < L; ++i) {
    if (phys_dim[i] < 1 || (i > 0 && (state_bond[i] < 1 || op_bond[i] < 1)))
      return fail(CBC_ERR_INVALID_ARG, "cbc_apply_tt_noalloc: site %d has a dimension < 1", i);
    if (!state_nodes[i] || !op_nodes[i])
      return fail(CBC_ERR_INVALID_ARG, "cbc_apply_tt_noalloc: node pointer %d is NULL", i);
  }
  // every extent the sweeps hand to a kernel is an int: reject chains whose dimension
  // products (with each compressed bond at its upper bound) exceed that range
  {
    auto bond_of = [&](const int64_t* b, int i) -> int64_t { return (i > 0 && i < L) ? b[i] : 1; };
    int64_t c = 1;  // upper bound of the compressed bond chi_i
    for (int i = 0; i < L; ++i) {
      const int64_t d = phys_dim[i], a_in = bond_of(state_bond, i), b_in = bond_of(op_bond, i);
      const int64_t a_out = bond_of(state_bond, i + 1), b_out = bond_of(op_bond, i + 1);
      const int64_t cn = std::min<int64_t>(c * d, a_out * b_out);  // chi_{i+1} and chi'_i bound
      const double big = std::max({(double)a_in * d * a_out, (double)b_in * d * d * b_out,
                                   (double)c * b_in * d * a_out, (double)c * d * b_out * a_out,
                                   (double)a_in * d * cn * b_out, (double)b_in * a_in * d * cn,
                                   (double)c * d * cn, (double)c * c});
      if (big > (double)INT32_MAX)
        return fail(CBC_ERR_INVALID_ARG,
                    "cbc_apply_tt_noalloc: site %d has a dimension product beyond 2^31 - 1", i);
      c = (max_bond > 0) ? std::min<int64_t>(cn, max_bond) : cn;
    }
  }
  void* base = nullptr;
  int rc = scratch_base(&base);
  if (rc != CBC_OK) return rc;
  Args a{L, phys_dim, state_bond, op_bond, state_nodes, op_nodes, max_bond, tol,
         static_cast<char*>(out_data), out_capacity, out_offsets, out_bonds, log_norm,
         static_cast<cudaStream_t>(cuda_stream)};
  // up-front size check with every rank at its upper bound
  Bump dry{nullptr, CBC_NOALLOC_SCRATCH_BYTES};
  rc = (dtype == CBC_C128) ? sweeps<zdbl>(a, dry, true) : sweeps<double>(a, dry, true);
  if (rc != CBC_OK) return rc;
  if (dry.peak > CBC_NOALLOC_SCRATCH_BYTES)
    return fail(CBC_ERR_INVALID_ARG,
                "cbc_apply_tt_noalloc: this chain needs up to %zu bytes of scratch; the "
                "no-allocation entry point holds %u bytes", dry.peak,
                (unsigned)CBC_NOALLOC_SCRATCH_BYTES);
  Bump run{static_cast<char*>(base), CBC_NOALLOC_SCRATCH_BYTES};
  return (dtype == CBC_C128) ? sweeps<zdbl>(a, run, false) : sweeps<double>(a, run, false);
}
