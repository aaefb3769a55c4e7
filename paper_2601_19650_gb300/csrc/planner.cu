// Sweep planners: they turn one cbc_apply into the sequence of kernel launches of
// Sec. III A (tensor train) and Sec. III B (trees).  All arithmetic runs in the
// kernels; the host only sizes buffers, picks leg views and reads back the rank chosen
// on the device after each compression.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <functional>
#include <utility>
#include <vector>

#include "kernels.cuh"
#include "planner.h"

namespace cbc {
namespace {

// stream-ordered scratch that is released when the call ends
struct Arena {
  cudaStream_t s;
  std::vector<void*> ptrs;
  cudaError_t err = cudaSuccess;
  explicit Arena(cudaStream_t st) : s(st) {}
  template <typename T>
  T* get(size_t n) {
    void* p = nullptr;
    size_t bytes = std::max<size_t>(n * sizeof(T), 256);
    cudaError_t e = pool_malloc(&p, bytes, s);
    if (e != cudaSuccess) {
      if (err == cudaSuccess) err = e;
      return nullptr;
    }
    ptrs.push_back(p);
    return static_cast<T*>(p);
  }
  // scopes: release() frees (stream-ordered) everything allocated after mark()
  size_t mark() const { return ptrs.size(); }
  void release(size_t mk) {
    while (ptrs.size() > mk) {
      cudaFreeAsync(ptrs.back(), s);
      ptrs.pop_back();
    }
  }
  // frees one allocation early
  void drop(void* p) {
    for (size_t i = 0; i < ptrs.size(); ++i)
      if (ptrs[i] == p) {
        cudaFreeAsync(p, s);
        ptrs.erase(ptrs.begin() + i);
        return;
      }
  }
  ~Arena() {
    for (void* p : ptrs) cudaFreeAsync(p, s);
  }
};



#define CK(expr)                                         \
  do {                                                   \
    cudaError_t e_ = (expr);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #expr);  \
  } while (0)

#define CKA(ptr)                                                          \
  do {                                                                    \
    if (!(ptr)) return cuda_fail(ar.err, "workspace allocation " #ptr);   \
  } while (0)

int status_to_rc(int st) {
  switch (st) {
    case CBC_ERR_NOT_POSITIVE_DEFINITE:
      return fail(st, "cbc_apply: Cholesky met a non-positive pivot (rank-deficient S)");
    case CBC_ERR_NUMERICAL:
      return fail(st, "cbc_apply: NaN or Inf in an intermediate, or O|psi> vanishes (an "
                      "environment of zero norm)");
    case CBC_ERR_TIMEOUT: return fail(st, "cbc_apply: a device-side wait timed out");
    default: return fail(st, "cbc_apply: device status %d", st);
  }
}

// device scalars of one call: one status word; k, the two log scales and the
// reduction scratch per instance of a group
struct Scalars {
  int* status;
  int* k;
  double* log_fwd;
  double* log_out;
  double* scratch;
};

template <typename T>
T host_one() {
  T v;
  if constexpr (ops<T>::cplx)
    v = zdbl{1.0, 0.0};
  else
    v = 1.0;
  return v;
}

// One contraction or Gram product, timed as a launch group: FP64 SIMT on the plain
// path, tensor-core slices on the mixed path (`fwd` picks the slice count of the first
// sweep, which feeds the truncations, or of the last one).  `gram` halves the
// algorithmic flops.
// `nb` instances of one shape run in lockstep: every operand of every call is then nb
// copies, View::bs elements apart.
struct Prec {
  bool mixed = false;
  bool cholqr_f64 = false;  // CholeskyQR2's Gram in FP64 even on the mixed path
  int s_fwd = 5, s_bwd = 4;
  Arena* ar = nullptr;
  int* status = nullptr;
  int nb = 1;
};

template <typename T>
cudaError_t tgemm(const Prec& pr, bool fwd, bool gram, int M, int N, int K, const T* A,
                  const View& va, bool ca, const T* B, const View& vb, bool cb, T* C,
                  const View& vc, cudaStream_t s) {
  double fl = (ops<T>::cplx ? 8.0 : 2.0) * (double)M * N * K * (gram ? 0.5 : 1.0) * pr.nb;
  if (pr.mixed && K > 0) {
    const int S = fwd ? pr.s_fwd : pr.s_bwd;
    const size_t mk = pr.ar->mark();
    void* ws = pr.ar->get<char>(gemm_tc_workspace_bytes(M, N, K, ops<T>::cplx, S, pr.nb));
    if (!ws) return pr.ar->err;
    cudaError_t e;
    {
      KTimer t(CBC_K_GEMM_TC, s, 0, fl);
      e = gemm_tc<T>(M, N, K, A, va, ca, B, vb, cb, C, vc, S, ws, pr.status, s, pr.nb);
    }
    pr.ar->release(mk);  // the slices are dead once the launch is queued
    return e;
  }
  KTimer t(CBC_K_GEMM_F64, s, 0, fl);
  return gemm_f64<T>(M, N, K, pr.nb, A, va, ca, B, vb, cb, C, vc, s);
}


// ---- truncation of a fused leg (Sec. III A, text after Eq. (tt_cbc_first_contraction);
// Sec. III B steps 1 and 2) --------------------------------------------------------------
//
// The paper names an SVD as one way to compress.  Here the candidate directions come from the
// Gram K = M M^H (or G = M^H M) and a Hermitian eigensolver, but the rank rule runs on
// weights measured on M itself: w_j = ||u_j^H M||^2 (or ||M v_j||^2) and, in tolerance
// mode, the exact weight outside the candidates ||M - U U^H M||_F^2.  A Gram holds the
// small singular values only to about eps * s_0^2 in absolute terms, so its eigenvalues
// cannot decide a tolerance of 1e-8 (discarded weight 1e-16 of the total); the weights
// measured on M resolve it, and when the rule keeps directions below what the Gram
// resolves, those directions are recomputed from the Gram of the residual
// M - U_r U_r^H M beyond the well-resolved ones (a second level).

// relative weight discarded by keeping the first k directions
double discarded_rel(const double* w, int kmax, int k, double beyond, double total) {
  if (!(total > 0.0)) return 0.0;
  double tail;
  if (beyond >= 0.0) {
    tail = std::max(beyond, 0.0);
    for (int j = k; j < kmax; ++j) tail += std::max(w[j], 0.0);
  } else {
    double kept = 0.0;
    for (int j = 0; j < k; ++j) kept += std::max(w[j], 0.0);
    tail = std::max(total - kept, 0.0);
  }
  return tail / total;
}

bool all_finite(const std::vector<double>& v) {
  for (double x : v)
    if (!std::isfinite(x)) return false;
  return true;
}

// Second level for one instance.  First level (rows orientation, m <= n): U1 (m x kmax,
// column j = direction j) and W1 = U1^H M (kmax x n).  Columns orientation (m > n): V1
// (n x kmax, the right directions, passed as U1) and W1 = M V1 (m x kmax).  jlo leading
// directions are kept as they are; k2 new candidates are recomputed from the Gram of the
// residual R = M - (the part of M along the kept ones), on the short side, orthogonalised
// against the kept ones.  Rows: their W rows replace W1's rows jlo .. jlo+k2-1.  Columns:
// their vectors replace V1's columns jlo .. jlo+k2-1 (the factor is then
// diag(sqrt(w)) V^H).  The rank is decided again on the combined weights (w is updated;
// w_dev receives them in the columns orientation).
template <typename T>
int refine_level2(Arena& ar, const Prec& pr, const T* M, int m, int n, int kmax, int jlo, int k2,
                  bool rows, T* U1, T* W1, std::vector<double>& w, double* w_dev, int64_t max_bond,
                  double tol, double floor_rel, const Options& o, const Scalars& sc,
                  cudaStream_t s, int* kout, double* disc) {
  const int64_t mn = (int64_t)m * n;
  const int g = rows ? m : n;  // the short side: the residual's Gram is g x g
  T* P = ar.get<T>((size_t)mn);
  T* R = ar.get<T>((size_t)mn);
  T* K2 = ar.get<T>((size_t)g * g);
  double* lam2 = ar.get<double>(g);
  T* U2 = ar.get<T>((size_t)g * k2);
  T* C = ar.get<T>((size_t)std::max(1, jlo) * k2);
  T* P2 = ar.get<T>((size_t)g * k2);
  T* W2c = rows ? nullptr : ar.get<T>((size_t)m * k2);
  char* work = ar.get<char>(eig_workspace_bytes(g, k2, ops<T>::cplx));
  double* dv = ar.get<double>(k2 + 4);
  CKA(P); CKA(R); CKA(K2); CKA(lam2); CKA(U2); CKA(C); CKA(P2); CKA(work); CKA(dv);
  if (!rows) CKA(W2c);
  CK(cudaMemsetAsync(dv, 0, sizeof(double) * (k2 + 4), s));
  // R = M - (the part along the kept directions)
  if (rows)   // U1r W1r
    CK(tgemm<T>(pr, true, false, m, n, jlo, U1, View::rowmajor(kmax), false, W1,
                View::rowmajor(n), false, P, View::rowmajor(n), s));
  else        // W1r V1r^H
    CK(tgemm<T>(pr, true, false, m, n, jlo, W1, View::rowmajor(kmax), false, U1,
                View::transposed(kmax), true, P, View::rowmajor(n), s));
  CK(diff_sumsq<T>(M, mn, P, R, mn, dv + k2, s));
  if (rows)   // R R^H
    CK(tgemm<T>(pr, true, true, m, m, n, R, View::rowmajor(n), false, R, View::transposed(n),
                true, K2, View::rowmajor(m), s));
  else        // R^H R
    CK(tgemm<T>(pr, true, true, n, n, m, R, View::transposed(n), true, R, View::rowmajor(n),
                false, K2, View::rowmajor(n), s));
  CK(heev_top<T>(K2, g, k2, k2, 0.0, -1.0, lam2, U2, sc.k, work, sc.status, num_sms(), s, 1,
                 o.concurrent, false));
  // U2 <- U2 - U1r (U1r^H U2)
  CK(tgemm<T>(pr, true, false, jlo, k2, g, U1, View::transposed(kmax), true, U2,
              View::rowmajor(k2), false, C, View::rowmajor(k2), s));
  CK(tgemm<T>(pr, true, false, g, k2, jlo, U1, View::rowmajor(kmax), false, C,
              View::rowmajor(k2), false, P2, View::rowmajor(k2), s));
  CK(diff_sumsq<T>(U2, (int64_t)g * k2, P2, U2, (int64_t)g * k2, dv + k2 + 1, s));
  if (rows) {
    T* W2 = W1 + (int64_t)jlo * n;  // rows jlo .. jlo+k2-1 of the new factor
    CK(tgemm<T>(pr, true, false, k2, n, m, U2, View::transposed(k2), true, M, View::rowmajor(n),
                false, W2, View::rowmajor(n), s));
    CK(row_norms2<T>(W2, k2, n, n, 0, dv, s));
    CK(tgemm<T>(pr, true, false, m, n, k2, U2, View::rowmajor(k2), false, W2, View::rowmajor(n),
                false, P, View::rowmajor(n), s));
  } else {
    CK(tgemm<T>(pr, true, false, m, k2, n, M, View::rowmajor(n), false, U2, View::rowmajor(k2),
                false, W2c, View::rowmajor(k2), s));
    CK(col_norms2<T>(W2c, m, k2, k2, 0, dv, s));
    CK(tgemm<T>(pr, true, false, m, n, k2, W2c, View::rowmajor(k2), false, U2,
                View::transposed(k2), true, P, View::rowmajor(n), s));
    // the new right directions become V1's columns jlo .. jlo+k2-1
    CK(copy_batched<T>(U2, k2, U1 + jlo, kmax, k2, s, n));
  }
  // weight outside all the directions: ||R - (the part along the new ones)||^2
  CK(diff_sumsq<T>(R, mn, P, nullptr, mn, dv + k2 + 2, s));
  std::vector<double> h(k2 + 3);
  int hs = 0;
  CK(cudaMemcpyAsync(h.data(), dv, sizeof(double) * (k2 + 3), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&hs, sc.status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (hs != 0) return status_to_rc(hs);
  if (!all_finite(h)) return fail(CBC_ERR_NUMERICAL, "cbc_apply: NaN or Inf in a truncation");
  const int kn = jlo + k2;
  for (int j = 0; j < k2; ++j) w[jlo + j] = h[j];
  const double beyond = h[k2 + 2];
  const int k = pick_rank(w.data(), kn, beyond, max_bond, tol, floor_rel);
  double total = beyond;
  for (int j = 0; j < kn; ++j) total += std::max(w[j], 0.0);
  *disc = discarded_rel(w.data(), kn, k, beyond, total);
  if (!rows && w_dev)
    CK(cudaMemcpyAsync(w_dev, w.data(), sizeof(double) * kn, cudaMemcpyHostToDevice, s));
  *kout = k;
  return CBC_OK;
}

template <typename T>
int lq_rows_inplace(Arena& ar, const Prec& pr, T* S, int m, int n, const Scalars& sc,
                    cudaStream_t s, bool shifted = false);

// Compression of the row leg of M (m x n, row-major): writes the k x n factor whose
// Gram reproduces the rank-k truncation of M^H M, normalised, and returns k (and the
// relative discarded weight per instance in disc, if given).  L (k x n per instance)
// comes from `keep` (default: ar); the rest is released on return when keep is given.
template <typename T>
int compress_rows(Arena& ar, const Prec& pr, const T* M, int m, int n, int64_t max_bond,
                  double tol, const Options& o, const Scalars& sc, cudaStream_t s, T** Lout,
                  int* kout, Arena* keep = nullptr, double* disc = nullptr) {
  const int g = std::min(m, n);
  const int kmax = (int)((max_bond > 0) ? std::min<int64_t>(max_bond, g) : g);
  const int nb = pr.nb;
  const int64_t mbs = (int64_t)m * n;  // M of consecutive instances
  const bool rows = (m <= n);          // K = M M^H, else G = M^H M
  const double floor_rel = o.eps_rank;
  const double res = pr.mixed ? kResolvedMixed : kResolvedFP64;
  Arena& kp = keep ? *keep : ar;
  const size_t mk = ar.mark();
  T* K = ar.get<T>((size_t)nb * g * g);
  double* lam = ar.get<double>((size_t)nb * g);
  T* U = ar.get<T>((size_t)nb * g * kmax);
  char* work = ar.get<char>(nb * eig_workspace_bytes(g, kmax, ops<T>::cplx));
  double* dv = ar.get<double>((size_t)nb * (kmax + 2));  // w [nb][kmax], beyond [nb], total [nb]
  CKA(K); CKA(lam); CKA(U); CKA(work); CKA(dv);
  double* w_dev = dv;
  double* beyond_dev = dv + (size_t)nb * kmax;
  double* total_dev = beyond_dev + nb;
  CK(cudaMemsetAsync(dv, 0, sizeof(double) * (size_t)nb * (kmax + 2), s));
  if (rows) {
    CK(tgemm<T>(pr, true, true, m, m, n, M, View::rowmajor(n, mbs), false, M,
                View::transposed(n, mbs), true, K, View::rowmajor(m, (int64_t)g * g), s));
  } else {
    CK(tgemm<T>(pr, true, true, n, n, m, M, View::transposed(n, mbs), true, M,
                View::rowmajor(n, mbs), false, K, View::rowmajor(n, (int64_t)g * g), s));
  }
  // ||M||_F^2, the weight of the cut: the trace of the Gram (g reads instead of m n)
  CK(trace_real<T>(K, g, (int64_t)g * g, total_dev, s, nb));
  // every candidate; the mixed path reduces batches to tridiagonal form in double-float
  CK(heev_top<T>(K, g, kmax, kmax, 0.0, -1.0, lam, U, sc.k, work, sc.status, num_sms(), s, nb,
                 o.concurrent, pr.mixed));
  const int64_t ubs = (int64_t)g * kmax;
  T* W = nullptr;
  int64_t wbs;
  if (rows) {  // W = U^H M (kmax x n): its first k rows are the new factor
    wbs = (int64_t)kmax * n;
    W = kp.get<T>((size_t)nb * wbs);
    if (!W) return cuda_fail(kp.err, "workspace allocation L");
    CK(tgemm<T>(pr, true, false, kmax, n, m, U, View::transposed(kmax, ubs), true, M,
                View::rowmajor(n, mbs), false, W, View::rowmajor(n, wbs), s));
    CK(row_norms2<T>(W, kmax, n, n, wbs, w_dev, s, nb));
  } else {     // W = M V (m x kmax): column j has norm s_j
    wbs = (int64_t)m * kmax;
    W = ar.get<T>((size_t)nb * wbs);
    CKA(W);
    CK(tgemm<T>(pr, true, false, m, kmax, n, M, View::rowmajor(n, mbs), false, U,
                View::rowmajor(kmax, ubs), false, W, View::rowmajor(kmax, wbs), s));
    CK(col_norms2<T>(W, m, kmax, kmax, wbs, w_dev, s, nb));
  }
  if (tol > 0.0) {  // the exact weight outside the candidates, ||M - U U^H M||^2
    T* P = ar.get<T>((size_t)nb * mbs);
    CKA(P);
    if (rows)
      CK(tgemm<T>(pr, true, false, m, n, kmax, U, View::rowmajor(kmax, ubs), false, W,
                  View::rowmajor(n, wbs), false, P, View::rowmajor(n, mbs), s));
    else
      CK(tgemm<T>(pr, true, false, m, n, kmax, W, View::rowmajor(kmax, wbs), false, U,
                  View::transposed(kmax, ubs), true, P, View::rowmajor(n, mbs), s));
    CK(diff_sumsq<T>(M, mbs, P, nullptr, mbs, beyond_dev, s, nb));
  }
  std::vector<double> h((size_t)nb * (kmax + 2));
  std::vector<double> hl(kmax < g ? (size_t)nb * g : 0);
  int hs = 0;
  CK(cudaMemcpyAsync(h.data(), dv, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s));
  if (!hl.empty())
    CK(cudaMemcpyAsync(hl.data(), lam, sizeof(double) * hl.size(), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&hs, sc.status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (hs != 0) return status_to_rc(hs);
  for (int b = 0; b < nb; ++b)
    if (h[(size_t)nb * (kmax + 1) + b] == 0.0)
      return fail(CBC_ERR_NUMERICAL, "cbc_apply: O|psi> vanishes (a compression of zero weight)");
  if (!all_finite(h)) return fail(CBC_ERR_NUMERICAL, "cbc_apply: NaN or Inf in a truncation");
  // the Gram's relative error (FP64: accumulation over the sqrt(g)-ish random walk of
  // g products; mixed: the operand slices and the double-float reduction) and the state
  // error a cut may add (a fraction of each path's bar, 1e-10 and 1e-6)
  const double nu = pr.mixed ? 5e-12 : 4.0 * std::sqrt((double)g) * 1.1102230246251565e-16;
  const double target = pr.mixed ? 1e-7 : 1e-11;
  std::vector<int> kb(nb), jlo(nb);
  std::vector<std::vector<double>> wb(nb);
  bool any_refine = false;
  for (int b = 0; b < nb; ++b) {
    wb[b].assign(h.begin() + (size_t)b * kmax, h.begin() + (size_t)(b + 1) * kmax);
    const double beyond = (tol > 0.0) ? h[(size_t)nb * kmax + b] : -1.0;
    const double total = h[(size_t)nb * (kmax + 1) + b];
    kb[b] = pick_rank(wb[b].data(), kmax, beyond, max_bond, tol, floor_rel);
    const double w_next = (kmax < g) ? hl[(size_t)b * g + kmax] : 0.0;
    jlo[b] = refine_start(wb[b].data(), kmax, g, kb[b], w_next, total, tol, nu, target, res);
    if (jlo[b] >= 0) any_refine = true;
    if (disc) disc[b] = discarded_rel(wb[b].data(), kmax, kb[b], beyond, total);
  }
  if (any_refine) {
    if (!rows && nb > 1) return kGroupSplit;
    Prec p1 = pr;
    p1.nb = 1;
    for (int b = 0; b < nb; ++b) {
      if (jlo[b] < 0) continue;
      const int k2 = second_level_size(kmax, kb[b], jlo[b]);
      double d = 0.0;
      int rc = refine_level2<T>(ar, p1, M + (size_t)b * mbs, m, n, kmax, jlo[b], k2, rows,
                                U + (size_t)b * ubs, W + (size_t)b * wbs, wb[b],
                                w_dev + (size_t)b * kmax, max_bond, tol, floor_rel, o, sc, s,
                                &kb[b], &d);
      if (rc != CBC_OK) return rc;
      if (disc) disc[b] = d;
    }
  }
  for (int b = 1; b < nb; ++b)
    if (kb[b] != kb[0]) return kGroupSplit;
  int k = kb[0];
  const int64_t lbs = (int64_t)k * n;
  T* L;
  if (rows) {
    L = W;
    if (nb > 1 && k < kmax) {  // instances back to back, k rows each
      L = kp.get<T>((size_t)nb * lbs);
      if (!L) return cuda_fail(kp.err, "workspace allocation L");
      CK(copy_batched<T>(W, wbs, L, lbs, lbs, s, nb));
      kp.drop(W);
    }
  } else {
    L = kp.get<T>((size_t)nb * lbs);
    if (!L) return cuda_fail(kp.err, "workspace allocation L");
    bool exact = false;  // some kept direction is below the Gram's resolution
    for (int b = 0; b < nb; ++b)
      if (resolved_prefix(wb[b].data(), k, res) < k) exact = true;
    if (!exact) {  // L = diag(sqrt(w_k)) V_k^H
      CK(scaled_adjoint_w<T>(U, kmax, w_dev, kmax, k, n, L, lbs, s, nb));
    } else {
      // diag(sqrt(w)) V^H keeps only the diagonal of V^H G V, whose off-diagonal rounding
      // (~eps w_0) is large next to the smallest kept weights; the exact factor is
      // L = Q' M with Q' an orthonormal basis of the row space of (M V_k)^H: then
      // L^H L = M^H P M, P the projector onto the span of M V_k
      const int64_t whs = (int64_t)k * m;
      T* Wh = ar.get<T>((size_t)nb * whs);
      CKA(Wh);
      CK(tgemm<T>(pr, true, false, k, m, n, U, View::transposed(kmax, ubs), true, M,
                  View::transposed(n, mbs), true, Wh, View::rowmajor(m, whs), s));
      int rc = lq_rows_inplace<T>(ar, pr, Wh, k, m, sc, s);
      if (rc != CBC_OK) return rc;
      CK(tgemm<T>(pr, true, false, k, n, m, Wh, View::rowmajor(m, whs), false, M,
                  View::rowmajor(n, mbs), false, L, View::rowmajor(n, lbs), s));
    }
  }
  CK(normalize_inplace<T>(L, lbs, sc.log_fwd, sc.status, sc.scratch, s, nb));
  if (keep) ar.release(mk);
  *Lout = L;
  *kout = k;
  return CBC_OK;
}

// S (m x n, row-major) -> Q with orthonormal rows spanning the row space of S, in place
// (CholeskyQR2; Eq. (tt_cbc_qr_decomp) is the LQ on chi_{i-1}).  Used for m < n.
// `shifted`: shifted CholeskyQR3 for S of any condition number (the first Cholesky
// factors S S^H + sigma I with sigma = 11 (m n + m (m + 1)) u ||S||^2, u the Gram's
// relative precision, which cannot break down and leaves a factor whose condition
// number CholeskyQR2 then handles; Fukaya et al., shifted CholeskyQR).
// (nb instances: S m*n elements apart.)
template <typename T>
int lq_rows_inplace(Arena& ar, const Prec& pr, T* S, int m, int n, const Scalars& sc,
                    cudaStream_t s, bool shifted) {
  const int nb = pr.nb;
  const size_t mk = ar.mark();
  T* G = ar.get<T>((size_t)nb * m * m);
  void* bar = ar.get<GridBarrier>(nb);
  double* rn = ar.get<double>((size_t)nb * m);
  CKA(G); CKA(bar); CKA(rn);
  // the mixed path solves in double-float arithmetic (FP32 pipes)
  void* dfb = nullptr;
  if (pr.mixed && !pr.cholqr_f64) {
    dfb = ar.get<char>(trsm_df_bytes(m, nb, ops<T>::cplx));
    CKA(dfb);
  }
  const int64_t sbs = (int64_t)m * n;
  // rows of S carry the graded singular values of the forward compression; scaling them
  // to unit norm keeps the row space (hence Q) and keeps the Gram well conditioned
  CK(row_norms2<T>(S, m, n, n, sbs, rn, s, nb));
  CK(scale_rows<T>(S, m, n, sbs, rn, s, nb));
  // the Gram with the first sweep's (finer) slices: CholeskyQR squares the condition
  // number, so it needs more of the product's bits than the contractions do
  Prec pg = pr;
  if (pr.cholqr_f64) pg.mixed = false;
  for (int rep = 0; rep < (shifted ? 3 : 2); ++rep) {
    CK(tgemm<T>(pg, true, true, m, m, n, S, View::rowmajor(n, sbs), false, S,
                View::transposed(n, sbs), true, G, View::rowmajor(m, (int64_t)m * m), s));
    if (shifted && rep == 0) {
      // rows of unit norm: ||S||_2^2 <= ||S||_F^2 = m; the slices' Gram carries ~2^-38
      const double u = pg.mixed ? 3.637978807091713e-12 : 1.1102230246251565e-16;
      const double shift = 11.0 * ((double)m * n + (double)m * (m + 1)) * u * m;
      CK(add_diagonal<T>(G, m, shift, s, nb));
    }
    KTimer t(CBC_K_CHOLQR, s, 0,
             nb * (ops<T>::cplx ? 4.0 : 1.0) * ((double)m * m * m / 3.0 + (double)m * m * n));
    CK(cholesky_lower<T>(G, m, sc.status, bar, num_sms(), s, nb));
    CK(trsm_lower_left<T>(G, S, m, n, sc.status, bar, num_sms(), s, nb, dfb));
  }
  ar.release(mk);
  return CBC_OK;
}

// ---- tensor train (Sec. III A) ---------------------------------------------------------
// One call runs nb instances of identical shapes in lockstep (nb = 1 for cbc_apply):
// every contraction, Gram product, eigensolve, CholeskyQR and normalisation below is one
// launch over the whole group.  Returns kGroupSplit when the instances stop agreeing on
// a rank (their outputs would differ in shape).
template <typename T>
int run_tt_group(const std::vector<const Net*>& sts, const std::vector<const Net*>& opv,
                 int64_t max_bond, double tol, const Options& o, const std::vector<Net*>& outs) {
  const Net& st = *sts[0];
  const Net& op = *opv[0];
  const int nb = (int)sts.size();
  cudaStream_t s = st.stream;
  const int L = st.n;
  // the group runs on the first instance's stream, after the others' pending work
  for (int b = 0; b < nb; ++b)
    for (cudaStream_t o2 : {sts[b]->stream, opv[b]->stream})
      if (o2 != s) {
        cudaEvent_t ev;
        CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        CK(cudaEventRecord(ev, o2));
        CK(cudaStreamWaitEvent(s, ev, 0));
        cudaEventDestroy(ev);
      }
  Arena ar(s);   // scalars, environments: the whole call
  Arena tmp(s);  // per-site temporaries, released after each site
  int* d_int = ar.get<int>(std::max(4, 1 + nb));
  double* d_dbl = ar.get<double>(std::max(4, 3 * nb));
  CKA(d_int); CKA(d_dbl);
  CK(cudaMemsetAsync(d_int, 0, std::max(4, 1 + nb) * sizeof(int), s));
  CK(cudaMemsetAsync(d_dbl, 0, std::max(4, 3 * nb) * sizeof(double), s));
  Scalars sc{d_int, d_int + 1, d_dbl, d_dbl + nb, d_dbl + 2 * nb};
  Prec pr;
  pr.mixed = (o.precision == CBC_PREC_MIXED);
  pr.cholqr_f64 = o.cholqr_f64;
  pr.s_fwd = o.slices_fwd;
  pr.s_bwd = o.slices_bwd;
  pr.ar = &tmp;
  pr.status = sc.status;
  pr.nb = nb;
  auto sb = [&](int i) { return i < L ? (int)st.bond[i] : 1; };  // alpha_{i-1} (site i's parent leg)
  auto ob = [&](int i) { return i < L ? (int)op.bond[i] : 1; };
  const std::vector<T> ones(nb, host_one<T>());
  // pointer table of the inputs, [site][state, op][instance], for the gathers
  T** in_ptrs = nullptr;
  if (nb > 1) {
    std::vector<void*> h((size_t)2 * L * nb);
    for (int i = 0; i < L; ++i)
      for (int b = 0; b < nb; ++b) {
        h[((size_t)i * 2 + 0) * nb + b] = sts[b]->data[i];
        h[((size_t)i * 2 + 1) * nb + b] = opv[b]->data[i];
      }
    in_ptrs = ar.get<T*>(h.size());
    CKA(in_ptrs);
    CK(cudaMemcpyAsync(in_ptrs, h.data(), sizeof(void*) * h.size(), cudaMemcpyHostToDevice, s));
  }
  // node tensor i of every instance, consecutive (one gather launch into `tmp` when nb > 1)
  auto site_in = [&](int i, bool opside, const T** p) -> int {
    const Net& ref = opside ? op : st;
    if (nb == 1) {
      *p = static_cast<const T*>(ref.data[i]);
      return CBC_OK;
    }
    const int64_t ne = ref.numel[i];
    T* g = tmp.get<T>((size_t)nb * ne);
    if (!g) return cuda_fail(tmp.err, "workspace allocation (gathered inputs)");
    CK(group_copy<T>(in_ptrs + ((size_t)i * 2 + (opside ? 1 : 0)) * nb, g, ne, ne, nb, true, s));
    *p = g;
    return CBC_OK;
  };

  // forward sweep: L^[0] = 1, Eq. (tt_cbc_first_contraction), compression of (chi, sigma')
  std::vector<std::vector<double>> disc(nb, std::vector<double>(L, 0.0));
  std::vector<double> dcut(nb, 0.0);
  std::vector<T*> env(L, nullptr);
  std::vector<int> chi(L, 1);
  env[0] = ar.get<T>(nb);
  CKA(env[0]);
  CK(cudaMemcpyAsync(env[0], ones.data(), sizeof(T) * nb, cudaMemcpyHostToDevice, s));
  // Zip-Up (Sec. III C) has no first sweep: it truncates during the single sweep below
  const int fwd_end = (o.method == kMethodZipUp) ? 0 : L - 1;
  for (int i = 0; i < fwd_end; ++i) {
    const int c = chi[i], b = ob(i), a = sb(i), d = (int)st.phys[i], a2 = sb(i + 1), b2 = ob(i + 1);
    const size_t mk = tmp.mark();
    const T *Ti = nullptr, *Wi = nullptr;
    int rc = site_in(i, false, &Ti);
    if (rc == CBC_OK) rc = site_in(i, true, &Wi);
    if (rc != CBC_OK) return rc;
    const int64_t tbs = (int64_t)a * d * a2, wbs = (int64_t)b * d * d * b2;
    const int64_t xbs = (int64_t)c * b * d * a2, lbs = (int64_t)c * d * b2 * a2;
    // F1: X[(chi b), (sigma a')] = sum_a L[(chi b), a] T[a, (sigma a')]
    T* X = tmp.get<T>((size_t)nb * xbs);
    if (!X) return cuda_fail(tmp.err, "workspace allocation X");
    CK(tgemm<T>(pr, true, false, c * b, d * a2, a, env[i], View::rowmajor(a, (int64_t)c * b * a),
                false, Ti, View::rowmajor(d * a2, tbs), false, X, View::rowmajor(d * a2, xbs), s));
    // F2: L'[chi, sigma', b', a'] = sum_{b, sigma} X[chi, b, sigma, a'] W[b, sigma', sigma, b']
    //     as C[(sigma' b'), (chi a')] = W[(sigma' b'), (b sigma)] X[(b sigma), (chi a')]
    T* Lp = tmp.get<T>((size_t)nb * lbs);
    if (!Lp) return cuda_fail(tmp.err, "workspace allocation L'");
    View vw;
    vw.rows2(b2, (int64_t)d * b2, 1).cols2(d, (int64_t)d * d * b2, b2);
    vw.bs = wbs;
    View vx;
    vx.rs_in = a2;
    vx.cols2(a2, (int64_t)b * d * a2, 1);
    vx.bs = xbs;
    View vl;
    vl.rs_in = a2;
    vl.cols2(a2, (int64_t)d * b2 * a2, 1);
    vl.bs = lbs;
    CK(tgemm<T>(pr, true, false, d * b2, c * a2, b * d, Wi, vw, false, X, vx, false, Lp, vl, s));
    int k = 0;
    if (o.method == kMethodSRC) {
      // SRC (Sec. III C): the sketch takes the place of the truncation, C[j, (b' a')] =
      // sum_sigma' L'[(j sigma'), (b' a')] Omega_i[sigma', j] (j shared by all sites)
      k = o.sketch;
      const int64_t cbs = (int64_t)k * b2 * a2;
      T* Cn = ar.get<T>((size_t)nb * cbs);
      CKA(Cn);
      CK(sketch_contract<T>(Lp, c, d, (int64_t)b2 * a2, static_cast<const T*>(o.sketch_mats[i]), k,
                            lbs, 0, Cn, cbs, s, nb));
      CK(normalize_inplace<T>(Cn, cbs, sc.log_fwd, sc.status, sc.scratch, s, nb));
      env[i + 1] = Cn;
    } else {
      // F3: compress M[(chi sigma'), (b' a')]
      rc = compress_rows<T>(tmp, pr, Lp, c * d, b2 * a2, max_bond, tol, o, sc, s, &env[i + 1], &k,
                            &ar, dcut.data());
      if (rc != CBC_OK) return rc;
      for (int b = 0; b < nb; ++b) disc[b][i + 1] = dcut[b];
    }
    chi[i + 1] = k;
    tmp.release(mk);
  }

  // backward sweep: R^[L] = 1, Eqs. (right_sweep_init_contr), (tt_cbc_qr_decomp),
  // (tt_cbc_final_contraction)
  for (int b = 0; b < nb; ++b) {
    Net* out = outs[b];
    out->kind = 0;
    out->n = L;
    out->root = 0;
    out->parent = sts[b]->parent;
    out->phys = sts[b]->phys;
    out->bond.assign(L, 1);
    out->children = sts[b]->children;
    out->cplx = sts[b]->cplx;
    out->stream = (nb == 1) ? s : sts[b]->stream;
    out->data.assign(L, nullptr);
    out->numel.assign(L, 0);
    out->discarded = disc[b];
  }
  T* R = ar.get<T>(nb);
  CKA(R);
  CK(cudaMemcpyAsync(R, ones.data(), sizeof(T) * nb, cudaMemcpyHostToDevice, s));
  int chiR = 1;
  for (int i = L - 1; i >= 0; --i) {
    const int a_in = sb(i), b_in = ob(i), d = (int)st.phys[i], a_out = sb(i + 1), b_out = ob(i + 1);
    const int cp = chiR, c = chi[i];
    const size_t mk = tmp.mark();
    const T *Ti = nullptr, *Wi = nullptr;
    int rc = site_in(i, false, &Ti);
    if (rc == CBC_OK) rc = site_in(i, true, &Wi);
    if (rc != CBC_OK) return rc;
    const int64_t tbs = (int64_t)a_in * d * a_out, wbs = (int64_t)b_in * d * d * b_out;
    const int64_t rbs = (int64_t)cp * b_out * a_out, ybs = (int64_t)a_in * d * cp * b_out;
    const int64_t zbs = (int64_t)b_in * a_in * d * cp;
    // B1: Y[(a sigma), (chi' b_out)] = sum_{a_out} T[(a sigma), a_out] R[(chi' b_out), a_out]
    T* Y = tmp.get<T>((size_t)nb * ybs);
    if (!Y) return cuda_fail(tmp.err, "workspace allocation Y");
    CK(tgemm<T>(pr, false, false, a_in * d, cp * b_out, a_out, Ti, View::rowmajor(a_out, tbs), false,
                R, View::transposed(a_out, rbs), false, Y, View::rowmajor(cp * b_out, ybs), s));
    // B2: Z[b_in, a, sigma', chi'] = sum_{sigma, b_out} W[b_in, sigma', sigma, b_out] Y[a, sigma, chi', b_out]
    //     as C[(b_in sigma'), (a chi')] = W[(b_in sigma'), (sigma b_out)] Y[(sigma b_out), (a chi')]
    T* Z = tmp.get<T>((size_t)nb * zbs);
    if (!Z) return cuda_fail(tmp.err, "workspace allocation Z");
    View vy;
    vy.rows2(b_out, (int64_t)cp * b_out, 1).cols2(cp, (int64_t)d * cp * b_out, b_out);
    vy.bs = ybs;
    View vz;
    vz.rows2(d, (int64_t)a_in * d * cp, cp).cols2(cp, (int64_t)d * cp, 1);
    vz.bs = zbs;
    CK(tgemm<T>(pr, false, false, b_in * d, a_in * cp, d * b_out, Wi, View::rowmajor(d * b_out, wbs),
                false, Y, vy, false, Z, vz, s));
    // B3: S[chi, (sigma' chi')] = sum_{(b a)} L^[i-1][chi, (b a)] Z[(b a), (sigma' chi')]
    const int n = d * cp;
    int m = c;
    T* Lz = nullptr;  // Zip-Up: a factor whose rows span the kept subspace (then its LQ)
    if (i > 0 && o.method == kMethodSRC) {
      // SRC: the rows of the sketch that enter the LQ, the generic rank of the sketched
      // block (beyond it the block is rank deficient): min(s, prod_{k<i} d_k, a b)
      int64_t pl = 1;
      for (int q = 0; q < i && pl < c; ++q) pl *= st.phys[q];
      m = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)c, pl, (int64_t)a_in * b_in}));
    } else if (i > 0 && o.method == kMethodZipUp) {
      // Zip-Up (Sec. III C): truncate the (sigma', chi') leg of Z[(b a), (sigma' chi')] at
      // once, by the rank rule on Z's singular values; the new tensor is an orthonormal row
      // basis of the kept right singular subspace
      int k = 0;
      rc = compress_rows<T>(tmp, pr, Z, b_in * a_in, n, max_bond, tol, o, sc, s, &Lz, &k, nullptr,
                            dcut.data());
      if (rc != CBC_OK) return rc;
      for (int b = 0; b < nb; ++b) outs[b]->discarded[i] = dcut[b];
      m = k;
    }
    // at least as many rows as columns: every unitary Q spans the whole row space, so the
    // identity is exact (and skips an ill-conditioned square CholeskyQR)
    const int cn = (m < n) ? m : n;
    const bool formed = (i == 0 || m < n);             // else Q is the identity
    const int64_t nbs = formed ? (int64_t)m * n : (int64_t)n * n;  // node stride in the group
    T* node = nullptr;
    if (nb == 1) {  // built in the output tensor itself
      CK(pool_malloc(reinterpret_cast<void**>(&node), sizeof(T) * std::max<size_t>((size_t)cn * n, (size_t)m * n), s));
      outs[0]->data[i] = node;
    } else {
      node = tmp.get<T>((size_t)nb * nbs);
      if (!node) return cuda_fail(tmp.err, "workspace allocation S");
    }
    for (int b = 0; b < nb; ++b) outs[b]->numel[i] = (int64_t)cn * n;
    if (formed && Lz) {
      CK(copy_batched<T>(Lz, (int64_t)m * n, node, nbs, (int64_t)m * n, s, nb));
    } else if (formed) {  // (SRC uses the first m of the c rows of its sketch)
      CK(tgemm<T>(pr, false, false, m, n, b_in * a_in, env[i], View::rowmajor(b_in * a_in, (int64_t)c * b_in * a_in),
                  false, Z, View::rowmajor(n, zbs), false, node, View::rowmajor(n, nbs), s));
    }
    // publishes the group's node tensors into the per-instance outputs
    auto emit = [&]() -> int {
      if (nb == 1) return CBC_OK;
      std::vector<void*> h(nb);
      for (int b = 0; b < nb; ++b) {
        CK(pool_malloc(&h[b], sizeof(T) * (size_t)cn * n, s));
        outs[b]->data[i] = h[b];
      }
      T** tab = tmp.get<T*>(nb);
      if (!tab) return cuda_fail(tmp.err, "workspace allocation (output table)");
      CK(cudaMemcpyAsync(tab, h.data(), sizeof(void*) * nb, cudaMemcpyHostToDevice, s));
      CK(group_copy<T>(tab, node, nbs, (int64_t)cn * n, nb, false, s));
      return CBC_OK;
    };
    if (i == 0) {  // T'^[1] = S^[1]
      CK(normalize_inplace<T>(node, (int64_t)n, sc.log_out, sc.status, sc.scratch, s, nb));
      for (int b = 0; b < nb; ++b) outs[b]->bond[0] = 1;
      rc = emit();
      if (rc != CBC_OK) return rc;
      tmp.release(mk);
      break;
    }
    // B4: S = R Q on chi_{i-1}; Q^[i] is the new tensor
    if (m < n) {
      // SRC: the sketched block can be arbitrarily ill conditioned (a fast-decaying
      // spectrum), so its LQ uses shifted CholeskyQR3
      rc = lq_rows_inplace<T>(tmp, pr, node, m, n, sc, s, o.method == kMethodSRC);
      if (rc != CBC_OK) return rc;
    } else {  // more rows than columns: any unitary basis of the columns; take the identity
      CK(fill_identity<T>(node, n, s, nb));
    }
    // B5: R^[i-1][chi'', (b a)] = sum_{(sigma' chi')} conj(Q[chi'', (sigma' chi')]) Z[(b a), (sigma' chi')]
    const int64_t rnbs = (int64_t)cn * b_in * a_in;
    T* Rn = ar.get<T>((size_t)nb * rnbs);
    CKA(Rn);
    CK(tgemm<T>(pr, false, false, cn, b_in * a_in, n, node, View::rowmajor(n, nbs), true, Z,
                View::transposed(n, zbs), false, Rn, View::rowmajor(b_in * a_in, rnbs), s));
    CK(normalize_inplace<T>(Rn, rnbs, sc.log_out, sc.status, sc.scratch, s, nb));
    ar.drop(R);
    R = Rn;
    chiR = cn;
    for (int b = 0; b < nb; ++b) outs[b]->bond[i] = cn;
    rc = emit();
    if (rc != CBC_OK) return rc;
    tmp.release(mk);
  }
  std::vector<int> h(1, 0);
  std::vector<double> hl(nb, 0.0);
  CK(cudaMemcpyAsync(h.data(), sc.status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(hl.data(), sc.log_out, sizeof(double) * nb, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (h[0] != 0) return status_to_rc(h[0]);
  for (int b = 0; b < nb; ++b) outs[b]->log_norm = hl[b];
  return CBC_OK;
}

template <typename T>
int run_tt_direct(const Net& st, const Net& op, int64_t max_bond, double tol, const Options& o,
                  Net* out);

template <typename T>
int run_tt(const Net& st, const Net& op, int64_t max_bond, double tol, const Options& o,
           Net* out) {
  if (o.method == kMethodDirect) return run_tt_direct<T>(st, op, max_bond, tol, o, out);
  return run_tt_group<T>({&st}, {&op}, max_bond, tol, o, {out});
}

// ---- the direct method (Sec. III C, a comparator): contract, then compress ------------
// 1. the product MPS N_i[(a b), sigma', (a' b')] = sum_sigma T[a, sigma, a'] W[b, sigma',
//    sigma, b'] (one GEMM with K = d per site, written through strided views);
// 2. sites 0 .. L-2 left-orthonormal: a tall site X (rows (l sigma') > columns r) by
//    shifted CholeskyQR3 of X^H (Q^H with orthonormal rows), R = Q^H X pushed into the next
//    site; a site that is not tall keeps the identity and passes X on whole (the reduced QR
//    then has min(l d, r) = l d columns, and any unitary gives the same state);
// 3. sites L-1 .. 1: the truncation of M = N_i[l, (sigma' r)] (compress_rows: CBC's rank
//    rule on M's singular values, which are Schmidt values since the left part is
//    orthonormal), the new tensor an orthonormal row basis of the kept subspace (LQ), the
//    carry M Q^H multiplied into site i-1.
template <typename T>
int run_tt_direct(const Net& st, const Net& op, int64_t max_bond, double tol, const Options& o,
                  Net* out) {
  cudaStream_t s = st.stream;
  const int L = st.n;
  Arena ar(s);   // the product MPS and scalars: the whole call
  Arena tmp(s);  // per-step temporaries
  int* d_int = ar.get<int>(4);
  double* d_dbl = ar.get<double>(4);
  CKA(d_int); CKA(d_dbl);
  CK(cudaMemsetAsync(d_int, 0, 4 * sizeof(int), s));
  CK(cudaMemsetAsync(d_dbl, 0, 4 * sizeof(double), s));
  Scalars sc{d_int, d_int + 1, d_dbl, d_dbl + 1, d_dbl + 2};
  Prec pr;
  pr.mixed = (o.precision == CBC_PREC_MIXED);
  pr.cholqr_f64 = o.cholqr_f64;
  pr.s_fwd = o.slices_fwd;
  pr.s_bwd = o.slices_bwd;
  pr.ar = &tmp;
  pr.status = sc.status;
  pr.nb = 1;
  auto sb = [&](int i) { return i < L ? (int)st.bond[i] : 1; };
  auto ob = [&](int i) { return i < L ? (int)op.bond[i] : 1; };
  out->kind = 0;
  out->n = L;
  out->root = 0;
  out->parent = st.parent;
  out->phys = st.phys;
  out->bond.assign(L, 1);
  out->children = st.children;
  out->cplx = st.cplx;
  out->stream = s;
  out->data.assign(L, nullptr);
  out->numel.assign(L, 0);
  out->discarded.assign(L, 0.0);
  // 1. product MPS
  std::vector<T*> N(L, nullptr);
  std::vector<int> lb(L), rb(L);  // left / right bond of N_i
  for (int i = 0; i < L; ++i) {
    const int a = sb(i), b = ob(i), d = (int)st.phys[i], A = sb(i + 1), B = ob(i + 1);
    lb[i] = a * b;
    rb[i] = A * B;
    N[i] = ar.get<T>((size_t)a * b * d * A * B);
    CKA(N[i]);
    // C[(a a'), (b sigma' b')] = T'[(a a'), sigma] W'[sigma, (b sigma' b')]
    View vt;
    vt.rows2(A, (int64_t)d * A, 1);
    vt.cs_in = A;
    View vw;
    vw.rs_in = B;
    vw.cols2(B, (int64_t)d * B, 1);  // (b sigma') has stride d B: the b stride d^2 B is d times it
    View vn;
    vn.rows2(A, (int64_t)b * d * A * B, B);
    vn.cols2(B, (int64_t)A * B, 1);
    CK(tgemm<T>(pr, false, false, a * A, b * d * B, d, static_cast<const T*>(st.data[i]), vt,
                false, static_cast<const T*>(op.data[i]), vw, false, N[i], vn, s));
  }
  // 2. left-orthonormal sites 0 .. L-2
  for (int i = 0; i + 1 < L; ++i) {
    const int d = (int)st.phys[i], p = lb[i] * d, r = rb[i];
    const int d2 = (int)st.phys[i + 1], r2 = rb[i + 1];
    const size_t mk = tmp.mark();
    T* Rm = nullptr;  // what the next site absorbs: R (r x r) or X itself (p x r)
    int nr = 0;       // its row count, the new bond
    if (p > r) {
      T* Sx = tmp.get<T>((size_t)r * p);
      Rm = tmp.get<T>((size_t)r * r);
      CKA(Sx); CKA(Rm);
      CK(adjoint_copy<T>(N[i], p, r, Sx, s));
      int rc = lq_rows_inplace<T>(tmp, pr, Sx, r, p, sc, s, true);
      if (rc != CBC_OK) return rc;
      // R = Q^H X, then X := Q
      CK(tgemm<T>(pr, false, false, r, r, p, Sx, View::rowmajor(p), false, N[i], View::rowmajor(r),
                  false, Rm, View::rowmajor(r), s));
      CK(adjoint_copy<T>(Sx, r, p, N[i], s));
      nr = r;
    } else {
      Rm = tmp.get<T>((size_t)p * r);
      CKA(Rm);
      CK(cudaMemcpyAsync(Rm, N[i], sizeof(T) * (size_t)p * r, cudaMemcpyDeviceToDevice, s));
      CK(fill_identity<T>(N[i], p, s));
      nr = p;
    }
    T* Nn = ar.get<T>((size_t)nr * d2 * r2);
    CKA(Nn);
    CK(tgemm<T>(pr, false, false, nr, d2 * r2, r, Rm, View::rowmajor(r), false, N[i + 1],
                View::rowmajor(d2 * r2), false, Nn, View::rowmajor(d2 * r2), s));
    CK(normalize_inplace<T>(Nn, (int64_t)nr * d2 * r2, sc.log_out, sc.status, sc.scratch, s));
    ar.drop(N[i + 1]);
    N[i + 1] = Nn;
    rb[i] = nr;
    lb[i + 1] = nr;
    tmp.release(mk);
  }
  // 3. truncating sweep, last site to first
  for (int i = L - 1; i >= 1; --i) {
    const int l = lb[i], d = (int)st.phys[i], n = d * rb[i];
    const size_t mk = tmp.mark();
    T* Lk = nullptr;
    int k = 0;
    double disc = 0.0;
    int rc = compress_rows<T>(tmp, pr, N[i], l, n, max_bond, tol, o, sc, s, &Lk, &k, nullptr, &disc);
    if (rc != CBC_OK) return rc;
    out->discarded[i] = disc;
    T* q = nullptr;
    CK(pool_malloc(reinterpret_cast<void**>(&q), sizeof(T) * (size_t)k * n, s));
    out->data[i] = q;
    out->numel[i] = (int64_t)k * n;
    out->bond[i] = k;
    if (k < n) {
      CK(cudaMemcpyAsync(q, Lk, sizeof(T) * (size_t)k * n, cudaMemcpyDeviceToDevice, s));
      rc = lq_rows_inplace<T>(tmp, pr, q, k, n, sc, s);
      if (rc != CBC_OK) return rc;
    } else {
      CK(fill_identity<T>(q, n, s));
    }
    // carry C = M Q^H (l x k), then N_{i-1} := N_{i-1} C
    T* Cc = tmp.get<T>((size_t)l * k);
    CKA(Cc);
    CK(tgemm<T>(pr, false, false, l, k, n, N[i], View::rowmajor(n), false, q, View::transposed(n),
                true, Cc, View::rowmajor(k), s));
    const int pl = lb[i - 1] * (int)st.phys[i - 1];
    T* Np = ar.get<T>((size_t)pl * k);
    CKA(Np);
    CK(tgemm<T>(pr, false, false, pl, k, l, N[i - 1], View::rowmajor(l), false, Cc,
                View::rowmajor(k), false, Np, View::rowmajor(k), s));
    CK(normalize_inplace<T>(Np, (int64_t)pl * k, sc.log_out, sc.status, sc.scratch, s));
    ar.drop(N[i - 1]);
    ar.drop(N[i]);
    N[i - 1] = Np;
    rb[i - 1] = k;
    tmp.release(mk);
  }
  // the first site: N_0 (1, sigma', chi_1), normalised
  {
    const int64_t n0 = (int64_t)lb[0] * st.phys[0] * rb[0];
    CK(normalize_inplace<T>(N[0], n0, sc.log_out, sc.status, sc.scratch, s));
    T* q = nullptr;
    CK(pool_malloc(reinterpret_cast<void**>(&q), sizeof(T) * (size_t)n0, s));
    CK(cudaMemcpyAsync(q, N[0], sizeof(T) * (size_t)n0, cudaMemcpyDeviceToDevice, s));
    out->data[0] = q;
    out->numel[0] = n0;
  }
  int hs = 0;
  double hl = 0.0;
  CK(cudaMemcpyAsync(&hs, sc.status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&hl, sc.log_out, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (hs != 0) return status_to_rc(hs);
  out->log_norm = hl;
  return CBC_OK;
}

// ---- trees (Sec. III B) ---------------------------------------------------------------
// Nodes with identical shapes at the same depth (and, in step 2, edges with identical
// shapes at the same depth) form groups that run in lockstep like the instances of a
// chain group: every contraction, Gram product, eigensolve, CholeskyQR and normalisation
// of a group is one launch, on node tensors and environments gathered into contiguous
// buffers.  In a perfect binary tree every depth is one group (two in step 2, one per
// child slot).  A group whose members choose different ranks runs one node at a time.

// nb tensors with named legs, row-major in the order of `legs`, size() elements apart
template <typename T>
struct DT {
  T* p = nullptr;
  std::vector<int> legs;
  std::vector<int64_t> dims;
  int nb = 1;
  int64_t size() const {
    int64_t n = 1;
    for (int64_t d : dims) n *= d;
    return n;
  }
  int pos(int leg) const {
    for (size_t i = 0; i < legs.size(); ++i)
      if (legs[i] == leg) return (int)i;
    return -1;
  }
};

// t with its legs in `order` (a copy through the permute kernel unless already so)
template <typename T>
int reorder(Arena& ar, const DT<T>& t, const std::vector<int>& order, DT<T>* out, cudaStream_t s) {
  if (order == t.legs) {
    *out = t;
    return CBC_OK;
  }
  std::vector<int> perm(order.size());
  DT<T> r;
  r.legs = order;
  r.nb = t.nb;
  for (size_t i = 0; i < order.size(); ++i) {
    perm[i] = t.pos(order[i]);
    if (perm[i] < 0) return fail(CBC_ERR_INVALID_ARG, "tree planner: leg %d missing", order[i]);
    r.dims.push_back(t.dims[perm[i]]);
  }
  r.p = ar.get<T>((size_t)t.size() * t.nb);
  CKA(r.p);
  CK(permute<T>(t.p, r.p, (int)t.legs.size(), t.dims.data(), perm.data(), s, t.nb));
  *out = r;
  return CBC_OK;
}

// Contract A and B over every leg they share; the result has A's other legs, then B's.
template <typename T>
int contract(Arena& ar, const Prec& pr, bool fwd, const DT<T>& A, const DT<T>& B, DT<T>* C,
             cudaStream_t s) {
  std::vector<int> shared, fa, fb;
  for (int l : A.legs) (B.pos(l) >= 0 ? shared : fa).push_back(l);
  for (int l : B.legs)
    if (A.pos(l) < 0) fb.push_back(l);
  std::vector<int> oa = fa, ob = shared;
  oa.insert(oa.end(), shared.begin(), shared.end());
  ob.insert(ob.end(), fb.begin(), fb.end());
  DT<T> A2, B2;
  int rc = reorder(ar, A, oa, &A2, s);
  if (rc != CBC_OK) return rc;
  rc = reorder(ar, B, ob, &B2, s);
  if (rc != CBC_OK) return rc;
  int64_t M = 1, K = 1, N = 1;
  DT<T> c;
  c.nb = A.nb;
  for (int l : fa) {
    M *= A.dims[A.pos(l)];
    c.legs.push_back(l);
    c.dims.push_back(A.dims[A.pos(l)]);
  }
  for (int l : shared) K *= A.dims[A.pos(l)];
  for (int l : fb) {
    N *= B.dims[B.pos(l)];
    c.legs.push_back(l);
    c.dims.push_back(B.dims[B.pos(l)]);
  }
  if (M > INT32_MAX || N > INT32_MAX || K > INT32_MAX)
    return fail(CBC_ERR_UNSUPPORTED, "tree planner: contraction dimension beyond 2^31");
  c.p = ar.get<T>((size_t)(M * N) * c.nb);
  CKA(c.p);
  Prec pg = pr;
  pg.nb = c.nb;
  CK(tgemm<T>(pg, fwd, false, (int)M, (int)N, (int)K, A2.p, View::rowmajor(K, M * K), false, B2.p,
              View::rowmajor(N, K * N), false, c.p, View::rowmajor(N, M * N), s));
  *C = c;
  return CBC_OK;
}

// nb tensors of ne elements (device pointers) back to back: one gather launch, none for
// a single tensor
template <typename T>
int gather(Arena& ar, const std::vector<const T*>& ptrs, int64_t ne, cudaStream_t s, T** out) {
  const int nb = (int)ptrs.size();
  if (nb == 1) {
    *out = const_cast<T*>(ptrs[0]);
    return CBC_OK;
  }
  T** tab = ar.get<T*>(nb);
  T* g = ar.get<T>((size_t)nb * ne);
  CKA(tab); CKA(g);
  CK(cudaMemcpyAsync(tab, ptrs.data(), sizeof(T*) * nb, cudaMemcpyHostToDevice, s));
  CK(group_copy<T>(tab, g, ne, ne, nb, true, s));
  *out = g;
  return CBC_OK;
}

// leg labels of one node contraction
constexpr int LG_SIN = 0, LG_SOUT = 1, LG_AP = 2, LG_BP = 3, LG_XP = 4;
inline int lg_a(int j) { return 10 + 3 * j; }
inline int lg_b(int j) { return 11 + 3 * j; }
inline int lg_x(int j) { return 12 + 3 * j; }

// groups of equal signature, in order of first appearance
std::vector<std::vector<int>> group_by(const std::vector<std::vector<int64_t>>& sig) {
  std::vector<std::vector<int>> groups;
  std::vector<int> rep;
  for (int q = 0; q < (int)sig.size(); ++q) {
    int g = -1;
    for (size_t h = 0; h < rep.size(); ++h)
      if (sig[rep[h]] == sig[q]) {
        g = (int)h;
        break;
      }
    if (g < 0) {
      rep.push_back(q);
      groups.push_back({q});
    } else {
      groups[g].push_back(q);
    }
  }
  return groups;
}

template <typename T>
int run_tree(const Net& st, const Net& op, int64_t max_bond, double tol, const Options& o,
             Net* out) {
  cudaStream_t s = st.stream;
  const int n = st.n;
  const auto& ch = st.children;
  Arena ar(s);   // environments and scalars: the whole call
  Arena tmp(s);  // per group: gathers, contractions, workspaces
  // scalars: status, k per group member, the output's log scale, and per member the
  // forward log scales (unused) and the normalisation scratch
  int* d_int = ar.get<int>(1 + n);
  double* d_dbl = ar.get<double>(1 + 2 * (size_t)n);
  CKA(d_int);
  CKA(d_dbl);
  CK(cudaMemsetAsync(d_int, 0, (1 + n) * sizeof(int), s));
  CK(cudaMemsetAsync(d_dbl, 0, (1 + 2 * (size_t)n) * sizeof(double), s));
  Scalars sc{d_int, d_int + 1, d_dbl + 1, d_dbl, d_dbl + 1 + n};
  Prec pr;
  pr.mixed = (o.precision == CBC_PREC_MIXED);
  pr.cholqr_f64 = o.cholqr_f64;
  pr.s_fwd = o.slices_fwd;
  pr.s_bwd = o.slices_bwd;
  pr.ar = &tmp;
  pr.status = sc.status;
  const T one = host_one<T>();
  std::vector<int> depth(n, 0);
  int maxd = 0;
  {
    std::vector<int> stack{st.root};
    while (!stack.empty()) {
      const int v = stack.back();
      stack.pop_back();
      for (int c : ch[v]) {
        depth[c] = depth[v] + 1;
        maxd = std::max(maxd, depth[c]);
        stack.push_back(c);
      }
    }
  }
  // node tensors of a group, gathered
  auto tensT = [&](const std::vector<int>& G, DT<T>* t) -> int {
    const int i = G[0];
    std::vector<const T*> ptrs;
    for (int g : G) ptrs.push_back(static_cast<const T*>(st.data[g]));
    t->legs = {LG_AP, LG_SIN};
    t->dims = {st.bond[i], st.phys[i]};
    for (size_t j = 0; j < ch[i].size(); ++j) {
      t->legs.push_back(lg_a((int)j));
      t->dims.push_back(st.bond[ch[i][j]]);
    }
    t->nb = (int)G.size();
    return gather<T>(tmp, ptrs, st.numel[i], s, &t->p);
  };
  auto tensW = [&](const std::vector<int>& G, DT<T>* t) -> int {
    const int i = G[0];
    std::vector<const T*> ptrs;
    for (int g : G) ptrs.push_back(static_cast<const T*>(op.data[g]));
    t->legs = {LG_BP, LG_SOUT, LG_SIN};
    t->dims = {op.bond[i], op.phys[i], op.phys[i]};
    for (size_t j = 0; j < ch[i].size(); ++j) {
      t->legs.push_back(lg_b((int)j));
      t->dims.push_back(op.bond[ch[i][j]]);
    }
    t->nb = (int)G.size();
    return gather<T>(tmp, ptrs, op.numel[i], s, &t->p);
  };
  // environments (chi, b, a) of node c (per member: envs[b]), gathered
  auto env_on = [&](const std::vector<const T*>& envs, int64_t chi, int c, int x, int b, int a,
                    DT<T>* t) -> int {
    t->legs = {x, b, a};
    t->dims = {chi, op.bond[c], st.bond[c]};
    t->nb = (int)envs.size();
    return gather<T>(tmp, envs, chi * op.bond[c] * st.bond[c], s, &t->p);
  };
  // T, the first environment, W, the remaining environments (pairwise, in this order)
  auto contract_node = [&](const DT<T>& Tt, const DT<T>& Wt, const std::vector<DT<T>>& envs,
                           const std::vector<int>& legs_out, bool fwd, DT<T>* res) -> int {
    DT<T> cur = Tt, nxt;
    int rc;
    size_t e = 0;
    if (!envs.empty()) {
      rc = contract(tmp, pr, fwd, cur, envs[0], &nxt, s);
      if (rc != CBC_OK) return rc;
      cur = nxt;
      e = 1;
    }
    rc = contract(tmp, pr, fwd, cur, Wt, &nxt, s);
    if (rc != CBC_OK) return rc;
    cur = nxt;
    for (; e < envs.size(); ++e) {
      rc = contract(tmp, pr, fwd, cur, envs[e], &nxt, s);
      if (rc != CBC_OK) return rc;
      cur = nxt;
    }
    return reorder(tmp, cur, legs_out, res, s);
  };
  std::vector<double> disc(n, 0.0);  // per edge: steps 1 and 2
  std::vector<double> dcut(n, 0.0);
  // a group, then its members one by one when they choose different ranks
  auto run_groups = [&](const std::vector<std::vector<int>>& groups,
                        const std::function<int(const std::vector<int>&)>& step) -> int {
    for (const auto& G : groups) {
      const size_t mk = tmp.mark();
      int rc = step(G);
      tmp.release(mk);
      if (rc == kGroupSplit) {
        for (int g : G) {
          const size_t mk2 = tmp.mark();
          rc = step({g});
          tmp.release(mk2);
          if (rc != CBC_OK) return rc;
        }
      } else if (rc != CBC_OK) {
        return rc;
      }
    }
    return CBC_OK;
  };

  // ---- step 1, Eq. (cbc_tree_first_contraction): subtree environments, deepest first
  std::vector<T*> Lsub(n, nullptr);
  std::vector<int64_t> chi_sub(n, 1);
  auto step1 = [&](const std::vector<int>& G) -> int {
    const int i = G[0];
    const int nb = (int)G.size();
    DT<T> Tt, Wt;
    int rc = tensT(G, &Tt);
    if (rc == CBC_OK) rc = tensW(G, &Wt);
    if (rc != CBC_OK) return rc;
    std::vector<DT<T>> envs;
    std::vector<int> lo{LG_SOUT};
    int64_t m = st.phys[i];
    for (size_t j = 0; j < ch[i].size(); ++j) {
      std::vector<const T*> ep;
      for (int g : G) ep.push_back(Lsub[ch[g][j]]);
      const int c = ch[i][j];
      DT<T> e;
      rc = env_on(ep, chi_sub[c], c, lg_x((int)j), lg_b((int)j), lg_a((int)j), &e);
      if (rc != CBC_OK) return rc;
      envs.push_back(e);
      lo.push_back(lg_x((int)j));
      m *= chi_sub[c];
    }
    lo.push_back(LG_BP);
    lo.push_back(LG_AP);
    DT<T> M;
    rc = contract_node(Tt, Wt, envs, lo, true, &M);
    if (rc != CBC_OK) return rc;
    Prec pg = pr;
    pg.nb = nb;
    const int n2 = (int)(op.bond[i] * st.bond[i]);
    T* L = nullptr;
    int k = 0;
    rc = compress_rows<T>(tmp, pg, M.p, (int)m, n2, max_bond, tol, o, sc, s, &L, &k, &ar,
                          dcut.data());
    if (rc != CBC_OK) return rc;
    for (int b = 0; b < nb; ++b) {
      Lsub[G[b]] = L + (size_t)b * k * n2;
      chi_sub[G[b]] = k;
      disc[G[b]] += dcut[b];
    }
    return CBC_OK;
  };
  for (int dd = maxd; dd >= 1; --dd) {
    std::vector<int> nodes;
    std::vector<std::vector<int64_t>> sig;
    for (int i = 0; i < n; ++i) {
      if (depth[i] != dd) continue;
      std::vector<int64_t> g{st.phys[i], st.bond[i], op.bond[i], (int64_t)ch[i].size()};
      for (int c : ch[i]) {
        g.push_back(chi_sub[c]);
        g.push_back(st.bond[c]);
        g.push_back(op.bond[c]);
      }
      nodes.push_back(i);
      sig.push_back(g);
    }
    std::vector<std::vector<int>> groups;
    for (const auto& q : group_by(sig)) {
      std::vector<int> G;
      for (int x : q) G.push_back(nodes[x]);
      groups.push_back(G);
    }
    int rc = run_groups(groups, step1);
    if (rc != CBC_OK) return rc;
  }

  // ---- step 2, Eq. (cbc_tree_second_contraction): complements, root first; an item is
  // an edge (node i, child slot jk), grouped by slot and shapes
  std::vector<T*> Ldown(n, nullptr);
  std::vector<int64_t> chi_down(n, 1);
  Ldown[st.root] = ar.get<T>(1);
  CKA(Ldown[st.root]);
  CK(cudaMemcpyAsync(Ldown[st.root], &one, sizeof(T), cudaMemcpyHostToDevice, s));
  std::vector<std::pair<int, int>> items;
  auto step2 = [&](const std::vector<int>& G) -> int {
    const int i = items[G[0]].first, jk = items[G[0]].second;
    const int nb = (int)G.size();
    std::vector<int> nodes;
    for (int q : G) nodes.push_back(items[q].first);
    DT<T> Tt, Wt;
    int rc = tensT(nodes, &Tt);
    if (rc == CBC_OK) rc = tensW(nodes, &Wt);
    if (rc != CBC_OK) return rc;
    std::vector<DT<T>> envs;
    {
      std::vector<const T*> ep;
      for (int g : nodes) ep.push_back(Ldown[g]);
      DT<T> e;
      rc = env_on(ep, chi_down[i], i, LG_XP, LG_BP, LG_AP, &e);
      if (rc != CBC_OK) return rc;
      envs.push_back(e);
    }
    std::vector<int> lo{LG_SOUT, LG_XP};
    int64_t m = st.phys[i] * chi_down[i];
    for (size_t j = 0; j < ch[i].size(); ++j) {
      if ((int)j == jk) continue;
      std::vector<const T*> ep;
      for (int g : nodes) ep.push_back(Lsub[ch[g][j]]);
      const int c = ch[i][j];
      DT<T> e;
      rc = env_on(ep, chi_sub[c], c, lg_x((int)j), lg_b((int)j), lg_a((int)j), &e);
      if (rc != CBC_OK) return rc;
      envs.push_back(e);
      lo.push_back(lg_x((int)j));
      m *= chi_sub[c];
    }
    lo.push_back(lg_b(jk));
    lo.push_back(lg_a(jk));
    DT<T> M;
    rc = contract_node(Tt, Wt, envs, lo, true, &M);
    if (rc != CBC_OK) return rc;
    const int k0 = ch[i][jk];
    Prec pg = pr;
    pg.nb = nb;
    const int n2 = (int)(op.bond[k0] * st.bond[k0]);
    T* L = nullptr;
    int kk = 0;
    rc = compress_rows<T>(tmp, pg, M.p, (int)m, n2, max_bond, tol, o, sc, s, &L, &kk, &ar,
                          dcut.data());
    if (rc != CBC_OK) return rc;
    for (int b = 0; b < nb; ++b) {
      const int kc = ch[nodes[b]][jk];
      Ldown[kc] = L + (size_t)b * kk * n2;
      chi_down[kc] = kk;
      disc[kc] += dcut[b];
    }
    return CBC_OK;
  };
  for (int dd = 0; dd < maxd; ++dd) {
    items.clear();
    std::vector<std::vector<int64_t>> sig;
    for (int i = 0; i < n; ++i) {
      if (depth[i] != dd) continue;
      for (size_t jk = 0; jk < ch[i].size(); ++jk) {
        std::vector<int64_t> g{(int64_t)jk, st.phys[i], st.bond[i], op.bond[i], chi_down[i],
                               (int64_t)ch[i].size()};
        for (size_t j = 0; j < ch[i].size(); ++j) {
          const int c = ch[i][j];
          g.push_back(j == jk ? -1 : chi_sub[c]);
          g.push_back(st.bond[c]);
          g.push_back(op.bond[c]);
        }
        items.push_back({i, (int)jk});
        sig.push_back(g);
      }
    }
    int rc = run_groups(group_by(sig), step2);
    if (rc != CBC_OK) return rc;
  }

  // ---- step 3, Eqs. (cbc_tree_third_contraction), (cbc_tree_qr), (cbc_final_contraction):
  // deepest first
  out->kind = 0;
  out->n = n;
  out->root = st.root;
  out->parent = st.parent;
  out->phys = st.phys;
  out->bond.assign(n, 1);
  out->children = st.children;
  out->cplx = st.cplx;
  out->stream = s;
  out->data.assign(n, nullptr);
  out->numel.assign(n, 0);
  out->discarded = disc;
  std::vector<T*> R(n, nullptr);
  std::vector<int64_t> chi_r(n, 1);
  auto step3 = [&](const std::vector<int>& G) -> int {
    const int i = G[0];
    const int nb = (int)G.size();
    const bool is_root = (i == st.root);
    DT<T> Tt, Wt;
    int rc = tensT(G, &Tt);
    if (rc == CBC_OK) rc = tensW(G, &Wt);
    if (rc != CBC_OK) return rc;
    // Z[(sigma', chi'_c...), (b_p, a_p)] = T W prod_c R^[c]; shared by S^[i] and R^[i]
    std::vector<DT<T>> envs;
    std::vector<int> lo{LG_SOUT};
    int64_t nz = st.phys[i];
    for (size_t j = 0; j < ch[i].size(); ++j) {
      std::vector<const T*> ep;
      for (int g : G) ep.push_back(R[ch[g][j]]);
      const int c = ch[i][j];
      DT<T> e;
      rc = env_on(ep, chi_r[c], c, lg_x((int)j), lg_b((int)j), lg_a((int)j), &e);
      if (rc != CBC_OK) return rc;
      envs.push_back(e);
      lo.push_back(lg_x((int)j));
      nz *= chi_r[c];
    }
    lo.push_back(LG_BP);
    lo.push_back(LG_AP);
    DT<T> Z;
    rc = contract_node(Tt, Wt, envs, lo, false, &Z);
    if (rc != CBC_OK) return rc;
    const int nba = (int)(op.bond[i] * st.bond[i]);
    const int m = (int)chi_down[i];
    const int nzi = (int)nz;
    const int cn = (m < nzi) ? m : nzi;  // square or tall: Q = I (exact, as on chains)
    const bool formed = is_root || m < nzi;
    const int64_t nbs = formed ? (int64_t)m * nzi : (int64_t)nzi * nzi;
    const int64_t zbs = (int64_t)nzi * nba;
    Prec pg = pr;
    pg.nb = nb;
    T* node = tmp.get<T>((size_t)nb * nbs);
    CKA(node);
    if (formed) {  // S^[i] = L^[(p_i, i)] contracted with Z over (b_p, a_p)
      std::vector<const T*> ep;
      for (int g : G) ep.push_back(Ldown[g]);
      T* Ld = nullptr;
      rc = gather<T>(tmp, ep, (int64_t)m * nba, s, &Ld);
      if (rc != CBC_OK) return rc;
      CK(tgemm<T>(pg, false, false, m, nzi, nba, Ld, View::rowmajor(nba, (int64_t)m * nba), false,
                  Z.p, View::transposed(nba, zbs), false, node, View::rowmajor(nzi, nbs), s));
    }
    if (is_root) {
      CK(normalize_inplace<T>(node, (int64_t)nzi, sc.log_out, sc.status, sc.scratch, s, nb, true));
    } else {
      if (m < nzi) {
        rc = lq_rows_inplace<T>(tmp, pg, node, m, nzi, sc, s);
        if (rc != CBC_OK) return rc;
      } else {
        CK(fill_identity<T>(node, nzi, s, nb));
      }
      // R^[i] = Q* Z over (sigma', chi'_c...)
      const int64_t rbs = (int64_t)cn * nba;
      T* Rn = ar.get<T>((size_t)nb * rbs);
      CKA(Rn);
      CK(tgemm<T>(pg, false, false, cn, nba, nzi, node, View::rowmajor(nzi, nbs), true, Z.p,
                  View::rowmajor(nba, zbs), false, Rn, View::rowmajor(nba, rbs), s));
      CK(normalize_inplace<T>(Rn, rbs, sc.log_out, sc.status, sc.scratch, s, nb, true));
      for (int b = 0; b < nb; ++b) {
        R[G[b]] = Rn + (size_t)b * rbs;
        chi_r[G[b]] = cn;
        out->bond[G[b]] = cn;
      }
    }
    // the node tensors into the output's own allocations
    const int64_t ne = is_root ? (int64_t)nzi : (int64_t)cn * nzi;
    std::vector<void*> dst(nb);
    for (int b = 0; b < nb; ++b) {
      CK(pool_malloc(&dst[b], sizeof(T) * (size_t)ne, s));
      out->data[G[b]] = dst[b];
      out->numel[G[b]] = ne;
    }
    T** tab = tmp.get<T*>(nb);
    CKA(tab);
    CK(cudaMemcpyAsync(tab, dst.data(), sizeof(void*) * nb, cudaMemcpyHostToDevice, s));
    CK(group_copy<T>(tab, node, nbs, ne, nb, false, s));
    return CBC_OK;
  };
  for (int dd = maxd; dd >= 0; --dd) {
    std::vector<int> nodes;
    std::vector<std::vector<int64_t>> sig;
    for (int i = 0; i < n; ++i) {
      if (depth[i] != dd) continue;
      std::vector<int64_t> g{st.phys[i], st.bond[i], op.bond[i], chi_down[i],
                             (int64_t)ch[i].size()};
      for (int c : ch[i]) {
        g.push_back(chi_r[c]);
        g.push_back(st.bond[c]);
        g.push_back(op.bond[c]);
      }
      nodes.push_back(i);
      sig.push_back(g);
    }
    std::vector<std::vector<int>> groups;
    for (const auto& q : group_by(sig)) {
      std::vector<int> G;
      for (int x : q) G.push_back(nodes[x]);
      groups.push_back(G);
    }
    int rc = run_groups(groups, step3);
    if (rc != CBC_OK) return rc;
  }
  int h[2];
  double hl = 0.0;
  CK(cudaMemcpyAsync(h, sc.status, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&hl, sc.log_out, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (h[0] != 0) return status_to_rc(h[0]);
  out->log_norm = hl;
  return CBC_OK;
}

bool is_chain(const Net& t) {
  for (int i = 0; i < t.n; ++i)
    if (t.parent[i] != i - 1) return false;
  return true;
}

}  // namespace

// The rank rule on weights w[0..kmax) in the order of the candidates (descending) and
// the weight `beyond` outside them (used by the tolerance rule only): keep w_j >
// floor^2 w_0 (a prefix), then the smallest k whose discarded weight sum_{j>=k} w_j +
// beyond <= tol^2 (sum_j w_j + beyond) when tol > 0, then at most max_bond; at least 1.
// This is the oracle's rule with w_j = s_j^2.
int pick_rank(const double* w, int kmax, double beyond, int64_t max_bond, double tol,
              double floor_rel) {
  if (kmax <= 0 || !(w[0] > 0.0)) return 1;
  int k = 0;
  const double fl = floor_rel * floor_rel * w[0];
  while (k < kmax && w[k] > fl) ++k;
  if (tol > 0.0) {
    std::vector<double> tail(kmax + 1);
    tail[kmax] = std::max(beyond, 0.0);
    for (int q = kmax - 1; q >= 0; --q) tail[q] = tail[q + 1] + std::max(w[q], 0.0);
    const double thr = tol * tol * tail[0];
    int kt = 0;
    while (kt < kmax && tail[kt] > thr) ++kt;
    k = std::min(k, std::max(kt, 1));
  }
  if (max_bond > 0 && k > max_bond) k = (int)max_bond;
  return std::max(k, 1);
}

// number of leading directions with w_j > res * w_0
int resolved_prefix(const double* w, int kmax, double res) {
  int j = 0;
  while (j < kmax && w[j] > res * w[0]) ++j;
  return j;
}

int refine_start(const double* w, int kmax, int g, int k, double w_next, double total,
                 double tol, double nu, double target, double res) {
  if (k < g) {
    // a direction at the cut is off by an angle ~ nu w_0 / (w_{k-1} - w_k); it mixes the
    // first dropped direction (weight w_k) into the kept ones, which moves the state by
    // about that angle times sqrt(w_k / total).  (A cut against zero-weight directions
    // moves nothing.)
    const double wk = (k < kmax) ? std::max(w[k], 0.0) : std::max(w_next, 0.0);
    const double gap = w[k - 1] - wk;
    const double est = (gap > 0.0) ? nu * w[0] / gap * std::sqrt(wk / total) : HUGE_VAL;
    if (!(est > target)) return -1;
    // the second level starts two orders of magnitude above the cut: its Gram's error
    // then scales with the weights near the cut instead of w_0
    int j = 0;
    while (j < k && w[j] > 100.0 * w[k - 1]) ++j;
    return (j >= 1) ? j : -1;
  }
  if (tol > 0.0) {  // nothing dropped, but the tolerance may cut among unresolved directions
    const int j0 = resolved_prefix(w, kmax, res);
    return (j0 >= 1 && j0 < g && g - j0 <= kMaxSecondLevel) ? j0 : -1;
  }
  return -1;
}

int second_level_size(int kmax, int k, int jlo) {
  const int near = std::max(k - jlo, 1);
  return std::min(kmax - jlo, near + std::max(16, near));
}

// frees what a failed run left in an output network, so it can be filled again
void release_outputs(Net* out) {
  bool any = false;
  for (void*& p : out->data)
    if (p) {
      cudaFreeAsync(p, out->stream);
      p = nullptr;
      any = true;
    }
  if (any) cudaStreamSynchronize(out->stream);
  cudaGetLastError();
  out->data.clear();
  out->numel.clear();
}

int run_cbc_group(const std::vector<const Net*>& sts, const std::vector<const Net*>& ops,
                  int64_t max_bond, double tol, const Options& o, const std::vector<Net*>& outs) {
  if (sts.empty() || sts.size() != ops.size() || sts.size() != outs.size())
    return fail(CBC_ERR_INVALID_ARG, "run_cbc_group: bad group");
  if (sts.size() == 1) return run_cbc(*sts[0], *ops[0], max_bond, tol, o, outs[0]);
  const Net& st = *sts[0];
  if (!is_chain(st)) return kGroupSplit;  // trees run one by one
  for (size_t b = 0; b < sts.size(); ++b)
    if (sts[b]->cplx != st.cplx || ops[b]->cplx != st.cplx || sts[b]->n != st.n ||
        sts[b]->phys != st.phys || sts[b]->bond != st.bond || ops[b]->bond != ops[0]->bond ||
        !is_chain(*sts[b]))
      return kGroupSplit;
  if (o.precision == CBC_PREC_MIXED && (o.slices_fwd < 2 || o.slices_fwd > 5 || o.slices_bwd < 2 ||
                                        o.slices_bwd > 5))
    return fail(CBC_ERR_INVALID_ARG, "cbc_apply: slice counts must be in [2, 5]");
  int rc = st.cplx ? run_tt_group<zdbl>(sts, ops, max_bond, tol, o, outs)
                   : run_tt_group<double>(sts, ops, max_bond, tol, o, outs);
  // a Cholesky breakdown on the mixed path: the members run one by one, each with the
  // FP64 fallback of run_cbc
  if (rc == CBC_ERR_NOT_POSITIVE_DEFINITE && o.precision == CBC_PREC_MIXED) return kGroupSplit;
  return rc;
}

int run_cbc(const Net& st, const Net& op, int64_t max_bond, double tol, const Options& o,
            Net* out) {
  if (st.cplx != op.cplx)
    return fail(CBC_ERR_UNSUPPORTED, "cbc_apply: state and operator must both be real or both complex");
  if (o.precision == CBC_PREC_MIXED && (o.slices_fwd < 2 || o.slices_fwd > 5 || o.slices_bwd < 2 ||
                                        o.slices_bwd > 5))
    return fail(CBC_ERR_INVALID_ARG, "cbc_apply: slice counts must be in [2, 5]");
  auto once = [&](const Options& oo) {
    if (is_chain(st)) {
      if (st.cplx) return run_tt<zdbl>(st, op, max_bond, tol, oo, out);
      return run_tt<double>(st, op, max_bond, tol, oo, out);
    }
    if (st.cplx) return run_tree<zdbl>(st, op, max_bond, tol, oo, out);
    return run_tree<double>(st, op, max_bond, tol, oo, out);
  };
  int rc = once(o);
  if (rc == CBC_ERR_NOT_POSITIVE_DEFINITE && o.precision == CBC_PREC_MIXED && !o.cholqr_f64) {
    // the slices' Gram of some backward factor S was too coarse for its condition
    // number: run the application again with FP64 Gram matrices in CholeskyQR2
    release_outputs(out);
    Options o2 = o;
    o2.cholqr_f64 = true;
    rc = once(o2);
  }
  return rc;
}

}  // namespace cbc
