// Internal launch interface of the CBC kernels (host side).  Not part of the C ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace cbc {

// A matrix view over strided memory.  Element (r, c) of batch b lives at
//   base + b*bs + (r / r_in)*rs_out + (r % r_in)*rs_in + (c / c_in)*cs_out + (c % c_in)*cs_in
// so a row or column index may itself be a pair of tensor legs with unrelated strides
// (a leg permutation of a node tensor is a view, never a copy).
struct View {
  int32_t r_in = 0x7fffffff;
  int64_t rs_out = 0, rs_in = 0;
  int32_t c_in = 0x7fffffff;
  int64_t cs_out = 0, cs_in = 0;
  int64_t bs = 0;

  static View rowmajor(int64_t ld, int64_t bs = 0) {
    View v;
    v.rs_in = ld;
    v.cs_in = 1;
    v.bs = bs;
    return v;
  }
  // the transpose of a row-major matrix with leading dimension ld
  static View transposed(int64_t ld, int64_t bs = 0) {
    View v;
    v.rs_in = 1;
    v.cs_in = ld;
    v.bs = bs;
    return v;
  }
  View& rows2(int32_t inner, int64_t s_out, int64_t s_in) {
    r_in = inner;
    rs_out = s_out;
    rs_in = s_in;
    return *this;
  }
  View& cols2(int32_t inner, int64_t s_out, int64_t s_in) {
    c_in = inner;
    cs_out = s_out;
    cs_in = s_in;
    return *this;
  }
  __host__ __device__ __forceinline__ int64_t roff(int32_t r) const {
    return (int64_t)(r / r_in) * rs_out + (int64_t)(r % r_in) * rs_in;
  }
  __host__ __device__ __forceinline__ int64_t coff(int32_t c) const {
    return (int64_t)(c / c_in) * cs_out + (int64_t)(c % c_in) * cs_in;
  }
};

// C = op(A) op(B), C: M x N, A: M x K, B: K x N, `batch` independent products.
// conjA / conjB take the complex conjugate of the operand elements (no transpose:
// transposes are views).  FP64 SIMT, FP64 accumulation; split over K when the output
// alone cannot fill the GPU.
template <typename T>
cudaError_t gemm_f64(int M, int N, int K, int batch, const T* A, const View& va, bool conjA,
                     const T* B, const View& vb, bool conjB, T* C, const View& vc,
                     cudaStream_t s);

// The same product on the tensor cores with S bf16 slices per operand (gemm_tc.cu);
// `ws` must hold gemm_tc_workspace_bytes(M, N, K, cplx, S, nb) bytes.  nb problems of
// one shape, their operands va.bs / vb.bs / vc.bs elements apart, in one launch.
size_t gemm_tc_workspace_bytes(int M, int N, int K, bool cplx, int S, int nb = 1);
template <typename T>
cudaError_t gemm_tc(int M, int N, int K, const T* A, const View& va, bool conjA, const T* B,
                    const View& vb, bool conjB, T* C, const View& vc, int S, void* ws,
                    int* status, cudaStream_t s, int nb = 1);

// ---- Hermitian eigensolver (FP64): A (m x m, row-major, overwritten) -----------------
// Finds the eigenvalues in descending order and the eigenvectors of the `k` largest,
// where k = min(max_bond (if > 0), #{lambda_j > floor * lambda_0}, smallest k with
// sum_{j>=k} lambda_j <= tol^2 sum_j lambda_j (if tol > 0)), at least 1; floor < 0 gives
// k = kmax (every candidate).  Outputs: lam[m], U (m x kmax, row-major, column j =
// eigenvector j), *k_dev.  Workspace: eig_workspace_bytes(m, kmax).
struct EigWork;
size_t eig_workspace_bytes(int m, int kmax, bool cplx);
template <typename T>
cudaError_t heev_top(T* A, int m, int kmax, int64_t max_bond, double tol, double floor_rel,
                     double* lam, T* U, int* k_dev, void* work, int* status, int num_sms,
                     cudaStream_t s, int nb = 1, bool prefer_cluster = false,
                     bool df = false);

// Householder tridiagonalisation by one thread-block cluster per matrix (rows in shared
// memory, exchanges through distributed shared memory; tridiag_cluster.cu).  Outputs as
// the eigensolver's first stage: d, e, tau, V (row j = [tau_j, 1, v_j...] from column j),
// per matrix wb bytes apart; A: nb matrices a_bs elements apart.  df: double-float rows.
// tridiag_cluster_size returns the cluster size that fits (4, 8 or 16), 0 if none.
template <typename T>
int tridiag_cluster_size(int m, bool df);
template <typename T>
cudaError_t tridiag_cluster(const T* A, int m, double* d, double* e, T* tau, T* V, int64_t a_bs,
                            size_t wb, int nb, int P, bool df, cudaStream_t s);

// ---- Cholesky QR (FP64) ------------------------------------------------------------
// Q = C^{-1} S with G = S S^H = C C^H, S: m x n (m <= n), row-major, in place on S.
// nb problems: G, C m*m and S m*n elements apart; `bar` holds nb GridBarriers.
template <typename T>
cudaError_t cholesky_lower(T* G, int m, int* status, void* bar, int num_sms, cudaStream_t s,
                           int nb = 1);
// dfbuf: NULL for the FP64 solve; else room for trsm_df_bytes(m, nb) bytes, and the solve
// runs in double-float arithmetic (the mixed path)
template <typename T>
cudaError_t trsm_lower_left(const T* C, T* S, int m, int n, int* status, void* bar,
                            int num_sms, cudaStream_t s, int nb = 1, void* dfbuf = nullptr);
inline size_t trsm_df_bytes(int m, int nb, bool cplx) {
  return (size_t)nb * ((size_t)m * m * (cplx ? 16 : 8) + (size_t)m * 8);
}

// ---- small helpers ------------------------------------------------------------------
// Let `func` use up to the device's opt-in shared memory per block.  Every caller sets
// the same value, so concurrent calls from several host threads cannot shrink the
// limit under another thread's launch.
cudaError_t allow_max_smem(const void* func);
// Largest feasible single-cluster size <= want (<= 16) for func; 0 if none.
int cluster_ctas(const void* func, int want, int threads, size_t smem);
// Launch func over `grid` CTAs in clusters of `cluster` CTAs (each cluster co-scheduled;
// clusters are concurrent with other streams' work).
cudaError_t launch_cluster(const void* func, int cluster, int grid, int threads, size_t smem,
                           void** args, cudaStream_t s);

// x[i] (i < n) scaled in place to unit Frobenius norm; log of the old norm added to
// *log_acc; non-finite norm sets CBC_ERR_NUMERICAL.  nb problems: x n elements apart,
// log_acc and scratch one double apart.
// shared_log: every problem's log is added into log_acc[0] (atomically) instead of
// log_acc[b]; scratch still needs nb doubles
template <typename T>
cudaError_t normalize_inplace(T* x, int64_t n, double* log_acc, int* status, double* scratch,
                              cudaStream_t s, int nb = 1, bool shared_log = false);
// L[r, c] = sqrt(lam[r]) * conj(V[c, r]) for r < k (V: n x ldv row-major), L: k x n;
// nb problems: V n*ldv, lam n, k_dev 1 and L l_bs elements apart
template <typename T>
cudaError_t scaled_adjoint(const T* V, int ldv, const double* lam, const int* k_dev, int n,
                           T* L, cudaStream_t s, int nb = 1, int64_t l_bs = 0);
// out = in with its axes permuted: out dims are in dims[perm[0]], in dims[perm[1]], ...
// (row-major, rank <= 8); nb tensors of the same shape, back to back in in and out
template <typename T>
cudaError_t permute(const T* in, T* out, int rank, const int64_t* in_dims, const int* perm,
                    cudaStream_t s, int nb = 1);
// Squared 2-norms of the rows (out[b * rows + r]) or of the columns (out[b * cols + c])
// of nb row-major matrices rows x cols with leading dimension ld, bs elements apart.
template <typename T>
cudaError_t row_norms2(const T* W, int rows, int cols, int64_t ld, int64_t bs, double* out,
                       cudaStream_t s, int nb = 1);
template <typename T>
cudaError_t col_norms2(const T* W, int rows, int cols, int64_t ld, int64_t bs, double* out,
                       cudaStream_t s, int nb = 1);
// rows r of nb row-major matrices (rows x cols, bs elements apart) scaled by
// 1 / sqrt(norms2[b * rows + r]) (rows of zero norm are left alone)
template <typename T>
cudaError_t scale_rows(T* X, int rows, int cols, int64_t bs, const double* norms2,
                       cudaStream_t s, int nb = 1);
// out[b] = sum_i |A_b[i] - B_b[i]|^2 over n contiguous elements (A_b = A + b * a_bs,
// B_b = B + b * n); C_b = A_b - B_b as well when C is not NULL (C_b = C + b * n)
template <typename T>
cudaError_t diff_sumsq(const T* A, int64_t a_bs, const T* B, T* C, int64_t n, double* out,
                       cudaStream_t s, int nb = 1);
// sum of |x|^2 over n contiguous elements per problem (problems n apart) into out[b]
template <typename T>
cudaError_t sum_squares(const T* x, int64_t n, double* out, cudaStream_t s, int nb = 1);
// L[r, c] = sqrt(w[r]) conj(V[c, r]) for r < k (V: n x ldv row-major), L: k x n; nb
// problems with V n*ldv, w w_bs and L l_bs elements apart
template <typename T>
cudaError_t scaled_adjoint_w(const T* V, int ldv, const double* w, int64_t w_bs, int k, int n,
                             T* L, int64_t l_bs, cudaStream_t s, int nb = 1);
// Sketch step of SRC (Sec. III C): C[j, col] = sum_p Lp[(cj, p), col] * om[p, j] with
// cj = j (c == s) or 0 (c == 1, the first site), Lp: (c d) x ncol row-major, om: d x s
// row-major, C: s x ncol; nb problems, Lp lp_bs, om om_bs and C c_bs elements apart.
template <typename T>
cudaError_t sketch_contract(const T* Lp, int c, int d, int64_t ncol, const T* om, int s,
                            int64_t lp_bs, int64_t om_bs, T* C, int64_t c_bs, cudaStream_t st,
                            int nb = 1);
// out[b] = the real part of the trace of G_b (g x g, nb matrices bs elements apart)
template <typename T>
cudaError_t trace_real(const T* G, int g, int64_t bs, double* out, cudaStream_t s, int nb = 1);
// out (cols x rows, row-major) = the conjugate transpose of in (rows x cols, row-major)
template <typename T>
cudaError_t adjoint_copy(const T* in, int rows, int cols, T* out, cudaStream_t s);
// G_b[i, i] += shift for i < m (nb matrices m*m elements apart)
template <typename T>
cudaError_t add_diagonal(T* G, int m, double shift, cudaStream_t s, int nb = 1);
// dst_b[i] = src_b[i] for i < n, src_b = src + b * s_bs, dst_b = dst + b * d_bs
template <typename T>
cudaError_t copy_batched(const T* src, int64_t s_bs, T* dst, int64_t d_bs, int64_t n,
                         cudaStream_t s, int nb = 1);
// dst (n_elem) = identity rows r < n of an n x n matrix
template <typename T>
cudaError_t fill_identity(T* dst, int n, cudaStream_t s, int nb = 1);
// nb tensors (device array ptrs of nb pointers, n elements each) <-> one buffer with them
// `stride` elements apart: to_group gathers into buf, else scatters out of it
template <typename T>
cudaError_t group_copy(T* const* ptrs, T* buf, int64_t stride, int64_t n, int nb, bool to_group,
                       cudaStream_t s);
// widen an input tensor to FP64 storage; *nonfinite (if given) is set to 1 when a value
// is NaN or infinite
cudaError_t widen_to_f64(const void* src, int src_dtype, void* dst, int64_t n_elem,
                         cudaStream_t s, int* nonfinite = nullptr);
// narrow FP64 storage to the requested dtype
cudaError_t narrow_from_f64(const void* src, bool cplx, void* dst, int dst_dtype,
                            int64_t n_elem, cudaStream_t s);

}  // namespace cbc
