// FP64 Hermitian eigensolver for the truncation of Sec. III A / III B.
//
// The paper compresses the fused leg "for example via SVD" (Sec. III A).  The GPU path
// reaches the same truncation through the Gram matrix K = M M^H (or M^H M): its
// eigenvectors are the singular vectors of M and its eigenvalues the squared singular
// values, so keeping the k largest eigenpairs keeps the same subspace as the truncated
// SVD.  Stages:
//   1. Householder reduction to a real symmetric tridiagonal T = Q^H K Q, one
//      cooperative launch; rows of K are dealt round-robin to the CTAs so the shrinking
//      trailing block stays balanced, two bounded grid barriers per column.  FP64 work
//      is spread over many SMs because one GB300 SM retires only ~2 DFMA per clock.
//   2. All eigenvalues of T by Sturm-count bisection, one thread per eigenvalue.
//   3. The rank rule (max_bond, relative floor, tolerance) on the device.
//   4. Eigenvectors of T for the kept eigenvalues by inverse iteration (LU with partial
//      pivoting of T - sigma I), modified Gram-Schmidt inside clusters of close
//      eigenvalues, Rayleigh-quotient eigenvalues.
//   5. Back transformation u = H_0 H_1 ... H_{m-2} x, one warp per kept eigenvector.
#include <float.h>

#include "kernels.cuh"
#include "planner.h"

namespace cbc {
namespace {

constexpr int TPB = 256;

template <typename T>
__device__ __forceinline__ T ldcg(const T* p);
template <>
__device__ __forceinline__ double ldcg<double>(const double* p) {
  return __ldcg(p);
}
template <>
__device__ __forceinline__ zdbl ldcg<zdbl>(const zdbl* p) {
  double2 v = __ldcg(reinterpret_cast<const double2*>(p));
  return {v.x, v.y};
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    t = warp_sum(t);
    if (threadIdx.x == 0) sh[0] = t;
  }
  __syncthreads();
  t = sh[0];
  __syncthreads();
  return t;
}

template <typename T>
struct TriArgs {
  T* A;
  int m;
  double* d;
  double* e;
  T* tau;
  T* V;     // (m-1) x m: row j = v_j (entries j+1 .. m-1, v_j[j+1] = 1)
  T* vbuf;  // 2 x m
  T* p;     // m
  double* dot;  // 2 x 2 (re, im) accumulators, double buffered
  GridBarrier* bar;
  int* status;
};

// Householder vector of column j (zlarfg convention: H = I - tau v v^H, H^H x = beta e_1,
// beta real), computed by the CTA that owns row j from its own (current) row.
template <typename T>
__device__ void householder_col(const TriArgs<T>& a, int j, double* sh) {
  using O = ops<T>;
  const int m = a.m;
  const T* row = a.A + (int64_t)j * m;
  // x_c = A[c][j] = conj(A[j][c]) for c > j
  double xn2 = 0.0;
  for (int c = j + 2 + threadIdx.x; c < m; c += blockDim.x) xn2 += O::abs2(row[c]);
  xn2 = block_sum(xn2, sh);
  T alpha = O::conj(row[j + 1]);
  double ar = O::real(alpha), ai = O::imag(alpha);
  T tau;
  double beta;
  T scale;
  bool trivial = (xn2 == 0.0 && ai == 0.0);
  if (trivial) {
    tau = O::zero();
    beta = ar;
    scale = O::zero();
  } else {
    double nrm = sqrt(ar * ar + ai * ai + xn2);
    beta = (ar >= 0.0) ? -nrm : nrm;
    tau = O::make((beta - ar) / beta, -ai / beta);
    // scale = 1 / (alpha - beta)
    double zr = ar - beta, zi = ai;
    double den = zr * zr + zi * zi;
    scale = O::make(zr / den, -zi / den);
  }
  T* vb = a.vbuf + (j & 1) * m;
  T* vs = a.V + (int64_t)j * m;
  for (int c = j + 1 + threadIdx.x; c < m; c += blockDim.x) {
    T v;
    if (c == j + 1)
      v = O::one();
    else
      v = trivial ? O::zero() : O::conj(row[c]) * scale;
    vb[c] = v;
    vs[c] = v;
  }
  if (threadIdx.x == 0) {
    a.tau[j] = tau;
    a.e[j] = beta;
    a.d[j] = O::real(row[j]);
    a.dot[(j & 1) * 2 + 0] = 0.0;
    a.dot[(j & 1) * 2 + 1] = 0.0;
  }
  __threadfence();
}

template <typename T>
__global__ void __launch_bounds__(TPB) tridiag_kernel(TriArgs<T> a) {
  using O = ops<T>;
  __shared__ double sh[64];
  const int m = a.m;
  const int P = gridDim.x, cta = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (m == 1) {
    if (cta == 0 && threadIdx.x == 0) a.d[0] = O::real(a.A[0]);
    return;
  }
  if (cta == 0) householder_col(a, 0, sh);
  if (!grid_sync(a.bar, a.status)) return;
  for (int j = 0; j < m - 1; ++j) {
    const T* v = a.vbuf + (j & 1) * m;
    const T tau = ldcg(a.tau + j);
    // ---- phase B: p_r = tau * sum_{c>j} A[r][c] v_c for own rows r > j
    // own rows: r = cta + P*t; the t-th own row goes to warp t % nw
    double dre = 0.0, dim = 0.0;
    int t0 = (j + 1 - cta + P - 1) / P;  // first t with cta + P t > j
    if (t0 < 0) t0 = 0;
    for (int t = t0 + warp; cta + P * t < m; t += nw) {
      int r = cta + P * t;
      const T* row = a.A + (int64_t)r * m;
      T acc = O::zero();
      for (int c = j + 1 + lane; c < m; c += 32) acc = O::fma(row[c], ldcg(v + c), acc);
      if constexpr (O::cplx) {
        acc = zdbl{warp_sum(O::real(acc)), warp_sum(O::imag(acc))};
      } else {
        acc = warp_sum(acc);
      }
      T pr = tau * acc;
      if (lane == 0) {
        a.p[r] = pr;
        T vd = O::conj(ldcg(v + r)) * pr;
        dre += O::real(vd);
        dim += O::imag(vd);
      }
    }
    dre = block_sum(dre, sh);
    if constexpr (O::cplx) dim = block_sum(dim, sh);
    if (threadIdx.x == 0) {
      atomicAdd(a.dot + (j & 1) * 2 + 0, dre);
      if constexpr (O::cplx) atomicAdd(a.dot + (j & 1) * 2 + 1, dim);
    }
    if (!grid_sync(a.bar, a.status)) return;
    // ---- phase C: A22 -= v w^H + w v^H, w = p - (conj(tau)/2) (v^H p) v
    T s = O::make(__ldcg(a.dot + (j & 1) * 2 + 0), __ldcg(a.dot + (j & 1) * 2 + 1));
    T coef = O::scale(-0.5, O::conj(tau) * s);
    for (int t = t0 + warp; cta + P * t < m; t += nw) {
      int r = cta + P * t;
      T* row = a.A + (int64_t)r * m;
      T vr = ldcg(v + r);
      T wr = O::fma(coef, vr, ldcg(a.p + r));
      for (int c = j + 1 + lane; c < m; c += 32) {
        T vc = ldcg(v + c);
        T wc = O::fma(coef, vc, ldcg(a.p + c));
        T upd = O::fma(vr, O::conj(wc), wr * O::conj(vc));
        row[c] = row[c] - upd;
      }
    }
    __syncthreads();
    if (j + 1 < m - 1) {
      if ((j + 1) % P == cta) householder_col(a, j + 1, sh);
    } else if ((m - 1) % P == cta && threadIdx.x == 0) {
      a.d[m - 1] = O::real(a.A[(int64_t)(m - 1) * m + (m - 1)]);
    }
    if (!grid_sync(a.bar, a.status)) return;
  }
}

// ---- Sturm count: number of eigenvalues of T smaller than x -------------------------
__device__ __forceinline__ int sturm_count(const double* d, const double* e, int m, double x,
                                           double pivmin) {
  int cnt = 0;
  double q = d[0] - x;
  if (q < 0.0) cnt++;
  for (int i = 1; i < m; ++i) {
    if (fabs(q) < pivmin) q = -pivmin;
    q = (d[i] - x) - (e[i - 1] * e[i - 1]) / q;
    if (q < 0.0) cnt++;
  }
  return cnt;
}

struct BisArgs {
  const double* d;
  const double* e;
  double* e2;  // scratch m
  int m;
  double* lam;  // out, descending
};

__global__ void bisect_kernel(BisArgs b) {
  __shared__ double s_lo, s_hi, s_piv;
  const int m = b.m;
  if (threadIdx.x == 0) {
    double lo = DBL_MAX, hi = -DBL_MAX, emax = 0.0;
    for (int i = 0; i < m; ++i) {
      double r = 0.0;
      if (i > 0) r += fabs(b.e[i - 1]);
      if (i < m - 1) r += fabs(b.e[i]);
      lo = fmin(lo, b.d[i] - r);
      hi = fmax(hi, b.d[i] + r);
      if (i < m - 1) emax = fmax(emax, b.e[i] * b.e[i]);
    }
    double span = fmax(fabs(lo), fabs(hi));
    s_lo = lo - 1e-14 * span - DBL_MIN;
    s_hi = hi + 1e-14 * span + DBL_MIN;
    s_piv = DBL_MIN * fmax(1.0, emax);
  }
  __syncthreads();
  int jj = blockIdx.x * blockDim.x + threadIdx.x;  // descending index
  if (jj >= m) return;
  const int target = m - 1 - jj;                    // ascending index
  double lo = s_lo, hi = s_hi;
  const double span = fmax(fabs(lo), fabs(hi));
  const double atol = 2e-12 * span + 4.0 * s_piv;
  for (int it = 0; it < 80 && (hi - lo) > atol; ++it) {
    double mid = 0.5 * (lo + hi);
    if (sturm_count(b.d, b.e, m, mid, s_piv) <= target)
      lo = mid;
    else
      hi = mid;
  }
  b.lam[jj] = 0.5 * (lo + hi);
}

// rank rule on the (descending) eigenvalues
__global__ void rank_kernel(const double* lam, int m, int kmax, long long max_bond, double tol,
                            double floor_rel, int* k_dev) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double l0 = lam[0];
  int k;
  if (!(l0 > 0.0)) {
    k = 1;
  } else {
    k = 0;
    while (k < m && lam[k] > floor_rel * l0) ++k;
    if (tol > 0.0) {
      double total = 0.0;
      for (int j = 0; j < m; ++j) total += fmax(lam[j], 0.0);
      double tail = total;
      int kt = 0;
      // smallest kt with sum_{j>=kt} <= tol^2 total
      while (kt < m && tail > tol * tol * total) {
        tail -= fmax(lam[kt], 0.0);
        ++kt;
      }
      if (kt < 1) kt = 1;
      if (kt < k) k = kt;
    }
    if (max_bond > 0 && k > max_bond) k = (int)max_bond;
    if (k < 1) k = 1;
  }
  if (k > kmax) k = kmax;
  *k_dev = k;
}

// ---- inverse iteration for the kept eigenvalues ------------------------------------
struct InvArgs {
  const double* d;
  const double* e;
  const double* lamb;  // bisection values (read only: cluster bounds and shifts)
  double* lam;         // out: Rayleigh quotients for kept j, bisection values otherwise
  int m;
  const int* k_dev;
  double* X;    // m x kmax (row i, column jj), eigenvectors of T
  int kmax;
  // per-thread scratch, layout [i][jj]
  double *dl, *dd, *du, *du2, *b;
  unsigned char* piv;
};

__device__ __forceinline__ uint32_t hash32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352dU;
  x ^= x >> 15;
  x *= 0x846ca68bU;
  x ^= x >> 16;
  return x;
}

__global__ void inverse_iter_kernel(InvArgs a) {
  const int m = a.m, K = a.kmax;
  const int k = *a.k_dev;
  const int jj = blockIdx.x * blockDim.x + threadIdx.x;
  if (jj >= m) return;
  if (jj >= k) {
    a.lam[jj] = a.lamb[jj];
    return;
  }
  const double span = fmax(fabs(a.lamb[0]), fabs(a.lamb[m - 1])) + DBL_MIN;
  const double ortol = 1e-3 * span;
  // only the first member of a cluster works; it computes the whole cluster in order
  if (jj > 0 && a.lamb[jj - 1] - a.lamb[jj] <= ortol) return;
  int cend = jj + 1;
  while (cend < k && a.lamb[cend - 1] - a.lamb[cend] <= ortol) ++cend;
#define AT(arr, i) arr[(int64_t)(i) * K + jj]
  const double eps = 2.220446049250313e-16;
  for (int jc = jj; jc < cend; ++jc) {
    double sigma = a.lamb[jc];
    // perturb members of a cluster apart so their shifts differ
    if (jc > jj) {
      double prev = a.lamb[jc - 1];
      if (prev - sigma < 10.0 * eps * span) sigma = prev - 10.0 * eps * span;
    }
    // LU with partial pivoting of T - sigma I (dgttrf layout)
    for (int i = 0; i < m; ++i) {
      AT(a.dd, i) = a.d[i] - sigma;
      if (i < m - 1) {
        AT(a.dl, i) = a.e[i];
        AT(a.du, i) = a.e[i];
      }
    }
    for (int i = 0; i < m - 1; ++i) {
      double di = AT(a.dd, i), li = AT(a.dl, i);
      if (fabs(di) >= fabs(li)) {
        AT(a.piv, i) = 0;
        double f = (di != 0.0) ? li / di : 0.0;
        AT(a.dl, i) = f;
        AT(a.dd, i + 1) -= f * AT(a.du, i);
        if (i < m - 2) AT(a.du2, i) = 0.0;
      } else {
        AT(a.piv, i) = 1;
        double f = di / li;
        AT(a.dd, i) = li;
        AT(a.dl, i) = f;
        double tmp = AT(a.du, i);
        AT(a.du, i) = AT(a.dd, i + 1);
        AT(a.dd, i + 1) = tmp - f * AT(a.dd, i + 1);
        if (i < m - 2) {
          AT(a.du2, i) = AT(a.du, i + 1);
          AT(a.du, i + 1) = -f * AT(a.du, i + 1);
        }
      }
    }
    const double tiny = eps * span;
    for (int i = 0; i < m; ++i)
      if (fabs(AT(a.dd, i)) < tiny) AT(a.dd, i) = (AT(a.dd, i) < 0.0) ? -tiny : tiny;
    // start vector
    for (int i = 0; i < m; ++i) {
      uint32_t h = hash32((uint32_t)(i * 7919 + jc * 104729 + 17));
      AT(a.b, i) = ((double)(h & 0xffffff) / 16777216.0) - 0.5;
    }
    for (int it = 0; it < 4; ++it) {
      // forward: L y = P b (in place in b)
      for (int i = 0; i < m - 1; ++i) {
        if (AT(a.piv, i) == 0) {
          AT(a.b, i + 1) -= AT(a.dl, i) * AT(a.b, i);
        } else {
          double t = AT(a.b, i);
          AT(a.b, i) = AT(a.b, i + 1);
          AT(a.b, i + 1) = t - AT(a.dl, i) * AT(a.b, i + 1);
        }
      }
      // back: U x = y
      for (int i = m - 1; i >= 0; --i) {
        double s = AT(a.b, i);
        if (i < m - 1) s -= AT(a.du, i) * AT(a.b, i + 1);
        if (i < m - 2) s -= AT(a.du2, i) * AT(a.b, i + 2);
        AT(a.b, i) = s / AT(a.dd, i);
      }
      // orthogonalise against earlier members of the cluster (their vectors are in X)
      for (int q = jj; q < jc; ++q) {
        double dotv = 0.0;
        for (int i = 0; i < m; ++i) dotv += a.X[(int64_t)i * K + q] * AT(a.b, i);
        for (int i = 0; i < m; ++i) AT(a.b, i) -= dotv * a.X[(int64_t)i * K + q];
      }
      double nrm = 0.0;
      for (int i = 0; i < m; ++i) nrm += AT(a.b, i) * AT(a.b, i);
      nrm = sqrt(nrm);
      double inv = (nrm > 0.0) ? 1.0 / nrm : 0.0;
      for (int i = 0; i < m; ++i) AT(a.b, i) *= inv;
    }
    // store and Rayleigh quotient
    double rq = 0.0;
    for (int i = 0; i < m; ++i) {
      double xi = AT(a.b, i);
      double tx = a.d[i] * xi;
      if (i > 0) tx += a.e[i - 1] * AT(a.b, i - 1);
      if (i < m - 1) tx += a.e[i] * AT(a.b, i + 1);
      rq += xi * tx;
      a.X[(int64_t)i * K + jc] = xi;
    }
    a.lam[jc] = rq;
  }
#undef AT
}

// ---- back transformation: U[:, jj] = H_0 ... H_{m-2} X[:, jj] ------------------------
template <typename T>
__global__ void backtransform_kernel(const T* V, const T* tau, const double* X, int m, int kmax,
                                     const int* k_dev, T* U) {
  using O = ops<T>;
  extern __shared__ unsigned char smem_raw[];
  T* u_all = reinterpret_cast<T*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int jj = blockIdx.x * (blockDim.x >> 5) + warp;
  const int k = *k_dev;
  if (jj >= k) return;
  T* u = u_all + warp * m;
  for (int i = lane; i < m; i += 32) u[i] = O::make(X[(int64_t)i * kmax + jj], 0.0);
  __syncwarp();
  for (int j = m - 2; j >= 0; --j) {
    const T* vj = V + (int64_t)j * m;
    T t = tau[j];
    if (O::real(t) == 0.0 && O::imag(t) == 0.0) continue;
    T s = O::zero();
    for (int r = j + 1 + lane; r < m; r += 32) s = O::fma(O::conj(vj[r]), u[r], s);
    if constexpr (O::cplx) {
      s = zdbl{warp_sum(O::real(s)), warp_sum(O::imag(s))};
    } else {
      s = warp_sum(s);
    }
    T ts = t * s;
    __syncwarp();
    for (int r = j + 1 + lane; r < m; r += 32) u[r] = u[r] - vj[r] * ts;
    __syncwarp();
  }
  for (int i = lane; i < m; i += 32) U[(int64_t)i * kmax + jj] = u[i];
}

}  // namespace

// workspace layout (all 256-byte aligned)
static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

size_t eig_workspace_bytes(int m, int kmax, bool cplx) {
  size_t ts = cplx ? sizeof(zdbl) : sizeof(double);
  size_t b = 0;
  b += align256(sizeof(double) * m);                 // d
  b += align256(sizeof(double) * m);                 // e
  b += align256(sizeof(double) * m);                 // e2
  b += align256(sizeof(double) * m);                 // lamb
  b += align256(ts * m);                             // tau
  b += align256(ts * (size_t)m * m);                 // V
  b += align256(ts * 2 * m);                         // vbuf
  b += align256(ts * m);                             // p
  b += align256(sizeof(double) * 4);                 // dot
  b += align256(sizeof(GridBarrier));                // barrier
  b += align256(sizeof(double) * (size_t)m * kmax);  // X
  b += 5 * align256(sizeof(double) * (size_t)m * kmax);  // dl dd du du2 b
  b += align256((size_t)m * kmax);                   // piv
  return b;
}

template <typename T>
cudaError_t heev_top(T* A, int m, int kmax, int64_t max_bond, double tol, double floor_rel,
                     double* lam, T* U, int* k_dev, void* work, int* status, int num_sms,
                     cudaStream_t s) {
  char* w = static_cast<char*>(work);
  auto take = [&](size_t bytes) {
    char* p = w;
    w += align256(bytes);
    return p;
  };
  const size_t ts = sizeof(T);
  double* d = (double*)take(sizeof(double) * m);
  double* e = (double*)take(sizeof(double) * m);
  double* e2 = (double*)take(sizeof(double) * m);
  double* lamb = (double*)take(sizeof(double) * m);
  T* tau = (T*)take(ts * m);
  T* V = (T*)take(ts * (size_t)m * m);
  T* vbuf = (T*)take(ts * 2 * m);
  T* p = (T*)take(ts * m);
  double* dot = (double*)take(sizeof(double) * 4);
  GridBarrier* bar = (GridBarrier*)take(sizeof(GridBarrier));
  double* X = (double*)take(sizeof(double) * (size_t)m * kmax);
  double* dl = (double*)take(sizeof(double) * (size_t)m * kmax);
  double* dd = (double*)take(sizeof(double) * (size_t)m * kmax);
  double* du = (double*)take(sizeof(double) * (size_t)m * kmax);
  double* du2 = (double*)take(sizeof(double) * (size_t)m * kmax);
  double* bb = (double*)take(sizeof(double) * (size_t)m * kmax);
  unsigned char* piv = (unsigned char*)take((size_t)m * kmax);

  cudaError_t err = cudaMemsetAsync(bar, 0, sizeof(GridBarrier), s);
  if (err != cudaSuccess) return err;
  err = cudaMemsetAsync(tau, 0, ts * m, s);
  if (err != cudaSuccess) return err;

  note_launches(CBC_K_EIG, 5);
  // 1. tridiagonalisation (cooperative)
  int P = m / 4;
  if (P < 1) P = 1;
  if (P > num_sms) P = num_sms;
  TriArgs<T> ta{A, m, d, e, tau, V, vbuf, p, dot, bar, status};
  void* args[] = {&ta};
  err = cudaLaunchCooperativeKernel((const void*)tridiag_kernel<T>, dim3(P), dim3(TPB), args, 0,
                                    s);
  if (err != cudaSuccess) return err;
  // 2. eigenvalues
  BisArgs ba{d, e, e2, m, lamb};
  bisect_kernel<<<(m + 63) / 64, 64, 0, s>>>(ba);
  // 3. rank
  rank_kernel<<<1, 32, 0, s>>>(lamb, m, kmax, (long long)max_bond, tol, floor_rel, k_dev);
  // 4. eigenvectors of T
  InvArgs ia{d, e, lamb, lam, m, k_dev, X, kmax, dl, dd, du, du2, bb, piv};
  inverse_iter_kernel<<<(m + 31) / 32, 32, 0, s>>>(ia);
  // 5. back transformation
  int wpb = 4;
  size_t shm = (size_t)wpb * m * ts;
  if (shm > 200 * 1024) {
    wpb = 1;
    shm = (size_t)m * ts;
  }
  if (shm > 48 * 1024) {
    err = cudaFuncSetAttribute(backtransform_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)shm);
    if (err != cudaSuccess) return err;
  }
  backtransform_kernel<T><<<(kmax + wpb - 1) / wpb, 32 * wpb, shm, s>>>(V, tau, X, m, kmax, k_dev,
                                                                         U);
  return cudaGetLastError();
}

template cudaError_t heev_top<double>(double*, int, int, int64_t, double, double, double*,
                                      double*, int*, void*, int*, int, cudaStream_t);
template cudaError_t heev_top<zdbl>(zdbl*, int, int, int64_t, double, double, double*, zdbl*,
                                    int*, void*, int*, int, cudaStream_t);

}  // namespace cbc
