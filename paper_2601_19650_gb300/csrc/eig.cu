// FP64 Hermitian eigensolver for the truncation of Sec. III A / III B.
//
// The paper names an SVD as one way to compress the fused leg (Sec. III A).  The GPU path
// reaches the same truncation through the Gram matrix K = M M^H (or M^H M): its
// eigenvectors are the singular vectors of M and its eigenvalues the squared singular
// values, so keeping the k largest eigenpairs keeps the same subspace as the truncated
// SVD.  Stages:
//   1. Householder reduction to a real symmetric tridiagonal T = Q^H K Q by one group
//      of CTAs that wait on each other (a thread-block cluster when the rows fit in its
//      shared memory, else a cooperative launch); rows of K are dealt round-robin to the
//      CTAs so the shrinking trailing block stays balanced.  FP64 work is spread over
//      several SMs because one GB300 SM retires only ~2 DFMA per clock.
//   2. Estimates of all eigenvalues of T by single-precision Sturm-count multisection,
//      one warp per eigenvalue (a dependent chain of FP64 divisions per Sturm step is
//      slow on this part; the estimates only need to separate the eigenvalues).
//   3. Eigenvectors of T for the candidates (the kmax largest) by FP64 inverse
//      iteration seeded with those estimates (one LU, four solves); eigenvalues =
//      Rayleigh quotients.
//   4. The rank rule (max_bond, relative floor, tolerance) on the refined eigenvalues,
//      with the discarded weight taken as trace(T) minus the kept eigenvalues.
//   5. Back transformation u = H_0 H_1 ... H_{m-2} x, one warp per kept eigenvector.
#include <float.h>

#include <algorithm>
#include <type_traits>
#include <cstdlib>

#include "df.cuh"
#include "kernels.cuh"
#include "planner.h"

namespace cbc {
namespace {

constexpr int TPB = 256;

// p moved by `bytes` (the per-instance stride of a batched workspace)
template <typename P>
__host__ __device__ __forceinline__ P* byte_shift(P* p, size_t bytes) {
  return reinterpret_cast<P*>(reinterpret_cast<uintptr_t>(p) + bytes);
}

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
    const double ib = rcp64(beta);
    tau = O::make((beta - ar) * ib, -ai * ib);
    // scale = 1 / (alpha - beta)
    double zr = ar - beta, zi = ai;
    const double iden = rcp64(zr * zr + zi * zi);
    scale = O::make(zr * iden, -zi * iden);
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

// ---- tridiagonalisation with the rows in shared memory -----------------------------
// Same reduction as tridiag_kernel, for m small enough that every CTA keeps its rows in
// shared memory.  Column j needs two exchanges through global memory: the Householder
// vector v_j (with tau_j) from the CTA that owns row j, and p = tau_j A v_j, one entry
// from the owner of each row.  Both travel as plain data: the receiving buffers are
// filled with the all-ones bit pattern before the launch, each entry is written once
// with a relaxed store, and readers poll every entry until it differs from that
// pattern, so no fence, counter or atomic sits on the dependency chain.  Each CTA also
// publishes its share of v^H p (its own rows); every CTA adds the P shares in one fixed
// order, so all CTAs apply the same rank-2 update.  Every wait is bounded.
template <typename T>
struct Tri2Args {
  const T* A;
  int m;
  double* d;
  double* e;
  T* tau;
  T* V;    // m x m; row j: [j] = tau_j, [j+1, m) = v_j; sentinel-filled before the launch
  T* Pg;   // m x m; row j: [j+1, m) = tau_j A v_j;     sentinel-filled before the launch
  T* Dg;   // (m-1) x P; [j][q] = CTA q's share of v_j^H p_j; sentinel-filled too
  int* status;
  int P;            // CTAs per matrix; CTA b handles matrix b / P of a batch
  int64_t a_bs;     // elements between consecutive matrices A
  size_t wb;        // bytes between the workspaces (d .. Pg) of consecutive matrices
};

constexpr long long kSentinel = -1LL;  // all bits set: a NaN that arithmetic never yields
constexpr long long kWaitCycles = 4000000000LL;

__device__ __forceinline__ double pub_value(double x) {
  return (__double_as_longlong(x) == kSentinel) ? __longlong_as_double(0x7ff8000000000000LL) : x;
}
__device__ __forceinline__ void st_pub(double* p, double v) {
  asm volatile("st.relaxed.gpu.global.f64 [%0], %1;" ::"l"(p), "d"(pub_value(v)) : "memory");
}
__device__ __forceinline__ void st_pub(zdbl* p, zdbl v) {
  asm volatile("st.relaxed.gpu.global.v2.f64 [%0], {%1, %2};" ::"l"(p), "d"(pub_value(v.re)),
               "d"(pub_value(v.im))
               : "memory");
}
__device__ __forceinline__ bool ld_pub(const double* p, double* v) {
  double x;
  asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(x) : "l"(p) : "memory");
  *v = x;
  return __double_as_longlong(x) != kSentinel;
}
__device__ __forceinline__ bool ld_pub(const zdbl* p, zdbl* v) {
  double x, y;
  asm volatile("ld.relaxed.gpu.global.v2.f64 {%0, %1}, [%2];" : "=d"(x), "=d"(y) : "l"(p) : "memory");
  *v = zdbl{x, y};
  return __double_as_longlong(x) != kSentinel && __double_as_longlong(y) != kSentinel;
}


// dst[lo, hi) <- src[lo, hi) as the entries get published (and their double-float forms
// into ddst when given).  False (for the whole CTA) when a wait ran out or another CTA
// has reported an error.
template <typename T>
__device__ bool gather_pub(const T* src, T* dst, int lo, int hi, int* status,
                           typename dfof<T>::type* ddst = nullptr) {
  bool ok = true;
  for (int c = lo + threadIdx.x; c < hi && ok; c += blockDim.x) {
    T v;
    if (!ld_pub(src + c, &v)) {
      const long long t0 = clock64();
      while (!ld_pub(src + c, &v)) {
        if (*((volatile int*)status) != 0) {
          ok = false;
          break;
        }
        if (clock64() - t0 > kWaitCycles) {
          set_status(status, CBC_ERR_TIMEOUT);
          ok = false;
          break;
        }
      }
    }
    dst[c] = v;
    if (ddst) ddst[c] = to_df(v);
  }
  return __syncthreads_and(ok) != 0;
}

// Two ranges in one polling pass (one barrier).
template <typename T>
__device__ bool gather_pub2(const T* s1, T* d1, int lo1, int hi1, const T* s2, T* d2, int lo2,
                            int hi2, int* status) {
  bool ok = true;
  const int n1 = hi1 - lo1, n = n1 + (hi2 - lo2);
  for (int q = threadIdx.x; q < n && ok; q += blockDim.x) {
    const T* src = (q < n1) ? s1 + lo1 + q : s2 + lo2 + (q - n1);
    T* dst = (q < n1) ? d1 + lo1 + q : d2 + lo2 + (q - n1);
    T v;
    if (!ld_pub(src, &v)) {
      const long long t0 = clock64();
      while (!ld_pub(src, &v)) {
        if (*((volatile int*)status) != 0) {
          ok = false;
          break;
        }
        if (clock64() - t0 > kWaitCycles) {
          set_status(status, CBC_ERR_TIMEOUT);
          ok = false;
          break;
        }
      }
    }
    *dst = v;
  }
  return __syncthreads_and(ok) != 0;
}

// (sum x, sum y) over the CTA; sh holds at least 66 doubles
__device__ __forceinline__ double2 block_sum2(double x, double y, double* sh) {
  x = warp_sum(x);
  y = warp_sum(y);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) {
    sh[w] = x;
    sh[32 + w] = y;
  }
  __syncthreads();
  if (w == 0) {
    double a = (lane < nw) ? sh[lane] : 0.0, b = (lane < nw) ? sh[32 + lane] : 0.0;
    a = warp_sum(a);
    b = warp_sum(b);
    if (lane == 0) {
      sh[64] = a;
      sh[65] = b;
    }
  }
  __syncthreads();
  return make_double2(sh[64], sh[65]);
}

// Householder vector of column j from the owner's updated row j (zlarfg convention:
// H = I - tau v v^H, H^H x = beta e_1 with beta real); written to vs (shared) and
// published to V.
template <typename T>
__device__ void householder_pub(const Tri2Args<T>& a, const T* row, int j, T* vs, double* sh) {
  using O = ops<T>;
  const int m = a.m;
  double xn2 = 0.0;
  for (int c = j + 2 + threadIdx.x; c < m; c += blockDim.x) xn2 += O::abs2(row[c]);
  xn2 = block_sum2(xn2, 0.0, sh).x;
  const T alpha = O::conj(row[j + 1]);
  const double ar = O::real(alpha), ai = O::imag(alpha);
  T tau, scale;
  double beta;
  const bool trivial = (xn2 == 0.0 && ai == 0.0);
  if (trivial) {
    tau = O::zero();
    beta = ar;
    scale = O::zero();
  } else {
    const double n2 = ar * ar + ai * ai + xn2;
    const double rn = rsqrt64(n2);  // 1 / ||x||
    const double nrm = n2 * rn;
    beta = (ar >= 0.0) ? -nrm : nrm;
    const double ib = (ar >= 0.0) ? -rn : rn;  // 1 / beta
    tau = O::make((beta - ar) * ib, -ai * ib);
    const double zr = ar - beta, zi = ai;
    const double iden = rcp64(zr * zr + zi * zi);
    scale = O::make(zr * iden, -zi * iden);
  }
  T* vg = a.V + (int64_t)j * m;
  for (int c = j + 1 + threadIdx.x; c < m; c += blockDim.x) {
    const T v = (c == j + 1) ? O::one() : (trivial ? O::zero() : O::conj(row[c]) * scale);
    vs[c] = v;
    st_pub(vg + c, v);
  }
  if (threadIdx.x == 0) {
    vs[j] = tau;
    st_pub(vg + j, tau);
    a.tau[j] = tau;
    a.e[j] = beta;
    a.d[j] = O::real(row[j]);
  }
  __syncthreads();
}

// householder_pub by one warp (lane = this thread's lane): no CTA barrier, so the other
// warps of the owner CTA keep updating their rows meanwhile.
template <typename T>
__device__ void householder_pub_warp(const Tri2Args<T>& a, const T* row, int j, T* vs,
                                     int lane) {
  using O = ops<T>;
  const int m = a.m;
  double xn2 = 0.0;
  for (int c = j + 2 + lane; c < m; c += 32) xn2 += O::abs2(row[c]);
  xn2 = warp_sum(xn2);
  const T alpha = O::conj(row[j + 1]);
  const double ar = O::real(alpha), ai = O::imag(alpha);
  T tau, scale;
  double beta;
  const bool trivial = (xn2 == 0.0 && ai == 0.0);
  if (trivial) {
    tau = O::zero();
    beta = ar;
    scale = O::zero();
  } else {
    const double n2 = ar * ar + ai * ai + xn2;
    const double rn = rsqrt64(n2);  // 1 / ||x||
    const double nrm = n2 * rn;
    beta = (ar >= 0.0) ? -nrm : nrm;
    const double ib = (ar >= 0.0) ? -rn : rn;  // 1 / beta
    tau = O::make((beta - ar) * ib, -ai * ib);
    const double zr = ar - beta, zi = ai;
    const double iden = rcp64(zr * zr + zi * zi);
    scale = O::make(zr * iden, -zi * iden);
  }
  T* vg = a.V + (int64_t)j * m;
  for (int c = j + 1 + lane; c < m; c += 32) {
    const T v = (c == j + 1) ? O::one() : (trivial ? O::zero() : O::conj(row[c]) * scale);
    st_pub(vg + c, v);
    vs[c] = v;
  }

  if (lane == 0) {
    vs[j] = tau;
    st_pub(vg + j, tau);
    a.tau[j] = tau;
    a.e[j] = beta;
    a.d[j] = O::real(row[j]);
  }
  __syncwarp();
}

// DF: rows as double-float pairs (mixed path); else FP64 throughout.
template <typename T, bool DF>
__global__ void __launch_bounds__(TPB) tridiag_smem_kernel(Tri2Args<T> a0) {
  using O = ops<T>;
  extern __shared__ unsigned char sm_raw[];
  __shared__ double sh[72];
  __shared__ T part[TPB / 32];
  const int P = a0.P, inst = blockIdx.x / P, cta = blockIdx.x % P;
  Tri2Args<T> a = a0;
  {
    const size_t off = (size_t)inst * a0.wb;
    a.A = a0.A + (int64_t)inst * a0.a_bs;
    a.d = byte_shift(a0.d, off);
    a.e = byte_shift(a0.e, off);
    a.tau = byte_shift(a0.tau, off);
    a.V = byte_shift(a0.V, off);
    a.Pg = byte_shift(a0.Pg, off);
    a.Dg = byte_shift(a0.Dg, off);
  }
  const int m = a.m;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int nr = (m - cta + P - 1) / P;  // own rows r = cta + P t
  T* rows = reinterpret_cast<T*>(sm_raw);
  T* vbuf = rows + (size_t)nr * m;  // v of two consecutive columns
  T* psm = vbuf + 2 * (size_t)m;    // p, then w
  T* pown = psm + m;                // p of the own rows (by local row index)
  T* dsm = pown + m;                // the P shares of v^H p
  // DF only: v and w as double-float, and the owner's row j+1 back in FP64
  using D = typename dfof<T>::type;
  D* rdf = reinterpret_cast<D*>(rows);
  D* vdfb = reinterpret_cast<D*>(dsm + P);  // two buffers, like vbuf
  D* wdf = vdfb + 2 * (size_t)m;
  T* hrow = reinterpret_cast<T*>(wdf + m);
  for (int t = 0; t < nr; ++t)
    for (int c = threadIdx.x; c < m; c += blockDim.x) {
      const T x = a.A[(int64_t)(cta + P * t) * m + c];
      if constexpr (DF)
        rdf[(size_t)t * m + c] = to_df(x);
      else
        rows[(size_t)t * m + c] = x;
    }
  __syncthreads();
  // own row t as FP64 (DF: converted into hrow from column `from` on)
  auto row64 = [&](int t, int from) -> const T* {
    if constexpr (DF) {
      for (int c = from + threadIdx.x; c < m; c += blockDim.x) hrow[c] = from_df(rdf[(size_t)t * m + c]);
      __syncthreads();
      return hrow;
    } else {
      return rows + (size_t)t * m;
    }
  };
  if (m == 1) {
    if (cta == 0) {
      const T* r0 = row64(0, 0);
      if (threadIdx.x == 0) a.d[0] = O::real(r0[0]);
    }
    return;
  }
  if (cta == 0) {
    householder_pub(a, row64(0, 0), 0, vbuf, sh);
    if constexpr (DF) {
      for (int c = 1 + threadIdx.x; c < m; c += blockDim.x) vdfb[c] = to_df(vbuf[c]);
      __syncthreads();
    }
  }
  for (int j = 0; j < m - 1; ++j) {
    T* vsm = vbuf + (size_t)(j & 1) * m;
    D* vdf = vdfb + (size_t)(j & 1) * m;
    // v_j and tau_j (the owner of row j computed them into vsm itself)
    // (the double-float copy of v goes with the gather; the owner converts its own v)
    if (j % P != cta) {
      if (!gather_pub(a.V + (int64_t)j * m, vsm, j, m, a.status, DF ? vdf : nullptr)) return;
    } else if (DF && j > 0) {
      for (int c = j + 1 + threadIdx.x; c < m; c += blockDim.x) vdf[c] = to_df(vsm[c]);
      __syncthreads();
    }
    const T tau = vsm[j];
    // phase B: p_r = tau sum_{c>j} A[r][c] v_c for own rows r > j
    const int t0 = (j + 1 - cta + P - 1) / P;  // first own row beyond j
    const int live = nr - t0;
    T* pg = a.Pg + (int64_t)j * m;
    if (live > 0) {
      int S = 1;
      while (S * 2 * live <= nw) S *= 2;
      if (S == 1) {
        // rows ta and ta + nw per warp pass; a reduce-scatter butterfly leaves row ta's
        // sum in lanes 0-15 and row tb's in lanes 16-31 (5 add levels for both rows)
        for (int item = warp; item < live; item += 2 * nw) {
          const int ta = t0 + item;
          const bool two = item + nw < live;
          const int tb = two ? ta + nw : ta;
          T xa = O::zero(), xb = O::zero();
          if constexpr (DF) {
            const D* ra = rdf + (size_t)ta * m;
            const D* rb = rdf + (size_t)tb * m;
            D ya = to_df(O::zero()), yb = ya;
            for (int c = j + 1 + lane; c < m; c += 32) {
              const D vc = vdf[c];
              ya = dff(ra[c], vc, ya);
              if (two) yb = dff(rb[c], vc, yb);
            }
            xa = from_df(ya);
            xb = from_df(yb);
          } else {
            const T* ra = rows + (size_t)ta * m;
            const T* rb = rows + (size_t)tb * m;
            for (int c = j + 1 + lane; c < m; c += 32) {
              const T vc = vsm[c];
              xa = O::fma(ra[c], vc, xa);
              if (two) xb = O::fma(rb[c], vc, xb);
            }
          }
          if (two) {
            T keep = (lane < 16) ? xa : xb;
            keep = keep + shfl_xor((lane < 16) ? xb : xa, 16);
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) keep = keep + shfl_xor(keep, o);
            if ((lane & 15) == 0) {
              const int t = (lane == 0) ? ta : tb;
              const T pr = tau * keep;
              pown[t] = pr;
              st_pub(pg + cta + P * t, pr);
            }
          } else {
            xa = warp_sum(xa);
            if (lane == 0) {
              const T pr = tau * xa;
              pown[ta] = pr;
              st_pub(pg + cta + P * ta, pr);
            }
          }
        }
      } else {
        for (int item = warp; item < live * S; item += nw) {
          const int t = t0 + item / S, sg = item % S;
          T acc = O::zero();
          if constexpr (DF) {
            const D* row = rdf + (size_t)t * m;
            D y = to_df(O::zero());
            for (int c = j + 1 + sg * 32 + lane; c < m; c += S * 32) y = dff(row[c], vdf[c], y);
            acc = from_df(y);
          } else {
            const T* row = rows + (size_t)t * m;
            for (int c = j + 1 + sg * 32 + lane; c < m; c += S * 32) acc = O::fma(row[c], vsm[c], acc);
          }
          acc = warp_sum(acc);
          if (lane == 0) part[item] = acc;
        }
        __syncthreads();
        if (threadIdx.x < live) {
          T sp = part[threadIdx.x * S];
          for (int q = 1; q < S; ++q) sp = sp + part[threadIdx.x * S + q];
          const T pr = tau * sp;
          pown[t0 + threadIdx.x] = pr;
          st_pub(pg + cta + P * (t0 + threadIdx.x), pr);
        }
      }
    }
    __syncthreads();
    // this CTA's share of v^H p, published next to p
    if (warp == 0) {
      T dv = O::zero();
      for (int t = t0 + lane; t < nr; t += 32) dv = O::fma(O::conj(vsm[cta + P * t]), pown[t], dv);
      dv = warp_sum(dv);
      if (lane == 0) st_pub(a.Dg + (int64_t)j * P + cta, dv);
    }
    // all of p and all shares; v^H p summed in one fixed order (the same in every CTA);
    // then w = p - (conj(tau)/2)(v^H p) v in place
    if (!gather_pub2(pg, psm, j + 1, m, a.Dg + (int64_t)j * P, dsm, 0, P, a.status)) return;
    T dot = O::zero();
    for (int q = lane; q < P; q += 32) dot = dot + dsm[q];
    dot = warp_sum(dot);
    const T coef = O::scale(-0.5, O::conj(tau) * dot);
    for (int c = j + 1 + threadIdx.x; c < m; c += blockDim.x) {
      psm[c] = O::fma(coef, vsm[c], psm[c]);
      if constexpr (DF) wdf[c] = to_df(psm[c]);
    }
    __syncthreads();
    // phase C: own rows r > j: A[r][c] -= v_r conj(w_c) + w_r conj(v_c), c > j
    auto update_row = [&](int t, int c0, int cstep) {
      const int r = cta + P * t;
      const T nvr = O::scale(-1.0, vsm[r]), nwr = O::scale(-1.0, psm[r]);
      if constexpr (DF) {
        D* row = rdf + (size_t)t * m;
        const D dvr = to_df(nvr), dwr = to_df(nwr);
        for (int c = j + 1 + c0; c < m; c += cstep)
          row[c] = dff(dwr, dfconj(vdf[c]), dff(dvr, dfconj(wdf[c]), row[c]));
      } else {
        T* row = rows + (size_t)t * m;
        for (int c = j + 1 + c0; c < m; c += cstep)
          row[c] = O::fma(nwr, O::conj(vsm[c]), O::fma(nvr, O::conj(psm[c]), row[c]));
      }
    };
    if (j + 1 < m - 1 && (j + 1) % P == cta) {
      // the next column's owner: warp 0 updates that row and publishes v_{j+1} while
      // the other warps update the remaining rows
      if (warp == 0) {
        update_row(t0, lane, 32);
        __syncwarp();
        const T* hr;
        if constexpr (DF) {
          for (int c = j + 1 + lane; c < m; c += 32) hrow[c] = from_df(rdf[(size_t)t0 * m + c]);
          __syncwarp();
          hr = hrow;
        } else {
          hr = rows + (size_t)t0 * m;
        }
        householder_pub_warp(a, hr, j + 1, vbuf + (size_t)((j + 1) & 1) * m, lane);
      } else {
        for (int t = t0 + 1 + (warp - 1); t < nr; t += nw - 1) update_row(t, lane, 32);
      }
    } else {
      for (int t = t0 + warp; t < nr; t += nw) update_row(t, lane, 32);
    }
    if (j + 1 == m - 1 && (m - 1) % P == cta) {
      __syncthreads();
      const T* rl = row64((m - 1 - cta) / P, m - 1);
      if (threadIdx.x == 0) a.d[m - 1] = O::real(rl[m - 1]);
    }
    __syncthreads();
  }
}

// ---- eigenvalues of T: single-precision multisection, one warp per eigenvalue --------
// The values only seed the shifts of the FP64 inverse iteration below, whose Rayleigh
// quotients are the eigenvalues used for the rank rule.
__device__ __forceinline__ int sturm32(const float* dd, const float* e2, int m, float x,
                                       float pivmin) {
  int cnt = 0;
  float q = dd[0] - x;
  if (q < 0.f) cnt++;
  for (int i = 1; i < m; ++i) {
    if (fabsf(q) < pivmin) q = -pivmin;
    q = (dd[i] - x) - __fdividef(e2[i - 1], q);
    if (q < 0.f) cnt++;
  }
  return cnt;
}

__global__ void bisect32_kernel(const double* d, const double* e, int m, float* lam32,
                                size_t wb) {
  extern __shared__ float shf[];
  d = byte_shift(d, blockIdx.y * wb);  // matrix blockIdx.y of a batch
  e = byte_shift(e, blockIdx.y * wb);
  lam32 = byte_shift(lam32, blockIdx.y * wb);
  float* dd = shf;
  float* e2 = shf + m;
  __shared__ float s_lo, s_hi, s_piv;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    dd[i] = (float)d[i];
    e2[i] = (i < m - 1) ? (float)(e[i] * e[i]) : 0.f;
  }
  if (threadIdx.x == 0) {
    double lo = DBL_MAX, hi = -DBL_MAX, emax = 0.0;
    for (int i = 0; i < m; ++i) {
      double r = 0.0;
      if (i > 0) r += fabs(e[i - 1]);
      if (i < m - 1) r += fabs(e[i]);
      lo = fmin(lo, d[i] - r);
      hi = fmax(hi, d[i] + r);
      if (i < m - 1) emax = fmax(emax, e[i] * e[i]);
    }
    double span = fmax(fabs(lo), fabs(hi));
    s_lo = (float)(lo - 1e-6 * span) - FLT_MIN;
    s_hi = (float)(hi + 1e-6 * span) + FLT_MIN;
    s_piv = FLT_MIN * (float)fmax(1.0, emax);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int jj = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);  // descending index
  if (jj >= m) return;
  const int target = m - 1 - jj;
  float lo = s_lo, hi = s_hi;
  for (int round = 0; round < 12; ++round) {
    const float x = lo + (hi - lo) * (float)(lane + 1) * (1.f / 33.f);
    const int cnt = sturm32(dd, e2, m, x, s_piv);
    const unsigned bits = __ballot_sync(0xffffffffu, cnt <= target);
    const int nle = __popc(bits);
    const float xl = __shfl_sync(0xffffffffu, x, max(nle - 1, 0));
    const float xh = __shfl_sync(0xffffffffu, x, min(nle, 31));
    if (nle > 0) lo = xl;
    if (nle < 32) hi = xh;
    if (hi - lo <= 2e-7f * fmaxf(fabsf(lo), fabsf(hi)) + s_piv) break;
  }
  if (lane == 0) lam32[jj] = 0.5f * (lo + hi);
}

// ---- eigenvectors of T by FP64 inverse iteration ----------------------------------
// The LU of T - sigma I with partial pivoting (the layout of LAPACK's tridiagonal
// factorisation) lives in shared memory, [i][member], with the pivots stored as
// reciprocals so the solves are division free.  A candidate whose single-precision
// eigenvalue is separated from its neighbours by more than 1e-4 of the spectral radius
// gets a thread of its own (invit_kernel); a run of closer candidates is a cluster that
// one warp iterates as a block, orthonormalising after every solve
// (invit_cluster_kernel).  The eigenvalue is the FP64 Rayleigh quotient of the vector.
__device__ __forceinline__ uint32_t hash32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352dU;
  x ^= x >> 15;
  x *= 0x846ca68bU;
  x ^= x >> 16;
  return x;
}

struct InvArgs {
  const double* d;
  const double* e;
  const float* lam32;  // descending
  int m;
  int kmax;            // candidates j < kmax
  double* X;           // m x kmax (row i, column j)
  double* rq;          // [kmax] Rayleigh quotients
  size_t wb;           // workspace bytes between the matrices of a batch (blockIdx.y)
};

// Shared-memory arrays of the members handled by one CTA: element i of member t at
// [i * tpb + t] (consecutive members' rows side by side).
struct InvSmem {
  double *dl, *di, *du, *du2, *b;  // multipliers, reciprocal pivots, U's two superdiagonals, vector
  unsigned char* piv;
  int tpb;
  __device__ InvSmem(double* base, int m, int tpb_) : tpb(tpb_) {
    dl = base;
    di = dl + (size_t)m * tpb;
    du = di + (size_t)m * tpb;
    du2 = du + (size_t)m * tpb;
    b = du2 + (size_t)m * tpb;
    piv = reinterpret_cast<unsigned char*>(b + (size_t)m * tpb);
  }
};
#define SH(arr, i) w.arr[(size_t)(i) * w.tpb + t]

// LU with partial pivoting of T - sigma I for member t (pivots kept as reciprocals, so the
// solves are division free)
__device__ void invit_factor(const double* d, const double* e, int m, double sigma, double tiny,
                             const InvSmem& w, int t) {
  double dcur = d[0] - sigma;
  double ucur = (m > 1) ? e[0] : 0.0;  // superdiagonal entry of the current row
  for (int i = 0; i < m - 1; ++i) {
    const double li = e[i];
    const double dn = d[i + 1] - sigma;
    const double un = (i + 1 < m - 1) ? e[i + 1] : 0.0;
    if (fabs(dcur) >= fabs(li)) {
      double dv = (fabs(dcur) < tiny) ? ((dcur < 0.0) ? -tiny : tiny) : dcur;
      double r = rcp64(dv);
      double f = li * r;
      SH(piv, i) = 0;
      SH(dl, i) = f;
      SH(di, i) = r;
      SH(du, i) = ucur;
      SH(du2, i) = 0.0;
      dcur = dn - f * ucur;
      ucur = un;
    } else {
      double r = rcp64(li);
      double f = dcur * r;
      SH(piv, i) = 1;
      SH(dl, i) = f;
      SH(di, i) = r;
      SH(du, i) = dn;
      SH(du2, i) = un;
      dcur = ucur - f * dn;
      ucur = -f * un;
    }
  }
  double dv = (fabs(dcur) < tiny) ? ((dcur < 0.0) ? -tiny : tiny) : dcur;
  SH(di, m - 1) = rcp64(dv);
}

// b <- (T - sigma I)^{-1} b for member t with its factors: L y = P b, then U x = y
__device__ void invit_solve(int m, const InvSmem& w, int t) {
  double carry = SH(b, 0);
  for (int i = 0; i < m - 1; ++i) {
    double nxt = SH(b, i + 1);
    if (SH(piv, i) == 0) {
      SH(b, i) = carry;
      carry = nxt - SH(dl, i) * carry;
    } else {
      SH(b, i) = nxt;
      carry = carry - SH(dl, i) * nxt;
    }
  }
  SH(b, m - 1) = carry;
  double x1 = 0.0, x2 = 0.0;
  for (int i = m - 1; i >= 0; --i) {
    double sv = SH(b, i) - SH(du, i) * x1 - SH(du2, i) * x2;
    if (i == m - 1) sv = SH(b, i);
    double xi = sv * SH(di, i);
    SH(b, i) = xi;
    x2 = x1;
    x1 = xi;
  }
}

// random start vector of candidate j (fixed hash, so every run is reproducible)
__device__ void invit_start(int m, int j, const InvSmem& w, int t) {
  for (int i = 0; i < m; ++i) {
    uint32_t h = hash32((uint32_t)(i * 7919 + j * 104729 + 17));
    SH(b, i) = ((double)(h & 0xffffff) / 16777216.0) - 0.5;
  }
}

// sum_i x_i y_i over strided arrays with four independent partial sums (the FP64
// latency chain is the cost of a lone thread's dot product)
__device__ __forceinline__ double dot4(const double* x, size_t sx, const double* y, size_t sy,
                                       int m) {
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int i = 0;
  for (; i + 3 < m; i += 4) {
    a0 = fma(x[(size_t)i * sx], y[(size_t)i * sy], a0);
    a1 = fma(x[(size_t)(i + 1) * sx], y[(size_t)(i + 1) * sy], a1);
    a2 = fma(x[(size_t)(i + 2) * sx], y[(size_t)(i + 2) * sy], a2);
    a3 = fma(x[(size_t)(i + 3) * sx], y[(size_t)(i + 3) * sy], a3);
  }
  for (; i < m; ++i) a0 = fma(x[(size_t)i * sx], y[(size_t)i * sy], a0);
  return (a0 + a1) + (a2 + a3);
}

// Rayleigh quotient of member t's (unit) vector, written with the vector to column j of X
__device__ void invit_finish(const InvArgs& a, int j, const InvSmem& w, int t) {
  const int m = a.m, K = a.kmax;
  double rqv = 0.0;
  for (int i = 0; i < m; ++i) {
    const double xi = SH(b, i);
    double tx = a.d[i] * xi;
    if (i > 0) tx += a.e[i - 1] * SH(b, i - 1);
    if (i < m - 1) tx += a.e[i] * SH(b, i + 1);
    rqv += xi * tx;
    a.X[(size_t)i * K + j] = xi;
  }
  a.rq[j] = rqv;
}

__device__ __forceinline__ void invit_shift(InvArgs& a) {
  const size_t off = blockIdx.y * a.wb;
  a.d = byte_shift(a.d, off);
  a.e = byte_shift(a.e, off);
  a.lam32 = byte_shift(a.lam32, off);
  a.X = byte_shift(a.X, off);
  a.rq = byte_shift(a.rq, off);
}

// Each solve shrinks the components along eigenvectors at distance delta by about
// |lambda - sigma| / delta with |lambda - sigma| ~ 1e-7 span (single-precision shifts);
// four solves reach FP64 accuracy for delta >= 1e-4 span.  Candidates closer than that
// to a neighbour form a cluster (invit_cluster_kernel).
__device__ __forceinline__ double invit_span(const InvArgs& a) {
  return fmax(fabs((double)a.lam32[0]), fabs((double)a.lam32[a.m - 1])) + DBL_MIN;
}
__device__ __forceinline__ bool close_pair(const InvArgs& a, int j, double ortol) {
  return (double)a.lam32[j] - (double)a.lam32[j + 1] <= ortol;  // descending
}

// candidates that are not part of a cluster: one thread each
__global__ void invit_kernel(InvArgs a) {
  extern __shared__ double shd[];
  invit_shift(a);
  const int m = a.m, K = a.kmax, t = threadIdx.x;
  const InvSmem w(shd, m, blockDim.x);
  const int jj = blockIdx.x * blockDim.x + t;
  if (jj >= K) return;
  const double span = invit_span(a);
  const double ortol = 1e-4 * span;
  if ((jj > 0 && close_pair(a, jj - 1, ortol)) || (jj + 1 < K && close_pair(a, jj, ortol))) return;
  const double tiny = 2.220446049250313e-16 * span;
  invit_factor(a.d, a.e, m, (double)a.lam32[jj], tiny, w, t);
  invit_start(m, jj, w, t);
  for (int it = 0; it < 4; ++it) {
    invit_solve(m, w, t);
    const double nrm = dot4(&SH(b, 0), w.tpb, &SH(b, 0), w.tpb, m);
    const double inv = (nrm > 0.0) ? rcp64(sqrt(nrm)) : 0.0;
    for (int i = 0; i < m; ++i) SH(b, i) *= inv;
  }
  invit_finish(a, jj, w, t);
}

// The clusters of candidates (runs of neighbours closer than 1e-4 of the spectral radius),
// each by one warp: `per` members at a time, one per lane, iterated as a block (block inverse
// iteration): every lane solves with its own shift (shifts at least 1e-10 span apart),
// then the block is orthonormalised (modified Gram-Schmidt, lanes in parallel) against
// the cluster's finished columns and within itself, four times.  The vectors then span
// the invariant subspace of the cluster's eigenvalues (any basis of it is a valid set of
// eigenvectors when they are not resolved individually).
// one cluster [jj, cend) by the warp, `per` members per pass
__device__ void invit_cluster(const InvArgs& a, const InvSmem& w, int jj, int cend, int per,
                              double span, double tiny) {
  const int m = a.m, K = a.kmax, lane = threadIdx.x;
  for (int j0 = jj; j0 < cend; j0 += per) {
    const int nact = min(per, cend - j0);
    const bool act = lane < nact;
    const int t = act ? lane : 0;
    const int j = j0 + lane;
    if (act) {
      double sigma = (double)a.lam32[jj];
      for (int q = jj + 1; q <= j; ++q) sigma = fmin((double)a.lam32[q], sigma - 1e-10 * span);
      invit_factor(a.d, a.e, m, sigma, tiny, w, t);
      invit_start(m, j, w, t);
    }
    __syncwarp();
    for (int it = 0; it < 4; ++it) {
      if (act) {
        invit_solve(m, w, t);
        // against the finished columns of the cluster
        for (int q = jj; q < j0; ++q) {
          const double dv = dot4(a.X + q, (size_t)K, &SH(b, 0), w.tpb, m);
          for (int i = 0; i < m; ++i) SH(b, i) -= dv * a.X[(size_t)i * K + q];
        }
      }
      __syncwarp();
      // within the block, in member order
      for (int q = 0; q < nact; ++q) {
        if (lane == q) {
          const double nrm = dot4(&SH(b, 0), w.tpb, &SH(b, 0), w.tpb, m);
          const double inv = (nrm > 0.0) ? rcp64(sqrt(nrm)) : 0.0;
          for (int i = 0; i < m; ++i) SH(b, i) *= inv;
        }
        __syncwarp();
        if (act && lane > q) {
          const double* bq = w.b + q;
          const double dv = dot4(bq, w.tpb, &SH(b, 0), w.tpb, m);
          for (int i = 0; i < m; ++i) SH(b, i) -= dv * bq[(size_t)i * w.tpb];
        }
        __syncwarp();
      }
    }
    if (act) invit_finish(a, j, w, t);
    __syncwarp();
  }
}

__global__ void invit_cluster_kernel(InvArgs a, int per) {
  extern __shared__ double shd[];
  invit_shift(a);
  const int K = a.kmax;
  const InvSmem w(shd, a.m, per);
  const double span = invit_span(a);
  const double ortol = 1e-4 * span;
  const double tiny = 2.220446049250313e-16 * span;
  // CTA c takes clusters c, c + gridDim.x, ... in order (a cluster: a run of two or more
  // candidates whose neighbours are close); every lane scans the same candidates
  int cidx = -1;
  for (int jj = 0; jj + 1 < K;) {
    if (!close_pair(a, jj, ortol)) {
      ++jj;
      continue;
    }
    int cend = jj + 2;
    while (cend < K && close_pair(a, cend - 1, ortol)) ++cend;
    ++cidx;
    if (cidx % (int)gridDim.x == (int)blockIdx.x) invit_cluster(a, w, jj, cend, per, span, tiny);
    jj = cend;
  }
}
#undef SH

// rank rule on the Rayleigh quotients of the candidates; the discarded weight is the
// exact trace of T minus the kept eigenvalues.  Writes k and the full eigenvalue list.
// floor_rel < 0 keeps all kmax candidates (the caller decides the rank from weights it
// measures on the factor itself).
__global__ void rank_kernel(const double* d, const double* rq, const float* lam32, int m,
                            int kmax, long long max_bond, double tol, double floor_rel,
                            int* k_dev, double* lam, size_t wb) {
  __shared__ double s_tr;
  // matrix blockIdx.x of a batch
  d = byte_shift(d, blockIdx.x * wb);
  rq = byte_shift(rq, blockIdx.x * wb);
  lam32 = byte_shift(lam32, blockIdx.x * wb);
  k_dev += blockIdx.x;
  lam += (size_t)blockIdx.x * m;
  if (threadIdx.x == 0) {
    double tr = 0.0;
    for (int i = 0; i < m; ++i) tr += d[i];
    s_tr = tr;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < m; j += blockDim.x) lam[j] = (j < kmax) ? rq[j] : (double)lam32[j];
  if (threadIdx.x != 0) return;
  const double l0 = rq[0];
  int k = 1;
  if (floor_rel < 0.0) {
    k = kmax;  // every candidate: the caller applies the rank rule itself
  } else if (l0 > 0.0) {
    k = 0;
    while (k < kmax && rq[k] > floor_rel * l0) ++k;
    if (tol > 0.0) {
      const double total = fmax(s_tr, 0.0);
      double tail = total;
      int kt = 0;
      while (kt < kmax && tail > tol * tol * total) {
        tail -= fmax(rq[kt], 0.0);
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

// ---- back transformation: U[:, jj] = H_0 ... H_{m-2} X[:, jj] ------------------------
// One CTA of four warps per kept eigenvector (one warp per SM sub-partition, since a
// warp alone reaches only its own partition's FP64 unit).  Each reflector application
// is a dot product over the rows (per-warp partial sums combined through shared
// memory) and an axpy; the rows are split across the 128 threads.
template <typename T>
__global__ void __launch_bounds__(128) backtransform_kernel(const T* V, const T* tau,
                                                            const double* X, int m, int kmax,
                                                            const int* k_dev, T* U, size_t wb) {
  using O = ops<T>;
  extern __shared__ unsigned char smem_raw[];
  T* u = reinterpret_cast<T*>(smem_raw);
  __shared__ T part[2][4];
  // matrix blockIdx.y of a batch
  V = byte_shift(V, blockIdx.y * wb);
  tau = byte_shift(tau, blockIdx.y * wb);
  X = byte_shift(X, blockIdx.y * wb);
  k_dev += blockIdx.y;
  U += (size_t)blockIdx.y * m * kmax;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int jj = blockIdx.x;
  const int k = *k_dev;
  if (jj >= k) return;
  for (int i = tid; i < m; i += 128) u[i] = O::make(X[(int64_t)i * kmax + jj], 0.0);
  __syncthreads();
  int par = 0;
  for (int j = m - 2; j >= 0; --j) {
    const T* vj = V + (int64_t)j * m;
    const T t = tau[j];
    T sacc = O::zero();
    // each thread owns rows r = tid (mod 128) for the whole loop, so u needs no barrier
    for (int r = tid; r < m; r += 128)
      if (r > j) sacc = O::fma(O::conj(vj[r]), u[r], sacc);
    if constexpr (O::cplx) {
      sacc = zdbl{warp_sum(O::real(sacc)), warp_sum(O::imag(sacc))};
    } else {
      sacc = warp_sum(sacc);
    }
    if (lane == 0) part[par][warp] = sacc;
    __syncthreads();
    const T tot = (part[par][0] + part[par][1]) + (part[par][2] + part[par][3]);
    const T ts = t * tot;
    for (int r = tid; r < m; r += 128)
      if (r > j) u[r] = u[r] - vj[r] * ts;
    par ^= 1;  // the next partial sums go to the other buffer: one barrier per reflector
  }
  __syncthreads();
  for (int i = tid; i < m; i += 128) U[(int64_t)i * kmax + jj] = u[i];
}

// Same back transformation with the lanes on the eigenvectors: a CTA takes 32 vectors
// (one per lane, held in shared memory as u[row][lane]) and 8 warps split the rows.
// Per reflector every lane sums conj(v_r) u_r over its warp's rows, the 8 partial sums
// meet in shared memory (one barrier), and every lane updates its rows.  No shuffle
// reductions and no half-empty warps: about a quarter of the FP64 instructions of the
// one-vector-per-CTA form.  u needs m * 32 elements of shared memory.
constexpr int BT_WARPS = 8;

// DF (mixed path, batches): u and the staged v as double-float pairs, the two O(m) loops
// per reflector in FP32 (the partial sums and tau * sum stay FP64).
template <typename T, bool DF>
__global__ void __launch_bounds__(32 * BT_WARPS) backtransform32_kernel(
    const T* V, const T* tau, const double* X, int m, int kmax, const int* k_dev, T* U,
    size_t wb) {
  using O = ops<T>;
  using D = typename dfof<T>::type;
  using E = typename std::conditional<DF, D, T>::type;  // element type of u and v in smem
  extern __shared__ unsigned char smem_raw[];
  E* u = reinterpret_cast<E*>(smem_raw);  // [m][32]
  E* vs = u + (size_t)m * 32;             // [3][m]: v_j in slot j % 3 (staged one ahead)
  // per-warp partial dots (double-float in the DF variant: the cross-warp sum and the
  // tau scaling then stay on the FP32 pipes, which every active warp repeats per reflector)
  __shared__ E part[2][BT_WARPS][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // matrix blockIdx.y of a batch
  V = byte_shift(V, blockIdx.y * wb);
  tau = byte_shift(tau, blockIdx.y * wb);
  X = byte_shift(X, blockIdx.y * wb);
  k_dev += blockIdx.y;
  U += (size_t)blockIdx.y * m * kmax;
  const int k = *k_dev;
  const int c0 = blockIdx.x * 32;
  if (c0 >= k) return;
  const int col = c0 + lane;
  const bool live = col < k;
  const int rb = (m + BT_WARPS - 1) / BT_WARPS;
  const int r0 = warp * rb, r1 = min(m, r0 + rb);
  auto to_e = [](const T& x) -> E {
    if constexpr (DF)
      return to_df(x);
    else
      return x;
  };
  for (int r = r0; r < r1; ++r)
    u[(size_t)r * 32 + lane] = to_e(O::make(live ? X[(int64_t)r * kmax + col] : 0.0, 0.0));
  if (m >= 2) {  // v_{m-2}: rows > m - 2
    const T* vg = V + (int64_t)(m - 2) * m;
    E* v0 = vs + (size_t)((m - 2) % 3) * m;
    for (int q = m - 1 + (int)threadIdx.x; q < m; q += blockDim.x) v0[q] = to_e(vg[q]);
  }
  __syncthreads();
  int par = 0;
  for (int j = m - 2; j >= 0; --j) {
    const E* v = vs + (size_t)(j % 3) * m;
    // partial dot over this warp's rows r > j, four independent accumulators
    const int rs = max(r0, j + 1);
    E psum;
    if constexpr (DF) {
      const D z = to_df(O::zero());
      D a0 = z, a1 = z, a2 = z, a3 = z;
      int r = rs;
      for (; r + 3 < r1; r += 4) {
        a0 = dff(dfconj(v[r]), u[(size_t)r * 32 + lane], a0);
        a1 = dff(dfconj(v[r + 1]), u[(size_t)(r + 1) * 32 + lane], a1);
        a2 = dff(dfconj(v[r + 2]), u[(size_t)(r + 2) * 32 + lane], a2);
        a3 = dff(dfconj(v[r + 3]), u[(size_t)(r + 3) * 32 + lane], a3);
      }
      for (; r < r1; ++r) a0 = dff(dfconj(v[r]), u[(size_t)r * 32 + lane], a0);
      psum = df_add(df_add(a0, a1), df_add(a2, a3));
    } else {
      T a0 = O::zero(), a1 = O::zero(), a2 = O::zero(), a3 = O::zero();
      int r = rs;
      for (; r + 3 < r1; r += 4) {
        a0 = O::fma(O::conj(v[r]), u[(size_t)r * 32 + lane], a0);
        a1 = O::fma(O::conj(v[r + 1]), u[(size_t)(r + 1) * 32 + lane], a1);
        a2 = O::fma(O::conj(v[r + 2]), u[(size_t)(r + 2) * 32 + lane], a2);
        a3 = O::fma(O::conj(v[r + 3]), u[(size_t)(r + 3) * 32 + lane], a3);
      }
      for (; r < r1; ++r) a0 = O::fma(O::conj(v[r]), u[(size_t)r * 32 + lane], a0);
      psum = (a0 + a1) + (a2 + a3);
    }
    part[par][warp][lane] = psum;
    // stage the next reflector's vector (rows > j - 1).  Its slot last held v_{j+2},
    // whose readers all finished before the barrier this warp passed last.
    if (j >= 1) {
      const T* vg = V + (int64_t)(j - 1) * m;
      E* vn = vs + (size_t)((j - 1) % 3) * m;
      for (int q = j + threadIdx.x; q < m; q += blockDim.x) vn[q] = to_e(vg[q]);
    }
    __syncthreads();
    if (rs < r1) {
      if constexpr (DF) {
        D tot = part[par][0][lane];
#pragma unroll
        for (int w = 1; w < BT_WARPS; ++w) tot = df_add(tot, part[par][w][lane]);
        const D ncf = df_neg(dff(to_df(tau[j]), tot, to_df(O::zero())));
        for (int q = rs; q < r1; ++q) u[(size_t)q * 32 + lane] = dff(v[q], ncf, u[(size_t)q * 32 + lane]);
      } else {
        T tot = part[par][0][lane];
#pragma unroll
        for (int w = 1; w < BT_WARPS; ++w) tot = tot + part[par][w][lane];
        const T cf = tau[j] * tot;
        for (int q = rs; q < r1; ++q) u[(size_t)q * 32 + lane] = u[(size_t)q * 32 + lane] - v[q] * cf;
      }
    }
    par ^= 1;
  }
  __syncthreads();
  if (live)
    for (int r = r0; r < r1; ++r) {
      if constexpr (DF)
        U[(int64_t)r * kmax + col] = from_df(u[(size_t)r * 32 + lane]);
      else
        U[(int64_t)r * kmax + col] = u[(size_t)r * 32 + lane];
    }
}

// Initial contents of a batch of eigensolver workspaces in one launch: up to 6 segments
// of 64-bit words per instance (instance blockIdx.y, workspaces wb bytes apart).
struct WsInit {
  unsigned long long* seg[6];
  int64_t words[6];
  unsigned long long val[6];
  int nseg;
  size_t wb;
};

__global__ void ws_init_kernel(WsInit a) {
  const size_t off = blockIdx.y * a.wb;
  for (int g = 0; g < a.nseg; ++g) {
    unsigned long long* p = byte_shift(a.seg[g], off);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.words[g];
         i += (int64_t)gridDim.x * blockDim.x)
      p[i] = a.val[g];
  }
}

}  // namespace

// workspace layout (all 256-byte aligned)
static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

size_t eig_workspace_bytes(int m, int kmax, bool cplx) {
  size_t ts = cplx ? sizeof(zdbl) : sizeof(double);
  size_t b = 0;
  b += align256(sizeof(double) * m);                 // d
  b += align256(sizeof(double) * m);                 // e
  b += align256(sizeof(float) * m);                  // lam32
  b += align256(sizeof(double) * m);                 // rq
  b += align256(ts * m);                             // tau
  b += align256(ts * (size_t)m * m);                 // V
  b += align256(ts * 2 * m);                         // vbuf
  b += align256(ts * 2 * m);                         // p (two buffers)
  b += align256(sizeof(double) * 4);                 // dot
  b += align256(sizeof(GridBarrier));                // barrier
  b += align256(sizeof(double) * (size_t)m * kmax);  // X
  b += align256(ts * (size_t)m * m);                 // p of every column (exchange)
  b += align256(ts * (size_t)m * m);                 // shares of v^H p (exchange)
  return b;
}

template <typename T>
cudaError_t heev_top(T* A, int m, int kmax, int64_t max_bond, double tol, double floor_rel,
                     double* lam, T* U, int* k_dev, void* work, int* status, int num_sms,
                     cudaStream_t s, int nb, bool prefer_cluster, bool df) {
  char* w = static_cast<char*>(work);
  auto take = [&](size_t bytes) {
    char* p = w;
    w += align256(bytes);
    return p;
  };
  const size_t ts = sizeof(T);
  const size_t wb = eig_workspace_bytes(m, kmax, ops<T>::cplx);  // per matrix
  double* d = (double*)take(sizeof(double) * m);
  double* e = (double*)take(sizeof(double) * m);
  float* lam32 = (float*)take(sizeof(float) * m);
  double* rq = (double*)take(sizeof(double) * m);
  T* tau = (T*)take(ts * m);
  T* V = (T*)take(ts * (size_t)m * m);
  T* vbuf = (T*)take(ts * 2 * m);
  T* p = (T*)take(ts * 2 * m);
  double* dot = (double*)take(sizeof(double) * 4);
  GridBarrier* bar = (GridBarrier*)take(sizeof(GridBarrier));
  double* X = (double*)take(sizeof(double) * (size_t)m * kmax);
  T* Pg = (T*)take(ts * (size_t)m * m);
  T* Dg = (T*)take(ts * (size_t)m * m);

  cudaError_t err = cudaSuccess;
  // algorithmic FP64 flops: Householder tridiagonalisation (16/3) m^3 complex,
  // (4/3) m^3 real; back transformation of kmax vectors 8 m^2 kmax complex, 2 m^2 kmax real
  const double cm = ops<T>::cplx ? 4.0 : 1.0;
  const double fl_tri = cm * (4.0 / 3.0) * m * (double)m * m * nb;
  const double fl_rest = cm * 2.0 * m * (double)m * kmax * nb;
  // 1. tridiagonalisation.  Rows in shared memory when they fit: one thread-block
  // cluster of up to 16 CTAs per matrix for a batch or when `prefer_cluster`
  // (co-scheduled and, unlike cooperative launches, concurrent with other streams'
  // work), else a cooperative launch over ~m/4 CTAs per matrix (the fastest single
  // reduction); rows in global memory beyond that.  CBC_TRIDIAG_CTAS overrides the CTA
  // count (1..16 selects a cluster).
  int Pw = 0;
  if (const char* env = getenv("CBC_TRIDIAG_CTAS")) Pw = std::max(0, std::min(num_sms, atoi(env)));
  auto shm_for = [&](int P) {
    return (((size_t)((m + P - 1) / P) + (df ? 8 : 4)) * m + P) * ts;
  };
  // double-float rows pay off when the batch makes the reduction throughput bound; a
  // lone reduction is latency bound and runs faster in FP64
  df = df && nb > 1;
  const void* ksm = df ? (const void*)tridiag_smem_kernel<T, true>
                       : (const void*)tridiag_smem_kernel<T, false>;
  const size_t shm_cap = 160 * 1024;
  int P = Pw > 0 ? Pw : std::max(1, std::min(16, m / 2));
  bool cluster = false;
  if ((Pw > 0 || prefer_cluster || nb > 1) && P <= 16 && shm_for(P) <= shm_cap) {
    err = allow_max_smem(ksm);
    if (err != cudaSuccess) return err;
    cluster = cluster_ctas(ksm, P, TPB, shm_for(P)) == P;
  }
  if (!cluster && Pw <= 0) P = std::max(1, std::min(num_sms, m / 4));
  // batches (and concurrent instances) use the cluster reduction with the rows' lower
  // triangles in shared memory and the exchanges through distributed shared memory
  // (tridiag_cluster.cu); CBC_TRIDIAG_CTAS selects the polling kernels above instead
  int Pc = 0;
  if ((nb > 1 || prefer_cluster) && Pw <= 0 && m >= 2) Pc = tridiag_cluster_size<T>(m, df);
  if (Pc > 0) cluster = false;
  const bool in_smem = Pc == 0 && (cluster || shm_for(P) <= shm_cap);
  {
    // barrier, tau and e[0] start at zero; with the rows in shared memory the exchange
    // buffers start as all-ones bit patterns (the "not yet written" mark)
    WsInit wi{};
    auto add = [&](void* p, size_t bytes, unsigned long long v) {
      wi.seg[wi.nseg] = static_cast<unsigned long long*>(p);
      wi.words[wi.nseg] = (int64_t)(bytes / 8);
      wi.val[wi.nseg] = v;
      ++wi.nseg;
    };
    add(bar, sizeof(GridBarrier), 0ull);
    add(tau, ts * m, 0ull);
    add(e, sizeof(double), 0ull);
    if (in_smem) {
      add(V, ts * (size_t)m * m, ~0ull);
      add(Pg, ts * (size_t)m * m, ~0ull);
      add(Dg, ts * (size_t)m * m, ~0ull);
    }
    wi.wb = wb;
    note_launches(CBC_K_AUX, 1);
    ws_init_kernel<<<dim3((unsigned)std::min<int64_t>(64, ((int64_t)m * m * (ts / 8) + 255) / 256), nb), 256, 0, s>>>(wi);
    err = cudaGetLastError();
    if (err == cudaSuccess && in_smem) err = allow_max_smem(ksm);
    if (err != cudaSuccess) return err;
  }
  {
  KTimer tt(CBC_K_TRIDIAG, s, (cluster || Pc > 0) ? 1 : nb, fl_tri);
  if (Pc > 0) {
    err = tridiag_cluster<T>(A, m, d, e, tau, V, (int64_t)m * m, wb, nb, Pc, df, s);
  } else if (cluster) {
    Tri2Args<T> ta{A, m, d, e, tau, V, Pg, Dg, status, P, (int64_t)m * m, wb};
    void* args[] = {&ta};
    err = launch_cluster(ksm, P, nb * P, TPB, shm_for(P), args, s);
  } else {
    for (int b = 0; b < nb && err == cudaSuccess; ++b) {
      const size_t off = (size_t)b * wb;
      T* Ab = A + (int64_t)b * m * m;
      if (in_smem) {
        Tri2Args<T> ta{Ab, m, byte_shift(d, off), byte_shift(e, off), byte_shift(tau, off),
                       byte_shift(V, off), byte_shift(Pg, off), byte_shift(Dg, off), status, P, 0, 0};
        void* args[] = {&ta};
        err = cudaLaunchCooperativeKernel(ksm, dim3(P), dim3(TPB),
                                          args, shm_for(P), s);
      } else {
        TriArgs<T> ta{Ab, m, byte_shift(d, off), byte_shift(e, off), byte_shift(tau, off),
                      byte_shift(V, off), byte_shift(vbuf, off), byte_shift(p, off),
                      byte_shift(dot, off), byte_shift(bar, off), status};
        void* args[] = {&ta};
        err = cudaLaunchCooperativeKernel((const void*)tridiag_kernel<T>, dim3(P), dim3(TPB), args,
                                          0, s);
      }
    }
  }
  }
  if (err != cudaSuccess) return err;
  KTimer te(CBC_K_EIG, s, 4, fl_rest);
  // 2. eigenvalue estimates
  const int wpb = 8;
  bisect32_kernel<<<dim3((m + wpb - 1) / wpb, nb), 32 * wpb, 2 * sizeof(float) * m, s>>>(
      d, e, m, lam32, wb);
  // 3. eigenvectors of T for the candidates, FP64.  The LU and the solves are long
  // dependent FP64 chains: alone, one candidate per CTA runs fastest (a whole SM and its
  // FP64 unit per chain); in a batch with many candidates per SM, up to 16 candidates
  // share a warp (one per lane), which issues 16x fewer FP64 warp instructions.
  int tpb = 1;
  if ((size_t)nb * kmax >= 4 * (size_t)num_sms)
    tpb = (int)std::max<size_t>(1, std::min<size_t>(16, (200 * 1024 - 64) / ((size_t)m * 41)));
  size_t shi = (size_t)tpb * m * 41 + 64;
  err = allow_max_smem((const void*)invit_kernel);
  if (err != cudaSuccess) return err;
  InvArgs ia{d, e, lam32, m, kmax, X, rq, wb};
  invit_kernel<<<dim3((kmax + tpb - 1) / tpb, nb), tpb, shi, s>>>(ia);
  // clusters: one warp each, four CTAs per matrix that share its clusters round robin, as
  // many members per pass as shared memory holds
  if (kmax >= 2) {
    const int per = (int)std::max<size_t>(1, std::min<size_t>(32, (200 * 1024 - 64) / ((size_t)m * 41)));
    const size_t shc = (size_t)per * m * 41 + 64;
    err = allow_max_smem((const void*)invit_cluster_kernel);
    if (err != cudaSuccess) return err;
    invit_cluster_kernel<<<dim3(std::min(4, kmax / 2), nb), 32, shc, s>>>(ia, per);
  }
  // 4. rank rule on the refined eigenvalues
  rank_kernel<<<nb, 256, 0, s>>>(d, rq, lam32, m, kmax, (long long)max_bond, tol, floor_rel,
                                 k_dev, lam, wb);
  // 5. back transformation: 32 vectors per CTA (fewer FP64 instructions) when u fits in
  // shared memory and the batch gives enough CTAs to spread the FP64 work over the SMs;
  // else one vector per CTA
  const size_t shm32 = ((size_t)m * 32 + 3 * (size_t)m) * ts;
  if (shm32 <= 200 * 1024 && (size_t)nb * ((kmax + 31) / 32) * 2 >= (size_t)num_sms) {
    const void* kbt = df ? (const void*)backtransform32_kernel<T, true>
                         : (const void*)backtransform32_kernel<T, false>;
    err = allow_max_smem(kbt);
    if (err != cudaSuccess) return err;
    if (df)
      backtransform32_kernel<T, true><<<dim3((kmax + 31) / 32, nb), 32 * BT_WARPS, shm32, s>>>(
          V, tau, X, m, kmax, k_dev, U, wb);
    else
      backtransform32_kernel<T, false><<<dim3((kmax + 31) / 32, nb), 32 * BT_WARPS, shm32, s>>>(
          V, tau, X, m, kmax, k_dev, U, wb);
    return cudaGetLastError();
  }
  size_t shm = (size_t)m * ts;
  if (shm > 48 * 1024) {
    err = allow_max_smem((const void*)backtransform_kernel<T>);
    if (err != cudaSuccess) return err;
  }
  backtransform_kernel<T><<<dim3(kmax, nb), 128, shm, s>>>(V, tau, X, m, kmax, k_dev, U, wb);
  return cudaGetLastError();
}

template cudaError_t heev_top<double>(double*, int, int, int64_t, double, double, double*,
                                      double*, int*, void*, int*, int, cudaStream_t, int, bool,
                                      bool);
template cudaError_t heev_top<zdbl>(zdbl*, int, int, int64_t, double, double, double*, zdbl*,
                                    int*, void*, int*, int, cudaStream_t, int, bool, bool);

}  // namespace cbc
