// FP64 SIMT strided GEMM: the arithmetic of the plain-FP64 CBC path.
//
// Every contraction of Sec. III (Eqs. (tt_cbc_first_contraction) ...
// (cbc_final_contraction)) and every Gram product is one call of this kernel on leg
// views of the node tensors (kernels.cuh: View).  On GB300 the FP64 pipe delivers
// about 2 DFMA per clock per SM, so this kernel is FP64-throughput bound by design: a
// 64x64 output tile per CTA, 16-deep K slices staged in shared memory, 4x4 outputs
// per thread, and a K split (FP64 atomics into a zeroed C) when the output tiles
// alone cannot occupy every SM.
#include <algorithm>

#include "kernels.cuh"
#include "planner.h"

namespace cbc {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

template <typename T>
struct GemmArgs {
  int M, N, K, splits, kchunk;
  const T* A;
  View va;
  const T* B;
  View vb;
  T* C;
  View vc;
};

template <typename T, bool CA, bool CB, bool ATOMIC>
__global__ void __launch_bounds__(NT) gemm_f64_kernel(GemmArgs<T> g) {
  using O = ops<T>;
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  __shared__ int64_t a_row[BM];
  __shared__ int64_t b_col[BN];

  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int bm = blockIdx.y * BM, bn = blockIdx.x * BN;
  const int batch = blockIdx.z / g.splits;
  const int split = blockIdx.z % g.splits;
  const int kbeg = split * g.kchunk;
  const int kend = min(g.K, kbeg + g.kchunk);

  const T* A = g.A + (int64_t)batch * g.va.bs;
  const T* B = g.B + (int64_t)batch * g.vb.bs;
  T* C = g.C + (int64_t)batch * g.vc.bs;

  for (int i = tid; i < BM; i += NT) a_row[i] = (bm + i < g.M) ? g.va.roff(bm + i) : -1;
  for (int i = tid; i < BN; i += NT) b_col[i] = (bn + i < g.N) ? g.vb.coff(bn + i) : -1;
  __syncthreads();

  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = O::zero();

  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    // A tile: BM x BK, consecutive threads walk K (the contiguous leg of most views)
#pragma unroll
    for (int q = 0; q < (BM * BK) / NT; ++q) {
      int idx = tid + q * NT;
      int kk = idx % BK, mm = idx / BK;
      int k = k0 + kk;
      T v = O::zero();
      int64_t ro = a_row[mm];
      if (ro >= 0 && k < kend) {
        v = A[ro + g.va.coff(k)];
        if (CA) v = O::conj(v);
      }
      As[kk][mm] = v;
    }
    // B tile: BK x BN, consecutive threads walk N
#pragma unroll
    for (int q = 0; q < (BN * BK) / NT; ++q) {
      int idx = tid + q * NT;
      int nn = idx % BN, kk = idx / BN;
      int k = k0 + kk;
      T v = O::zero();
      int64_t co = b_col[nn];
      if (co >= 0 && k < kend) {
        v = B[g.vb.roff(k) + co];
        if (CB) v = O::conj(v);
      }
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = O::fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }

#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int r = bm + ty + 16 * i;
    if (r >= g.M) continue;
    int64_t ro = g.vc.roff(r);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int c = bn + tx + 16 * j;
      if (c >= g.N) continue;
      T* dst = C + ro + g.vc.coff(c);
      if (ATOMIC) {
        if constexpr (O::cplx) {
          double* d = reinterpret_cast<double*>(dst);
          atomicAdd(d, O::real(acc[i][j]));
          atomicAdd(d + 1, O::imag(acc[i][j]));
        } else {
          atomicAdd(reinterpret_cast<double*>(dst), O::real(acc[i][j]));
        }
      } else {
        *dst = acc[i][j];
      }
    }
  }
}

template <typename T>
__global__ void zero_view_kernel(T* C, View vc, int M, int N, int batch) {
  int64_t total = (int64_t)M * N * batch;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int c = (int)(t % N);
    int64_t rb = t / N;
    int r = (int)(rb % M);
    int b = (int)(rb / M);
    C[(int64_t)b * vc.bs + vc.roff(r) + vc.coff(c)] = ops<T>::zero();
  }
}

int g_num_sms = 0;

}  // namespace

template <typename T>
cudaError_t gemm_f64(int M, int N, int K, int batch, const T* A, const View& va, bool conjA,
                     const T* B, const View& vb, bool conjB, T* C, const View& vc,
                     cudaStream_t s) {
  if (M <= 0 || N <= 0 || batch <= 0) return cudaSuccess;
  if (g_num_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 148;
  }
  int tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN) * batch;
  int ksteps = (K + BK - 1) / BK;
  int splits = 1;
  int target = 2 * g_num_sms;
  if (tiles < target && ksteps >= 16) {
    splits = (target + tiles - 1) / tiles;
    splits = min(splits, ksteps / 8);
    splits = max(splits, 1);
  }
  int kchunk = ((ksteps + splits - 1) / splits) * BK;
  splits = max(1, (K + kchunk - 1) / kchunk);
  if (K <= 0) {  // empty contraction: C = 0
    note_launches(CBC_K_GEMM_F64, 1);
    zero_view_kernel<T><<<256, 256, 0, s>>>(C, vc, M, N, batch);
    return cudaGetLastError();
  }
  GemmArgs<T> g{M, N, K, splits, kchunk, A, va, B, vb, C, vc};
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, batch * splits);
  note_launches(CBC_K_GEMM_F64, splits > 1 ? 2 : 1);
  if (splits > 1) {
    int zb = (int)std::min<int64_t>(4096, ((int64_t)M * N * batch + 255) / 256);
    zero_view_kernel<T><<<zb, 256, 0, s>>>(C, vc, M, N, batch);
  }
#define CBC_GEMM_LAUNCH(CA, CB)                                                     \
  if (splits > 1)                                                                   \
    gemm_f64_kernel<T, CA, CB, true><<<grid, NT, 0, s>>>(g);                        \
  else                                                                              \
    gemm_f64_kernel<T, CA, CB, false><<<grid, NT, 0, s>>>(g);
  if (conjA && conjB) {
    CBC_GEMM_LAUNCH(true, true)
  } else if (conjA) {
    CBC_GEMM_LAUNCH(true, false)
  } else if (conjB) {
    CBC_GEMM_LAUNCH(false, true)
  } else {
    CBC_GEMM_LAUNCH(false, false)
  }
#undef CBC_GEMM_LAUNCH
  return cudaGetLastError();
}

template cudaError_t gemm_f64<double>(int, int, int, int, const double*, const View&, bool,
                                      const double*, const View&, bool, double*, const View&,
                                      cudaStream_t);
template cudaError_t gemm_f64<zdbl>(int, int, int, int, const zdbl*, const View&, bool,
                                    const zdbl*, const View&, bool, zdbl*, const View&,
                                    cudaStream_t);

}  // namespace cbc
