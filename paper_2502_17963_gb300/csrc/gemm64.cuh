// Register-blocked FP64 GEMM used by the plain-FP64 path and the metric
// solve:  C = beta C + alpha sum_{k1 < K1} sum_{k2 < K2} A(m, k1, k2) B(k1, k2, n)
// with row-major operands
//   A(m,k1,k2) = A[k1 sA1 + m lda + k2]          (kAN)
//              = A[k1 sA1 + k2 lda + m]          (kAT)
//              = Bsym_{k1}(m, k2), packed lower  (kASym: A[k1 sA1 + tri(max, min)])
//   B(k1,k2,n) = B[k1 sB1 + k2 ldb + n]   or  B[k1 sB1 + n ldb + k2] (transB).
// The two-level contraction index lets one launch contract over (P, i) for
// K = sum_P X_P X_P^T.  Batched over gridDim.z with per-batch strides.
// 64x64 tile, 16-deep k-steps, 256 threads, 4x4 outputs per thread.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "bqc_internal.h"

namespace bqc {

enum AMode { kAN = 0, kAT = 1, kASym = 2 };

struct Gemm64Args {
  int M = 0, N = 0;
  int K1 = 1, K2 = 0;
  double alpha = 1.0, beta = 0.0;
  const double *A = nullptr;
  int64_t lda = 0, sA1 = 0, bsA = 0;  // bsA: batch stride
  const double *B = nullptr;
  int64_t ldb = 0, sB1 = 0, bsB = 0;
  double *C = nullptr;
  int64_t ldc = 0, bsC = 0;
  int batch = 1;
  int lower_only = 0;  // compute only tiles with tile_n <= tile_m
  int mirror = 0;      // with lower_only and beta == 0: also write C^T into the upper part
};

template <int AM, bool TB>
__global__ void __launch_bounds__(256) k_gemm64(Gemm64Args g) {
  constexpr int T = 64, KT = 16;
  __shared__ double As[KT][T + 1];
  __shared__ double Bs[KT][T + 1];
  const int tm = blockIdx.y, tn = blockIdx.x;
  if (g.lower_only && tn > tm) return;
  const int z = blockIdx.z;
  const double *A = g.A + (int64_t)z * g.bsA;
  const double *B = g.B + (int64_t)z * g.bsB;
  double *C = g.C + (int64_t)z * g.bsC;
  const int m0 = tm * T, n0 = tn * T;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  for (int k1 = 0; k1 < g.K1; ++k1) {
    const double *Ak = A + (int64_t)k1 * g.sA1;
    const double *Bk = B + (int64_t)k1 * g.sB1;
    for (int k0 = 0; k0 < g.K2; k0 += KT) {
      // A tile: 64 (m) x 16 (k)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int e = threadIdx.x + r * 256;
        int mm, kk;
        if (AM == kAT) {
          mm = e % T;
          kk = e / T;
        } else {
          kk = e % KT;
          mm = e / KT;
        }
        const int gm = m0 + mm, gk = k0 + kk;
        double v = 0.0;
        if (gm < g.M && gk < g.K2) {
          if (AM == kAN) {
            v = Ak[(int64_t)gm * g.lda + gk];
          } else if (AM == kAT) {
            v = Ak[(int64_t)gk * g.lda + gm];
          } else {
            const int64_t hi = gm > gk ? gm : gk, lo = gm > gk ? gk : gm;
            v = Ak[hi * (hi + 1) / 2 + lo];
          }
        }
        As[kk][mm] = v;
      }
      // B tile: 16 (k) x 64 (n)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int e = threadIdx.x + r * 256;
        int kk, nn;
        if (TB) {
          kk = e % KT;
          nn = e / KT;
        } else {
          nn = e % T;
          kk = e / T;
        }
        const int gk = k0 + kk, gn = n0 + nn;
        double v = 0.0;
        if (gn < g.N && gk < g.K2)
          v = TB ? Bk[(int64_t)gn * g.ldb + gk] : Bk[(int64_t)gk * g.ldb + gn];
        Bs[kk][nn] = v;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < KT; ++kk) {
        double a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gm = m0 + ty + 16 * i, gn = n0 + tx + 16 * j;
      if (gm >= g.M || gn >= g.N) continue;
      if (g.lower_only && gn > gm) continue;
      double *c = C + (int64_t)gm * g.ldc + gn;
      const double v = g.alpha * acc[i][j] + (g.beta != 0.0 ? g.beta * *c : 0.0);
      *c = v;
      if (g.mirror && gn != gm) C[(int64_t)gn * g.ldc + gm] = v;
    }
}

inline int launch_gemm64(int amode, bool transB, const Gemm64Args &g, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0) return BQC_OK;
  const int64_t gx = (g.N + 63) / 64, gy = (g.M + 63) / 64;
  if (gy > 65535 || g.batch > 65535 || g.batch < 1) return BQC_E_INVALID;
  dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)g.batch);
  if (amode == kAN) {
    if (transB) k_gemm64<kAN, true><<<grid, 256, 0, s>>>(g);
    else k_gemm64<kAN, false><<<grid, 256, 0, s>>>(g);
  } else if (amode == kAT) {
    if (transB) k_gemm64<kAT, true><<<grid, 256, 0, s>>>(g);
    else k_gemm64<kAT, false><<<grid, 256, 0, s>>>(g);
  } else {
    if (transB) k_gemm64<kASym, true><<<grid, 256, 0, s>>>(g);
    else k_gemm64<kASym, false><<<grid, 256, 0, s>>>(g);
  }
  BQC_LAUNCH_CHECK();
  return BQC_OK;
}

}  // namespace bqc
