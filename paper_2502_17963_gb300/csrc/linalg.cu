// FP64 dense kernels of the DF pipeline: a DFMA GEMM (the plain-FP64
// contractions and the metric solve), blocked Cholesky of the Coulomb metric
// V = L L^T, and the in-place triangular solve B = L^{-1} (Q|mu nu) that
// turns raw three-centre integrals into the Cholesky-decomposed ERIs (CD-ERIs) of
// Sec. 2.2.
//
// On GB300 FP64 runs at ~1.2 TFLOP/s (about 2 DFMA per clock per SM), so a
// 64x64 register-blocked tile already saturates the FP64 pipe; the kernels
// are written for that pipe, not for the tensor cores.
#include <cuda_runtime.h>

#include <algorithm>

#include "bqc_internal.h"
#include "gemm64.cuh"

namespace bqc {

int dgemm(bool tA, bool tB, int M, int N, int K, double alpha, const double *A, int64_t lda,
          const double *B, int64_t ldb, double beta, double *C, int64_t ldc, cudaStream_t s) {
  Gemm64Args g;
  g.M = M;
  g.N = N;
  g.K1 = 1;
  g.K2 = K;
  g.alpha = alpha;
  g.beta = beta;
  g.A = A;
  g.lda = lda;
  g.sA1 = 0;
  g.B = B;
  g.ldb = ldb;
  g.sB1 = 0;
  g.C = C;
  g.ldc = ldc;
  return launch_gemm64(tA ? kAT : kAN, tB, g, s);
}

// ----------------------------------------------------------- Cholesky ---

constexpr int kNB = 64;

// Unblocked Cholesky of the kNB x kNB diagonal block at (k0, k0), in shared
// memory; writes L (lower) and zeros above.  flag <- 1 when not positive.
__global__ void __launch_bounds__(256) k_potrf_diag(double *A, int n, int k0, int *flag) {
  __shared__ double a[kNB][kNB + 1];
  const int nb = min(kNB, n - k0);
  for (int i = threadIdx.x; i < kNB * kNB; i += blockDim.x) {
    const int r = i / kNB, c = i % kNB;
    a[r][c] = (r < nb && c < nb) ? A[(int64_t)(k0 + r) * n + k0 + c] : 0.0;
  }
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (threadIdx.x == 0) {
      const double d = a[j][j];
      if (!(d > 0.0)) {
        atomicExch(flag, 1);
        a[j][j] = 1.0;
      } else {
        a[j][j] = sqrt(d);
      }
    }
    __syncthreads();
    const double djj = a[j][j];
    for (int i = j + 1 + threadIdx.x; i < nb; i += blockDim.x) a[i][j] /= djj;
    __syncthreads();
    const int m = nb - j - 1;
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
      const int r = j + 1 + t / m, c = j + 1 + t % m;
      if (c <= r) a[r][c] -= a[r][j] * a[c][j];
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < nb * nb; i += blockDim.x) {
    const int r = i / nb, c = i % nb;
    A[(int64_t)(k0 + r) * n + k0 + c] = (c <= r) ? a[r][c] : 0.0;
  }
}

// Rows below the diagonal block: A_rk := A_rk L_kk^{-T} (forward substitution
// per row, one thread per row); also zeroes the block above the diagonal.
__global__ void __launch_bounds__(128) k_chol_panel(double *A, int n, int k0) {
  __shared__ double L[kNB][kNB + 1];
  const int nb = min(kNB, n - k0);
  for (int i = threadIdx.x; i < kNB * kNB; i += blockDim.x) {
    const int r = i / kNB, c = i % kNB;
    L[r][c] = (r < nb && c < nb) ? A[(int64_t)(k0 + r) * n + k0 + c] : 0.0;
  }
  __syncthreads();
  const int row = k0 + nb + blockIdx.x * blockDim.x + threadIdx.x;
  if (row < n) {
    double x[kNB];
    double *ar = A + (int64_t)row * n + k0;
    for (int j = 0; j < nb; ++j) {
      double v = ar[j];
      for (int l = 0; l < j; ++l) v -= x[l] * L[j][l];
      x[j] = v / L[j][j];
    }
    for (int j = 0; j < nb; ++j) ar[j] = x[j];
    // upper block (row k0 + j, column `row`) = 0
    for (int j = 0; j < nb; ++j) A[(int64_t)(k0 + j) * n + row] = 0.0;
  }
}

int cholesky_lower(Ctx *ctx, double *A, int n, cudaStream_t s) {
  for (int k0 = 0; k0 < n; k0 += kNB) {
    const int nb = std::min(kNB, n - k0);
    k_potrf_diag<<<1, 256, 0, s>>>(A, n, k0, ctx->flag);
    BQC_LAUNCH_CHECK();
    const int rem = n - k0 - nb;
    if (rem <= 0) break;
    k_chol_panel<<<(rem + 127) / 128, 128, 0, s>>>(A, n, k0);
    BQC_LAUNCH_CHECK();
    // trailing update, lower triangle only: A22 -= L21 L21^T
    Gemm64Args g;
    g.M = rem;
    g.N = rem;
    g.K1 = 1;
    g.K2 = nb;
    g.alpha = -1.0;
    g.beta = 1.0;
    g.A = A + (int64_t)(k0 + nb) * n + k0;
    g.lda = n;
    g.sA1 = 0;
    g.B = g.A;
    g.ldb = n;
    g.sB1 = 0;
    g.C = A + (int64_t)(k0 + nb) * n + k0 + nb;
    g.ldc = n;
    g.lower_only = 1;
    BQC_TRY(launch_gemm64(kAN, true, g, s));
  }
  return BQC_OK;
}

// ------------------------------------------------------ triangular solve ---

// X_k := L_kk^{-1} X_k for the kNB rows of block k, one thread per column.
__global__ void __launch_bounds__(128) k_trsm_diag(const double *L, int n, int k0, double *X,
                                                   int64_t ncol, int64_t ld) {
  __shared__ double Lk[kNB][kNB + 1];
  const int nb = min(kNB, n - k0);
  for (int i = threadIdx.x; i < kNB * kNB; i += blockDim.x) {
    const int r = i / kNB, c = i % kNB;
    Lk[r][c] = (r < nb && c < nb) ? L[(int64_t)(k0 + r) * n + k0 + c] : 0.0;
  }
  __syncthreads();
  const int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= ncol) return;
  double x[kNB];
  double *xc = X + (int64_t)k0 * ld + col;
  for (int j = 0; j < nb; ++j) {
    double v = xc[(int64_t)j * ld];
    for (int l = 0; l < j; ++l) v -= Lk[j][l] * x[l];
    x[j] = v / Lk[j][j];
    xc[(int64_t)j * ld] = x[j];
  }
}

int trsm_lower_left(Ctx *ctx, const double *L, int n, double *X, int64_t ncol, int64_t ld,
                    cudaStream_t s) {
  (void)ctx;
  if (ncol <= 0) return BQC_OK;
  for (int k0 = 0; k0 < n; k0 += kNB) {
    const int nb = std::min(kNB, n - k0);
    k_trsm_diag<<<(unsigned)((ncol + 127) / 128), 128, 0, s>>>(L, n, k0, X, ncol, ld);
    BQC_LAUNCH_CHECK();
    const int rem = n - k0 - nb;
    if (rem <= 0) break;
    // X[k0+nb:, :] -= L[k0+nb:, k0:k0+nb] X[k0:k0+nb, :]
    Gemm64Args g;
    g.M = rem;
    g.N = (int)std::min<int64_t>(ncol, (int64_t)1 << 30);
    g.K1 = 1;
    g.K2 = nb;
    g.alpha = -1.0;
    g.beta = 1.0;
    g.A = L + (int64_t)(k0 + nb) * n + k0;
    g.lda = n;
    g.sA1 = 0;
    g.B = X + (int64_t)k0 * ld;
    g.ldb = ld;
    g.sB1 = 0;
    g.C = X + (int64_t)(k0 + nb) * ld;
    g.ldc = ld;
    BQC_TRY(launch_gemm64(kAN, false, g, s));
  }
  return BQC_OK;
}

}  // namespace bqc
