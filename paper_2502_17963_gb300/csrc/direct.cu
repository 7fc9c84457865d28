// Direct (on-the-fly, slice-by-slice) density fitting (Sec. 2.2): when B does
// not fit in HBM, (Q|mu nu) is regenerated in aux blocks at every Fock build.
// The Coulomb matrix needs two passes of regeneration, as the paper notes:
//   pass 1, per block:  gamma_Q = (Q|D) = sum_{mu nu} (Q|mu nu) D_mu nu   and
//                       X_Q = (Q|..) C_occ (the exchange intermediate);
//   then                c = V^{-1} gamma = L^{-T} L^{-1} gamma,
//                       Y = L^{-1} X,  K = sum_{P,i} Y_P,mu i Y_P,nu i;
//   pass 2, per block:  J += sum_Q c_Q (Q|mu nu).
// (These equal the stored-mode J and K: J = sum_P B_P (B_P:D) with
// B = L^{-1}(Q|..) gives sum_{QQ'} (Q|..) (V^{-1})_{QQ'} (Q'|D).)
// Integrals and the gamma / c / J parts are FP64; X, Y and K run either in
// FP64 (DFMA, small systems) or on the tensor cores (tc.cu).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "bqc_internal.h"
#include "df_internal.h"
#include "gemm64.cuh"

namespace bqc {

// D2[col(mu,nu)] = (2 - delta_mu nu) sum_i C[mu][i] C[nu][i], packed lower triangle.
__global__ void k_density_packed(const double *__restrict__ C, int n, int nocc, double *D2) {
  const int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t npair = (int64_t)n * (n + 1) / 2;
  if (col >= npair) return;
  int64_t mu = (int64_t)((sqrt(8.0 * (double)col + 1.0) - 1.0) * 0.5);
  while ((mu + 1) * (mu + 2) / 2 <= col) ++mu;
  while (mu * (mu + 1) / 2 > col) --mu;
  const int64_t nu = col - mu * (mu + 1) / 2;
  const double *a = C + mu * nocc, *b = C + nu * nocc;
  double s = 0.0;
  for (int i = 0; i < nocc; ++i) s = fma(a[i], b[i], s);
  D2[col] = (mu == nu) ? s : 2.0 * s;
}

// g[q] = sum_col raw[q][col] D2[col]  (one block per aux row).
__global__ void __launch_bounds__(256) k_rows_dot(const double *__restrict__ raw, int64_t npair,
                                                  const double *__restrict__ D2, double *g) {
  const int q = blockIdx.x;
  const double *r = raw + (int64_t)q * npair;
  double s = 0.0;
  for (int64_t c = threadIdx.x; c < npair; c += blockDim.x) s = fma(r[c], D2[c], s);
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) g[q] = red[0];
}

// Jp[col] += sum_q c[q] raw[q][col]  (thread per column, coalesced over columns).
__global__ void __launch_bounds__(256) k_cols_axpy(const double *__restrict__ raw, int nq,
                                                   int64_t npair, const double *__restrict__ c,
                                                   double *__restrict__ Jp) {
  const int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= npair) return;
  double s = 0.0;
  for (int q = 0; q < nq; ++q) s = fma(__ldg(c + q), raw[(int64_t)q * npair + col], s);
  Jp[col] += s;
}

// y = L^{-1} x (L^{-1} lower, n x n): one block per row.
__global__ void __launch_bounds__(256) k_lower_gemv(const double *__restrict__ Li, int n,
                                                    const double *__restrict__ x, double *y) {
  const int r = blockIdx.x;
  double s = 0.0;
  for (int q = threadIdx.x; q <= r; q += blockDim.x) s = fma(Li[(int64_t)r * n + q], x[q], s);
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) y[r] = red[0];
}

// y = L^{-T} x: thread per column q, coalesced reads along rows.
__global__ void k_lower_gemv_t(const double *__restrict__ Li, int n, const double *__restrict__ x,
                               double *y) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  double s = 0.0;
  for (int r = q; r < n; ++r) s = fma(Li[(int64_t)r * n + q], x[r], s);
  y[q] = s;
}

__global__ void k_identity(double *A, int n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)n * n) return;
  A[i] = (i / n == i % n) ? 1.0 : 0.0;
}

__global__ void k_unpack_sym3(const double *Jp, int n, double *J) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)n * n) return;
  const int64_t r = i / n, c = i % n;
  const int64_t hi = r > c ? r : c, lo = r > c ? c : r;
  J[i] = Jp[hi * (hi + 1) / 2 + lo];
}

static inline unsigned nb(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

int direct_setup(Df *df, cudaStream_t s) {
  Ctx *ctx = df->ctx;
  const Basis *b = df->basis;
  const int n = b->nbf, naux = b->naux, no = b->nocc;
  df->aux_block = std::max(1, std::min(df->opts.aux_block, naux));
  // L^{-1} (FP64), once
  BQC_TRY(df->Linv.alloc(ctx, (size_t)naux * naux * 8));
  k_identity<<<nb((int64_t)naux * naux), 256, 0, s>>>(df->Linv.as<double>(), naux);
  BQC_LAUNCH_CHECK();
  BQC_TRY(trsm_lower_left(ctx, df->L.as<double>(), naux, df->Linv.as<double>(), naux, naux, s));
  BQC_TRY(df->raw.alloc(ctx, (size_t)df->aux_block * df->npair * 8));
  BQC_TRY(df->gamma.alloc(ctx, (size_t)naux * 8 * 2));
  BQC_TRY(df->D2.alloc(ctx, (size_t)df->npair * 8));
  BQC_TRY(df->Jp.alloc(ctx, (size_t)df->npair * 8));
  if (df->opts.keep_fp32) {
    // largest X-pass sub-block (multiple of 32 aux rows) that fits the free memory
    size_t fr = 0, tot = 0;
    BQC_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
    const size_t budget = (size_t)(fr * 0.92);
    int bs = ((df->aux_block + 31) / 32) * 32;
    while (bs > 32 && direct_mixed_bytes(n, naux, no, bs) > budget) bs -= 32;
    if (direct_mixed_bytes(n, naux, no, bs) > budget) return BQC_E_OOM;
    BQC_TRY(direct_mixed_setup(df, df->Linv.as<double>(), bs, s));
  }
  return BQC_OK;
}

int jk_direct(Df *df, const double *C, int prec, double *J, double *K, cudaStream_t s) {
  Ctx *ctx = df->ctx;
  const Basis *b = df->basis;
  const int n = b->nbf, naux = b->naux, no = b->nocc;
  const int64_t npair = df->npair;
  const int bk = df->aux_block;
  if (prec == BQC_PREC_MIXED_F16X3) {
    set_error("direct mode runs FP64, MIXED_TF32 and MIXED_TF32X3 builds", __FILE__, __LINE__);
    return BQC_E_UNSUPPORTED;
  }
  const bool mixed = prec != BQC_PREC_FP64;
  const int split = prec == BQC_PREC_MIXED_TF32X3 ? 3 : 1;
  if (mixed && !df->dmixed) return BQC_E_INVALID;
  if (!mixed && !df->Xraw.p) BQC_TRY(df->Xraw.alloc(ctx, (size_t)naux * n * no * 8));
  double *raw = df->raw.as<double>();
  double *gam = df->gamma.as<double>(), *cvec = gam + naux;
  df->mark(0, s);
  k_density_packed<<<nb(npair), 256, 0, s>>>(C, n, no, df->D2.as<double>());
  BQC_LAUNCH_CHECK();
  if (mixed) BQC_TRY(direct_mixed_prep_c(df, C, split, s));
  df->mark(1, s);
  // pass 1: gamma and X
  for (int q0 = 0; q0 < naux; q0 += bk) {
    const int nq = std::min(bk, naux - q0);
    BQC_CUDA_TRY(cudaMemsetAsync(raw, 0, (size_t)nq * npair * 8, s));
    BQC_TRY(launch_eri3c(b, &df->plan, q0, q0 + nq, raw, npair, s));
    k_rows_dot<<<nq, 256, 0, s>>>(raw, npair, df->D2.as<double>(), gam + q0);
    BQC_LAUNCH_CHECK();
    if (mixed) {
      BQC_TRY(direct_mixed_block(df, raw, q0, nq, split, s));
    } else {
      Gemm64Args g;  // X_Q = (Q|..)sym C
      g.M = n;
      g.N = no;
      g.K1 = 1;
      g.K2 = n;
      g.A = raw;
      g.bsA = npair;
      g.B = C;
      g.ldb = no;
      g.C = df->Xraw.as<double>() + (int64_t)q0 * n * no;
      g.ldc = no;
      g.bsC = (int64_t)n * no;
      g.batch = nq;
      BQC_TRY(launch_gemm64(kASym, false, g, s));
    }
  }
  df->mark(2, s);
  // c = L^{-T} L^{-1} gamma
  k_lower_gemv<<<naux, 256, 0, s>>>(df->Linv.as<double>(), naux, gam, cvec);
  BQC_LAUNCH_CHECK();
  k_lower_gemv_t<<<nb(naux, 128), 128, 0, s>>>(df->Linv.as<double>(), naux, cvec, gam);
  BQC_LAUNCH_CHECK();  // gam now holds c
  // K
  if (mixed) {
    BQC_TRY(direct_mixed_finish(df, split, K, s));
  } else {
    BQC_TRY(trsm_lower_left(ctx, df->L.as<double>(), naux, df->Xraw.as<double>(),
                            (int64_t)n * no, (int64_t)n * no, s));
    Gemm64Args k;
    k.M = n;
    k.N = n;
    k.K1 = naux;
    k.K2 = no;
    k.A = df->Xraw.as<double>();
    k.lda = no;
    k.sA1 = (int64_t)n * no;
    k.B = k.A;
    k.ldb = no;
    k.sB1 = (int64_t)n * no;
    k.C = K;
    k.ldc = n;
    k.lower_only = 1;
    k.mirror = 1;
    BQC_TRY(launch_gemm64(kAN, true, k, s));
  }
  df->mark(3, s);
  // pass 2: J = sum_Q c_Q (Q|..)
  BQC_CUDA_TRY(cudaMemsetAsync(df->Jp.p, 0, (size_t)npair * 8, s));
  for (int q0 = 0; q0 < naux; q0 += bk) {
    const int nq = std::min(bk, naux - q0);
    BQC_CUDA_TRY(cudaMemsetAsync(raw, 0, (size_t)nq * npair * 8, s));
    BQC_TRY(launch_eri3c(b, &df->plan, q0, q0 + nq, raw, npair, s));
    k_cols_axpy<<<nb(npair), 256, 0, s>>>(raw, nq, npair, gam + q0, df->Jp.as<double>());
    BQC_LAUNCH_CHECK();
  }
  k_unpack_sym3<<<nb((int64_t)n * n), 256, 0, s>>>(df->Jp.as<double>(), n, J);
  BQC_LAUNCH_CHECK();
  df->mark(4, s);
  return BQC_OK;
}

}  // namespace bqc
