// DF-MP2 on the resident three-index tensor (Sec. 2.3).
//
// The paper's MP2 stage reuses the CD-ERIs of the mean field: in canonical
// SCF orbitals, B_P,ia = sum_{mu nu} C_mu i B_P,mu nu C_nu a, the
// integrals (ia|jb) = sum_P B_P,ia B_P,jb are formed block by block as
// matrix products, and the closed-shell second-order energy
//   E2 = sum_{ijab} (ia|jb) [2 (ia|jb) - (ib|ja)] / (e_i + e_j - e_a - e_b)
// (Szabo & Ostlund Eq. 6.74) is accumulated with the denominator applied in
// place, one block of occupied pairs at a time, so no four-index array is
// ever held.  FP64: the register-blocked DFMA GEMM of gemm64.cuh;
// MIXED_F16X3: the pair blocks on the tensor cores (tc.cu).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <memory>
#include <vector>

#include "bqc_internal.h"
#include "df_internal.h"
#include "gemm64.cuh"

namespace bqc {

// Energy of the occupied pairs (i, j), i >= j, of one block of
// V[(ii, a)][(jj, b)] = (i a | j b) with i = i0 + ii, j = j0 + jj: one CTA per
// pair, a fixed-order reduction, epair[i * nocc + j] = weight * sum_ab; the
// weight is 2 for i > j (the (j, i) term is equal) and 1 for i = j.
__global__ void __launch_bounds__(256) k_mp2_pairs(const double *__restrict__ V, int64_t ldv,
                                                   int i0, int j0, int nvir,
                                                   const double *__restrict__ eps, int nocc,
                                                   double *__restrict__ epair) {
  const int ii = blockIdx.x, jj = blockIdx.y;
  const int i = i0 + ii, j = j0 + jj;
  if (j > i) return;  // uniform over the block
  const double eij = eps[i] + eps[j];
  const double *ev = eps + nocc;
  const double *Vi = V + (int64_t)ii * nvir * ldv + (int64_t)jj * nvir;
  double s = 0.0;
  const int64_t nab = (int64_t)nvir * nvir;
  for (int64_t e = threadIdx.x; e < nab; e += blockDim.x) {
    const int a = (int)(e / nvir), b = (int)(e % nvir);
    const double v = Vi[(int64_t)a * ldv + b];
    const double x = Vi[(int64_t)b * ldv + a];
    s += v * (2.0 * v - x) / (eij - ev[a] - ev[b]);
  }
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) epair[(int64_t)i * nocc + j] = (i == j ? 1.0 : 2.0) * red[0];
}

// *out = sum of the lower triangle of epair (nocc x nocc), in a fixed order.
__global__ void __launch_bounds__(256) k_mp2_sum(const double *__restrict__ epair, int nocc,
                                                 double *out) {
  double s = 0.0;
  for (int64_t e = threadIdx.x; e < (int64_t)nocc * nocc; e += blockDim.x) {
    const int i = (int)(e / nocc), j = (int)(e % nocc);
    if (j <= i) s += epair[e];
  }
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// Occupied-index block size: (bi * nvir)^2 doubles of (ia|jb) at most ~1 GiB,
// and at most 16 occupied orbitals (small systems still run several blocks).
static int mp2_block(int nocc, int nvir) {
  const double cap = (double)(1 << 27);  // doubles
  int bi = std::max(1, (int)(std::sqrt(cap) / std::max(1, nvir)));
  return std::max(1, std::min({bi, 16, nocc}));
}

// prec FP64: every GEMM on the DFMA path; MIXED_F16X3: the MO transform in
// FP64, the pair blocks as split-FP16 tensor-core GEMMs (FP32 accumulation in
// short chains, float-float drains, FP64 blocks), the energy in FP64.
static int mp2_run(Df *df, const double *C, const double *eps, int nmo, int prec, double *e2,
                   cudaStream_t s) {
  const Basis *b = df->basis;
  const int n = b->nbf, naux = b->naux, no = b->nocc, nv = nmo - no;
  Ctx *ctx = df->ctx;
  DBuf Bt, V, ep, out;
  BQC_TRY(ep.alloc(ctx, (size_t)no * no * 8));
  BQC_TRY(out.alloc(ctx, 8));
  BQC_CUDA_TRY(cudaMemsetAsync(ep.p, 0, ep.n, s));
  if (nv > 0) {
    // X_P = B_P C_occ (N x nocc per P), into the handle's FP64 X buffer
    Gemm64Args g;
    g.M = n;
    g.N = no;
    g.K1 = 1;
    g.K2 = n;
    g.A = df->B64.as<double>();
    g.bsA = df->npair;
    g.B = C;
    g.ldb = nmo;
    g.C = df->X64.as<double>();
    g.ldc = no;
    g.bsC = (int64_t)n * no;
    g.batch = naux;
    BQC_TRY(launch_gemm64(kASym, false, g, s));
    // B_P,ia = sum_nu X_P[nu][i] C[nu][no + a]  ->  Bt[P][i][a]
    BQC_TRY(Bt.alloc(ctx, (size_t)naux * no * nv * 8));
    Gemm64Args t;
    t.M = no;
    t.N = nv;
    t.K1 = 1;
    t.K2 = n;
    t.A = df->X64.as<double>();
    t.lda = no;
    t.bsA = (int64_t)n * no;
    t.B = C + no;
    t.ldb = nmo;
    t.C = Bt.as<double>();
    t.ldc = nv;
    t.bsC = (int64_t)no * nv;
    t.batch = naux;
    BQC_TRY(launch_gemm64(kAT, false, t, s));
    std::unique_ptr<Mp2Tc, Mp2TcDeleter> tcs;
    if (prec == BQC_PREC_MIXED_F16X3) {
      BQC_TRY(mp2_tc_setup(ctx, Bt.as<double>(), naux, no, nv, ctx->flag, tcs, s));
      BQC_CUDA_TRY(cudaStreamSynchronize(s));
      Bt.release();  // the split operand replaces it
    }
    const int bi = mp2_block(no, nv);
    BQC_TRY(V.alloc(ctx, (size_t)bi * nv * bi * nv * 8));
    const int64_t ldt = (int64_t)no * nv;
    for (int i0 = 0; i0 < no; i0 += bi) {
      const int ni = std::min(bi, no - i0);
      for (int j0 = 0; j0 <= i0; j0 += bi) {
        const int nj = std::min(bi, no - j0);
        // V[(ii,a)][(jj,b)] = sum_P Bt[P][i0+ii][a] Bt[P][j0+jj][b]
        if (tcs) {
          BQC_TRY(mp2_tc_block(tcs.get(), nv, i0, ni, j0, nj, V.as<double>(), (int64_t)nj * nv,
                               ctx->flag, s));
          k_mp2_pairs<<<dim3((unsigned)ni, (unsigned)nj), 256, 0, s>>>(
              V.as<double>(), (int64_t)nj * nv, i0, j0, nv, eps, no, ep.as<double>());
          BQC_LAUNCH_CHECK();
          continue;
        }
        Gemm64Args v;
        v.M = ni * nv;
        v.N = nj * nv;
        v.K1 = 1;
        v.K2 = naux;
        v.A = Bt.as<double>() + (int64_t)i0 * nv;
        v.lda = ldt;
        v.B = Bt.as<double>() + (int64_t)j0 * nv;
        v.ldb = ldt;
        v.C = V.as<double>();
        v.ldc = (int64_t)nj * nv;
        BQC_TRY(launch_gemm64(kAT, false, v, s));
        k_mp2_pairs<<<dim3((unsigned)ni, (unsigned)nj), 256, 0, s>>>(
            V.as<double>(), (int64_t)nj * nv, i0, j0, nv, eps, no, ep.as<double>());
        BQC_LAUNCH_CHECK();
      }
    }
  }
  k_mp2_sum<<<1, 256, 0, s>>>(ep.as<double>(), no, out.as<double>());
  BQC_LAUNCH_CHECK();
  BQC_CUDA_TRY(cudaMemcpyAsync(e2, out.p, 8, cudaMemcpyDeviceToHost, s));
  BQC_CUDA_TRY(cudaStreamSynchronize(s));
  return ctx->check_flag(s);
}

}  // namespace bqc

using namespace bqc;

extern "C" int bqc_mp2(bqc_df *df, const double *C_dev, const double *eps_dev, int nmo, int prec,
                       double *e2, bqc_stream_t stream) {
  if (!df || !C_dev || !eps_dev || !e2) return BQC_E_INVALID;
  NvtxRange nv("bqc_mp2");
  if (df->mode != BQC_DF_STORED || !df->B64.p || !df->X64.p || df->is_shard()) {
    set_error("bqc_mp2 needs a stored-mode DF handle holding the whole tensor", __FILE__, __LINE__);
    return BQC_E_INVALID;
  }
  if (nmo < df->basis->nocc || nmo > df->basis->nbf) return BQC_E_INVALID;
  BQC_CUDA_TRY(cudaSetDevice(df->ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == BQC_PREC_FP64 || prec == BQC_PREC_MIXED_F16X3)
    return mp2_run(df, C_dev, eps_dev, nmo, prec, e2, s);
  set_error("bqc_mp2: precision not available", __FILE__, __LINE__);
  return BQC_E_UNSUPPORTED;
}
