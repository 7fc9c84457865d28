// Density-fitting tensor and the J/K build (Sec. 2.2).
//
// Stored mode (the three-index tensor depends only on basis and geometry, so
// it is computed once and kept):
//   V = (P|Q) -> L (Cholesky) -> raw (Q|mu nu) packed lower triangle in FP64
//   -> B = L^{-1} raw in place -> optional TF32-rounded full-square shadow.
// Each Fock build then makes two passes over B, as the paper notes for the
// Coulomb matrix: the X pass (X_P = B_P C_occ, with w_P = <X_P, C_occ>) and
// the J pass (J = sum_P w_P B_P); K = sum_P X_P X_P^T.
// Direct mode (regenerated per aux block at every build): see direct.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "bqc_internal.h"
#include "df_internal.h"
#include "gemm64.cuh"

namespace bqc {

// w[P] = sum_{mu,i} X[P][mu][i] C[mu][i]  (one block per P, FP64).
__global__ void __launch_bounds__(256) k_wdot(const double *X, const double *C, int64_t nc,
                                              double *w) {
  const int P = blockIdx.x;
  const double *x = X + (int64_t)P * nc;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < nc; i += blockDim.x) s = fma(x[i], C[i], s);
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) w[P] = red[0];
}

// J pass over packed FP64 B: out[col] = sum_{P in [Pa, Pb)} w_P B[P][col] for
// the two adjacent columns c2, c2 + 1 a thread owns; P streams in increasing
// order (one read of B, coalesced), eight 16-byte loads in flight per thread.
__device__ __forceinline__ void jpass64_cols(const double *__restrict__ B,
                                             const double *__restrict__ w, int Pa, int Pb,
                                             int64_t npair, int64_t c2, double *__restrict__ out) {
  double a0 = 0.0, a1 = 0.0;
  if (c2 + 1 < npair && (npair % 2 == 0)) {
    const double2 *b2 = reinterpret_cast<const double2 *>(B + c2);
    const int64_t st = npair / 2;
    int P = Pa;
    for (; P + 8 <= Pb; P += 8) {
      double2 v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = __ldg(b2 + (int64_t)(P + k) * st);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const double wp = __ldg(w + P + k);
        a0 = fma(wp, v[k].x, a0);
        a1 = fma(wp, v[k].y, a1);
      }
    }
    for (; P < Pb; ++P) {
      const double2 v = __ldg(b2 + (int64_t)P * st);
      const double wp = __ldg(w + P);
      a0 = fma(wp, v.x, a0);
      a1 = fma(wp, v.y, a1);
    }
    out[c2] = a0;
    out[c2 + 1] = a1;
  } else {
    for (int P = Pa; P < Pb; ++P) {
      const double wp = __ldg(w + P);
      a0 = fma(wp, B[(int64_t)P * npair + c2], a0);
      if (c2 + 1 < npair) a1 = fma(wp, B[(int64_t)P * npair + c2 + 1], a1);
    }
    out[c2] = a0;
    if (c2 + 1 < npair) out[c2 + 1] = a1;
  }
}

// Jp[y][col] = sum_{P in chunk y} w_P B[P][col]: gridDim.y aux chunks give
// small systems enough blocks; the chunk partials are summed in a fixed order
// by k_unpack_jsum.
__global__ void __launch_bounds__(256) k_jpass64(const double *__restrict__ B,
                                                 const double *__restrict__ w, int naux,
                                                 int64_t npair, double *__restrict__ Jp) {
  const int64_t c2 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 2;
  if (c2 >= npair) return;
  const int per = (naux + gridDim.y - 1) / gridDim.y;
  const int Pa = blockIdx.y * per, Pb = min(naux, Pa + per);
  jpass64_cols(B, w, Pa, Pb, npair, c2, Jp + (int64_t)blockIdx.y * npair);
}

// The same for aux functions [P0, P1), partials into the slices y0 .. y0 +
// gridDim.y - 1 (the pieces of the split-FP16 build's pipeline).
__global__ void __launch_bounds__(256) k_jpass64_range(const double *__restrict__ B,
                                                       const double *__restrict__ w, int P0,
                                                       int P1, int64_t npair, int y0,
                                                       double *__restrict__ Jp) {
  const int64_t c2 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 2;
  if (c2 >= npair) return;
  const int per = (P1 - P0 + gridDim.y - 1) / gridDim.y;
  const int Pa = P0 + blockIdx.y * per, Pb = min(P1, Pa + per);
  jpass64_cols(B, w, Pa, Pb, npair, c2, Jp + (int64_t)(y0 + blockIdx.y) * npair);
}

// (sh, sl) += (wh + wl) (bh + bl) in float-float arithmetic: the exact
// product wh*bh (its rounding error from one FMA), the two cross terms (wl*bl
// is below 2^-48 of the product), and a two-sum into the running pair.
__device__ __forceinline__ void ff_acc(float &sh, float &sl, float wh, float wl, float bh,
                                       float bl) {
  const float p = wh * bh;
  float e = fmaf(wh, bh, -p);
  e = fmaf(wh, bl, e);
  e = fmaf(wl, bh, e);
  const float t = sh + p;
  const float bp = t - sh;
  const float err = (sh - (t - bp)) + (p - bp);
  sh = t;
  sl += err + e;
}

// out[col] = sum_{P in [Pa, Pb)} w_P B[P][col] for the columns c2, c2 + 1 of
// a thread, from the float-pair B (one 16-byte load per P: hi0 lo0 hi1 lo1)
// and float-pair w, accumulated in float-float: the FP32 pipe does what the
// FP64 pipe (1/64 of its rate) would, at ~2^-46 relative per term, so the
// pass runs at the memory's speed.
__device__ __forceinline__ void jpass_ff_cols(const float4 *__restrict__ B2,
                                              const float2 *__restrict__ w2, int Pa, int Pb,
                                              int64_t npair, int64_t c2,
                                              double *__restrict__ out) {
  float h0 = 0.0f, l0 = 0.0f, h1 = 0.0f, l1 = 0.0f;
  if (c2 + 1 < npair && (npair % 2 == 0)) {
    const float4 *b = B2 + c2 / 2;
    const int64_t st = npair / 2;
    int P = Pa;
    for (; P + 8 <= Pb; P += 8) {
      float4 v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = __ldg(b + (int64_t)(P + k) * st);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const float2 wp = __ldg(w2 + P + k);
        ff_acc(h0, l0, wp.x, wp.y, v[k].x, v[k].y);
        ff_acc(h1, l1, wp.x, wp.y, v[k].z, v[k].w);
      }
    }
    for (; P < Pb; ++P) {
      const float4 v = __ldg(b + (int64_t)P * st);
      const float2 wp = __ldg(w2 + P);
      ff_acc(h0, l0, wp.x, wp.y, v.x, v.y);
      ff_acc(h1, l1, wp.x, wp.y, v.z, v.w);
    }
    out[c2] = (double)h0 + (double)l0;
    out[c2 + 1] = (double)h1 + (double)l1;
  } else {
    const float2 *b = reinterpret_cast<const float2 *>(B2);
    for (int P = Pa; P < Pb; ++P) {
      const float2 wp = __ldg(w2 + P);
      const float2 v0 = __ldg(b + (int64_t)P * npair + c2);
      ff_acc(h0, l0, wp.x, wp.y, v0.x, v0.y);
      if (c2 + 1 < npair) {
        const float2 v1 = __ldg(b + (int64_t)P * npair + c2 + 1);
        ff_acc(h1, l1, wp.x, wp.y, v1.x, v1.y);
      }
    }
    out[c2] = (double)h0 + (double)l0;
    if (c2 + 1 < npair) out[c2 + 1] = (double)h1 + (double)l1;
  }
}

__global__ void __launch_bounds__(256) k_jpass_ff_range(const float4 *__restrict__ B2,
                                                        const float2 *__restrict__ w2, int P0,
                                                        int P1, int64_t npair, int y0,
                                                        double *__restrict__ Jp) {
  const int64_t c2 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 2;
  if (c2 >= npair) return;
  const int per = (P1 - P0 + gridDim.y - 1) / gridDim.y;
  const int Pa = P0 + blockIdx.y * per, Pb = min(P1, Pa + per);
  jpass_ff_cols(B2, w2, Pa, Pb, npair, c2, Jp + (int64_t)(y0 + blockIdx.y) * npair);
}

// B (FP64) -> float pairs (hi, lo), hi = fl(B), lo = fl(B - hi).
__global__ void k_split_ff(const double *__restrict__ B, int64_t count, float2 *__restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const double d = B[i];
  const float h = (float)d;
  out[i] = make_float2(h, (float)(d - (double)h));
}

// Grouped J pass of independent problems in one launch: problem k owns the
// blocks [off[k], off[k + 1]) as xb[k] column blocks times sp[k] aux chunks.
struct JGroup {
  const double *B[kMaxGroup];
  const double *w[kMaxGroup];
  const float4 *B2[kMaxGroup];  // float-pair B and w (ff variant)
  const float2 *w2[kMaxGroup];
  double *Jp[kMaxGroup];
  double *J[kMaxGroup];
  int64_t npair[kMaxGroup];
  int naux[kMaxGroup], sp[kMaxGroup], xb[kMaxGroup], n[kMaxGroup];
  int off[kMaxGroup + 1];
  int nprob;
};

template <bool FF>
__global__ void __launch_bounds__(256) k_jpass64_grp(const __grid_constant__ JGroup g) {
  const int bid = blockIdx.x;
  int k = 0;
  while (k + 1 < g.nprob && bid >= g.off[k + 1]) ++k;
  const int lb = bid - g.off[k], y = lb / g.xb[k], xb = lb % g.xb[k];
  const int64_t npair = g.npair[k];
  const int64_t c2 = ((int64_t)xb * blockDim.x + threadIdx.x) * 2;
  if (c2 >= npair) return;
  const int per = (g.naux[k] + g.sp[k] - 1) / g.sp[k];
  const int Pa = y * per, Pb = min(g.naux[k], Pa + per);
  if (FF)
    jpass_ff_cols(g.B2[k], g.w2[k], Pa, Pb, npair, c2, g.Jp[k] + (int64_t)y * npair);
  else
    jpass64_cols(g.B[k], g.w[k], Pa, Pb, npair, c2, g.Jp[k] + (int64_t)y * npair);
}

__device__ __forceinline__ void unpack_jsum_one(const double *Jp, int nsplit, int64_t npair, int n,
                                                double *J, int64_t i) {
  if (i >= (int64_t)n * n) return;
  const int64_t r = i / n, c = i % n;
  const int64_t hi = r > c ? r : c, lo = r > c ? c : r;
  const int64_t q = hi * (hi + 1) / 2 + lo;
  double s = Jp[q];
  for (int y = 1; y < nsplit; ++y) s += Jp[(int64_t)y * npair + q];
  J[i] = s;
}

__global__ void k_unpack_jsum(const double *Jp, int nsplit, int64_t npair, int n, double *J) {
  unpack_jsum_one(Jp, nsplit, npair, n, J, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

__global__ void k_unpack_jsum_grp(const __grid_constant__ JGroup g) {
  const int k = blockIdx.y;
  unpack_jsum_one(g.Jp[k], g.sp[k], g.npair[k], g.n[k], g.J[k],
                  (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

// aux chunks of the J pass: enough blocks for four per SM, at least 64 P each
int jpass_split(int64_t npair, int naux) {
  const int64_t blocks = (npair / 2 + 256) / 256;
  int sp = (int)std::min<int64_t>(16, (4 * (int64_t)sm_count() + blocks - 1) / blocks);
  sp = std::max(1, std::min(sp, naux / 64));
  return sp;
}

// Packed lower triangle -> full symmetric N x N.
__global__ void k_unpack_sym(const double *Jp, int n, double *J) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)n * n) return;
  const int64_t r = i / n, c = i % n;
  const int64_t hi = r > c ? r : c, lo = r > c ? c : r;
  J[i] = Jp[hi * (hi + 1) / 2 + lo];
}

int jpass_fp64(Df *df, double *J, cudaStream_t s) {
  const int n = df->basis->nbf, naux = df->naux_loc;
  const int64_t npair = df->npair;
  if (!df->B64.p) return BQC_E_INVALID;
  const int sp = jpass_split(npair, naux);
  if (df->Jp.n < (size_t)sp * npair * 8) return BQC_E_INVALID;
  k_jpass64<<<dim3((unsigned)((npair / 2 + 256) / 256), (unsigned)sp), 256, 0, s>>>(
      df->B64.as<double>(), df->w.as<double>(), naux, npair, df->Jp.as<double>());
  BQC_LAUNCH_CHECK();
  k_unpack_jsum<<<(unsigned)(((int64_t)n * n + 255) / 256), 256, 0, s>>>(df->Jp.as<double>(), sp,
                                                                         npair, n, J);
  BQC_LAUNCH_CHECK();
  return BQC_OK;
}


// Packed lower triangle of a symmetric N x N matrix with the off-diagonal
// doubled: D2[mu(mu+1)/2 + nu] = (2 - delta_mu nu) D[mu][nu] (so that
// B_P : D = sum over the packed entries of B_P D2).
__global__ void k_pack_sym2(const double *__restrict__ D, int n, double *__restrict__ D2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)n * (n + 1) / 2) return;
  int mu = (int)((sqrt(8.0 * (double)i + 1.0) - 1.0) * 0.5);
  while ((int64_t)(mu + 1) * (mu + 2) / 2 <= i) ++mu;
  while ((int64_t)mu * (mu + 1) / 2 > i) --mu;
  const int nu = (int)(i - (int64_t)mu * (mu + 1) / 2);
  D2[i] = (mu == nu ? 1.0 : 2.0) * D[(int64_t)mu * n + nu];
}

// w[P] = sum_c B[P][c] D2[c] over the packed FP64 B (one block per P).
__global__ void __launch_bounds__(256) k_bdot(const double *__restrict__ B, int64_t npair,
                                              const double *__restrict__ D2, double *w) {
  const double *b = B + (int64_t)blockIdx.x * npair;
  double s = 0.0;
  for (int64_t c = threadIdx.x; c < npair; c += blockDim.x) s = fma(b[c], D2[c], s);
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) w[blockIdx.x] = red[0];
}

// The packed, off-diagonal-doubled density as float pairs (hi, lo).
__global__ void k_pack_sym2_ff(const double *__restrict__ D, int n, float2 *__restrict__ D2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)n * (n + 1) / 2) return;
  int mu = (int)((sqrt(8.0 * (double)i + 1.0) - 1.0) * 0.5);
  while ((int64_t)(mu + 1) * (mu + 2) / 2 <= i) ++mu;
  while ((int64_t)mu * (mu + 1) / 2 > i) --mu;
  const int nu = (int)(i - (int64_t)mu * (mu + 1) / 2);
  const double v = (mu == nu ? 1.0 : 2.0) * D[(int64_t)mu * n + nu];
  const float h = (float)v;
  D2[i] = make_float2(h, (float)(v - (double)h));
}

// w[P] = sum_c B[P][c] D2[c] from the float pairs of B and D2 in float-float
// arithmetic (one block per P; the block's partial pairs summed in FP64);
// also w as float pairs for the J pass.
__global__ void __launch_bounds__(256) k_bdot_ff(const float2 *__restrict__ B2, int64_t npair,
                                                 const float2 *__restrict__ D2, double *w,
                                                 float2 *w2) {
  const float2 *b = B2 + (int64_t)blockIdx.x * npair;
  float h = 0.0f, l = 0.0f;
  if (npair % 2 == 0) {
    const float4 *b4 = reinterpret_cast<const float4 *>(b);
    const float4 *d4 = reinterpret_cast<const float4 *>(D2);
    for (int64_t c = threadIdx.x; c < npair / 2; c += blockDim.x) {
      const float4 x = __ldg(b4 + c), d = __ldg(d4 + c);
      ff_acc(h, l, d.x, d.y, x.x, x.y);
      ff_acc(h, l, d.z, d.w, x.z, x.w);
    }
  } else {
    for (int64_t c = threadIdx.x; c < npair; c += blockDim.x) {
      const float2 x = __ldg(b + c), d = __ldg(D2 + c);
      ff_acc(h, l, d.x, d.y, x.x, x.y);
    }
  }
  __shared__ double red[256];
  red[threadIdx.x] = (double)h + (double)l;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double v = red[0];
    w[blockIdx.x] = v;
    const float fh = (float)v;
    w2[blockIdx.x] = make_float2(fh, (float)(v - (double)fh));
  }
}

int jff_of_density(Df *df, const double *D, double *D2, double *J, cudaStream_t s) {
  if (df->mode != BQC_DF_STORED || !df->B2f.p || !df->w2f.p) return BQC_E_INVALID;
  const int n = df->basis->nbf;
  float2 *d2 = reinterpret_cast<float2 *>(D2);  // npair doubles hold npair float pairs
  k_pack_sym2_ff<<<(unsigned)((df->npair + 255) / 256), 256, 0, s>>>(D, n, d2);
  BQC_LAUNCH_CHECK();
  k_bdot_ff<<<(unsigned)df->naux_loc, 256, 0, s>>>(df->B2f.as<float2>(), df->npair, d2,
                                                   df->w.as<double>(), df->w2f.as<float2>());
  BQC_LAUNCH_CHECK();
  const int sp = jpass_split(df->npair, df->naux_loc);
  BQC_TRY(jpass_ff_range(df, 0, df->naux_loc, 0, s));
  return jpass_unpack(df, sp, J, s);
}

int jfp64_of_density(Df *df, const double *D, double *D2, double *J, cudaStream_t s) {
  if (df->mode != BQC_DF_STORED || !df->B64.p) return BQC_E_INVALID;
  const int n = df->basis->nbf;
  k_pack_sym2<<<(unsigned)((df->npair + 255) / 256), 256, 0, s>>>(D, n, D2);
  BQC_LAUNCH_CHECK();
  k_bdot<<<(unsigned)df->naux_loc, 256, 0, s>>>(df->B64.as<double>(), df->npair, D2,
                                                df->w.as<double>());
  BQC_LAUNCH_CHECK();
  return jpass_fp64(df, J, s);
}

int jpass_fp64_range(Df *df, int P0, int P1, int y0, cudaStream_t s) {
  const int64_t npair = df->npair;
  const int sp = jpass_split(npair, P1 - P0);
  if (df->Jp.n < (size_t)(y0 + sp) * npair * 8) return BQC_E_INVALID;
  k_jpass64_range<<<dim3((unsigned)((npair / 2 + 256) / 256), (unsigned)sp), 256, 0, s>>>(
      df->B64.as<double>(), df->w.as<double>(), P0, P1, npair, y0, df->Jp.as<double>());
  BQC_LAUNCH_CHECK();
  return BQC_OK;
}

int jpass_ff_setup(Df *df, cudaStream_t s) {
  const int64_t count = (int64_t)df->naux_loc * df->npair;
  BQC_TRY(df->B2f.alloc(df->ctx, (size_t)count * 8));
  BQC_TRY(df->w2f.alloc(df->ctx, (size_t)df->naux_loc * 8));
  k_split_ff<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(df->B64.as<double>(), count,
                                                             df->B2f.as<float2>());
  BQC_LAUNCH_CHECK();
  return BQC_OK;
}

int jpass_ff_range(Df *df, int P0, int P1, int y0, cudaStream_t s) {
  const int64_t npair = df->npair;
  const int sp = jpass_split(npair, P1 - P0);
  if (!df->B2f.p || !df->w2f.p || df->Jp.n < (size_t)(y0 + sp) * npair * 8)
    return BQC_E_INVALID;
  k_jpass_ff_range<<<dim3((unsigned)((npair / 2 + 256) / 256), (unsigned)sp), 256, 0, s>>>(
      df->B2f.as<float4>(), df->w2f.as<float2>(), P0, P1, npair, y0, df->Jp.as<double>());
  BQC_LAUNCH_CHECK();
  return BQC_OK;
}

int jpass_unpack(Df *df, int nslice, double *J, cudaStream_t s) {
  const int n = df->basis->nbf;
  k_unpack_jsum<<<(unsigned)(((int64_t)n * n + 255) / 256), 256, 0, s>>>(df->Jp.as<double>(),
                                                                         nslice, df->npair, n, J);
  BQC_LAUNCH_CHECK();
  return BQC_OK;
}

int group_jpass(Df *const *dfs, double *const *J, int n, cudaStream_t s) {
  if (n <= 0 || n > kMaxGroup) return BQC_E_INVALID;
  JGroup g;
  std::memset(&g, 0, sizeof(g));
  int blocks = 0;
  bool ff = true;
  int64_t nn_max = 0;
  for (int k = 0; k < n; ++k) {
    Df *df = dfs[k];
    if (!df->B64.p) return BQC_E_INVALID;
    const int64_t npair = df->npair;
    const int naux = df->naux_loc, nb = df->basis->nbf;
    const int sp = jpass_split(npair, naux);
    if (df->Jp.n < (size_t)sp * npair * 8) return BQC_E_INVALID;
    g.B[k] = df->B64.as<double>();
    g.w[k] = df->w.as<double>();
    g.B2[k] = df->B2f.as<float4>();
    g.w2[k] = df->w2f.as<float2>();
    ff = ff && df->B2f.p && df->w2f.p;
    g.Jp[k] = df->Jp.as<double>();
    g.J[k] = J[k];
    g.npair[k] = npair;
    g.naux[k] = naux;
    g.sp[k] = sp;
    g.xb[k] = (int)((npair / 2 + 256) / 256);
    g.n[k] = nb;
    g.off[k] = blocks;
    blocks += g.xb[k] * sp;
    nn_max = std::max(nn_max, (int64_t)nb * nb);
  }
  g.off[n] = blocks;
  g.nprob = n;
  if (ff)
    k_jpass64_grp<true><<<(unsigned)blocks, 256, 0, s>>>(g);
  else
    k_jpass64_grp<false><<<(unsigned)blocks, 256, 0, s>>>(g);
  BQC_LAUNCH_CHECK();
  k_unpack_jsum_grp<<<dim3((unsigned)((nn_max + 255) / 256), (unsigned)n), 256, 0, s>>>(g);
  BQC_LAUNCH_CHECK();
  return BQC_OK;
}

int jk_fp64_stored(Df *df, const double *C, double *J, double *K, cudaStream_t s) {
  const Basis *b = df->basis;
  const int n = b->nbf, naux = df->naux_loc, no = b->nocc;
  const int64_t npair = df->npair;
  double *X = df->X64.as<double>();
  df->mark(0, s);
  df->mark(1, s);
  // X_P = Bsym_P C  (batched over P)
  Gemm64Args g;
  g.M = n;
  g.N = no;
  g.K1 = 1;
  g.K2 = n;
  g.A = df->B64.as<double>();
  g.bsA = npair;
  g.B = C;
  g.ldb = no;
  g.C = X;
  g.ldc = no;
  g.bsC = (int64_t)n * no;
  g.batch = naux;
  BQC_TRY(launch_gemm64(kASym, false, g, s));
  k_wdot<<<naux, 256, 0, s>>>(X, C, (int64_t)n * no, df->w.as<double>());
  BQC_LAUNCH_CHECK();
  df->mark(2, s);
  // J pass
  BQC_TRY(jpass_fp64(df, J, s));
  df->mark(3, s);
  // K = sum_{P,i} X_P,mu i X_P,nu i
  Gemm64Args k;
  k.M = n;
  k.N = n;
  k.K1 = naux;
  k.K2 = no;
  k.A = X;
  k.lda = no;
  k.sA1 = (int64_t)n * no;
  k.B = X;
  k.ldb = no;
  k.sB1 = (int64_t)n * no;
  k.C = K;
  k.ldc = n;
  k.lower_only = 1;
  k.mirror = 1;
  BQC_TRY(launch_gemm64(kAN, true, k, s));
  df->mark(4, s);
  return BQC_OK;
}

size_t df_stored_bytes(int n, int naux, int nocc, int shadow) {
  const size_t npair = (size_t)n * (n + 1) / 2;
  size_t b = (size_t)naux * naux * 8 + (size_t)naux * npair * 8;  // L, B64
  b += (size_t)naux * n * nocc * 8;                                // X64
  b += (size_t)jpass_split((int64_t)npair, naux) * npair * 8 + (size_t)naux * 8 * 2;
  if (shadow == BQC_SHADOW_TF32 || shadow == BQC_SHADOW_F16)
    b += mixed_workspace_bytes(n, naux, nocc, shadow);
  if (shadow == BQC_SHADOW_F16) {  // float-pair B and w of the J pass, the pieces' J partials
    b += (size_t)naux * npair * 8 + (size_t)naux * 8;
    const int np = std::min(kJPieces, std::max(naux, 1));
    for (int k = 0; k < np; ++k)
      b += (size_t)jpass_split((int64_t)npair, (int)((int64_t)naux * (k + 1) / np) -
                                                   (int)((int64_t)naux * k / np)) *
           npair * 8;
  }
  return b;
}

}  // namespace bqc

using namespace bqc;

extern "C" {

int bqc_df_coulomb(bqc_df *df, const double *D_dev, double *J_dev, int variant,
                   bqc_stream_t stream) {
  if (!df || !D_dev || !J_dev || (variant != BQC_COULOMB_FP64 && variant != BQC_COULOMB_FF))
    return BQC_E_INVALID;
  if (df->mode != BQC_DF_STORED || !df->B64.p) {
    set_error("bqc_df_coulomb needs a stored handle", __FILE__, __LINE__);
    return BQC_E_UNSUPPORTED;
  }
  if (variant == BQC_COULOMB_FF && !df->B2f.p) {
    set_error("the float-float Coulomb pass needs a handle built with BQC_SHADOW_F16",
              __FILE__, __LINE__);
    return BQC_E_UNSUPPORTED;
  }
  BQC_CUDA_TRY(cudaSetDevice(df->ctx->device));
  if (df->D2.n < (size_t)df->npair * 8) BQC_TRY(df->D2.alloc(df->ctx, (size_t)df->npair * 8));
  const int need = jpass_split(df->npair, df->naux_loc);
  if (df->Jp.n < (size_t)need * df->npair * 8)
    BQC_TRY(df->Jp.alloc(df->ctx, (size_t)need * df->npair * 8));
  cudaStream_t s = (cudaStream_t)stream;
  return variant == BQC_COULOMB_FF ? jff_of_density(df, D_dev, df->D2.as<double>(), J_dev, s)
                                   : jfp64_of_density(df, D_dev, df->D2.as<double>(), J_dev, s);
}

int bqc_df_build(bqc_ctx *ctx, const bqc_basis *basis, const bqc_df_opts *opts,
                 bqc_stream_t stream, bqc_df **out) {
  if (!ctx || !basis || !out) return BQC_E_INVALID;
  *out = nullptr;
  NvtxRange nv("bqc_df_build");
  BQC_CUDA_TRY(cudaSetDevice(ctx->device));
  bqc_df_opts o;
  o.mode = BQC_DF_STORED;
  o.schwarz = -1.0;
  o.aux_block = 1024;
  o.keep_fp32 = 1;
  o.hbm_limit = 0;
  o.aux_begin = 0;
  o.aux_end = 0;
  if (opts) o = *opts;
  cudaStream_t s = (cudaStream_t)stream;
  const int n = basis->nbf, naux = basis->naux, no = basis->nocc;
  const int64_t npair = (int64_t)n * (n + 1) / 2;
  int mode = o.mode;
  if (mode == BQC_DF_AUTO) {
    size_t limit = o.hbm_limit;
    if (!limit) {
      size_t fr = 0, tot = 0;
      BQC_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
      limit = (size_t)(fr * 0.9);
    }
    mode = df_stored_bytes(n, naux, no, o.keep_fp32) <= limit ? BQC_DF_STORED : BQC_DF_DIRECT;
  }
  if (mode != BQC_DF_STORED && mode != BQC_DF_DIRECT && mode != BQC_DF_NONE) return BQC_E_INVALID;
  if (o.keep_fp32 < BQC_SHADOW_NONE || o.keep_fp32 > BQC_SHADOW_F16) return BQC_E_INVALID;
  // aux shard [P0, P1) (stored mode): both 0 selects every aux function
  int P0 = o.aux_begin, P1 = o.aux_end;
  if (P0 == 0 && P1 == 0) P1 = naux;
  if (P0 < 0 || P1 > naux || P0 >= P1) {
    set_error("bqc_df_build: aux shard outside [0, Naux) or empty", __FILE__, __LINE__);
    return BQC_E_INVALID;
  }
  const bool shard = P0 != 0 || P1 != naux;
  if (shard && mode == BQC_DF_NONE) return BQC_E_INVALID;
  if (shard && mode != BQC_DF_STORED) {
    set_error("bqc_df_build: aux shards are a stored-mode feature", __FILE__, __LINE__);
    return BQC_E_UNSUPPORTED;
  }
  if (o.schwarz < 0.0) o.schwarz = (mode == BQC_DF_DIRECT) ? 1e-10 : 1e-12;
  if (o.aux_block <= 0) o.aux_block = 1024;
  bqc_df *df = new (std::nothrow) bqc_df();
  if (!df) return BQC_E_OOM;
  df->ctx = ctx;
  df->basis = basis;
  df->mode = mode;
  df->npair = npair;
  df->opts = o;
  df->p0 = P0;
  df->naux_loc = P1 - P0;
  auto fail = [&](int st) {
    cudaStreamSynchronize(s);
    delete df;
    return st;
  };
  int st;
  if (mode == BQC_DF_NONE) {  // conventional four-centre J/K: no auxiliary tensor
    if ((st = jk4c_setup(df, s)) != BQC_OK) return fail(st);
    if ((st = ctx->check_flag(s)) != BQC_OK) return fail(st);
    *out = df;
    return BQC_OK;
  }
  // metric and its Cholesky factor
  if ((st = df->L.alloc(ctx, (size_t)naux * naux * 8)) != BQC_OK) return fail(st);
  if ((st = launch_int2c(basis, df->L.as<double>(), s)) != BQC_OK) return fail(st);
  if ((st = df->Vdiag.alloc(ctx, (size_t)naux * naux * 8)) != BQC_OK) return fail(st);
  if (cudaMemcpyAsync(df->Vdiag.p, df->L.p, (size_t)naux * naux * 8, cudaMemcpyDeviceToDevice,
                      s) != cudaSuccess)
    return fail(BQC_E_CUDA);
  if ((st = cholesky_lower(ctx, df->L.as<double>(), naux, s)) != BQC_OK) return fail(st);
  if ((st = ctx->check_flag(s)) != BQC_OK) return fail(st);
  if ((st = eri3c_plan(basis, o.schwarz, df->Vdiag.as<double>(), s, &df->plan)) != BQC_OK)
    return fail(st);
  if ((st = df->w.alloc(ctx, (size_t)naux * 8)) != BQC_OK) return fail(st);
  if (mode == BQC_DF_STORED) {
    df->Vdiag.release();  // metric only needed for the screening plan
    if (!shard) {
      if ((st = df->B64.alloc(ctx, (size_t)naux * npair * 8)) != BQC_OK) return fail(st);
      if (cudaMemsetAsync(df->B64.p, 0, (size_t)naux * npair * 8, s) != cudaSuccess)
        return fail(BQC_E_CUDA);
      if ((st = launch_eri3c(basis, &df->plan, 0, naux, df->B64.as<double>(), npair, s)) !=
          BQC_OK)
        return fail(st);
      if ((st = trsm_lower_left(ctx, df->L.as<double>(), naux, df->B64.as<double>(), npair,
                                npair, s)) != BQC_OK)
        return fail(st);
    } else {
      // B_P for P in [P0, P1) depends on (Q|mu nu) for every Q <= P (the
      // triangular solve couples them): solve rows [0, P1) with the leading
      // P1 x P1 block of L and keep the shard's rows
      DBuf raw, Lb;
      if ((st = raw.alloc(ctx, (size_t)P1 * npair * 8)) != BQC_OK) return fail(st);
      if (cudaMemsetAsync(raw.p, 0, (size_t)P1 * npair * 8, s) != cudaSuccess)
        return fail(BQC_E_CUDA);
      if ((st = launch_eri3c(basis, &df->plan, 0, P1, raw.as<double>(), npair, s)) != BQC_OK)
        return fail(st);
      if ((st = Lb.alloc(ctx, (size_t)P1 * P1 * 8)) != BQC_OK) return fail(st);
      if (cudaMemcpy2DAsync(Lb.p, (size_t)P1 * 8, df->L.p, (size_t)naux * 8, (size_t)P1 * 8, P1,
                            cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return fail(BQC_E_CUDA);
      if ((st = trsm_lower_left(ctx, Lb.as<double>(), P1, raw.as<double>(), npair, npair, s)) !=
          BQC_OK)
        return fail(st);
      if ((st = df->B64.alloc(ctx, (size_t)(P1 - P0) * npair * 8)) != BQC_OK) return fail(st);
      if (cudaMemcpyAsync(df->B64.p, raw.as<double>() + (size_t)P0 * npair,
                          (size_t)(P1 - P0) * npair * 8, cudaMemcpyDeviceToDevice,
                          s) != cudaSuccess)
        return fail(BQC_E_CUDA);
      if (cudaStreamSynchronize(s) != cudaSuccess) return fail(BQC_E_CUDA);
    }
    const int nl = df->naux_loc;
    if ((st = df->X64.alloc(ctx, (size_t)nl * n * no * 8)) != BQC_OK) return fail(st);
    if ((st = df->Jp.alloc(ctx, (size_t)jpass_split(npair, nl) * npair * 8)) != BQC_OK)
      return fail(st);
    if (o.keep_fp32 != BQC_SHADOW_NONE)
      if ((st = mixed_setup(df, o.keep_fp32, s)) != BQC_OK) return fail(st);
  } else {
    if ((st = direct_setup(df, s)) != BQC_OK) return fail(st);
  }
  if ((st = ctx->check_flag(s)) != BQC_OK) return fail(st);
  *out = df;
  return BQC_OK;
}

int bqc_df_destroy(bqc_df *df) {
  if (!df) return BQC_E_INVALID;
  cudaSetDevice(df->ctx->device);
  cudaDeviceSynchronize();
  delete df;
  return BQC_OK;
}

int bqc_df_info(const bqc_df *df, int *mode, size_t *bytes) {
  if (!df) return BQC_E_INVALID;
  if (mode) *mode = df->mode;
  if (bytes) *bytes = df->device_bytes();
  return BQC_OK;
}

int bqc_df_shard(const bqc_df *df, int *aux_begin, int *aux_end) {
  if (!df) return BQC_E_INVALID;
  if (aux_begin) *aux_begin = df->p0;
  if (aux_end) *aux_end = df->p0 + df->naux_loc;
  return BQC_OK;
}

int bqc_df_screening(const bqc_df *df, int64_t *candidates, int64_t *survivors) {
  if (!df) return BQC_E_INVALID;
  if (candidates) *candidates = df->plan.candidates;
  if (survivors) *survivors = df->plan.survivors;
  return BQC_OK;
}

int bqc_df_copy(const bqc_df *df, int which, double *out, bqc_stream_t stream) {
  if (!df || !out) return BQC_E_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  const int naux = df->basis->naux;
  if (which == 0) {
    if (df->mode != BQC_DF_STORED) return BQC_E_INVALID;
    BQC_CUDA_TRY(cudaMemcpyAsync(out, df->B64.p, (size_t)df->naux_loc * df->npair * 8,
                                 cudaMemcpyDeviceToDevice, s));
  } else if (which == 1) {
    if (!df->L.p) return BQC_E_INVALID;
    BQC_CUDA_TRY(
        cudaMemcpyAsync(out, df->L.p, (size_t)naux * naux * 8, cudaMemcpyDeviceToDevice, s));
  } else {
    return BQC_E_INVALID;
  }
  return BQC_OK;
}

int bqc_int3c_screened(const bqc_df *df, int p0, int p1, int variant, double *out,
                       bqc_stream_t stream) {
  if (!df || !out || variant < 0 || variant > 2 || df->mode == BQC_DF_NONE)
    return BQC_E_INVALID;
  if (p0 < 0 || p1 > df->basis->naux || p0 >= p1) return BQC_E_INVALID;
  BQC_CUDA_TRY(cudaSetDevice(df->ctx->device));
  return launch_eri3c_variant(df->basis, &df->plan, p0, p1, out, df->npair, variant,
                              (cudaStream_t)stream);
}

int bqc_df_timing(bqc_df *df, int enable) {
  if (!df) return BQC_E_INVALID;
  if (enable) {
    for (auto &e : df->ev)
      if (!e) BQC_CUDA_TRY(cudaEventCreate(&e));
  }
  df->timing = enable != 0;
  return BQC_OK;
}

int bqc_df_phase_ms(bqc_df *df, float *ms, int n) {
  if (!df || !ms || n <= 0) return BQC_E_INVALID;
  if (!df->timed) return BQC_E_NOT_READY;
  BQC_CUDA_TRY(cudaEventSynchronize(df->ev[4]));
  float t[4] = {0, 0, 0, 0};
  BQC_CUDA_TRY(cudaEventElapsedTime(&t[0], df->ev[1], df->ev[2]));
  BQC_CUDA_TRY(cudaEventElapsedTime(&t[3], df->ev[0], df->ev[1]));
  if (df->mode == BQC_DF_STORED && df->side && df->last_mixed) {
    // mixed stored build: J (side stream, ev[j_from] -> ev5) runs beside the
    // tensor-core passes; K is the SYRK (ev2 -> ev3)
    BQC_CUDA_TRY(cudaEventElapsedTime(&t[1], df->ev[df->j_from], df->ev[5]));
    BQC_CUDA_TRY(cudaEventElapsedTime(&t[2], df->ev[2], df->ev[3]));
  } else {
    BQC_CUDA_TRY(cudaEventElapsedTime(&t[1], df->ev[2], df->ev[3]));
    BQC_CUDA_TRY(cudaEventElapsedTime(&t[2], df->ev[3], df->ev[4]));
  }
  for (int i = 0; i < n && i < 4; ++i) ms[i] = t[i];
  return BQC_OK;
}

int bqc_jk(bqc_df *df, const double *C, int nocc, int prec, double *J, double *K,
           bqc_stream_t stream) {
  if (!df || !C || !J || !K) return BQC_E_INVALID;
  if (nocc != df->basis->nocc) return BQC_E_INVALID;
  NvtxRange nv(prec == BQC_PREC_FP64 ? "bqc_jk fp64" : "bqc_jk mixed");
  cudaStream_t s = (cudaStream_t)stream;
  if (df->timing) df->timed = true;
  df->last_mixed = prec != BQC_PREC_FP64;
  if (df->mode == BQC_DF_DIRECT) return jk_direct(df, C, prec, J, K, s);
  if (df->mode == BQC_DF_NONE) return jk_4c(df, C, prec, J, K, s);
  if (prec == BQC_PREC_FP64) return jk_fp64_stored(df, C, J, K, s);
  if (prec == BQC_PREC_MIXED_TF32 || prec == BQC_PREC_MIXED_TF32X3 ||
      prec == BQC_PREC_MIXED_F16X3) {
    if (!df->mixed) {
      set_error("mixed precision needs split shadows (bqc_df_opts.keep_fp32)", __FILE__, __LINE__);
      return BQC_E_INVALID;
    }
    return jk_mixed_stored(df, C, prec, J, K, s);
  }
  return BQC_E_INVALID;
}

int bqc_jk_host(bqc_df *df, const double *C, int nocc, int prec, double *J, double *K,
                bqc_stream_t stream) {
  if (!df || !C || !J || !K) return BQC_E_INVALID;
  if (nocc != df->basis->nocc) return BQC_E_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  const int n = df->basis->nbf;
  // a NaN or an infinity in the orbitals would poison every element of J
  // and K: refuse it on the host, before anything is copied or launched
  for (size_t i = 0, e = (size_t)n * nocc; i < e; ++i)
    if (!std::isfinite(C[i])) {
      char msg[96];
      std::snprintf(msg, sizeof(msg), "bqc_jk_host: C_occ[%zu] is not finite", i);
      set_error(msg, __FILE__, __LINE__);
      return BQC_E_INVALID;
    }
  if (!df->host_io.p) {
    BQC_TRY(df->host_io.alloc(df->ctx, ((size_t)n * nocc + 2 * (size_t)n * n) * 8));
  }
  double *dC = df->host_io.as<double>();
  double *dJ = dC + (size_t)n * nocc, *dK = dJ + (size_t)n * n;
  BQC_CUDA_TRY(cudaMemcpyAsync(dC, C, (size_t)n * nocc * 8, cudaMemcpyHostToDevice, s));
  BQC_TRY(bqc_jk(df, dC, nocc, prec, dJ, dK, stream));
  BQC_CUDA_TRY(cudaMemcpyAsync(J, dJ, (size_t)n * n * 8, cudaMemcpyDeviceToHost, s));
  BQC_CUDA_TRY(cudaMemcpyAsync(K, dK, (size_t)n * n * 8, cudaMemcpyDeviceToHost, s));
  BQC_CUDA_TRY(cudaStreamSynchronize(s));
  return df->ctx->check_flag(s);
}

}  // extern "C"
