// Mixed-precision Fock build on the 5th-generation tensor cores (tcgen05).
//
// The two passes over the CD-ERIs that the paper describes for the Coulomb
// and exchange matrices (Sec. 2.2) become, with B held as a TF32-rounded
// full-square shadow B32[P][mu][nu]:
//   X pass  X[(P,mu)][i] = sum_nu B32[(P,mu)][nu] C[nu][i]       (one GEMM,
//           M = Naux*N, N = nocc, K = N) with the Coulomb contraction
//           w_P = sum_{mu,i} X[(P,mu)][i] C[mu][i] fused into the epilogue;
//   SYRK    K[mu][nu] = sum_{P,i} X[P][mu][i] X[P][nu][i], lower tiles only,
//           split over aux chunks whose FP32 partials are summed in FP64;
//   J pass  J[mu][nu<=mu] = sum_P w_P B32[P][mu][nu]  (HBM-bound stream).
// Tensor-core kernels: TMA (128-byte swizzle) -> shared memory ring ->
// tcgen05.mma kind::tf32 issued by one thread -> FP32 accumulators in TMEM
// -> tcgen05.ld epilogue.  Warp 0 produces, warp 1 issues MMAs, all four
// warps drain TMEM.  Every mbarrier wait is bounded; on timeout the kernel
// records an error code in the context's device flag and skips its work.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "bqc_internal.h"
#include "df_internal.h"
#include "tc_util.cuh"

namespace bqc {

using namespace tc;

// --------------------------------------------------------- tensor maps ---

static PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}

// fp32 tensor map, rank 2 or 3, 128-byte swizzle; dims/box innermost first;
// strides in bytes for dims 1.. (rank-1 entries).
int make_tmap_f32(CUtensorMap *map, const void *base, int rank, const uint64_t *dims,
                  const uint64_t *strides_bytes, const uint32_t *box) {
  auto enc = get_encode();
  if (!enc) {
    set_error("cuTensorMapEncodeTiled unavailable", __FILE__, __LINE__);
    return BQC_E_CUDA;
  }
  cuuint32_t estr[3] = {1, 1, 1};
  cuuint64_t d[3], s[2];
  cuuint32_t b[3];
  for (int i = 0; i < rank; ++i) {
    d[i] = dims[i];
    b[i] = box[i];
  }
  for (int i = 0; i < rank - 1; ++i) s[i] = strides_bytes[i];
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, const_cast<void *>(base),
                   d, s, b, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed", __FILE__, __LINE__);
    return BQC_E_CUDA;
  }
  return BQC_OK;
}

__device__ __forceinline__ uint8_t *align1024(uint8_t *p) {
  const uint32_t a = smem_u32(p);
  return p + ((1024 - (a & 1023)) & 1023);
}

// ------------------------------------------------------------- X pass ----

__device__ __forceinline__ float tf32r(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

struct XpassParams {
  int64_t rows;      // Naux * N
  int n;             // N (rows per aux function)
  int ldx;           // nocc_pad (row length of X32 and Cf)
  int col0;          // first C column of this CTA's column group (blockIdx.y * cols)
  int cols;          // columns per CTA (<= 512, multiple of 32)
  int sub_n;         // columns per MMA (<= 256, multiple of 16)
  int n_sub;         // MMAs per k-step
  int kblocks;       // ceil(K / 32)
  int stages;
  float *X;          // rows x ldx
  const float *Cf;   // N x ldx, fp32 C_occ
  double *wrow;      // [ncg][rows]
  int tmem_cols;     // power of two >= cols
  int *flag;
};

constexpr int kBM = 128;
constexpr uint32_t kAStage = kBM * 128;  // 128 rows x 128 bytes

__global__ void __launch_bounds__(128, 1)
    k_xpass_tf32(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                 const XpassParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = align1024(smem_raw);
  const uint32_t bstage = (uint32_t)p.cols * 128;
  const uint32_t stage_bytes = kAStage + bstage;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + (size_t)p.stages * stage_bytes);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2 * p.stages + 1);
  const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * p.stages,
                 done = full0 + 16 * p.stages;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    prefetch_tmap(&mapA);
    prefetch_tmap(&mapB);
    for (int s = 0; s < p.stages; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(done, 1);
    fence_barrier_init();
  }
  if (warp == 0) tmem_alloc(smem_u32(tslot), p.tmem_cols);
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;
  const int64_t m0 = (int64_t)blockIdx.x * kBM;
  const int cg = blockIdx.y;
  const uint32_t sbase = smem_u32(smem);
  bool ok = true;
  if (warp == 0 && lane == 0) {
    for (int kb = 0; kb < p.kblocks && ok; ++kb) {
      const int s = kb % p.stages;
      if (kb >= p.stages) ok = mbar_wait(empty0 + 8 * s, ((kb / p.stages) - 1) & 1, p.flag, 11);
      if (!ok) break;
      const uint32_t a = sbase + s * stage_bytes, b = a + kAStage;
      mbar_arrive_expect_tx(full0 + 8 * s, stage_bytes);
      tma_load_2d(a, &mapA, full0 + 8 * s, kb * 32, (int)m0);
      for (int j = 0; j < p.n_sub; ++j)
        tma_load_2d(b + j * p.sub_n * 128, &mapB, full0 + 8 * s, kb * 32,
                    p.col0 + cg * p.cols + j * p.sub_n);
    }
  } else if (warp == 1 && lane == 0) {
    const uint32_t idesc = idesc_tf32(kBM, p.sub_n);
    for (int kb = 0; kb < p.kblocks && ok; ++kb) {
      const int s = kb % p.stages;
      ok = mbar_wait(full0 + 8 * s, (kb / p.stages) & 1, p.flag, 12);
      if (!ok) break;
      tc_fence_after();
      const uint32_t a = sbase + s * stage_bytes, b = a + kAStage;
#pragma unroll
      for (int k4 = 0; k4 < 4; ++k4) {
        const uint64_t ad = sdesc_sw128(a + k4 * 32);
        for (int j = 0; j < p.n_sub; ++j) {
          const uint64_t bd = sdesc_sw128(b + j * p.sub_n * 128 + k4 * 32);
          mma_tf32(tbase + j * p.sub_n, ad, bd, idesc, (kb | k4) != 0);
        }
      }
      mma_commit(empty0 + 8 * s);
    }
    mma_commit(done);
  }
  __syncwarp();
  // epilogue: thread = accumulator row
  ok = mbar_wait(done, 0, p.flag, 13);
  __syncwarp();
  tc_fence_after();
  const int64_t row = m0 + warp * 32 + lane;
  const bool valid = ok && row < p.rows;
  const int mu = (int)(row % p.n);
  double wsum = 0.0;
  float wpart = 0.0f;
  const int cbase = cg * p.cols;
  for (int c = 0; c < p.n_sub * p.sub_n; c += 16) {
    float v[16];
    tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16) + c, v);
    if (valid) {
      float *xr = p.X + row * p.ldx + cbase + c;
      const float *cr = p.Cf + (int64_t)mu * p.ldx + cbase + c;
#pragma unroll
      for (int q = 0; q < 16; q += 4) {
        // stored TF32-rounded (round to nearest): the SYRK operand is exact TF32
        *reinterpret_cast<float4 *>(xr + q) =
            make_float4(tf32r(v[q]), tf32r(v[q + 1]), tf32r(v[q + 2]), tf32r(v[q + 3]));
        const float4 cc = *reinterpret_cast<const float4 *>(cr + q);
        wpart = fmaf(v[q], cc.x, wpart);
        wpart = fmaf(v[q + 1], cc.y, wpart);
        wpart = fmaf(v[q + 2], cc.z, wpart);
        wpart = fmaf(v[q + 3], cc.w, wpart);
      }
    }
    if ((c & 127) == 112) {  // fold every 128 columns into FP64
      wsum += wpart;
      wpart = 0.0f;
    }
  }
  wsum += wpart;
  if (valid) p.wrow[(int64_t)cg * p.rows + row] = wsum;
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tbase, p.tmem_cols);
}

// w[P] = sum_cg sum_mu wrow[cg][P*N + mu]; also the fp32 copy for the J pass.
__global__ void __launch_bounds__(256) k_wreduce(const double *wrow, int64_t rows, int ncg, int n,
                                                 double *w, float *w32) {
  const int P = blockIdx.x;
  double s = 0.0;
  for (int g = 0; g < ncg; ++g)
    for (int m = threadIdx.x; m < n; m += blockDim.x) s += wrow[g * rows + (int64_t)P * n + m];
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    w[P] = red[0];
    w32[P] = (float)red[0];
  }
}

// ---------------------------------------------------------------- SYRK ---

struct SyrkParams {
  int n, ldx, naux;
  int ntile, ntri;
  int p_per_chunk;
  int nib;     // ldx / 32
  int stages;
  float *part; // [chunk][ntri][128][128]
  int *flag;
};

__global__ void __launch_bounds__(128, 1)
    k_syrk_tf32(const __grid_constant__ CUtensorMap mapX, const SyrkParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = align1024(smem_raw);
  constexpr uint32_t stage_bytes = 2 * kAStage;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + (size_t)p.stages * stage_bytes);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2 * p.stages + 1);
  const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * p.stages,
                 done = full0 + 16 * p.stages;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.x, chunk = blockIdx.y;
  int tm = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
  while ((tm + 1) * (tm + 2) / 2 <= t) ++tm;
  while (tm * (tm + 1) / 2 > t) --tm;
  const int tn = t - tm * (tm + 1) / 2;
  const int P0 = chunk * p.p_per_chunk;
  const int P1 = min(p.naux, P0 + p.p_per_chunk);
  const int kblocks = max(0, P1 - P0) * p.nib;
  if (threadIdx.x == 0) {
    prefetch_tmap(&mapX);
    for (int s = 0; s < p.stages; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(done, 1);
    fence_barrier_init();
  }
  if (warp == 0) tmem_alloc(smem_u32(tslot), 128);
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;
  const uint32_t sbase = smem_u32(smem);
  bool ok = true;
  if (warp == 0 && lane == 0) {
    for (int kb = 0; kb < kblocks && ok; ++kb) {
      const int s = kb % p.stages;
      if (kb >= p.stages) ok = mbar_wait(empty0 + 8 * s, ((kb / p.stages) - 1) & 1, p.flag, 21);
      if (!ok) break;
      const int P = P0 + kb / p.nib, i0 = (kb % p.nib) * 32;
      const uint32_t a = sbase + s * stage_bytes, b = a + kAStage;
      mbar_arrive_expect_tx(full0 + 8 * s, stage_bytes);
      tma_load_3d(a, &mapX, full0 + 8 * s, i0, tm * kBM, P);
      tma_load_3d(b, &mapX, full0 + 8 * s, i0, tn * kBM, P);
    }
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t idesc = idesc_tf32(kBM, kBM);
    for (int kb = 0; kb < kblocks && ok; ++kb) {
      const int s = kb % p.stages;
      ok = mbar_wait(full0 + 8 * s, (kb / p.stages) & 1, p.flag, 22);
      if (!ok) break;
      tc_fence_after();
      const uint32_t a = sbase + s * stage_bytes, b = a + kAStage;
#pragma unroll
      for (int k4 = 0; k4 < 4; ++k4)
        mma_tf32(tbase, sdesc_sw128(a + k4 * 32), sdesc_sw128(b + k4 * 32), idesc,
                 (kb | k4) != 0);
      mma_commit(empty0 + 8 * s);
    }
    mma_commit(done);
  }
  __syncwarp();
  if (kblocks > 0) ok = mbar_wait(done, 0, p.flag, 23);
  __syncwarp();
  tc_fence_after();
  const int r = warp * 32 + lane;
  float *dst = p.part + (((int64_t)chunk * p.ntri + t) * kBM + r) * kBM;
  for (int c = 0; c < kBM; c += 16) {
    float v[16];
    tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16) + c, v);
    if (kblocks == 0 || !ok) {
#pragma unroll
      for (int q = 0; q < 16; ++q) v[q] = 0.0f;
    }
#pragma unroll
    for (int q = 0; q < 16; q += 4)
      *reinterpret_cast<float4 *>(dst + c + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tbase, 128);
}

// K = sum over chunks of the partial tiles, in FP64, symmetric.  One block
// per (lower tile, 32-row strip): sums into shared memory, writes the strip
// and its mirror image coalesced.
__global__ void __launch_bounds__(256) k_syrk_reduce(const float *part, int nchunk, int ntri,
                                                     int n, double *K) {
  __shared__ double strip[32][kBM + 1];
  const int t = blockIdx.x, sr = blockIdx.y;  // strip of 32 rows
  int tm = 0;
  while ((tm + 1) * (tm + 2) / 2 <= t) ++tm;
  const int tn = t - tm * (tm + 1) / 2;
  for (int e = threadIdx.x; e < 32 * kBM; e += blockDim.x) {
    const int rr = e / kBM, c = e % kBM;
    const int r = sr * 32 + rr;
    double s = 0.0;
    for (int ch = 0; ch < nchunk; ++ch)
      s += part[(((int64_t)ch * ntri + t) * kBM + r) * kBM + c];
    strip[rr][c] = s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 32 * kBM; e += blockDim.x) {
    const int rr = e / kBM, c = e % kBM;
    const int mu = tm * kBM + sr * 32 + rr, nu = tn * kBM + c;
    if (mu < n && nu < n && (tm != tn || nu <= mu)) K[(int64_t)mu * n + nu] = strip[rr][c];
  }
  // mirror: K[nu][mu] for nu in the tn tile, mu in this strip
  for (int e = threadIdx.x; e < 32 * kBM; e += blockDim.x) {
    const int c = e / 32, rr = e % 32;
    const int mu = tm * kBM + sr * 32 + rr, nu = tn * kBM + c;
    if (mu < n && nu < n && (tm != tn || nu < mu)) K[(int64_t)nu * n + mu] = strip[rr][c];
  }
}

// -------------------------------------------------------------- J pass ---

// J[mu][nu <= mu] = sum_P w_P B32[P][mu][nu] into packed FP64.  Block b owns
// rows b and N-1-b (balanced work); a thread owns 4 consecutive columns of
// one row and streams every P (float4 loads, FP32 partial sums over 64 P,
// folded into FP64).
__global__ void __launch_bounds__(512) k_jpass_tf32(const float *__restrict__ B32,
                                                    const float *__restrict__ w32, int naux, int n,
                                                    int ld, double *__restrict__ Jp) {
  const int b = blockIdx.x;
  const int r1 = b, r2 = n - 1 - b;
  const int c1 = r1 / 4 + 1;
  const int c2 = (r2 != r1) ? r2 / 4 + 1 : 0;
  const int64_t nn = (int64_t)n * ld;
  for (int it = threadIdx.x; it < c1 + c2; it += blockDim.x) {
  const int row = it < c1 ? r1 : r2;
  const int q = it < c1 ? it : it - c1;
  const float *src = B32 + (int64_t)row * ld + 4 * q;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int P0 = 0; P0 < naux; P0 += 64) {
    const int P1 = min(naux, P0 + 64);
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 8
    for (int P = P0; P < P1; ++P) {
      const float4 v = __ldg(reinterpret_cast<const float4 *>(src + P * nn));
      const float wp = __ldg(w32 + P);
      a.x = fmaf(wp, v.x, a.x);
      a.y = fmaf(wp, v.y, a.y);
      a.z = fmaf(wp, v.z, a.z);
      a.w = fmaf(wp, v.w, a.w);
    }
    acc[0] += a.x;
    acc[1] += a.y;
    acc[2] += a.z;
    acc[3] += a.w;
  }
  const int64_t base = (int64_t)row * (row + 1) / 2;
  for (int k = 0; k < 4; ++k) {
    const int col = 4 * q + k;
    if (col <= row) Jp[base + col] = acc[k];
  }
  }
}

__global__ void k_unpack_sym2(const double *Jp, int n, double *J) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)n * n) return;
  const int64_t r = i / n, c = i % n;
  const int64_t hi = r > c ? r : c, lo = r > c ? c : r;
  J[i] = Jp[hi * (hi + 1) / 2 + lo];
}

// Ct[i][nu] = tf32(C[nu][i]) (zero padded to ldx x ld), Cf[mu][i] = fp32 C.
__global__ void k_prep_c(const double *C, int n, int nocc, int ld, int ldx, float *Ct,
                         float *Cf) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t tot = (int64_t)ldx * ld;
  if (i < tot) {
    const int oi = (int)(i / ld), nu = (int)(i % ld);
    float v = 0.0f;
    if (oi < nocc && nu < n) {
      uint32_t r;
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"((float)C[(int64_t)nu * nocc + oi]));
      v = __uint_as_float(r);
    }
    Ct[i] = v;
  }
  if (i < (int64_t)n * ldx) {
    const int mu = (int)(i / ldx), oi = (int)(i % ldx);
    Cf[i] = oi < nocc ? (float)C[(int64_t)mu * nocc + oi] : 0.0f;
  }
}

// ------------------------------------------------------------- driver ----

static int round_up(int x, int m) { return (x + m - 1) / m * m; }

struct MixedPlan {
  int ld;        // B32 row length (N rounded to 4)
  int ldx;       // nocc rounded to 32
  int ncg;       // column groups of the X pass
  int cols;      // columns per group
  int sub_n, n_sub;
  int xp_stages;
  size_t xp_smem;
  int ntile, ntri, nchunk, ppc;
  int sy_stages;
  size_t sy_smem;
};

static MixedPlan mixed_plan(int n, int naux, int nocc) {
  MixedPlan m;
  m.ld = round_up(n, 4);
  const int ldx0 = round_up(std::max(nocc, 1), 32);
  m.ncg = (ldx0 + 511) / 512;
  m.cols = round_up((ldx0 + m.ncg - 1) / m.ncg, 32);
  m.ldx = m.ncg * m.cols;  // every column group is full
  m.n_sub = (m.cols + 255) / 256;
  m.sub_n = m.cols / m.n_sub;  // multiple of 16 since cols is a multiple of 32
  const size_t stage = kAStage + (size_t)m.cols * 128;
  const size_t avail = 232448 - 1024 - 256;
  m.xp_stages = (int)std::min<size_t>(4, avail / stage);
  m.xp_smem = m.xp_stages * stage + 1024 + 256;
  m.ntile = (n + kBM - 1) / kBM;
  m.ntri = m.ntile * (m.ntile + 1) / 2;
  m.nchunk = std::max(1, std::min(naux, (2 * 152 + m.ntri - 1) / m.ntri));
  m.ppc = (naux + m.nchunk - 1) / m.nchunk;
  m.nchunk = (naux + m.ppc - 1) / m.ppc;
  m.sy_stages = 6;
  m.sy_smem = m.sy_stages * 2 * kAStage + 1024 + 256;
  return m;
}

size_t mixed_workspace_bytes(int n, int naux, int nocc) {
  const MixedPlan m = mixed_plan(n, naux, nocc);
  size_t b = (size_t)m.ldx * m.ld * 4 + (size_t)n * m.ldx * 4;
  b += (size_t)m.ncg * naux * n * 8 + (size_t)naux * 4;
  b += (size_t)m.nchunk * m.ntri * kBM * kBM * 4;
  b += (size_t)naux * n * (m.ldx - nocc) * 4;  // X32 padding beyond nocc
  return b;
}

struct MixedState {
  MixedPlan plan;
  CUtensorMap mapA, mapB, mapX;
  DBuf Cf, wrow, w32;
};

void MixedDeleter::operator()(MixedState *p) const { delete p; }

int mixed_ld(int n) { return round_up(n, 4); }

int mixed_setup(Df *df, cudaStream_t s) {
  (void)s;
  const Basis *b = df->basis;
  const int n = b->nbf, naux = b->naux, no = b->nocc;
  MixedState *ms = new MixedState();
  df->mixed.reset(ms);
  ms->plan = mixed_plan(n, naux, no);
  const MixedPlan &m = ms->plan;
  if (m.xp_stages < 2) return BQC_E_UNSUPPORTED;
  Ctx *ctx = df->ctx;
  BQC_TRY(df->X32.alloc(ctx, (size_t)naux * n * m.ldx * 4));
  BQC_TRY(df->Ct32.alloc(ctx, (size_t)m.ldx * m.ld * 4));
  BQC_TRY(ms->Cf.alloc(ctx, (size_t)n * m.ldx * 4));
  BQC_TRY(ms->wrow.alloc(ctx, (size_t)m.ncg * naux * n * 8));
  BQC_TRY(ms->w32.alloc(ctx, (size_t)naux * 4));
  BQC_TRY(df->Kpart.alloc(ctx, (size_t)m.nchunk * m.ntri * kBM * kBM * 4));
  if (!df->Jp.p) BQC_TRY(df->Jp.alloc(ctx, (size_t)df->npair * 8));
  // A: B32 as (Naux*N) rows x ld columns
  {
    const uint64_t dims[2] = {(uint64_t)m.ld, (uint64_t)naux * n};
    const uint64_t str[1] = {(uint64_t)m.ld * 4};
    const uint32_t box[2] = {32, kBM};
    BQC_TRY(make_tmap_f32(&ms->mapA, df->B32.p, 2, dims, str, box));
  }
  // B: Ct32 as ldx rows x ld columns, boxes of sub_n rows
  {
    const uint64_t dims[2] = {(uint64_t)m.ld, (uint64_t)m.ldx};
    const uint64_t str[1] = {(uint64_t)m.ld * 4};
    const uint32_t box[2] = {32, (uint32_t)m.sub_n};
    BQC_TRY(make_tmap_f32(&ms->mapB, df->Ct32.p, 2, dims, str, box));
  }
  // X32 as (ldx, N, Naux)
  {
    const uint64_t dims[3] = {(uint64_t)m.ldx, (uint64_t)n, (uint64_t)naux};
    const uint64_t str[2] = {(uint64_t)m.ldx * 4, (uint64_t)n * m.ldx * 4};
    const uint32_t box[3] = {32, kBM, 1};
    BQC_TRY(make_tmap_f32(&ms->mapX, df->X32.p, 3, dims, str, box));
  }
  BQC_CUDA_TRY(cudaFuncSetAttribute(k_xpass_tf32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)m.xp_smem));
  BQC_CUDA_TRY(cudaFuncSetAttribute(k_syrk_tf32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)m.sy_smem));
  return BQC_OK;
}

int mixed_xpass(Df *df, const double *C, cudaStream_t s, const CUtensorMap *mapA, int64_t rows,
                float *X, double *w_out) {
  MixedState *ms = df->mixed.get();
  const MixedPlan &m = ms->plan;
  const Basis *b = df->basis;
  const int n = b->nbf, no = b->nocc;
  const int64_t tot = std::max<int64_t>((int64_t)m.ldx * m.ld, (int64_t)n * m.ldx);
  df->mark(0, s);
  k_prep_c<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(C, n, no, m.ld, m.ldx,
                                                          df->Ct32.as<float>(),
                                                          ms->Cf.as<float>());
  BQC_LAUNCH_CHECK();
  df->mark(1, s);
  XpassParams p;
  p.rows = rows;
  p.n = n;
  p.ldx = m.ldx;
  p.col0 = 0;
  p.cols = m.cols;
  p.sub_n = m.sub_n;
  p.n_sub = m.n_sub;
  p.kblocks = (m.ld + 31) / 32;
  p.stages = m.xp_stages;
  p.tmem_cols = 32;
  while (p.tmem_cols < m.cols) p.tmem_cols *= 2;
  p.X = X;
  p.Cf = ms->Cf.as<float>();
  p.wrow = ms->wrow.as<double>();
  p.flag = df->ctx->flag;
  dim3 grid((unsigned)((rows + kBM - 1) / kBM), (unsigned)m.ncg);
  k_xpass_tf32<<<grid, 128, m.xp_smem, s>>>(*mapA, ms->mapB, p);
  BQC_LAUNCH_CHECK();
  if (w_out) {
    k_wreduce<<<(unsigned)(rows / n), 256, 0, s>>>(ms->wrow.as<double>(), rows, m.ncg, n, w_out,
                                                    ms->w32.as<float>());
    BQC_LAUNCH_CHECK();
  }
  return BQC_OK;
}

int mixed_syrk(Df *df, const CUtensorMap *mapX, int naux, double *K, cudaStream_t s) {
  MixedState *ms = df->mixed.get();
  const MixedPlan &m = ms->plan;
  const int n = df->basis->nbf;
  SyrkParams q;
  q.n = n;
  q.ldx = m.ldx;
  q.naux = naux;
  q.ntile = m.ntile;
  q.ntri = m.ntri;
  q.p_per_chunk = m.ppc;
  q.nib = m.ldx / 32;
  q.stages = m.sy_stages;
  q.part = df->Kpart.as<float>();
  q.flag = df->ctx->flag;
  const int nchunk = (naux + m.ppc - 1) / m.ppc;
  k_syrk_tf32<<<dim3((unsigned)m.ntri, (unsigned)nchunk), 128, m.sy_smem, s>>>(*mapX, q);
  BQC_LAUNCH_CHECK();
  k_syrk_reduce<<<dim3((unsigned)m.ntri, kBM / 32), 256, 0, s>>>(df->Kpart.as<float>(), nchunk,
                                                                  m.ntri, n, K);
  BQC_LAUNCH_CHECK();
  return BQC_OK;
}

int jk_mixed_stored(Df *df, const double *C, double *J, double *K, cudaStream_t s) {
  MixedState *ms = df->mixed.get();
  if (!ms) return BQC_E_INVALID;
  const MixedPlan &m = ms->plan;
  const Basis *b = df->basis;
  const int n = b->nbf, naux = b->naux;
  const int64_t rows = (int64_t)naux * n;
  BQC_TRY(mixed_xpass(df, C, s, &ms->mapA, rows, df->X32.as<float>(), df->w.as<double>()));
  df->mark(2, s);
  // J pass (HBM-bound) over the lower triangle of B32
  const int threads = std::min(512, round_up((n - 1) / 4 + 3, 32));
  k_jpass_tf32<<<(unsigned)((n + 1) / 2), threads, 0, s>>>(df->B32.as<float>(), ms->w32.as<float>(),
                                                          naux, n, m.ld, df->Jp.as<double>());
  BQC_LAUNCH_CHECK();
  k_unpack_sym2<<<(unsigned)(((int64_t)n * n + 255) / 256), 256, 0, s>>>(df->Jp.as<double>(), n, J);
  BQC_LAUNCH_CHECK();
  df->mark(3, s);
  BQC_TRY(mixed_syrk(df, &ms->mapX, naux, K, s));
  df->mark(4, s);
  return BQC_OK;
}

}  // namespace bqc
