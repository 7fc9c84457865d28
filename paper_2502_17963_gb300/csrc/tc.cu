// Mixed-precision Fock build on the 5th-generation tensor cores (tcgen05).
//
// The two passes over the CD-ERIs that the paper describes for the Coulomb
// and exchange matrices (Sec. 2.2) become, with B held as TF32 split
// full-square shadows Bh/Bl[P][mu][nu]:
//   X pass  X[(P,mu)][i] = sum_nu B[(P,mu)][nu] C[nu][i]         (one GEMM,
//           M = Naux*N, N = nocc, K = N) with the Coulomb contraction
//           w_P = sum_{mu,i} X[(P,mu)][i] C[mu][i] fused into the epilogue;
//   SYRK    K[mu][nu] = sum_{P,i} X[P][mu][i] X[P][nu][i], lower tiles only,
//           split over aux chunks whose partials are summed in FP64;
//   J pass  J = sum_P w_P B_P over the packed FP64 B (df.cu, 3xTF32) or the
//           TF32 shadow (single-pass TF32), on a side stream beside the SYRK.
// Tensor-core kernels: TMA (128-byte swizzle) -> shared memory ring ->
// tcgen05.mma kind::tf32 issued by one thread -> FP32 accumulators in TMEM
// -> tcgen05.ld epilogue.  Warp 0 produces, warp 1 issues MMAs, eight warps
// drain TMEM.  Every mbarrier wait is bounded; on timeout the kernel
// records an error code in the context's device flag and skips its work.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

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
static int make_tmap(CUtensorMap *map, CUtensorMapDataType dtype, const void *base, int rank,
                     const uint64_t *dims, const uint64_t *strides_bytes, const uint32_t *box);

int make_tmap_f32(CUtensorMap *map, const void *base, int rank, const uint64_t *dims,
                  const uint64_t *strides_bytes, const uint32_t *box) {
  return make_tmap(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, base, rank, dims, strides_bytes, box);
}

// fp16 tensor map with the same conventions (boxes of 64 elements = 128 bytes).
static int make_tmap_f16(CUtensorMap *map, const void *base, int rank, const uint64_t *dims,
                         const uint64_t *strides_bytes, const uint32_t *box) {
  return make_tmap(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, base, rank, dims, strides_bytes, box);
}

static int make_tmap(CUtensorMap *map, CUtensorMapDataType dtype, const void *base, int rank,
                     const uint64_t *dims, const uint64_t *strides_bytes, const uint32_t *box) {
  auto enc = get_encode();
  if (!enc) {
    set_error("cuTensorMapEncodeTiled unavailable", __FILE__, __LINE__);
    return BQC_E_CUDA;
  }
  if (rank < 1 || rank > 5) {
    set_error("tensor map rank out of range", __FILE__, __LINE__);
    return BQC_E_INVALID;
  }
  cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  cuuint64_t d[5], s[4];
  cuuint32_t b[5];
  for (int i = 0; i < rank; ++i) {
    d[i] = dims[i];
    b[i] = box[i];
  }
  for (int i = 0; i < rank - 1; ++i) s[i] = strides_bytes[i];
  CUresult r = enc(map, dtype, (cuuint32_t)rank, const_cast<void *>(base),
                   d, s, b, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed", __FILE__, __LINE__);
    return BQC_E_CUDA;
  }
  return BQC_OK;
}

constexpr int kBM = 128;
constexpr uint32_t kAStage = kBM * 128;  // 128 rows x 128 bytes

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

// Precision design.
//  * Split operands: an FP32 value f is held as hi = tf32(f), lo = tf32(f - hi)
//    (hi + lo = f to ~2^-22).  SPLIT = 3 issues hi*hi + hi*lo + lo*hi per
//    k-step ("3xTF32"), SPLIT = 1 only hi*hi (plain TF32, ~2^-11 per product).
//  * Short accumulation chains: the tensor core adds into its FP32 TMEM
//    accumulator with truncation, so a chain of S MMAs carries a relative bias
//    growing with S (measured ~3e-5 after 390 steps).  Every chain here is one
//    group of kGroupKb k-blocks; TMEM holds two accumulators, and while the
//    MMA warp fills one, eight epilogue warps drain the other into register
//    accumulators with round-to-nearest adds (X pass: FP32; SYRK:
//    float-float, the compensation term kept in spare TMEM columns).  Within
//    a chain the cross terms go first, while the accumulator is still small,
//    so that only the hi*hi MMAs add into a full-size accumulator.  At the
//    end of the chain the bias is what decides the SCF's error floor in
//    mixed precision (the orthogonalisation amplifies a relative shift of K
//    by the inverse square root of the smallest overlap eigenvalue).

constexpr int kEpiWarps = 8;
constexpr int kThreads = 64 + 32 * kEpiWarps;  // TMA warp, MMA warp, 8 epilogue warps
constexpr int kGroupKb = 4;   // k-blocks (of 32) per TMEM chain: X pass (contraction N)
constexpr int kGroupKbS = 4;  // SYRK (contraction Naux x nocc)
constexpr int kGroupKbT = 2;  // TRMM (contraction Naux)

// Power-of-two scales of the FP16 split (written on the device by
// k_scales for each build, read by the X-pass and SYRK epilogues).  FP16 has
// TF32's 11-bit significand but a narrow exponent range (normal numbers from
// 2^-14 to 65504), so every operand is scaled to a largest magnitude of at
// most 2^14 before it is split: B by s_B (fixed at setup), C by s_C, X by
// s_X.  Powers of two make the scaling and unscaling exact.
struct MixScale {
  float x_out;       // s_X / (s_B s_C): X-pass accumulator -> scaled X
  float x_unscale;   // 1 / (s_B s_C): X-pass accumulator -> X
  float c_scale;     // s_C
  float pad;
  double k_unscale;  // 1 / s_X^2: SYRK accumulator -> K
};

struct XpassParams {
  int64_t rows;      // rows of this launch (M of the GEMM), starting at row0
  int64_t row0;      // first row (a launch may cover a range of aux functions)
  int64_t wstride;   // row stride of the w partials (all rows of the tensor)
  int n;             // N (rows per aux function)
  int ldx;           // row length of X and Cf
  int ncg;           // column groups (tile columns = XN each)
  int kblocks;       // ceil(K / 32)
  int stages;
  int64_t tiles;     // row tiles x ncg
  float *Xh, *Xl;    // rows x ldx (TF32 hi / lo parts)
  __half *Xh16, *Xl16;      // rows x ldx (FP16 hi / lo parts of s_X X), KIND f16
  const MixScale *scale;    // KIND f16
  const float *Cf;   // N x ldx, fp32 C_occ
  float *wpart;      // [2 * ncg][rows] partial w per row
  int *flag;
  // transposed epilogue (EPI = 1, direct mode): rows are (mu, q) with q the
  // aux function within a block of bk, written to X^T(mu, i, P = q0 + q)
  // stored as [P block][i][mu][32] (xrows = ldx * N rows per P block)
  int bk, q0, bkv;   // bkv: valid rows per mu (a ragged last sub-block)
  int64_t xrows;
};

// Whether the X pass keeps its chain sums in TMEM (two accumulator buffers
// and the running sum, 3 XN columns, fit in the 512 columns of an SM).
__host__ __device__ constexpr bool xpass_acc_tmem(int XN) { return 3 * XN <= 512; }
// Resident CTAs the register budget is sized for: 2 leaves room for other
// kernels' blocks (the J pass) beside a persistent CTA that needs few
// registers.
__host__ __device__ constexpr int xpass_min_blocks(int XN) { return xpass_acc_tmem(XN) ? 2 : 1; }

// One X-pass tile as the kernel body sees it: the operand maps, the
// parameters of its problem, its first row, column group and width (xn <= the
// kernel's XN; one problem per launch has xn = XN, a grouped launch takes the
// width of each problem's own plan).
struct XTile {
  const CUtensorMap *Ah, *Al, *Ch, *Cl;
  const XpassParams *p;
  int64_t m0;
  int cg, xn;
  const CUtensorMap *ChH = nullptr, *ClH = nullptr;  // half-height C boxes (cluster pairs)
};

// Tile locator of a single-problem launch.
template <int XN> struct XLocOne {
  const CUtensorMap *Ah, *Al, *Ch, *Cl;
  const XpassParams *p;
  __device__ __forceinline__ XTile at(int64_t t) const {
    return XTile{Ah, Al, Ch, Cl, p, p->row0 + (t / p->ncg) * kBM, (int)(t % p->ncg), XN};
  }
};

// Tile locator of a cluster pair: pair tile u = (row tiles 2 (u / ncg) and
// 2 (u / ncg) + 1, column group u % ncg); the CTA of rank r takes row tile
// 2 (u / ncg) + r.  Both CTAs need the same C tile: each loads one half and
// multicasts it to both.  A row tile past the end is computed from the
// (zero-filled or next) rows and discarded by the epilogue's row guard.
template <int XN> struct XLocPair {
  const CUtensorMap *Ah, *Al, *Ch, *Cl, *ChH, *ClH;
  const XpassParams *p;
  int rank;
  __device__ __forceinline__ XTile at(int64_t u) const {
    const int64_t rt = 2 * (u / p->ncg) + rank;
    return XTile{Ah, Al, Ch, Cl, p, p->row0 + rt * kBM, (int)(u % p->ncg), XN, ChH, ClH};
  }
};

// Persistent: CTA c processes tiles c, c + grid, ...; tile t = (row tile
// t / ncg, column group t % ncg), so neighbouring CTAs share A rows in L2.
// MC: the CTAs run in clusters of two over pair tiles (XLocPair), the C tile
// multicast to both, and a stage is free only when both CTAs' MMAs have
// released it (each MMA warp's commit arrives on both CTAs' empty barrier).
// EPI 0: X[row][i] (hi/lo) and the fused w_P partials; EPI 1: X^T layout
// (TF32 only).  KIND: TF32 or FP16 operands (k-blocks of 32 or 64 elements).
// LOC maps a tile index to its problem (one problem, or a grouped table).
template <int KIND, int XN, int SPLIT, int EPI, class LOC, bool MC = false>
__device__ __forceinline__ void xpass_body(const LOC &loc, int64_t tiles, int stages,
                                           int *flag) {
  static_assert(KIND == kKindTF32 || EPI == 0, "the transposed epilogue is TF32 only");
  using KD = Kind<KIND>;
  constexpr int KE = KD::kElems;
  constexpr int HALF = XN / 2;
  constexpr int NS = SPLIT == 3 ? 2 : 1;  // operand parts per side
  constexpr uint32_t a_bytes = kAStage, c_bytes = XN * 128;
  constexpr uint32_t stage_bytes = NS * (a_bytes + c_bytes);
  // ACC_T: the running sum of the chains lives in a third TMEM region
  // (columns 2 XN .. 3 XN) instead of registers, so the epilogue needs few
  // registers and other kernels' blocks fit beside the persistent CTA
  constexpr bool ACC_T = xpass_acc_tmem(XN);
  constexpr int UCOLS = ACC_T ? 3 * XN : 2 * XN;
  constexpr int TCOLS = (UCOLS <= 32) ? 32 : (UCOLS <= 64) ? 64 : (UCOLS <= 128) ? 128
                                            : (UCOLS <= 256) ? 256 : 512;
  constexpr int AREG = ACC_T ? 1 : HALF;  // register accumulators per thread
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = align1024(smem_raw);
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + (size_t)stages * stage_bytes);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2 * stages + 4);
  const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * stages;
  const uint32_t tfull0 = full0 + 16 * stages, tempty0 = tfull0 + 16;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, MC ? 2 : 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull0 + 8 * b, 1);
      mbar_init(tempty0 + 8 * b, kEpiWarps);
    }
    fence_barrier_init();
  }
  if (warp == 0) tmem_alloc(smem_u32(tslot), TCOLS);
  __syncthreads();
  if (MC) cluster_sync();  // the peer's barriers exist before anything is multicast
  tc_fence_after();
  const uint32_t tbase = *tslot;
  const uint32_t sbase = smem_u32(smem);
  const int64_t tbeg = MC ? blockIdx.x / 2 : blockIdx.x;
  const int64_t tstep = MC ? gridDim.x / 2 : gridDim.x;
  const uint32_t rank = MC ? cluster_rank() : 0;
  bool ok = true;
  if (warp == 0) {
    if (lane == 0) {
      int64_t kg = 0;  // k-blocks issued by this CTA
      for (int64_t t = tbeg; t < tiles && ok; t += tstep) {
        const XTile T = loc.at(t);
        const int kblocks = T.p->kblocks;
        const int c0 = T.cg * T.xn;
        const uint32_t tx = (uint32_t)NS * (a_bytes + (uint32_t)T.xn * 128);
        for (int kb = 0; kb < kblocks && ok; ++kb, ++kg) {
          const int s = (int)(kg % stages);
          if (kg >= stages)
            ok = mbar_wait(empty0 + 8 * s, (uint32_t)(((kg / stages) - 1) & 1), flag, 11);
          if (!ok) break;
          const uint32_t a = sbase + s * stage_bytes;  // [Ah][Al][Ch][Cl]
          const uint32_t bar = full0 + 8 * s;
          mbar_arrive_expect_tx(bar, tx);
          tma_load_2d(a, T.Ah, bar, kb * KE, (int)T.m0);
          if (SPLIT == 3) tma_load_2d(a + a_bytes, T.Al, bar, kb * KE, (int)T.m0);
          if (MC) {  // this CTA's half of the C tile, to both CTAs of the pair
            const int hr = T.xn / 2;
            const uint32_t ho = rank * (uint32_t)hr * 128;
            tma_load_2d_mc(a + NS * a_bytes + ho, T.ChH, bar, kb * KE, c0 + (int)rank * hr, 3);
            if (SPLIT == 3)
              tma_load_2d_mc(a + NS * a_bytes + c_bytes + ho, T.ClH, bar, kb * KE,
                             c0 + (int)rank * hr, 3);
          } else {
            tma_load_2d(a + NS * a_bytes, T.Ch, bar, kb * KE, c0);
            if (SPLIT == 3) tma_load_2d(a + NS * a_bytes + c_bytes, T.Cl, bar, kb * KE, c0);
          }
        }
      }
      // MC tail: wait until both CTAs' MMAs have released the last stages,
      // so that no commit of the peer can still be on its way to this CTA's
      // barriers when the CTA exits
      for (int64_t j = kg > stages ? kg - stages : 0; MC && ok && j < kg; ++j)
        ok = mbar_wait(empty0 + 8 * (int)(j % stages), (uint32_t)((j / stages) & 1), flag, 15);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int64_t kg = 0, g = 0;
      for (int64_t t = tbeg; t < tiles && ok; t += tstep) {
        const XTile T = loc.at(t);
        const int kblocks = T.p->kblocks;
        const int ngroups = (kblocks + kGroupKb - 1) / kGroupKb;
        const uint32_t idesc = KD::idesc(kBM, T.xn);
        for (int gr = 0; gr < ngroups && ok; ++gr, ++g) {
          const int b = (int)(g & 1);
          if (g >= 2) ok = mbar_wait(tempty0 + 8 * b, (uint32_t)(((g >> 1) - 1) & 1), flag, 14);
          if (!ok) break;
          tc_fence_after();
          const uint32_t d = tbase + b * XN;
          const int kb0 = gr * kGroupKb, kb1 = min(kblocks, kb0 + kGroupKb);
          for (int kb = kb0; kb < kb1 && ok; ++kb, ++kg) {
            const int s = (int)(kg % stages);
            ok = mbar_wait(full0 + 8 * s, (uint32_t)((kg / stages) & 1), flag, 12);
            if (!ok) break;
            tc_fence_after();
            const uint32_t ah = sbase + s * stage_bytes, al = ah + a_bytes;
            const uint32_t ch = ah + NS * a_bytes, cl = ch + c_bytes;
            if (SPLIT == 3) {
              // cross terms first: their running sum stays ~2^-11 of the
              // result, so the accumulator's truncation there is negligible;
              // then the hi*hi terms
#pragma unroll
              for (int k4 = 0; k4 < 4; ++k4) {
                const uint32_t acc = ((kb - kb0) | k4) != 0;
                KD::mma(d, sdesc_sw128(ah + k4 * 32), sdesc_sw128(cl + k4 * 32), acc, idesc);
                KD::mma(d, sdesc_sw128(al + k4 * 32), sdesc_sw128(ch + k4 * 32), 1, idesc);
              }
#pragma unroll
              for (int k4 = 0; k4 < 4; ++k4)
                KD::mma(d, sdesc_sw128(ah + k4 * 32), sdesc_sw128(ch + k4 * 32), 1, idesc);
            } else {
#pragma unroll
              for (int k4 = 0; k4 < 4; ++k4) {
                const uint32_t acc = ((kb - kb0) | k4) != 0;
                KD::mma(d, sdesc_sw128(ah + k4 * 32), sdesc_sw128(ch + k4 * 32), acc, idesc);
              }
            }
            if (MC)
              mma_commit_mc(empty0 + 8 * s, 3);
            else
              mma_commit(empty0 + 8 * s);
          }
          mma_commit(tfull0 + 8 * b);
        }
      }
    }
  } else {
    // epilogue warps: quadrant q of TMEM lanes, column half h
    const int q = warp & 3, h = (warp - 2) >> 2;
    int64_t g = 0;
    for (int64_t t = tbeg; t < tiles; t += tstep) {
      const XTile T = loc.at(t);
      const XpassParams &p = *T.p;
      const int half = T.xn / 2;  // a multiple of 16
      const int ngroups = (p.kblocks + kGroupKb - 1) / kGroupKb;
      const int64_t m0 = T.m0;
      const int cg = T.cg;
      const int64_t row_end = p.row0 + p.rows;
      const uint32_t tacc = tbase + ((uint32_t)(q * 32) << 16) + 2 * XN + h * half;
      float acc[AREG];
#pragma unroll
      for (int c = 0; c < AREG; ++c) acc[c] = 0.0f;
      for (int gr = 0; gr < ngroups; ++gr, ++g) {
        const int b = (int)(g & 1);
        if (ok) ok = mbar_wait(tfull0 + 8 * b, (uint32_t)((g >> 1) & 1), flag, 13);
        __syncwarp();
        tc_fence_after();
        const uint32_t ta = tbase + ((uint32_t)(q * 32) << 16) + b * XN + h * half;
#pragma unroll (ACC_T ? 1 : HALF / 16)
        for (int c = 0; c < HALF; c += 16) {
          if (c < half) {
            float v[16];
            tmem_ld16(ta + c, v);
            if (ACC_T) {
              if (gr > 0) {
                float a[16];
                tmem_ld16(tacc + c, a);
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] = a[i] + v[i];
              }
              tmem_st16(tacc + c, v);
            } else {
#pragma unroll
              for (int i = 0; i < 16; ++i) acc[(c + i) % AREG] += v[i];
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(tempty0 + 8 * b);
      }
      // the 16 accumulated columns c .. c + 15 of this thread's half
      auto acc16 = [&](int c, float *a) {
        if (ACC_T) {
          tmem_ld16(tacc + c, a);
        } else {
#pragma unroll
          for (int i = 0; i < 16; ++i) a[i] = acc[(c + i) % AREG];
        }
      };
      // tcgen05.ld is warp-collective: every lane reads the accumulators
      // (acc16), and only the lanes of valid rows store
      const int64_t row = m0 + q * 32 + lane;
      const bool act = ok && row < row_end;
      if (KIND == kKindF16) {
        // scaled X split into FP16 hi + lo (each rounded to nearest), and the
        // fused w partial sum_i X[row][i] C[mu][i] of the unscaled X
        const float xo = p.scale->x_out, xu = p.scale->x_unscale;
        const int mu = (int)(row % p.n);
        const int col = cg * T.xn + h * half;
        __half *xh = p.Xh16 + row * p.ldx + col;
        __half *xl = p.Xl16 + row * p.ldx + col;
        const float *cr = p.Cf + (int64_t)mu * p.ldx + col;
        float wsum = 0.0f;
#pragma unroll (ACC_T ? 1 : HALF / 16)
        for (int c16 = 0; c16 < HALF; c16 += 16) {
          if (c16 < half) {
            float a16[16];
            acc16(c16, a16);
#pragma unroll
            for (int e = 0; e < 16 && act; e += 8) {
              const int c = c16 + e;
              const float *av = a16 + e;
              const float4 ca = *reinterpret_cast<const float4 *>(cr + c);
              const float4 cb = *reinterpret_cast<const float4 *>(cr + c + 4);
              wsum = fmaf(av[0], ca.x, wsum);
              wsum = fmaf(av[1], ca.y, wsum);
              wsum = fmaf(av[2], ca.z, wsum);
              wsum = fmaf(av[3], ca.w, wsum);
              wsum = fmaf(av[4], cb.x, wsum);
              wsum = fmaf(av[5], cb.y, wsum);
              wsum = fmaf(av[6], cb.z, wsum);
              wsum = fmaf(av[7], cb.w, wsum);
              __align__(16) __half hv[8], lv[8];
#pragma unroll
              for (int k = 0; k < 8; ++k) {
                const float v = av[k] * xo;
                hv[k] = __float2half_rn(v);
                lv[k] = __float2half_rn(v - __half2float(hv[k]));
              }
              *reinterpret_cast<uint4 *>(xh + c) = *reinterpret_cast<const uint4 *>(hv);
              *reinterpret_cast<uint4 *>(xl + c) = *reinterpret_cast<const uint4 *>(lv);
            }
          }
        }
        if (act) p.wpart[(int64_t)(2 * cg + h) * p.wstride + row] = wsum * xu;
      }
      if (KIND == kKindTF32 && EPI == 0) {
        const int mu = (int)(row % p.n);
        const int col = cg * T.xn + h * half;
        float *xh = p.Xh + row * p.ldx + col;
        float *xl = p.Xl + row * p.ldx + col;
        const float *cr = p.Cf + (int64_t)mu * p.ldx + col;
        float wsum = 0.0f;
#pragma unroll (ACC_T ? 1 : HALF / 16)
        for (int c16 = 0; c16 < HALF; c16 += 16) {
          if (c16 < half) {
            float a16[16];
            acc16(c16, a16);
#pragma unroll
            for (int e = 0; e < 16 && act; e += 4) {
              const int c = c16 + e;
              const float *av = a16 + e;
              const float4 cc = *reinterpret_cast<const float4 *>(cr + c);
              wsum = fmaf(av[0], cc.x, wsum);
              wsum = fmaf(av[1], cc.y, wsum);
              wsum = fmaf(av[2], cc.z, wsum);
              wsum = fmaf(av[3], cc.w, wsum);
              float4 hv, lv;
              hv.x = tf32r(av[0]);
              hv.y = tf32r(av[1]);
              hv.z = tf32r(av[2]);
              hv.w = tf32r(av[3]);
              *reinterpret_cast<float4 *>(xh + c) = hv;
              if (SPLIT == 3) {
                lv.x = tf32r(av[0] - hv.x);
                lv.y = tf32r(av[1] - hv.y);
                lv.z = tf32r(av[2] - hv.z);
                lv.w = tf32r(av[3] - hv.w);
                *reinterpret_cast<float4 *>(xl + c) = lv;
              }
            }
          }
        }
        if (act) p.wpart[(int64_t)(2 * cg + h) * p.wstride + row] = wsum;
      }
      if (KIND == kKindTF32 && EPI == 1) {
        const bool act1 = act && (int)(row % p.bk) < p.bkv;
        // consecutive lanes hold consecutive q of one mu: coalesced per column
        const int64_t mu = row / p.bk, qq = p.q0 + row % p.bk;
        const int col = cg * T.xn + h * half;
        const int64_t base = ((qq >> 5) * p.xrows + (int64_t)col * p.n + mu) * 32 + (qq & 31);
        const int64_t step = (int64_t)p.n * 32;
#pragma unroll (ACC_T ? 1 : HALF / 16)
        for (int c16 = 0; c16 < HALF; c16 += 16) {
          if (c16 < half) {
            float a16[16];
            acc16(c16, a16);
#pragma unroll
            for (int e = 0; e < 16 && act1; ++e) {
              const int c = c16 + e;
              const float hv = tf32r(a16[e]);
              p.Xh[base + (int64_t)c * step] = hv;
              if (SPLIT == 3) p.Xl[base + (int64_t)c * step] = tf32r(a16[e] - hv);
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  // the peer's MMAs (whose commits arrive here) and its copies into this
  // CTA's shared memory are complete once both CTAs reach this barrier
  if (MC) cluster_sync();
  if (warp == 0) tmem_dealloc(tbase, TCOLS);
}

template <int KIND, int XN, int SPLIT, int EPI>
__global__ void __launch_bounds__(kThreads, xpass_min_blocks(XN))
    k_xpass(const __grid_constant__ CUtensorMap mapAh, const __grid_constant__ CUtensorMap mapAl,
            const __grid_constant__ CUtensorMap mapCh, const __grid_constant__ CUtensorMap mapCl,
            const __grid_constant__ XpassParams p) {
  if (threadIdx.x == 0) {
    prefetch_tmap(&mapAh);
    prefetch_tmap(&mapCh);
    if (SPLIT == 3) {
      prefetch_tmap(&mapAl);
      prefetch_tmap(&mapCl);
    }
  }
  const XLocOne<XN> loc{&mapAh, &mapAl, &mapCh, &mapCl, &p};
  xpass_body<KIND, XN, SPLIT, EPI>(loc, p.tiles, p.stages, p.flag);
}

// The split-FP16 X pass in clusters of two CTAs over pair tiles: each CTA
// loads its own 128 rows of B and one half of the shared C tile, multicast to
// both, so the C operand crosses from L2 once per pair instead of twice.
template <int XN>
__global__ void __launch_bounds__(kThreads, xpass_min_blocks(XN))
    k_xpass_mc(const __grid_constant__ CUtensorMap mapAh, const __grid_constant__ CUtensorMap mapAl,
               const __grid_constant__ CUtensorMap mapChH,
               const __grid_constant__ CUtensorMap mapClH, const __grid_constant__ XpassParams p) {
  if (threadIdx.x == 0) {
    prefetch_tmap(&mapAh);
    prefetch_tmap(&mapAl);
    prefetch_tmap(&mapChH);
    prefetch_tmap(&mapClH);
  }
  const XLocPair<XN> loc{&mapAh, &mapAl, &mapChH, &mapClH, &mapChH, &mapClH, &p,
                         (int)cluster_rank()};
  const int64_t rt = (p.rows + kBM - 1) / kBM;
  xpass_body<kKindF16, XN, 3, 0, XLocPair<XN>, true>(loc, (rt + 1) / 2 * p.ncg, p.stages,
                                                     p.flag);
}

// w[P] = sum over partials and mu of wpart[k][P*N + mu] (FP64); also fp32 w.
// One 256-thread block per P.
__device__ __forceinline__ void wreduce_one(const float *wpart, int64_t rows, int nparts, int n,
                                            double *w, float *w32, float2 *w2, int P) {
  double s = 0.0;
  for (int g = 0; g < nparts; ++g)
    for (int m = threadIdx.x; m < n; m += blockDim.x) s += wpart[g * rows + (int64_t)P * n + m];
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
    if (w2) {  // float pair (hi, lo) for the float-float J pass
      const float h = (float)red[0];
      w2[P] = make_float2(h, (float)(red[0] - (double)h));
    }
  }
}

__global__ void __launch_bounds__(256) k_wreduce(const float *wpart, int64_t rows, int nparts,
                                                 int n, double *w, float *w32, float2 *w2,
                                                 int P0) {
  wreduce_one(wpart, rows, nparts, n, w, w32, w2, P0 + blockIdx.x);
}

// ---------------------------------------------------------------- SYRK ---

struct SyrkParams {
  int n, ldx, naux;
  int ntri;
  int nchunk, p_per_chunk;
  int nib;       // k-blocks per aux function: ceil(ldx / elements per k-block)
  int stages;
  double *part;  // [chunk][ntri][128][128]
  int *flag;
  const MixScale *scale;  // KIND f16: partial tiles are unscaled by scale->k_unscale
  // two-operand mode (3-D operands): tile (tm, tn) = sum X[tm] Y[tn]^T +
  // Y[tm] X[tn]^T over the chunk, the lower tiles of a symmetric rank-2k update
  int two;
  // blocked operand mode (direct mode): Y^T stored as [P block][i][mu][32];
  // rows mu, K = (i, P) with k-block kb = i * npb + P block; chunks are ranges
  // of kb_per_chunk k-blocks of kb_total
  int mode2d;
  int npb;
  int64_t kb_total;
  int64_t kb_per_chunk;
};

__device__ __forceinline__ void tile_of(int t, int &tm, int &tn) {
  int m = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
  while ((m + 1) * (m + 2) / 2 <= t) ++m;
  while (m * (m + 1) / 2 > t) --m;
  tm = m;
  tn = t - m * (m + 1) / 2;
}

constexpr int kSyCols = kBM / (kEpiWarps / 4);  // columns per epilogue thread
constexpr uint32_t kLoCol = 2 * kBM;             // TMEM columns of the compensation term
constexpr uint32_t kHiCol = 3 * kBM;             // TMEM columns of the running sum

// One SYRK work item: operand maps, problem parameters, lower tile and aux
// chunk.
struct SyItem {
  const CUtensorMap *Xh, *Xl, *Yh, *Yl;
  const SyrkParams *p;
  int tile, chunk;
};

// Work-item locator of a single-problem launch: item i -> tile i % ntri,
// chunk i / ntri.
struct SyLocOne {
  const CUtensorMap *Xh, *Xl, *Yh, *Yl;
  const SyrkParams *p;
  __device__ __forceinline__ SyItem at(int it) const {
    return SyItem{Xh, Xl, Yh, Yl, p, it % p->ntri, it / p->ntri};
  }
};

// Persistent SYRK over work items (lower tile, aux chunk).  Partial tiles are written in FP64.  KIND: TF32
// or FP16 operands (the blocked operand mode of direct mode is TF32 only).
template <int KIND, int SPLIT, class LOC>
__device__ __forceinline__ void syrk_body(const LOC &loc, int items, int stages, int *flag) {
  using KD = Kind<KIND>;
  constexpr int KE = KD::kElems;
  constexpr int NS = SPLIT == 3 ? 2 : 1;
  constexpr uint32_t stage_bytes = NS * 2 * kAStage;  // [Xh(tm)][Xh(tn)][Xl(tm)][Xl(tn)]
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = align1024(smem_raw);
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + (size_t)stages * stage_bytes);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2 * stages + 4);
  const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * stages;
  const uint32_t tfull0 = full0 + 16 * stages, tempty0 = tfull0 + 16;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull0 + 8 * b, 1);
      mbar_init(tempty0 + 8 * b, kEpiWarps);
    }
    fence_barrier_init();
  }
  if (warp == 0) tmem_alloc(smem_u32(tslot), 512);
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;
  const uint32_t sbase = smem_u32(smem);
  bool ok = true;
  // chunk ch -> first aux function P0 (3-D mode) or first k-block (2-D mode), k-block count
  auto chunk_kb = [&](const SyrkParams &p, int ch, int64_t &P0, int &nkb) {
    if (p.mode2d) {
      P0 = (int64_t)ch * p.kb_per_chunk;
      nkb = (int)max((int64_t)0, min(p.kb_total, P0 + p.kb_per_chunk) - P0);
    } else {
      P0 = (int64_t)ch * p.p_per_chunk;
      nkb = max(0, min(p.naux, (int)P0 + p.p_per_chunk) - (int)P0) * p.nib;
      if (p.two) nkb *= 2;  // first half X[tm] Y[tn], second half Y[tm] X[tn]
    }
  };
  if (warp == 0) {
    if (lane == 0) {
      int64_t kg = 0;
      for (int it = blockIdx.x; it < items && ok; it += gridDim.x) {
        const SyItem I = loc.at(it);
        const SyrkParams &p = *I.p;
        int tm, tn, nkb;
        int64_t P0;
        tile_of(I.tile, tm, tn);
        chunk_kb(p, I.chunk, P0, nkb);
        for (int kb = 0; kb < nkb && ok; ++kb, ++kg) {
          const int s = (int)(kg % stages);
          if (kg >= stages)
            ok = mbar_wait(empty0 + 8 * s, (uint32_t)(((kg / stages) - 1) & 1), flag, 21);
          if (!ok) break;
          const uint32_t a = sbase + s * stage_bytes, bar = full0 + 8 * s;
          mbar_arrive_expect_tx(bar, stage_bytes);
          if (p.mode2d) {
            // one box = 128 consecutive mu of one (i, P block): 16 KB contiguous
            const int64_t kk = P0 + kb;
            const int pb = (int)(kk % p.npb), ii = (int)(kk / p.npb);
            tma_load_4d(a, I.Xh, bar, 0, tm * kBM, ii, pb);
            tma_load_4d(a + kAStage, I.Xh, bar, 0, tn * kBM, ii, pb);
            if (SPLIT == 3) {
              tma_load_4d(a + 2 * kAStage, I.Xl, bar, 0, tm * kBM, ii, pb);
              tma_load_4d(a + 3 * kAStage, I.Xl, bar, 0, tn * kBM, ii, pb);
            }
          } else {
            const int half = p.two ? nkb / 2 : nkb;
            const bool second = kb >= half;
            const int kk = second ? kb - half : kb;
            const int P = (int)P0 + kk / p.nib, i0 = (kk % p.nib) * KE;
            // one-operand: X[tm], X[tn]; two-operand: X[tm], Y[tn] then Y[tm], X[tn]
            const CUtensorMap *mh = (p.two && second) ? I.Yh : I.Xh;
            const CUtensorMap *ml = (p.two && second) ? I.Yl : I.Xl;
            const CUtensorMap *nh = (p.two && !second) ? I.Yh : I.Xh;
            const CUtensorMap *nl = (p.two && !second) ? I.Yl : I.Xl;
            tma_load_3d(a, mh, bar, i0, tm * kBM, P);
            tma_load_3d(a + kAStage, nh, bar, i0, tn * kBM, P);
            if (SPLIT == 3) {
              tma_load_3d(a + 2 * kAStage, ml, bar, i0, tm * kBM, P);
              tma_load_3d(a + 3 * kAStage, nl, bar, i0, tn * kBM, P);
            }
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = KD::idesc(kBM, kBM);
      int64_t kg = 0, g = 0;
      for (int it = blockIdx.x; it < items && ok; it += gridDim.x) {
        const SyItem I = loc.at(it);
        int nkb;
        int64_t P0;
        chunk_kb(*I.p, I.chunk, P0, nkb);
        for (int kb0 = 0; kb0 < nkb && ok; kb0 += kGroupKbS, ++g) {
          const int b = (int)(g & 1);
          if (g >= 2) ok = mbar_wait(tempty0 + 8 * b, (uint32_t)(((g >> 1) - 1) & 1), flag, 24);
          if (!ok) break;
          tc_fence_after();
          const uint32_t d = tbase + b * kBM;
          const int kb1 = min(nkb, kb0 + kGroupKbS);
          for (int kb = kb0; kb < kb1 && ok; ++kb, ++kg) {
            const int s = (int)(kg % stages);
            ok = mbar_wait(full0 + 8 * s, (uint32_t)((kg / stages) & 1), flag, 22);
            if (!ok) break;
            tc_fence_after();
            const uint32_t hm = sbase + s * stage_bytes, hn = hm + kAStage;
            const uint32_t lm = hm + 2 * kAStage, ln = hm + 3 * kAStage;
            if (SPLIT == 3) {  // cross terms first, as in the X pass
#pragma unroll
              for (int k4 = 0; k4 < 4; ++k4) {
                const uint32_t acc = ((kb - kb0) | k4) != 0;
                KD::mma(d, sdesc_sw128(hm + k4 * 32), sdesc_sw128(ln + k4 * 32), acc, idesc);
                KD::mma(d, sdesc_sw128(lm + k4 * 32), sdesc_sw128(hn + k4 * 32), 1, idesc);
              }
#pragma unroll
              for (int k4 = 0; k4 < 4; ++k4)
                KD::mma(d, sdesc_sw128(hm + k4 * 32), sdesc_sw128(hn + k4 * 32), 1, idesc);
            } else {
#pragma unroll
              for (int k4 = 0; k4 < 4; ++k4) {
                const uint32_t acc = ((kb - kb0) | k4) != 0;
                KD::mma(d, sdesc_sw128(hm + k4 * 32), sdesc_sw128(hn + k4 * 32), acc, idesc);
              }
            }
            mma_commit(empty0 + 8 * s);
          }
          mma_commit(tfull0 + 8 * b);
        }
      }
    }
  } else {
    const int q = warp & 3, h = (warp - 2) >> 2;
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    int64_t g = 0;
    for (int it = blockIdx.x; it < items; it += gridDim.x) {
      const SyItem I = loc.at(it);
      const SyrkParams &p = *I.p;
      int nkb;
      int64_t P0;
      chunk_kb(p, I.chunk, P0, nkb);
      // float-float running sum (hi, lo) of the chains, both halves in TMEM
      const uint32_t tl = tbase + lane_base + kLoCol + h * kSyCols;
      const uint32_t th = tbase + lane_base + kHiCol + h * kSyCols;
      {
        float z[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) z[i] = 0.0f;
#pragma unroll
        for (int c = 0; c < kSyCols; c += 16) {
          tmem_st16(tl + c, z);
          tmem_st16(th + c, z);
        }
      }
      for (int kb0 = 0; kb0 < nkb; kb0 += kGroupKbS, ++g) {
        const int b = (int)(g & 1);
        if (ok) ok = mbar_wait(tfull0 + 8 * b, (uint32_t)((g >> 1) & 1), flag, 23);
        __syncwarp();
        tc_fence_after();
        const uint32_t ta = tbase + lane_base + b * kBM + h * kSyCols;
#pragma unroll 1
        for (int c = 0; c < kSyCols; c += 16) {
          float v[16], lo[16], hi[16];
          tmem_ld16(ta + c, v);
          tmem_ld16(tl + c, lo);
          tmem_ld16(th + c, hi);
#pragma unroll
          for (int i = 0; i < 16; ++i) {  // two-sum: (hi, lo) += v
            const float s = hi[i] + v[i];
            const float bp = s - hi[i];
            lo[i] += (hi[i] - (s - bp)) + (v[i] - bp);
            hi[i] = s;
          }
          tmem_st16(tl + c, lo);
          tmem_st16(th + c, hi);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(tempty0 + 8 * b);
      }
      const int r = q * 32 + lane;
      double *dst =
          p.part + (((int64_t)I.chunk * p.ntri + I.tile) * kBM + r) * kBM + h * kSyCols;
      const double ku = (KIND == kKindF16) ? p.scale->k_unscale : 1.0;
#pragma unroll 1
      for (int c = 0; c < kSyCols; c += 16) {
        float lo[16], hi[16];
        tmem_ld16(tl + c, lo);
        tmem_ld16(th + c, hi);
#pragma unroll
        for (int i = 0; i < 16; i += 2) {
          const double2 v =
              make_double2(ok ? ((double)hi[i] + (double)lo[i]) * ku : 0.0,
                           ok ? ((double)hi[i + 1] + (double)lo[i + 1]) * ku : 0.0);
          *reinterpret_cast<double2 *>(dst + c + i) = v;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tbase, 512);
}

template <int KIND, int SPLIT>
__global__ void __launch_bounds__(kThreads, 2)
    k_syrk(const __grid_constant__ CUtensorMap mapXh, const __grid_constant__ CUtensorMap mapXl,
           const __grid_constant__ CUtensorMap mapYh, const __grid_constant__ CUtensorMap mapYl,
           const __grid_constant__ SyrkParams p) {
  if (threadIdx.x == 0) {
    prefetch_tmap(&mapXh);
    if (SPLIT == 3) prefetch_tmap(&mapXl);
    if (p.two) {
      prefetch_tmap(&mapYh);
      prefetch_tmap(&mapYl);
    }
  }
  const SyLocOne loc{&mapXh, &mapXl, &mapYh, &mapYl, &p};
  syrk_body<KIND, SPLIT>(loc, p.ntri * p.nchunk, p.stages, p.flag);
}

// ------------------------------------------------- grouped (serving) ---
//
// Several independent molecules' X passes (or SYRKs) in one persistent
// launch: the problem table travels as one kernel parameter (tensor maps
// included, so the TMA reads them from parameter space and nothing is
// uploaded), and the locator maps a global tile index to its problem by the
// table's prefix of tile counts.  Each problem keeps its own plan (column
// groups, tile width, k-blocks, aux chunks), so every tile computes exactly
// what the single-problem launch computes for it.

struct XGroupProb {  // tensor maps first (128-byte aligned)
  CUtensorMap Ah, Al, Ch, Cl;
  XpassParams p;
  int xn;
};

struct XGroupTab {
  XGroupProb prob[kMaxGroup];
  int64_t tile0[kMaxGroup + 1];  // prefix of the problems' tile counts
  int nprob, stages;
  int *flag;
};

template <int XN> struct XLocGroup {
  const XGroupTab *g;
  __device__ __forceinline__ XTile at(int64_t t) const {
    int k = 0;
    while (k + 1 < g->nprob && t >= g->tile0[k + 1]) ++k;
    const XGroupProb &q = g->prob[k];
    const int64_t lt = t - g->tile0[k];
    return XTile{&q.Ah, &q.Al, &q.Ch, &q.Cl, &q.p, q.p.row0 + (lt / q.p.ncg) * kBM,
                 (int)(lt % q.p.ncg), q.xn};
  }
};

template <int XN>
__global__ void __launch_bounds__(kThreads, xpass_min_blocks(XN))
    k_xpass_grp(const __grid_constant__ XGroupTab g) {
  if (threadIdx.x < 4 * g.nprob) {
    const XGroupProb &q = g.prob[threadIdx.x >> 2];
    const int m = threadIdx.x & 3;
    prefetch_tmap(m == 0 ? &q.Ah : m == 1 ? &q.Al : m == 2 ? &q.Ch : &q.Cl);
  }
  const XLocGroup<XN> loc{&g};
  xpass_body<kKindF16, XN, 3, 0>(loc, g.tile0[g.nprob], g.stages, g.flag);
}

struct SyGroupProb {
  CUtensorMap Xh, Xl;
  SyrkParams p;
};

struct SyGroupTab {
  SyGroupProb prob[kMaxGroup];
  int item0[kMaxGroup + 1];  // prefix of the problems' work items
  int nprob, stages;
  int *flag;
};

struct SyLocGroup {
  const SyGroupTab *g;
  __device__ __forceinline__ SyItem at(int it) const {
    int k = 0;
    while (k + 1 < g->nprob && it >= g->item0[k + 1]) ++k;
    const SyGroupProb &q = g->prob[k];
    const int lt = it - g->item0[k];
    return SyItem{&q.Xh, &q.Xl, &q.Xh, &q.Xl, &q.p, lt % q.p.ntri, lt / q.p.ntri};
  }
};

__global__ void __launch_bounds__(kThreads, 2) k_syrk_grp(const __grid_constant__ SyGroupTab g) {
  if (threadIdx.x < 2 * g.nprob) {
    const SyGroupProb &q = g.prob[threadIdx.x >> 1];
    prefetch_tmap((threadIdx.x & 1) ? &q.Xl : &q.Xh);
  }
  const SyLocGroup loc{&g};
  syrk_body<kKindF16, 3>(loc, g.item0[g.nprob], g.stages, g.flag);
}

// C = scale * A B^T for row ranges of two K-major split-FP16 operands (the
// DF-MP2 pair blocks: rows (i, a) of the MO tensor against rows (j, b),
// contraction over the aux index).  Persistent over output tiles; tile it ->
// (it / nt, it % nt); each tile is one K loop (no aux chunks), drained from
// TMEM in short chains into float-float registers as in the SYRK, and
// written in FP64.
struct GemmNtParams {
  int mt, nt;              // output tiles along M and N
  int64_t a_row0, b_row0;  // first rows of the A and B ranges in the maps
  int kblocks;             // k-blocks of 64 elements
  int stages;
  double *out;
  int64_t ldo;
  int mvalid, nvalid;      // valid rows / columns of C
  double scale;
  int *flag;
};

template <int KIND>
__global__ void __launch_bounds__(kThreads, 1)
    k_gemm_nt(const __grid_constant__ CUtensorMap mapAh, const __grid_constant__ CUtensorMap mapAl,
              const __grid_constant__ CUtensorMap mapBh, const __grid_constant__ CUtensorMap mapBl,
              const GemmNtParams p) {
  using KD = Kind<KIND>;
  constexpr int KE = KD::kElems;
  constexpr uint32_t stage_bytes = 4 * kAStage;  // [Ah][Bh][Al][Bl]
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = align1024(smem_raw);
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + (size_t)p.stages * stage_bytes);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2 * p.stages + 4);
  const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * p.stages;
  const uint32_t tfull0 = full0 + 16 * p.stages, tempty0 = tfull0 + 16;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int items = p.mt * p.nt;
  if (threadIdx.x == 0) {
    prefetch_tmap(&mapAh);
    prefetch_tmap(&mapAl);
    prefetch_tmap(&mapBh);
    prefetch_tmap(&mapBl);
    for (int st = 0; st < p.stages; ++st) {
      mbar_init(full0 + 8 * st, 1);
      mbar_init(empty0 + 8 * st, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull0 + 8 * b, 1);
      mbar_init(tempty0 + 8 * b, kEpiWarps);
    }
    fence_barrier_init();
  }
  if (warp == 0) tmem_alloc(smem_u32(tslot), 512);
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;
  const uint32_t sbase = smem_u32(smem);
  bool ok = true;
  if (warp == 0) {
    if (lane == 0) {
      int64_t kg = 0;
      for (int it = blockIdx.x; it < items && ok; it += gridDim.x) {
        const int tm = it / p.nt, tn = it % p.nt;
        const int ra = (int)(p.a_row0 + (int64_t)tm * kBM), rb = (int)(p.b_row0 + (int64_t)tn * kBM);
        for (int kb = 0; kb < p.kblocks && ok; ++kb, ++kg) {
          const int st = (int)(kg % p.stages);
          if (kg >= p.stages)
            ok = mbar_wait(empty0 + 8 * st, (uint32_t)(((kg / p.stages) - 1) & 1), p.flag, 41);
          if (!ok) break;
          const uint32_t a = sbase + st * stage_bytes, bar = full0 + 8 * st;
          mbar_arrive_expect_tx(bar, stage_bytes);
          tma_load_2d(a, &mapAh, bar, kb * KE, ra);
          tma_load_2d(a + kAStage, &mapBh, bar, kb * KE, rb);
          tma_load_2d(a + 2 * kAStage, &mapAl, bar, kb * KE, ra);
          tma_load_2d(a + 3 * kAStage, &mapBl, bar, kb * KE, rb);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = KD::idesc(kBM, kBM);
      int64_t kg = 0, g = 0;
      for (int it = blockIdx.x; it < items && ok; it += gridDim.x) {
        for (int kb0 = 0; kb0 < p.kblocks && ok; kb0 += kGroupKbS, ++g) {
          const int b = (int)(g & 1);
          if (g >= 2) ok = mbar_wait(tempty0 + 8 * b, (uint32_t)(((g >> 1) - 1) & 1), p.flag, 44);
          if (!ok) break;
          tc_fence_after();
          const uint32_t d = tbase + b * kBM;
          const int kb1 = min(p.kblocks, kb0 + kGroupKbS);
          for (int kb = kb0; kb < kb1 && ok; ++kb, ++kg) {
            const int st = (int)(kg % p.stages);
            ok = mbar_wait(full0 + 8 * st, (uint32_t)((kg / p.stages) & 1), p.flag, 42);
            if (!ok) break;
            tc_fence_after();
            const uint32_t ah = sbase + st * stage_bytes, bh = ah + kAStage;
            const uint32_t al = ah + 2 * kAStage, bl = ah + 3 * kAStage;
#pragma unroll
            for (int k4 = 0; k4 < 4; ++k4) {  // cross terms first
              const uint32_t acc = ((kb - kb0) | k4) != 0;
              KD::mma(d, sdesc_sw128(ah + k4 * 32), sdesc_sw128(bl + k4 * 32), acc, idesc);
              KD::mma(d, sdesc_sw128(al + k4 * 32), sdesc_sw128(bh + k4 * 32), 1, idesc);
            }
#pragma unroll
            for (int k4 = 0; k4 < 4; ++k4)
              KD::mma(d, sdesc_sw128(ah + k4 * 32), sdesc_sw128(bh + k4 * 32), 1, idesc);
            mma_commit(empty0 + 8 * st);
          }
          mma_commit(tfull0 + 8 * b);
        }
      }
    }
  } else {
    const int q = warp & 3, h = (warp - 2) >> 2;
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    int64_t g = 0;
    for (int it = blockIdx.x; it < items; it += gridDim.x) {
      const int tm = it / p.nt, tn = it % p.nt;
      float hi[kSyCols];
#pragma unroll
      for (int c = 0; c < kSyCols; ++c) hi[c] = 0.0f;
      {
        float z[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) z[i] = 0.0f;
#pragma unroll
        for (int c = 0; c < kSyCols; c += 16)
          tmem_st16(tbase + lane_base + kLoCol + h * kSyCols + c, z);
      }
      for (int kb0 = 0; kb0 < p.kblocks; kb0 += kGroupKbS, ++g) {
        const int b = (int)(g & 1);
        if (ok) ok = mbar_wait(tfull0 + 8 * b, (uint32_t)((g >> 1) & 1), p.flag, 43);
        __syncwarp();
        tc_fence_after();
        const uint32_t ta = tbase + lane_base + b * kBM + h * kSyCols;
        const uint32_t tl = tbase + lane_base + kLoCol + h * kSyCols;
#pragma unroll
        for (int c = 0; c < kSyCols; c += 16) {
          float v[16], lo[16];
          tmem_ld16(ta + c, v);
          tmem_ld16(tl + c, lo);
#pragma unroll
          for (int i = 0; i < 16; ++i) {  // two-sum: (hi, lo) += v
            const float sm = hi[c + i] + v[i];
            const float bp = sm - hi[c + i];
            lo[i] += (hi[c + i] - (sm - bp)) + (v[i] - bp);
            hi[c + i] = sm;
          }
          tmem_st16(tl + c, lo);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(tempty0 + 8 * b);
      }
      const int r = tm * kBM + q * 32 + lane;
      const int c0 = tn * kBM + h * kSyCols;
      const uint32_t tl = tbase + lane_base + kLoCol + h * kSyCols;
#pragma unroll
      for (int c = 0; c < kSyCols; c += 16) {
        float lo[16];
        tmem_ld16(tl + c, lo);
        if (ok && r < p.mvalid) {
          double *dst = p.out + (int64_t)r * p.ldo + c0 + c;
#pragma unroll
          for (int i = 0; i < 16; ++i)
            if (c0 + c + i < p.nvalid) dst[i] = ((double)hi[c + i] + (double)lo[i]) * p.scale;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tbase, 512);
}

// K = sum over chunks of the FP64 partial tiles, symmetric.  One block per
// (lower tile, 32-row strip): sums into shared memory, writes the strip and
// its mirror image coalesced.
__device__ __forceinline__ void syrk_reduce_strip(const double *part, int nchunk, int ntri, int n,
                                                  double *K, int t, int sr) {
  __shared__ double strip[32][kBM + 1];
  int tm = 0;
  while ((tm + 1) * (tm + 2) / 2 <= t) ++tm;
  const int tn = t - tm * (tm + 1) / 2;
  for (int e = threadIdx.x; e < 32 * kBM; e += blockDim.x) {
    const int rr = e / kBM, c = e % kBM;
    const int r = sr * 32 + rr;
    double s = 0.0;
    for (int ch = 0; ch < nchunk; ++ch) s += part[(((int64_t)ch * ntri + t) * kBM + r) * kBM + c];
    strip[rr][c] = s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 32 * kBM; e += blockDim.x) {
    const int rr = e / kBM, c = e % kBM;
    const int mu = tm * kBM + sr * 32 + rr, nu = tn * kBM + c;
    if (mu < n && nu < n && (tm != tn || nu <= mu)) K[(int64_t)mu * n + nu] = strip[rr][c];
  }
  for (int e = threadIdx.x; e < 32 * kBM; e += blockDim.x) {
    const int c = e / 32, rr = e % 32;
    const int mu = tm * kBM + sr * 32 + rr, nu = tn * kBM + c;
    if (mu < n && nu < n && (tm != tn || nu < mu)) K[(int64_t)nu * n + mu] = strip[rr][c];
  }
}

__global__ void __launch_bounds__(256) k_syrk_reduce(const double *part, int nchunk, int ntri,
                                                     int n, double *K) {
  syrk_reduce_strip(part, nchunk, ntri, n, K, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------- TRMM ---

// In-place Y = X L^{-T} on the rows of X^T:  Y[r][P] = sum_{Q <= P} X[r][Q] Linv[P][Q]
// (r = (mu, i), so Y^T holds the metric-orthogonalised Y_P = (L^{-1} X)_P of
// direct mode).  A CTA owns row tiles exclusively and walks the P tiles of a
// row tile from the last to the first: tile pt reads columns Q < (pt+1)*128
// and writes columns [pt*128, pt*128+128), which later (smaller) tiles never
// read, so the product can overwrite X.
struct TrmmParams {
  int64_t rows;      // N * ldx rows r = i * N + mu of X^T, stored as [P block][r][32]
  int naux;          // columns (P and Q)
  int ntp;           // P tiles of 128
  int stages;
  int64_t mtiles;
  float *Xh, *Xl;
  int *flag;
};

template <int SPLIT>
__global__ void __launch_bounds__(kThreads, 1)
    k_trmm_tf32(const __grid_constant__ CUtensorMap mapXh, const __grid_constant__ CUtensorMap mapXl,
                const __grid_constant__ CUtensorMap mapLh, const __grid_constant__ CUtensorMap mapLl,
                const TrmmParams p) {
  constexpr int NS = SPLIT == 3 ? 2 : 1;
  constexpr uint32_t stage_bytes = NS * 2 * kAStage;  // [Xh][Lh][Xl][Ll]
  constexpr int HALF = kBM / 2;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = align1024(smem_raw);
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + (size_t)p.stages * stage_bytes);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2 * p.stages + 4);
  const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * p.stages;
  const uint32_t tfull0 = full0 + 16 * p.stages, tempty0 = tfull0 + 16;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    prefetch_tmap(&mapXh);
    prefetch_tmap(&mapLh);
    if (SPLIT == 3) {
      prefetch_tmap(&mapXl);
      prefetch_tmap(&mapLl);
    }
    for (int st = 0; st < p.stages; ++st) {
      mbar_init(full0 + 8 * st, 1);
      mbar_init(empty0 + 8 * st, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull0 + 8 * b, 1);
      mbar_init(tempty0 + 8 * b, kEpiWarps);
    }
    fence_barrier_init();
  }
  if (warp == 0) tmem_alloc(smem_u32(tslot), 256);
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;
  const uint32_t sbase = smem_u32(smem);
  auto kblocks_of = [&](int pt) { return (min(p.naux, (pt + 1) * kBM) + 31) / 32; };
  bool ok = true;
  if (warp == 0) {
    if (lane == 0) {
      int64_t kg = 0;
      for (int64_t t = blockIdx.x; t < p.mtiles && ok; t += gridDim.x) {
        const int m0 = (int)(t * kBM);
        for (int pt = p.ntp - 1; pt >= 0 && ok; --pt) {
          const int nkb = kblocks_of(pt);
          for (int kb = 0; kb < nkb && ok; ++kb, ++kg) {
            const int st = (int)(kg % p.stages);
            if (kg >= p.stages)
              ok = mbar_wait(empty0 + 8 * st, (uint32_t)(((kg / p.stages) - 1) & 1), p.flag, 31);
            if (!ok) break;
            const uint32_t a = sbase + st * stage_bytes, bar = full0 + 8 * st;
            mbar_arrive_expect_tx(bar, stage_bytes);
            tma_load_3d(a, &mapXh, bar, 0, m0, kb);
            tma_load_2d(a + kAStage, &mapLh, bar, kb * 32, pt * kBM);
            if (SPLIT == 3) {
              tma_load_3d(a + 2 * kAStage, &mapXl, bar, 0, m0, kb);
              tma_load_2d(a + 3 * kAStage, &mapLl, bar, kb * 32, pt * kBM);
            }
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_tf32(kBM, kBM);
      int64_t kg = 0, g = 0;
      for (int64_t t = blockIdx.x; t < p.mtiles && ok; t += gridDim.x) {
        for (int pt = p.ntp - 1; pt >= 0 && ok; --pt) {
          const int nkb = kblocks_of(pt);
          for (int kb0 = 0; kb0 < nkb && ok; kb0 += kGroupKbT, ++g) {
            const int b = (int)(g & 1);
            if (g >= 2)
              ok = mbar_wait(tempty0 + 8 * b, (uint32_t)(((g >> 1) - 1) & 1), p.flag, 34);
            if (!ok) break;
            tc_fence_after();
            const uint32_t d = tbase + b * kBM;
            const int kb1 = min(nkb, kb0 + kGroupKbT);
            for (int kb = kb0; kb < kb1 && ok; ++kb, ++kg) {
              const int st = (int)(kg % p.stages);
              ok = mbar_wait(full0 + 8 * st, (uint32_t)((kg / p.stages) & 1), p.flag, 32);
              if (!ok) break;
              tc_fence_after();
              const uint32_t xh = sbase + st * stage_bytes, lh = xh + kAStage;
              const uint32_t xl = xh + 2 * kAStage, ll = xh + 3 * kAStage;
              if (SPLIT == 3) {  // cross terms first, as in the X pass
#pragma unroll
                for (int k4 = 0; k4 < 4; ++k4) {
                  const uint32_t acc = ((kb - kb0) | k4) != 0;
                  mma_tf32(d, sdesc_sw128(xh + k4 * 32), sdesc_sw128(ll + k4 * 32), idesc, acc);
                  mma_tf32(d, sdesc_sw128(xl + k4 * 32), sdesc_sw128(lh + k4 * 32), idesc, 1);
                }
#pragma unroll
                for (int k4 = 0; k4 < 4; ++k4)
                  mma_tf32(d, sdesc_sw128(xh + k4 * 32), sdesc_sw128(lh + k4 * 32), idesc, 1);
              } else {
#pragma unroll
                for (int k4 = 0; k4 < 4; ++k4) {
                  const uint32_t acc = ((kb - kb0) | k4) != 0;
                  mma_tf32(d, sdesc_sw128(xh + k4 * 32), sdesc_sw128(lh + k4 * 32), idesc, acc);
                }
              }
              mma_commit(empty0 + 8 * st);
            }
            mma_commit(tfull0 + 8 * b);
          }
        }
      }
    }
  } else {
    const int q = warp & 3, h = (warp - 2) >> 2;
    int64_t g = 0;
    for (int64_t t = blockIdx.x; t < p.mtiles; t += gridDim.x) {
      for (int pt = p.ntp - 1; pt >= 0; --pt) {
        const int nkb = kblocks_of(pt);
        float acc[HALF];
#pragma unroll
        for (int c = 0; c < HALF; ++c) acc[c] = 0.0f;
        for (int kb0 = 0; kb0 < nkb; kb0 += kGroupKbT, ++g) {
          const int b = (int)(g & 1);
          if (ok) ok = mbar_wait(tfull0 + 8 * b, (uint32_t)((g >> 1) & 1), p.flag, 33);
          __syncwarp();
          tc_fence_after();
          const uint32_t ta = tbase + ((uint32_t)(q * 32) << 16) + b * kBM + h * HALF;
#pragma unroll
          for (int c = 0; c < HALF; c += 16) {
            float v[16];
            tmem_ld16(ta + c, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) acc[c + i] += v[i];
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(tempty0 + 8 * b);
        }
        const int64_t row = t * kBM + q * 32 + lane;
        const int col0 = pt * kBM + h * HALF;
        if (ok && row < p.rows) {
          // columns col0 .. col0 + HALF - 1 span HALF / 32 P blocks of 32
#pragma unroll
          for (int c = 0; c < HALF; ++c) {
            const int P = col0 + c;
            if (P < p.naux) {
              const int64_t e = ((int64_t)(P >> 5) * p.rows + row) * 32 + (P & 31);
              const float hv = tf32r(acc[c]);
              p.Xh[e] = hv;
              if (SPLIT == 3) p.Xl[e] = tf32r(acc[c] - hv);
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tbase, 256);
}

// -------------------------------------------------------------- J pass ---

// J[mu][nu <= mu] = sum_P w_P Bh[P][mu][nu] into packed FP64 from the TF32
// shadow (the single-pass TF32 build; the 3xTF32 build reads the FP64 B).
// Block b owns rows b and N-1-b (balanced work); a thread owns 4 consecutive
// columns of one row and streams every P (float4 loads, FP32 partial sums
// over 64 P, folded into FP64).
// Blocks are small (kJThreads) so that one fits beside a persistent SYRK CTA
// on each SM: the J pass streams HBM while the SYRK keeps the tensor cores
// busy.
constexpr int kJThreads = 128;

__global__ void __launch_bounds__(kJThreads) k_jpass_tf32(const float *__restrict__ Bh,
                                                          const float *__restrict__ w32, int naux,
                                                          int n, int ld, double *__restrict__ Jp) {
  const int b = blockIdx.x;
  const int r1 = b, r2 = n - 1 - b;
  const int c1 = r1 / 4 + 1;
  const int c2 = (r2 != r1) ? r2 / 4 + 1 : 0;
  const int64_t nn = (int64_t)n * ld;
  for (int it = blockIdx.y * blockDim.x + threadIdx.x; it < c1 + c2;
       it += gridDim.y * blockDim.x) {
    const int row = it < c1 ? r1 : r2;
    const int q = it < c1 ? it : it - c1;
    const int64_t off = (int64_t)row * ld + 4 * q;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int P0 = 0; P0 < naux; P0 += 64) {
      const int P1 = min(naux, P0 + 64);
      float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 8
      for (int P = P0; P < P1; ++P) {
        const float wp = __ldg(w32 + P);
        const float4 v = __ldg(reinterpret_cast<const float4 *>(Bh + off + P * nn));
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

// Split of C_occ: Ch[i][nu] = tf32(c), Cl[i][nu] = tf32(c - Ch) with c = fp32(C[nu][i])
// (zero padded to ldx x ld), and Cf[mu][i] = fp32 C.
__global__ void k_prep_c(const double *C, int n, int nocc, int ld, int ldx, float *Ch, float *Cl,
                         float *Cf) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t tot = (int64_t)ldx * ld;
  if (i < tot) {
    const int oi = (int)(i / ld), nu = (int)(i % ld);
    float h = 0.0f, l = 0.0f;
    if (oi < nocc && nu < n) {
      const float f = (float)C[(int64_t)nu * nocc + oi];
      h = tf32r(f);
      l = tf32r(f - h);
    }
    Ch[i] = h;
    if (Cl) Cl[i] = l;
  }
  if (i < (int64_t)n * ldx) {
    const int mu = (int)(i / ldx), oi = (int)(i % ldx);
    Cf[i] = oi < nocc ? (float)C[(int64_t)mu * nocc + oi] : 0.0f;
  }
}

// B (FP64 packed lower triangle) -> full-square split shadows Bh, Bl
// ([P][mu][ld], rows zero-padded to ld columns: TMA strides are multiples of 16 B).
__global__ void k_expand_split(const double *__restrict__ B, int n, int ld, int64_t npair, int p0,
                               int np, float *__restrict__ Bh, float *__restrict__ Bl) {
  const int64_t nn = (int64_t)n * ld;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nn * np) return;
  const int64_t P = i / nn, rc = i % nn;
  const int64_t r = rc / ld, c = rc % ld;
  float h = 0.0f, l = 0.0f;
  if (c < n) {
    const int64_t hi = r > c ? r : c, lo = r > c ? c : r;
    const float f = (float)B[(p0 + P) * npair + hi * (hi + 1) / 2 + lo];
    h = tf32r(f);
    l = tf32r(f - h);
  }
  Bh[i] = h;
  if (Bl) Bl[i] = l;
}

// ------------------------------------------------------- FP16 split prep ---

// atomicMax on non-negative floats through their bit patterns (order-preserving).
__device__ __forceinline__ void atomic_max_nonneg(unsigned *addr, float v) {
  atomicMax(addr, __float_as_uint(v));
}

// *out = max |a[i]| over n doubles (as the bits of a float; *out zeroed before).
__global__ void __launch_bounds__(256) k_absmax_f64(const double *__restrict__ a, int64_t n,
                                                    unsigned *out) {
  float m = 0.0f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    m = fmaxf(m, (float)fabs(a[i]));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomic_max_nonneg(out, m);
}

// B (FP64 packed lower triangle) -> scaled full-square FP16 split shadows:
// f = s_B B, Bh = fp16(f), Bl = fp16(f - Bh), rows zero-padded to ld.
__global__ void k_expand_split16(const double *__restrict__ B, int n, int ld, int64_t npair,
                                 int np, float sB, __half *__restrict__ Bh,
                                 __half *__restrict__ Bl) {
  const int64_t nn = (int64_t)n * ld;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nn * np) return;
  const int64_t P = i / nn, rc = i % nn;
  const int64_t r = rc / ld, c = rc % ld;
  float h = 0.0f, l = 0.0f;
  if (c < n) {
    const int64_t hi = r > c ? r : c, lo = r > c ? c : r;
    const float f = (float)(B[P * npair + hi * (hi + 1) / 2 + lo] * (double)sB);
    h = __half2float(__float2half_rn(f));
    l = f - h;
  }
  Bh[i] = __float2half_rn(h);
  Bl[i] = __float2half_rn(l);
}

// *out = max over rows of sum_c Bh[row][c]^2 (one warp per row; float bits).
__global__ void __launch_bounds__(256) k_rowsq_max16(const __half *__restrict__ Bh, int64_t rows,
                                                     int ld, unsigned *out) {
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  float best = 0.0f;
  for (int64_t r = w0; r < rows; r += nw) {
    const __half *row = Bh + r * ld;
    float s = 0.0f;
    for (int c = lane; c < ld; c += 32) {
      const float v = __half2float(row[c]);
      s = fmaf(v, v, s);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    best = fmaxf(best, s);
  }
  if (lane == 0) atomic_max_nonneg(out, best);
}

// Per-build statistics of C_occ (N x nocc, row-major): st[0] = bits of
// max|C|, st[1 + i] = sum_nu C[nu][i]^2 (float, atomically accumulated; st
// zeroed before).  Block b covers rows 32b .. 32b + 31.
__global__ void __launch_bounds__(256) k_cstats(const double *__restrict__ C, int n, int nocc,
                                                float *st) {
  const int r0 = blockIdx.x * 32, r1 = min(n, r0 + 32);
  float m = 0.0f;
  for (int i = threadIdx.x; i < nocc; i += blockDim.x) {
    float sq = 0.0f;
    for (int r = r0; r < r1; ++r) {
      const float v = (float)C[(int64_t)r * nocc + i];
      sq = fmaf(v, v, sq);
      m = fmaxf(m, fabsf(v));
    }
    atomicAdd(st + 1 + i, sq);
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomic_max_nonneg(reinterpret_cast<unsigned *>(st), m);
}

// Exponent e with x <= 2^e (x >= 0; 0 for x == 0).
__device__ __forceinline__ int ceil_exp2(double x) {
  if (!(x > 0.0)) return 0;
  int e = 0;
  const double m = frexp(x, &e);  // x = m 2^e, m in [0.5, 1)
  return m == 0.5 ? e - 1 : e;
}

// The build's scales (one thread): s_C = 2^(14 - e(max|C|)) and, from
// |X_P,mu i| <= ||B_P,mu .||_2 ||C_. i||_2 (Cauchy-Schwarz), s_X = 2^(14 - e(bound))
// with bound = rownorm * max_i ||C_. i||_2 * 1.01 (the factor covers the
// float column sums).  s_B = 2^eB_scale was fixed at setup.
__global__ void k_scales(const float *st, int nocc, int eB_scale, double rownorm,
                         MixScale *out) {
  if (threadIdx.x != 0) return;
  const float maxc = __uint_as_float(reinterpret_cast<const unsigned *>(st)[0]);
  float mc2 = 0.0f;
  for (int i = 0; i < nocc; ++i) mc2 = fmaxf(mc2, st[1 + i]);
  const int eC = 14 - ceil_exp2((double)maxc);
  const int eX = 14 - ceil_exp2(rownorm * sqrt((double)mc2) * 1.01);
  MixScale sc;
  sc.c_scale = ldexpf(1.0f, eC);
  sc.x_out = ldexpf(1.0f, eX - eB_scale - eC);
  sc.x_unscale = ldexpf(1.0f, -eB_scale - eC);
  sc.pad = 0.0f;
  sc.k_unscale = ldexp(1.0, -2 * eX);
  *out = sc;
}

// FP16 split of C_occ: Ch[i][nu] = fp16(s_C c), Cl = fp16(s_C c - Ch) with
// c = C[nu][i] (zero padded to ldx x ld), and Cf[mu][i] = fp32 C (unscaled,
// for the fused w).
__global__ void k_prep_c16(const double *C, int n, int nocc, int ld, int ldx,
                           const MixScale *sc, __half *Ch, __half *Cl, float *Cf) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t tot = (int64_t)ldx * ld;
  if (i < tot) {
    const int oi = (int)(i / ld), nu = (int)(i % ld);
    float h = 0.0f, l = 0.0f;
    if (oi < nocc && nu < n) {
      const float f = (float)(C[(int64_t)nu * nocc + oi] * (double)sc->c_scale);
      h = __half2float(__float2half_rn(f));
      l = f - h;
    }
    Ch[i] = __float2half_rn(h);
    Cl[i] = __float2half_rn(l);
  }
  if (i < (int64_t)n * ldx) {
    const int mu = (int)(i / ldx), oi = (int)(i % ldx);
    Cf[i] = oi < nocc ? (float)C[(int64_t)mu * nocc + oi] : 0.0f;
  }
}

// ------------------------------------------------------------- driver ----

static int round_up(int x, int m) { return (x + m - 1) / m * m; }

struct MixedPlan {
  int ld;        // TF32 B shadow row length (N rounded to 4)
  int ld16;      // FP16 B shadow row length (N rounded to 8: 16-byte rows)
  int ldx;       // X row length = ncg * xn
  int ncg, xn;   // X-pass column groups and tile width
  int xp_stages[2];   // [split1, split3]
  size_t xp_smem[2];
  int ntile, ntri, nchunk, ppc;
  int sy_stages[2];
  size_t sy_smem[2];
  int grid;      // persistent grid size (SM count)
};

static MixedPlan mixed_plan(int n, int naux, int nocc, int nsm) {
  MixedPlan m;
  m.grid = nsm;
  m.ld = round_up(n, 4);
  m.ld16 = round_up(n, 8);
  const int ldx0 = round_up(std::max(nocc, 1), 32);
  m.ncg = (ldx0 + 255) / 256;
  m.xn = round_up((ldx0 + m.ncg - 1) / m.ncg, 32);
  m.ldx = m.ncg * m.xn;
  // a stage holds one 128-byte k-block row per operand tile row: the same
  // bytes for TF32 (32 elements) and FP16 (64 elements)
  const size_t avail = 232448 - 1024 - 256;
  for (int k = 0; k < 2; ++k) {
    const size_t stage = (size_t)(k + 1) * (kAStage + (size_t)m.xn * 128);
    m.xp_stages[k] = (int)std::min<size_t>(8, avail / stage);
    m.xp_smem[k] = m.xp_stages[k] * stage + 1024 + 256;
    const size_t sst = (size_t)(k + 1) * 2 * kAStage;
    m.sy_stages[k] = (int)std::min<size_t>(8, avail / sst);
    m.sy_smem[k] = m.sy_stages[k] * sst + 1024 + 256;
  }
  m.ntile = (n + kBM - 1) / kBM;
  m.ntri = m.ntile * (m.ntile + 1) / 2;
  // work items (tile, aux chunk): at least two per SM, chunks of at least 16
  // aux functions, and the chunk count whose items split most evenly over
  // the persistent CTAs (the makespan is ceil(items / nsm) items)
  int nchunk = std::max(1, (nsm + m.ntri - 1) / m.ntri);
  while (nchunk * m.ntri < 2 * nsm && nchunk * 16 < naux) ++nchunk;
  {
    int best = nchunk;
    double best_eff = 0.0;
    const int cmax = std::max(2 * nchunk, nchunk + 8);
    for (int c = nchunk; c <= cmax && c * 16 <= std::max(16, naux); ++c) {
      const double items = (double)c * m.ntri;
      const double eff = items / ((double)((c * m.ntri + nsm - 1) / nsm) * nsm);
      if (eff > best_eff + 1e-3) {
        best_eff = eff;
        best = c;
      }
    }
    nchunk = best;
  }
  nchunk = std::min(nchunk, std::max(1, naux));
  m.ppc = (naux + nchunk - 1) / nchunk;
  m.nchunk = (naux + m.ppc - 1) / m.ppc;
  return m;
}

size_t mixed_workspace_bytes(int n, int naux, int nocc, int shadow) {
  const MixedPlan m = mixed_plan(n, naux, nocc, sm_count());
  size_t b = (size_t)2 * m.ncg * naux * n * 4 + (size_t)naux * 4;  // w partials, w32
  b += (size_t)m.nchunk * m.ntri * kBM * kBM * 8;                    // SYRK partials
  if (shadow == BQC_SHADOW_F16) {
    b += (size_t)2 * naux * n * m.ld16 * 2;                          // Bh16, Bl16
    b += (size_t)2 * naux * n * m.ldx * 2;                           // Xh16, Xl16
    b += (size_t)2 * m.ldx * m.ld16 * 2 + (size_t)n * m.ldx * 4;     // C split, Cf
    b += (size_t)(nocc + 1) * 4 + 256;                               // statistics, scales
    b += (size_t)kJPieces * n * (n + 1) / 2 * 8;                   // J partials of the pieces
  } else {
    b += (size_t)2 * naux * n * m.ld * 4;                            // Bh, Bl
    b += (size_t)2 * naux * n * m.ldx * 4;                           // Xh, Xl
    b += (size_t)2 * m.ldx * m.ld * 4 + (size_t)n * m.ldx * 4;       // C split, Cf
  }
  return b;
}

struct MixedState {
  MixedPlan plan;
  int shadow = BQC_SHADOW_TF32;
  CUtensorMap mapAh, mapAl, mapCh, mapCl, mapXh, mapXl;
  // split-FP16 X pass in cluster pairs: C boxes of xn / 2 rows, and the
  // number of two-CTA clusters that fit at once (0: pairs not used)
  CUtensorMap mapChH, mapClH;
  int mc_clusters = 0;
  DBuf Bl, Xl, Cl, Cf, wpart, w32;
  // FP16 split
  DBuf Bh16, Bl16, Xh16, Xl16, Ch16, Cl16, cstat, scale;
  // second X operand of the two-operand (rank-2k) K build, allocated on first use
  DBuf Yh16, Yl16, cstatB, scaleB, scaleK;
  CUtensorMap mapYh, mapYl;
  int eB = 0;            // s_B = 2^eB
  double rownorm = 0.0;  // max_{P,mu} ||B_P,mu .||_2, unscaled, with a safety factor
  size_t bytes() const {
    return Bl.n + Xl.n + Cl.n + Cf.n + wpart.n + w32.n + Bh16.n + Bl16.n + Xh16.n + Xl16.n +
           Ch16.n + Cl16.n + cstat.n + scale.n + Yh16.n + Yl16.n + cstatB.n + scaleB.n +
           scaleK.n;
  }
};

void MixedDeleter::operator()(MixedState *p) const { delete p; }

size_t mixed_bytes(const MixedState *ms) { return ms ? ms->bytes() : 0; }

int mixed_ld(int n) { return round_up(n, 4); }

#define BQC_XN_LIST(X) X(32) X(64) X(96) X(128) X(160) X(192) X(224) X(256)

template <int KIND, int XN, int SPLIT, int EPI>
static int xpass_run(size_t smem, const XpassParams *p, const CUtensorMap *Ah,
                     const CUtensorMap *Al, const CUtensorMap *Ch, const CUtensorMap *Cl, int grid,
                     cudaStream_t s) {
  if (!p) {
    BQC_CUDA_TRY(cudaFuncSetAttribute(k_xpass<KIND, XN, SPLIT, EPI>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    return BQC_OK;
  }
  k_xpass<KIND, XN, SPLIT, EPI><<<grid, kThreads, smem, s>>>(*Ah, *Al, *Ch, *Cl, *p);
  BQC_LAUNCH_CHECK();
  return BQC_OK;
}

// kind f16 exists only as the three-product split with the row epilogue.
template <int XN>
static int xpass_split_epi(int kind, int split, int epi, size_t smem, const XpassParams *p,
                           const CUtensorMap *Ah, const CUtensorMap *Al, const CUtensorMap *Ch,
                           const CUtensorMap *Cl, int grid, cudaStream_t s) {
  if (kind == kKindF16) {
    if (split != 3 || epi != 0) return BQC_E_UNSUPPORTED;
    return xpass_run<kKindF16, XN, 3, 0>(smem, p, Ah, Al, Ch, Cl, grid, s);
  }
  if (split == 3)
    return epi ? xpass_run<kKindTF32, XN, 3, 1>(smem, p, Ah, Al, Ch, Cl, grid, s)
               : xpass_run<kKindTF32, XN, 3, 0>(smem, p, Ah, Al, Ch, Cl, grid, s);
  return epi ? xpass_run<kKindTF32, XN, 1, 1>(smem, p, Ah, Ah, Ch, Ch, grid, s)
             : xpass_run<kKindTF32, XN, 1, 0>(smem, p, Ah, Ah, Ch, Ch, grid, s);
}

// p == nullptr: only set the kernel's shared-memory attribute.
static int dispatch_xn(int xn, int kind, int split, int epi, size_t smem, const XpassParams *p,
                       const CUtensorMap *Ah, const CUtensorMap *Al, const CUtensorMap *Ch,
                       const CUtensorMap *Cl, int grid, cudaStream_t s) {
#define BQC_XN_CASE(V) \
  case V:              \
    return xpass_split_epi<V>(kind, split, epi, smem, p, Ah, Al, Ch, Cl, grid, s);
  switch (xn) { BQC_XN_LIST(BQC_XN_CASE) }
#undef BQC_XN_CASE
  return BQC_E_UNSUPPORTED;
}

static int make_side_stream(Df *df, cudaStream_t s) {
  if (df->side) return BQC_OK;
  // the side stream (J) inherits the caller's priority (serving ranks
  // requests by it); the tensor-core stream runs one level above it, so that
  // the block scheduler starts a persistent tensor-core kernel's CTAs before
  // pending J blocks (otherwise J blocks fill every SM first and the two
  // passes serialise)
  int prio = 0, least = 0, greatest = 0;
  if (s && cudaStreamGetPriority(s, &prio) != cudaSuccess) {
    cudaGetLastError();
    prio = 0;
  }
  BQC_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
  BQC_CUDA_TRY(cudaStreamCreateWithPriority(&df->side, cudaStreamNonBlocking, prio));
  BQC_CUDA_TRY(cudaStreamCreateWithPriority(&df->tcs, cudaStreamNonBlocking,
                                            std::max(greatest, prio - 1)));
  BQC_CUDA_TRY(cudaEventCreateWithFlags(&df->fork, cudaEventDisableTiming));
  BQC_CUDA_TRY(cudaEventCreateWithFlags(&df->join, cudaEventDisableTiming));
  BQC_CUDA_TRY(cudaEventCreateWithFlags(&df->fork2, cudaEventDisableTiming));
  BQC_CUDA_TRY(cudaEventCreateWithFlags(&df->prep, cudaEventDisableTiming));
  for (auto &e : df->piece) BQC_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  BQC_CUDA_TRY(cudaEventCreateWithFlags(&df->tjoin, cudaEventDisableTiming));
  return BQC_OK;
}

// k_xpass_mc for a runtime tile width; p == nullptr: set its shared-memory
// attribute and count the two-CTA clusters that fit (into *clusters).
template <int XN>
static int xpass_mc_launch(size_t smem, const XpassParams *p, const MixedState *ms, int grid,
                           cudaStream_t s, int *clusters) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (!p) {
    BQC_CUDA_TRY(cudaFuncSetAttribute(k_xpass_mc<XN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
    cfg.gridDim = dim3(2 * (unsigned)sm_count());
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_xpass_mc<XN>, &cfg) != cudaSuccess) {
      cudaGetLastError();
      n = 0;
    }
    *clusters = n;
    return BQC_OK;
  }
  cfg.gridDim = dim3((unsigned)grid);
  BQC_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_xpass_mc<XN>, ms->mapAh, ms->mapAl, ms->mapChH,
                                  ms->mapClH, *p));
  return BQC_OK;
}

static int xpass_mc_dispatch(int xn, size_t smem, const XpassParams *p, const MixedState *ms,
                             int grid, cudaStream_t s, int *clusters) {
#define BQC_XN_MC(V) \
  case V:            \
    return xpass_mc_launch<V>(smem, p, ms, grid, s, clusters);
  switch (xn) { BQC_XN_LIST(BQC_XN_MC) }
#undef BQC_XN_MC
  return BQC_E_UNSUPPORTED;
}

static int xpass_mc_setup(MixedState *ms, int xn, size_t smem) {
  int n = 0;
  BQC_TRY(xpass_mc_dispatch(xn, smem, nullptr, ms, 0, nullptr, &n));
  ms->mc_clusters = n;
  return BQC_OK;
}

// FP16 split shadows of the stored B: the scale s_B from max|B| and the
// largest row norm of B (for the per-build bound on |X|), read back once.
static int mixed_setup_f16(Df *df, MixedState *ms, cudaStream_t s) {
  const Basis *b = df->basis;
  const int n = b->nbf, naux = df->naux_loc;
  const MixedPlan &m = ms->plan;
  Ctx *ctx = df->ctx;
  DBuf stat;
  BQC_TRY(stat.alloc(ctx, 256));
  BQC_CUDA_TRY(cudaMemsetAsync(stat.p, 0, 256, s));
  const int64_t nb = (int64_t)naux * df->npair;
  const unsigned grid = (unsigned)std::min<int64_t>((nb + 255) / 256, (int64_t)sm_count() * 8);
  k_absmax_f64<<<std::max(1u, grid), 256, 0, s>>>(df->B64.as<double>(), nb, stat.as<unsigned>());
  BQC_LAUNCH_CHECK();
  unsigned hb = 0;
  BQC_CUDA_TRY(cudaMemcpyAsync(&hb, stat.p, 4, cudaMemcpyDeviceToHost, s));
  BQC_CUDA_TRY(cudaStreamSynchronize(s));
  float maxb = 0.0f;
  std::memcpy(&maxb, &hb, 4);
  int e = 0;
  if (maxb > 0.0f) {
    const double mt = std::frexp((double)maxb, &e);
    if (mt == 0.5) --e;
  }
  ms->eB = 14 - e;
  const float sB = std::ldexp(1.0f, ms->eB);
  BQC_TRY(ms->Bh16.alloc(ctx, (size_t)naux * n * m.ld16 * 2));
  BQC_TRY(ms->Bl16.alloc(ctx, (size_t)naux * n * m.ld16 * 2));
  {
    const int64_t tot = (int64_t)n * m.ld16 * naux;
    k_expand_split16<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(
        df->B64.as<double>(), n, m.ld16, df->npair, naux, sB, ms->Bh16.as<__half>(),
        ms->Bl16.as<__half>());
    BQC_LAUNCH_CHECK();
  }
  BQC_CUDA_TRY(cudaMemsetAsync(stat.p, 0, 256, s));
  k_rowsq_max16<<<(unsigned)sm_count() * 8, 256, 0, s>>>(ms->Bh16.as<__half>(), (int64_t)naux * n,
                                                         m.ld16, stat.as<unsigned>());
  BQC_LAUNCH_CHECK();
  BQC_CUDA_TRY(cudaMemcpyAsync(&hb, stat.p, 4, cudaMemcpyDeviceToHost, s));
  BQC_CUDA_TRY(cudaStreamSynchronize(s));
  float maxsq = 0.0f;
  std::memcpy(&maxsq, &hb, 4);
  // |B row| <= |Bh row| / (1 - 2^-11); the factor also covers the float sums
  ms->rownorm = std::sqrt((double)maxsq) / (double)sB * (1.0 + 1.0 / 256.0);
  // float-pair B for the J pass on the FP32 pipe (8 bytes per packed
  // element, like the FP64 B it is split from)
  BQC_TRY(jpass_ff_setup(df, s));
  {  // room for the J partials of the pieces
    const int np = std::min(kJPieces, naux);
    int slices = 0;
    for (int k = 0; k < np; ++k)
      slices += jpass_split(df->npair, (int)((int64_t)naux * (k + 1) / np) -
                                           (int)((int64_t)naux * k / np));
    const size_t need =
        (size_t)std::max(jpass_split(df->npair, naux), slices) * df->npair * 8;
    if (df->Jp.n < need) BQC_TRY(df->Jp.alloc(ctx, need));
  }
  BQC_TRY(ms->Xh16.alloc(ctx, (size_t)naux * n * m.ldx * 2));
  BQC_TRY(ms->Xl16.alloc(ctx, (size_t)naux * n * m.ldx * 2));
  BQC_TRY(ms->Ch16.alloc(ctx, (size_t)m.ldx * m.ld16 * 2));
  BQC_TRY(ms->Cl16.alloc(ctx, (size_t)m.ldx * m.ld16 * 2));
  BQC_TRY(ms->cstat.alloc(ctx, (size_t)(b->nocc + 1) * 4));
  BQC_TRY(ms->scale.alloc(ctx, sizeof(MixScale)));
  {  // A operands: B shadows as (Naux*N) rows x ld16 columns
    const uint64_t dims[2] = {(uint64_t)m.ld16, (uint64_t)naux * n};
    const uint64_t str[1] = {(uint64_t)m.ld16 * 2};
    const uint32_t box[2] = {64, kBM};
    BQC_TRY(make_tmap_f16(&ms->mapAh, ms->Bh16.p, 2, dims, str, box));
    BQC_TRY(make_tmap_f16(&ms->mapAl, ms->Bl16.p, 2, dims, str, box));
  }
  {  // B operands: C^T split as ldx rows x ld16 columns, boxes of xn rows
    const uint64_t dims[2] = {(uint64_t)m.ld16, (uint64_t)m.ldx};
    const uint64_t str[1] = {(uint64_t)m.ld16 * 2};
    const uint32_t box[2] = {64, (uint32_t)m.xn};
    BQC_TRY(make_tmap_f16(&ms->mapCh, ms->Ch16.p, 2, dims, str, box));
    BQC_TRY(make_tmap_f16(&ms->mapCl, ms->Cl16.p, 2, dims, str, box));
    const uint32_t hbox[2] = {64, (uint32_t)m.xn / 2};
    BQC_TRY(make_tmap_f16(&ms->mapChH, ms->Ch16.p, 2, dims, str, hbox));
    BQC_TRY(make_tmap_f16(&ms->mapClH, ms->Cl16.p, 2, dims, str, hbox));
  }
  BQC_TRY(xpass_mc_setup(ms, m.xn, m.xp_smem[1]));
  {  // X split as (ldx, N, Naux)
    const uint64_t dims[3] = {(uint64_t)m.ldx, (uint64_t)n, (uint64_t)naux};
    const uint64_t str[2] = {(uint64_t)m.ldx * 2, (uint64_t)n * m.ldx * 2};
    const uint32_t box[3] = {64, kBM, 1};
    BQC_TRY(make_tmap_f16(&ms->mapXh, ms->Xh16.p, 3, dims, str, box));
    BQC_TRY(make_tmap_f16(&ms->mapXl, ms->Xl16.p, 3, dims, str, box));
  }
  BQC_TRY(dispatch_xn(m.xn, kKindF16, 3, 0, m.xp_smem[1], nullptr, nullptr, nullptr, nullptr,
                      nullptr, 0, s));
  BQC_CUDA_TRY(cudaFuncSetAttribute(k_syrk<kKindF16, 3>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)m.sy_smem[1]));
  return BQC_OK;
}

int mixed_setup(Df *df, int shadow, cudaStream_t s) {
  const Basis *b = df->basis;
  const int n = b->nbf, naux = df->naux_loc, no = b->nocc;
  MixedState *ms = new MixedState();
  df->mixed.reset(ms);
  ms->shadow = shadow;
  ms->plan = mixed_plan(n, naux, no, sm_count());
  const MixedPlan &m = ms->plan;
  if (m.xp_stages[1] < 2 || m.sy_stages[1] < 2) return BQC_E_UNSUPPORTED;
  BQC_TRY(make_side_stream(df, s));
  Ctx *ctx = df->ctx;
  BQC_TRY(ms->Cf.alloc(ctx, (size_t)n * m.ldx * 4));
  BQC_TRY(ms->wpart.alloc(ctx, (size_t)2 * m.ncg * naux * n * 4));
  BQC_TRY(ms->w32.alloc(ctx, (size_t)naux * 4));
  BQC_TRY(df->Kpart.alloc(ctx, (size_t)m.nchunk * m.ntri * kBM * kBM * 8));
  if (!df->Jp.p) BQC_TRY(df->Jp.alloc(ctx, (size_t)df->npair * 8));
  if (shadow == BQC_SHADOW_F16) return mixed_setup_f16(df, ms, s);
  // TF32 split shadow of B (Bh lives in df->B32)
  BQC_TRY(df->B32.alloc(ctx, (size_t)naux * n * m.ld * 4));
  BQC_TRY(ms->Bl.alloc(ctx, (size_t)naux * n * m.ld * 4));
  {
    const int64_t tot = (int64_t)n * m.ld * naux;
    k_expand_split<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(
        df->B64.as<double>(), n, m.ld, df->npair, 0, naux, df->B32.as<float>(), ms->Bl.as<float>());
    BQC_LAUNCH_CHECK();
  }
  BQC_TRY(df->X32.alloc(ctx, (size_t)naux * n * m.ldx * 4));
  BQC_TRY(ms->Xl.alloc(ctx, (size_t)naux * n * m.ldx * 4));
  BQC_TRY(df->Ct32.alloc(ctx, (size_t)m.ldx * m.ld * 4));
  BQC_TRY(ms->Cl.alloc(ctx, (size_t)m.ldx * m.ld * 4));
  {  // A operands: B shadows as (Naux*N) rows x ld columns
    const uint64_t dims[2] = {(uint64_t)m.ld, (uint64_t)naux * n};
    const uint64_t str[1] = {(uint64_t)m.ld * 4};
    const uint32_t box[2] = {32, kBM};
    BQC_TRY(make_tmap_f32(&ms->mapAh, df->B32.p, 2, dims, str, box));
    BQC_TRY(make_tmap_f32(&ms->mapAl, ms->Bl.p, 2, dims, str, box));
  }
  {  // B operands: C^T split as ldx rows x ld columns, boxes of xn rows
    const uint64_t dims[2] = {(uint64_t)m.ld, (uint64_t)m.ldx};
    const uint64_t str[1] = {(uint64_t)m.ld * 4};
    const uint32_t box[2] = {32, (uint32_t)m.xn};
    BQC_TRY(make_tmap_f32(&ms->mapCh, df->Ct32.p, 2, dims, str, box));
    BQC_TRY(make_tmap_f32(&ms->mapCl, ms->Cl.p, 2, dims, str, box));
  }
  {  // X split as (ldx, N, Naux)
    const uint64_t dims[3] = {(uint64_t)m.ldx, (uint64_t)n, (uint64_t)naux};
    const uint64_t str[2] = {(uint64_t)m.ldx * 4, (uint64_t)n * m.ldx * 4};
    const uint32_t box[3] = {32, kBM, 1};
    BQC_TRY(make_tmap_f32(&ms->mapXh, df->X32.p, 3, dims, str, box));
    BQC_TRY(make_tmap_f32(&ms->mapXl, ms->Xl.p, 3, dims, str, box));
  }
  for (int k = 0; k < 2; ++k)
    for (int epi = 0; epi < 2; ++epi)
      BQC_TRY(dispatch_xn(m.xn, kKindTF32, k ? 3 : 1, epi, m.xp_smem[k], nullptr, nullptr,
                          nullptr, nullptr, nullptr, 0, s));
  BQC_CUDA_TRY(cudaFuncSetAttribute(k_syrk<kKindTF32, 1>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)m.sy_smem[0]));
  BQC_CUDA_TRY(cudaFuncSetAttribute(k_syrk<kKindTF32, 3>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)m.sy_smem[1]));
  return BQC_OK;
}

// X pass over `rows` rows of the A operands, writing the X split (TF32 into
// Xh / Xl, FP16 into the state's Xh16 / Xl16) and, if w_out, the Coulomb
// contraction w.
static int mixed_xpass(Df *df, const double *C, int kind, int split, cudaStream_t s,
                       const CUtensorMap *Ah, const CUtensorMap *Al, int64_t rows, float *Xh,
                       float *Xl, double *w_out, int P0 = 0, int P1 = -1, bool prep = true,
                       __half *x16h = nullptr, __half *x16l = nullptr, float *cst = nullptr,
                       MixScale *scl = nullptr) {
  // rows: all rows of the A operands; the launch covers aux functions [P0, P1);
  // FP16: X into (x16h, x16l) with statistics cst and scales scl when given
  MixedState *ms = df->mixed.get();
  if (!x16h) {
    x16h = ms->Xh16.as<__half>();
    x16l = ms->Xl16.as<__half>();
    cst = ms->cstat.as<float>();
    scl = ms->scale.as<MixScale>();
  }
  const MixedPlan &m = ms->plan;
  const Basis *b = df->basis;
  const int n = b->nbf, no = b->nocc;
  if (P1 < 0) P1 = (int)(rows / n);
  if (prep && P1 > P0) df->mark(0, s);
  if (!prep) {
  } else if (kind == kKindF16) {
    const int64_t tot = std::max<int64_t>((int64_t)m.ldx * m.ld16, (int64_t)n * m.ldx);
    BQC_CUDA_TRY(cudaMemsetAsync(cst, 0, (size_t)(no + 1) * 4, s));
    k_cstats<<<(unsigned)((n + 31) / 32), 256, 0, s>>>(C, n, no, cst);
    BQC_LAUNCH_CHECK();
    k_scales<<<1, 32, 0, s>>>(cst, no, ms->eB, ms->rownorm, scl);
    BQC_LAUNCH_CHECK();
    k_prep_c16<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(
        C, n, no, m.ld16, m.ldx, scl, ms->Ch16.as<__half>(), ms->Cl16.as<__half>(),
        ms->Cf.as<float>());
    BQC_LAUNCH_CHECK();
  } else {
    const int64_t tot = std::max<int64_t>((int64_t)m.ldx * m.ld, (int64_t)n * m.ldx);
    k_prep_c<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(
        C, n, no, m.ld, m.ldx, df->Ct32.as<float>(), split == 3 ? ms->Cl.as<float>() : nullptr,
        ms->Cf.as<float>());
    BQC_LAUNCH_CHECK();
  }
  if (prep) df->mark(1, s);
  if (P1 <= P0) return BQC_OK;
  XpassParams p;
  p.row0 = (int64_t)P0 * n;
  p.rows = (int64_t)(P1 - P0) * n;
  p.wstride = rows;
  p.n = n;
  p.ldx = m.ldx;
  p.ncg = m.ncg;
  const int ke = kind == kKindF16 ? 64 : 32;
  p.kblocks = ((kind == kKindF16 ? m.ld16 : m.ld) + ke - 1) / ke;
  const int k = split == 3 ? 1 : 0;
  p.stages = m.xp_stages[k];
  p.tiles = (p.rows + kBM - 1) / kBM * m.ncg;
  p.Xh = Xh;
  p.Xl = Xl;
  p.Xh16 = kind == kKindF16 ? x16h : nullptr;
  p.Xl16 = kind == kKindF16 ? x16l : nullptr;
  p.scale = kind == kKindF16 ? scl : nullptr;
  p.Cf = ms->Cf.as<float>();
  p.wpart = ms->wpart.as<float>();
  p.flag = df->ctx->flag;
  const int grid = (int)std::min<int64_t>(m.grid, p.tiles);
  p.bk = 0;
  p.q0 = 0;
  p.bkv = 0;
  p.xrows = 0;
  const int64_t pairs = ((p.rows + kBM - 1) / kBM + 1) / 2 * m.ncg;
  if (kind == kKindF16 && ms->mc_clusters > 0 && Ah == &ms->mapAh && pairs >= 2) {
    const int g2 = 2 * (int)std::min<int64_t>(ms->mc_clusters, pairs);
    BQC_TRY(xpass_mc_dispatch(m.xn, m.xp_smem[k], &p, ms, g2, s, nullptr));
  } else {
    BQC_TRY(dispatch_xn(m.xn, kind, split, 0, m.xp_smem[k], &p, Ah, Al, &ms->mapCh, &ms->mapCl,
                        grid, s));
  }
  if (w_out) {
    k_wreduce<<<(unsigned)(P1 - P0), 256, 0, s>>>(ms->wpart.as<float>(), rows, 2 * m.ncg, n,
                                                   w_out, ms->w32.as<float>(),
                                                   w_out == df->w.as<double>() ? df->w2f.as<float2>()
                                                                               : nullptr,
                                                   P0);
    BQC_LAUNCH_CHECK();
  }
  return BQC_OK;
}

static int mixed_syrk(Df *df, int kind, int split, const CUtensorMap *Xh, const CUtensorMap *Xl,
                      int naux, double *K, cudaStream_t s, const CUtensorMap *Yh = nullptr,
                      const CUtensorMap *Yl = nullptr, const MixScale *scl = nullptr) {
  MixedState *ms = df->mixed.get();
  const MixedPlan &m = ms->plan;
  const int n = df->basis->nbf;
  SyrkParams q;
  q.n = n;
  q.ldx = m.ldx;
  q.naux = naux;
  q.ntri = m.ntri;
  q.p_per_chunk = m.ppc;
  q.nchunk = (naux + m.ppc - 1) / m.ppc;
  const int ke = kind == kKindF16 ? 64 : 32;
  q.nib = (m.ldx + ke - 1) / ke;
  const int k = split == 3 ? 1 : 0;
  q.stages = m.sy_stages[k];
  q.part = df->Kpart.as<double>();
  q.flag = df->ctx->flag;
  q.scale = kind == kKindF16 ? (scl ? scl : ms->scale.as<MixScale>()) : nullptr;
  q.mode2d = 0;
  q.npb = 0;
  q.kb_total = 0;
  q.kb_per_chunk = 0;
  q.two = Yh != nullptr;
  if (q.two && kind != kKindF16) return BQC_E_UNSUPPORTED;
  const int grid = std::min(m.grid, q.ntri * q.nchunk);
  if (kind == kKindF16)
    k_syrk<kKindF16, 3><<<grid, kThreads, m.sy_smem[1], s>>>(*Xh, *Xl, Yh ? *Yh : *Xh,
                                                             Yl ? *Yl : *Xl, q);
  else if (split == 3)
    k_syrk<kKindTF32, 3><<<grid, kThreads, m.sy_smem[1], s>>>(*Xh, *Xl, *Xh, *Xl, q);
  else
    k_syrk<kKindTF32, 1><<<grid, kThreads, m.sy_smem[0], s>>>(*Xh, *Xh, *Xh, *Xh, q);
  BQC_LAUNCH_CHECK();
  k_syrk_reduce<<<dim3((unsigned)m.ntri, kBM / 32), 256, 0, s>>>(df->Kpart.as<double>(), q.nchunk,
                                                                  m.ntri, n, K);
  BQC_LAUNCH_CHECK();
  return BQC_OK;
}

// k_unscale of a product of two differently scaled operands: 1 / (s_X s_Y),
// the square root of the product of their 1 / s^2 (exact: powers of two).
__global__ void k_scale_pair(const MixScale *a, const MixScale *b, MixScale *out) {
  if (threadIdx.x != 0) return;
  MixScale sc = *a;
  sc.k_unscale = sqrt(a->k_unscale * b->k_unscale);
  *out = sc;
}

// K = sum_P (W_P DY_P^T + DY_P W_P^T) with W_P = B_P Cw and DY_P = B_P Cd
// (both N x nocc, row-major device inputs): the exchange matrix of the
// symmetric density Cw Cd^T + Cd Cw^T, as two split-FP16 X passes and the
// SYRK kernel in its two-operand mode.  The rounding error is relative to
// |W||DY|, so a small Cd gives a small error (split-FP16 handles only).
int jk_k_rank2(Df *df, const double *Cw, const double *Cd, double *K, cudaStream_t s) {
  MixedState *ms = df->mixed.get();
  if (!ms || ms->shadow != BQC_SHADOW_F16) return BQC_E_UNSUPPORTED;
  const MixedPlan &m = ms->plan;
  const Basis *b = df->basis;
  const int n = b->nbf, naux = df->naux_loc;
  const int64_t rows = (int64_t)naux * n;
  Ctx *ctx = df->ctx;
  if (!ms->Yh16.p) {
    BQC_TRY(ms->Yh16.alloc(ctx, (size_t)naux * n * m.ldx * 2));
    BQC_TRY(ms->Yl16.alloc(ctx, (size_t)naux * n * m.ldx * 2));
    BQC_TRY(ms->cstatB.alloc(ctx, (size_t)(b->nocc + 1) * 4));
    BQC_TRY(ms->scaleB.alloc(ctx, sizeof(MixScale)));
    BQC_TRY(ms->scaleK.alloc(ctx, sizeof(MixScale)));
    const uint64_t dims[3] = {(uint64_t)m.ldx, (uint64_t)n, (uint64_t)naux};
    const uint64_t str[2] = {(uint64_t)m.ldx * 2, (uint64_t)n * m.ldx * 2};
    const uint32_t box[3] = {64, kBM, 1};
    BQC_TRY(make_tmap_f16(&ms->mapYh, ms->Yh16.p, 3, dims, str, box));
    BQC_TRY(make_tmap_f16(&ms->mapYl, ms->Yl16.p, 3, dims, str, box));
  }
  BQC_TRY(mixed_xpass(df, Cw, kKindF16, 3, s, &ms->mapAh, &ms->mapAl, rows, nullptr, nullptr,
                      nullptr));
  BQC_TRY(mixed_xpass(df, Cd, kKindF16, 3, s, &ms->mapAh, &ms->mapAl, rows, nullptr, nullptr,
                      nullptr, 0, -1, true, ms->Yh16.as<__half>(), ms->Yl16.as<__half>(),
                      ms->cstatB.as<float>(), ms->scaleB.as<MixScale>()));
  k_scale_pair<<<1, 32, 0, s>>>(ms->scale.as<MixScale>(), ms->scaleB.as<MixScale>(),
                                ms->scaleK.as<MixScale>());
  BQC_LAUNCH_CHECK();
  return mixed_syrk(df, kKindF16, 3, &ms->mapXh, &ms->mapXl, naux, K, s, &ms->mapYh, &ms->mapYl,
                    ms->scaleK.as<MixScale>());
}

// ------------------------------------------- grouped passes (serving) ---

// Small reductions of a group: one launch, blockIdx.y (w) or blockIdx.z (K)
// selects the problem; blocks past a problem's own extent return at once.
struct WredGroup {
  const float *wpart[kMaxGroup];
  double *w[kMaxGroup];
  float *w32[kMaxGroup];
  float2 *w2[kMaxGroup];
  int64_t rows[kMaxGroup];
  int nparts[kMaxGroup], n[kMaxGroup], naux[kMaxGroup];
};

__global__ void __launch_bounds__(256) k_wreduce_grp(const __grid_constant__ WredGroup g) {
  const int k = blockIdx.y;
  if ((int)blockIdx.x >= g.naux[k]) return;
  wreduce_one(g.wpart[k], g.rows[k], g.nparts[k], g.n[k], g.w[k], g.w32[k], g.w2[k], blockIdx.x);
}

struct SyRedGroup {
  const double *part[kMaxGroup];
  double *K[kMaxGroup];
  int nchunk[kMaxGroup], ntri[kMaxGroup], n[kMaxGroup];
};

__global__ void __launch_bounds__(256) k_syrk_reduce_grp(const __grid_constant__ SyRedGroup g) {
  const int k = blockIdx.z;
  if ((int)blockIdx.x >= g.ntri[k]) return;
  syrk_reduce_strip(g.part[k], g.nchunk[k], g.ntri[k], g.n[k], g.K[k], blockIdx.x, blockIdx.y);
}

static bool groupable(const Df *df) {
  const MixedState *ms = df->mixed.get();
  return df->mode == BQC_DF_STORED && ms && ms->shadow == BQC_SHADOW_F16 && !df->is_shard() &&
         df->B64.p;
}

int group_prep(Df *df, const double *C, cudaStream_t s) {
  if (!groupable(df)) {
    set_error("grouped builds need a stored, unsharded handle with FP16 shadows", __FILE__,
              __LINE__);
    return BQC_E_UNSUPPORTED;
  }
  MixedState *ms = df->mixed.get();
  const int64_t rows = (int64_t)df->naux_loc * df->basis->nbf;
  return mixed_xpass(df, C, kKindF16, 3, s, &ms->mapAh, &ms->mapAl, rows, nullptr, nullptr,
                     nullptr, 0, 0, true);
}

template <int XN>
static int xpass_grp_launch(const XGroupTab &tab, size_t smem, int grid, cudaStream_t s) {
  BQC_CUDA_TRY(cudaFuncSetAttribute(k_xpass_grp<XN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
  k_xpass_grp<XN><<<grid, kThreads, smem, s>>>(tab);
  BQC_LAUNCH_CHECK();
  return BQC_OK;
}

// X pass and w of n problems (their C split by group_prep) in one launch
// each: X into each handle's FP16 X split, w into df->w.
int group_xpass(Df *const *dfs, int n, cudaStream_t s) {
  if (n <= 0 || n > kMaxGroup) return BQC_E_INVALID;
  int xnmax = 0, naux_max = 0;
  for (int k = 0; k < n; ++k) {
    if (!groupable(dfs[k])) return BQC_E_UNSUPPORTED;
    xnmax = std::max(xnmax, dfs[k]->mixed->plan.xn);
    naux_max = std::max(naux_max, dfs[k]->naux_loc);
  }
  const int XN = xnmax <= 64 ? 64 : xnmax <= 128 ? 128 : 256;
  auto tab = std::make_unique<XGroupTab>();
  std::memset(tab.get(), 0, sizeof(XGroupTab));
  auto wr = std::make_unique<WredGroup>();
  std::memset(wr.get(), 0, sizeof(WredGroup));
  int64_t t0 = 0;
  for (int k = 0; k < n; ++k) {
    Df *df = dfs[k];
    MixedState *ms = df->mixed.get();
    const MixedPlan &m = ms->plan;
    const int nb = df->basis->nbf, naux = df->naux_loc;
    XGroupProb &q = tab->prob[k];
    q.Ah = ms->mapAh;
    q.Al = ms->mapAl;
    q.Ch = ms->mapCh;
    q.Cl = ms->mapCl;
    q.xn = m.xn;
    XpassParams &p = q.p;
    p.row0 = 0;
    p.rows = (int64_t)naux * nb;
    p.wstride = p.rows;
    p.n = nb;
    p.ldx = m.ldx;
    p.ncg = m.ncg;
    p.kblocks = (m.ld16 + 63) / 64;
    p.stages = 0;  // the group's
    p.tiles = (p.rows + kBM - 1) / kBM * m.ncg;
    p.Xh16 = ms->Xh16.as<__half>();
    p.Xl16 = ms->Xl16.as<__half>();
    p.scale = ms->scale.as<MixScale>();
    p.Cf = ms->Cf.as<float>();
    p.wpart = ms->wpart.as<float>();
    p.flag = df->ctx->flag;
    tab->tile0[k] = t0;
    t0 += p.tiles;
    wr->wpart[k] = ms->wpart.as<float>();
    wr->w[k] = df->w.as<double>();
    wr->w32[k] = ms->w32.as<float>();
    wr->w2[k] = df->w2f.as<float2>();
    wr->rows[k] = p.rows;
    wr->nparts[k] = 2 * m.ncg;
    wr->n[k] = nb;
    wr->naux[k] = naux;
  }
  tab->tile0[n] = t0;
  tab->nprob = n;
  tab->flag = dfs[0]->ctx->flag;
  const size_t stage = 2 * ((size_t)kAStage + (size_t)XN * 128);
  tab->stages = (int)std::min<size_t>(8, (232448 - 1024 - 256) / stage);
  const size_t smem = tab->stages * stage + 1024 + 256;
  const int grid = (int)std::min<int64_t>(sm_count(), t0);
  if (grid > 0) {
    if (XN == 64) BQC_TRY(xpass_grp_launch<64>(*tab, smem, grid, s));
    else if (XN == 128) BQC_TRY(xpass_grp_launch<128>(*tab, smem, grid, s));
    else BQC_TRY(xpass_grp_launch<256>(*tab, smem, grid, s));
  }
  k_wreduce_grp<<<dim3((unsigned)naux_max, (unsigned)n), 256, 0, s>>>(*wr);
  BQC_LAUNCH_CHECK();
  return BQC_OK;
}

// K of n problems from their X split (group_xpass) in one SYRK launch and
// one reduction launch.
int group_syrk(Df *const *dfs, double *const *K, int n, cudaStream_t s) {
  if (n <= 0 || n > kMaxGroup) return BQC_E_INVALID;
  auto tab = std::make_unique<SyGroupTab>();
  std::memset(tab.get(), 0, sizeof(SyGroupTab));
  auto red = std::make_unique<SyRedGroup>();
  std::memset(red.get(), 0, sizeof(SyRedGroup));
  int items = 0, ntri_max = 0;
  for (int k = 0; k < n; ++k) {
    Df *df = dfs[k];
    if (!groupable(df)) return BQC_E_UNSUPPORTED;
    MixedState *ms = df->mixed.get();
    const MixedPlan &m = ms->plan;
    SyGroupProb &g = tab->prob[k];
    g.Xh = ms->mapXh;
    g.Xl = ms->mapXl;
    SyrkParams &q = g.p;
    q.n = df->basis->nbf;
    q.ldx = m.ldx;
    q.naux = df->naux_loc;
    q.ntri = m.ntri;
    q.p_per_chunk = m.ppc;
    q.nchunk = (q.naux + m.ppc - 1) / m.ppc;
    q.nib = (m.ldx + 63) / 64;
    q.stages = 0;  // the group's
    q.part = df->Kpart.as<double>();
    q.flag = df->ctx->flag;
    q.scale = ms->scale.as<MixScale>();
    q.two = 0;
    q.mode2d = 0;
    q.npb = 0;
    q.kb_total = 0;
    q.kb_per_chunk = 0;
    tab->item0[k] = items;
    items += q.ntri * q.nchunk;
    red->part[k] = q.part;
    red->K[k] = K[k];
    red->nchunk[k] = q.nchunk;
    red->ntri[k] = q.ntri;
    red->n[k] = q.n;
    ntri_max = std::max(ntri_max, q.ntri);
  }
  tab->item0[n] = items;
  tab->nprob = n;
  tab->flag = dfs[0]->ctx->flag;
  const MixedPlan &m0 = dfs[0]->mixed->plan;  // the SYRK stage size is the same for every plan
  tab->stages = m0.sy_stages[1];
  const int grid = std::min(sm_count(), items);
  if (grid > 0) {
    BQC_CUDA_TRY(cudaFuncSetAttribute(k_syrk_grp, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)m0.sy_smem[1]));
    k_syrk_grp<<<grid, kThreads, m0.sy_smem[1], s>>>(*tab);
    BQC_LAUNCH_CHECK();
  }
  k_syrk_reduce_grp<<<dim3((unsigned)ntri_max, kBM / 32, (unsigned)n), 256, 0, s>>>(*red);
  BQC_LAUNCH_CHECK();
  return BQC_OK;
}

// w comes fused from the X pass in every mixed precision (FP32 row partials
// of X C, summed in FP64).  The J pass then runs on the side stream beside
// the tensor-core passes: the three-product builds read the packed FP64 B
// with FP64 w (FP64 FMAs), single-pass TF32 reads the TF32 shadow.  The
// precision of J matters: J = sum_P w_P B_P cancels heavily, and in a
// diffuse basis the orthogonalisation amplifies its error (by up to
// 1/sqrt(s_min)) into the DIIS error: the 22-bit split of B there set the
// mixed SCF's floor at ~2e-3, and a packed FP32 B with FP32 w at ~1e-2
// (measured), against ~1e-4 from K; with FP64 B and w the J share is
// ~3e-7.  The error of the fused w, a smooth Coulomb-like perturbation,
// stays ~1e-7.
int jk_mixed_stored(Df *df, const double *C, int prec, double *J, double *K, cudaStream_t s) {
  MixedState *ms = df->mixed.get();
  if (!ms) return BQC_E_INVALID;
  const int kind = prec == BQC_PREC_MIXED_F16X3 ? kKindF16 : kKindTF32;
  if ((kind == kKindF16) != (ms->shadow == BQC_SHADOW_F16)) {
    set_error(kind == kKindF16 ? "MIXED_F16X3 needs FP16 shadows (BQC_SHADOW_F16)"
                               : "TF32 precisions need TF32 shadows (BQC_SHADOW_TF32)",
              __FILE__, __LINE__);
    return BQC_E_INVALID;
  }
  const int split = prec == BQC_PREC_MIXED_TF32 ? 1 : 3;
  if (kind == kKindF16 && df->group) return jk_grouped(df, C, J, K, s);
  const MixedPlan &m = ms->plan;
  const Basis *b = df->basis;
  const int n = b->nbf, naux = df->naux_loc;
  const int64_t rows = (int64_t)naux * n;
  const bool j64 = split == 3 && df->B64.p;
  if (kind == kKindF16 && df->side && df->tcs && naux >= 2) {
    // The X pass in kJPieces pieces of the aux index on the tensor-core
    // stream, then the SYRK; the FP64 J pass of each piece follows it on the
    // side stream, beside the next piece (the J stream needs about as long
    // as the X pass and the SYRK together at the memory parallelism a J
    // block gets beside a persistent tensor-core CTA, so it has to start
    // early to end with them).
    const int np = std::min(kJPieces, naux);
    cudaStream_t ts = df->tcs, js = df->side;
    df->mark(0, s);
    BQC_TRY(mixed_xpass(df, C, kind, split, s, &ms->mapAh, &ms->mapAl, rows, nullptr, nullptr,
                        nullptr, 0, 0, true));  // C split and scales only (no rows)
    BQC_CUDA_TRY(cudaEventRecord(df->prep, s));
    BQC_CUDA_TRY(cudaStreamWaitEvent(ts, df->prep, 0));
    for (int k = 0; k < np; ++k) {
      const int Pa = (int)((int64_t)naux * k / np), Pb = (int)((int64_t)naux * (k + 1) / np);
      BQC_TRY(mixed_xpass(df, C, kind, split, ts, &ms->mapAh, &ms->mapAl, rows, nullptr, nullptr,
                          df->w.as<double>(), Pa, Pb, false));
      if (k == 0 && df->timing && df->ev[6]) cudaEventRecord(df->ev[6], ts);
      BQC_CUDA_TRY(cudaEventRecord(df->piece[k], ts));
    }
    df->j_from = 6;
    if (df->timing && df->ev[2]) cudaEventRecord(df->ev[2], ts);
    BQC_TRY(mixed_syrk(df, kind, split, &ms->mapXh, &ms->mapXl, naux, K, ts));
    if (df->timing && df->ev[3]) cudaEventRecord(df->ev[3], ts);
    BQC_CUDA_TRY(cudaEventRecord(df->tjoin, ts));
    int y = 0;
    for (int k = 0; k < np; ++k) {
      const int Pa = (int)((int64_t)naux * k / np), Pb = (int)((int64_t)naux * (k + 1) / np);
      BQC_CUDA_TRY(cudaStreamWaitEvent(js, df->piece[k], 0));
      if (df->B2f.p)
        BQC_TRY(jpass_ff_range(df, Pa, Pb, y, js));
      else
        BQC_TRY(jpass_fp64_range(df, Pa, Pb, y, js));
      y += jpass_split(df->npair, Pb - Pa);
    }
    BQC_TRY(jpass_unpack(df, y, J, js));
    if (df->timing && df->ev[5]) cudaEventRecord(df->ev[5], js);
    BQC_CUDA_TRY(cudaEventRecord(df->join, js));
    BQC_CUDA_TRY(cudaStreamWaitEvent(s, df->tjoin, 0));
    BQC_CUDA_TRY(cudaStreamWaitEvent(s, df->join, 0));
    df->mark(4, s);
    return BQC_OK;
  }
  BQC_TRY(mixed_xpass(df, C, kind, split, s, &ms->mapAh, &ms->mapAl, rows,
                      kind == kKindF16 ? nullptr : df->X32.as<float>(),
                      kind == kKindF16 ? nullptr : ms->Xl.as<float>(), df->w.as<double>()));
  df->mark(2, s);
  df->j_from = 2;
  cudaStream_t js = s;
  if (df->side) {
    BQC_CUDA_TRY(cudaEventRecord(df->fork, s));
    BQC_CUDA_TRY(cudaStreamWaitEvent(df->side, df->fork, 0));
    js = df->side;
  }
  if (j64) {
    BQC_TRY(jpass_fp64(df, J, js));
  } else {
    const dim3 jgrid((unsigned)((n + 1) / 2),
                     (unsigned)(((n - 1) / 4 + 2 + kJThreads - 1) / kJThreads));
    k_jpass_tf32<<<jgrid, kJThreads, 0, js>>>(df->B32.as<float>(), ms->w32.as<float>(), naux,
                                              n, m.ld, df->Jp.as<double>());
    BQC_LAUNCH_CHECK();
    k_unpack_sym2<<<(unsigned)(((int64_t)n * n + 255) / 256), 256, 0, js>>>(df->Jp.as<double>(),
                                                                             n, J);
    BQC_LAUNCH_CHECK();
  }
  if (df->timing && df->ev[5]) cudaEventRecord(df->ev[5], js);
  // the SYRK on the higher-priority tensor-core stream (forked from the
  // same point as J), so its persistent CTAs are placed before J's blocks
  cudaStream_t ks = (df->side && df->tcs) ? df->tcs : s;
  if (ks != s) BQC_CUDA_TRY(cudaStreamWaitEvent(ks, df->fork, 0));
  BQC_TRY(mixed_syrk(df, kind, split, &ms->mapXh, &ms->mapXl, naux, K, ks));
  if (df->timing && df->ev[3]) cudaEventRecord(df->ev[3], ks);
  if (ks != s) {
    BQC_CUDA_TRY(cudaEventRecord(df->tjoin, ks));
    BQC_CUDA_TRY(cudaStreamWaitEvent(s, df->tjoin, 0));
  }
  if (df->side) {
    BQC_CUDA_TRY(cudaEventRecord(df->join, df->side));
    BQC_CUDA_TRY(cudaStreamWaitEvent(s, df->join, 0));
  }
  df->mark(4, s);
  return BQC_OK;
}

}  // namespace bqc

// ------------------------------------------------- direct mode (mixed) ---

namespace bqc {

// Raw FP64 block (packed lower triangles, rows qs .. qs + nq of the block) ->
// split TF32 shadows laid out mu-major, Rh/Rl[mu][q][nu], so that the X-pass
// epilogue can write X^T[mu][i][q] with coalesced stores.  One block
// (32 x 8 threads) per 32 x 32 tile pair (I >= J) of the symmetric B_q and
// one aux row q: the packed lower triangle is read once with coalesced rows
// (tri(mu) + nu is contiguous in nu), and the tile and its mirror image are
// written through a padded shared-memory transpose, so the writes are
// coalesced too.  Rows are zero-padded to ld; rows q >= nq are zero.
__global__ void __launch_bounds__(256) k_expand_raw_mu_t(const double *__restrict__ raw,
                                                         int64_t npair, int n, int ld, int bs,
                                                         int qs, int nq, float *__restrict__ Rh,
                                                         float *__restrict__ Rl) {
  const int q = blockIdx.y;
  const int t = blockIdx.x;
  int I = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
  while ((I + 1) * (I + 2) / 2 <= t) ++I;
  while (I * (I + 1) / 2 > t) --I;
  const int J = t - I * (I + 1) / 2;
  __shared__ float th[32][33], tl[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const double *rq = raw + (int64_t)(qs + q) * npair;
#pragma unroll
  for (int r = ty; r < 32; r += 8) {
    const int mu = I * 32 + r, nu = J * 32 + tx;
    float h = 0.0f, l = 0.0f;
    if (q < nq && mu < n && nu < n) {
      const int64_t hi = mu > nu ? mu : nu, lo = mu > nu ? nu : mu;
      const float f = (float)rq[hi * (hi + 1) / 2 + lo];
      h = tf32r(f);
      l = tf32r(f - h);
    }
    th[r][tx] = h;
    tl[r][tx] = l;
  }
  __syncthreads();
  const int64_t row = (int64_t)bs * ld;
#pragma unroll
  for (int r = ty; r < 32; r += 8) {
    const int mu = I * 32 + r, nu = J * 32 + tx;
    if (mu < n && nu < ld) {
      const int64_t e = (int64_t)mu * row + (int64_t)q * ld + nu;
      Rh[e] = th[r][tx];
      if (Rl) Rl[e] = tl[r][tx];
    }
  }
  if (I != J) {
#pragma unroll
    for (int r = ty; r < 32; r += 8) {
      const int mu = J * 32 + r, nu = I * 32 + tx;
      if (mu < n && nu < ld) {
        const int64_t e = (int64_t)mu * row + (int64_t)q * ld + nu;
        Rh[e] = th[tx][r];
        if (Rl) Rl[e] = tl[tx][r];
      }
    }
  }
}

// FP64 L^{-1} (n x n) -> split shadows with rows padded to ld (zeros beyond n).
__global__ void k_split_f64(const double *__restrict__ a, int n, int ld, float *__restrict__ h,
                            float *__restrict__ l) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)n * ld) return;
  const int64_t r = i / ld, c = i % ld;
  float hv = 0.0f, lv = 0.0f;
  if (c < n) {
    const float f = (float)a[r * n + c];
    hv = tf32r(f);
    lv = tf32r(f - hv);
  }
  h[i] = hv;
  l[i] = lv;
}

struct DirectMixed {
  MixedPlan plan;      // X-pass / SYRK tile geometry (shared with stored mode)
  int bs;              // aux rows per X-pass sub-block
  int ntp;             // P tiles of the TRMM
  int tr_stages[2];
  size_t tr_smem[2];
  int64_t kb_total;    // SYRK k-blocks (ldx * naux_ld / 32)
  int naux_ld;         // Naux rounded up to 32: P blocks of X^T, row length of the L^{-1} shadows
  int sy_nchunk;
  int64_t sy_kbpc;
  CUtensorMap mapRh, mapRl, mapCh, mapCl, mapXAh, mapXAl, mapLh, mapLl, mapYh, mapYl;
  DBuf Rh, Rl, Xh, Xl, Lh, Ll, Ch, Cl, Cf, Kpart;
};

void DirectMixedDeleter::operator()(DirectMixed *p) const { delete p; }

size_t direct_mixed_bytes(int n, int naux, int nocc, int bs) {
  const MixedPlan m = mixed_plan(n, naux, nocc, sm_count());
  size_t b = (size_t)2 * n * bs * m.ld * 4;               // raw shadows of one sub-block
  const size_t nl = (size_t)round_up(naux, 4);
  b += (size_t)2 * n * m.ldx * nl * 4;                    // X^T / Y^T hi, lo
  b += (size_t)2 * naux * nl * 4;                         // L^{-1} hi, lo
  b += (size_t)3 * m.ldx * m.ld * 4;                      // C split + Cf
  b += (size_t)m.ntri * std::max(1, 2 * sm_count() / std::max(1, m.ntri)) * kBM * kBM * 8;
  return b;
}

int direct_mixed_setup(Df *df, const double *Linv, int bs, cudaStream_t s) {
  const Basis *b = df->basis;
  const int n = b->nbf, naux = b->naux, no = b->nocc;
  DirectMixed *dm = new DirectMixed();
  df->dmixed.reset(dm);
  dm->plan = mixed_plan(n, naux, no, sm_count());
  const MixedPlan &m = dm->plan;
  if (m.xp_stages[1] < 2) return BQC_E_UNSUPPORTED;
  dm->bs = bs;
  dm->ntp = (naux + kBM - 1) / kBM;
  const size_t avail = 232448 - 1024 - 256;
  for (int k = 0; k < 2; ++k) {
    const size_t st = (size_t)(k + 1) * 2 * kAStage;
    dm->tr_stages[k] = (int)std::min<size_t>(8, avail / st);
    dm->tr_smem[k] = dm->tr_stages[k] * st + 1024 + 256;
  }
  dm->naux_ld = round_up(naux, 32);
  const int nl = dm->naux_ld;
  dm->kb_total = (int64_t)m.ldx * (nl / 32);
  int nch = std::max(1, (2 * m.grid + m.ntri - 1) / m.ntri);
  nch = (int)std::min<int64_t>(nch, dm->kb_total);
  dm->sy_kbpc = (dm->kb_total + nch - 1) / nch;
  dm->sy_nchunk = (int)((dm->kb_total + dm->sy_kbpc - 1) / dm->sy_kbpc);
  Ctx *ctx = df->ctx;
  BQC_TRY(dm->Rh.alloc(ctx, (size_t)n * bs * m.ld * 4));
  BQC_TRY(dm->Rl.alloc(ctx, (size_t)n * bs * m.ld * 4));
  BQC_TRY(dm->Xh.alloc(ctx, (size_t)n * m.ldx * nl * 4));
  BQC_TRY(dm->Xl.alloc(ctx, (size_t)n * m.ldx * nl * 4));
  // padding columns (Q >= Naux) are never written and must read as zero
  BQC_CUDA_TRY(cudaMemsetAsync(dm->Xh.p, 0, dm->Xh.n, s));
  BQC_CUDA_TRY(cudaMemsetAsync(dm->Xl.p, 0, dm->Xl.n, s));
  BQC_TRY(dm->Lh.alloc(ctx, (size_t)naux * nl * 4));
  BQC_TRY(dm->Ll.alloc(ctx, (size_t)naux * nl * 4));
  BQC_TRY(dm->Ch.alloc(ctx, (size_t)m.ldx * m.ld * 4));
  BQC_TRY(dm->Cl.alloc(ctx, (size_t)m.ldx * m.ld * 4));
  BQC_TRY(dm->Cf.alloc(ctx, (size_t)n * m.ldx * 4));
  BQC_TRY(dm->Kpart.alloc(ctx, (size_t)dm->sy_nchunk * m.ntri * kBM * kBM * 8));
  {
    const int64_t nn = (int64_t)naux * nl;
    k_split_f64<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(Linv, naux, nl, dm->Lh.as<float>(),
                                                              dm->Ll.as<float>());
    BQC_LAUNCH_CHECK();
  }
  {  // raw sub-block shadows: rows (mu, q), K = nu
    const uint64_t dims[2] = {(uint64_t)m.ld, (uint64_t)n * bs};
    const uint64_t str[1] = {(uint64_t)m.ld * 4};
    const uint32_t box[2] = {32, kBM};
    BQC_TRY(make_tmap_f32(&dm->mapRh, dm->Rh.p, 2, dims, str, box));
    BQC_TRY(make_tmap_f32(&dm->mapRl, dm->Rl.p, 2, dims, str, box));
  }
  {  // C^T split
    const uint64_t dims[2] = {(uint64_t)m.ld, (uint64_t)m.ldx};
    const uint64_t str[1] = {(uint64_t)m.ld * 4};
    const uint32_t box[2] = {32, (uint32_t)m.xn};
    BQC_TRY(make_tmap_f32(&dm->mapCh, dm->Ch.p, 2, dims, str, box));
    BQC_TRY(make_tmap_f32(&dm->mapCl, dm->Cl.p, 2, dims, str, box));
  }
  // X^T is stored in P blocks of 32: [P block][i][mu][32] (rows r = i * N + mu)
  const uint64_t xrows = (uint64_t)n * m.ldx;
  {  // X^T as the TRMM A operand: rows r, K = Q in blocks
    const uint64_t dims[3] = {32, xrows, (uint64_t)(nl / 32)};
    const uint64_t str[2] = {32 * 4, xrows * 32 * 4};
    const uint32_t box[3] = {32, kBM, 1};
    BQC_TRY(make_tmap_f32(&dm->mapXAh, dm->Xh.p, 3, dims, str, box));
    BQC_TRY(make_tmap_f32(&dm->mapXAl, dm->Xl.p, 3, dims, str, box));
  }
  {  // L^{-1}: rows P, K = Q
    const uint64_t dims[2] = {(uint64_t)naux, (uint64_t)naux};
    const uint64_t str[1] = {(uint64_t)nl * 4};
    const uint32_t box[2] = {32, kBM};
    BQC_TRY(make_tmap_f32(&dm->mapLh, dm->Lh.p, 2, dims, str, box));
    BQC_TRY(make_tmap_f32(&dm->mapLl, dm->Ll.p, 2, dims, str, box));
  }
  {  // Y^T as the SYRK operand: rows mu, K = (i, P block, P % 32)
    const uint64_t dims[4] = {32, (uint64_t)n, (uint64_t)m.ldx, (uint64_t)(nl / 32)};
    const uint64_t str[3] = {32 * 4, (uint64_t)n * 32 * 4, xrows * 32 * 4};
    const uint32_t box[4] = {32, kBM, 1, 1};
    BQC_TRY(make_tmap_f32(&dm->mapYh, dm->Xh.p, 4, dims, str, box));
    BQC_TRY(make_tmap_f32(&dm->mapYl, dm->Xl.p, 4, dims, str, box));
  }
  for (int k = 0; k < 2; ++k)
    BQC_TRY(dispatch_xn(m.xn, kKindTF32, k ? 3 : 1, 1, m.xp_smem[k], nullptr, nullptr, nullptr,
                        nullptr, nullptr, 0, s));
  BQC_CUDA_TRY(cudaFuncSetAttribute(k_trmm_tf32<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)dm->tr_smem[0]));
  BQC_CUDA_TRY(cudaFuncSetAttribute(k_trmm_tf32<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)dm->tr_smem[1]));
  BQC_CUDA_TRY(cudaFuncSetAttribute(k_syrk<kKindTF32, 1>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)m.sy_smem[0]));
  BQC_CUDA_TRY(cudaFuncSetAttribute(k_syrk<kKindTF32, 3>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)m.sy_smem[1]));
  return BQC_OK;
}

int direct_mixed_prep_c(Df *df, const double *C, int split, cudaStream_t s) {
  DirectMixed *dm = df->dmixed.get();
  const MixedPlan &m = dm->plan;
  const int n = df->basis->nbf, no = df->basis->nocc;
  const int64_t tot = std::max<int64_t>((int64_t)m.ldx * m.ld, (int64_t)n * m.ldx);
  k_prep_c<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(
      C, n, no, m.ld, m.ldx, dm->Ch.as<float>(), split == 3 ? dm->Cl.as<float>() : nullptr,
      dm->Cf.as<float>());
  BQC_LAUNCH_CHECK();
  return BQC_OK;
}

// X^T[mu][i][q0 + q] = sum_nu raw[q][mu nu] C[nu][i] for the nq aux rows of a
// packed FP64 raw block (in sub-blocks of bs rows).
int direct_mixed_block(Df *df, const double *raw, int q0, int nq, int split, cudaStream_t s) {
  DirectMixed *dm = df->dmixed.get();
  const MixedPlan &m = dm->plan;
  const int n = df->basis->nbf;
  const int k = split == 3 ? 1 : 0;
  for (int qs = 0; qs < nq; qs += dm->bs) {
    const int nv = std::min(dm->bs, nq - qs);
    const int nt = (m.ld + 31) / 32;
    k_expand_raw_mu_t<<<dim3((unsigned)(nt * (nt + 1) / 2), (unsigned)dm->bs), 256, 0, s>>>(
        raw, df->npair, n, m.ld, dm->bs, qs, nv, dm->Rh.as<float>(),
        split == 3 ? dm->Rl.as<float>() : nullptr);
    BQC_LAUNCH_CHECK();
    XpassParams p;
    p.rows = (int64_t)n * dm->bs;
    p.row0 = 0;
    p.wstride = p.rows;
    p.n = n;
    p.ldx = m.ldx;
    p.ncg = m.ncg;
    p.kblocks = (m.ld + 31) / 32;
    p.stages = m.xp_stages[k];
    p.tiles = (p.rows + kBM - 1) / kBM * m.ncg;
    p.Xh = dm->Xh.as<float>();
    p.Xl = dm->Xl.as<float>();
    p.Cf = dm->Cf.as<float>();
    p.wpart = nullptr;
    p.flag = df->ctx->flag;
    p.bk = dm->bs;
    p.q0 = q0 + qs;
    p.bkv = nv;
    p.xrows = (int64_t)n * m.ldx;
    const int grid = (int)std::min<int64_t>(m.grid, p.tiles);
    p.Xh16 = nullptr;
    p.Xl16 = nullptr;
    p.scale = nullptr;
    BQC_TRY(dispatch_xn(m.xn, kKindTF32, split, 1, m.xp_smem[k], &p, &dm->mapRh, &dm->mapRl,
                        &dm->mapCh, &dm->mapCl, grid, s));
  }
  return BQC_OK;
}

// After all blocks: Y = L^{-1} X in place on X^T, then K = sum_{P,i} Y Y^T.
int direct_mixed_finish(Df *df, int split, double *K, cudaStream_t s) {
  DirectMixed *dm = df->dmixed.get();
  const MixedPlan &m = dm->plan;
  const int n = df->basis->nbf, naux = df->basis->naux;
  const int k = split == 3 ? 1 : 0;
  TrmmParams t;
  t.rows = (int64_t)n * m.ldx;
  t.naux = naux;
  t.ntp = dm->ntp;
  t.stages = dm->tr_stages[k];
  t.mtiles = (t.rows + kBM - 1) / kBM;
  t.Xh = dm->Xh.as<float>();
  t.Xl = dm->Xl.as<float>();
  t.flag = df->ctx->flag;
  const int tg = (int)std::min<int64_t>(m.grid, t.mtiles);
  if (split == 3)
    k_trmm_tf32<3><<<tg, kThreads, dm->tr_smem[1], s>>>(dm->mapXAh, dm->mapXAl, dm->mapLh,
                                                        dm->mapLl, t);
  else
    k_trmm_tf32<1><<<tg, kThreads, dm->tr_smem[0], s>>>(dm->mapXAh, dm->mapXAh, dm->mapLh,
                                                        dm->mapLh, t);
  BQC_LAUNCH_CHECK();
  SyrkParams q;
  q.n = n;
  q.ldx = m.ldx;
  q.naux = naux;
  q.ntri = m.ntri;
  q.nchunk = dm->sy_nchunk;
  q.p_per_chunk = 0;
  q.nib = m.ldx / 32;
  q.stages = m.sy_stages[k];
  q.part = dm->Kpart.as<double>();
  q.flag = df->ctx->flag;
  q.mode2d = 1;
  q.npb = dm->naux_ld / 32;
  q.kb_total = dm->kb_total;
  q.kb_per_chunk = dm->sy_kbpc;
  q.scale = nullptr;
  q.two = 0;
  const int grid = std::min(m.grid, q.ntri * q.nchunk);
  if (split == 3)
    k_syrk<kKindTF32, 3><<<grid, kThreads, m.sy_smem[1], s>>>(dm->mapYh, dm->mapYl, dm->mapYh,
                                                             dm->mapYl, q);
  else
    k_syrk<kKindTF32, 1><<<grid, kThreads, m.sy_smem[0], s>>>(dm->mapYh, dm->mapYh, dm->mapYh,
                                                             dm->mapYh, q);
  BQC_LAUNCH_CHECK();
  k_syrk_reduce<<<dim3((unsigned)m.ntri, kBM / 32), 256, 0, s>>>(dm->Kpart.as<double>(),
                                                                  q.nchunk, m.ntri, n, K);
  BQC_LAUNCH_CHECK();
  return BQC_OK;
}

}  // namespace bqc

// ------------------------------------------- bounded-wait self-test -----

namespace bqc {

// One thread waits on an mbarrier that nothing ever arrives on, through the
// same bounded wait the tensor-core kernels use; the wait gives up after
// `limit` clocks and records code 99 in the context's device flag.
__global__ void k_wait_selftest(int *flag, long long limit) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    fence_barrier_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_wait(smem_u32(&bar), 0, flag, 99, limit);
}

}  // namespace bqc

extern "C" int bqc_wait_selftest(bqc_ctx *ctx, long long cycles, bqc_stream_t stream) {
  if (!ctx || cycles <= 0 || cycles > 4000000000LL) return BQC_E_INVALID;
  BQC_CUDA_TRY(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  bqc::k_wait_selftest<<<1, 32, 0, s>>>(ctx->flag, cycles);
  BQC_LAUNCH_CHECK();
  return ctx->check_flag(s);
}

// ----------------------------------------------------- DF-MP2 pair GEMMs --

namespace bqc {

// Bt ([P][q], q = (i, a), FP64) -> A[q][P] = split FP16 of s * Bt, the rows
// of (ia|jb)'s K-major operands (P padded with zeros to ldp), through a
// 32 x 32 shared-memory transpose (coalesced reads over q, writes over P).
__global__ void k_transpose_split16(const double *__restrict__ Bt, int naux, int64_t Q, int ldp,
                                    double scale, __half *__restrict__ Ah,
                                    __half *__restrict__ Al) {
  __shared__ float t[32][33];
  const int64_t q0 = (int64_t)blockIdx.x * 32;
  const int p0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int P = p0 + r;
    const int64_t q = q0 + threadIdx.x;
    t[r][threadIdx.x] = (P < naux && q < Q) ? (float)(Bt[(int64_t)P * Q + q] * scale) : 0.0f;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t q = q0 + r;
    const int P = p0 + threadIdx.x;
    if (q < Q && P < ldp) {
      const float f = t[threadIdx.x][r];
      const __half h = __float2half_rn(f);
      Ah[q * ldp + P] = h;
      Al[q * ldp + P] = __float2half_rn(f - __half2float(h));
    }
  }
}

struct Mp2Tc {
  int naux = 0, ldp = 0;
  int64_t Q = 0;
  double inv_scale2 = 1.0;
  int stages = 0;
  size_t smem = 0;
  DBuf Ah, Al;
  CUtensorMap mapAh, mapAl;
};

void Mp2TcDeleter::operator()(Mp2Tc *p) const { delete p; }

int mp2_tc_setup(Ctx *ctx, const double *Bt, int naux, int nocc, int nv, int *flag,
                 std::unique_ptr<Mp2Tc, Mp2TcDeleter> &out, cudaStream_t s) {
  Mp2Tc *m = new Mp2Tc();
  out.reset(m);
  m->naux = naux;
  m->Q = (int64_t)nocc * nv;
  m->ldp = round_up(naux, 8);
  // scale: largest |B_P,ia| to at most 2^14
  DBuf stat;
  BQC_TRY(stat.alloc(ctx, 256));
  BQC_CUDA_TRY(cudaMemsetAsync(stat.p, 0, 256, s));
  const int64_t nb = (int64_t)naux * m->Q;
  const unsigned grid = (unsigned)std::min<int64_t>((nb + 255) / 256, (int64_t)sm_count() * 8);
  k_absmax_f64<<<std::max(1u, grid), 256, 0, s>>>(Bt, nb, stat.as<unsigned>());
  BQC_LAUNCH_CHECK();
  unsigned hb = 0;
  BQC_CUDA_TRY(cudaMemcpyAsync(&hb, stat.p, 4, cudaMemcpyDeviceToHost, s));
  BQC_CUDA_TRY(cudaStreamSynchronize(s));
  float mx = 0.0f;
  std::memcpy(&mx, &hb, 4);
  int e = 0;
  if (mx > 0.0f) {
    const double mt = std::frexp((double)mx, &e);
    if (mt == 0.5) --e;
  }
  const double sc = std::ldexp(1.0, 14 - e);
  m->inv_scale2 = 1.0 / (sc * sc);
  BQC_TRY(m->Ah.alloc(ctx, (size_t)m->Q * m->ldp * 2));
  BQC_TRY(m->Al.alloc(ctx, (size_t)m->Q * m->ldp * 2));
  k_transpose_split16<<<dim3((unsigned)((m->Q + 31) / 32), (unsigned)((m->ldp + 31) / 32)),
                        dim3(32, 8), 0, s>>>(Bt, naux, m->Q, m->ldp, sc, m->Ah.as<__half>(),
                                             m->Al.as<__half>());
  BQC_LAUNCH_CHECK();
  const uint64_t dims[2] = {(uint64_t)m->ldp, (uint64_t)m->Q};
  const uint64_t str[1] = {(uint64_t)m->ldp * 2};
  const uint32_t box[2] = {64, kBM};
  BQC_TRY(make_tmap_f16(&m->mapAh, m->Ah.p, 2, dims, str, box));
  BQC_TRY(make_tmap_f16(&m->mapAl, m->Al.p, 2, dims, str, box));
  const size_t avail = 232448 - 1024 - 256;
  m->stages = (int)std::min<size_t>(8, avail / (4 * kAStage));
  m->smem = (size_t)m->stages * 4 * kAStage + 1024 + 256;
  BQC_CUDA_TRY(cudaFuncSetAttribute(k_gemm_nt<kKindF16>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)m->smem));
  (void)flag;
  return BQC_OK;
}

// V[(ii, a)][(jj, b)] = sum_P B_P,(i0+ii) a B_P,(j0+jj) b for ni x nj occupied
// orbitals, FP64 out (ldv), from the split FP16 operand.
int mp2_tc_block(Mp2Tc *m, int nv, int i0, int ni, int j0, int nj, double *V, int64_t ldv,
                 int *flag, cudaStream_t s) {
  GemmNtParams p;
  p.mvalid = ni * nv;
  p.nvalid = nj * nv;
  p.mt = (p.mvalid + kBM - 1) / kBM;
  p.nt = (p.nvalid + kBM - 1) / kBM;
  p.a_row0 = (int64_t)i0 * nv;
  p.b_row0 = (int64_t)j0 * nv;
  p.kblocks = (m->ldp + 63) / 64;
  p.stages = m->stages;
  p.out = V;
  p.ldo = ldv;
  p.scale = m->inv_scale2;
  p.flag = flag;
  const int grid = std::min(sm_count(), p.mt * p.nt);
  k_gemm_nt<kKindF16><<<grid, kThreads, m->smem, s>>>(m->mapAh, m->mapAl, m->mapAh, m->mapAl, p);
  BQC_LAUNCH_CHECK();
  return BQC_OK;
}

}  // namespace bqc
