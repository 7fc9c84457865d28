// Gaussian integrals on the GPU: Boys function, Obara-Saika / Head-Gordon-Pople
// recursions for the three-centre (P|mu nu) Cholesky-decomposed ERIs (CD-ERIs) of
// the density-fitted mean field (Sec. 2.2), the Coulomb metric (P|Q), the
// Schwarz diagonals (mu nu|mu nu) and the one-electron matrices.
//
// Design (GB300): FP64 throughput on this part is ~1/64 of FP32, so the
// kernels are DFMA-bound.  One shell quartet is processed by a group of G
// lanes of a warp; each recursion level is a set of independent entries that
// the G lanes split, with the level tables in shared memory (the paper's
// local-memory problem for high angular momentum, Sec. 2.2.2 item 1, does not
// arise: nothing spills).  G is chosen per class from the table size, so
// small classes run one quartet per lane and (f|dd) runs 16-32 lanes on one.
//
// Recursions (Obara & Saika 1986; Head-Gordon & Pople 1988), with
// p = a+b, q = c+d, rho = pq/(p+q), W = (pP + qQ)/(p+q):
//   [e+1_i|f]^m = PA_i [e|f]^m + WP_i [e|f]^{m+1}
//                 + e_i/(2p) ([e-1_i|f]^m - rho/p [e-1_i|f]^{m+1}),      (f = 0)
//   [e|f+1_i]^m = QC_i [e|f]^m + WQ_i [e|f]^{m+1}
//                 + f_i/(2q) ([e|f-1_i]^m - rho/q [e|f-1_i]^{m+1})
//                 + e_i/(2(p+q)) [e-1_i|f]^{m+1},
//   [0|0]^m = 2 pi^{5/2} / (p q sqrt(p+q)) K_ab K_cd F_m(rho |PQ|^2),
//   (a, b+1_i| = (a+1_i, b| + AB_i (a, b|   (and likewise on the ket).
// The three-centre integral is the case d = s with exponent 0 at C; the
// nuclear attraction is the point-charge limit q -> infinity of the same
// recursion.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cub/cub.cuh>
#include <type_traits>
#include <vector>

#include "bqc_internal.h"
#include "os_eri.cuh"

namespace bqc {
// ------------------------------------------------------------ Boys -------

// F_m(T) at the grid points from the power series
// F_m(T) = exp(-T) sum_k (2T)^k / ((2m+1)(2m+3)...(2m+2k+1)), summed in long
// double; the device evaluates F_m by an 8-term Taylor expansion about the
// nearest grid point (dF_m/dT = -F_{m+1}), and for T >= 36 by
// F_0 = sqrt(pi/T)/2 with the upward recursion F_{m+1} = ((2m+1)F_m - e^{-T})/(2T).
int boys_table_build(Ctx *ctx) {
  std::vector<double> tab((size_t)kBoysNT * kBoysNM);
  for (int k = 0; k < kBoysNT; ++k) {
    const long double T = (long double)k * kBoysH;
    for (int m = 0; m < kBoysNM; ++m) {
      long double den = 2.0L * m + 1.0L, term = 1.0L / den, sum = term;
      for (int t = 1; t < 4000; ++t) {
        term *= 2.0L * T / (den + 2.0L * t);
        sum += term;
        if (term < 1e-22L * sum) break;
      }
      tab[(size_t)k * kBoysNM + m] = (double)(expl(-T) * sum);
    }
  }
  void *p = ctx->dmalloc(tab.size() * sizeof(double));
  if (!p) return BQC_E_OOM;
  ctx->boys = (double *)p;
  BQC_CUDA_TRY(cudaMemcpy(ctx->boys, tab.data(), tab.size() * sizeof(double),
                          cudaMemcpyHostToDevice));
  return upload_cart_tables();
}

__global__ void k_boys_eval(const double *__restrict__ tab, int n, const double *__restrict__ T,
                            int mmax, double *__restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= (int64_t)n * (mmax + 1)) return;
  const int64_t t = i / (mmax + 1);
  const int m = (int)(i - t * (mmax + 1));
  const double x = T[t];
  const double e = x >= kBoysTCut ? exp(-x) : 0.0;
  out[i] = boys_one(tab, m, x, e);
}

int launch_boys_eval(Ctx *ctx, int n, const double *T, int mmax, double *out, cudaStream_t s) {
  if (n < 0 || mmax < 0 || mmax > kBoysMaxM) return BQC_E_INVALID;
  if (n == 0) return BQC_OK;
  const int64_t tot = (int64_t)n * (mmax + 1);
  k_boys_eval<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(ctx->boys, n, T, mmax, out);
  BQC_LAUNCH_CHECK();
  return BQC_OK;
}

// ------------------------------------------------ three-centre kernel ----

// Shipped compaction: pairs of a class sorted by decreasing Schwarz factor,
// so the survivors of aux shell P are the prefix [0, cut_P) of the list; the
// scanned cuts map a dense triplet index t onto (P, pair) by binary search,
// and every lane computes a surviving triplet (no test, no divergence).
template <int LC, int LA, int LB>
__global__ void __launch_bounds__(256) k_eri3c(Eri3cArgs a) {
  using O = Os<LA, LB, LC, 0>;
  constexpr int G = O::G;
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31;
  const int gl = lane % G;
  const int group_in_block = threadIdx.x / G;
  const int groups_per_block = blockDim.x / G;
  double *scr = smem + (size_t)group_in_block * O::SCR;
  // triplet index space of this launch: [prefix[0], prefix[n_aux]) (a window
  // of aux shells may start past the first shell of the l-list)
  const int64_t pbase = a.prefix[0];
  const int64_t total = a.prefix[a.n_aux] - pbase;
  const int64_t gstride = (int64_t)gridDim.x * groups_per_block;
  // warp-uniform trip count: all groups of a warp iterate together
  const int warp_first_group = (threadIdx.x >> 5) * (32 / G);
  const int64_t base0 = (int64_t)blockIdx.x * groups_per_block + warp_first_group;
  for (int64_t base = base0; base < total; base += gstride) {
    int64_t t = base + (group_in_block - warp_first_group);
    const bool active = t < total;
    if (!active) t = total - 1;
    t += pbase;
    // aux shell: largest i with prefix[i] <= t
    int lo = 0, hi = a.n_aux;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (a.prefix[mid] <= t) lo = mid; else hi = mid;
    }
    eri3c_triplet<LC, LA, LB>(a, scr, gl, a.aux_list[lo], a.pairs[t - a.prefix[lo]], active);
    __syncwarp();
  }
}

template <int LC, int LA, int LB>
static int launch3(const Eri3cArgs &a, int64_t total, cudaStream_t s) {
  using O = Os<LA, LB, LC, 0>;
  constexpr int G = O::G;
  // groups per block: up to 256 threads and ~196 KB of tables
  int groups = 256 / G;
  while (groups > 32 / G && (size_t)groups * O::SCR * 8 > 196 * 1024) groups -= 32 / G;
  const size_t smem = (size_t)groups * O::SCR * 8;
  if (smem > 227 * 1024) return BQC_E_UNSUPPORTED;
  auto kern = k_eri3c<LC, LA, LB>;
  BQC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
  int64_t blocks = (total + groups - 1) / groups;
  blocks = std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)sm_count() * 16));
  kern<<<(unsigned)blocks, groups * G, smem, s>>>(a);
  BQC_LAUNCH_CHECK();
  return BQC_OK;
}

template <int LC>
static int dispatch3_pair(int cls, const Eri3cArgs &a, int64_t total, cudaStream_t s) {
  switch (cls) {
    case 0: return launch3<LC, 0, 0>(a, total, s);
    case 1: return launch3<LC, 1, 0>(a, total, s);
    case 2: return launch3<LC, 1, 1>(a, total, s);
    case 3: return launch3<LC, 2, 0>(a, total, s);
    case 4: return launch3<LC, 2, 1>(a, total, s);
    case 5: return launch3<LC, 2, 2>(a, total, s);
  }
  return BQC_E_UNSUPPORTED;
}

static int dispatch3(int lc, int cls, const Eri3cArgs &a, int64_t total, cudaStream_t s) {
  switch (lc) {
    case 0: return dispatch3_pair<0>(cls, a, total, s);
    case 1: return dispatch3_pair<1>(cls, a, total, s);
    case 2: return dispatch3_pair<2>(cls, a, total, s);
    case 3: return dispatch3_pair<3>(cls, a, total, s);
  }
  return BQC_E_UNSUPPORTED;
}

// The loop-buffer and index-list variants (eri3c_ablation.cu).
int dispatch3v(int lc, int cls, const Eri3cArgs &a, int64_t total, int v, cudaStream_t s);

int launch_eri3c(const Basis *b, const Eri3cPlan *plan, int p0, int p1, double *out, int64_t ld,
                 cudaStream_t s) {
  return launch_eri3c_variant(b, plan, p0, p1, out, ld, 0, s);
}

int launch_eri3c_variant(const Basis *b, const Eri3cPlan *plan, int p0, int p1, double *out,
                         int64_t ld, int variant, cudaStream_t s) {
  if (p0 < 0 || p1 > b->naux || p0 > p1 || variant < 0 || variant > 2) return BQC_E_INVALID;
  if (p0 == p1) return BQC_OK;
  DBuf list, count;
  if (variant == 2) {
    int64_t maxc = 0;
    for (int lc = 0; lc <= kMaxLAux; ++lc)
      for (int cls = 0; cls < kNPairClass; ++cls)
        maxc = std::max<int64_t>(maxc, (int64_t)(b->auxl_off[lc + 1] - b->auxl_off[lc]) *
                                           (b->pair_off[cls + 1] - b->pair_off[cls]));
    BQC_TRY(list.alloc(b->ctx, (size_t)std::max<int64_t>(1, maxc) * 8));
    BQC_TRY(count.alloc(b->ctx, 8));
  }
  for (int lc = 0; lc <= kMaxLAux; ++lc) {
    const int na = b->auxl_off[lc + 1] - b->auxl_off[lc];
    if (na == 0) continue;
    // shells of this l whose functions meet [p0, p1): a contiguous sub-range
    // [s0, s1) of the l-list, since function offsets grow with shell index
    int s0 = 0, s1 = 0;
    {
      int k = 0;
      s0 = -1;
      for (int sh = 0; sh < (int)b->aux.l.size(); ++sh) {
        if (b->aux.l[sh] != lc) continue;
        const int f0 = b->aux.fn[sh], f1 = f0 + (lc + 1) * (lc + 2) / 2;
        if (f1 > p0 && f0 < p1) {
          if (s0 < 0) s0 = k;
          s1 = k + 1;
        }
        ++k;
      }
      if (s0 < 0) continue;
    }
    for (int cls = 0; cls < kNPairClass; ++cls) {
      const int np = b->pair_off[cls + 1] - b->pair_off[cls];
      if (np == 0 || plan->total[cls][lc] == 0) continue;
      const int64_t *hp = plan->h_prefix.data() + plan->prefix_off[cls][lc];
      const int64_t ntrip = hp[s1] - hp[s0];
      if (ntrip == 0) continue;
      Eri3cArgs a;
      a.orb = b->orb.dev;
      a.aux = b->aux.dev;
      a.boys = b->ctx->boys;
      a.pairs = plan->d_pairs_sorted.as<int2>() + b->pair_off[cls];
      a.aux_list = b->d_aux_by_l.as<int>() + b->auxl_off[lc] + s0;
      a.prefix = plan->d_prefix.as<int64_t>() + plan->prefix_off[cls][lc] + s0;
      a.n_aux = s1 - s0;
      a.p0 = p0;
      a.p1 = p1;
      a.out = out;
      a.ld = ld;
      a.flag = b->ctx->flag;
      a.out_elems = (int64_t)(p1 - p0) * ld;
      a.pairs_orig = b->d_pairs.as<int2>() + b->pair_off[cls];
      a.qpair_orig = plan->d_qpair.as<double>() + b->pair_off[cls];
      a.qaux = plan->d_qaux.as<double>();
      a.tau = plan->tau;
      a.np = np;
      a.list = list.as<int64_t>();
      a.count = count.as<unsigned long long>();
      if (variant == 0)
        BQC_TRY(dispatch3(lc, cls, a, ntrip, s));
      else
        BQC_TRY(dispatch3v(lc, cls, a, ntrip, variant, s));
    }
  }
  if (variant == 2) BQC_CUDA_TRY(cudaStreamSynchronize(s));  // before the list is released
  return BQC_OK;
}

// ------------------------------------------------------ Schwarz kernel ---

struct SchwarzArgs {
  ShellSetDev orb;
  const double *boys;
  const int2 *pairs;
  int npair;
  double *Q;
};

template <int LA, int LB>
__global__ void __launch_bounds__(256) k_schwarz(SchwarzArgs a) {
  using O = Os<LA, LB, LA, LB>;
  constexpr int G = O::G;
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31, gl = lane % G;
  const int gib = threadIdx.x / G, gpb = blockDim.x / G;
  double *scr = smem + (size_t)gib * O::SCR;
  const int wfg = (threadIdx.x >> 5) * (32 / G);
  for (int64_t base = (int64_t)blockIdx.x * gpb + wfg; base < a.npair;
       base += (int64_t)gridDim.x * gpb) {
    int64_t t = base + (gib - wfg);
    const bool active = t < a.npair;
    if (!active) t = a.npair - 1;
    const int2 pr = a.pairs[t];
    const ShellRef sa = load_shell(a.orb, pr.x), sb = load_shell(a.orb, pr.y);
    const double *ea = a.orb.exps + sa.poff, *ca = a.orb.coefs + sa.poff;
    const double *eb = a.orb.exps + sb.poff, *cb = a.orb.coefs + sb.poff;
    const double *res =
        os_quartet<LA, LB, LA, LB, G>(a.boys, scr, gl, sa, ea, ca, &sb, eb, cb, sa, ea, ca, &sb,
                                      eb, cb);
    if (active && gl == 0) {
      constexpr int NA = ncart(LA), NB = ncart(LB);
      double mx = 0.0;
      for (int ia = 0; ia < NA; ++ia)
        for (int ib = 0; ib < NB; ++ib) {
          const double n = c_cnorm[ncum(LA) + ia] * c_cnorm[ncum(LB) + ib];
          const double v = res[((ia * NB + ib) * NA + ia) * NB + ib] * n * n;
          mx = fmax(mx, fabs(v));
        }
      a.Q[t] = sqrt(mx);
    }
    __syncwarp();
  }
}

template <int LA, int LB>
static int launch_schwarz_cls(const SchwarzArgs &a, cudaStream_t s) {
  using O = Os<LA, LB, LA, LB>;
  constexpr int G = O::G;
  int groups = 256 / G;
  while (groups > 32 / G && (size_t)groups * O::SCR * 8 > 196 * 1024) groups -= 32 / G;
  const size_t smem = (size_t)groups * O::SCR * 8;
  if (smem > 227 * 1024) return BQC_E_UNSUPPORTED;
  auto kern = k_schwarz<LA, LB>;
  BQC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
  int64_t blocks = (a.npair + groups - 1) / groups;
  blocks = std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)sm_count() * 16));
  kern<<<(unsigned)blocks, groups * G, smem, s>>>(a);
  BQC_LAUNCH_CHECK();
  return BQC_OK;
}

int launch_schwarz_pairs(const Basis *b, double *Qpair, cudaStream_t s) {
  for (int cls = 0; cls < kNPairClass; ++cls) {
    const int np = b->pair_off[cls + 1] - b->pair_off[cls];
    if (np == 0) continue;
    SchwarzArgs a;
    a.orb = b->orb.dev;
    a.boys = b->ctx->boys;
    a.pairs = b->d_pairs.as<int2>() + b->pair_off[cls];
    a.npair = np;
    a.Q = Qpair + b->pair_off[cls];
    int st = BQC_E_UNSUPPORTED;
    switch (cls) {
      case 0: st = launch_schwarz_cls<0, 0>(a, s); break;
      case 1: st = launch_schwarz_cls<1, 0>(a, s); break;
      case 2: st = launch_schwarz_cls<1, 1>(a, s); break;
      case 3: st = launch_schwarz_cls<2, 0>(a, s); break;
      case 4: st = launch_schwarz_cls<2, 1>(a, s); break;
      case 5: st = launch_schwarz_cls<2, 2>(a, s); break;
    }
    BQC_TRY(st);
  }
  return BQC_OK;
}

// ------------------------------------------------------- metric (P|Q) ----

struct Int2cArgs {
  ShellSetDev aux;
  const double *boys;
  const int *listP, *listQ;
  int nP, nQ;
  double *V;
  int naux;
};

template <int LP, int LQ>
__global__ void __launch_bounds__(256) k_int2c(Int2cArgs a) {
  using O = Os<LP, 0, LQ, 0>;
  constexpr int G = O::G;
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31, gl = lane % G;
  const int gib = threadIdx.x / G, gpb = blockDim.x / G;
  double *scr = smem + (size_t)gib * O::SCR;
  const int wfg = (threadIdx.x >> 5) * (32 / G);
  const int64_t total = (int64_t)a.nP * a.nQ;
  for (int64_t base = (int64_t)blockIdx.x * gpb + wfg; base < total;
       base += (int64_t)gridDim.x * gpb) {
    int64_t t = base + (gib - wfg);
    const bool active = t < total;
    if (!active) t = total - 1;
    const int iP = a.listP[t / a.nQ], iQ = a.listQ[t % a.nQ];
    const ShellRef sp = load_shell(a.aux, iP), sq = load_shell(a.aux, iQ);
    const double *res = os_quartet<LP, 0, LQ, 0, G>(
        a.boys, scr, gl, sp, a.aux.exps + sp.poff, a.aux.coefs + sp.poff, nullptr, nullptr,
        nullptr, sq, a.aux.exps + sq.poff, a.aux.coefs + sq.poff, nullptr, nullptr, nullptr);
    if (active) {
      constexpr int NP = ncart(LP), NQ = ncart(LQ);
      for (int idx = gl; idx < NP * NQ; idx += G) {
        const int iq = idx % NQ, ip = idx / NQ;
        a.V[(int64_t)(sp.fn + ip) * a.naux + sq.fn + iq] =
            res[idx] * c_cnorm[ncum(LP) + ip] * c_cnorm[ncum(LQ) + iq];
      }
    }
    __syncwarp();
  }
}

template <int LP, int LQ>
static int launch_int2c_cls(const Int2cArgs &a, cudaStream_t s) {
  using O = Os<LP, 0, LQ, 0>;
  constexpr int G = O::G;
  int groups = 256 / G;
  while (groups > 32 / G && (size_t)groups * O::SCR * 8 > 196 * 1024) groups -= 32 / G;
  const size_t smem = (size_t)groups * O::SCR * 8;
  auto kern = k_int2c<LP, LQ>;
  BQC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
  const int64_t total = (int64_t)a.nP * a.nQ;
  int64_t blocks = (total + groups - 1) / groups;
  blocks = std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)sm_count() * 16));
  kern<<<(unsigned)blocks, groups * G, smem, s>>>(a);
  BQC_LAUNCH_CHECK();
  return BQC_OK;
}

template <int LP>
static int int2c_q(int lq, const Int2cArgs &a, cudaStream_t s) {
  switch (lq) {
    case 0: return launch_int2c_cls<LP, 0>(a, s);
    case 1: return launch_int2c_cls<LP, 1>(a, s);
    case 2: return launch_int2c_cls<LP, 2>(a, s);
    case 3: return launch_int2c_cls<LP, 3>(a, s);
  }
  return BQC_E_UNSUPPORTED;
}

int launch_int2c(const Basis *b, double *V, cudaStream_t s) {
  for (int lp = 0; lp <= kMaxLAux; ++lp)
    for (int lq = 0; lq <= kMaxLAux; ++lq) {
      const int nP = b->auxl_off[lp + 1] - b->auxl_off[lp];
      const int nQ = b->auxl_off[lq + 1] - b->auxl_off[lq];
      if (!nP || !nQ) continue;
      Int2cArgs a;
      a.aux = b->aux.dev;
      a.boys = b->ctx->boys;
      a.listP = b->d_aux_by_l.as<int>() + b->auxl_off[lp];
      a.listQ = b->d_aux_by_l.as<int>() + b->auxl_off[lq];
      a.nP = nP;
      a.nQ = nQ;
      a.V = V;
      a.naux = b->naux;
      int st = BQC_E_UNSUPPORTED;
      switch (lp) {
        case 0: st = int2c_q<0>(lq, a, s); break;
        case 1: st = int2c_q<1>(lq, a, s); break;
        case 2: st = int2c_q<2>(lq, a, s); break;
        case 3: st = int2c_q<3>(lq, a, s); break;
      }
      BQC_TRY(st);
    }
  return BQC_OK;
}

// -------------------------------------------------- one-electron parts ---

struct OneArgs {
  ShellSetDev orb;
  const double *boys;
  const int2 *pairs;
  int npair;
  const double *atoms;  // natom x 4 (x, y, z, Z)
  int natom;
  double *S, *T, *V;
  int nbf;
};

// Nuclear attraction: point-charge limit of the OS recursion, summed over
// nuclei (Obara & Saika 1986: [a+1_i]^m = PA_i [a]^m - PC_i [a]^{m+1} + ...).
template <int LA, int LB>
__global__ void __launch_bounds__(256) k_nuclear(OneArgs a) {
  using O = Os<LA, LB, 0, 0>;
  constexpr int G = O::G;
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31, gl = lane % G;
  const int gib = threadIdx.x / G, gpb = blockDim.x / G;
  double *scr = smem + (size_t)gib * O::SCR;
  const int wfg = (threadIdx.x >> 5) * (32 / G);
  for (int64_t base = (int64_t)blockIdx.x * gpb + wfg; base < a.npair;
       base += (int64_t)gridDim.x * gpb) {
    int64_t t = base + (gib - wfg);
    const bool active = t < a.npair;
    if (!active) t = a.npair - 1;
    const int2 pr = a.pairs[t];
    const ShellRef sa = load_shell(a.orb, pr.x), sb = load_shell(a.orb, pr.y);
    const double *ea = a.orb.exps + sa.poff, *ca = a.orb.coefs + sa.poff;
    const double *eb = a.orb.exps + sb.poff, *cb = a.orb.coefs + sb.poff;
    double *acc = scr;
    double *s1 = scr + O::ACC;
    for (int i = gl; i < O::ACC; i += G) acc[i] = 0.0;
    __syncwarp();
    for (int n = 0; n < a.natom; ++n) {
      const double C[3] = {a.atoms[4 * n], a.atoms[4 * n + 1], a.atoms[4 * n + 2]};
      const double Z = a.atoms[4 * n + 3];
      for (int ia = 0; ia < sa.nprim; ++ia)
        for (int ib = 0; ib < sb.nprim; ++ib) {
          PrimQ g;
          prim_setup(ea[ia], sa.xyz, eb[ib], sb.xyz, 0.0, C, 0.0, C, -Z * ca[ia] * cb[ib], 1, g);
          os_vrr_accumulate<LA, LB, 0, 0, G>(g, a.boys, acc, s1, nullptr, gl);
        }
    }
    double AB[3], CD[3] = {0.0, 0.0, 0.0};
    for (int x = 0; x < 3; ++x) AB[x] = sa.xyz[x] - sb.xyz[x];
    double *bufA = scr + O::ACC;
    double *bufB = bufA + O::HMAX;
    const double *res = os_hrr<LA, LB, 0, 0, G>(acc, bufA, bufB, gl, AB, CD);
    if (active) {
      constexpr int NA = ncart(LA), NB = ncart(LB);
      for (int idx = gl; idx < NA * NB; idx += G) {
        const int ib = idx % NB, ia = idx / NB;
        const double v = res[idx] * c_cnorm[ncum(LA) + ia] * c_cnorm[ncum(LB) + ib];
        const int mu = sa.fn + ia, nu = sb.fn + ib;
        a.V[(int64_t)mu * a.nbf + nu] = v;
        a.V[(int64_t)nu * a.nbf + mu] = v;
      }
    }
    __syncwarp();
  }
}

template <int LA, int LB>
static int launch_nuclear_cls(const OneArgs &a, cudaStream_t s) {
  using O = Os<LA, LB, 0, 0>;
  constexpr int G = O::G;
  const int groups = 256 / G;
  const size_t smem = (size_t)groups * O::SCR * 8;
  auto kern = k_nuclear<LA, LB>;
  BQC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
  int64_t blocks = (a.npair + groups - 1) / groups;
  blocks = std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)sm_count() * 16));
  kern<<<(unsigned)blocks, groups * G, smem, s>>>(a);
  BQC_LAUNCH_CHECK();
  return BQC_OK;
}

// Overlap and kinetic energy by the 1-D Obara-Saika overlap recursion
// S(i+1,j) = PA S(i,j) + (i S(i-1,j) + j S(i,j-1)) / (2p), and
// T_x = [i j S(i-1,j-1) - 2b i S(i-1,j+1) - 2a j S(i+1,j-1) + 4ab S(i+1,j+1)] / 2
// (the symmetric form of -1/2 d^2/dx^2).  One thread per shell pair.
__global__ void k_overlap_kinetic(OneArgs a) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.npair) return;
  const int2 pr = a.pairs[t];
  const ShellRef sa = load_shell(a.orb, pr.x), sb = load_shell(a.orb, pr.y);
  constexpr int LM = kMaxLOrb + 2;  // i, j up to l + 1
  double Sv[36], Tv[36];
  const int na = ncart(sa.l), nb = ncart(sb.l);
  for (int k = 0; k < na * nb; ++k) Sv[k] = Tv[k] = 0.0;
  for (int ia = 0; ia < sa.nprim; ++ia)
    for (int ib = 0; ib < sb.nprim; ++ib) {
      const double al = a.orb.exps[sa.poff + ia], be = a.orb.exps[sb.poff + ib];
      const double p = al + be, ip = 1.0 / p;
      double s1d[3][LM][LM];
      double K = 1.0;
      for (int x = 0; x < 3; ++x) {
        const double P = (al * sa.xyz[x] + be * sb.xyz[x]) * ip;
        const double PA = P - sa.xyz[x], PB = P - sb.xyz[x];
        const double dAB = sa.xyz[x] - sb.xyz[x];
        double (*S)[LM] = s1d[x];
        S[0][0] = sqrt(3.141592653589793 * ip) * exp(-al * be * ip * dAB * dAB);
        for (int j = 1; j < LM; ++j)
          S[0][j] = PB * S[0][j - 1] + (j - 1) * 0.5 * ip * (j >= 2 ? S[0][j - 2] : 0.0);
        for (int i = 1; i < LM; ++i)
          for (int j = 0; j < LM; ++j) {
            double v = PA * S[i - 1][j];
            if (i >= 2) v += (i - 1) * 0.5 * ip * S[i - 2][j];
            if (j >= 1) v += j * 0.5 * ip * S[i - 1][j - 1];
            S[i][j] = v;
          }
        (void)K;
      }
      const double w = a.orb.coefs[sa.poff + ia] * a.orb.coefs[sb.poff + ib];
      for (int ia2 = 0; ia2 < na; ++ia2) {
        const unsigned char *ni = c_cart[ncum(sa.l) + ia2];
        for (int ib2 = 0; ib2 < nb; ++ib2) {
          const unsigned char *nj = c_cart[ncum(sb.l) + ib2];
          double s[3], tk[3];
          for (int x = 0; x < 3; ++x) {
            const int i = ni[x], j = nj[x];
            const double (*S)[LM] = s1d[x];
            s[x] = S[i][j];
            double v = 4.0 * al * be * S[i + 1][j + 1];
            if (i >= 1) v -= 2.0 * be * i * S[i - 1][j + 1];
            if (j >= 1) v -= 2.0 * al * j * S[i + 1][j - 1];
            if (i >= 1 && j >= 1) v += i * j * S[i - 1][j - 1];
            tk[x] = 0.5 * v;
          }
          Sv[ia2 * nb + ib2] += w * s[0] * s[1] * s[2];
          Tv[ia2 * nb + ib2] += w * (tk[0] * s[1] * s[2] + s[0] * tk[1] * s[2] + s[0] * s[1] * tk[2]);
        }
      }
    }
  for (int ia2 = 0; ia2 < na; ++ia2)
    for (int ib2 = 0; ib2 < nb; ++ib2) {
      const double n = c_cnorm[ncum(sa.l) + ia2] * c_cnorm[ncum(sb.l) + ib2];
      const int mu = sa.fn + ia2, nu = sb.fn + ib2;
      if (a.S) {
        a.S[(int64_t)mu * a.nbf + nu] = Sv[ia2 * nb + ib2] * n;
        a.S[(int64_t)nu * a.nbf + mu] = Sv[ia2 * nb + ib2] * n;
      }
      if (a.T) {
        a.T[(int64_t)mu * a.nbf + nu] = Tv[ia2 * nb + ib2] * n;
        a.T[(int64_t)nu * a.nbf + mu] = Tv[ia2 * nb + ib2] * n;
      }
    }
}

int launch_one_electron(const Basis *b, double *S, double *T, double *V, cudaStream_t s) {
  OneArgs a;
  a.orb = b->orb.dev;
  a.boys = b->ctx->boys;
  a.atoms = b->d_atoms.as<double>();
  a.natom = b->natom;
  a.S = S;
  a.T = T;
  a.V = V;
  a.nbf = b->nbf;
  if (S || T) {
    a.pairs = b->d_pairs.as<int2>();
    a.npair = (int)b->npair_sh;
    k_overlap_kinetic<<<(a.npair + 127) / 128, 128, 0, s>>>(a);
    BQC_LAUNCH_CHECK();
  }
  if (V) {
    for (int cls = 0; cls < kNPairClass; ++cls) {
      const int np = b->pair_off[cls + 1] - b->pair_off[cls];
      if (!np) continue;
      a.pairs = b->d_pairs.as<int2>() + b->pair_off[cls];
      a.npair = np;
      int st = BQC_E_UNSUPPORTED;
      switch (cls) {
        case 0: st = launch_nuclear_cls<0, 0>(a, s); break;
        case 1: st = launch_nuclear_cls<1, 0>(a, s); break;
        case 2: st = launch_nuclear_cls<1, 1>(a, s); break;
        case 3: st = launch_nuclear_cls<2, 0>(a, s); break;
        case 4: st = launch_nuclear_cls<2, 1>(a, s); break;
        case 5: st = launch_nuclear_cls<2, 2>(a, s); break;
      }
      BQC_TRY(st);
    }
  }
  return BQC_OK;
}

// ------------------------------------------------------ screening plan ---

__global__ void k_diag_sqrt_max(const double *V, int naux, const int *fn_of_shell,
                                const int *l_of_shell, int nshell, double *q) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nshell) return;
  const int f0 = fn_of_shell[i], nc = ncart(l_of_shell[i]);
  double m = 0.0;
  for (int c = 0; c < nc; ++c) m = fmax(m, fabs(V[(int64_t)(f0 + c) * naux + f0 + c]));
  q[i] = sqrt(m);
}

// cut[P] = number of class pairs with Q_pair * Q_P >= tau (pairs sorted descending).
__global__ void k_cut(const double *qpair, int np, const int *aux_list, int na,
                      const double *qaux, double tau, int64_t *cut) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= na) return;
  const double qp = qaux[aux_list[i]];
  int lo = 0, hi = np;  // first index with qpair*qp < tau
  if (tau > 0.0) {
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (qpair[mid] * qp >= tau) lo = mid + 1; else hi = mid;
    }
  } else {
    lo = np;
  }
  cut[i] = lo;
}

int eri3c_plan(const Basis *b, double tau, const double *V_diag_dev, cudaStream_t s,
               Eri3cPlan *plan) {
  Ctx *ctx = b->ctx;
  plan->ctx = ctx;
  plan->tau = tau;
  const int64_t np = b->npair_sh;
  const int nas = b->aux.dev.n;
  BQC_TRY(plan->d_pairs_sorted.alloc(ctx, np * sizeof(int2)));
  BQC_TRY(plan->d_qpair_sorted.alloc(ctx, np * sizeof(double)));
  BQC_TRY(plan->d_qaux.alloc(ctx, nas * sizeof(double)));
  DBuf &qpair = plan->d_qpair;
  BQC_TRY(qpair.alloc(ctx, np * sizeof(double)));
  BQC_TRY(launch_schwarz_pairs(b, qpair.as<double>(), s));
  k_diag_sqrt_max<<<(nas + 127) / 128, 128, 0, s>>>(V_diag_dev, b->naux, b->aux.dev.fn,
                                                      b->aux.dev.l, nas, plan->d_qaux.as<double>());
  BQC_LAUNCH_CHECK();
  // sort each class segment by decreasing Q
  for (int cls = 0; cls < kNPairClass; ++cls) {
    const int o = b->pair_off[cls], n = b->pair_off[cls + 1] - o;
    if (!n) continue;
    size_t tmp = 0;
    const double *kin = qpair.as<double>() + o;
    double *kout = plan->d_qpair_sorted.as<double>() + o;
    const int2 *vin = b->d_pairs.as<int2>() + o;
    int2 *vout = plan->d_pairs_sorted.as<int2>() + o;
    BQC_CUDA_TRY(cub::DeviceRadixSort::SortPairsDescending(nullptr, tmp, kin, kout, vin, vout, n,
                                                           0, 64, s));
    DBuf t;
    BQC_TRY(t.alloc(ctx, std::max<size_t>(tmp, 16)));
    BQC_CUDA_TRY(cub::DeviceRadixSort::SortPairsDescending(t.p, tmp, kin, kout, vin, vout, n, 0,
                                                           64, s));
    BQC_CUDA_TRY(cudaStreamSynchronize(s));  // t is released at scope end
  }
  // survivor counts and prefixes per (class, aux l)
  int64_t off = 0;
  for (int cls = 0; cls < kNPairClass; ++cls)
    for (int lc = 0; lc <= kMaxLAux; ++lc) {
      plan->prefix_off[cls][lc] = off;
      off += (b->auxl_off[lc + 1] - b->auxl_off[lc]) + 1;
    }
  BQC_TRY(plan->d_prefix.alloc(ctx, off * sizeof(int64_t)));
  BQC_CUDA_TRY(cudaMemsetAsync(plan->d_prefix.p, 0, off * sizeof(int64_t), s));
  DBuf cut;
  BQC_TRY(cut.alloc(ctx, std::max<int64_t>(1, nas) * sizeof(int64_t)));
  for (int cls = 0; cls < kNPairClass; ++cls) {
    const int po = b->pair_off[cls], pn = b->pair_off[cls + 1] - po;
    for (int lc = 0; lc <= kMaxLAux; ++lc) {
      const int ao = b->auxl_off[lc], an = b->auxl_off[lc + 1] - ao;
      if (!an) continue;
      int64_t *pre = plan->d_prefix.as<int64_t>() + plan->prefix_off[cls][lc];
      if (!pn) continue;
      k_cut<<<(an + 127) / 128, 128, 0, s>>>(plan->d_qpair_sorted.as<double>() + po, pn,
                                             b->d_aux_by_l.as<int>() + ao, an,
                                             plan->d_qaux.as<double>(), tau, cut.as<int64_t>());
      BQC_LAUNCH_CHECK();
      size_t tmp = 0;
      BQC_CUDA_TRY(cub::DeviceScan::InclusiveSum(nullptr, tmp, cut.as<int64_t>(), pre + 1, an, s));
      DBuf t;
      BQC_TRY(t.alloc(ctx, std::max<size_t>(tmp, 16)));
      BQC_CUDA_TRY(cub::DeviceScan::InclusiveSum(t.p, tmp, cut.as<int64_t>(), pre + 1, an, s));
      BQC_CUDA_TRY(cudaStreamSynchronize(s));
    }
  }
  // read the totals (one small copy)
  std::vector<int64_t> &h = plan->h_prefix;
  h.assign(off, 0);
  BQC_CUDA_TRY(cudaMemcpyAsync(h.data(), plan->d_prefix.p, off * sizeof(int64_t),
                               cudaMemcpyDeviceToHost, s));
  BQC_CUDA_TRY(cudaStreamSynchronize(s));
  plan->survivors = plan->candidates = 0;
  for (int cls = 0; cls < kNPairClass; ++cls) {
    const int pn = b->pair_off[cls + 1] - b->pair_off[cls];
    for (int lc = 0; lc <= kMaxLAux; ++lc) {
      const int an = b->auxl_off[lc + 1] - b->auxl_off[lc];
      plan->total[cls][lc] = h[plan->prefix_off[cls][lc] + an];
      plan->survivors += plan->total[cls][lc];
      plan->candidates += (int64_t)an * pn;
    }
  }
  return BQC_OK;
}

}  // namespace bqc
