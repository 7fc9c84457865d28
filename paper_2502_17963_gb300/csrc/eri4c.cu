// Conventional (non-DF) direct J and K from four-centre integrals.
//
// The paper's mean field for molecules builds the Fock matrix on the fly from
// the four-centre ERIs rather than from fitted ones (Sec. 2.2.2).  Here:
//   J_mu nu = sum_{lambda sigma} (mu nu|lambda sigma) D_lambda sigma,
//   K_mu lambda = sum_{nu sigma} (mu nu|lambda sigma) D_nu sigma,
// with D = C_occ C_occ^T, over the unique shell quartets (ab|cd) of the
// eight-fold permutational symmetry: oriented shell pairs p = (a, b) and
// q = (c, d) of pair classes X >= Y, and q <= p within one class.  A quartet
// is kept when Q_p Q_q >= tau (Schwarz, Q = sqrt(max (ab|ab))); with each
// class's pairs sorted by decreasing Q the kept partners of p are a prefix,
// so the kept quartets map onto a dense index as in the three-centre kernel.
//
// Digestion.  A computed integral v stands for its eight symmetric images;
// where shells coincide (a = b, c = d, or p = q) images repeat, so v is
// weighted by 1/2 for each coincidence.  Summing the images gives, with D
// symmetric, Jacc_ij += 2 w v D_kl, Jacc_kl += 2 w v D_ij and
// Kacc_ik += w v D_jl, Kacc_jk += w v D_il, Kacc_il += w v D_jk,
// Kacc_jl += w v D_ik, and J = Jacc + Jacc^T, K = Kacc + Kacc^T.  Each lane
// group first contracts its quartet over the indices a target does not
// depend on (e.g. J_ij sums over all (k, l) of the quartet) and then issues
// one FP64 atomic per target element, instead of one per integral.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "bqc_internal.h"
#include "df_internal.h"
#include "gemm64.cuh"
#include "os_eri.cuh"

namespace bqc {

struct Jk4Args {
  ShellSetDev orb;
  const double *boys;
  const int2 *pX, *pY;      // sorted pairs of the two classes
  const int64_t *prefix;    // npX + 1 kept-quartet prefix over the pairs of X
  int npX;
  int same;                 // X == Y
  const double *D;          // N x N
  double *Jacc, *Kacc;      // N x N
  int n;
};

template <int LA, int LB, int LC, int LD>
__global__ void __launch_bounds__(256) k_jk4c(Jk4Args a) {
  using O = Os<LA, LB, LC, LD>;
  constexpr int G = O::G;
  constexpr int NA = ncart(LA), NB = ncart(LB), NC = ncart(LC), ND = ncart(LD);
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31;
  const int gl = lane % G;
  const int group_in_block = threadIdx.x / G;
  const int groups_per_block = blockDim.x / G;
  double *scr = smem + (size_t)group_in_block * O::SCR;
  const int64_t total = a.prefix[a.npX];
  const int64_t gstride = (int64_t)gridDim.x * groups_per_block;
  const int warp_first_group = (threadIdx.x >> 5) * (32 / G);
  const int64_t base0 = (int64_t)blockIdx.x * groups_per_block + warp_first_group;
  const int n = a.n;
  for (int64_t base = base0; base < total; base += gstride) {
    int64_t t = base + (group_in_block - warp_first_group);
    const bool active = t < total;
    if (!active) t = total - 1;
    int lo = 0, hi = a.npX;  // largest i with prefix[i] <= t
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (a.prefix[mid] <= t) lo = mid; else hi = mid;
    }
    const int jq = (int)(t - a.prefix[lo]);
    const int2 p = a.pX[lo], q = a.pY[jq];
    const ShellRef sa = load_shell(a.orb, p.x), sb = load_shell(a.orb, p.y);
    const ShellRef sc = load_shell(a.orb, q.x), sd = load_shell(a.orb, q.y);
    const double *res = os_quartet<LA, LB, LC, LD, G>(
        a.boys, scr, gl, sa, a.orb.exps + sa.poff, a.orb.coefs + sa.poff, &sb,
        a.orb.exps + sb.poff, a.orb.coefs + sb.poff, sc, a.orb.exps + sc.poff,
        a.orb.coefs + sc.poff, &sd, a.orb.exps + sd.poff, a.orb.coefs + sd.poff);
    if (active) {
      double w = 1.0;
      if (p.x == p.y) w *= 0.5;
      if (q.x == q.y) w *= 0.5;
      if (a.same && jq == lo) w *= 0.5;
      auto val = [&](int ia, int ib, int ic, int id) {
        return res[((ia * NB + ib) * NC + ic) * ND + id] * c_cnorm[ncum(LA) + ia] *
               c_cnorm[ncum(LB) + ib] * c_cnorm[ncum(LC) + ic] * c_cnorm[ncum(LD) + id];
      };
      const double *D = a.D;
      // J_ij += 2 w sum_kl v D_kl
      for (int e = gl; e < NA * NB; e += G) {
        const int ia = e / NB, ib = e % NB;
        double s = 0.0;
        for (int ic = 0; ic < NC; ++ic)
          for (int id = 0; id < ND; ++id)
            s += val(ia, ib, ic, id) * D[(int64_t)(sc.fn + ic) * n + sd.fn + id];
        atomicAdd(a.Jacc + (int64_t)(sa.fn + ia) * n + sb.fn + ib, 2.0 * w * s);
      }
      // J_kl += 2 w sum_ij v D_ij
      for (int e = gl; e < NC * ND; e += G) {
        const int ic = e / ND, id = e % ND;
        double s = 0.0;
        for (int ia = 0; ia < NA; ++ia)
          for (int ib = 0; ib < NB; ++ib)
            s += val(ia, ib, ic, id) * D[(int64_t)(sa.fn + ia) * n + sb.fn + ib];
        atomicAdd(a.Jacc + (int64_t)(sc.fn + ic) * n + sd.fn + id, 2.0 * w * s);
      }
      // K_ik += w sum_jl v D_jl ; K_jk += w sum_il v D_il
      for (int e = gl; e < NA * NC; e += G) {
        const int ia = e / NC, ic = e % NC;
        double s = 0.0;
        for (int ib = 0; ib < NB; ++ib)
          for (int id = 0; id < ND; ++id)
            s += val(ia, ib, ic, id) * D[(int64_t)(sb.fn + ib) * n + sd.fn + id];
        atomicAdd(a.Kacc + (int64_t)(sa.fn + ia) * n + sc.fn + ic, w * s);
      }
      for (int e = gl; e < NB * NC; e += G) {
        const int ib = e / NC, ic = e % NC;
        double s = 0.0;
        for (int ia = 0; ia < NA; ++ia)
          for (int id = 0; id < ND; ++id)
            s += val(ia, ib, ic, id) * D[(int64_t)(sa.fn + ia) * n + sd.fn + id];
        atomicAdd(a.Kacc + (int64_t)(sb.fn + ib) * n + sc.fn + ic, w * s);
      }
      // K_il += w sum_jk v D_jk ; K_jl += w sum_ik v D_ik
      for (int e = gl; e < NA * ND; e += G) {
        const int ia = e / ND, id = e % ND;
        double s = 0.0;
        for (int ib = 0; ib < NB; ++ib)
          for (int ic = 0; ic < NC; ++ic)
            s += val(ia, ib, ic, id) * D[(int64_t)(sb.fn + ib) * n + sc.fn + ic];
        atomicAdd(a.Kacc + (int64_t)(sa.fn + ia) * n + sd.fn + id, w * s);
      }
      for (int e = gl; e < NB * ND; e += G) {
        const int ib = e / ND, id = e % ND;
        double s = 0.0;
        for (int ia = 0; ia < NA; ++ia)
          for (int ic = 0; ic < NC; ++ic)
            s += val(ia, ib, ic, id) * D[(int64_t)(sa.fn + ia) * n + sc.fn + ic];
        atomicAdd(a.Kacc + (int64_t)(sb.fn + ib) * n + sd.fn + id, w * s);
      }
    }
    __syncwarp();
  }
}

// out = acc + acc^T (N x N)
__global__ void k_sym_add(const double *acc, int n, double *out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)n * n) return;
  const int64_t r = i / n, c = i % n;
  out[i] = acc[i] + acc[c * n + r];
}

template <int LA, int LB, int LC, int LD>
static int launch4(const Jk4Args &a, int64_t total, cudaStream_t s) {
  using O = Os<LA, LB, LC, LD>;
  constexpr int G = O::G;
  int groups = 256 / G;
  while (groups > 32 / G && (size_t)groups * O::SCR * 8 > 196 * 1024) groups -= 32 / G;
  const size_t smem = (size_t)groups * O::SCR * 8;
  if (smem > 227 * 1024) return BQC_E_UNSUPPORTED;
  auto kern = k_jk4c<LA, LB, LC, LD>;
  BQC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
  int64_t blocks = (total + groups - 1) / groups;
  blocks = std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)sm_count() * 16));
  kern<<<(unsigned)blocks, groups * G, smem, s>>>(a);
  BQC_LAUNCH_CHECK();
  return BQC_OK;
}

// class index -> (la, lb): 00, 10, 11, 20, 21, 22
template <int X> struct Cls;
template <> struct Cls<0> { static constexpr int a = 0, b = 0; };
template <> struct Cls<1> { static constexpr int a = 1, b = 0; };
template <> struct Cls<2> { static constexpr int a = 1, b = 1; };
template <> struct Cls<3> { static constexpr int a = 2, b = 0; };
template <> struct Cls<4> { static constexpr int a = 2, b = 1; };
template <> struct Cls<5> { static constexpr int a = 2, b = 2; };

template <int X, int Y>
static int launch_xy(const Jk4Args &a, int64_t total, cudaStream_t s) {
  return launch4<Cls<X>::a, Cls<X>::b, Cls<Y>::a, Cls<Y>::b>(a, total, s);
}

template <int X>
static int dispatch_y(int y, const Jk4Args &a, int64_t total, cudaStream_t s) {
  switch (y) {
    case 0: return launch_xy<X, 0>(a, total, s);
    case 1: if constexpr (X >= 1) return launch_xy<X, 1>(a, total, s); break;
    case 2: if constexpr (X >= 2) return launch_xy<X, 2>(a, total, s); break;
    case 3: if constexpr (X >= 3) return launch_xy<X, 3>(a, total, s); break;
    case 4: if constexpr (X >= 4) return launch_xy<X, 4>(a, total, s); break;
    case 5: if constexpr (X >= 5) return launch_xy<X, 5>(a, total, s); break;
  }
  return BQC_E_UNSUPPORTED;
}

static int dispatch_xy(int x, int y, const Jk4Args &a, int64_t total, cudaStream_t s) {
  switch (x) {
    case 0: return dispatch_y<0>(y, a, total, s);
    case 1: return dispatch_y<1>(y, a, total, s);
    case 2: return dispatch_y<2>(y, a, total, s);
    case 3: return dispatch_y<3>(y, a, total, s);
    case 4: return dispatch_y<4>(y, a, total, s);
    case 5: return dispatch_y<5>(y, a, total, s);
  }
  return BQC_E_UNSUPPORTED;
}

struct Jk4Plan {
  double tau = 0.0;
  DBuf pairs;    // int2 per pair, sorted by decreasing Q within each class
  DBuf prefix;   // concatenated npX + 1 prefixes of the class pairs (X >= Y)
  int64_t pre_off[kNPairClass][kNPairClass] = {{0}};
  int64_t total[kNPairClass][kNPairClass] = {{0}};
  int64_t kept = 0, candidates = 0;
  DBuf D, Jacc, Kacc;
};

void Jk4Deleter::operator()(Jk4Plan *p) const { delete p; }

// Schwarz factors of every pair (device), sorted per class on the host, and
// the kept-partner counts of every pair of class X against class Y <= X.
int jk4c_setup(Df *df, cudaStream_t s) {
  const Basis *b = df->basis;
  Ctx *ctx = df->ctx;
  BQC_TRY(upload_cart_tables());
  Jk4Plan *pl = new Jk4Plan();
  df->jk4.reset(pl);
  pl->tau = df->opts.schwarz;
  const int64_t np = b->npair_sh;
  DBuf q;
  BQC_TRY(q.alloc(ctx, (size_t)std::max<int64_t>(1, np) * 8));
  BQC_TRY(launch_schwarz_pairs(b, q.as<double>(), s));
  std::vector<double> hq(np);
  std::vector<int2> hp(np);
  BQC_CUDA_TRY(cudaMemcpyAsync(hq.data(), q.p, np * 8, cudaMemcpyDeviceToHost, s));
  BQC_CUDA_TRY(cudaMemcpyAsync(hp.data(), b->d_pairs.p, np * sizeof(int2), cudaMemcpyDeviceToHost,
                               s));
  BQC_CUDA_TRY(cudaStreamSynchronize(s));
  std::vector<int2> sp(np);
  std::vector<double> sq(np);
  for (int c = 0; c < kNPairClass; ++c) {
    const int o = b->pair_off[c], m = b->pair_off[c + 1] - o;
    std::vector<int> idx(m);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(),
                     [&](int u, int v) { return hq[o + u] > hq[o + v]; });
    for (int k = 0; k < m; ++k) {
      sp[o + k] = hp[o + idx[k]];
      sq[o + k] = hq[o + idx[k]];
    }
  }
  std::vector<int64_t> pre;
  for (int x = 0; x < kNPairClass; ++x)
    for (int y = 0; y <= x; ++y) {
      const int ox = b->pair_off[x], nx = b->pair_off[x + 1] - ox;
      const int oy = b->pair_off[y], ny = b->pair_off[y + 1] - oy;
      pl->pre_off[x][y] = (int64_t)pre.size();
      int64_t acc = 0;
      pre.push_back(0);
      for (int i = 0; i < nx; ++i) {
        // partners: a prefix of class y's sorted list (Q_p Q_q >= tau)
        int lo = 0, hi = ny;
        if (pl->tau > 0.0) {
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (sq[ox + i] * sq[oy + mid] >= pl->tau) lo = mid + 1; else hi = mid;
          }
        } else {
          lo = ny;
        }
        int64_t cnt = lo;
        if (x == y) cnt = std::min<int64_t>(cnt, i + 1);
        acc += cnt;
        pre.push_back(acc);
      }
      pl->total[x][y] = acc;
      pl->kept += acc;
      pl->candidates += (x == y) ? (int64_t)nx * (nx + 1) / 2 : (int64_t)nx * ny;
    }
  BQC_TRY(pl->pairs.alloc(ctx, (size_t)std::max<int64_t>(1, np) * sizeof(int2)));
  BQC_TRY(pl->prefix.alloc(ctx, pre.size() * 8));
  BQC_CUDA_TRY(cudaMemcpyAsync(pl->pairs.p, sp.data(), np * sizeof(int2), cudaMemcpyHostToDevice, s));
  BQC_CUDA_TRY(cudaMemcpyAsync(pl->prefix.p, pre.data(), pre.size() * 8, cudaMemcpyHostToDevice, s));
  const int n = b->nbf;
  BQC_TRY(pl->D.alloc(ctx, (size_t)n * n * 8));
  BQC_TRY(pl->Jacc.alloc(ctx, (size_t)n * n * 8));
  BQC_TRY(pl->Kacc.alloc(ctx, (size_t)n * n * 8));
  BQC_CUDA_TRY(cudaStreamSynchronize(s));  // the host vectors go out of scope
  df->plan.candidates = pl->candidates;
  df->plan.survivors = pl->kept;
  return BQC_OK;
}

int jk_4c(Df *df, const double *C, int prec, double *J, double *K, cudaStream_t s) {
  if (prec != BQC_PREC_FP64) {
    set_error("four-centre J/K runs in FP64 only", __FILE__, __LINE__);
    return BQC_E_UNSUPPORTED;
  }
  Jk4Plan *pl = df->jk4.get();
  if (!pl) return BQC_E_INVALID;
  const Basis *b = df->basis;
  const int n = b->nbf, no = b->nocc;
  df->mark(0, s);
  df->mark(1, s);
  Gemm64Args g;  // D = C C^T
  g.M = n;
  g.N = n;
  g.K1 = 1;
  g.K2 = no;
  g.A = C;
  g.lda = no;
  g.B = C;
  g.ldb = no;
  g.C = pl->D.as<double>();
  g.ldc = n;
  BQC_TRY(launch_gemm64(kAN, true, g, s));
  BQC_CUDA_TRY(cudaMemsetAsync(pl->Jacc.p, 0, pl->Jacc.n, s));
  BQC_CUDA_TRY(cudaMemsetAsync(pl->Kacc.p, 0, pl->Kacc.n, s));
  df->mark(2, s);
  Jk4Args a;
  a.orb = b->orb.dev;
  a.boys = b->ctx->boys;
  a.D = pl->D.as<double>();
  a.Jacc = pl->Jacc.as<double>();
  a.Kacc = pl->Kacc.as<double>();
  a.n = n;
  for (int x = 0; x < kNPairClass; ++x)
    for (int y = 0; y <= x; ++y) {
      if (pl->total[x][y] == 0) continue;
      a.pX = pl->pairs.as<int2>() + b->pair_off[x];
      a.pY = pl->pairs.as<int2>() + b->pair_off[y];
      a.prefix = pl->prefix.as<int64_t>() + pl->pre_off[x][y];
      a.npX = b->pair_off[x + 1] - b->pair_off[x];
      a.same = x == y;
      BQC_TRY(dispatch_xy(x, y, a, pl->total[x][y], s));
    }
  df->mark(3, s);
  const unsigned nb = (unsigned)(((int64_t)n * n + 255) / 256);
  k_sym_add<<<nb, 256, 0, s>>>(pl->Jacc.as<double>(), n, J);
  BQC_LAUNCH_CHECK();
  k_sym_add<<<nb, 256, 0, s>>>(pl->Kacc.as<double>(), n, K);
  BQC_LAUNCH_CHECK();
  df->mark(4, s);
  return BQC_OK;
}

}  // namespace bqc
