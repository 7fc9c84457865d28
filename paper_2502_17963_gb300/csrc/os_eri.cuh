// Device-side Obara-Saika / Head-Gordon-Pople engine shared by the integral
// translation units (three-centre, metric, Schwarz and one-electron kernels in
// eri.cu; the direct four-centre J/K in eri4c.cu): Cartesian component
// tables, the Boys-function evaluator, the recursion tables and the
// group-cooperative quartet routine.  The constant tables have internal
// linkage: every translation unit that includes this header holds its own
// copy and uploads it (upload_cart_tables) before its first launch.
#pragma once
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <type_traits>

#include "bqc_internal.h"

namespace bqc {

__host__ __device__ constexpr int ncart(int l) { return (l + 1) * (l + 2) / 2; }
__host__ __device__ constexpr int ncum(int l) { return l * (l + 1) * (l + 2) / 6; }
__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }

constexpr int kCartLevels = 9;               // components for l = 0..8
constexpr int kCartN = 165;                  // ncum(9)
static __constant__ unsigned char c_cart[kCartN][3];
static __constant__ double c_cnorm[kCartN];         // 1/sqrt((2i-1)!!(2j-1)!!(2k-1)!!)

__device__ __forceinline__ int cart_index(int i, int j, int k) {
  const int l = i + j + k, jk = j + k;
  return ncum(l) + jk * (jk + 1) / 2 + k;
}

static void cart_tables_host(unsigned char (*cart)[3], double *cn) {
  int n = 0;
  for (int l = 0; l < kCartLevels; ++l)
    for (int i = l; i >= 0; --i)
      for (int j = l - i; j >= 0; --j) {
        const int k = l - i - j;
        cart[n][0] = (unsigned char)i;
        cart[n][1] = (unsigned char)j;
        cart[n][2] = (unsigned char)k;
        auto df = [](int m) {
          double r = 1.0;
          for (int t = 2 * m - 1; t > 1; t -= 2) r *= t;
          return r;
        };
        cn[n] = 1.0 / std::sqrt(df(i) * df(j) * df(k));
        ++n;
      }
}

static int upload_cart_tables() {
  static std::once_flag once;
  static int status = BQC_OK;
  std::call_once(once, [] {
    unsigned char cart[kCartN][3];
    double cn[kCartN];
    cart_tables_host(cart, cn);
    if (cudaMemcpyToSymbol(c_cart, cart, sizeof(cart)) != cudaSuccess ||
        cudaMemcpyToSymbol(c_cnorm, cn, sizeof(cn)) != cudaSuccess)
      status = BQC_E_CUDA;
  });
  return status;
}


__device__ __forceinline__ double boys_one(const double *__restrict__ tab, int m, double T,
                                           double expmT_large) {
  if (T < kBoysTCut) {
    const int k = __double2int_rn(T * (1.0 / kBoysH));
    const double d = -(T - k * kBoysH);
    const double *row = tab + (size_t)k * kBoysNM + m;
    // sum_j F_{m+j}(T_k) d^j / j!  (Horner)
    double r = __ldg(row + 7) * (1.0 / 5040.0);
    r = fma(r, d, __ldg(row + 6) * (1.0 / 720.0));
    r = fma(r, d, __ldg(row + 5) * (1.0 / 120.0));
    r = fma(r, d, __ldg(row + 4) * (1.0 / 24.0));
    r = fma(r, d, __ldg(row + 3) * (1.0 / 6.0));
    r = fma(r, d, __ldg(row + 2) * 0.5);
    r = fma(r, d, __ldg(row + 1));
    r = fma(r, d, __ldg(row + 0));
    return r;
  }
  const double inv2T = 0.5 / T;
  double f = 0.5 * sqrt(3.141592653589793 / T);
  for (int j = 0; j < m; ++j) f = ((2 * j + 1) * f - expmT_large) * inv2T;
  return f;
}

// --------------------------------------------------- OS/HGP engine -------

template <int I, int N, class Fn>
__device__ __forceinline__ void static_for(Fn &&fn) {
  if constexpr (I < N) {
    fn(std::integral_constant<int, I>{});
    static_for<I + 1, N>(fn);
  }
}

// Table geometry of one class (all sizes in doubles).
template <int LA, int LB, int LC, int LD>
struct Os {
  static constexpr int E = LA + LB, F = LC + LD, L = E + F;
  static constexpr int NE = ncum(E + 1);
  static constexpr int S1 = NE * (L + 1);  // [e][m], m <= L - |e|
  __host__ __device__ static constexpr int elo(int f) { return cmax(LA - (F - f), 0); }
  __host__ __device__ static constexpr int lne(int f) { return NE - ncum(elo(f)); }
  __host__ __device__ static constexpr int lm(int f) { return F - f + 1; }
  __host__ __device__ static constexpr int lsz(int f) { return lne(f) * ncart(f) * lm(f); }
  __host__ __device__ static constexpr int loff(int f) {
    int o = 0;
    for (int g = 1; g < f; ++g) o += lsz(g);
    return o;
  }
  static constexpr int GSZ = loff(F + 1);
  static constexpr int NEA = NE - ncum(LA);
  static constexpr int NFC = ncum(F + 1) - ncum(LC);
  static constexpr int ACC = NEA * NFC;
  static constexpr int NAB = ncart(LA) * ncart(LB);
  __host__ __device__ static constexpr int hbsz(int j) {
    return (ncum(E - j + 1) - ncum(LA)) * ncart(j) * NFC;
  }
  __host__ __device__ static constexpr int hksz(int j) {
    return NAB * (ncum(F - j + 1) - ncum(LC)) * ncart(j);
  }
  __host__ __device__ static constexpr int hmax() {
    int m = 0;
    for (int j = 1; j <= LB; ++j) m = cmax(m, hbsz(j));
    for (int j = 1; j <= LD; ++j) m = cmax(m, hksz(j));
    return m;
  }
  static constexpr int HMAX = hmax();
  static constexpr int NOUT = NAB * ncart(LC) * ncart(LD);
  static constexpr int PH1 = S1 + GSZ;
  static constexpr int PH2 = 2 * HMAX;
  static constexpr int SCR = ACC + cmax(PH1, PH2);
  // lanes per quartet: keep <= ~96 doubles of table per lane
  static constexpr int lanes() {
    int g = 1;
    while (g < 32 && SCR > 96 * g) g *= 2;
    return g;
  }
  static constexpr int G = lanes();
};

// Scalars of one primitive quartet.
struct PrimQ {
  double PA[3], WP[3], QC[3], WQ[3];
  double inv2p, rho_p, inv2q, rho_q, inv2pq, T, pref;
};

// Geometry of a primitive quartet (a,b|c,d).  point != 0: ket is a point
// charge at C (nuclear attraction): rho = p, W = C, prefactor 2 pi / p.
__device__ __forceinline__ void prim_setup(double a, const double *A, double b, const double *B,
                                           double c, const double *C, double d, const double *D,
                                           double cabcd, int point, PrimQ &g) {
  const double p = a + b, ip = 1.0 / p;
  double P[3], AB2 = 0.0;
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    P[x] = (a * A[x] + b * B[x]) * ip;
    const double t = A[x] - B[x];
    AB2 += t * t;
    g.PA[x] = P[x] - A[x];
  }
  const double Kab = exp(-a * b * ip * AB2);
  if (point) {
    double PC2 = 0.0;
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      const double t = C[x] - P[x];
      g.WP[x] = t;
      PC2 += t * t;
      g.QC[x] = 0.0;
      g.WQ[x] = 0.0;
    }
    g.inv2p = 0.5 * ip;
    g.rho_p = 1.0;
    g.inv2q = g.rho_q = g.inv2pq = 0.0;
    g.T = p * PC2;
    g.pref = 2.0 * 3.141592653589793 * ip * Kab * cabcd;
    return;
  }
  const double q = c + d, iq = 1.0 / q;
  double Q[3], CD2 = 0.0;
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    Q[x] = (c * C[x] + d * D[x]) * iq;
    const double t = C[x] - D[x];
    CD2 += t * t;
    g.QC[x] = Q[x] - C[x];
  }
  const double Kcd = (d == 0.0) ? 1.0 : exp(-c * d * iq * CD2);
  const double ipq = 1.0 / (p + q);
  const double rho = p * q * ipq;
  double PQ2 = 0.0;
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    const double W = (p * P[x] + q * Q[x]) * ipq;
    g.WP[x] = W - P[x];
    g.WQ[x] = W - Q[x];
    const double t = P[x] - Q[x];
    PQ2 += t * t;
  }
  g.inv2p = 0.5 * ip;
  g.rho_p = rho * ip;
  g.inv2q = 0.5 * iq;
  g.rho_q = rho * iq;
  g.inv2pq = 0.5 * ipq;
  g.T = rho * PQ2;
  // 2 pi^{5/2} = 34.98683665524972
  g.pref = 34.98683665524972 * ip * iq * sqrt(ipq) * Kab * Kcd * cabcd;
}

__device__ __forceinline__ int first_dir(const unsigned char *n) {
  return n[0] > 0 ? 0 : (n[1] > 0 ? 1 : 2);
}

// VRR for one primitive quartet and accumulation into acc.  Group-cooperative:
// lane gl of G.  scr: S1 table then ket levels.  The caller syncs after.
template <int LA, int LB, int LC, int LD, int G>
__device__ __forceinline__ void os_vrr_accumulate(const PrimQ &g, const double *__restrict__ boys,
                                                  double *__restrict__ acc,
                                                  double *__restrict__ s1,
                                                  double *__restrict__ gk, int gl) {
  using O = Os<LA, LB, LC, LD>;
  constexpr int L = O::L, E = O::E, F = O::F;
  // level 0: [0|0]^m
  {
    const double e = g.T >= kBoysTCut ? exp(-g.T) : 0.0;
    for (int m = gl; m <= L; m += G) s1[m] = g.pref * boys_one(boys, m, g.T, e);
  }
  __syncwarp();
  // bra levels e = 1..E on f = 0
  static_for<1, E + 1>([&](auto ei) {
    constexpr int e = decltype(ei)::value;
    constexpr int M = L - e + 1;
    constexpr int CNT = ncart(e) * M;
    for (int idx = gl; idx < CNT; idx += G) {
      const int c = idx / M, m = idx - c * M;
      const int ci = ncum(e) + c;
      const unsigned char *n = c_cart[ci];
      const int d = first_dir(n);
      const int nd = n[d];
      int i1[3] = {n[0], n[1], n[2]};
      i1[d] -= 1;
      const int e1 = cart_index(i1[0], i1[1], i1[2]);
      double v = g.PA[d] * s1[e1 * (L + 1) + m] + g.WP[d] * s1[e1 * (L + 1) + m + 1];
      if (nd >= 2) {
        i1[d] -= 1;
        const int e2 = cart_index(i1[0], i1[1], i1[2]);
        v += (nd - 1) * g.inv2p * (s1[e2 * (L + 1) + m] - g.rho_p * s1[e2 * (L + 1) + m + 1]);
      }
      s1[ci * (L + 1) + m] = v;
    }
    __syncwarp();
  });
  // ket levels f = 1..F
  auto get = [&](auto lvl, int ecum, int fc, int m) -> double {
    constexpr int gg = decltype(lvl)::value;
    if constexpr (gg == 0) {
      return s1[ecum * (L + 1) + m];
    } else {
      return gk[O::loff(gg) + ((ecum - ncum(O::elo(gg))) * ncart(gg) + fc) * O::lm(gg) + m];
    }
  };
  static_for<1, F + 1>([&](auto fi) {
    constexpr int f = decltype(fi)::value;
    constexpr int LM = O::lm(f), NF = ncart(f);
    constexpr int CNT = O::lne(f) * NF * LM;
    for (int idx = gl; idx < CNT; idx += G) {
      const int m = idx % LM;
      const int t = idx / LM;
      const int fc = t % NF, er = t / NF;
      const int ecum = ncum(O::elo(f)) + er;
      const unsigned char *ne = c_cart[ecum];
      const unsigned char *nf = c_cart[ncum(f) + fc];
      const int d = first_dir(nf);
      const int nd = nf[d];
      int j1[3] = {nf[0], nf[1], nf[2]};
      j1[d] -= 1;
      const int f1 = cart_index(j1[0], j1[1], j1[2]) - ncum(f - 1);
      std::integral_constant<int, f - 1> lv1;
      double v = g.QC[d] * get(lv1, ecum, f1, m) + g.WQ[d] * get(lv1, ecum, f1, m + 1);
      if constexpr (f >= 2) {
        if (nd >= 2) {
          j1[d] -= 1;
          const int f2 = cart_index(j1[0], j1[1], j1[2]) - ncum(f - 2);
          std::integral_constant<int, f - 2> lv2;
          v += (nd - 1) * g.inv2q * (get(lv2, ecum, f2, m) - g.rho_q * get(lv2, ecum, f2, m + 1));
        }
      }
      const int ed = ne[d];
      if (ed >= 1) {
        int i1[3] = {ne[0], ne[1], ne[2]};
        i1[d] -= 1;
        const int e1 = cart_index(i1[0], i1[1], i1[2]);
        v += ed * g.inv2pq * get(lv1, e1, f1, m + 1);
      }
      gk[O::loff(f) + (er * NF + fc) * LM + m] = v;
    }
    __syncwarp();
  });
  // accumulate [e|f]^0 for e in [LA, E], f in [LC, F]
  static_for<LC, F + 1>([&](auto fi) {
    constexpr int f = decltype(fi)::value;
    constexpr int NF = ncart(f);
    constexpr int CNT = O::NEA * NF;
    for (int idx = gl; idx < CNT; idx += G) {
      const int fc = idx % NF, er = idx / NF;
      const int ecum = ncum(LA) + er;
      acc[er * O::NFC + (ncum(f) - ncum(LC)) + fc] += get(fi, ecum, fc, 0);
    }
  });
  __syncwarp();
}

// Horizontal recursions after the primitive loops.  Returns the table holding
// [ab][c][d] (layout (a*nb + b) * nc * nd + c * nd + d).
template <int LA, int LB, int LC, int LD, int G>
__device__ __forceinline__ const double *os_hrr(const double *acc, double *bufA, double *bufB,
                                                int gl, const double *AB, const double *CD) {
  using O = Os<LA, LB, LC, LD>;
  constexpr int E = O::E, F = O::F, NFC = O::NFC;
  const double *src = acc;
  double *dst = bufA;
  static_for<1, LB + 1>([&](auto ji) {
    constexpr int j = decltype(ji)::value;
    constexpr int NB = ncart(j), NBP = ncart(j - 1);
    constexpr int CNT = (ncum(E - j + 1) - ncum(LA)) * NB * NFC;
    for (int idx = gl; idx < CNT; idx += G) {
      const int fr = idx % NFC;
      const int t = idx / NFC;
      const int bc = t % NB, ar = t / NB;
      const unsigned char *na = c_cart[ncum(LA) + ar];
      const unsigned char *nb = c_cart[ncum(j) + bc];
      const int d = first_dir(nb);
      int b1[3] = {nb[0], nb[1], nb[2]};
      b1[d] -= 1;
      const int bp = cart_index(b1[0], b1[1], b1[2]) - ncum(j - 1);
      int a1[3] = {na[0], na[1], na[2]};
      a1[d] += 1;
      const int a1r = cart_index(a1[0], a1[1], a1[2]) - ncum(LA);
      dst[(ar * NB + bc) * NFC + fr] =
          src[(a1r * NBP + bp) * NFC + fr] + AB[d] * src[(ar * NBP + bp) * NFC + fr];
    }
    __syncwarp();
    src = dst;
    dst = (dst == bufA) ? bufB : bufA;
  });
  static_for<1, LD + 1>([&](auto ji) {
    constexpr int j = decltype(ji)::value;
    constexpr int ND = ncart(j), NDP = ncart(j - 1);
    constexpr int NCJ = ncum(F - j + 1) - ncum(LC), NCP = ncum(F - j + 2) - ncum(LC);
    constexpr int CNT = O::NAB * NCJ * ND;
    for (int idx = gl; idx < CNT; idx += G) {
      const int dc = idx % ND;
      const int t = idx / ND;
      const int cr = t % NCJ, ab = t / NCJ;
      const unsigned char *nc = c_cart[ncum(LC) + cr];
      const unsigned char *nd = c_cart[ncum(j) + dc];
      const int d = first_dir(nd);
      int d1[3] = {nd[0], nd[1], nd[2]};
      d1[d] -= 1;
      const int dp = cart_index(d1[0], d1[1], d1[2]) - ncum(j - 1);
      int c1[3] = {nc[0], nc[1], nc[2]};
      c1[d] += 1;
      const int c1r = cart_index(c1[0], c1[1], c1[2]) - ncum(LC);
      dst[(ab * NCJ + cr) * ND + dc] =
          src[(ab * NCP + c1r) * NDP + dp] + CD[d] * src[(ab * NCP + cr) * NDP + dp];
    }
    __syncwarp();
    src = dst;
    dst = (dst == bufA) ? bufB : bufA;
  });
  return src;
}

struct ShellRef {
  int l, nprim, poff, fn;
  double xyz[3];
};

__device__ __forceinline__ ShellRef load_shell(const ShellSetDev &s, int i) {
  ShellRef r;
  r.l = s.l[i];
  r.nprim = s.nprim[i];
  r.poff = s.poff[i];
  r.fn = s.fn[i];
  r.xyz[0] = s.xyz[3 * i];
  r.xyz[1] = s.xyz[3 * i + 1];
  r.xyz[2] = s.xyz[3 * i + 2];
  return r;
}

// One quartet (a b|c d) by a group; d may be "unit" (exponent 0 at C) and b
// may be unit too.  Result via os_hrr.
template <int LA, int LB, int LC, int LD, int G>
__device__ __forceinline__ const double *os_quartet(
    const double *boys, double *scr, int gl, const ShellRef &sa, const double *ea,
    const double *ca, const ShellRef *sb, const double *eb, const double *cb, const ShellRef &sc,
    const double *ec, const double *cc, const ShellRef *sd, const double *ed, const double *cd) {
  using O = Os<LA, LB, LC, LD>;
  double *acc = scr;
  double *s1 = scr + O::ACC;
  double *gk = s1 + O::S1;
  for (int i = gl; i < O::ACC; i += G) acc[i] = 0.0;
  __syncwarp();
  const double *B = sb ? sb->xyz : sa.xyz;
  const double *D = sd ? sd->xyz : sc.xyz;
  const int nb = sb ? sb->nprim : 1, nd = sd ? sd->nprim : 1;
  for (int ia = 0; ia < sa.nprim; ++ia)
    for (int ib = 0; ib < nb; ++ib)
      for (int ic = 0; ic < sc.nprim; ++ic)
        for (int id = 0; id < nd; ++id) {
          PrimQ g;
          const double xb = sb ? eb[ib] : 0.0, wb = sb ? cb[ib] : 1.0;
          const double xd = sd ? ed[id] : 0.0, wd = sd ? cd[id] : 1.0;
          prim_setup(ea[ia], sa.xyz, xb, B, ec[ic], sc.xyz, xd, D, ca[ia] * wb * cc[ic] * wd, 0,
                     g);
          os_vrr_accumulate<LA, LB, LC, LD, G>(g, boys, acc, s1, gk, gl);
        }
  double AB[3], CD[3];
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    AB[x] = sa.xyz[x] - B[x];
    CD[x] = sc.xyz[x] - D[x];
  }
  double *bufA = scr + O::ACC;
  double *bufB = bufA + O::HMAX;
  return os_hrr<LA, LB, LC, LD, G>(acc, bufA, bufB, gl, AB, CD);
}

// ------------------------------------------------ three-centre triplet ----

struct Eri3cArgs {
  ShellSetDev orb, aux;
  const double *boys;
  const int2 *pairs;       // class segment, sorted by Schwarz factor
  const int *aux_list;     // aux shells of this l
  const int64_t *prefix;   // n_aux + 1 survivor prefix
  int n_aux;
  int p0, p1;              // aux function window [p0, p1)
  double *out;
  int64_t ld;
  int *flag;
  int64_t out_elems;
  // screening-ablation variants (ring buffer, index list): the class's pairs
  // in their original order with their Schwarz factors, the aux-shell factors
  const int2 *pairs_orig;
  const double *qpair_orig;
  const double *qaux;
  double tau;
  int np;
  int64_t *list;           // index-list variant: survivors (capacity n_aux * np)
  unsigned long long *count;
};

// One shell triplet (P | a b) by a group of G lanes (gl = lane in the group),
// written into the packed output; inactive groups compute a copy of a valid
// triplet (so the warp stays convergent) and write nothing.
template <int LC, int LA, int LB>
__device__ __forceinline__ void eri3c_triplet(const Eri3cArgs &a, double *scr, int gl, int Pi,
                                              int2 pr, bool active) {
  using O = Os<LA, LB, LC, 0>;
  constexpr int G = O::G;
  const ShellRef sc = load_shell(a.aux, Pi);
  const ShellRef sa = load_shell(a.orb, pr.x);
  const ShellRef sb = load_shell(a.orb, pr.y);
  const double *res = os_quartet<LA, LB, LC, 0, G>(
      a.boys, scr, gl, sa, a.orb.exps + sa.poff, a.orb.coefs + sa.poff, &sb,
      a.orb.exps + sb.poff, a.orb.coefs + sb.poff, sc, a.aux.exps + sc.poff,
      a.aux.coefs + sc.poff, nullptr, nullptr, nullptr);
  if (active) {
    constexpr int NA = ncart(LA), NB = ncart(LB), NC = ncart(LC);
    const bool diag = pr.x == pr.y;
    for (int idx = gl; idx < O::NOUT; idx += G) {
      const int ic = idx % NC;
      const int ab = idx / NC;
      const int ib = ab % NB, ia = ab / NB;
      const int P = sc.fn + ic;
      if (P < a.p0 || P >= a.p1) continue;
      int mu = sa.fn + ia, nu = sb.fn + ib;
      if (diag && mu < nu) continue;
      if (mu < nu) { const int t2 = mu; mu = nu; nu = t2; }
      const int64_t col = (int64_t)mu * (mu + 1) / 2 + nu;
      const int64_t o = (int64_t)(P - a.p0) * a.ld + col;
      if (o < 0 || o >= a.out_elems) { atomicExch(a.flag, 3); continue; }
      a.out[o] = res[idx] * c_cnorm[ncum(LA) + ia] * c_cnorm[ncum(LB) + ib] *
                 c_cnorm[ncum(LC) + ic];
    }
  }
}

}  // namespace bqc
