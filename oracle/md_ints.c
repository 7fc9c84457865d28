/*
 * Oracle integrals: a plain, slow FP64 CPU reference for the Gaussian
 * integrals of the density-fitted mean-field method (Sec. 2.2: the
 * Cholesky-decomposition ERIs and the metric they are fitted in).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only tests, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code with the CUDA library.
 *
 * Method: McMurchie-Davidson Hermite expansion (Helgaker, Jorgensen & Olsen,
 * "Molecular Electronic-Structure Theory", Sec. 9.5 for the E coefficients,
 * Sec. 9.9 for the R_tuv Coulomb integrals), Boys function by its power
 * series and the large-T asymptote with the downward/upward recursions
 * (same book, Sec. 9.8).  The paper itself prints no integral formulas.
 *
 * Conventions: Cartesian components of a shell of angular momentum l are
 * enumerated lexicographically (i from l down to 0, then j from l-i down to
 * 0, k = l-i-j: xx, xy, xz, yy, yz, zz).  Every component of every primitive
 * is unit-normalised, N = (2a/pi)^(3/4) (4a)^(l/2) / sqrt((2i-1)!!(2j-1)!!(2k-1)!!),
 * and each contracted shell is rescaled to unit self-overlap using this
 * file's own overlap integral.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define OL_MAX 4          /* maximum angular momentum of one shell        */
#define OL_SUM 16         /* maximum total angular momentum in one integral */
#define OE_I (OL_MAX + 3) /* E table extent (kinetic needs j + 2)          */
#define OE_T (2 * OL_MAX + 4)

/* ------------------------------------------------------------------ Boys */

/* F_m(T) = int_0^1 t^(2m) exp(-T t^2) dt for m = 0..mmax (HJO Sec. 9.8). */
void orc_boys(int mmax, double T, double *F) {
  if (T < 40.0) {
    /* Series F_m(T) = exp(-T) sum_k (2T)^k / ((2m+1)(2m+3)...(2m+2k+1)). */
    double denom = 2.0 * mmax + 1.0;
    double term = 1.0 / denom, sum = term;
    for (int k = 1; k < 2000; ++k) {
      term *= 2.0 * T / (denom + 2.0 * k);
      sum += term;
      if (term < 1e-18 * sum) break;
    }
    double e = exp(-T);
    F[mmax] = e * sum;
    /* Downward recursion F_{m-1} = (2T F_m + exp(-T)) / (2m - 1). */
    for (int m = mmax; m > 0; --m) F[m - 1] = (2.0 * T * F[m] + e) / (2.0 * m - 1.0);
  } else {
    /* erf(sqrt(T)) = 1 to double precision for T >= 40. */
    double e = exp(-T);
    F[0] = 0.5 * sqrt(M_PI / T);
    /* Upward recursion F_{m+1} = ((2m+1) F_m - exp(-T)) / (2T), stable here. */
    for (int m = 0; m < mmax; ++m) F[m + 1] = ((2.0 * m + 1.0) * F[m] - e) / (2.0 * T);
  }
}

/* -------------------------------------------------------------- shells */

typedef struct {
  int l, nprim;
  double A[3];
  const double *exps;
  double coef[64]; /* contraction coefficient x primitive radial norm x renorm */
} oshell;

static int ncart(int l) { return (l + 1) * (l + 2) / 2; }

static void cart_list(int l, int (*ijk)[3]) {
  int n = 0;
  for (int i = l; i >= 0; --i)
    for (int j = l - i; j >= 0; --j) {
      ijk[n][0] = i;
      ijk[n][1] = j;
      ijk[n][2] = l - i - j;
      ++n;
    }
}

static double dfact_odd(int n) { /* (2n-1)!! with (-1)!! = 1 */
  double r = 1.0;
  for (int k = 2 * n - 1; k > 1; k -= 2) r *= k;
  return r;
}

static double comp_norm(int i, int j, int k) {
  return 1.0 / sqrt(dfact_odd(i) * dfact_odd(j) * dfact_odd(k));
}

/* --------------------------------------------------- Hermite E (HJO 9.5) */

/* E[i][j][t] for one Cartesian axis of the product of x_A^i e^{-a x_A^2} and
 * x_B^j e^{-b x_B^2}.  E^{00}_0 = exp(-ab/p X_AB^2);
 * E^{i+1,j}_t = E^{ij}_{t-1}/(2p) + X_PA E^{ij}_t + (t+1) E^{ij}_{t+1},
 * E^{i,j+1}_t = E^{ij}_{t-1}/(2p) + X_PB E^{ij}_t + (t+1) E^{ij}_{t+1}. */
static void hermite_e(int imax, int jmax, double a, double b, double Ax, double Bx,
                      double E[OE_I][OE_I][OE_T]) {
  double p = a + b;
  double Px = (a * Ax + b * Bx) / p;
  double XPA = Px - Ax, XPB = Px - Bx, XAB = Ax - Bx;
  memset(E, 0, sizeof(double) * OE_I * OE_I * OE_T);
  E[0][0][0] = exp(-a * b / p * XAB * XAB);
  double h = 0.5 / p;
  for (int i = 0; i <= imax; ++i) {
    for (int j = 0; j <= jmax; ++j) {
      if (i == 0 && j == 0) continue;
      if (j == 0) {
        /* raise i from i-1 */
        for (int t = 0; t <= i + j; ++t) {
          double v = XPA * E[i - 1][j][t];
          if (t > 0) v += h * E[i - 1][j][t - 1];
          if (t + 1 <= i - 1 + j) v += (t + 1) * E[i - 1][j][t + 1];
          E[i][j][t] = v;
        }
      } else {
        /* raise j from j-1 */
        for (int t = 0; t <= i + j; ++t) {
          double v = XPB * E[i][j - 1][t];
          if (t > 0) v += h * E[i][j - 1][t - 1];
          if (t + 1 <= i + j - 1) v += (t + 1) * E[i][j - 1][t + 1];
          E[i][j][t] = v;
        }
      }
    }
  }
}

/* ------------------------------------------------ R_tuv (HJO 9.9.18-20) */

#define RI(t, u, v) (((t) * (OL_SUM + 1) + (u)) * (OL_SUM + 1) + (v))
#define RSZ ((OL_SUM + 1) * (OL_SUM + 1) * (OL_SUM + 1))

/* R^0_{tuv} for t+u+v <= L: R^n_000 = (-2 alpha)^n F_n(alpha R^2),
 * R^n_{t+1,u,v} = t R^{n+1}_{t-1,u,v} + X R^{n+1}_{tuv} (and likewise u, v). */
static void hermite_r(int L, double alpha, const double PC[3], double *R0) {
  double F[OL_SUM + 1];
  double T = alpha * (PC[0] * PC[0] + PC[1] * PC[1] + PC[2] * PC[2]);
  orc_boys(L, T, F);
  double bufA[RSZ], bufB[RSZ];
  double *cur = bufA, *nxt = bufB;
  /* level n = L: only R_000.  Every entry read at level n (t+u+v <= L-n-1
   * at level n+1) was written at level n+1, so no clearing is needed. */
  double m2a = -2.0 * alpha, pw = 1.0;
  for (int n = 0; n < L; ++n) pw *= m2a;
  nxt[RI(0, 0, 0)] = pw * F[L];
  for (int n = L - 1; n >= 0; --n) {
    int lim = L - n;
    pw = 1.0;
    for (int k = 0; k < n; ++k) pw *= m2a;
    for (int t = 0; t <= lim; ++t)
      for (int u = 0; u <= lim - t; ++u)
        for (int v = 0; v <= lim - t - u; ++v) {
          double val;
          if (t == 0 && u == 0 && v == 0) {
            val = pw * F[n];
          } else if (t > 0) {
            val = PC[0] * nxt[RI(t - 1, u, v)];
            if (t > 1) val += (t - 1) * nxt[RI(t - 2, u, v)];
          } else if (u > 0) {
            val = PC[1] * nxt[RI(t, u - 1, v)];
            if (u > 1) val += (u - 1) * nxt[RI(t, u - 2, v)];
          } else {
            val = PC[2] * nxt[RI(t, u, v - 1)];
            if (v > 1) val += (v - 1) * nxt[RI(t, u, v - 2)];
          }
          cur[RI(t, u, v)] = val;
        }
    double *tmp = cur;
    cur = nxt;
    nxt = tmp;
  }
  for (int t = 0; t <= L; ++t)
    for (int u = 0; u <= L - t; ++u)
      for (int v = 0; v <= L - t - u; ++v) R0[RI(t, u, v)] = nxt[RI(t, u, v)];
}

/* --------------------------------------- generic 4-index Coulomb quartet */

/* (ab|cd) for contracted shells; b and/or d may be a "unit" shell (l = 0,
 * exponent 0, coefficient 1).  out[ia][ib][ic][id], components unnormalised
 * by the per-component factor (the caller applies it). */
static void quartet(const oshell *a, const oshell *b, const oshell *c, const oshell *d,
                    double *out) {
  int na = ncart(a->l), nb = ncart(b->l), nc = ncart(c->l), nd = ncart(d->l);
  int ca[15][3], cb[15][3], cc[15][3], cd[15][3];
  cart_list(a->l, ca);
  cart_list(b->l, cb);
  cart_list(c->l, cc);
  cart_list(d->l, cd);
  int L = a->l + b->l + c->l + d->l;
  int nout = na * nb * nc * nd;
  memset(out, 0, sizeof(double) * nout);
  double *R = (double *)malloc(sizeof(double) * RSZ);
  double Eab[3][OE_I][OE_I][OE_T];
  double Ecd[3][OE_I][OE_I][OE_T];
  for (int pa = 0; pa < a->nprim; ++pa)
    for (int pb = 0; pb < b->nprim; ++pb) {
      double al = a->exps[pa], be = b->exps[pb], p = al + be;
      double P[3];
      for (int x = 0; x < 3; ++x) {
        P[x] = (al * a->A[x] + be * b->A[x]) / p;
        hermite_e(a->l, b->l, al, be, a->A[x], b->A[x], Eab[x]);
      }
      double cab = a->coef[pa] * b->coef[pb];
      for (int pc = 0; pc < c->nprim; ++pc)
        for (int pd = 0; pd < d->nprim; ++pd) {
          double ga = c->exps[pc], de = d->exps[pd], q = ga + de;
          double Q[3], PQ[3];
          for (int x = 0; x < 3; ++x) {
            Q[x] = (ga * c->A[x] + de * d->A[x]) / q;
            PQ[x] = P[x] - Q[x];
            hermite_e(c->l, d->l, ga, de, c->A[x], d->A[x], Ecd[x]);
          }
          double alpha = p * q / (p + q);
          hermite_r(L, alpha, PQ, R);
          double pref = cab * c->coef[pc] * d->coef[pd] * 2.0 * pow(M_PI, 2.5) /
                        (p * q * sqrt(p + q));
          int idx = 0;
          for (int ia = 0; ia < na; ++ia)
            for (int ib = 0; ib < nb; ++ib)
              for (int ic = 0; ic < nc; ++ic)
                for (int id = 0; id < nd; ++id, ++idx) {
                  int ax = ca[ia][0], ay = ca[ia][1], az = ca[ia][2];
                  int bx = cb[ib][0], by = cb[ib][1], bz = cb[ib][2];
                  int cx = cc[ic][0], cy = cc[ic][1], cz = cc[ic][2];
                  int dx = cd[id][0], dy = cd[id][1], dz = cd[id][2];
                  double s = 0.0;
                  for (int t = 0; t <= ax + bx; ++t)
                    for (int u = 0; u <= ay + by; ++u)
                      for (int v = 0; v <= az + bz; ++v) {
                        double e1 = Eab[0][ax][bx][t] * Eab[1][ay][by][u] * Eab[2][az][bz][v];
                        if (e1 == 0.0) continue;
                        double s2 = 0.0;
                        for (int tt = 0; tt <= cx + dx; ++tt)
                          for (int uu = 0; uu <= cy + dy; ++uu)
                            for (int vv = 0; vv <= cz + dz; ++vv) {
                              double e2 = Ecd[0][cx][dx][tt] * Ecd[1][cy][dy][uu] *
                                          Ecd[2][cz][dz][vv];
                              double sg = ((tt + uu + vv) & 1) ? -1.0 : 1.0;
                              s2 += sg * e2 * R[RI(t + tt, u + uu, v + vv)];
                            }
                        s += e1 * s2;
                      }
                  out[idx] += pref * s;
                }
        }
    }
  free(R);
}

/* ------------------------------------------------------ basis handling */

typedef struct {
  int nshell, nfn;
  oshell *sh;
  int *off; /* first function of each shell */
} obasis;

static void overlap_prim_shell(const oshell *a, const oshell *b, double *out);

/* Builds the shell array from flat arrays; applies primitive radial norms and
 * rescales each contracted shell to unit self-overlap (of its first
 * component, which fixes all components, see comp_norm). */
static obasis make_basis(int nshell, const int *l, const int *nprim, const int *poff,
                         const double *xyz, const double *exps, const double *coefs) {
  obasis B;
  B.nshell = nshell;
  B.sh = (oshell *)calloc(nshell, sizeof(oshell));
  B.off = (int *)calloc(nshell + 1, sizeof(int));
  int f = 0;
  for (int s = 0; s < nshell; ++s) {
    oshell *S = &B.sh[s];
    S->l = l[s];
    S->nprim = nprim[s];
    S->exps = exps + poff[s];
    for (int x = 0; x < 3; ++x) S->A[x] = xyz[3 * s + x];
    for (int k = 0; k < S->nprim; ++k) {
      double a = S->exps[k];
      S->coef[k] = coefs[poff[s] + k] * pow(2.0 * a / M_PI, 0.75) * pow(4.0 * a, 0.5 * S->l);
    }
    /* self-overlap of component 0 (x^l), then renormalise */
    int nc = ncart(S->l);
    double *ov = (double *)malloc(sizeof(double) * nc * nc);
    overlap_prim_shell(S, S, ov);
    double n0 = comp_norm(S->l, 0, 0);
    double self = ov[0] * n0 * n0;
    double sc = 1.0 / sqrt(self);
    for (int k = 0; k < S->nprim; ++k) S->coef[k] *= sc;
    free(ov);
    B.off[s] = f;
    f += nc;
  }
  B.off[nshell] = f;
  B.nfn = f;
  return B;
}

static void free_basis(obasis *B) {
  free(B->sh);
  free(B->off);
}

static oshell unit_shell(const double *A) {
  static const double zero = 0.0;
  oshell u;
  memset(&u, 0, sizeof(u));
  u.l = 0;
  u.nprim = 1;
  u.exps = &zero;
  u.coef[0] = 1.0;
  for (int x = 0; x < 3; ++x) u.A[x] = A[x];
  return u;
}

/* ----------------------------------------------------- one-electron parts */

/* Overlap block without component norms (HJO 9.5.41: S_ij = E^{ij}_0 sqrt(pi/p)). */
static void overlap_prim_shell(const oshell *a, const oshell *b, double *out) {
  int na = ncart(a->l), nb = ncart(b->l);
  int ca[15][3], cb[15][3];
  cart_list(a->l, ca);
  cart_list(b->l, cb);
  memset(out, 0, sizeof(double) * na * nb);
  double E[3][OE_I][OE_I][OE_T];
  for (int pa = 0; pa < a->nprim; ++pa)
    for (int pb = 0; pb < b->nprim; ++pb) {
      double al = a->exps[pa], be = b->exps[pb], p = al + be;
      for (int x = 0; x < 3; ++x) hermite_e(a->l, b->l, al, be, a->A[x], b->A[x], E[x]);
      double f = a->coef[pa] * b->coef[pb] * pow(M_PI / p, 1.5);
      for (int i = 0; i < na; ++i)
        for (int j = 0; j < nb; ++j)
          out[i * nb + j] += f * E[0][ca[i][0]][cb[j][0]][0] * E[1][ca[i][1]][cb[j][1]][0] *
                             E[2][ca[i][2]][cb[j][2]][0];
    }
}

/* Kinetic block: per axis T_ij = -1/2 [j(j-1) S_{i,j-2} - 2b(2j+1) S_ij + 4b^2 S_{i,j+2}]
 * with 1-D overlaps S_ij = E^{ij}_0 sqrt(pi/p) (HJO 9.3.38-40 in Hermite form). */
static void kinetic_shell(const oshell *a, const oshell *b, double *out) {
  int na = ncart(a->l), nb = ncart(b->l);
  int ca[15][3], cb[15][3];
  cart_list(a->l, ca);
  cart_list(b->l, cb);
  memset(out, 0, sizeof(double) * na * nb);
  double E[3][OE_I][OE_I][OE_T];
  for (int pa = 0; pa < a->nprim; ++pa)
    for (int pb = 0; pb < b->nprim; ++pb) {
      double al = a->exps[pa], be = b->exps[pb], p = al + be;
      for (int x = 0; x < 3; ++x) hermite_e(a->l, b->l + 2, al, be, a->A[x], b->A[x], E[x]);
      double sq = sqrt(M_PI / p);
      double f = a->coef[pa] * b->coef[pb];
      for (int i = 0; i < na; ++i)
        for (int j = 0; j < nb; ++j) {
          double S1[3], T1[3];
          for (int x = 0; x < 3; ++x) {
            int ii = ca[i][x], jj = cb[j][x];
            S1[x] = E[x][ii][jj][0] * sq;
            double t = -2.0 * be * (2 * jj + 1) * E[x][ii][jj][0] +
                       4.0 * be * be * E[x][ii][jj + 2][0];
            if (jj >= 2) t += jj * (jj - 1) * E[x][ii][jj - 2][0];
            T1[x] = -0.5 * t * sq;
          }
          out[i * nb + j] += f * (T1[0] * S1[1] * S1[2] + S1[0] * T1[1] * S1[2] +
                                  S1[0] * S1[1] * T1[2]);
        }
    }
}

/* Nuclear attraction -sum_C Z_C (2 pi / p) sum_tuv E_t E_u E_v R_tuv(p, P - C). */
static void nuclear_shell(const oshell *a, const oshell *b, int natom, const int *Z,
                          const double *C, double *out) {
  int na = ncart(a->l), nb = ncart(b->l);
  int ca[15][3], cb[15][3];
  cart_list(a->l, ca);
  cart_list(b->l, cb);
  memset(out, 0, sizeof(double) * na * nb);
  double E[3][OE_I][OE_I][OE_T];
  double *R = (double *)malloc(sizeof(double) * RSZ);
  int L = a->l + b->l;
  for (int pa = 0; pa < a->nprim; ++pa)
    for (int pb = 0; pb < b->nprim; ++pb) {
      double al = a->exps[pa], be = b->exps[pb], p = al + be;
      double P[3];
      for (int x = 0; x < 3; ++x) {
        P[x] = (al * a->A[x] + be * b->A[x]) / p;
        hermite_e(a->l, b->l, al, be, a->A[x], b->A[x], E[x]);
      }
      for (int n = 0; n < natom; ++n) {
        double PC[3] = {P[0] - C[3 * n], P[1] - C[3 * n + 1], P[2] - C[3 * n + 2]};
        hermite_r(L, p, PC, R);
        double f = -Z[n] * a->coef[pa] * b->coef[pb] * 2.0 * M_PI / p;
        for (int i = 0; i < na; ++i)
          for (int j = 0; j < nb; ++j) {
            double s = 0.0;
            for (int t = 0; t <= ca[i][0] + cb[j][0]; ++t)
              for (int u = 0; u <= ca[i][1] + cb[j][1]; ++u)
                for (int v = 0; v <= ca[i][2] + cb[j][2]; ++v)
                  s += E[0][ca[i][0]][cb[j][0]][t] * E[1][ca[i][1]][cb[j][1]][u] *
                       E[2][ca[i][2]][cb[j][2]][v] * R[RI(t, u, v)];
            out[i * nb + j] += f * s;
          }
      }
    }
  free(R);
}

static void comp_norms(int l, double *nrm) {
  int c[15][3];
  cart_list(l, c);
  for (int i = 0; i < ncart(l); ++i) nrm[i] = comp_norm(c[i][0], c[i][1], c[i][2]);
}

/* which: 0 overlap, 1 kinetic, 2 nuclear attraction.  out is nfn x nfn. */
int orc_one_electron(int which, int nshell, const int *l, const int *nprim, const int *poff,
                     const double *xyz, const double *exps, const double *coefs, int natom,
                     const int *Z, const double *C, double *out) {
  obasis B = make_basis(nshell, l, nprim, poff, xyz, exps, coefs);
  int N = B.nfn;
#pragma omp parallel for schedule(dynamic)
  for (int s1 = 0; s1 < nshell; ++s1)
    for (int s2 = 0; s2 < nshell; ++s2) {
      double blk[15 * 15], n1[15], n2[15];
      const oshell *a = &B.sh[s1], *b = &B.sh[s2];
      if (which == 0)
        overlap_prim_shell(a, b, blk);
      else if (which == 1)
        kinetic_shell(a, b, blk);
      else
        nuclear_shell(a, b, natom, Z, C, blk);
      comp_norms(a->l, n1);
      comp_norms(b->l, n2);
      int na = ncart(a->l), nb = ncart(b->l);
      for (int i = 0; i < na; ++i)
        for (int j = 0; j < nb; ++j)
          out[(size_t)(B.off[s1] + i) * N + B.off[s2] + j] = blk[i * nb + j] * n1[i] * n2[j];
    }
  free_basis(&B);
  return N;
}

/* --------------------------------------------------- two-electron parts */

/* (P|Q) over the auxiliary basis: out is naux x naux. */
int orc_int2c(int nshell, const int *l, const int *nprim, const int *poff, const double *xyz,
              const double *exps, const double *coefs, double *out) {
  obasis B = make_basis(nshell, l, nprim, poff, xyz, exps, coefs);
  int N = B.nfn;
#pragma omp parallel for schedule(dynamic)
  for (int s1 = 0; s1 < nshell; ++s1)
    for (int s2 = 0; s2 < nshell; ++s2) {
      double blk[15 * 15], n1[15], n2[15];
      const oshell *a = &B.sh[s1], *c = &B.sh[s2];
      oshell ua = unit_shell(a->A), uc = unit_shell(c->A);
      quartet(a, &ua, c, &uc, blk);
      comp_norms(a->l, n1);
      comp_norms(c->l, n2);
      int na = ncart(a->l), nc = ncart(c->l);
      for (int i = 0; i < na; ++i)
        for (int j = 0; j < nc; ++j)
          out[(size_t)(B.off[s1] + i) * N + B.off[s2] + j] = blk[i * nc + j] * n1[i] * n2[j];
    }
  free_basis(&B);
  return N;
}

/* (P|mu nu) for the aux shells listed in psel and the orbital shell pairs
 * (asel[k], bsel[k]).  Output layout: for each selected aux shell (in psel
 * order) its components, times for each pair k its na x nb block:
 * out[(fP)][k-block] packed consecutively per P component row; row length is
 * the sum over k of na_k * nb_k.  Returns the row length. */
int orc_int3c(int naux_sh, const int *la, const int *npa, const int *poffa, const double *xyza,
              const double *expsa, const double *coefsa, int norb_sh, const int *lo,
              const int *npo, const int *poffo, const double *xyzo, const double *expso,
              const double *coefso, int npsel, const int *psel, int npair, const int *asel,
              const int *bsel, double *out) {
  obasis A = make_basis(naux_sh, la, npa, poffa, xyza, expsa, coefsa);
  obasis O = make_basis(norb_sh, lo, npo, poffo, xyzo, expso, coefso);
  int *col = (int *)malloc(sizeof(int) * (npair + 1));
  col[0] = 0;
  for (int k = 0; k < npair; ++k)
    col[k + 1] = col[k] + ncart(O.sh[asel[k]].l) * ncart(O.sh[bsel[k]].l);
  int rowlen = col[npair];
  int *prow = (int *)malloc(sizeof(int) * (npsel + 1));
  prow[0] = 0;
  for (int i = 0; i < npsel; ++i) prow[i + 1] = prow[i] + ncart(A.sh[psel[i]].l);
#pragma omp parallel for schedule(dynamic) collapse(2)
  for (int i = 0; i < npsel; ++i)
    for (int k = 0; k < npair; ++k) {
      double blk[15 * 15 * 15], nP[15], n1[15], n2[15];
      const oshell *P = &A.sh[psel[i]];
      const oshell *a = &O.sh[asel[k]], *b = &O.sh[bsel[k]];
      oshell uP = unit_shell(P->A);
      quartet(P, &uP, a, b, blk);
      comp_norms(P->l, nP);
      comp_norms(a->l, n1);
      comp_norms(b->l, n2);
      int np = ncart(P->l), na = ncart(a->l), nb = ncart(b->l);
      for (int ip = 0; ip < np; ++ip)
        for (int ia = 0; ia < na; ++ia)
          for (int ib = 0; ib < nb; ++ib)
            out[(size_t)(prow[i] + ip) * rowlen + col[k] + ia * nb + ib] =
                blk[(ip * na + ia) * nb + ib] * nP[ip] * n1[ia] * n2[ib];
    }
  free(col);
  free(prow);
  free_basis(&A);
  free_basis(&O);
  return rowlen;
}

/* Full (mu nu|lambda sigma) over the orbital basis, N^4 (small systems only). */
int orc_int4c(int nshell, const int *l, const int *nprim, const int *poff, const double *xyz,
              const double *exps, const double *coefs, double *out) {
  obasis B = make_basis(nshell, l, nprim, poff, xyz, exps, coefs);
  size_t N = B.nfn;
#pragma omp parallel for schedule(dynamic) collapse(2)
  for (int s1 = 0; s1 < nshell; ++s1)
    for (int s2 = 0; s2 < nshell; ++s2) {
      double *blk = (double *)malloc(sizeof(double) * 15 * 15 * 15 * 15);
      double n1[15], n2[15], n3[15], n4[15];
      for (int s3 = 0; s3 < nshell; ++s3)
        for (int s4 = 0; s4 < nshell; ++s4) {
          const oshell *a = &B.sh[s1], *b = &B.sh[s2], *c = &B.sh[s3], *d = &B.sh[s4];
          quartet(a, b, c, d, blk);
          comp_norms(a->l, n1);
          comp_norms(b->l, n2);
          comp_norms(c->l, n3);
          comp_norms(d->l, n4);
          int na = ncart(a->l), nb = ncart(b->l), nc = ncart(c->l), nd = ncart(d->l);
          for (int i = 0; i < na; ++i)
            for (int j = 0; j < nb; ++j)
              for (int k = 0; k < nc; ++k)
                for (int m = 0; m < nd; ++m) {
                  size_t I = B.off[s1] + i, J = B.off[s2] + j, K = B.off[s3] + k,
                         M = B.off[s4] + m;
                  out[((I * N + J) * N + K) * N + M] =
                      blk[((i * nb + j) * nc + k) * nd + m] * n1[i] * n2[j] * n3[k] * n4[m];
                }
        }
      free(blk);
    }
  free_basis(&B);
  return (int)N;
}

/* Nuclear repulsion sum_{A<B} Z_A Z_B / R_AB. */
double orc_nuclear_repulsion(int natom, const int *Z, const double *C) {
  double e = 0.0;
  for (int a = 0; a < natom; ++a)
    for (int b = 0; b < a; ++b) {
      double dx = C[3 * a] - C[3 * b], dy = C[3 * a + 1] - C[3 * b + 1],
             dz = C[3 * a + 2] - C[3 * b + 2];
      e += Z[a] * Z[b] / sqrt(dx * dx + dy * dy + dz * dz);
    }
  return e;
}
