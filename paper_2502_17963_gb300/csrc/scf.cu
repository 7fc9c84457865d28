// Closed-shell SCF driver around the DF Fock build (bqc_jk).
//
// Protocol (Szabo & Ostlund Sec. 3.4.6 with Pulay DIIS; identical to the
// oracle's): canonical orthogonalisation X = U s^{-1/2} over eigenvalues of S
// above orth_thresh; core-Hamiltonian guess; each iteration builds J, K from
// C_occ, F = H + 2J - K, E = sum D (H + F) + E_nn, e = X^T (F D S - S D F) X;
// converged when max|e| < diis_tol and |E - E_prev| < max(energy_tol,
// eps_64 * N * |E|) (the second term is the rounding noise of the energy
// itself, a sum over N^2 products, which exceeds 1e-10 Eh from N of about
// 800); otherwise DIIS over the last diis_space (F, e) pairs once two are
// stored, and diagonalise X^T F X.  Precision staging: a MIXED first stage
// switches to FP64 (DIIS history cleared) at stage_tol or at the mixed
// stage's error floor (see the rule at the switch below).
//
// Linear algebra here (eigh, small GEMMs, dots) uses cuSOLVER / cuBLAS in
// FP64; everything is column-major; symmetric matrices need no conversion.
#include <cublas_v2.h>
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <vector>

#include "bqc_internal.h"
#include "df_internal.h"

namespace bqc {

#define BQC_BLAS_TRY(expr)                                                   \
  do {                                                                       \
    if ((expr) != CUBLAS_STATUS_SUCCESS) {                                   \
      ::bqc::set_error("cuBLAS call failed: " #expr, __FILE__, __LINE__);    \
      return BQC_E_CUDA;                                                     \
    }                                                                        \
  } while (0)
#define BQC_SOLVER_TRY(expr)                                                 \
  do {                                                                       \
    if ((expr) != CUSOLVER_STATUS_SUCCESS) {                                 \
      ::bqc::set_error("cuSOLVER call failed: " #expr, __FILE__, __LINE__);  \
      return BQC_E_CUDA;                                                     \
    }                                                                        \
  } while (0)

__global__ void k_axpby3(int64_t n, const double *a, double ca, const double *b, double cb,
                         const double *c, double cc, double *out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = ca * a[i] + cb * b[i] + (c ? cc * c[i] : 0.0);
}

// out = M - M^T (column-major n x n)
__global__ void k_antisym(int n, const double *M, double *out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)n * n) return;
  const int64_t r = i % n, c = i / n;
  out[i] = M[i] - M[r * n + c];
}

// X[:, j] = U[:, k0 + j] / sqrt(s[k0 + j])
__global__ void k_orth(int n, int nmo, int k0, const double *U, const double *s, double *X) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)n * nmo) return;
  const int64_t r = i % n, j = i / n;
  X[i] = U[(k0 + j) * (int64_t)n + r] * rsqrt(s[k0 + j]);
}

// row-major out[r][c] = colmajor in[c * rows + r]  (rows x cols)
// out (column-major, leading dimension ld) = in (row-major rows x cols)
__global__ void k_rm_to_cm(int rows, int cols, const double *in, double *out, int64_t ld) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)rows * cols) return;
  const int64_t r = i / cols, c = i % cols;
  out[c * ld + r] = in[i];
}

__global__ void k_cm_to_rm(int rows, int cols, const double *in, int64_t ld, double *out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)rows * cols) return;
  const int64_t r = i / cols, c = i % cols;
  out[i] = in[c * ld + r];
}

// V[nu][c] = U[k0 + c][nu] * sqrt(|ev[k0 + c]|) for c < cnt, 0 for cnt <= c < ncol
// (U column-major n x n eigenvectors; V row-major n x ncol): the scaled
// eigenvector factor of one sign of a symmetric matrix.
__global__ void k_eig_factor(int n, const double *U, const double *ev, int k0, int cnt,
                             int ncol, double *V) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)n * ncol) return;
  const int64_t nu = i / ncol;
  const int c = (int)(i % ncol);
  V[i] = c < cnt ? U[(int64_t)(k0 + c) * n + nu] * sqrt(fabs(ev[k0 + c])) : 0.0;
}

// Cw = (Ca + Ct) / 2, Cd = Ct - Ca (row-major n x no) from column-major Ca,
// Ct (n x no): the midpoint and difference of two sets of occupied orbitals.
__global__ void k_procrustes_pair(int n, int no, const double *Ca, const double *Ct, double *Cw,
                                  double *Cd) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)n * no) return;
  const int64_t r = i / no, c = i % no;
  const double a = Ca[c * n + r], t = Ct[c * n + r];
  Cw[i] = 0.5 * (a + t);
  Cd[i] = t - a;
}

// W[:, j] = V[:, j] / sqrt(lam[j]) (column-major no x no)
__global__ void k_scale_cols_rsqrt(int no, const double *V, const double *lam, double *W) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)no * no) return;
  W[i] = V[i] / sqrt(lam[i / no]);
}

// incremental_build's answer when the increment cannot be formed: the
// iteration is built in full instead
constexpr int kIncFull = 1;

// F = Fref + 2 (Jp - Jm) - (Kp - Km)
__global__ void k_inc_fock(int64_t n, const double *Fref, const double *Jp, const double *Jm,
                           const double *Kp, const double *Km, double *F) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) F[i] = Fref[i] + 2.0 * (Jp[i] - Jm[i]) - (Kp[i] - Km[i]);
}

static inline unsigned nblk(int64_t n) { return (unsigned)((n + 255) / 256); }

// Instantiated CUDA graphs of the Fock build, one per precision, destroyed on
// every exit path.
struct GraphSet {
  cudaGraphExec_t g[4] = {nullptr, nullptr, nullptr, nullptr};
  void clear() {
    for (auto &e : g)
      if (e) cudaGraphExecDestroy(e), e = nullptr;
  }
  ~GraphSet() { clear(); }
};

// Solves the (m+1) x (m+1) Pulay system by Gaussian elimination with partial
// pivoting; returns false if singular.
static bool diis_solve(const std::vector<double> &Bm, int m, std::vector<double> &c) {
  const int n = m + 1;
  std::vector<double> A((size_t)n * (n + 1), 0.0);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) A[(size_t)i * (n + 1) + j] = Bm[(size_t)i * m + j];
  for (int i = 0; i < m; ++i) {
    A[(size_t)i * (n + 1) + m] = -1.0;
    A[(size_t)m * (n + 1) + i] = -1.0;
  }
  A[(size_t)m * (n + 1) + n] = -1.0;  // rhs
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(A[(size_t)i * (n + 1) + k]) > std::fabs(A[(size_t)p * (n + 1) + k])) p = i;
    if (A[(size_t)p * (n + 1) + k] == 0.0) return false;
    if (p != k)
      for (int j = 0; j <= n; ++j) std::swap(A[(size_t)p * (n + 1) + j], A[(size_t)k * (n + 1) + j]);
    for (int i = k + 1; i < n; ++i) {
      const double f = A[(size_t)i * (n + 1) + k] / A[(size_t)k * (n + 1) + k];
      for (int j = k; j <= n; ++j) A[(size_t)i * (n + 1) + j] -= f * A[(size_t)k * (n + 1) + j];
    }
  }
  std::vector<double> x(n);
  for (int i = n - 1; i >= 0; --i) {
    double v = A[(size_t)i * (n + 1) + n];
    for (int j = i + 1; j < n; ++j) v -= A[(size_t)i * (n + 1) + j] * x[j];
    x[i] = v / A[(size_t)i * (n + 1) + i];
  }
  c.assign(x.begin(), x.begin() + m);
  for (double v : c)
    if (!std::isfinite(v)) return false;
  return true;
}

// cuBLAS / cuSOLVER handles cached per host thread and device: creating a
// handle allocates device memory, which synchronises the device and would
// serialise concurrent solves (serving slots run one thread each).
struct ScfWork {
  cublasHandle_t blas = nullptr;
  cusolverDnHandle_t sol = nullptr;
};

struct HandleCache {
  int device = -1;
  cublasHandle_t blas = nullptr;
  cusolverDnHandle_t sol = nullptr;
};

static int get_handles(int device, ScfWork &w) {
  static thread_local HandleCache hc;
  if (hc.device != device) {
    if (hc.blas) cublasDestroy(hc.blas);
    if (hc.sol) cusolverDnDestroy(hc.sol);
    hc.blas = nullptr;
    hc.sol = nullptr;
    BQC_BLAS_TRY(cublasCreate(&hc.blas));
    BQC_SOLVER_TRY(cusolverDnCreate(&hc.sol));
    hc.device = device;
  }
  w.blas = hc.blas;
  w.sol = hc.sol;
  return BQC_OK;
}

// Symmetric eigen-decomposition in place (columns of A become eigenvectors).
static int eigh(ScfWork &w, Ctx *ctx, double *A, int n, double *evals, DBuf &work, DBuf &info,
                cudaStream_t s) {
  int lwork = 0;
  BQC_SOLVER_TRY(cusolverDnDsyevd_bufferSize(w.sol, CUSOLVER_EIG_MODE_VECTOR,
                                             CUBLAS_FILL_MODE_LOWER, n, A, n, evals, &lwork));
  if (work.n < (size_t)lwork * 8) BQC_TRY(work.alloc(ctx, (size_t)std::max(lwork, 1) * 8));
  if (!info.p) BQC_TRY(info.alloc(ctx, sizeof(int)));
  BQC_SOLVER_TRY(cusolverDnDsyevd(w.sol, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, A,
                                  n, evals, work.as<double>(), lwork, info.as<int>()));
  int h = 0;
  BQC_CUDA_TRY(cudaMemcpyAsync(&h, info.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  BQC_CUDA_TRY(cudaStreamSynchronize(s));
  if (h != 0) {
    set_error("syevd did not converge", __FILE__, __LINE__);
    return BQC_E_CUDA;
  }
  return BQC_OK;
}

int scf_run(Ctx *ctx, Df *df, const bqc_scf_opts &o, cudaStream_t s, bqc_scf_result *res) {
  const Basis *b = df->basis;
  const int n = b->nbf, no = b->nocc;
  const int64_t nn = (int64_t)n * n;
  ScfWork w;
  BQC_TRY(get_handles(ctx->device, w));
  BQC_BLAS_TRY(cublasSetStream(w.blas, s));
  BQC_BLAS_TRY(cublasSetPointerMode(w.blas, CUBLAS_POINTER_MODE_HOST));
  BQC_BLAS_TRY(cublasSetMathMode(w.blas, CUBLAS_PEDANTIC_MATH));
  BQC_SOLVER_TRY(cusolverDnSetStream(w.sol, s));
  DBuf S, T, V, H, F, J, K, D, X, U, ev, Cc, Fp, t1, t2, Crm, work, info, Fx;
  for (DBuf *p : {&S, &T, &V, &H, &F, &J, &K, &D, &X, &U, &Cc, &Fp, &t1, &t2, &Fx})
    BQC_TRY(p->alloc(ctx, nn * 8));
  BQC_TRY(ev.alloc(ctx, (size_t)n * 8));
  BQC_TRY(Crm.alloc(ctx, (size_t)n * no * 8));
  BQC_TRY(launch_one_electron(b, S.as<double>(), T.as<double>(), V.as<double>(), s));
  k_axpby3<<<nblk(nn), 256, 0, s>>>(nn, T.as<double>(), 1.0, V.as<double>(), 1.0, nullptr, 0.0,
                                    H.as<double>());
  BQC_LAUNCH_CHECK();
  // canonical orthogonalisation
  BQC_CUDA_TRY(cudaMemcpyAsync(U.p, S.p, nn * 8, cudaMemcpyDeviceToDevice, s));
  BQC_TRY(eigh(w, ctx, U.as<double>(), n, ev.as<double>(), work, info, s));
  std::vector<double> sv(n);
  BQC_CUDA_TRY(cudaMemcpyAsync(sv.data(), ev.p, (size_t)n * 8, cudaMemcpyDeviceToHost, s));
  BQC_CUDA_TRY(cudaStreamSynchronize(s));
  int k0 = 0;
  while (k0 < n && !(sv[k0] > o.orth_thresh)) ++k0;
  const int nmo = n - k0;
  if (nmo < no) return BQC_E_INVALID;
  k_orth<<<nblk((int64_t)n * nmo), 256, 0, s>>>(n, nmo, k0, U.as<double>(), ev.as<double>(),
                                                X.as<double>());
  BQC_LAUNCH_CHECK();
  const double one = 1.0, zero = 0.0;
  double *Xp = X.as<double>();
  // diagonalise X^T M X -> C (n x nmo, column-major), eps
  auto diag = [&](const double *M) -> int {
    BQC_BLAS_TRY(cublasDgemm(w.blas, CUBLAS_OP_N, CUBLAS_OP_N, n, nmo, n, &one, M, n, Xp, n,
                             &zero, t1.as<double>(), n));
    BQC_BLAS_TRY(cublasDgemm(w.blas, CUBLAS_OP_T, CUBLAS_OP_N, nmo, nmo, n, &one, Xp, n,
                             t1.as<double>(), n, &zero, Fp.as<double>(), nmo));
    BQC_TRY(eigh(w, ctx, Fp.as<double>(), nmo, ev.as<double>(), work, info, s));
    BQC_BLAS_TRY(cublasDgemm(w.blas, CUBLAS_OP_N, CUBLAS_OP_N, n, nmo, nmo, &one, Xp, n,
                             Fp.as<double>(), nmo, &zero, Cc.as<double>(), n));
    return BQC_OK;
  };
  BQC_TRY(diag(H.as<double>()));
  if (o.guess_C) {  // resume: the given occupied orbitals replace the core guess's
    k_rm_to_cm<<<nblk((int64_t)n * no), 256, 0, s>>>(n, no, o.guess_C, Cc.as<double>(), n);
    BQC_LAUNCH_CHECK();
  }
  const int space = std::max(1, o.diis_space);
  std::vector<DBuf> hF(space), hE(space);
  for (int i = 0; i < space; ++i) {
    BQC_TRY(hF[i].alloc(ctx, nn * 8));
    BQC_TRY(hE[i].alloc(ctx, (size_t)nmo * nmo * 8));
  }
  std::vector<int> slot;  // DIIS entries in age order (slot indices)
  std::vector<double> Bm; // Gram matrix of errors in age order
  int stage = o.prec;
  // a solve whose mixed builds join a group (serving) is counted there while
  // it is in the mixed stage, so a batch leader knows whom to wait for
  struct GroupSeat {
    FockGroup *g = nullptr;
    void release() {
      if (g) group_leave(g);
      g = nullptr;
    }
    ~GroupSeat() { release(); }
  } seat;
  if (df->group && stage == BQC_PREC_MIXED_F16X3) {
    seat.g = df->group;
    group_enter(seat.g);
  }
  int mixed_iters = 0, since_best = 0;
  double best = INFINITY;
  double E = 0.0, Eprev = 0.0, emax = INFINITY;
  bool have_prev = false, converged = false;
  int it = 0;
  // anchored incremental FP64 stage (see bqc.h): state
  const bool inc_on = o.incremental != 0 && o.prec != BQC_PREC_FP64;
  const int mixed_prec = o.prec;
  DBuf Facc, Dref, Dk, Vp, Vm, J2, K2, evd, Jx, D2p;
  // rank-2k increments (split-FP16 stored handles): the anchor's occupied
  // orbitals, the Procrustes rotation and its work space
  const bool rank2 = inc_on && mixed_prec == BQC_PREC_MIXED_F16X3 &&
                     df->mode == BQC_DF_STORED && df->B64.p && df->mixed && !df->is_shard();
  DBuf Ca, Sca, Mo, Uo, VTo, So, Ro, Ct;
  if (inc_on) {
    for (DBuf *p : {&Facc, &Dref, &Dk, &J2, &K2, &Jx}) BQC_TRY(p->alloc(ctx, nn * 8));
    BQC_TRY(evd.alloc(ctx, (size_t)n * 8));
    BQC_TRY(D2p.alloc(ctx, (size_t)n * (n + 1) / 2 * 8));
    BQC_TRY(Vp.alloc(ctx, (size_t)n * no * 8));
    BQC_TRY(Vm.alloc(ctx, (size_t)n * no * 8));
  }
  if (rank2) {
    const size_t on = (size_t)n * no * 8, oo = (size_t)no * no * 8;
    for (DBuf *p : {&Ca, &Sca, &Ct}) BQC_TRY(p->alloc(ctx, on));
    for (DBuf *p : {&Mo, &Uo, &VTo, &Ro}) BQC_TRY(p->alloc(ctx, oo));
    BQC_TRY(So.alloc(ctx, (size_t)no * 8));
  }
  bool need_anchor = true;    // the first FP64-stage build is full
  bool last_incremental = false;
  bool confirming = false;     // a full build redoing a converged incremental iteration
  int anchors = 0, inc_since_anchor = 0, inc_stalled = 0;
  double anchor_err = INFINITY, inc_best = INFINITY;
  std::vector<double> hev;
  // The Fock build of an iteration (C -> C_occ row-major, J, K, F) has no
  // host synchronisation in stored mode, so it is captured once per precision
  // stage into a CUDA graph and replayed (thread-local capture mode: other
  // threads, e.g. other serving slots, keep launching meanwhile).
  GraphSet graphs;
  cudaGraphExec_t *gexec = graphs.g;
  // F = Facc + G[D_k - Dref] in the mixed precision, relative to the last
  // anchor (Facc, Dref = its full FP64 Fock matrix and density), so the
  // errors of successive increments do not accumulate (no graph: the
  // eigen-decomposition reads its status on the host).
  auto incremental_build = [&]() -> int {
    BQC_BLAS_TRY(cublasDgemm(w.blas, CUBLAS_OP_N, CUBLAS_OP_T, n, n, no, &one, Cc.as<double>(), n,
                             Cc.as<double>(), n, &zero, Dk.as<double>(), n));
    const double mone = -1.0;
    BQC_BLAS_TRY(cublasDgeam(w.blas, CUBLAS_OP_N, CUBLAS_OP_N, n, n, &one, Dk.as<double>(), n,
                             &mone, Dref.as<double>(), n, t1.as<double>(), n));
    // the Coulomb part of the increment in FP64 straight from dD (stored
    // mode): J is linear in the density, so no factorisation and no
    // cancellation between the two signed parts
    const bool jexact = df->mode == BQC_DF_STORED && df->B64.p;
    if (jexact) {
      if (df->B2f.p)
        BQC_TRY(jff_of_density(df, t1.as<double>(), D2p.as<double>(), Jx.as<double>(), s));
      else
        BQC_TRY(jfp64_of_density(df, t1.as<double>(), D2p.as<double>(), Jx.as<double>(), s));
    }
    if (rank2) {
      // Exchange part as a rank-2k update: rotate the current occupied
      // orbitals Ck onto the anchor's Ca (orthogonal Procrustes in the S
      // metric: M = Ck^T S Ca = U s V^T, R = U V^T, Ct = Ck R, so that
      // Ct Ct^T = D_k), then dD = Cw Cd^T + Cd Cw^T with Cw = (Ca + Ct) / 2
      // and Cd = Ct - Ca small; K[dD] from W = B Cw and DY = B Cd carries
      // rounding relative to |W||DY|, not to |D|.
      BQC_BLAS_TRY(cublasDgemm(w.blas, CUBLAS_OP_N, CUBLAS_OP_N, n, no, n, &one, S.as<double>(),
                               n, Ca.as<double>(), n, &zero, Sca.as<double>(), n));
      BQC_BLAS_TRY(cublasDgemm(w.blas, CUBLAS_OP_T, CUBLAS_OP_N, no, no, n, &one, Cc.as<double>(),
                               n, Sca.as<double>(), n, &zero, Mo.as<double>(), no));
      // R = M (M^T M)^(-1/2), the orthogonal polar factor of M (= U V^T of
      // its SVD), from the eigen-decomposition of M^T M = V diag(lam) V^T
      BQC_BLAS_TRY(cublasDgemm(w.blas, CUBLAS_OP_T, CUBLAS_OP_N, no, no, no, &one, Mo.as<double>(),
                               no, Mo.as<double>(), no, &zero, Uo.as<double>(), no));
      BQC_TRY(eigh(w, ctx, Uo.as<double>(), no, So.as<double>(), work, info, s));
      double lam_min = 0.0;
      BQC_CUDA_TRY(cudaMemcpyAsync(&lam_min, So.p, 8, cudaMemcpyDeviceToHost, s));
      BQC_CUDA_TRY(cudaStreamSynchronize(s));
      // the occupied spaces of C_k and C_a nearly orthogonal in some
      // direction: no small rank-2k difference exists, build in full instead
      if (!(lam_min > 1e-8)) return kIncFull;
      k_scale_cols_rsqrt<<<nblk((int64_t)no * no), 256, 0, s>>>(no, Uo.as<double>(),
                                                                So.as<double>(), VTo.as<double>());
      BQC_LAUNCH_CHECK();
      // Sca (n x no, no longer needed) holds T = V diag(lam^-1/2) V^T
      BQC_BLAS_TRY(cublasDgemm(w.blas, CUBLAS_OP_N, CUBLAS_OP_T, no, no, no, &one, VTo.as<double>(),
                               no, Uo.as<double>(), no, &zero, Sca.as<double>(), no));
      BQC_BLAS_TRY(cublasDgemm(w.blas, CUBLAS_OP_N, CUBLAS_OP_N, no, no, no, &one, Mo.as<double>(),
                               no, Sca.as<double>(), no, &zero, Ro.as<double>(), no));
      BQC_BLAS_TRY(cublasDgemm(w.blas, CUBLAS_OP_N, CUBLAS_OP_N, n, no, no, &one, Cc.as<double>(),
                               n, Ro.as<double>(), no, &zero, Ct.as<double>(), n));
      k_procrustes_pair<<<nblk((int64_t)n * no), 256, 0, s>>>(n, no, Ca.as<double>(),
                                                              Ct.as<double>(), Vp.as<double>(),
                                                              Vm.as<double>());
      BQC_LAUNCH_CHECK();
      BQC_TRY(jk_k_rank2(df, Vp.as<double>(), Vm.as<double>(), K.as<double>(), s));
      BQC_CUDA_TRY(cudaMemsetAsync(K2.p, 0, nn * 8, s));
      BQC_CUDA_TRY(cudaMemcpyAsync(J.p, Jx.p, nn * 8, cudaMemcpyDeviceToDevice, s));
      BQC_CUDA_TRY(cudaMemsetAsync(J2.p, 0, nn * 8, s));
      k_inc_fock<<<nblk(nn), 256, 0, s>>>(nn, Facc.as<double>(), J.as<double>(), J2.as<double>(),
                                          K.as<double>(), K2.as<double>(), F.as<double>());
      BQC_LAUNCH_CHECK();
      return BQC_OK;
    }
    BQC_TRY(eigh(w, ctx, t1.as<double>(), n, evd.as<double>(), work, info, s));
    hev.resize(n);
    BQC_CUDA_TRY(cudaMemcpyAsync(hev.data(), evd.p, (size_t)n * 8, cudaMemcpyDeviceToHost, s));
    BQC_CUDA_TRY(cudaStreamSynchronize(s));
    double amax = 0.0;
    for (double v : hev) amax = std::max(amax, std::fabs(v));
    const double thr = amax * 1e-15;
    int nneg = 0, npos = 0;
    while (nneg < n && hev[nneg] < -thr) ++nneg;
    while (npos < n - nneg && hev[n - 1 - npos] > thr) ++npos;
    nneg = std::min(nneg, no);  // most negative first
    npos = std::min(npos, no);  // the largest positive ones are the last
    const unsigned g = nblk((int64_t)n * no);
    k_eig_factor<<<g, 256, 0, s>>>(n, t1.as<double>(), evd.as<double>(), 0, nneg, no,
                                   Vm.as<double>());
    BQC_LAUNCH_CHECK();
    k_eig_factor<<<g, 256, 0, s>>>(n, t1.as<double>(), evd.as<double>(), n - npos, npos, no,
                                   Vp.as<double>());
    BQC_LAUNCH_CHECK();
    BQC_TRY(bqc_jk(static_cast<bqc_df *>(df), Vp.as<double>(), no, mixed_prec, J.as<double>(),
                   K.as<double>(), (bqc_stream_t)s));
    BQC_TRY(bqc_jk(static_cast<bqc_df *>(df), Vm.as<double>(), no, mixed_prec, J2.as<double>(),
                   K2.as<double>(), (bqc_stream_t)s));
    if (jexact) {  // J[dD] exact: J+ - J- replaced by Jx
      BQC_CUDA_TRY(cudaMemcpyAsync(J.p, Jx.p, nn * 8, cudaMemcpyDeviceToDevice, s));
      BQC_CUDA_TRY(cudaMemsetAsync(J2.p, 0, nn * 8, s));
    }
    k_inc_fock<<<nblk(nn), 256, 0, s>>>(nn, Facc.as<double>(), J.as<double>(), J2.as<double>(),
                                        K.as<double>(), K2.as<double>(), F.as<double>());
    BQC_LAUNCH_CHECK();
    return BQC_OK;
  };
  auto fock_build = [&](int prec) -> int {
    k_cm_to_rm<<<nblk((int64_t)n * no), 256, 0, s>>>(n, no, Cc.as<double>(), n, Crm.as<double>());
    BQC_LAUNCH_CHECK();
    BQC_TRY(bqc_jk(static_cast<bqc_df *>(df), Crm.as<double>(), no, prec, J.as<double>(),
                   K.as<double>(), (bqc_stream_t)s));
    k_axpby3<<<nblk(nn), 256, 0, s>>>(nn, H.as<double>(), 1.0, J.as<double>(), 2.0,
                                      K.as<double>(), -1.0, F.as<double>());
    BQC_LAUNCH_CHECK();
    return BQC_OK;
  };
  const bool use_graph = df->mode == BQC_DF_STORED && !df->timing && s != nullptr;
  auto graph_free = [&]() { graphs.clear(); };
  for (it = 1; it <= o.max_iter; ++it) {
    NvtxRange nv(stage != BQC_PREC_FP64 ? "scf iteration, mixed"
                 : inc_on && !need_anchor ? "scf iteration, incremental"
                                          : "scf iteration, fp64");
    if (cancel_requested()) {  // between iterations: nothing of ours in flight
      BQC_CUDA_TRY(cudaStreamSynchronize(s));
      return BQC_E_CANCELLED;
    }
    const bool inc_stage = inc_on && stage == BQC_PREC_FP64 && anchors < 8;
    last_incremental = inc_stage && !need_anchor;
    if (last_incremental) {
      const int ist = incremental_build();
      if (ist == kIncFull) {
        last_incremental = false;  // this iteration becomes a full build (an anchor)
      } else {
        BQC_TRY(ist);
        ++res->builds_incremental;
        ++inc_since_anchor;
      }
    }
    if (last_incremental) {
    } else if (use_graph && stage >= 0 && stage < 4 && !(df->group && stage != BQC_PREC_FP64)) {
      if (!gexec[stage]) {
        cudaGraph_t graph = nullptr;
        BQC_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        const int st = fock_build(stage);
        const cudaError_t ce = cudaStreamEndCapture(s, &graph);
        if (st != BQC_OK || ce != cudaSuccess) {
          if (graph) cudaGraphDestroy(graph);
          graph_free();
          if (st != BQC_OK) return st;
          BQC_CUDA_TRY(ce);
        }
        const cudaError_t ie = cudaGraphInstantiate(&gexec[stage], graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) {
          graph_free();
          BQC_CUDA_TRY(ie);
        }
      }
      const cudaError_t le = cudaGraphLaunch(gexec[stage], s);
      if (le != cudaSuccess) {
        graph_free();
        BQC_CUDA_TRY(le);
      }
    } else {
      BQC_TRY(fock_build(stage));
    }
    if (!last_incremental) ++(stage == BQC_PREC_FP64 ? res->builds_fp64 : res->builds_mixed);
    BQC_BLAS_TRY(cublasDgemm(w.blas, CUBLAS_OP_N, CUBLAS_OP_T, n, n, no, &one, Cc.as<double>(), n,
                             Cc.as<double>(), n, &zero, D.as<double>(), n));
    if (inc_stage && !last_incremental) {
      // an anchor: the reference of the next increments
      BQC_CUDA_TRY(cudaMemcpyAsync(Facc.p, F.p, nn * 8, cudaMemcpyDeviceToDevice, s));
      BQC_CUDA_TRY(cudaMemcpyAsync(Dref.p, D.p, nn * 8, cudaMemcpyDeviceToDevice, s));
      if (rank2)  // the anchor's occupied orbitals: the first nocc columns of Cc
        BQC_CUDA_TRY(
            cudaMemcpyAsync(Ca.p, Cc.p, (size_t)n * no * 8, cudaMemcpyDeviceToDevice, s));
    }
    k_axpby3<<<nblk(nn), 256, 0, s>>>(nn, H.as<double>(), 1.0, F.as<double>(), 1.0, nullptr, 0.0,
                                      t2.as<double>());
    BQC_LAUNCH_CHECK();
    double eel = 0.0;
    BQC_BLAS_TRY(cublasDdot(w.blas, (int)nn, D.as<double>(), 1, t2.as<double>(), 1, &eel));
    E = eel + b->enuc;
    // e = X^T (F D S - S D F) X
    BQC_BLAS_TRY(cublasDgemm(w.blas, CUBLAS_OP_N, CUBLAS_OP_N, n, n, n, &one, F.as<double>(), n,
                             D.as<double>(), n, &zero, t1.as<double>(), n));
    BQC_BLAS_TRY(cublasDgemm(w.blas, CUBLAS_OP_N, CUBLAS_OP_N, n, n, n, &one, t1.as<double>(), n,
                             S.as<double>(), n, &zero, t2.as<double>(), n));
    k_antisym<<<nblk(nn), 256, 0, s>>>(n, t2.as<double>(), t1.as<double>());
    BQC_LAUNCH_CHECK();
    BQC_BLAS_TRY(cublasDgemm(w.blas, CUBLAS_OP_N, CUBLAS_OP_N, n, nmo, n, &one, t1.as<double>(),
                             n, Xp, n, &zero, t2.as<double>(), n));
    // choose the DIIS slot for this iteration's error
    int sl;
    if ((int)slot.size() < space) {
      std::vector<bool> used(space, false);
      for (int q : slot) used[q] = true;
      sl = 0;
      while (used[sl]) ++sl;
    } else {
      sl = slot.front();
    }
    double *err = hE[sl].as<double>();
    BQC_BLAS_TRY(cublasDgemm(w.blas, CUBLAS_OP_T, CUBLAS_OP_N, nmo, nmo, n, &one, Xp, n,
                             t2.as<double>(), n, &zero, err, nmo));
    int imax = 1;
    BQC_BLAS_TRY(cublasIdamax(w.blas, nmo * nmo, err, 1, &imax));
    double hv = 0.0;
    BQC_CUDA_TRY(cudaMemcpyAsync(&hv, err + (imax - 1), 8, cudaMemcpyDeviceToHost, s));
    BQC_CUDA_TRY(cudaStreamSynchronize(s));
    emax = std::fabs(hv);
    if (res->history && res->history_len < res->history_cap) {
      double *h = res->history + 3 * (size_t)res->history_len++;
      h[0] = last_incremental ? -1.0 : stage;
      h[1] = emax;
      h[2] = E;
    }
    const bool e_stable =
        have_prev && std::fabs(E - Eprev) < std::max(o.energy_tol, DBL_EPSILON * n * std::fabs(E));
    if (stage == BQC_PREC_FP64 && emax < o.diis_tol &&
        (e_stable || confirming || last_incremental)) {
      if (!last_incremental) {
        converged = true;
        break;
      }
      // converged on an incremental Fock matrix: redo the iteration as a full
      // FP64 build, which must confirm the DIIS error (an incremental energy
      // carries the increment's rounding, so its stability is not required
      // here; the confirming build's own DIIS error decides)
      need_anchor = true;
      confirming = true;
      --it;
      continue;
    }
    confirming = false;
    if (inc_stage) {
      if (!last_incremental) {
        ++anchors;
        anchor_err = emax;
        inc_since_anchor = 0;
        inc_stalled = 0;
        inc_best = emax;
        need_anchor = false;
      } else if (rank2) {
        // rank-2k increments carry errors of order |C - C_a| times the mixed
        // rounding, far below the DIIS tolerance, so one anchor serves the
        // whole stage; re-anchor only when the DIIS error stops falling
        // (four increments without a 30 % gain) or after 30 increments
        if (emax < 0.7 * inc_best) {
          inc_best = emax;
          inc_stalled = 0;
        } else {
          ++inc_stalled;
        }
        if (inc_stalled >= 4 || inc_since_anchor >= 30) need_anchor = true;
      } else if ((emax < 100.0 * o.diis_tol && anchor_err >= 100.0 * o.diis_tol) ||
                 inc_since_anchor >= 10) {
        need_anchor = true;  // the next build is full
      }
    }
    if (stage != BQC_PREC_FP64) {
      // Switch to FP64 at stage_tol, or once the mixed stage has reached its
      // floor: the DIIS error of a mixed Fock matrix cannot fall below about
      // max|dF| / sqrt(s_min) (s_min the smallest kept overlap eigenvalue;
      // the orthogonalisation amplifies dF by that much), which in diffuse
      // bases lies well above stage_tol.  The floor shows as a best error that
      // stops halving.  Early iterations from the core guess oscillate at
      // large errors, so stagnation counts only below 1e-2, with a hard
      // bound of 8 iterations without progress and max_iter / 2 in total.
      ++mixed_iters;
      if (emax < best * 0.5) {
        best = emax;
        since_best = 0;
      } else {
        ++since_best;
      }
      const bool at_floor = (since_best >= 3 && best < 1e-2) || since_best >= 8 ||
                            mixed_iters >= std::max(2, o.max_iter / 2);
      if (emax < o.stage_tol || at_floor) {
        // switch to FP64: discard the mixed history, redo this iteration in FP64
        res->switch_rule = emax < o.stage_tol ? BQC_SWITCH_STAGE_TOL : BQC_SWITCH_FLOOR;
        res->switch_err = emax;
        stage = BQC_PREC_FP64;
        seat.release();
        slot.clear();
        Bm.clear();
        have_prev = false;
        --it;
        continue;
      }
    }
    Eprev = E;
    have_prev = true;
    // DIIS bookkeeping
    if ((int)slot.size() == space) {
      // drop the oldest entry (row/col 0 of Bm)
      const int m = (int)slot.size();
      std::vector<double> nb((size_t)(m - 1) * (m - 1));
      for (int i = 1; i < m; ++i)
        for (int j = 1; j < m; ++j) nb[(size_t)(i - 1) * (m - 1) + j - 1] = Bm[(size_t)i * m + j];
      Bm.swap(nb);
      slot.erase(slot.begin());
    }
    BQC_CUDA_TRY(cudaMemcpyAsync(hF[sl].p, F.p, nn * 8, cudaMemcpyDeviceToDevice, s));
    {
      const int m = (int)slot.size();
      std::vector<double> nb((size_t)(m + 1) * (m + 1));
      for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) nb[(size_t)i * (m + 1) + j] = Bm[(size_t)i * m + j];
      for (int i = 0; i <= m; ++i) {
        const int si = (i < m) ? slot[i] : sl;
        double d = 0.0;
        BQC_BLAS_TRY(cublasDdot(w.blas, nmo * nmo, hE[si].as<double>(), 1, err, 1, &d));
        nb[(size_t)i * (m + 1) + m] = d;
        nb[(size_t)m * (m + 1) + i] = d;
      }
      Bm.swap(nb);
      slot.push_back(sl);
    }
    const double *Fuse = F.as<double>();
    const int m = (int)slot.size();
    if (m >= 2) {
      std::vector<double> c;
      if (diis_solve(Bm, m, c)) {
        BQC_CUDA_TRY(cudaMemsetAsync(Fx.p, 0, nn * 8, s));
        for (int i = 0; i < m; ++i)
          BQC_BLAS_TRY(cublasDaxpy(w.blas, (int)nn, &c[i], hF[slot[i]].as<double>(), 1,
                                   Fx.as<double>(), 1));
        Fuse = Fx.as<double>();
      }
    }
    BQC_TRY(diag(Fuse));
  }
  graph_free();
  if (it > o.max_iter) it = o.max_iter;
  // results (library-owned buffers, row-major C)
  res->energy = E;
  res->e_nuc = b->enuc;
  res->diis_err = emax;
  res->iterations = it;
  res->converged = converged ? 1 : 0;
  res->iterations_mixed = mixed_iters;
  res->nmo = nmo;
  if (res->C_dev) {
    k_cm_to_rm<<<nblk((int64_t)n * nmo), 256, 0, s>>>(n, nmo, Cc.as<double>(), n, res->C_dev);
    BQC_LAUNCH_CHECK();
  }
  if (res->eps_dev)
    BQC_CUDA_TRY(
        cudaMemcpyAsync(res->eps_dev, ev.p, (size_t)nmo * 8, cudaMemcpyDeviceToDevice, s));
  if (res->F_dev)
    BQC_CUDA_TRY(cudaMemcpyAsync(res->F_dev, F.p, nn * 8, cudaMemcpyDeviceToDevice, s));
  BQC_CUDA_TRY(cudaStreamSynchronize(s));
  BQC_TRY(ctx->check_flag(s));
  return converged ? BQC_OK : BQC_E_NOT_CONVERGED;
}

}  // namespace bqc

using namespace bqc;

extern "C" {

int bqc_scf_run(bqc_ctx *ctx, bqc_df *df, const bqc_scf_opts *opts, bqc_stream_t stream,
                bqc_scf_result *out) {
  if (!ctx || !df || !out) return BQC_E_INVALID;
  if (df->is_shard()) {
    set_error("bqc_scf_run needs the whole three-index tensor, not an aux shard", __FILE__,
              __LINE__);
    return BQC_E_INVALID;
  }
  BQC_CUDA_TRY(cudaSetDevice(ctx->device));
  bqc_scf_opts o;
  o.diis_tol = 1e-8;
  o.energy_tol = 1e-10;
  o.stage_tol = 1e-5;
  o.max_iter = 100;
  o.diis_space = 8;
  o.prec = BQC_PREC_FP64;
  o.orth_thresh = 1e-8;
  if (opts) {
    o = *opts;
    if (o.diis_tol <= 0) o.diis_tol = 1e-8;
    if (o.energy_tol <= 0) o.energy_tol = 1e-10;
    if (o.stage_tol <= 0) o.stage_tol = 1e-5;
    if (o.max_iter <= 0) o.max_iter = 100;
    if (o.diis_space <= 0) o.diis_space = 8;
    if (o.orth_thresh <= 0) o.orth_thresh = 1e-8;
  }
  double *C = out->C_dev, *eps = out->eps_dev, *F = out->F_dev, *hist = out->history;
  const int cap = out->history_cap;
  *out = bqc_scf_result{};
  out->C_dev = C;
  out->eps_dev = eps;
  out->F_dev = F;
  out->history = hist;
  out->history_cap = hist ? std::max(cap, 0) : 0;
  return scf_run(ctx, df, o, (cudaStream_t)stream, out);
}

}  // extern "C"
