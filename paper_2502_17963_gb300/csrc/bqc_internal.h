// Internal declarations of the bqc library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "bqc.h"

namespace bqc {

// NVTX range over a host scope (a profiler attached by nsys or ncu's NVTX
// filter shows it; without one it costs two calls into a stub).
struct NvtxRange {
  explicit NvtxRange(const char *name);
  ~NvtxRange();
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

// Cancellation flag of the request the calling thread is solving (serving),
// read by the SCF between iterations; null outside the server.
extern thread_local const std::atomic<int> *tl_cancel;
inline bool cancel_requested() {
  return tl_cancel && tl_cancel->load(std::memory_order_relaxed) != 0;
}

// ------------------------------------------------------------ errors ----

void set_error(const char *what, const char *file, int line);
const char *last_error();

#define BQC_CUDA_TRY(expr)                                                   \
  do {                                                                       \
    cudaError_t e__ = (expr);                                                \
    if (e__ != cudaSuccess) {                                                \
      ::bqc::set_error(cudaGetErrorString(e__), __FILE__, __LINE__);         \
      return BQC_E_CUDA;                                                     \
    }                                                                        \
  } while (0)

#define BQC_TRY(expr)                                                        \
  do {                                                                       \
    int s__ = (expr);                                                        \
    if (s__ != BQC_OK) return s__;                                           \
  } while (0)

// Multiprocessor count of the current device (cached per device); grids of
// persistent kernels and the memory plans that depend on them use it.
int sm_count();

// Launch check: reports launch-configuration errors without synchronising.
#define BQC_LAUNCH_CHECK() BQC_CUDA_TRY(cudaPeekAtLastError())

constexpr int kMaxLOrb = 2;   // orbital shells up to d
constexpr int kMaxLAux = 3;   // auxiliary shells up to f
constexpr int kMaxPrim = 32;  // primitives per shell

// Boys table: F_m(k h) for k = 0..kBoysNT-1, m = 0..kBoysNM-1, Taylor order 8.
constexpr int kBoysTaylor = 8;
constexpr double kBoysH = 1.0 / 16.0;
constexpr double kBoysTCut = 36.0;
constexpr int kBoysNT = 577;                   // 36 / h + 1
constexpr int kBoysMaxM = 16;                  // largest m served
constexpr int kBoysNM = kBoysMaxM + kBoysTaylor;

// --------------------------------------------------------- context -----

struct Ctx {
  int device = 0;
  size_t budget = 0;
  bqc_alloc_fn alloc = nullptr;
  bqc_free_fn dealloc = nullptr;
  void *user = nullptr;
  double *boys = nullptr;  // device table [kBoysNT][kBoysNM]
  int *flag = nullptr;     // device error word (0 = fine)
  std::mutex mu;
  std::atomic<size_t> bytes_live{0};
  std::unordered_map<void *, size_t> sizes;  // live allocations (guarded by mu)

  void *dmalloc(size_t bytes);
  void dfree(void *p, size_t bytes_hint = 0);
  int check_flag(cudaStream_t s);  // reads and clears the device flag
};

// Device buffer owned by a context.
struct DBuf {
  Ctx *ctx = nullptr;
  void *p = nullptr;
  size_t n = 0;
  DBuf() = default;
  DBuf(const DBuf &) = delete;
  DBuf &operator=(const DBuf &) = delete;
  ~DBuf() { release(); }
  int alloc(Ctx *c, size_t bytes);
  void release();
  template <class T> T *as() const { return static_cast<T *>(p); }
};

// ---------------------------------------------------------- basis ------

// Structure-of-arrays shell set on the device.
struct ShellSetDev {
  int n = 0;
  const int *l = nullptr;
  const int *nprim = nullptr;
  const int *poff = nullptr;   // first primitive
  const int *fn = nullptr;     // first function
  const double *xyz = nullptr; // n x 3
  const double *exps = nullptr;
  const double *coefs = nullptr; // includes radial norms and contraction renorm
};

struct ShellSetHost {
  std::vector<int> l, nprim, poff, fn, atom;
  std::vector<double> xyz, exps, coefs;
  int nfn = 0;
  DBuf d_int, d_dbl;  // packed device copies
  ShellSetDev dev;
  int upload(Ctx *ctx);
};

// Orbital shell-pair classes (la >= lb): 00, 10, 11, 20, 21, 22.
constexpr int kNPairClass = 6;
inline int pair_class(int la, int lb) { return la * (la + 1) / 2 + lb; }

struct Basis {
  Ctx *ctx = nullptr;
  int natom = 0;
  std::vector<int> Z;
  std::vector<double> xyz;
  ShellSetHost orb, aux;
  int nbf = 0, naux = 0, nocc = 0;
  double enuc = 0.0;
  int64_t npair_sh = 0;
  // oriented orbital shell pairs (a, b), l(a) >= l(b), grouped by class
  int pair_off[kNPairClass + 1] = {0};
  DBuf d_pairs;  // int2 per pair
  // aux shells grouped by l
  int auxl_off[kMaxLAux + 2] = {0};
  DBuf d_aux_by_l;
  DBuf d_atoms;  // natom x (x, y, z, Z) doubles
};

// ---------------------------------------------------- integral API -----

// Device Boys table construction (host series, upload).
int boys_table_build(Ctx *ctx);
int launch_boys_eval(Ctx *ctx, int n, const double *T, int mmax, double *out, cudaStream_t s);

int launch_one_electron(const Basis *b, double *S, double *T, double *V, cudaStream_t s);
int launch_int2c(const Basis *b, double *V, cudaStream_t s);
// Schwarz factors of oriented pairs: Q[k] = sqrt(max_ij (a_i b_j|a_i b_j)).
int launch_schwarz_pairs(const Basis *b, double *Qpair, cudaStream_t s);

// Screened work lists of the three-centre kernel (Sec. 2.2 prescreening).
// Pairs of each class are sorted by decreasing Schwarz factor; for each aux
// shell P the survivors are a prefix of that list, counted in `cut` and
// scanned into `prefix` so that surviving triplets map densely to threads.
struct Eri3cPlan {
  Ctx *ctx = nullptr;
  double tau = 0.0;
  DBuf d_pairs_sorted;  // int2 per pair, sorted within class
  DBuf d_qpair_sorted;  // double per pair
  DBuf d_qaux;          // double per aux shell
  DBuf d_qpair;         // double per pair, in the basis' (unsorted) pair order
  DBuf d_prefix;        // per (pair class, aux l): n_aux(l)+1 int64 prefix
  int64_t prefix_off[kNPairClass][kMaxLAux + 1] = {{0}};
  int64_t total[kNPairClass][kMaxLAux + 1] = {{0}};
  int64_t survivors = 0, candidates = 0;
  std::vector<int64_t> h_prefix;  // host copy of d_prefix
};
// Builds the plan on `s` (one stream sync at the end to read the counts).
int eri3c_plan(const Basis *b, double tau, const double *V_diag_dev, cudaStream_t s,
               Eri3cPlan *plan);
// (P|mu nu) for aux functions [p0, p1) into out[(P - p0) * ld + col(mu,nu)],
// packed lower triangle; screened-out entries are left untouched.
int launch_eri3c(const Basis *b, const Eri3cPlan *plan, int p0, int p1, double *out,
                 int64_t ld, cudaStream_t s);
// The same with a choice of survivor compaction (0: sorted prefix, the
// default; 1: per-warp loop buffer; 2: two-kernel global index list).
int launch_eri3c_variant(const Basis *b, const Eri3cPlan *plan, int p0, int p1, double *out,
                         int64_t ld, int variant, cudaStream_t s);

// --------------------------------------------------------- linalg ------

// C = beta C + alpha op(A) op(B), FP64, row-major with leading dimensions.
int dgemm(bool transA, bool transB, int M, int N, int K, double alpha, const double *A,
          int64_t lda, const double *B, int64_t ldb, double beta, double *C, int64_t ldc,
          cudaStream_t s);
// In-place lower Cholesky of an n x n SPD matrix (upper part zeroed).
int cholesky_lower(Ctx *ctx, double *A, int n, cudaStream_t s);
// In-place X := L^{-1} X for L n x n lower, X n x ncol with leading dim ld.
int trsm_lower_left(Ctx *ctx, const double *L, int n, double *X, int64_t ncol, int64_t ld,
                    cudaStream_t s);

}  // namespace bqc

// Opaque handle types of the C ABI.
struct bqc_ctx : bqc::Ctx {};
struct bqc_basis : bqc::Basis {};
