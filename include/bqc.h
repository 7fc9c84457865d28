/*
 * bqc.h - C ABI of the GB300 density-fitted RHF Fock-build library.
 *
 * The method is the mean-field stage of arXiv 2502.17963 (ByteQC), Sec. 2.2:
 * three-index Cholesky-decomposed ERIs built from an auxiliary basis, stored
 * once when they fit (they depend only on the basis and the geometry, not on
 * the SCF iterate), regenerated in slices of the auxiliary basis when they do
 * not, and contracted into the Coulomb and exchange matrices inside the SCF.
 * The paper prints no equations for this path; the operations below are the
 * textbook ones (Szabo & Ostlund Ch. 3; Helgaker, Jorgensen & Olsen Ch. 9).
 *
 * Notation.  N orbital and Naux auxiliary Cartesian Gaussian functions,
 * nocc doubly occupied orbitals, Npair = N(N+1)/2.  D = C_occ C_occ^T (no
 * factor 2).  V_PQ = (P|Q) = L L^T (L lower, positive diagonal).
 * B_P,mu nu = sum_Q (L^{-1})_PQ (Q|mu nu).  J = sum_P B_P (B_P : D),
 * K = sum_P B_P D B_P, F = H + 2J - K, E = sum D (H + F) + E_nn.
 *
 * Conventions for every call.
 *  - Return value: BQC_OK (0) or a negative status; bqc_strerror() names it.
 *    No call aborts, throws or traps; a device-side check that trips is
 *    reported as BQC_E_DEVICE_FLAG by the next call that reads the flag.
 *  - Pointers named *_dev are device pointers on the context's device; all
 *    other pointers are host memory.  Matrices are row-major, FP64 unless a
 *    name says otherwise.
 *  - Ownership: the caller owns every array it passes; the library copies
 *    what it keeps.  Handles are owned by the library until their _destroy.
 *  - Streams: a cudaStream_t argument may be NULL (the legacy default
 *    stream).  Calls marked "async" enqueue work and return without waiting.
 *  - Units: bohr and hartree.  Cartesian components of a shell of angular
 *    momentum l are ordered lexicographically (xx, xy, xz, yy, yz, zz ...);
 *    every Cartesian primitive component is unit-normalised and each
 *    contracted shell is rescaled to unit self-overlap.
 */
#ifndef BQC_H
#define BQC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *bqc_stream_t; /* = cudaStream_t */

enum {
  BQC_OK = 0,
  BQC_E_INVALID = -1,       /* bad argument or size                         */
  BQC_E_OOM = -2,           /* allocation failed                            */
  BQC_E_ADMISSION = -3,     /* request exceeds the HBM budget               */
  BQC_E_NOT_CONVERGED = -4, /* SCF hit max_iter                             */
  BQC_E_CUDA = -5,          /* a CUDA runtime / library call failed         */
  BQC_E_TIMEOUT = -6,       /* a bounded device or host wait ran out        */
  BQC_E_DEVICE_FLAG = -7,   /* a kernel's own bounds check tripped          */
  BQC_E_NOT_READY = -8,     /* serving: result not available yet            */
  BQC_E_UNSUPPORTED = -9,   /* angular momentum / size the library lacks    */
  BQC_E_CANCELLED = -10     /* serving: the request was cancelled           */
};

/* Precision of the Fock build (the X = B C and K contractions, the B.D
 * products).  FP64: all FP64 (DFMA).  MIXED_TF32: tcgen05 kind::tf32 MMAs on
 * TF32-rounded B and C_occ (one product per term, ~2^-11 relative per
 * product), FP32 accumulation in short chains, FP64 chunk sums; J from the
 * TF32 shadow of B.  MIXED_TF32X3: K the same with every operand split
 * hi + lo into two TF32 parts and three products per term (hi*hi + hi*lo +
 * lo*hi, ~2^-22); J in FP64 from the FP64 B on the CUDA cores, concurrently
 * with the tensor-core passes (the direct mode's J is FP64 in every
 * precision).  MIXED_F16X3: as MIXED_TF32X3 with FP16 split parts (FP16 has
 * TF32's 11-bit significand; B, C_occ and X are scaled by powers of two to a
 * largest magnitude of 2^14 before the split, so the narrow FP16 exponent
 * range costs nothing above ~2^-40 of the largest element) and kind::f16
 * MMAs, which run at twice the TF32 rate; stored mode only. */
typedef enum {
  BQC_PREC_FP64 = 0,
  BQC_PREC_MIXED_TF32 = 1,
  BQC_PREC_MIXED_TF32X3 = 2,
  BQC_PREC_MIXED_F16X3 = 3
} bqc_prec;

typedef struct bqc_ctx bqc_ctx;
typedef struct bqc_basis bqc_basis;
typedef struct bqc_df bqc_df;
typedef struct bqc_server bqc_server;

/* Device-memory callbacks.  alloc returns a device pointer (or NULL) of at
 * least `bytes` bytes on the context's device; free releases it.  Both may be
 * NULL, in which case cudaMalloc / cudaFree are used. */
typedef void *(*bqc_alloc_fn)(size_t bytes, void *user);
typedef void (*bqc_free_fn)(void *ptr, void *user);

/* Create a context on `device`.  hbm_budget (bytes) caps what the serving
 * loop admits (0 = no cap).  Builds the Boys-function table on the device. */
int bqc_ctx_create(int device, size_t hbm_budget, bqc_alloc_fn alloc, bqc_free_fn dealloc,
                   void *alloc_user, bqc_ctx **out);
int bqc_ctx_destroy(bqc_ctx *ctx);

/* One contracted Cartesian shell.  exps/coefs: nprim entries each; coefs
 * multiply unit-normalised primitives. */
typedef struct {
  int atom;
  int l;
  int nprim;
  const double *exps;
  const double *coefs;
} bqc_shell;

/* Load a molecule and its orbital and auxiliary bases (Sec. 2.2: DF expands
 * orbital products in an auxiliary basis on the same atoms).  Z: natom
 * nuclear charges; xyz_bohr: natom x 3.  Orbital l <= 2 and auxiliary
 * l <= 3 (compiled limits; up to the
 * (f|dd) class), else BQC_E_UNSUPPORTED; sum Z must be even (closed shell),
 * else BQC_E_INVALID.  Copies everything; the shell setup (normalisation,
 * pair classes) runs here. */
int bqc_basis_load(bqc_ctx *ctx, int natom, const int *Z, const double *xyz_bohr,
                   const bqc_shell *orb, int norb_shell, const bqc_shell *aux, int naux_shell,
                   bqc_basis **out);
int bqc_basis_destroy(bqc_basis *basis);
/* Sizes: N, Naux, nocc, number of orbital shell pairs (a >= b). */
int bqc_basis_info(const bqc_basis *basis, int *nbf, int *naux, int *nocc, int64_t *nshell_pair);
/* Nuclear repulsion energy sum_{A<B} Z_A Z_B / R_AB. */
int bqc_basis_enuc(const bqc_basis *basis, double *enuc);

/* One-electron matrices (overlap S, kinetic T, nuclear attraction Vne),
 * N x N into device buffers; any pointer may be NULL to skip it.  Async. */
int bqc_one_electron(const bqc_basis *basis, double *S_dev, double *T_dev, double *Vne_dev,
                     bqc_stream_t stream);

/* Boys function F_m(T) = int_0^1 t^(2m) exp(-T t^2) dt, m = 0..mmax (<= 16)
 * for n arguments: out_dev is n x (mmax+1).  The device evaluator used by the
 * integral kernels (Taylor table + recursions), exposed for testing.  Async. */
int bqc_boys(bqc_ctx *ctx, int n, const double *T_dev, int mmax, double *out_dev,
             bqc_stream_t stream);

/* Coulomb metric V_PQ = (P|Q), Naux x Naux, FP64.  Async. */
int bqc_int2c(const bqc_basis *basis, double *V_dev, bqc_stream_t stream);

/* Raw three-centre integrals (P|mu nu) over all aux functions and the packed
 * lower triangle mu >= nu: out_dev is Naux x Npair, column mu(mu+1)/2 + nu.
 * Integrals whose Schwarz bound sqrt((P|P)) sqrt((mu nu|mu nu)) is below
 * `schwarz` are written as 0 (schwarz <= 0 computes everything).  Async. */
int bqc_int3c(const bqc_basis *basis, double schwarz, double *out_dev, bqc_stream_t stream);

/* ---------------------------------------------------------- DF tensor --- */

/* NONE: no density fitting; bqc_jk builds J and K directly from Schwarz-
 * screened four-centre integrals (mu nu|lambda sigma), the conventional
 * on-the-fly mean field the paper uses for molecules (Sec. 2.2.2), FP64 only;
 * the auxiliary basis is ignored. */
typedef enum { BQC_DF_STORED = 0, BQC_DF_DIRECT = 1, BQC_DF_AUTO = 2, BQC_DF_NONE = 3 } bqc_df_mode;

/* Split shadows of B kept for the mixed precisions: NONE (FP64 builds only),
 * TF32 (full-square hi/lo TF32 parts: MIXED_TF32 and MIXED_TF32X3; 8 bytes
 * per element of the square), F16 (scaled hi/lo FP16 parts: MIXED_F16X3;
 * 4 bytes per element).  Direct mode uses TF32 for either non-NONE value. */
enum { BQC_SHADOW_NONE = 0, BQC_SHADOW_TF32 = 1, BQC_SHADOW_F16 = 2 };

typedef struct {
  int mode;            /* bqc_df_mode                                         */
  double schwarz;      /* screening threshold; default 1e-12 stored, 1e-10 direct */
  int aux_block;       /* direct mode: aux functions per block (default 1024)  */
  int keep_fp32;       /* split shadows of B for the mixed precisions: one of
                          BQC_SHADOW_NONE / _TF32 / _F16 (default TF32)       */
  size_t hbm_limit;    /* AUTO: choose DIRECT when STORED needs more (0 = free memory) */
  int aux_begin;       /* stored mode: keep only the rows P in [aux_begin, aux_end) */
  int aux_end;         /* of B (an aux shard); 0, 0 = every aux function         */
} bqc_df_opts;

/* Build the DF machinery (Sec. 2.2).  STORED: metric, Cholesky, raw (Q|mu nu),
 * in-place B = L^{-1}(Q|mu nu) in FP64 (packed), plus the TF32 full-square
 * shadow when keep_fp32.  DIRECT: metric, Cholesky and screening data only;
 * (Q|mu nu) is regenerated in aux blocks at each bqc_jk (Sec. 2.2: computed
 * again slice by slice when too large to keep); with keep_fp32 its tensor-core
 * sub-blocks are
 * sized from the device memory free at build time (memory held by a caching
 * allocator counts as used).  Work on `stream`; returns after the build has
 * been enqueued and its workspaces allocated (synchronises the stream once to
 * size the screened work lists).  opts may be NULL for defaults. */
int bqc_df_build(bqc_ctx *ctx, const bqc_basis *basis, const bqc_df_opts *opts,
                 bqc_stream_t stream, bqc_df **out);
int bqc_df_destroy(bqc_df *df);
/* Mode actually built and bytes of device memory held. */
int bqc_df_info(const bqc_df *df, int *mode, size_t *device_bytes);
/* Aux shards (the per-GPU partition of the CD-ERIs, Sec. 2.2.2 and the
 * multi-GPU scaling of Sec. 3.2, applied to the aux index).  J and K are
 * sums over P of per-P terms, so a handle built with
 * opts.aux_begin/aux_end = [P0, P1) holds only the rows P0 <= P < P1 of B,
 * and bqc_jk on it returns the partial J and K of those rows; the partials
 * of shards that cover [0, Naux) once add up to the full J and K (one
 * all-reduce per Fock build across the processes that hold them).  The rows
 * of B = L^-1 (Q|mu nu) up to P1 need the integrals of every Q < P1, so the
 * build solves rows [0, P1) and keeps its own (the one-GPU construction; a
 * multi-GPU build would solve pair-column slices and exchange them once).
 * bqc_scf_run and bqc_mp2 need the whole tensor and refuse a shard
 * (BQC_E_INVALID); direct mode has no shards (BQC_E_UNSUPPORTED).  This
 * call returns the handle's range ([0, Naux) for a whole tensor). */
int bqc_df_shard(const bqc_df *df, int *aux_begin, int *aux_end);
/* Schwarz screening of the 3-centre integrals (Sec. 2.2): shell triplets
 * (aux shell, orbital shell pair) considered and kept (Q_P Q_mu nu >= tau). */
int bqc_df_screening(const bqc_df *df, int64_t *candidates, int64_t *survivors);
/* Survivor compaction of the screened three-centre integrals, as a
 * measured choice (the paper's GPU prescreening, Sec. 2.2.1 and Algorithm 1,
 * against the alternatives it discusses).  Writes (P|mu nu) for the aux
 * functions [p0, p1) into out_dev ((p1 - p0) x Npair, packed as bqc_int3c),
 * with the handle's Schwarz screening; screened entries are left untouched
 * (zero the buffer first).  variant 0: the library's compaction (pairs
 * sorted by Schwarz factor, survivors a prefix per aux shell, dense
 * triplet index, no divergence); 1: the paper's per-warp loop buffer
 * (screen 32 candidates per warp, append survivors to a 64-entry ring in
 * shared memory, compute a warp's worth at a time); 2: a screening kernel
 * that appends survivors to a global index list, then a kernel over the
 * list.  All three compute the same triplets with the same arithmetic, so
 * their outputs are identical.  Async except variant 2, which allocates the
 * list from the context and synchronises the stream before releasing it. */
int bqc_int3c_screened(const bqc_df *df, int p0, int p1, int variant, double *out_dev,
                       bqc_stream_t stream);

/* Copy B (Naux x Npair packed, FP64, stored mode) into a device buffer; or
 * the Cholesky factor L (Naux x Naux, lower, zeros above) when which = 1.  Async. */
int bqc_df_copy(const bqc_df *df, int which, double *out_dev, bqc_stream_t stream);

/* J and K for the occupied orbitals C_occ (N x nocc, row-major, device):
 * J_mu nu = sum_P B_P,mu nu w_P with w_P = sum_lambda sigma B_P,lambda sigma D_lambda sigma,
 * K_mu nu = sum_{P,i} X_P,mu i X_P,nu i with X_P = B_P C_occ (Sec. 2.2: the
 * Coulomb matrix needs two passes over the CD-ERIs; exchange re-reads them).
 * J_dev, K_dev: N x N, FP64, full symmetric.  nocc must equal the basis'
 * nocc.  Async; no host synchronisation and no allocation inside, so the
 * call can be captured into a CUDA graph (stored mode). */
int bqc_jk(bqc_df *df, const double *C_occ_dev, int nocc, int prec, double *J_dev,
           double *K_dev, bqc_stream_t stream);

/* Allocation-free FP64 Fock build (no counterpart in the paper; it exists
 * for callers that cannot allocate device memory at call time, e.g. a host
 * framework that has already reserved the GPU's memory in its own pool, or a
 * latency-critical loop that cannot afford the device-wide synchronisation
 * that cudaMalloc / cudaFree may cause).
 * Computes the same J and K as bqc_jk with BQC_PREC_FP64 from caller-owned
 * device buffers: B_dev is the packed FP64 B (Naux x Npair, as bqc_df_copy
 * returns it), C_occ_dev N x nocc, J_dev and K_dev N x N.  Its working memory
 * (Naux*N*nocc + Naux + Npair doubles, each part rounded up to 256 bytes) comes
 * from a fixed array of BQC_NOALLOC_SCRATCH_BYTES inside the library, which
 * every GPU that loads the library holds until the process exits; larger
 * sizes return BQC_E_INVALID (bqc_last_error names the size) before any work.
 * The first call on a device looks up that array's device address (one-time
 * set-up, with the device current); make that first call before any stream
 * capture.  The address is kept for the life of the process: after a
 * cudaDeviceReset() of a device it is stale, so do not call this entry
 * point on that device again in the same process.  The limit admits the
 * single water up to (H2O)_7 of the cluster workloads.  All calls on a device share the array: calls whose work overlaps
 * on the GPU (different streams, or host threads without ordering) race and
 * must be serialised by the caller.  Async. */
#define BQC_NOALLOC_SCRATCH_BYTES (32u << 20)
int bqc_jk_fp64_noalloc(const double *B_dev, int naux, int nbf, const double *C_occ_dev,
                        int nocc, double *J_dev, double *K_dev, bqc_stream_t stream);

/* Same as bqc_jk with host buffers: copies C_occ in, J and K out, and
 * waits for the stream.  The end-to-end entry point.  A non-finite entry of
 * C_occ returns BQC_E_INVALID before anything is copied or launched. */
int bqc_jk_host(bqc_df *df, const double *C_occ, int nocc, int prec, double *J, double *K,
                bqc_stream_t stream);

/* The Coulomb matrix of any symmetric density from the stored tensor, as the
 * two passes over the CD-ERIs of Sec. 2.2: w_P = sum_{mu nu} B_P,mu nu D_mu nu,
 * then J = sum_P w_P B_P.  D_dev and J_dev are device N x N, row-major (D
 * symmetric; its lower triangle is read).  BQC_COULOMB_FP64 runs both passes
 * with FP64 FMAs over the FP64 B; BQC_COULOMB_FF runs them on the FP32 pipe
 * in float-float arithmetic (~2^-46 relative per term) over the float-pair
 * copy of B that handles built with BQC_SHADOW_F16 hold (else
 * BQC_E_UNSUPPORTED).  Each pass reads the packed B once (8 bytes per packed
 * element); the FP64 pipe of this GPU runs 1/64 of the FP32 rate, so only the
 * float-float passes run at the memory's speed.  Stored mode only; the first
 * call allocates a packed-density scratch.  Async. */
#define BQC_COULOMB_FP64 0
#define BQC_COULOMB_FF 1
int bqc_df_coulomb(bqc_df *df, const double *D_dev, double *J_dev, int variant,
                   bqc_stream_t stream);

/* Grouped split-FP16 Fock builds of n independent molecules (the batching
 * of launch-bound small kernels of Sec. 2.4.2 applied to Sec. 2.2's two
 * passes): J[k], K[k] of dfs[k] with C_dev[k] (device, row-major N_k x
 * nocc_k, as bqc_jk), all at MIXED_F16X3.  Every handle must be stored mode,
 * unsharded and built with BQC_SHADOW_F16 (else BQC_E_UNSUPPORTED), on one
 * device, and appear once.  The X passes of all molecules run as one
 * persistent tensor-core launch, then their FP64 J passes as one launch and
 * their SYRKs as one launch (up to 12 molecules per launch; more are taken
 * twelve at a time), each molecule keeping its own plan, so K[k] equals
 * bqc_jk's K exactly and J[k] its J to the float-float rounding of a
 * different aux chunking (~1e-12 of max|J|).  Uses each handle's own
 * workspace: no handle may have another build in flight.  Async on
 * `stream`. */
int bqc_jk_grouped(int n, bqc_df *const *dfs, const double *const *C_dev, double *const *J,
                   double *const *K, bqc_stream_t stream);

/* Per-phase device timing of bqc_jk (a profiling aid).  enable != 0 makes
 * every following bqc_jk on this handle record CUDA events at its phase
 * boundaries on its stream (leave it off while capturing a graph).
 * bqc_df_phase_ms waits for the last call's events and writes up to n
 * durations in ms.  Stored mode: [0] X pass (X = B C, with the fused w
 * contraction in FP64 and MIXED_TF32), [1] J (mixed builds: on a side stream,
 * overlapping [0] in MIXED_TF32X3 and [2] in MIXED_TF32), [2] K (SYRK and
 * its FP64 reduction), [3] operand preparation.  Direct mode: [0] first integral pass (integrals, gamma, X),
 * [1] metric solve and K, [2] second integral pass (J), [3] preparation.
 * BQC_E_NOT_READY if no timed call has been made. */
int bqc_df_timing(bqc_df *df, int enable);
int bqc_df_phase_ms(bqc_df *df, float *ms, int n);

/* --------------------------------------------------------------- MP2 --- */

/* Closed-shell DF-MP2 correlation energy on the resident three-index tensor
 * (Sec. 2.3: MO-basis tensor B_P,ia = sum C_mu,i B_P,mu nu C_nu,a, integrals
 * (ia|jb) = sum_P B_P,ia B_P,jb formed block by block, the denominator
 * applied in place):
 *   E2 = sum_{i,j,a,b} (ia|jb) [2 (ia|jb) - (ib|ja)] / (e_i + e_j - e_a - e_b).
 * df: a stored-mode handle.  C_dev: N x nmo row-major canonical orbitals
 * (columns; the first nocc occupied, the rest virtual), eps_dev: their nmo
 * orbital energies (bqc_scf_run's C_dev / eps_dev outputs have this layout).
 * prec: BQC_PREC_FP64 (every GEMM on the DFMA path) or BQC_PREC_MIXED_F16X3
 * (the MO transform in FP64, the (ia|jb) blocks as split-FP16 tensor-core
 * GEMMs with FP32 accumulation in short chains and FP64 blocks, ~2^-22
 * relative per integral); other precisions BQC_E_UNSUPPORTED.
 * Writes *e2 (host).  Allocates its working memory from the context
 * (Naux * nocc * nvir doubles and a block of (ia|jb) of at most 1 GiB) and
 * synchronises the stream; reuses the handle's X buffer, so it must not
 * overlap a bqc_jk on the same handle. */
int bqc_mp2(bqc_df *df, const double *C_dev, const double *eps_dev, int nmo, int prec,
            double *e2, bqc_stream_t stream);

/* ---------------------------------------------------------------- SCF --- */

typedef struct {
  double diis_tol;     /* max |X^T (FDS - SDF) X| to converge (default 1e-8)   */
  double energy_tol;   /* |E - E_prev| to converge (default 1e-10); the bar is
                          max(energy_tol, eps_64 * N * |E|), the energy's own
                          rounding noise, which is larger from N ~ 800 */
  double stage_tol;    /* mixed -> FP64 switch when DIIS error below (1e-5)   */
  int max_iter;        /* default 100                                         */
  int diis_space;      /* default 8                                           */
  int prec;            /* bqc_prec of the first stage; FP64 = unstaged        */
  double orth_thresh;  /* canonical orthogonalisation cut on S eigenvalues (1e-8) */
  int incremental;     /* staged SCF only (prec mixed): 0 = every FP64-stage Fock
                          build is a full FP64 build; 1 = anchored incremental
                          FP64 stage (see bqc_scf_run)                         */
  const double *guess_C; /* optional start (resume from a checkpoint): device
                          N x nocc row-major occupied orbitals, e.g. the first
                          nocc columns of an earlier result's C_dev; the first
                          Fock build uses D = C C^T instead of the
                          core-Hamiltonian guess, and the DIIS history starts
                          empty.  NULL: core guess.  Ignored by the server.   */
} bqc_scf_opts;

typedef struct {
  double energy;       /* total energy at convergence (last iteration)        */
  double e_nuc;
  double diis_err;     /* max-abs DIIS error of the last iteration            */
  int iterations;
  int converged;
  int iterations_mixed;/* iterations run in the mixed stage                    */
  int nmo;             /* orbitals kept by canonical orthogonalisation          */
  /* Optional caller-owned device outputs (set before the call, NULL = skip):
   * C_dev N x N buffer receiving C as N x nmo row-major (first N*nmo
   * entries); eps_dev N doubles (first nmo used); F_dev N x N last Fock
   * matrix. */
  double *C_dev;
  double *eps_dev;
  double *F_dev;
  /* Optional caller-owned host output (NULL = skip): 3 * history_cap doubles
   * receiving, per Fock build in order, (bqc_prec of the build, max-abs DIIS
   * error, energy); history_len (output) counts the builds written. */
  double *history;
  int history_cap;
  int history_len;
  /* Precision staging (output): which rule ended the mixed stage
   * (BQC_SWITCH_NONE if the SCF ran in one precision, BQC_SWITCH_STAGE_TOL
   * when the DIIS error fell below stage_tol, BQC_SWITCH_FLOOR when the mixed
   * stage stopped improving above it) and the max-abs DIIS error of the last
   * mixed iteration. */
  int switch_rule;
  double switch_err;
  /* Fock builds of the run by kind (output): full FP64 builds, mixed builds of
   * the first stage, incremental FP64-stage builds (opts.incremental). */
  int builds_fp64;
  int builds_mixed;
  int builds_incremental;
} bqc_scf_result;

enum { BQC_SWITCH_NONE = 0, BQC_SWITCH_STAGE_TOL = 1, BQC_SWITCH_FLOOR = 2 };

/* Closed-shell SCF (canonical orthogonalisation, core-Hamiltonian guess,
 * Pulay DIIS on e = X^T (FDS - SDF) X, aufbau) with the Fock build of
 * bqc_jk.
 * Anchored incremental FP64 stage (opts.incremental = 1 with a mixed first
 * stage; no counterpart in the paper, the incremental Fock build of direct
 * SCF codes): F_k = F_a + 2 J[dD] - K[dD] with F_a the full FP64 Fock matrix
 * of the last anchor build, dD = D_k - D_a factored as V+ V+^T - V- V-^T
 * (eigenvectors of dD scaled by the square roots of its positive and
 * negative eigenvalues, at most nocc of each) and J, K of V+ and V- built in
 * the first stage's mixed precision, so the rounding error of F_k scales
 * with |D_k - D_a|, not with |D|; in stored mode the Coulomb part J[dD] is
 * instead formed in FP64 from dD itself (two streaming passes over the FP64
 * B), which avoids the cancellation between the J of V+ and of V-; and with
 * MIXED_F16X3 on a stored handle K[dD] is a rank-2k update: the occupied
 * orbitals are rotated onto the anchor's (orthogonal Procrustes in the S
 * metric), dD = Cw Cd^T + Cd Cw^T with Cd the small orbital difference, and
 * the error of K[dD] scales with |Cd|.  Anchors (full FP64 builds) are made at
 * the switch, when the DIIS error first falls below 100 x diis_tol, after
 * 10 increments, and on every iteration that would converge: an
 * incremental iteration with max|e| < diis_tol and a stable energy is
 * redone as a full FP64 build, which must confirm max|e| < diis_tol, so the
 * reported energy and DIIS error are always those of a full FP64 Fock
 * matrix.  After 8 anchors the stage falls back to full builds.  History
 * entries of incremental builds carry the precision code -1.  With prec = MIXED_TF32 the first stage runs mixed and switches to
 * FP64 (DIIS subspace cleared) when the DIIS error drops below stage_tol, or
 * earlier once the mixed stage stops improving (its error floor, about
 * max|dF_mixed| / sqrt(smallest kept overlap eigenvalue), can lie above
 * stage_tol in diffuse bases): best error not halved for 3 iterations while
 * below 1e-2, for 8 iterations at any size, or max_iter / 2 mixed iterations.
 * Blocks until done.  Returns BQC_E_NOT_CONVERGED (result still filled) if
 * max_iter is reached.  out's C_dev / eps_dev / F_dev / history /
 * history_cap are read as inputs (caller buffers or NULL); everything else
 * in *out is written. */
int bqc_scf_run(bqc_ctx *ctx, bqc_df *df, const bqc_scf_opts *opts, bqc_stream_t stream,
                bqc_scf_result *out);

/* ------------------------------------------------------------ serving --- */

typedef enum {
  /* Queue order, except that a later request that fits the HBM ledger may be
   * admitted while the queue head does not (the head is passed over at most
   * max_skips times, then waits alone); smaller molecules run on
   * higher-priority streams.  Default. */
  BQC_SERVE_BACKFILL = 0,
  /* Strict arrival order, every stream at the same priority. */
  BQC_SERVE_FIFO = 1
} bqc_serve_policy;

typedef struct {
  int max_slots;       /* concurrent SCF solves on the device (default 4)     */
  size_t hbm_budget;   /* bytes the admitted requests may hold (0 = ctx's)    */
  int prec;            /* bqc_prec of every request (MIXED_F16X3 when the
                          server is created with opts NULL)                    */
  bqc_scf_opts scf;    /* SCF options for every request                       */
  int policy;          /* bqc_serve_policy                                    */
  int max_skips;       /* backfill starvation bound (<= 0: 8)                 */
  /* != 0 (prec MIXED_F16X3 only): the mixed-stage Fock builds of the solves
   * in flight are batched into grouped launches (bqc_jk_grouped); the first
   * solve to hand in a build waits at most group_window_us (<= 0: 1000) for
   * the other solves of the mixed stage before the batch launches. */
  int grouped;
  double group_window_us;
} bqc_serve_opts;

typedef struct {
  int natom;
  const int *Z;
  const double *xyz_bohr;
  const bqc_shell *orb;
  int norb_shell;
  const bqc_shell *aux;
  int naux_shell;
} bqc_request;

typedef struct {
  int status;          /* BQC_OK, BQC_E_NOT_CONVERGED, BQC_E_ADMISSION, ...   */
  double energy;
  double diis_err;
  int iterations;
  int nbf;
  double t_submit;     /* seconds on the server's monotonic clock              */
  double t_admit;
  double t_done;
  int iterations_mixed; /* SCF iterations before the switch to FP64            */
  int priority;         /* CUDA stream priority the solve ran at               */
} bqc_serve_result;

/* Continuous-batching server: a scheduler thread admits queued requests as
 * slots and HBM budget free up; each admitted request runs its DF build and
 * SCF on its own stream, so solves overlap on the device. */
int bqc_serve_create(bqc_ctx *ctx, const bqc_serve_opts *opts, bqc_server **out);
/* Copies the request; returns a ticket.  BQC_E_ADMISSION if the request could
 * never fit the budget. */
int bqc_serve_submit(bqc_server *srv, const bqc_request *req, uint64_t *ticket);
/* BQC_OK with the result once done, BQC_E_NOT_READY before. */
int bqc_serve_poll(bqc_server *srv, uint64_t ticket, bqc_serve_result *res);
/* Cancels a request.  A queued one completes at once with status
 * BQC_E_CANCELLED; a running one stops at its next step boundary (before the
 * DF build, before the SCF, or between SCF iterations, never with work of
 * its own in flight) and completes with BQC_E_CANCELLED, its memory
 * returned to the ledger; one already done is left as it is.  BQC_OK, or
 * BQC_E_INVALID for an unknown ticket. */
int bqc_serve_cancel(bqc_server *srv, uint64_t ticket);
/* Wait (at most timeout_s seconds, <= 0 = no limit) until all submitted
 * requests are done; BQC_E_TIMEOUT otherwise. */
int bqc_serve_drain(bqc_server *srv, double timeout_s);
int bqc_serve_destroy(bqc_server *srv);
/* Grouped-build counters of a server created with grouped != 0: batches
 * launched, builds they held, and the largest batch (all 0 otherwise). */
int bqc_serve_group_stats(bqc_server *srv, uint64_t *batches, uint64_t *builds, int *max_batch);
/* Predicted device bytes of a request of this size solved with `prec` (the
 * admission ledger); 0 for an invalid argument. */
size_t bqc_serve_footprint(int nbf, int naux, int nocc, int prec);

/* Failure-detection self-test (no counterpart in the paper): launches one
 * kernel whose only thread waits on a device barrier that nothing completes,
 * through the bounded wait every tensor-core kernel uses, and reads the
 * context's device flag.  The wait gives up after `cycles` SM clocks
 * (1 .. 4e9), records its code, and the kernel returns normally, so the call
 * returns BQC_E_DEVICE_FLAG and the context stays usable.  BQC_E_INVALID for
 * cycles out of range.  Synchronises the stream. */
int bqc_wait_selftest(bqc_ctx *ctx, long long cycles, bqc_stream_t stream);

const char *bqc_strerror(int status);
/* Text of the last error recorded on the calling thread (file:line of the failing call). */
const char *bqc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* BQC_H */
