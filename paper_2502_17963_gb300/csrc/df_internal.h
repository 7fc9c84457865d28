// Internal state of a DF handle (stored or direct mode).
#pragma once
#include <memory>

#include "bqc_internal.h"

namespace bqc {

// Aux pieces of the split-FP16 build's X pass (each followed by its J pass).
constexpr int kJPieces = 4;
// Problems of one grouped launch (the problem table is a kernel parameter).
constexpr int kMaxGroup = 12;
struct FockGroup;

struct MixedState;
size_t mixed_bytes(const MixedState *ms);
struct MixedDeleter {
  void operator()(MixedState *p) const;
};
struct DirectMixed;
struct DirectMixedDeleter {
  void operator()(DirectMixed *p) const;
};
struct Jk4Plan;
struct Jk4Deleter {
  void operator()(Jk4Plan *p) const;
};

struct Df {
  Ctx *ctx = nullptr;
  const Basis *basis = nullptr;
  int mode = BQC_DF_STORED;
  int64_t npair = 0;
  bqc_df_opts opts{};
  int p0 = 0;        // first aux function of the handle's shard
  int naux_loc = 0;  // aux functions held (Naux unless the handle is a shard)
  bool is_shard() const { return naux_loc != basis->naux; }
  DBuf L;      // Naux x Naux lower Cholesky factor of the metric
  DBuf Vdiag;  // metric copy (screening; direct mode keeps it)
  Eri3cPlan plan;
  // stored mode
  DBuf B64;    // Naux x Npair, FP64, packed lower triangle
  DBuf X64;    // Naux x N x nocc, FP64
  DBuf Jp;     // Npair FP64 (packed J)
  DBuf w;      // Naux FP64: w_P = B_P : D
  // float-pair copy of B for the J pass of the split-FP16 build on the FP32
  // pipe: [P][Npair][2] = (hi, lo), hi = fl(B), lo = fl(B - hi); and w as
  // float pairs [Naux][2]
  DBuf B2f, w2f;
  DBuf host_io;
  // mixed precision (TF32 tensor cores)
  DBuf B32;    // Naux x N x ld, TF32 hi part of B, full square (MMA A operand)
  DBuf X32;    // Naux x N x nocc_pad FP32
  DBuf Ct32;   // nocc_pad x N FP32 (C_occ^T, TF32-rounded: MMA B operand, K-major)
  DBuf wpart;  // per X-pass tile partial w (FP64)
  DBuf Kpart;  // SYRK partial tiles (FP32)
  std::unique_ptr<MixedState, MixedDeleter> mixed;  // plan, tensor maps, epilogue buffers
  // direct mode
  DBuf raw;    // aux block x Npair FP64 raw integrals
  DBuf Linv;   // Naux x Naux FP64 L^{-1}
  DBuf Xraw;   // FP64 path: Naux x N x nocc, then Y = L^{-1} X in place
  DBuf gamma;  // Naux FP64: gamma_Q = (Q|D), then c = V^{-1} gamma
  DBuf D2;     // Npair FP64 packed density, off-diagonal doubled
  DBuf Kpart64;
  int aux_block = 1024;
  std::unique_ptr<DirectMixed, DirectMixedDeleter> dmixed;  // tensor-core state
  // conventional four-centre mode (no density fitting)
  std::unique_ptr<Jk4Plan, Jk4Deleter> jk4;
  // phase timing (bqc_df_timing)
  bool timing = false, timed = false, last_mixed = false;
  int j_from = 2;  // event that opens the J phase of the last mixed stored build
  cudaEvent_t ev[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  void mark(int i, cudaStream_t s) {
    if (timing && ev[i]) cudaEventRecord(ev[i], s);
  }
  // side stream of the mixed build: J runs there concurrently with the tensor-core passes
  cudaStream_t side = nullptr;
  cudaStream_t tcs = nullptr;  // tensor-core stream, one priority level above side
  cudaEvent_t fork = nullptr, join = nullptr, fork2 = nullptr, prep = nullptr, tjoin = nullptr;
  cudaEvent_t piece[kJPieces] = {};  // end of each X-pass piece (split-FP16 pipeline)
  // grouped builds (serving): the group this handle's mixed builds join, and
  // the events that hand a build to the group and back
  FockGroup *group = nullptr;
  cudaEvent_t gready = nullptr, gdone = nullptr;
  ~Df() {
    if (gready) cudaEventDestroy(gready);
    if (gdone) cudaEventDestroy(gdone);
    for (auto &e : ev)
      if (e) cudaEventDestroy(e);
    if (fork) cudaEventDestroy(fork);
    if (fork2) cudaEventDestroy(fork2);
    if (prep) cudaEventDestroy(prep);
    for (auto &e : piece)
      if (e) cudaEventDestroy(e);
    if (tjoin) cudaEventDestroy(tjoin);
    if (tcs) cudaStreamDestroy(tcs);
    if (join) cudaEventDestroy(join);
    if (side) cudaStreamDestroy(side);
  }
  size_t device_bytes() const {
    return L.n + Vdiag.n + B64.n + B2f.n + w2f.n + X64.n + Jp.n + w.n + host_io.n + B32.n +
           X32.n + Ct32.n +
           wpart.n + Kpart.n + raw.n + Linv.n + Xraw.n + gamma.n + D2.n +
           plan.d_pairs_sorted.n + plan.d_qpair_sorted.n + plan.d_qaux.n + plan.d_prefix.n +
           plan.d_qpair.n +
           mixed_bytes(mixed.get());
  }
};

// Device bytes of the mixed-precision state beyond the Df buffers (shadow:
// BQC_SHADOW_TF32 or BQC_SHADOW_F16).
size_t mixed_workspace_bytes(int n, int naux, int nocc, int shadow);
int mixed_ld(int n);  // row length of the TF32 shadow (N rounded up to 4)
int mixed_setup(Df *df, int shadow, cudaStream_t s);
int jk_mixed_stored(Df *df, const double *C, int prec, double *J, double *K, cudaStream_t s);
// K of the symmetric density Cw Cd^T + Cd Cw^T (N x nocc row-major inputs)
// on the split-FP16 tensor cores; BQC_E_UNSUPPORTED without FP16 shadows.
int jk_k_rank2(Df *df, const double *Cw, const double *Cd, double *K, cudaStream_t s);
int jk_fp64_stored(Df *df, const double *C, double *J, double *K, cudaStream_t s);
// J = sum_P w_P B_P from the packed FP64 B and df->w (FP64), full symmetric.
int jpass_fp64(Df *df, double *J, cudaStream_t s);
// The FP64 J pass in pieces: partials of aux functions [P0, P1) (df->w) into
// partial slices starting at y0, then the sum of nslice slices into J.
int jpass_fp64_range(Df *df, int P0, int P1, int y0, cudaStream_t s);
int jpass_unpack(Df *df, int nslice, double *J, cudaStream_t s);
// The same J partials from the float-pair B and w (df->B2f, df->w2f) in
// float-float arithmetic on the FP32 pipe; jpass_ff_setup builds B2f.
int jpass_ff_setup(Df *df, cudaStream_t s);
int jpass_ff_range(Df *df, int P0, int P1, int y0, cudaStream_t s);
int jpass_split(int64_t npair, int naux);
// J[D] = sum_P (B_P : D) B_P in FP64 over the stored FP64 B for a symmetric
// N x N matrix D (any sign), D2 an Npair scratch.
int jfp64_of_density(Df *df, const double *D, double *D2, double *J, cudaStream_t s);
// The same on the FP32 pipe from the float-pair B (float-float arithmetic).
int jff_of_density(Df *df, const double *D, double *D2, double *J, cudaStream_t s);
int direct_setup(Df *df, cudaStream_t s);
size_t direct_mixed_bytes(int n, int naux, int nocc, int bs);
int direct_mixed_setup(Df *df, const double *Linv, int bs, cudaStream_t s);
int direct_mixed_prep_c(Df *df, const double *C, int split, cudaStream_t s);
int direct_mixed_block(Df *df, const double *raw, int q0, int nq, int split, cudaStream_t s);
int direct_mixed_finish(Df *df, int split, double *K, cudaStream_t s);
int jk_direct(Df *df, const double *C, int prec, double *J, double *K, cudaStream_t s);
size_t df_stored_bytes(int n, int naux, int nocc, int shadow);
// Split-FP16 tensor-core pair blocks of DF-MP2 (tc.cu).
struct Mp2Tc;
struct Mp2TcDeleter {
  void operator()(Mp2Tc *p) const;
};
int mp2_tc_setup(Ctx *ctx, const double *Bt, int naux, int nocc, int nv, int *flag,
                 std::unique_ptr<Mp2Tc, Mp2TcDeleter> &out, cudaStream_t s);
int mp2_tc_block(Mp2Tc *m, int nv, int i0, int ni, int j0, int nj, double *V, int64_t ldv,
                 int *flag, cudaStream_t s);
int jk4c_setup(Df *df, cudaStream_t s);
// Grouped split-FP16 builds of independent handles (stored, unsharded, FP16
// shadows): group_prep splits one handle's C (its own stream); group_xpass
// (X and w), group_jpass (FP64 J) and group_syrk (K) then each run n <=
// kMaxGroup problems in one launch (plus one small reduction launch).
int group_prep(Df *df, const double *C, cudaStream_t s);
int group_xpass(Df *const *dfs, int n, cudaStream_t s);
int group_jpass(Df *const *dfs, double *const *J, int n, cudaStream_t s);
int group_syrk(Df *const *dfs, double *const *K, int n, cudaStream_t s);
// All three for n handles whose C was split by group_prep, on stream s.
int group_build(Df *const *dfs, double *const *J, double *const *K, int n, cudaStream_t s);
// A mixed build of one handle through its group (blocks until the group has
// launched it; the build is complete in stream order on s on return).
int jk_grouped(Df *df, const double *C, double *J, double *K, cudaStream_t s);
void group_enter(FockGroup *g);
void group_leave(FockGroup *g);
// A group whose batches launch on a new stream of the given priority; window_s
// bounds how long a leader waits for the registered solves.
FockGroup *group_create(double window_s, int max_jobs, int priority, int *status);
void group_destroy(FockGroup *g);
void group_stats(FockGroup *g, uint64_t *batches, uint64_t *jobs, int *max_batch);
int jk_4c(Df *df, const double *C, int prec, double *J, double *K, cudaStream_t s);

}  // namespace bqc

struct bqc_df : bqc::Df {};
