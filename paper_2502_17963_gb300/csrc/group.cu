// Grouped Fock builds of independent molecules (the serving workload).
//
// A server runs many small DF-RHF solves at once; one split-FP16 Fock build
// of a molecule with N <= 1200 fills a fraction of the 152 SMs, and each of
// its passes is a separate launch.  A FockGroup batches the mixed-stage
// builds of the solves that are in flight: each solve prepares its own C
// split on its own stream and hands the build to the group; the first solve
// to arrive leads, waits (a bounded window) until every solve registered in
// the mixed stage has arrived, and launches the X pass, the FP64 J pass and
// the SYRK of the whole batch as one persistent launch each (plus their
// reductions) on the group's stream.  Every solve's stream then waits for
// that work in stream order, so the SCF around it is unchanged.  The kernels
// compute every tile exactly as the single-problem launch does.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <mutex>
#include <vector>

#include "bqc_internal.h"
#include "df_internal.h"

namespace bqc {

struct GroupJob {
  Df *df = nullptr;
  double *J = nullptr, *K = nullptr;
  int status = BQC_OK;
  bool finished = false;
};

struct FockGroup {
  std::mutex mu;
  std::condition_variable cv;
  std::mutex launch_mu;         // one batch's launches at a time on gs
  std::vector<GroupJob *> open;  // handed in, not yet taken into a batch
  bool gathering = false;        // a leader is waiting for the batch to fill
  int active = 0;                // solves registered in the mixed stage
  int max_jobs = kMaxGroup;
  double window_s = 1e-3;
  cudaStream_t gs = nullptr;
  uint64_t batches = 0, jobs = 0;
  int max_batch = 0;
};

int group_build(Df *const *dfs, double *const *J, double *const *K, int n, cudaStream_t s) {
  for (int a = 0; a < n; ++a)
    for (int b = a + 1; b < n; ++b)
      if (dfs[a] == dfs[b]) {
        set_error("a handle appears twice in one grouped build", __FILE__, __LINE__);
        return BQC_E_INVALID;
      }
  for (int k0 = 0; k0 < n; k0 += kMaxGroup) {
    const int m = std::min(kMaxGroup, n - k0);
    BQC_TRY(group_xpass(dfs + k0, m, s));
    BQC_TRY(group_jpass(dfs + k0, J + k0, m, s));
    BQC_TRY(group_syrk(dfs + k0, K + k0, m, s));
  }
  return BQC_OK;
}

static void run_batch(FockGroup *g, const std::vector<GroupJob *> &batch) {
  std::lock_guard<std::mutex> lg(g->launch_mu);
  int st = BQC_OK;
  std::vector<Df *> dfs;
  std::vector<double *> J, K;
  for (GroupJob *j : batch) {
    if (cudaStreamWaitEvent(g->gs, j->df->gready, 0) != cudaSuccess) st = BQC_E_CUDA;
    dfs.push_back(j->df);
    J.push_back(j->J);
    K.push_back(j->K);
  }
  if (st == BQC_OK) st = group_build(dfs.data(), J.data(), K.data(), (int)dfs.size(), g->gs);
  for (GroupJob *j : batch) {
    if (cudaEventRecord(j->df->gdone, g->gs) != cudaSuccess && st == BQC_OK) st = BQC_E_CUDA;
  }
  for (GroupJob *j : batch) j->status = st;
}

int jk_grouped(Df *df, const double *C, double *J, double *K, cudaStream_t s) {
  FockGroup *g = df->group;
  if (!g) return BQC_E_INVALID;
  BQC_TRY(group_prep(df, C, s));
  if (!df->gready) BQC_CUDA_TRY(cudaEventCreateWithFlags(&df->gready, cudaEventDisableTiming));
  if (!df->gdone) BQC_CUDA_TRY(cudaEventCreateWithFlags(&df->gdone, cudaEventDisableTiming));
  BQC_CUDA_TRY(cudaEventRecord(df->gready, s));
  GroupJob job;
  job.df = df;
  job.J = J;
  job.K = K;
  std::unique_lock<std::mutex> lk(g->mu);
  g->open.push_back(&job);
  g->cv.notify_all();
  while (!job.finished) {
    const bool queued = std::find(g->open.begin(), g->open.end(), &job) != g->open.end();
    if (!g->gathering && queued) {
      // lead: wait until every registered solve has handed in its build, or
      // the window ends
      g->gathering = true;
      const auto deadline = std::chrono::steady_clock::now() +
                            std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                                std::chrono::duration<double>(g->window_s));
      while ((int)g->open.size() < std::max(1, std::min(g->active, g->max_jobs)) &&
             std::chrono::steady_clock::now() < deadline)
        g->cv.wait_until(lk, deadline);
      const int take = std::min((int)g->open.size(), g->max_jobs);
      std::vector<GroupJob *> batch(g->open.begin(), g->open.begin() + take);
      g->open.erase(g->open.begin(), g->open.begin() + take);
      g->gathering = false;
      ++g->batches;
      g->jobs += (uint64_t)take;
      g->max_batch = std::max(g->max_batch, take);
      g->cv.notify_all();  // jobs left over elect the next leader
      lk.unlock();
      run_batch(g, batch);
      lk.lock();
      for (GroupJob *j : batch) j->finished = true;
      g->cv.notify_all();
      continue;
    }
    g->cv.wait(lk);
  }
  lk.unlock();
  if (job.status != BQC_OK) return job.status;
  BQC_CUDA_TRY(cudaStreamWaitEvent(s, df->gdone, 0));
  return BQC_OK;
}

void group_enter(FockGroup *g) {
  if (!g) return;
  std::lock_guard<std::mutex> lk(g->mu);
  ++g->active;
  g->cv.notify_all();
}

void group_leave(FockGroup *g) {
  if (!g) return;
  std::lock_guard<std::mutex> lk(g->mu);
  --g->active;
  g->cv.notify_all();
}

FockGroup *group_create(double window_s, int max_jobs, int priority, int *status) {
  auto *g = new FockGroup();
  g->window_s = window_s > 0.0 ? window_s : 1e-3;
  g->max_jobs = std::max(1, std::min(max_jobs > 0 ? max_jobs : kMaxGroup, kMaxGroup));
  const cudaError_t e = cudaStreamCreateWithPriority(&g->gs, cudaStreamNonBlocking, priority);
  if (e != cudaSuccess) {
    set_error(cudaGetErrorString(e), __FILE__, __LINE__);
    delete g;
    *status = BQC_E_CUDA;
    return nullptr;
  }
  *status = BQC_OK;
  return g;
}

void group_destroy(FockGroup *g) {
  if (!g) return;
  if (g->gs) {
    cudaStreamSynchronize(g->gs);
    cudaStreamDestroy(g->gs);
  }
  delete g;
}

void group_stats(FockGroup *g, uint64_t *batches, uint64_t *jobs, int *max_batch) {
  if (!g) {
    *batches = *jobs = 0;
    *max_batch = 0;
    return;
  }
  std::lock_guard<std::mutex> lk(g->mu);
  *batches = g->batches;
  *jobs = g->jobs;
  *max_batch = g->max_batch;
}

}  // namespace bqc

using namespace bqc;

extern "C" int bqc_jk_grouped(int n, bqc_df *const *dfs, const double *const *C_dev,
                              double *const *J, double *const *K, bqc_stream_t stream) {
  if (n <= 0 || !dfs || !C_dev || !J || !K) return BQC_E_INVALID;
  for (int k = 0; k < n; ++k)
    if (!dfs[k] || !C_dev[k] || !J[k] || !K[k]) return BQC_E_INVALID;
  const int dev = dfs[0]->ctx->device;
  for (int k = 1; k < n; ++k)
    if (dfs[k]->ctx->device != dev) {
      set_error("grouped handles live on different devices", __FILE__, __LINE__);
      return BQC_E_INVALID;
    }
  BQC_CUDA_TRY(cudaSetDevice(dev));
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<Df *> v(dfs, dfs + n);
  for (int k = 0; k < n; ++k) BQC_TRY(group_prep(v[k], C_dev[k], s));
  return group_build(v.data(), J, K, n, s);
}
