// Continuous-batching server for DF-RHF solves (the serving workload).
//
// Requests of different molecule sizes arrive at any time.  A request is
// admitted as soon as a slot is free and the HBM ledger has room for its
// predicted footprint (queue order, with bounded backfill past a head that
// does not fit); every admitted request runs its basis setup, DF build and
// SCF on its own CUDA stream, prioritised by molecule size, so the work of
// several molecules overlaps on the device while new requests keep arriving.  All device memory comes
// from one arena reserved when the server is created, so the serving loop
// never calls cudaMalloc / cudaFree (both can synchronise the device and
// would serialise the slots).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "bqc_internal.h"
#include "df_internal.h"

namespace bqc {

// ------------------------------------------------------------- arena ----

// Sub-allocator over one device allocation; blocks are 256-byte aligned and
// neighbouring free blocks are merged on release.  Small blocks are placed
// first-fit from the bottom, large ones (>= kLarge) best-fit at the top end
// of their free block, so that the many small buffers of concurrent solves
// do not split the space the multi-GB DF tensors need.
struct Arena {
  char *base = nullptr;
  size_t size = 0;
  std::mutex mu;
  std::map<size_t, size_t> free_;   // offset -> size
  std::unordered_map<size_t, size_t> used_;
  size_t in_use = 0, peak = 0;

  int init(size_t bytes) {
    size = (bytes + 255) & ~(size_t)255;
    if (cudaMalloc(&base, size) != cudaSuccess) {
      cudaGetLastError();
      base = nullptr;
      set_error("arena reservation failed", __FILE__, __LINE__);
      return BQC_E_OOM;
    }
    free_[0] = size;
    return BQC_OK;
  }
  ~Arena() {
    if (base) cudaFree(base);
  }
  static constexpr size_t kLarge = (size_t)256 << 20;
  void *alloc(size_t bytes) {
    bytes = (std::max<size_t>(bytes, 1) + 255) & ~(size_t)255;
    std::lock_guard<std::mutex> g(mu);
    auto pick = free_.end();
    if (bytes < kLarge) {
      for (auto it = free_.begin(); it != free_.end(); ++it)
        if (it->second >= bytes) {
          pick = it;
          break;
        }
    } else {
      for (auto it = free_.begin(); it != free_.end(); ++it)
        if (it->second >= bytes && (pick == free_.end() || it->second < pick->second)) pick = it;
    }
    if (pick == free_.end()) return nullptr;
    const size_t off0 = pick->first, len = pick->second, rest = len - bytes;
    free_.erase(pick);
    size_t off = off0;
    if (bytes < kLarge) {
      if (rest) free_[off0 + bytes] = rest;
    } else {
      off = off0 + rest;  // top end of the block
      if (rest) free_[off0] = rest;
    }
    used_[off] = bytes;
    in_use += bytes;
    peak = std::max(peak, in_use);
    return base + off;
  }
  void release(void *p) {
    if (!p) return;
    std::lock_guard<std::mutex> g(mu);
    const size_t off = (size_t)((char *)p - base);
    auto u = used_.find(off);
    if (u == used_.end()) return;
    size_t sz = u->second;
    used_.erase(u);
    in_use -= sz;
    size_t start = off;
    auto nx = free_.lower_bound(off);
    if (nx != free_.end() && nx->first == off + sz) {
      sz += nx->second;
      nx = free_.erase(nx);
    }
    if (nx != free_.begin()) {
      auto pv = std::prev(nx);
      if (pv->first + pv->second == start) {
        start = pv->first;
        sz += pv->second;
        free_.erase(pv);
      }
    }
    free_[start] = sz;
  }
};

static void *arena_alloc(size_t bytes, void *user) { return static_cast<Arena *>(user)->alloc(bytes); }
static void arena_free(void *p, void *user) { static_cast<Arena *>(user)->release(p); }

// ------------------------------------------------------------ requests --

struct Request {
  uint64_t id = 0;
  std::vector<int> Z;
  std::vector<double> xyz;
  std::vector<int> shl_atom[2], shl_l[2], shl_np[2];
  std::vector<double> exps[2], coefs[2];
  int nbf = 0, naux = 0, nocc = 0;
  size_t footprint = 0;
  int skipped = 0;  // times a later request was admitted ahead of this one
  int retries = 0;  // re-admissions after an allocation failure
  bool wait_for_release = false;  // requeued: wait until another solve ends
  uint64_t release_mark = 0;      // srv->releases when it was requeued
  double t_submit = 0.0;
  bool done = false;
  bool running = false;
  std::atomic<int> cancel{0};
  bqc_serve_result res{};
};

static int ncart_s(int l) { return (l + 1) * (l + 2) / 2; }

}  // namespace bqc

struct bqc_server {
  bqc::Ctx *outer = nullptr;
  bqc_ctx *ctx = nullptr;  // internal context allocating from the arena
  bqc::Arena arena;
  bqc_serve_opts opts{};
  size_t budget = 0, ledger = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, std::unique_ptr<bqc::Request>> reqs;
  std::vector<std::thread> workers;
  uint64_t next_id = 1;
  int pending = 0;
  bool stop = false;
  int prio_least = 0, prio_greatest = 0;  // CUDA stream priority range
  uint64_t releases = 0;                  // solves finished (their memory freed)
  bqc::FockGroup *group = nullptr;        // grouped mixed-stage builds (opts.grouped)
  std::chrono::steady_clock::time_point t0;
  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace bqc {

// Shadow kind a precision needs.
static int shadow_of_prec(int prec) {
  return prec == BQC_PREC_MIXED_F16X3 ? BQC_SHADOW_F16
         : prec == BQC_PREC_FP64      ? BQC_SHADOW_NONE
                                      : BQC_SHADOW_TF32;
}

// Predicted device bytes of one solve: stored DF tensors (FP64 B, split TF32
// shadows, X), the integral screening plan, and the SCF work matrices.
size_t serve_footprint(int n, int naux, int nocc, int shadow) {
  const size_t nn = (size_t)n * n;
  size_t b = df_stored_bytes(n, naux, nocc, shadow);
  b += (size_t)naux * naux * 8;             // metric copy during the build
  b += (size_t)(16 + 2 * 8) * nn * 8;       // SCF matrices + DIIS history
  b += (size_t)3 * n * n / 2 * 16;          // shell-pair plan (generous)
  b += (size_t)64 << 20;                    // Boys table, small buffers, alignment
  return b;
}

static void run_request(bqc_server *srv, Request *r, cudaStream_t s) {
  NvtxRange nv("serve request");
  std::vector<bqc_shell> sh[2];
  for (int k = 0; k < 2; ++k) {
    size_t po = 0;
    for (size_t i = 0; i < r->shl_l[k].size(); ++i) {
      sh[k].push_back(bqc_shell{r->shl_atom[k][i], r->shl_l[k][i], r->shl_np[k][i],
                                r->exps[k].data() + po, r->coefs[k].data() + po});
      po += r->shl_np[k][i];
    }
  }
  bqc_basis *basis = nullptr;
  bqc_df *df = nullptr;
  tl_cancel = &r->cancel;
  int st = cancel_requested() ? BQC_E_CANCELLED : BQC_OK;
  if (st == BQC_OK)
    st = bqc_basis_load(srv->ctx, (int)r->Z.size(), r->Z.data(), r->xyz.data(), sh[0].data(),
                          (int)sh[0].size(), sh[1].data(), (int)sh[1].size(), &basis);
  bqc_scf_result res{};
  if (st == BQC_OK) {
    bqc_df_opts o{};
    o.mode = BQC_DF_STORED;
    o.schwarz = -1.0;
    o.aux_block = 1024;
    o.keep_fp32 = shadow_of_prec(srv->opts.prec);
    o.hbm_limit = 0;
    st = bqc_df_build(srv->ctx, basis, &o, (bqc_stream_t)s, &df);
  }
  if (st == BQC_OK && cancel_requested()) st = BQC_E_CANCELLED;
  if (st == BQC_OK && srv->group) df->group = srv->group;
  if (st == BQC_OK) {
    bqc_scf_opts so = srv->opts.scf;
    so.guess_C = nullptr;  // every request starts from its own core guess
    so.prec = srv->opts.prec;
    st = bqc_scf_run(srv->ctx, df, &so, (bqc_stream_t)s, &res);
  }
  // the stream is idle now: free without the device-wide synchronisation of
  // the public destroy calls, which would stall the other slots
  cudaStreamSynchronize(s);
  tl_cancel = nullptr;
  delete df;
  delete basis;
  r->res.status = st;
  r->res.energy = res.energy;
  r->res.diis_err = res.diis_err;
  r->res.iterations = res.iterations;
  r->res.iterations_mixed = res.iterations_mixed;
}

// Stream priority of a request: one level above the lowest per halving of N
// below 1536, so a small molecule's blocks are scheduled ahead of a large
// one's when both are pending (running blocks are never preempted).
static int request_priority(const bqc_server *srv, int nbf) {
  if (srv->opts.policy == BQC_SERVE_FIFO) return srv->prio_least;
  int lvl = 0;
  for (int m = 1536; lvl < srv->prio_least - srv->prio_greatest && 2 * nbf <= m; m /= 2) ++lvl;
  return srv->prio_least - lvl;
}

// Next request to admit (called with srv->mu held), or nullptr.  The queue
// head is admitted when it fits the ledger.  Otherwise, with backfill, the
// first later request that fits is admitted instead and the head's skip
// count grows; once it reaches max_skips nothing passes the head any more.
static Request *pick_request(bqc_server *srv) {
  if (srv->queue.empty()) return nullptr;
  auto fits = [&](const Request *r) {
    if (r->wait_for_release && srv->releases <= r->release_mark) return false;
    return srv->ledger + r->footprint <= srv->budget;
  };
  Request *h = srv->reqs[srv->queue.front()].get();
  if (fits(h)) {
    srv->queue.pop_front();
    return h;
  }
  const int max_skips = srv->opts.max_skips > 0 ? srv->opts.max_skips : 8;
  if (srv->opts.policy == BQC_SERVE_FIFO || h->skipped >= max_skips) return nullptr;
  for (auto it = srv->queue.begin() + 1; it != srv->queue.end(); ++it) {
    Request *r = srv->reqs[*it].get();
    if (fits(r)) {
      srv->queue.erase(it);
      ++h->skipped;
      return r;
    }
  }
  return nullptr;
}

static void worker_main(bqc_server *srv) {
  cudaSetDevice(srv->ctx->device);
  // one stream per priority level, created on first use
  std::vector<cudaStream_t> streams(srv->prio_least - srv->prio_greatest + 1, nullptr);
  while (true) {
    Request *r = nullptr;
    {
      std::unique_lock<std::mutex> lk(srv->mu);
      while (!srv->stop && !(r = pick_request(srv))) srv->cv_work.wait(lk);
      if (!r) break;
      srv->ledger += r->footprint;
      r->res.t_admit = srv->now();
      r->res.priority = request_priority(srv, r->nbf);
    }
    cudaStream_t &s = streams[srv->prio_least - r->res.priority];
    if (!s && cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, r->res.priority) != cudaSuccess) {
      cudaGetLastError();
      s = nullptr;
    }
    if (s) {
      run_request(srv, r, s);
    } else {
      r->res.status = BQC_E_CUDA;
    }
    bool requeued = false;
    {
      std::lock_guard<std::mutex> lk(srv->mu);
      srv->ledger -= r->footprint;
      // The ledger admitted it, so an allocation failure means the free space
      // was split by the solves in flight: retry at the head of the queue once
      // some of them have finished (a bounded number of times).
      if (r->res.status == BQC_E_OOM && srv->ledger > 0 && r->retries < 4) {
        ++r->retries;
        r->res = bqc_serve_result{};
        r->res.status = BQC_E_NOT_READY;
        r->res.nbf = r->nbf;
        r->res.t_submit = r->t_submit;
        r->wait_for_release = true;
        r->release_mark = srv->releases;
        srv->queue.push_front(r->id);
        requeued = true;
      } else {
        r->res.t_done = srv->now();
        r->done = true;
        --srv->pending;
        ++srv->releases;
      }
    }
    srv->cv_work.notify_all();
    if (!requeued) srv->cv_done.notify_all();
  }
  for (cudaStream_t s : streams)
    if (s) cudaStreamDestroy(s);
}

}  // namespace bqc

using namespace bqc;

extern "C" {

size_t bqc_serve_footprint(int nbf, int naux, int nocc, int prec) {
  if (nbf <= 0 || naux <= 0 || nocc <= 0 || prec < BQC_PREC_FP64 || prec > BQC_PREC_MIXED_F16X3)
    return 0;
  return serve_footprint(nbf, naux, nocc, shadow_of_prec(prec));
}

int bqc_serve_create(bqc_ctx *ctx, const bqc_serve_opts *opts, bqc_server **out) {
  if (!ctx || !out) return BQC_E_INVALID;
  *out = nullptr;
  BQC_CUDA_TRY(cudaSetDevice(ctx->device));
  std::unique_ptr<bqc_server> srv(new bqc_server());
  srv->outer = ctx;
  bqc_serve_opts o{};
  o.max_slots = 4;
  o.hbm_budget = 0;
  o.prec = BQC_PREC_MIXED_F16X3;
  o.scf.diis_tol = 1e-8;
  o.scf.energy_tol = 1e-10;
  o.scf.stage_tol = 1e-5;
  o.scf.max_iter = 100;
  o.scf.diis_space = 8;
  o.scf.orth_thresh = 1e-8;
  o.policy = BQC_SERVE_BACKFILL;
  o.max_skips = 8;
  if (opts) o = *opts;
  if (o.max_slots <= 0) o.max_slots = 4;
  if (o.policy != BQC_SERVE_FIFO) o.policy = BQC_SERVE_BACKFILL;
  if (o.max_skips <= 0) o.max_skips = 8;
  srv->opts = o;
  BQC_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&srv->prio_least, &srv->prio_greatest));
  size_t budget = o.hbm_budget ? o.hbm_budget : ctx->budget;
  if (!budget) {
    size_t fr = 0, tot = 0;
    BQC_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
    budget = fr / 2;
  }
  srv->budget = budget;
  BQC_TRY(srv->arena.init(budget + ((size_t)64 << 20)));
  bqc_ctx *ic = nullptr;
  BQC_TRY(bqc_ctx_create(ctx->device, budget, arena_alloc, arena_free, &srv->arena, &ic));
  srv->ctx = ic;
  if (o.grouped && o.prec == BQC_PREC_MIXED_F16X3) {
    int gst = BQC_OK;
    const double win = o.group_window_us > 0.0 ? o.group_window_us * 1e-6 : 1e-3;
    srv->group = group_create(win, o.max_slots, srv->prio_greatest, &gst);
    if (!srv->group) return gst;
  }
  srv->t0 = std::chrono::steady_clock::now();
  for (int i = 0; i < o.max_slots; ++i) srv->workers.emplace_back(worker_main, srv.get());
  *out = srv.release();
  return BQC_OK;
}

int bqc_serve_submit(bqc_server *srv, const bqc_request *q, uint64_t *ticket) {
  if (!srv || !q || !ticket || q->natom <= 0 || !q->Z || !q->xyz_bohr || !q->orb || !q->aux)
    return BQC_E_INVALID;
  std::unique_ptr<Request> r(new Request());
  r->Z.assign(q->Z, q->Z + q->natom);
  r->xyz.assign(q->xyz_bohr, q->xyz_bohr + 3 * q->natom);
  int zsum = 0;
  for (int z : r->Z) zsum += z;
  const bqc_shell *lists[2] = {q->orb, q->aux};
  const int counts[2] = {q->norb_shell, q->naux_shell};
  int nf[2] = {0, 0};
  for (int k = 0; k < 2; ++k) {
    if (counts[k] <= 0) return BQC_E_INVALID;
    for (int i = 0; i < counts[k]; ++i) {
      const bqc_shell &s = lists[k][i];
      if (s.nprim <= 0 || s.nprim > kMaxPrim || !s.exps || !s.coefs) return BQC_E_INVALID;
      r->shl_atom[k].push_back(s.atom);
      r->shl_l[k].push_back(s.l);
      r->shl_np[k].push_back(s.nprim);
      r->exps[k].insert(r->exps[k].end(), s.exps, s.exps + s.nprim);
      r->coefs[k].insert(r->coefs[k].end(), s.coefs, s.coefs + s.nprim);
      nf[k] += ncart_s(s.l);
    }
  }
  r->nbf = nf[0];
  r->naux = nf[1];
  r->nocc = zsum / 2;
  r->footprint = serve_footprint(r->nbf, r->naux, std::max(1, r->nocc),
                                 shadow_of_prec(srv->opts.prec));
  if (r->footprint > srv->budget) return BQC_E_ADMISSION;
  std::lock_guard<std::mutex> lk(srv->mu);
  r->id = srv->next_id++;
  r->res.status = BQC_E_NOT_READY;
  r->res.nbf = r->nbf;
  r->res.t_submit = srv->now();
  r->t_submit = r->res.t_submit;
  *ticket = r->id;
  srv->queue.push_back(r->id);
  ++srv->pending;
  srv->reqs[r->id] = std::move(r);
  srv->cv_work.notify_all();
  return BQC_OK;
}

int bqc_serve_poll(bqc_server *srv, uint64_t ticket, bqc_serve_result *res) {
  if (!srv || !res) return BQC_E_INVALID;
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(ticket);
  if (it == srv->reqs.end()) return BQC_E_INVALID;
  if (!it->second->done) return BQC_E_NOT_READY;
  *res = it->second->res;
  return BQC_OK;
}

int bqc_serve_cancel(bqc_server *srv, uint64_t ticket) {
  if (!srv) return BQC_E_INVALID;
  bool finished_now = false;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return BQC_E_INVALID;
    Request *r = it->second.get();
    if (r->done) return BQC_OK;
    r->cancel.store(1, std::memory_order_relaxed);
    auto q = std::find(srv->queue.begin(), srv->queue.end(), ticket);
    if (q != srv->queue.end()) {  // still queued: complete it now
      srv->queue.erase(q);
      r->res.status = BQC_E_CANCELLED;
      r->res.t_done = srv->now();
      r->done = true;
      --srv->pending;
      finished_now = true;
    }
  }
  if (finished_now) {
    srv->cv_work.notify_all();
    srv->cv_done.notify_all();
  }
  return BQC_OK;
}

int bqc_serve_drain(bqc_server *srv, double timeout_s) {
  if (!srv) return BQC_E_INVALID;
  std::unique_lock<std::mutex> lk(srv->mu);
  auto pred = [&] { return srv->pending == 0; };
  if (timeout_s <= 0) {
    srv->cv_done.wait(lk, pred);
    return BQC_OK;
  }
  const bool ok = srv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred);
  return ok ? BQC_OK : BQC_E_TIMEOUT;
}

int bqc_serve_destroy(bqc_server *srv) {
  if (!srv) return BQC_E_INVALID;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
  }
  srv->cv_work.notify_all();
  for (auto &t : srv->workers) t.join();
  group_destroy(srv->group);
  if (srv->ctx) bqc_ctx_destroy(srv->ctx);
  delete srv;
  return BQC_OK;
}

int bqc_serve_group_stats(bqc_server *srv, uint64_t *batches, uint64_t *builds, int *max_batch) {
  if (!srv || !batches || !builds || !max_batch) return BQC_E_INVALID;
  group_stats(srv->group, batches, builds, max_batch);
  return BQC_OK;
}

}  // extern "C"
