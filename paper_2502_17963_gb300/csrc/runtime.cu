// Context, device memory, basis setup and the integral entry points of the
// C ABI.  The basis setup follows the paper's point that preparation belongs
// on the device (Sec. 2.2.2 item 3): the host only normalises the shells and
// lays out index lists; every integral is evaluated by the kernels in eri.cu.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "bqc_internal.h"

namespace bqc {

thread_local const std::atomic<int> *tl_cancel = nullptr;

NvtxRange::NvtxRange(const char *name) { nvtxRangePushA(name); }
NvtxRange::~NvtxRange() { nvtxRangePop(); }

static thread_local char g_err[512] = "";

void set_error(const char *what, const char *file, int line) {
  std::snprintf(g_err, sizeof(g_err), "%s (%s:%d)", what, file, line);
}
const char *last_error() { return g_err; }

// Multiprocessor count of the current device, queried once per device.
int sm_count() {
  constexpr int kMaxDev = 64;
  static std::atomic<int> cache[kMaxDev];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    dev = 0;
  }
  if (dev >= 0 && dev < kMaxDev) {
    const int c = cache[dev].load(std::memory_order_relaxed);
    if (c > 0) return c;
  }
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
    cudaGetLastError();
    return 1;  // no device: a one-SM plan is valid, only slower
  }
  if (dev >= 0 && dev < kMaxDev) cache[dev].store(n, std::memory_order_relaxed);
  return n;
}

void *Ctx::dmalloc(size_t bytes) {
  if (bytes == 0) bytes = 16;
  void *p = nullptr;
  if (alloc) {
    p = alloc(bytes, user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) {
    std::lock_guard<std::mutex> g(mu);
    sizes[p] = bytes;
    bytes_live += bytes;
  }
  return p;
}

void Ctx::dfree(void *p, size_t) {
  if (!p) return;
  {
    std::lock_guard<std::mutex> g(mu);
    auto it = sizes.find(p);
    if (it != sizes.end()) {
      bytes_live -= it->second;
      sizes.erase(it);
    }
  }
  if (dealloc)
    dealloc(p, user);
  else
    cudaFree(p);
}

int Ctx::check_flag(cudaStream_t s) {
  int h = 0;
  BQC_CUDA_TRY(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  BQC_CUDA_TRY(cudaStreamSynchronize(s));
  if (h != 0) {
    BQC_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int), s));
    char msg[64];
    std::snprintf(msg, sizeof(msg), "device check tripped (code %d)", h);
    set_error(msg, __FILE__, __LINE__);
    return BQC_E_DEVICE_FLAG;
  }
  return BQC_OK;
}

int DBuf::alloc(Ctx *c, size_t bytes) {
  release();
  ctx = c;
  p = c->dmalloc(bytes);
  if (!p) {
    set_error("device allocation failed", __FILE__, __LINE__);
    return BQC_E_OOM;
  }
  n = bytes;
  return BQC_OK;
}

void DBuf::release() {
  if (p && ctx) ctx->dfree(p, n);
  p = nullptr;
  n = 0;
}

static int ncart_h(int l) { return (l + 1) * (l + 2) / 2; }

// Primitive radial norm (2a/pi)^{3/4} (4a)^{l/2} times the contraction
// coefficient; then the whole shell rescaled so that its x^l component has
// unit self-overlap: S = sum_kl c_k c_l N_k N_l (pi/(a_k+a_l))^{3/2} / (2(a_k+a_l))^l.
static int load_shells(const bqc_shell *sh, int n, int natom, const double *xyz, int lmax,
                       ShellSetHost &out) {
  out.l.clear(); out.nprim.clear(); out.poff.clear(); out.fn.clear(); out.atom.clear();
  out.xyz.clear(); out.exps.clear(); out.coefs.clear();
  int fn = 0, po = 0;
  for (int i = 0; i < n; ++i) {
    const bqc_shell &s = sh[i];
    if (s.l < 0 || s.l > lmax) return BQC_E_UNSUPPORTED;
    if (s.nprim < 1 || s.nprim > kMaxPrim || !s.exps || !s.coefs) return BQC_E_INVALID;
    if (s.atom < 0 || s.atom >= natom) return BQC_E_INVALID;
    out.l.push_back(s.l);
    out.nprim.push_back(s.nprim);
    out.poff.push_back(po);
    out.fn.push_back(fn);
    out.atom.push_back(s.atom);
    for (int x = 0; x < 3; ++x) out.xyz.push_back(xyz[3 * s.atom + x]);
    std::vector<double> c(s.nprim);
    for (int k = 0; k < s.nprim; ++k) {
      const double a = s.exps[k];
      if (!(a > 0.0) || !std::isfinite(a) || !std::isfinite(s.coefs[k])) return BQC_E_INVALID;
      c[k] = s.coefs[k] * std::pow(2.0 * a / M_PI, 0.75) * std::pow(4.0 * a, 0.5 * s.l);
    }
    double S = 0.0;
    for (int k = 0; k < s.nprim; ++k)
      for (int m = 0; m < s.nprim; ++m) {
        const double ab = s.exps[k] + s.exps[m];
        S += c[k] * c[m] * std::pow(M_PI / ab, 1.5) / std::pow(2.0 * ab, s.l);
      }
    if (!(S > 0.0)) return BQC_E_INVALID;
    const double r = 1.0 / std::sqrt(S);
    for (int k = 0; k < s.nprim; ++k) {
      out.exps.push_back(s.exps[k]);
      out.coefs.push_back(c[k] * r);
    }
    po += s.nprim;
    fn += ncart_h(s.l);
  }
  out.nfn = fn;
  return BQC_OK;
}

int ShellSetHost::upload(Ctx *ctx) {
  const int n = (int)l.size();
  std::vector<int> iv;
  iv.insert(iv.end(), l.begin(), l.end());
  iv.insert(iv.end(), nprim.begin(), nprim.end());
  iv.insert(iv.end(), poff.begin(), poff.end());
  iv.insert(iv.end(), fn.begin(), fn.end());
  std::vector<double> dv;
  dv.insert(dv.end(), xyz.begin(), xyz.end());
  dv.insert(dv.end(), exps.begin(), exps.end());
  dv.insert(dv.end(), coefs.begin(), coefs.end());
  BQC_TRY(d_int.alloc(ctx, std::max<size_t>(1, iv.size()) * sizeof(int)));
  BQC_TRY(d_dbl.alloc(ctx, std::max<size_t>(1, dv.size()) * sizeof(double)));
  BQC_CUDA_TRY(cudaMemcpy(d_int.p, iv.data(), iv.size() * sizeof(int), cudaMemcpyHostToDevice));
  BQC_CUDA_TRY(
      cudaMemcpy(d_dbl.p, dv.data(), dv.size() * sizeof(double), cudaMemcpyHostToDevice));
  const int *ip = d_int.as<int>();
  const double *dp = d_dbl.as<double>();
  const int np = (int)exps.size();
  dev.n = n;
  dev.l = ip;
  dev.nprim = ip + n;
  dev.poff = ip + 2 * n;
  dev.fn = ip + 3 * n;
  dev.xyz = dp;
  dev.exps = dp + 3 * n;
  dev.coefs = dp + 3 * n + np;
  return BQC_OK;
}

}  // namespace bqc

using namespace bqc;

extern "C" {

const char *bqc_strerror(int status) {
  switch (status) {
    case BQC_OK: return "ok";
    case BQC_E_INVALID: return "invalid argument";
    case BQC_E_OOM: return "out of device memory";
    case BQC_E_ADMISSION: return "request exceeds the HBM budget";
    case BQC_E_NOT_CONVERGED: return "SCF not converged";
    case BQC_E_CUDA: return "CUDA error";
    case BQC_E_TIMEOUT: return "timeout";
    case BQC_E_DEVICE_FLAG: return "device-side check tripped";
    case BQC_E_NOT_READY: return "not ready";
    case BQC_E_UNSUPPORTED: return "unsupported (angular momentum or size)";
    case BQC_E_CANCELLED: return "cancelled";
  }
  return "unknown status";
}

const char *bqc_last_error(void) { return last_error(); }

int bqc_ctx_create(int device, size_t hbm_budget, bqc_alloc_fn alloc, bqc_free_fn dealloc,
                   void *alloc_user, bqc_ctx **out) {
  if (!out) return BQC_E_INVALID;
  *out = nullptr;
  if ((alloc == nullptr) != (dealloc == nullptr)) return BQC_E_INVALID;
  int ndev = 0;
  BQC_CUDA_TRY(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return BQC_E_INVALID;
  BQC_CUDA_TRY(cudaSetDevice(device));
  bqc_ctx *c = new (std::nothrow) bqc_ctx();
  if (!c) return BQC_E_OOM;
  c->device = device;
  c->budget = hbm_budget;
  c->alloc = alloc;
  c->dealloc = dealloc;
  c->user = alloc_user;
  c->flag = (int *)c->dmalloc(sizeof(int));
  if (!c->flag) {
    delete c;
    return BQC_E_OOM;
  }
  if (cudaMemset(c->flag, 0, sizeof(int)) != cudaSuccess) {
    bqc_ctx_destroy(c);
    return BQC_E_CUDA;
  }
  const int st = boys_table_build(c);
  if (st != BQC_OK) {
    bqc_ctx_destroy(c);
    return st;
  }
  *out = c;
  return BQC_OK;
}

int bqc_ctx_destroy(bqc_ctx *ctx) {
  if (!ctx) return BQC_E_INVALID;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  ctx->dfree(ctx->boys, (size_t)kBoysNT * kBoysNM * sizeof(double));
  ctx->dfree(ctx->flag, sizeof(int));
  delete ctx;
  return BQC_OK;
}

int bqc_basis_load(bqc_ctx *ctx, int natom, const int *Z, const double *xyz_bohr,
                   const bqc_shell *orb, int norb_shell, const bqc_shell *aux, int naux_shell,
                   bqc_basis **out) {
  if (!ctx || !out || natom <= 0 || !Z || !xyz_bohr || !orb || !aux || norb_shell <= 0 ||
      naux_shell <= 0)
    return BQC_E_INVALID;
  *out = nullptr;
  BQC_CUDA_TRY(cudaSetDevice(ctx->device));
  bqc_basis *b = new (std::nothrow) bqc_basis();
  if (!b) return BQC_E_OOM;
  auto fail = [&](int st) {
    delete b;
    return st;
  };
  b->ctx = ctx;
  b->natom = natom;
  int zsum = 0;
  for (int i = 0; i < natom; ++i) {
    if (Z[i] < 0) return fail(BQC_E_INVALID);
    b->Z.push_back(Z[i]);
    zsum += Z[i];
    for (int x = 0; x < 3; ++x) {
      if (!std::isfinite(xyz_bohr[3 * i + x])) return fail(BQC_E_INVALID);
      b->xyz.push_back(xyz_bohr[3 * i + x]);
    }
  }
  if (zsum % 2 != 0 || zsum == 0) return fail(BQC_E_INVALID);
  int st = load_shells(orb, norb_shell, natom, xyz_bohr, kMaxLOrb, b->orb);
  if (st != BQC_OK) return fail(st);
  st = load_shells(aux, naux_shell, natom, xyz_bohr, kMaxLAux, b->aux);
  if (st != BQC_OK) return fail(st);
  b->nbf = b->orb.nfn;
  b->naux = b->aux.nfn;
  b->nocc = zsum / 2;
  if (b->nocc > b->nbf) return fail(BQC_E_INVALID);
  double e = 0.0;
  for (int a = 0; a < natom; ++a)
    for (int c = 0; c < a; ++c) {
      double r2 = 0.0;
      for (int x = 0; x < 3; ++x) {
        const double d = b->xyz[3 * a + x] - b->xyz[3 * c + x];
        r2 += d * d;
      }
      if (r2 == 0.0) {
        if (b->Z[a] * b->Z[c] != 0) return fail(BQC_E_INVALID);
        continue;
      }
      e += b->Z[a] * b->Z[c] / std::sqrt(r2);
    }
  b->enuc = e;
  // oriented orbital shell pairs grouped by class
  std::vector<std::vector<int2>> cls(kNPairClass);
  for (int i = 0; i < norb_shell; ++i)
    for (int j = 0; j <= i; ++j) {
      int a = i, c = j;
      if (b->orb.l[c] > b->orb.l[a]) std::swap(a, c);
      cls[pair_class(b->orb.l[a], b->orb.l[c])].push_back(make_int2(a, c));
    }
  std::vector<int2> pairs;
  for (int k = 0; k < kNPairClass; ++k) {
    b->pair_off[k] = (int)pairs.size();
    pairs.insert(pairs.end(), cls[k].begin(), cls[k].end());
  }
  b->pair_off[kNPairClass] = (int)pairs.size();
  b->npair_sh = (int64_t)pairs.size();
  std::vector<int> auxl;
  for (int l = 0; l <= kMaxLAux; ++l) {
    b->auxl_off[l] = (int)auxl.size();
    for (int i = 0; i < naux_shell; ++i)
      if (b->aux.l[i] == l) auxl.push_back(i);
  }
  b->auxl_off[kMaxLAux + 1] = (int)auxl.size();
  std::vector<double> atoms(4 * natom);
  for (int a = 0; a < natom; ++a) {
    for (int x = 0; x < 3; ++x) atoms[4 * a + x] = b->xyz[3 * a + x];
    atoms[4 * a + 3] = b->Z[a];
  }
  if ((st = b->orb.upload(ctx)) != BQC_OK) return fail(st);
  if ((st = b->aux.upload(ctx)) != BQC_OK) return fail(st);
  if ((st = b->d_pairs.alloc(ctx, pairs.size() * sizeof(int2))) != BQC_OK) return fail(st);
  if ((st = b->d_aux_by_l.alloc(ctx, auxl.size() * sizeof(int))) != BQC_OK) return fail(st);
  if ((st = b->d_atoms.alloc(ctx, atoms.size() * sizeof(double))) != BQC_OK) return fail(st);
  if (cudaMemcpy(b->d_pairs.p, pairs.data(), pairs.size() * sizeof(int2),
                 cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_aux_by_l.p, auxl.data(), auxl.size() * sizeof(int),
                 cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_atoms.p, atoms.data(), atoms.size() * sizeof(double),
                 cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(BQC_E_CUDA);
  *out = b;
  return BQC_OK;
}

int bqc_basis_destroy(bqc_basis *basis) {
  if (!basis) return BQC_E_INVALID;
  cudaSetDevice(basis->ctx->device);
  cudaDeviceSynchronize();
  delete basis;
  return BQC_OK;
}

int bqc_basis_info(const bqc_basis *b, int *nbf, int *naux, int *nocc, int64_t *npair) {
  if (!b) return BQC_E_INVALID;
  if (nbf) *nbf = b->nbf;
  if (naux) *naux = b->naux;
  if (nocc) *nocc = b->nocc;
  if (npair) *npair = b->npair_sh;
  return BQC_OK;
}

int bqc_basis_enuc(const bqc_basis *b, double *enuc) {
  if (!b || !enuc) return BQC_E_INVALID;
  *enuc = b->enuc;
  return BQC_OK;
}

int bqc_one_electron(const bqc_basis *b, double *S, double *T, double *V, bqc_stream_t stream) {
  if (!b) return BQC_E_INVALID;
  BQC_CUDA_TRY(cudaSetDevice(b->ctx->device));
  return launch_one_electron(b, S, T, V, (cudaStream_t)stream);
}

int bqc_boys(bqc_ctx *ctx, int n, const double *T, int mmax, double *out, bqc_stream_t stream) {
  if (!ctx || (n > 0 && (!T || !out))) return BQC_E_INVALID;
  BQC_CUDA_TRY(cudaSetDevice(ctx->device));
  return launch_boys_eval(ctx, n, T, mmax, out, (cudaStream_t)stream);
}

int bqc_int2c(const bqc_basis *b, double *V, bqc_stream_t stream) {
  if (!b || !V) return BQC_E_INVALID;
  BQC_CUDA_TRY(cudaSetDevice(b->ctx->device));
  return launch_int2c(b, V, (cudaStream_t)stream);
}

int bqc_int3c(const bqc_basis *b, double schwarz, double *out, bqc_stream_t stream) {
  if (!b || !out) return BQC_E_INVALID;
  BQC_CUDA_TRY(cudaSetDevice(b->ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t npair = (int64_t)b->nbf * (b->nbf + 1) / 2;
  DBuf V;
  BQC_TRY(V.alloc(b->ctx, (size_t)b->naux * b->naux * sizeof(double)));
  BQC_TRY(launch_int2c(b, V.as<double>(), s));
  Eri3cPlan plan;
  BQC_TRY(eri3c_plan(b, schwarz, V.as<double>(), s, &plan));
  BQC_CUDA_TRY(cudaMemsetAsync(out, 0, (size_t)b->naux * npair * sizeof(double), s));
  BQC_TRY(launch_eri3c(b, &plan, 0, b->naux, out, npair, s));
  BQC_CUDA_TRY(cudaStreamSynchronize(s));  // plan buffers are released on return
  return b->ctx->check_flag(s);
}

}  // extern "C"
