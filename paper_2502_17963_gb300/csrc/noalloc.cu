// Allocation-free FP64 Fock build (J and K from a stored B and C_occ).
//
// Who needs this.  Some callers cannot obtain device memory from
// cudaMalloc at the moment they want a Fock build: a host framework that has
// already reserved the GPU's memory for its own pool (cudaMalloc then fails
// or fragments that pool), or a latency-critical loop that must not pay for
// cudaMalloc / cudaFree, which can synchronise the whole device.  For them
// this entry point takes its working memory from one fixed array that is part
// of the library image instead of allocating it.
//
// The array is a file-scope __device__ object of kScratchBytes.  Every GPU
// that loads the library holds it until the process exits.  Host code never
// dereferences the symbol itself (on the host it is only a stand-in for the
// device object); the device address is obtained once per device with
// cudaGetSymbolAddress and passed to the kernels.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <mutex>

#include "bqc_internal.h"
#include "gemm64.cuh"

namespace bqc {

// Kernels of the regular FP64 build (df.cu), reused unchanged.
__global__ void k_wdot(const double *X, const double *C, int64_t nc, double *w);
__global__ void k_jpass64(const double *__restrict__ B, const double *__restrict__ w, int naux,
                          int64_t npair, double *__restrict__ Jp);
__global__ void k_unpack_sym(const double *Jp, int n, double *J);

constexpr size_t kScratchBytes = (size_t)32 << 20;  // 32 MiB
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
static std::mutex g_mu;
static void *g_scratch_dev[kMaxDevices] = {nullptr};

// Device address of g_scratch on the current device (set up once per device,
// with that device current, and kept for the life of the process; a
// cudaDeviceReset() of the device leaves the kept address stale).
static int scratch_address(void **out) {
  int dev = 0;
  BQC_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return BQC_E_INVALID;
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_scratch_dev[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) {
      set_error(e != cudaSuccess ? cudaGetErrorString(e) : "null scratch address", __FILE__,
                __LINE__);
      return BQC_E_CUDA;
    }
    g_scratch_dev[dev] = p;
  }
  *out = g_scratch_dev[dev];
  return BQC_OK;
}

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace bqc

using namespace bqc;

extern "C" int bqc_jk_fp64_noalloc(const double *B, int naux, int nbf, const double *C,
                                   int nocc, double *J, double *K, bqc_stream_t stream) {
  if (!B || !C || !J || !K || naux <= 0 || nbf <= 0 || nocc <= 0 || nocc > nbf)
    return BQC_E_INVALID;
  const int64_t npair = (int64_t)nbf * (nbf + 1) / 2;
  // scratch: X (Naux x N x nocc), w (Naux), packed J (Npair), each 256-byte aligned
  const size_t bx = align256((size_t)naux * nbf * nocc * sizeof(double));
  const size_t bw = align256((size_t)naux * sizeof(double));
  const size_t bj = align256((size_t)npair * sizeof(double));
  if (bx + bw + bj > kScratchBytes) {
    char msg[160];
    std::snprintf(msg, sizeof(msg),
                  "bqc_jk_fp64_noalloc: needs %zu bytes of scratch, limit is %zu", bx + bw + bj,
                  kScratchBytes);
    set_error(msg, __FILE__, __LINE__);
    return BQC_E_INVALID;
  }
  void *base = nullptr;
  BQC_TRY(scratch_address(&base));
  double *X = reinterpret_cast<double *>(base);
  double *w = reinterpret_cast<double *>(static_cast<unsigned char *>(base) + bx);
  double *Jp = reinterpret_cast<double *>(static_cast<unsigned char *>(base) + bx + bw);
  cudaStream_t s = (cudaStream_t)stream;
  // Every scratch entry below is written before it is read, so nothing needs
  // clearing between calls.
  Gemm64Args g;  // X_P = Bsym_P C, batched over P
  g.M = nbf;
  g.N = nocc;
  g.K1 = 1;
  g.K2 = nbf;
  g.A = B;
  g.bsA = npair;
  g.B = C;
  g.ldb = nocc;
  g.C = X;
  g.ldc = nocc;
  g.bsC = (int64_t)nbf * nocc;
  g.batch = naux;
  BQC_TRY(launch_gemm64(kASym, false, g, s));
  k_wdot<<<naux, 256, 0, s>>>(X, C, (int64_t)nbf * nocc, w);
  BQC_LAUNCH_CHECK();
  k_jpass64<<<(unsigned)((npair / 2 + 256) / 256), 256, 0, s>>>(B, w, naux, npair, Jp);
  BQC_LAUNCH_CHECK();
  k_unpack_sym<<<(unsigned)(((int64_t)nbf * nbf + 255) / 256), 256, 0, s>>>(Jp, nbf, J);
  BQC_LAUNCH_CHECK();
  Gemm64Args k;  // K = sum_{P,i} X_P,mu i X_P,nu i
  k.M = nbf;
  k.N = nbf;
  k.K1 = naux;
  k.K2 = nocc;
  k.A = X;
  k.lda = nocc;
  k.sA1 = (int64_t)nbf * nocc;
  k.B = X;
  k.ldb = nocc;
  k.sB1 = (int64_t)nbf * nocc;
  k.C = K;
  k.ldc = nbf;
  k.lower_only = 1;
  k.mirror = 1;
  return launch_gemm64(kAN, true, k, s);
}
