// Survivor compaction variants of the screened three-centre integrals, kept
// as a measured ablation beside the library's sorted-prefix compaction
// (eri.cu): the paper's per-warp loop buffer (Sec. 2.2.1, Algorithm 1) and a
// two-kernel global index list.  Same triplet routine, so the outputs are
// bitwise those of the shipped kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "bqc_internal.h"
#include "os_eri.cuh"

namespace bqc {

// The paper's warp-specialised prescreening (Sec. 2.2.1, Algorithm 1), kept
// as a measured variant: every warp screens batches of 32 consecutive
// candidate triplets (aux shell of the window x pair of the class, pairs in
// their original order), one per lane, and appends the survivors to a
// 64-entry loop buffer in shared memory (warp ballot for the slots); as soon
// as the buffer holds a warp's worth of work (32 / G triplets, G lanes per
// triplet) the warp computes them together, and at the end the remainder.
// head and tail are warp-uniform registers.  The buffer cannot overflow: it
// holds fewer than 32 / G entries before a batch adds at most 32.
template <int LC, int LA, int LB>
__global__ void __launch_bounds__(256) k_eri3c_ring(Eri3cArgs a) {
  using O = Os<LA, LB, LC, 0>;
  constexpr int G = O::G, W = 32 / G;
  extern __shared__ double smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gl = lane % G, gw = lane / G;
  const int groups_per_block = blockDim.x / G;
  double *scr = smem + (size_t)(threadIdx.x / G) * O::SCR;
  int64_t *ring = reinterpret_cast<int64_t *>(smem + (size_t)groups_per_block * O::SCR) + warp * 64;
  const int64_t ncand = (int64_t)a.n_aux * a.np;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t gwarp = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  int head = 0, tail = 0;
  auto consume = [&](int cnt) {
    const bool act = gw < cnt;
    const int64_t c = ring[(head + (act ? gw : 0)) & 63];
    eri3c_triplet<LC, LA, LB>(a, scr, gl, a.aux_list[c / a.np], a.pairs_orig[c % a.np], act);
    __syncwarp();
    head += cnt;
  };
  for (int64_t b0 = gwarp * 32; b0 < ncand; b0 += nwarps * 32) {
    const int64_t c = b0 + lane;
    bool keep = false;
    if (c < ncand) keep = a.qaux[a.aux_list[c / a.np]] * a.qpair_orig[c % a.np] >= a.tau;
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    if (keep) ring[(tail + __popc(m & ((1u << lane) - 1u))) & 63] = c;
    tail += __popc(m);
    __syncwarp();
    while (tail - head >= W) consume(W);
  }
  if (tail > head) consume(tail - head);
}

// The two-kernel alternative the paper argues against: a screening kernel
// appends every surviving candidate to a global index list (capacity for
// all candidates, since the count is unknown in advance), then a second
// kernel computes the listed triplets.
__global__ void __launch_bounds__(256) k_screen_list(Eri3cArgs a) {
  const int64_t ncand = (int64_t)a.n_aux * a.np;
  const int lane = threadIdx.x & 31;
  for (int64_t b0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) & ~(int64_t)31; b0 < ncand;
       b0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = b0 + lane;
    bool keep = false;
    if (c < ncand) keep = a.qaux[a.aux_list[c / a.np]] * a.qpair_orig[c % a.np] >= a.tau;
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    unsigned long long pos = 0;
    if (lane == 0 && m) pos = atomicAdd(a.count, (unsigned long long)__popc(m));
    pos = __shfl_sync(0xffffffffu, pos, 0);
    if (keep) a.list[pos + __popc(m & ((1u << lane) - 1u))] = c;
  }
}

template <int LC, int LA, int LB>
__global__ void __launch_bounds__(256) k_eri3c_list(Eri3cArgs a) {
  using O = Os<LA, LB, LC, 0>;
  constexpr int G = O::G;
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31;
  const int gl = lane % G;
  const int group_in_block = threadIdx.x / G;
  const int groups_per_block = blockDim.x / G;
  double *scr = smem + (size_t)group_in_block * O::SCR;
  const int64_t total = (int64_t)*a.count;
  const int64_t gstride = (int64_t)gridDim.x * groups_per_block;
  const int warp_first_group = (threadIdx.x >> 5) * (32 / G);
  const int64_t base0 = (int64_t)blockIdx.x * groups_per_block + warp_first_group;
  for (int64_t base = base0; base < total; base += gstride) {
    int64_t t = base + (group_in_block - warp_first_group);
    const bool active = t < total;
    if (!active) t = total - 1;
    const int64_t c = a.list[t];
    eri3c_triplet<LC, LA, LB>(a, scr, gl, a.aux_list[c / a.np], a.pairs_orig[c % a.np], active);
    __syncwarp();
  }
}

// variant 0: sorted prefix (k_eri3c), 1: loop buffer, 2: index list
template <int LC, int LA, int LB>
static int launch3v(const Eri3cArgs &a, int64_t total, int variant, cudaStream_t s) {
  using O = Os<LA, LB, LC, 0>;
  constexpr int G = O::G;
  int groups = 256 / G;
  while (groups > 32 / G && (size_t)groups * O::SCR * 8 + 8 * 64 * 8 > 196 * 1024)
    groups -= 32 / G;
  const size_t smem = (size_t)groups * O::SCR * 8 + (variant == 1 ? (size_t)(groups * G / 32) * 512 : 0);
  if (smem > 227 * 1024) return BQC_E_UNSUPPORTED;
  const int64_t cap = (int64_t)sm_count() * 16;
  if (variant == 1) {
    auto kern = k_eri3c_ring<LC, LA, LB>;
    BQC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
    const int64_t ncand = (int64_t)a.n_aux * a.np;
    const int warps = groups * G / 32;
    int64_t blocks = (ncand + 32 * warps - 1) / (32 * warps);
    blocks = std::max<int64_t>(1, std::min<int64_t>(blocks, cap));
    kern<<<(unsigned)blocks, groups * G, smem, s>>>(a);
  } else {
    auto kern = k_eri3c_list<LC, LA, LB>;
    BQC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
    const int64_t ncand = (int64_t)a.n_aux * a.np;
    int64_t sb = std::max<int64_t>(1, std::min<int64_t>((ncand + 255) / 256, cap));
    BQC_CUDA_TRY(cudaMemsetAsync(a.count, 0, sizeof(unsigned long long), s));
    k_screen_list<<<(unsigned)sb, 256, 0, s>>>(a);
    BQC_LAUNCH_CHECK();
    // the survivor count stays on the device: size the grid for all candidates
    int64_t blocks = (ncand + groups - 1) / groups;
    blocks = std::max<int64_t>(1, std::min<int64_t>(blocks, cap));
    kern<<<(unsigned)blocks, groups * G, smem, s>>>(a);
  }
  (void)total;
  BQC_LAUNCH_CHECK();
  return BQC_OK;
}

template <int LC>
static int dispatch3v_pair(int cls, const Eri3cArgs &a, int64_t total, int v, cudaStream_t s) {
  switch (cls) {
    case 0: return launch3v<LC, 0, 0>(a, total, v, s);
    case 1: return launch3v<LC, 1, 0>(a, total, v, s);
    case 2: return launch3v<LC, 1, 1>(a, total, v, s);
    case 3: return launch3v<LC, 2, 0>(a, total, v, s);
    case 4: return launch3v<LC, 2, 1>(a, total, v, s);
    case 5: return launch3v<LC, 2, 2>(a, total, v, s);
  }
  return BQC_E_UNSUPPORTED;
}

int dispatch3v(int lc, int cls, const Eri3cArgs &a, int64_t total, int v, cudaStream_t s) {
  BQC_TRY(upload_cart_tables());
  switch (lc) {
    case 0: return dispatch3v_pair<0>(cls, a, total, v, s);
    case 1: return dispatch3v_pair<1>(cls, a, total, v, s);
    case 2: return dispatch3v_pair<2>(cls, a, total, v, s);
    case 3: return dispatch3v_pair<3>(cls, a, total, v, s);
  }
  return BQC_E_UNSUPPORTED;
}

}  // namespace bqc
