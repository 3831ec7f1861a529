// tl_noalloc.cu -- the yield reduction for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc: code running inside another
// framework's memory pool or under a strict memory budget, or a host
// process that must not change the device's allocation state while a
// simulation it does not own is running.  They can still pass their own
// input and output buffers.  This entry point reduces a hit list to
// (count, sum of w_i w_j, checksums) -- the same quantities the yield
// reduction of trilens_collide_step produces -- using as scratch a
// file-scope device array instead of allocated workspace.
//
// Scratch: one 32-byte partial per chunk of 65536 hits, for at most 4096
// chunks (128 KiB), plus a completion counter.  Every GPU that loads the
// library holds this array until the process exits.  Every call shares it:
// calls that overlap on the GPU race with each other.  The completion
// counter is cleared at the start of every call.
#include <stdint.h>

#include <mutex>

#include "tl_yield.cuh"
#include "trilens.h"

namespace {

using tl::YieldPartial;

constexpr int kChunk = 65536;
constexpr int kMaxChunks = 4096;
constexpr int kThreads = 256;
static_assert((long long)kMaxChunks * kChunk == TRILENS_NOALLOC_MAX_HITS,
              "the scratch array must hold one partial per chunk of the largest list");

struct NaScratch {
  YieldPartial part[kMaxChunks];
  unsigned int done;
};

static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NaScratch)];

// One block per chunk of hits; the last block to finish adds the chunk
// partials in a fixed order (strided over its threads, then the block's
// fixed-order reduction) and writes the result.
__global__ void __launch_bounds__(kThreads) k_yield_noalloc(NaScratch *sc, const uint2 *hits,
                                                            int64_t n, const double *wA,
                                                            const double *wB, YieldPartial *out) {
  __shared__ YieldPartial sp[kThreads / 32];
  __shared__ bool last;
  const int64_t lo = (int64_t)blockIdx.x * kChunk;
  const int64_t hi = lo + kChunk < n ? lo + kChunk : n;
  YieldPartial p = tl::yield_zero();
  for (int64_t i = lo + threadIdx.x; i < hi; i += kThreads) {
    const uint2 h = hits[i];
    tl::yield_hit(p, h.x, h.y, wA ? wA[h.x] : 1.0, wB ? wB[h.y] : 1.0);
  }
  const YieldPartial b = tl::yield_block_reduce(p, sp);
  if (threadIdx.x == 0) {
    sc->part[blockIdx.x] = b;
    __threadfence();
    last = atomicAdd(&sc->done, 1u) == gridDim.x - 1u;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  YieldPartial t = tl::yield_zero();
  for (unsigned q = threadIdx.x; q < gridDim.x; q += kThreads)
    tl::yield_add(t, tl::yield_load_volatile(sc->part + q));
  const YieldPartial tot = tl::yield_block_reduce(t, sp);
  if (threadIdx.x == 0) *out = tot;
}

// Device address of the scratch array, looked up once per device with that
// device current.
std::mutex g_mu;
NaScratch *g_addr[64] = {nullptr};

cudaError_t scratch_for_current_device(NaScratch **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = reinterpret_cast<NaScratch *>(p);
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int trilens_yield_reduce_noalloc(const uint32_t *hits, int64_t n_hits,
                                            const double *w_a, const double *w_b,
                                            void *out_result, trilens_stream_t stream) {
  if (n_hits < 0 || n_hits > (int64_t)TRILENS_NOALLOC_MAX_HITS) return TRILENS_ERR_INVALID;
  if (!out_result || (n_hits > 0 && !hits)) return TRILENS_ERR_INVALID;
  // the kernel reads hits as 8-byte pairs and writes one 32-byte result of
  // 8-byte fields: a misaligned pointer would fault in the caller's context
  if (((uintptr_t)hits & 7u) || ((uintptr_t)out_result & 7u)) return TRILENS_ERR_INVALID;
  NaScratch *sc = nullptr;
  if (scratch_for_current_device(&sc) != cudaSuccess) return TRILENS_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  // the completion counter must start at zero; the partials are overwritten
  if (cudaMemsetAsync(&sc->done, 0, sizeof(unsigned int), s) != cudaSuccess) return TRILENS_ERR_CUDA;
  const int64_t blocks = n_hits > 0 ? (n_hits + kChunk - 1) / kChunk : 1;
  k_yield_noalloc<<<(unsigned)blocks, kThreads, 0, s>>>(
      sc, reinterpret_cast<const uint2 *>(hits), n_hits, w_a, w_b,
      reinterpret_cast<YieldPartial *>(out_result));
  return cudaGetLastError() == cudaSuccess ? TRILENS_OK : TRILENS_ERR_CUDA;
}
