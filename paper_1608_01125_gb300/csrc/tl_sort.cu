// tl_sort.cu -- stable LSD radix sort of (64-bit key, 32-bit value) pairs.
//
// 8-bit digits.  The key kernel counts every digit of every pass while it
// writes the keys; one scan turns the counts into digit offsets; then one
// kernel per digit pass ranks a 2048-key tile in shared memory
// (warp match-any ranking keeps the order of equal digits), obtains the
// tile's global offsets by decoupled look-back over the preceding tiles'
// published digit counts (Merrill & Garland 2016, "Single-pass parallel
// prefix scan with decoupled look-back"; as used by one-sweep radix sorting,
// Adinets & Merrill 2022), and writes the tile out digit by digit.
// Tiles are numbered in the order blocks start (an atomic counter), so a
// tile only ever waits on tiles whose blocks are already running.  Every wait
// is bounded by spin_limit; on expiry the tile records TL_ST_TIMEOUT and
// proceeds (the result is then invalid, and the host reports the error).
//
// Status words: 2 flag bits (aggregate / inclusive prefix published), a
// 3-bit pass epoch and a 27-bit count (beams hold fewer than 2^27 photons).
// Every pass rewrites every tile's 256 words, so a word left by the previous
// pass carries the previous epoch and reads as "not published": the array
// needs no clearing between passes.  The epochs live on the device (the scan
// picks them), so a captured graph's replays cycle them too.
#include "tl_common.cuh"

namespace tl {

constexpr int kSortThreads = 256;
constexpr int kSortItems = TL_SORT_TILE / kSortThreads;
constexpr int kSortTile = TL_SORT_TILE;
constexpr int kRadix = 256;
constexpr uint32_t kAgg = 1u << 30;     // tile aggregate published
constexpr uint32_t kPre = 2u << 30;     // inclusive prefix published
constexpr uint32_t kFlagMask = 3u << 30;
constexpr int kEpochShift = 27;
constexpr uint32_t kEpochMask = 7u << kEpochShift;
constexpr uint32_t kValMask = (1u << kEpochShift) - 1u;
constexpr int kLookback = 8;  // preceding tiles' words read per look-back round trip

// exclusive scan of each pass's 256 digit counts (raw, counted by the key
// kernel) into hist (one block of 256); then clears the raw counts and the
// tile counters for the next sort.  Also picks the passes' epochs: ep[8] is
// the last epoch used, ep[p] that of pass p (1..7, cycling), so that a
// replayed graph moves on as eager launches do.
__global__ void k_sort_scan(uint32_t *raw, uint32_t *hist, uint32_t *tile_ctr, uint32_t *ep,
                            int passes) {
  __shared__ uint32_t s[kRadix];
  if (threadIdx.x < 8) tile_ctr[threadIdx.x] = 0u;
  if (threadIdx.x == 0) {
    uint32_t e = ep[8];
    for (int p = 0; p < passes; ++p) {
      e = e % 7u + 1u;
      ep[p] = e;
    }
    ep[8] = e;
  }
  for (int p = 0; p < passes; ++p) {
    uint32_t v = raw[p * kRadix + threadIdx.x];
    raw[p * kRadix + threadIdx.x] = 0u;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < kRadix; off <<= 1) {
      uint32_t t = threadIdx.x >= off ? s[threadIdx.x - off] : 0u;
      __syncthreads();
      s[threadIdx.x] += t;
      __syncthreads();
    }
    hist[p * kRadix + threadIdx.x] = s[threadIdx.x] - v;
    __syncthreads();
  }
}

struct SortSmem {
  unsigned long long keys[kSortTile];
  uint32_t vals[kSortTile];
  uint32_t wcnt[8][kRadix];  // per-warp digit counts, then per-warp offsets
  uint32_t dexcl[kRadix];    // tile-local exclusive digit offsets
  uint32_t gbase[kRadix];    // global destination of each digit's first key
  uint32_t scan[kRadix];
  uint32_t tile;
};

__global__ void __launch_bounds__(256, 4) k_sort_pass(
    const unsigned long long *__restrict__ kin, const uint32_t *__restrict__ vin,
    unsigned long long *__restrict__ kout, uint32_t *__restrict__ vout, int64_t n, int shift,
    const uint32_t *__restrict__ digit_base, uint32_t *status, uint32_t *tile_ctr,
    const uint32_t *epoch_p, long long spin_limit, int debug_stall, unsigned int *st_flags,
    const float4 *__restrict__ pos_u, const float4 *__restrict__ dir_u, float4 *__restrict__ pos,
    float4 *__restrict__ dir) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SortSmem &sm = *reinterpret_cast<SortSmem *>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) sm.tile = atomicAdd(tile_ctr, 1u);
  for (int i = tid; i < 8 * kRadix; i += kSortThreads) (&sm.wcnt[0][0])[i] = 0;
  __syncthreads();
  const uint32_t tile = sm.tile;
  const int64_t base = (int64_t)tile * kSortTile;
  const unsigned lt = (1u << lane) - 1u;

  unsigned long long k[kSortItems];
  uint32_t v[kSortItems];
  uint32_t rank[kSortItems];
  uint32_t dig[kSortItems];
#pragma unroll
  for (int it = 0; it < kSortItems; ++it) {
    const int64_t idx = base + warp * (32 * kSortItems) + it * 32 + lane;
    const bool valid = idx < n;
    k[it] = valid ? kin[idx] : 0ull;
    v[it] = valid ? vin[idx] : 0u;
    dig[it] = valid ? (uint32_t)((k[it] >> shift) & 255u) : 256u;
  }
#pragma unroll
  for (int it = 0; it < kSortItems; ++it) {
    const unsigned peers = __match_any_sync(0xffffffffu, dig[it]);
    uint32_t before = 0;
    if (dig[it] < 256u) before = sm.wcnt[warp][dig[it]];
    __syncwarp();
    if (dig[it] < 256u && lane == __ffs(peers) - 1) sm.wcnt[warp][dig[it]] = before + __popc(peers);
    rank[it] = before + __popc(peers & lt);
    __syncwarp();
  }
  __syncthreads();
  // per-digit exclusive offsets across warps; tile total per digit
  uint32_t cnt;
  {
    const int d = tid;
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      uint32_t t = sm.wcnt[w][d];
      sm.wcnt[w][d] = run;
      run += t;
    }
    cnt = run;
    // publish the tile aggregate, then look back over preceding tiles
    uint32_t *my = status + (int64_t)tile * kRadix + d;
    const uint32_t ep = *epoch_p << kEpochShift;
    uint32_t excl = 0;
    if (tile == 0) {
      if (!debug_stall) atomicExch(my, kPre | ep | cnt);
    } else {
      atomicExch(my, kAgg | ep | cnt);
      // walk back over the preceding tiles kLookback at a time (independent loads),
      // adding published aggregates until an inclusive prefix is found
      int64_t j = (int64_t)tile - 1;
      long long spins = 0;
      bool done = false;
      while (j >= 0 && !done) {
        uint32_t sv[kLookback];
#pragma unroll
        for (int q = 0; q < kLookback; ++q)
          sv[q] = j - q >= 0 ? *(volatile uint32_t *)(status + (j - q) * kRadix + d) : (kPre | ep);
        int used = 0;
        for (int q = 0; q < kLookback && !done; ++q) {
          const uint32_t flag = sv[q] & kFlagMask;
          // not published in this pass yet: reload from here
          if (flag == 0u || (sv[q] & kEpochMask) != ep) break;
          if (j - q >= 0) excl += sv[q] & kValMask;
          ++used;
          if (flag == kPre) done = true;
        }
        j -= used;
        if (!done && used == 0) {
          if (++spins > spin_limit) {
            atomicOr(st_flags, (unsigned)TL_ST_TIMEOUT);
            break;
          }
          __nanosleep(32);
        }
      }
      atomicExch(my, kPre | ep | ((excl + cnt) & kValMask));
    }
    sm.gbase[d] = digit_base[d] + excl;
    sm.scan[d] = cnt;
  }
  __syncthreads();
  // tile-local exclusive scan over digits (Hillis-Steele in shared memory)
  for (int off = 1; off < kRadix; off <<= 1) {
    uint32_t t = tid >= off ? sm.scan[tid - off] : 0u;
    __syncthreads();
    sm.scan[tid] += t;
    __syncthreads();
  }
  sm.dexcl[tid] = sm.scan[tid] - cnt;
  __syncthreads();
#pragma unroll
  for (int it = 0; it < kSortItems; ++it) {
    if (dig[it] < 256u) {
      const uint32_t pos = sm.dexcl[dig[it]] + sm.wcnt[warp][dig[it]] + rank[it];
      sm.keys[pos] = k[it];
      sm.vals[pos] = v[it];
    }
  }
  __syncthreads();
  const int64_t rem = n - base;
  const int tcount = rem < kSortTile ? (int)rem : kSortTile;
  for (int j = tid; j < tcount; j += kSortThreads) {
    const unsigned long long kk = sm.keys[j];
    const uint32_t d = (uint32_t)((kk >> shift) & 255u);
    const uint32_t g = sm.gbase[d] + (uint32_t)j - sm.dexcl[d];
    if ((int64_t)g < n) {  // always true unless a wait expired (then the result is discarded)
      kout[g] = kk;
      if (pos) {  // last pass: gather the photon itself into Morton order
        const uint32_t src = sm.vals[j];
        pos[g] = pos_u[src];
        dir[g] = dir_u[src];
      } else {
        vout[g] = sm.vals[j];
      }
    }
  }
}

// Kernel attributes of the sort (before any launch or stream capture).
cudaError_t sort_prepare() {
  return cudaFuncSetAttribute(k_sort_pass, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sizeof(SortSmem));
}

// Sort w.key[0]/w.val[0] by the low key_bits bits and gather the SoA into
// w.pos / w.dir in the sorted order (the last pass does it).  *out_sel
// receives the buffer index holding the sorted keys.  The key kernel has
// counted every pass's digits into w.sort_raw (which the scan clears again, as
// it does the tile counters; both are zero when allocated).  n <= 1: nothing
// is sorted or gathered.
cudaError_t launch_sort(BuildBufs &w, int64_t n, int key_bits, long long spin_limit,
                        int debug_stall, unsigned int *status, int *out_sel, cudaStream_t s) {
  *out_sel = 0;
  if (n <= 1) return cudaSuccess;
  const int passes = (key_bits + 7) / 8;
  const int64_t tiles = (n + kSortTile - 1) / kSortTile;
  cudaError_t e;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if ((e = cudaStreamIsCapturing(s, &cap))) return e;
  const bool capturing = cap != cudaStreamCaptureStatusNone;
  if (w.sort_epoch == 0) {  // fresh buffers, or a wait expired: clear the words once
    if ((e = cudaMemsetAsync(w.sort_status, 0, sizeof(uint32_t) * kRadix * tiles, s))) return e;
    if ((e = cudaMemsetAsync(w.sort_ep, 0, sizeof(uint32_t) * 9, s))) return e;
    if (!capturing) w.sort_epoch = 1;
  }
  k_sort_scan<<<1, kRadix, 0, s>>>(w.sort_raw, w.sort_hist, w.sort_tile, w.sort_ep, passes);
  int sel = 0;
  for (int p = 0; p < passes; ++p) {
    const bool last = p == passes - 1;
    k_sort_pass<<<(unsigned)tiles, kSortThreads, sizeof(SortSmem), s>>>(
        w.key[sel], w.val[sel], w.key[sel ^ 1], w.val[sel ^ 1], n, 8 * p, w.sort_hist + p * kRadix,
        w.sort_status, w.sort_tile + p, w.sort_ep + p, spin_limit, debug_stall && p == 0, status,
        last ? w.pos_u : nullptr, last ? w.dir_u : nullptr, last ? w.pos : nullptr,
        last ? w.dir : nullptr);
    if ((e = cudaGetLastError())) return e;
    sel ^= 1;
  }
  *out_sel = sel;
  return cudaSuccess;
}

}  // namespace tl
