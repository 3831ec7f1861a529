// tl_traverse.cu -- dual-hierarchy traversal, narrow phase, FP64 band
// re-test and the per-step yield reduction.
//
// The two hierarchies are traversed against each other (Sec. 2.2: depth-first
// descent; a failed overlap test, Eq. CollDet, skips the whole subtree pair).
// The frontier of node pairs comes from the refit's seed lists (large beams:
// every overlapping pair of cut nodes) or from a few breadth-first expansion
// levels of the root pair; then persistent warps take frontier pairs and
// descend depth first with a stack of node pairs in shared memory, handing
// large items on to a device work queue (see k_traverse).  Each
// iteration a warp pops up to 32 pairs, one per lane; a lane loads both
// node records of its pair once and tests the up-to-4 child combinations
// (both children of each side); survivors are pushed (or, when both sides
// are leaf buckets, appended to the step's leaf-pair list in blocks of at
// least 32) with ballot/popc compaction.  A separate kernel (k_narrow) then
// flattens the listed bucket pairs over its warps' lanes, one photon pair
// per lane, and gives them the narrow-phase test; hits leave with one atomic
// per warp.  Splitting the two keeps each kernel's registers low and its
// warps many, which hides the latency both are bound by.
#include "tl_common.cuh"
#include "tl_exact.cuh"
#include "tl_narrow.cuh"
#include "tl_yield.cuh"

namespace tl {


// One side of a child pair: the child `slot` of an inner node, or a bucket
// itself (slot ignored) when ref names a bucket.
struct Side {
  TLBox box;
  uint32_t sref;   // stack reference of this child
  uint32_t first;  // first photon (buckets)
  uint32_t cnt;    // photons under it
  bool bucket;
};

__device__ __forceinline__ Side side_of(const TLTree &T, uint32_t ref, int slot) {
  Side s;
  uint32_t node, sl;
  if (!(ref & TL_FLAG)) {
    node = ref;
    sl = (uint32_t)slot;
  } else {
    node = (ref & ~TL_FLAG) >> 1;
    sl = ref & 1u;
  }
  const TLNode *nd = T.nodes + node;
  const float4 *f = reinterpret_cast<const float4 *>(nd);
  TLNode v;
  v.b0 = __ldg(f + 0);
  v.b1 = __ldg(f + 1);
  v.b2 = __ldg(f + 2);
  v.c = __ldg(reinterpret_cast<const int4 *>(f + 3));
  s.box = tl_child_box(v, (int)sl);
  const uint32_t cr = (uint32_t)(sl ? v.c.y : v.c.x);
  s.cnt = (uint32_t)(sl ? v.c.w : v.c.z);
  s.bucket = (cr & TL_FLAG) != 0u;
  s.first = cr & ~TL_FLAG;
  if (ref & TL_FLAG) s.sref = ref;
  else s.sref = s.bucket ? (TL_FLAG | (node << 1) | sl) : cr;
  return s;
}

__device__ __forceinline__ uint32_t pack_bucket(uint32_t first, uint32_t cnt) {
  return first | ((cnt - 1u) << 27);
}

// For a pair (ra, rb) and a combination index 0..3, the child pair it names.
// Returns false if the combination does not exist for this pair.
__device__ __forceinline__ bool child_pair(const TLTree &A, const TLTree &B, uint2 pr, int combo,
                                           Side &sa, Side &sb) {
  const bool ain = !(pr.x & TL_FLAG), bin = !(pr.y & TL_FLAG);
  int ia, ib;
  if (ain && bin) {
    ia = combo >> 1;
    ib = combo & 1;
  } else if (ain) {
    if (combo >= 2) return false;
    ia = combo;
    ib = 0;
  } else if (bin) {
    if (combo >= 2) return false;
    ia = 0;
    ib = combo;
  } else {
    return false;
  }
  sa = side_of(A, pr.x, ia);
  sb = side_of(B, pr.y, ib);
  return true;
}

// Child i (0 or 1) of one side of a popped pair, from the side's node record
// rec: for an inner node (ref without FLAG) its child i; for a bucket (ref =
// FLAG | parent << 1 | slot, rec = the parent's record) the bucket itself
// (i = 0 only).
struct Kid {
  TLBox box;
  uint32_t sref;  // stack reference
  uint32_t pack;  // bucket as (first photon | (count - 1) << 27)
  bool bucket;
};

__device__ __forceinline__ Kid kid_of(const TLNode &rec, uint32_t ref, int i) {
  Kid k;
  uint32_t node, sl;
  if (ref & TL_FLAG) {
    node = (ref & ~TL_FLAG) >> 1;
    sl = ref & 1u;
  } else {
    node = ref;
    sl = (uint32_t)i;
  }
  k.box = tl_child_box(rec, (int)sl);
  const uint32_t cr = (uint32_t)(sl ? rec.c.y : rec.c.x);
  const uint32_t cnt = (uint32_t)(sl ? rec.c.w : rec.c.z);
  k.bucket = (cr & TL_FLAG) != 0u;
  k.pack = pack_bucket(cr & ~TL_FLAG, cnt);
  k.sref = (ref & TL_FLAG) ? ref : (k.bucket ? (TL_FLAG | (node << 1) | sl) : cr);
  return k;
}

__device__ __forceinline__ TLNode node_record(const TLTree &T, uint32_t ref) {
  const uint32_t node = (ref & TL_FLAG) ? ((ref & ~TL_FLAG) >> 1) : ref;
  const float4 *f = reinterpret_cast<const float4 *>(T.nodes + node);
  TLNode v;
  v.b0 = __ldg(f + 0);
  v.b1 = __ldg(f + 1);
  v.b2 = __ldg(f + 2);
  v.c = __ldg(reinterpret_cast<const int4 *>(f + 3));
  return v;
}

// warp-aggregated append of (x, y) for lanes with pred
__device__ __forceinline__ void emit(bool pred, uint32_t x, uint32_t y, uint2 *buf,
                                     unsigned long long cap, unsigned long long *counter,
                                     unsigned *status, unsigned ovf_bit, int lane) {
  const unsigned m = __ballot_sync(0xffffffffu, pred);
  if (!m) return;
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(counter, (unsigned long long)__popc(m));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (pred) {
    const unsigned long long idx = base + __popc(m & ((1u << lane) - 1u));
    if (idx < cap) buf[idx] = make_uint2(x, y);
  }
  if (lane == 0 && base + __popc(m) > cap) atomicOr(status, ovf_bit);
}

// ------------------------------------------------------------ init

// run_status (captured runs, else NULL): a queue overflow or an expired wait
// in an earlier step of the run carries over, so that no later step runs on
// a queue that may still hold chunks nobody takes (the host repeats the run)
__global__ void k_step_init(TLCounters *ctr, uint2 *F0, uint32_t superA, uint32_t superB,
                            int nonempty, const unsigned *build_status,
                            const unsigned *run_status) {
  unsigned *w = reinterpret_cast<unsigned *>(ctr);
  for (int i = threadIdx.x; i < (int)(sizeof(TLCounters) / 4); i += blockDim.x) w[i] = 0u;
  if (threadIdx.x == 0) F0[0] = make_uint2(superA, superB);
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned bs = *build_status & (unsigned)TL_ST_TIMEOUT;
    const unsigned rs =
        run_status ? *run_status & (unsigned)(TL_ST_SPILL_OVF | TL_ST_TIMEOUT) : 0u;
    ctr->status = bs | rs;
    // after a failed build there is nothing valid to traverse
    ctr->counts[0] = (nonempty && !bs && !rs) ? 1u : 0u;
  }
}

// Several instances: the frontier starts from each instance's pair of
// subtree roots, so no pair of photons from different instances is tested.
__global__ void k_seed_instances(TLCounters *ctr, uint2 *F0, const uint32_t *rootA,
                                 const uint32_t *rootB, int n_inst) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n_inst || (ctr->status & (TL_ST_TIMEOUT | TL_ST_SPILL_OVF))) return;
  const uint32_t ra = rootA[q], rb = rootB[q];
  if (ra == TL_NONE || rb == TL_NONE) return;
  const unsigned idx = atomicAdd(&ctr->counts[0], 1u);
  F0[idx] = make_uint2(ra, rb);
}

// ------------------------------------------------------------ frontier

// Seeds from the two cut lists written by the refit: every pair (cut node of
// A, cut node of B) whose boxes overlap (Eq. CollDet).  Every photon lies in
// exactly one cut node of its beam and a box contains its descendants' boxes,
// so every overlapping pair of leaf buckets lies below exactly one seed: the
// traversal from the seeds reaches the same leaf pairs as from the roots.
__global__ void __launch_bounds__(256) k_seed_cut(TravArgs a, const uint32_t *cutA,
                                                  const unsigned *cntA, uint32_t capA,
                                                  const uint32_t *cutB, const unsigned *cntB,
                                                  uint32_t capB, uint2 *F0, unsigned cap) {
  TLCounters *ctr = a.ctr;
  // the build failed, or the queue overflowed earlier in a captured run: nothing to traverse
  if (ctr->status & (TL_ST_TIMEOUT | TL_ST_SPILL_OVF)) return;
  const unsigned na = *cntA, nb = *cntB;
  if (na > capA || nb > capB) {  // a list overflowed: start from the root pair
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      F0[0] = make_uint2(a.A.super, a.B.super);
      ctr->counts[0] = 1u;
    }
    return;
  }
  const unsigned long long total = (unsigned long long)na * nb;
  const unsigned long long rounded = (total + 31ull) & ~31ull;
  const int lane = threadIdx.x & 31;
  unsigned long long tests = 0;
  for (unsigned long long q = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
       q < rounded; q += (unsigned long long)gridDim.x * blockDim.x) {
    bool ok = false;
    uint2 o = make_uint2(0u, 0u);
    if (q < total) {
      const uint32_t ea = cutA[q / nb], eb = cutB[q % nb];
      const Side sa = side_of(a.A, ea >> 1, (int)(ea & 1u));
      const Side sb = side_of(a.B, eb >> 1, (int)(eb & 1u));
      ++tests;
      ok = tl_overlap(sa.box, sb.box);
      o = make_uint2(sa.sref, sb.sref);
    }
    const unsigned m = __ballot_sync(0xffffffffu, ok);
    if (m) {
      unsigned base = 0;
      if (lane == 0) base = atomicAdd(&ctr->counts[0], (unsigned)__popc(m));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (ok) {
        const unsigned idx = base + __popc(m & ((1u << lane) - 1u));
        if (idx < cap) F0[idx] = o;
        else atomicOr(&ctr->status, (unsigned)TL_ST_FRONT_OVF);
      }
    }
  }
  for (int off = 16; off; off >>= 1) tests += __shfl_xor_sync(0xffffffffu, tests, off);
  if (lane == 0 && tests) atomicAdd(&ctr->node_tests, tests);
}

// One block expands the root pair breadth first, level by level, until the
// frontier holds at least `target` pairs (or nothing is left to expand).
// Bucket pairs pass through unchanged; failed overlap tests prune.
__global__ void __launch_bounds__(1024) k_expand(TravArgs a, uint2 *F0, uint2 *F1, unsigned cap,
                                                 unsigned target, int max_levels) {
  __shared__ unsigned s_count[2];
  __shared__ unsigned long long s_tests;
  TLCounters *ctr = a.ctr;
  if (threadIdx.x == 0) {
    s_count[0] = ctr->counts[0];
    s_count[1] = 0u;
    s_tests = 0ull;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  unsigned long long tests = 0;
  int level = 0;
  while (true) {
    const unsigned nin = s_count[level & 1];
    if (nin >= target || nin == 0u || level >= max_levels) break;
    const uint2 *in = (level & 1) ? F1 : F0;
    uint2 *out = (level & 1) ? F0 : F1;
    unsigned *ocount = &s_count[(level + 1) & 1];
    const unsigned nround = (nin + 31u) & ~31u;
    for (unsigned i = threadIdx.x; i < nround; i += blockDim.x) {
      const bool valid = i < nin;
      const uint2 pr = valid ? in[i] : make_uint2(0u, 0u);
      const bool both_buckets = valid && (pr.x & TL_FLAG) && (pr.y & TL_FLAG);
      for (int combo = 0; combo < 4; ++combo) {
        Side sa, sb;
        bool ok = false;
        uint2 o = make_uint2(0u, 0u);
        if (valid && !both_buckets && child_pair(a.A, a.B, pr, combo, sa, sb)) {
          ++tests;
          ok = tl_overlap(sa.box, sb.box);
          o = make_uint2(sa.sref, sb.sref);
        } else if (both_buckets && combo == 0) {
          ok = true;  // already tested when it was produced: pass through
          o = pr;
        }
        const unsigned m = __ballot_sync(0xffffffffu, ok);
        if (m) {
          unsigned base = 0;
          if (lane == 0) base = atomicAdd(ocount, (unsigned)__popc(m));
          base = __shfl_sync(0xffffffffu, base, 0);
          if (ok) {
            const unsigned idx = base + __popc(m & ((1u << lane) - 1u));
            if (idx < cap) out[idx] = o;
            else atomicOr(&ctr->status, (unsigned)TL_ST_FRONT_OVF);
          }
        }
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) s_count[level & 1] = 0u;  // the next level's output count
    ++level;
    __syncthreads();
  }
  for (int off = 16; off; off >>= 1) tests += __shfl_xor_sync(0xffffffffu, tests, off);
  if (lane == 0 && tests) atomicAdd(&s_tests, tests);
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned n = s_count[level & 1];
    ctr->counts[level] = n < cap ? n : cap;
    ctr->final_level = (unsigned)level;
    ctr->frozen = 1u;
    ctr->node_tests += s_tests;
  }
}

// One breadth-first level of the frontier across the whole grid.  Launched
// for a fixed number of levels after the seeds; level `level` acts only if it
// is the frontier's current level and that frontier has fewer than `target`
// pairs (and its children cannot overflow the buffer, at most 4 per pair):
// every pair is replaced by its overlapping child pairs (Eq. CollDet; bucket
// pairs pass through) and the last block to finish moves the frontier on to
// level + 1.  The decision reads values earlier launches wrote, so every
// block takes the same one.  A wide frontier gives every traversal warp
// full 32-pair items from the start.
__global__ void __launch_bounds__(256) k_widen(TravArgs a, uint2 *F0, uint2 *F1, unsigned cap,
                                               unsigned target, int level) {
  TLCounters *ctr = a.ctr;
  // the build failed, or the queue overflowed earlier in a captured run: nothing to traverse
  if (ctr->status & (TL_ST_TIMEOUT | TL_ST_SPILL_OVF)) return;
  if ((int)ctr->final_level != level || level + 1 >= 32) return;
  const unsigned nin = ctr->counts[level];
  if (nin == 0u || nin >= target || 4ull * nin > (unsigned long long)cap) return;
  const uint2 *in = (level & 1) ? F1 : F0;
  uint2 *out = (level & 1) ? F0 : F1;
  unsigned *ocount = &ctr->counts[level + 1];
  const int lane = threadIdx.x & 31;
  unsigned long long tests = 0;
  const unsigned nround = (nin + 31u) & ~31u;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < nround;
       i += gridDim.x * blockDim.x) {
    const bool valid = i < nin;
    const uint2 pr = valid ? in[i] : make_uint2(0u, 0u);
    const bool both_buckets = valid && (pr.x & TL_FLAG) && (pr.y & TL_FLAG);
    for (int combo = 0; combo < 4; ++combo) {
      Side sa, sb;
      bool ok = false;
      uint2 o = make_uint2(0u, 0u);
      if (valid && !both_buckets && child_pair(a.A, a.B, pr, combo, sa, sb)) {
        ++tests;
        ok = tl_overlap(sa.box, sb.box);
        o = make_uint2(sa.sref, sb.sref);
      } else if (both_buckets && combo == 0) {
        ok = true;  // already tested when it was produced: pass through
        o = pr;
      }
      const unsigned m = __ballot_sync(0xffffffffu, ok);
      if (m) {
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(ocount, (unsigned)__popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (ok) out[base + __popc(m & ((1u << lane) - 1u))] = o;  // < 4 nin <= cap
      }
    }
  }
  for (int off = 16; off; off >>= 1) tests += __shfl_xor_sync(0xffffffffu, tests, off);
  if (lane == 0 && tests) atomicAdd(&ctr->node_tests, tests);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();  // this block's outputs and count before its finish
    if (atomicAdd(&ctr->widen_done, 1u) == gridDim.x - 1u) {
      ctr->widen_done = 0u;
      __threadfence();
      ctr->final_level = (unsigned)(level + 1);
    }
  }
}

// ------------------------------------------------------------ narrow phase

// a warp's leaf-pair queue: fewer than 32 entries before an iteration, at
// most 4 new ones per lane in it
constexpr int kLeafQ = 32 + 4 * 32;

struct WarpSmem {
  uint2 leafq[kLeafQ];
  uint2 pend[64];  // narrow phase: photon pairs the test's prefix left undecided
  int scan[32];
};

// The full FP32 test of up to 32 pending photon pairs (sorted positions in
// ws.pend[0 .. cnt)), one per lane; hits and band pairs leave with one
// atomic per warp each.
__device__ __forceinline__ void decide_pending(const TravArgs &a, const WarpSmem &ws, int cnt,
                                               int lane, const float *sbin) {
  int outcome = TL_MISS;
  uint32_t oi = 0u, oj = 0u;
  if (lane < cnt) {
    const uint2 pr = ws.pend[lane];
    const float4 da = __ldg(a.A.dir + pr.x), db = __ldg(a.B.dir + pr.y);
    const float4 pa = __ldg(a.A.pos + pr.x), pb = __ldg(a.B.pos + pr.y);
    oi = __float_as_uint(da.w);
    oj = __float_as_uint(db.w);
    outcome = tl_narrow32(pa, da, pb, db, a.nk, sbin);
  }
  emit(outcome == TL_HIT, oi, oj, a.hits, a.hit_cap, &a.ctr->hits, &a.ctr->status,
       TL_ST_HIT_OVF, lane);
  emit(outcome == TL_BAND, oi, oj, a.band, a.band_cap, &a.ctr->band, &a.ctr->status,
       TL_ST_BAND_OVF, lane);
}

// The narrow phase of nq leaf pairs in ws.leafq: their photon pairs are
// flattened over the lanes (a scan of the pairs' sizes, then each lane finds
// its pair by binary search).  FP64: each photon pair is decided by the
// definition.  FP32: the test's prefix (threshold, quick miss) runs on every
// photon pair and decides most of them; the undecided ones are queued in
// ws.pend (npend of them, warp-uniform) and given the full test 32 at a time,
// so that the long path runs on full warps.
template <bool FP64>
__device__ __forceinline__ void flush_leaves(const TravArgs &a, WarpSmem &ws, int nq, int lane,
                                             unsigned long long &tests, int &npend,
                                             const float *sbin) {
  const unsigned lt = (1u << lane) - 1u;
  for (int e0 = 0; e0 < nq; e0 += 32) {
    const int m = min(32, nq - e0);
    int sz = 0;
    if (lane < m) {
      const uint2 q = ws.leafq[e0 + lane];
      sz = (int)(((q.x >> 27) + 1u) * ((q.y >> 27) + 1u));
    }
    int inc = sz;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, inc, off);
      if (lane >= off) inc += t;
    }
    const int total = __shfl_sync(0xffffffffu, inc, 31);
    ws.scan[lane] = inc - sz;
    __syncwarp();
    tests += (unsigned long long)total;
    for (int t0 = 0; t0 < total; t0 += 32) {
      const int t = t0 + lane;
      int outcome = TL_MISS;
      bool undecided = false;
      uint32_t oi = 0u, oj = 0u, si = 0u, sj = 0u;
      if (t < total) {
        // largest entry e with scan[e] <= t
        int lo = 0, hi = m - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (ws.scan[mid] <= t) lo = mid;
          else hi = mid - 1;
        }
        const uint2 q = ws.leafq[e0 + lo];
        const uint32_t fa = q.x & 0x7FFFFFFu, fb = q.y & 0x7FFFFFFu;
        const uint32_t cb = (q.y >> 27) + 1u;
        const uint32_t loc = (uint32_t)(t - ws.scan[lo]);
        const uint32_t ia = loc / cb, jb = loc - ia * cb;
        si = fa + ia;
        sj = fb + jb;
        const float4 da = __ldg(a.A.dir + si), db = __ldg(a.B.dir + sj);
        if (FP64) {
          oi = __float_as_uint(da.w);
          oj = __float_as_uint(db.w);
          outcome = tl_exact_hit(a.mA, oi, a.mB, oj, a.ct, a.dt, a.kappa) ? TL_HIT : TL_MISS;
        } else {
          const float4 pa = __ldg(a.A.pos + si), pb = __ldg(a.B.pos + sj);
          undecided = !tl_narrow32_quick_miss(pa, da, pb, db, a.nk, sbin);
        }
      }
      if (FP64) {
        emit(outcome == TL_HIT, oi, oj, a.hits, a.hit_cap, &a.ctr->hits, &a.ctr->status,
             TL_ST_HIT_OVF, lane);
      } else {
        const unsigned mu = __ballot_sync(0xffffffffu, undecided);
        if (undecided) ws.pend[npend + __popc(mu & lt)] = make_uint2(si, sj);
        npend += __popc(mu);
        __syncwarp();
        if (npend >= 32) {
          decide_pending(a, ws, 32, lane, sbin);
          // the rest (fewer than 32) move to the front
          const int rest = npend - 32;
          uint2 v = make_uint2(0u, 0u);
          if (lane < rest) v = ws.pend[32 + lane];
          __syncwarp();
          if (lane < rest) ws.pend[lane] = v;
          __syncwarp();
          npend = rest;
        }
      }
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------ traversal

// Persistent warps share one work queue.  Its items come first from the
// frontier, in groups of up to 32 node pairs (indices below nf), then from
// the queue's chunks of up to 32 node pairs each (256 bytes).  A warp that
// waits for a chunk is counted in ctr->hungry while it waits; a warp that
// has spent `budget` iterations on its item while h > 0 warps wait hands on
// up to h chunks.  A warp's own stack has two
// levels: the top in shared memory (D entries), the bottom in its private
// spill area in global memory.  A warp pops at most P = min(32, D / 8) pairs
// per iteration (so it pushes at most 4P); when the next iteration's pushes
// might not fit its shared stack, the bottom of it (up to D / 2 entries)
// moves to the spill area, and when the shared stack runs dry it is refilled from the
// spill area's top.  So no work leaves a warp except the chunks it hands on
// to waiting warps, taken from the bottom of its spill area first (the
// shallowest pairs it holds), else from the bottom of its shared stack.
// Unused and free entries hold a sentinel.  A writer fills a chunk's entries
// 1..31, fences, then swaps entry 0 in; a taker swaps the sentinel back into
// entry 0 as it reads it (atomic exchange) and waits while it is still free
// and work is in flight.  The traversal ends when the items finished equal
// nf plus the chunks handed on.  Every wait is bounded by spin_limit (then
// TL_ST_TIMEOUT).
constexpr unsigned long long kQFree = 0xffffffffffffffffull;
constexpr int kGroup = 32;  // frontier pairs per item, node pairs per queue chunk

__device__ __forceinline__ unsigned long long pack2(uint2 v) {
  return (unsigned long long)v.x | ((unsigned long long)v.y << 32);
}

// chunks a working warp hands on per waiting warp, at most
#ifndef TL_DONATE_MAX
#define TL_DONATE_MAX 1
#endif

// Launch bounds: at most 8 warps per block and registers for 4 such blocks
// per SM (63 registers, no spills; the narrow phase is a kernel of its own).
#ifndef TL_TRAV_MINBLOCKS
#define TL_TRAV_MINBLOCKS 4
#endif
// A warp's queued leaf pairs to the step's list (one atomic per warp), from
// the current part's start lbase.  The count keeps every leaf pair; pairs
// past the list's end are dropped and the step is flagged (TL_ST_LEAFQ): the
// host grows the list, or splits the step into more parts, and repeats it.
__device__ __forceinline__ void spill_leaves(const TravArgs &a, const WarpSmem &ws, int nq,
                                             int lane, unsigned long long lbase) {
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(&a.ctr->leaf_pairs, (unsigned long long)nq) - lbase;
  base = __shfl_sync(0xffffffffu, base, 0);
  for (int e = lane; e < nq; e += 32)
    if (base + e < a.leaf_cap) a.leaves[base + e] = ws.leafq[e];
  if (lane == 0 && base + nq > a.leaf_cap) atomicOr(&a.ctr->status, (unsigned)TL_ST_LEAFQ);
}

__global__ void __launch_bounds__(TL_TRAV_MAX_WARPS * 32, TL_TRAV_MINBLOCKS) k_traverse(
    TravArgs a, const uint2 *F0, const uint2 *F1, const uint2 *list, unsigned long long list_n,
    int from_frontier, int budget, int part, int nparts) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int D = a.stack_depth;
  uint2 *stack = reinterpret_cast<uint2 *>(smem_raw) + (size_t)warp * D;
  WarpSmem &ws = reinterpret_cast<WarpSmem *>(
      smem_raw + sizeof(uint2) * (size_t)D * (blockDim.x >> 5))[warp];
  TLCounters *ctr = a.ctr;
  // After a queue overflow or an expired wait in this step (an earlier part)
  // or this run, the queue may hold chunks that no warp will take: a warp
  // taking one would count an item the counters never handed on, and the
  // step's end would no longer be seen.  The host repeats the step (or run)
  // with the queue reset, so nothing more is traversed here.
  if (*(volatile unsigned *)&ctr->status & (TL_ST_SPILL_OVF | TL_ST_TIMEOUT)) return;
  const uint2 *src0;
  unsigned long long n0;
  if (from_frontier) {
    const unsigned lvl = ctr->final_level;
    src0 = (lvl & 1u) ? F1 : F0;
    n0 = ctr->counts[lvl];
  } else {
    src0 = list;
    n0 = list_n;
  }
  {  // this launch's part of the frontier: every leaf pair lies below exactly
     // one frontier pair, so the parts split the step's work
    const unsigned long long lo = n0 * (unsigned long long)part / (unsigned long long)nparts;
    const unsigned long long hi = n0 * (unsigned long long)(part + 1) / (unsigned long long)nparts;
    src0 += lo;
    n0 = hi - lo;
  }
  const unsigned long long lbase = ctr->leaf_base;  // the list of this part starts here
  const unsigned long long nf = (n0 + kGroup - 1) / kGroup;  // frontier groups
  unsigned long long *Q = a.queue;
  const unsigned long long qcap = a.queue_cap / kGroup;  // chunks
  const unsigned lt = (1u << lane) - 1u;
  // the private spill area: entries [gbot, gtop) hold the stack's bottom
  uint2 *gs = a.spill + (size_t)(blockIdx.x * (blockDim.x >> 5) + warp) * a.spill_per_warp;
  const int W = (int)a.spill_per_warp;
  const int P = min(32, D >> 3);  // pops per iteration at most
  int gbot = 0, gtop = 0;
  int sp = 0, nq = 0, iters = 0;
  bool holding = false;  // this warp holds an item (counted in flight)
  bool handed = false;   // ... and has handed pieces of it on
  unsigned long long node_tests = 0;
  while (true) {
    // the bottom of a shared stack that could not take the next iteration's
    // pushes (min(sp, P) pops, 4 pushes each) moves to the spill area
    if (sp + 3 * min(sp, P) > D) {
      const int m = min(D >> 1, sp - P);
      if (gbot > 0 && gtop + m > W) {  // compact the spill area first
        const int cnt = gtop - gbot;
        for (int e0 = 0; e0 < cnt; e0 += 32) {
          uint2 v = make_uint2(0u, 0u);
          if (e0 + lane < cnt) v = gs[gbot + e0 + lane];
          __syncwarp();
          if (e0 + lane < cnt) gs[e0 + lane] = v;
          __syncwarp();
        }
        gtop = cnt;
        gbot = 0;
      }
      if (gtop + m <= W) {
        for (int e = lane; e < m; e += 32) gs[gtop + e] = stack[e];
        __syncwarp();
        for (int e0 = 0; e0 < sp - m; e0 += 32) {
          uint2 v = make_uint2(0u, 0u);
          if (e0 + lane < sp - m) v = stack[m + e0 + lane];
          __syncwarp();
          if (e0 + lane < sp - m) stack[e0 + lane] = v;
          __syncwarp();
        }
        gtop += m;
        sp -= m;
      } else if (lane == 0) {
        atomicOr(&ctr->status, (unsigned)TL_ST_PRIV_OVF);  // the host grows it, repeats the step
      }
    }
    // the shared stack ran dry: refill it from the spill area's top
    if (sp == 0 && gtop > gbot) {
      const int m = min(gtop - gbot, D >> 1);
      for (int e = lane; e < m; e += 32) stack[e] = gs[gtop - m + e];
      __syncwarp();
      gtop -= m;
      sp = m;
      if (gtop == gbot) gtop = gbot = 0;
    }
    if ((sp > 1 || gtop > gbot) && budget > 0 && iters >= budget) {
      unsigned h = 0;
      if (lane == 0) h = *(volatile unsigned *)&ctr->hungry;
      h = __shfl_sync(0xffffffffu, h, 0);
      iters = 0;
      if (h > 0u) {
        // hand on chunks of 32 to the waiting warps, at most TL_DONATE_MAX
        // per waiting warp: the spill area's entries (its bottom first), then
        // all but the top 32 entries of the shared stack (or half of a stack
        // of at most 64); they are counted (q_tail) before this item is
        // counted finished
        // chunks available, each non-empty: the spill area's, then those the
        // loop below cuts from the shared stack (every reserved chunk must be
        // published, so the count follows the loop's own cuts)
        int avail = (gtop - gbot + kGroup - 1) / kGroup;
        for (int r = sp; ; ) {
          const int g = min(kGroup, r > 2 * kGroup ? r - kGroup : r / 2);
          if (g < 1) break;
          ++avail;
          r -= g;
        }
        const int nch = (int)min((unsigned)avail, (unsigned)TL_DONATE_MAX * h);
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&ctr->q_tail, (unsigned long long)nch);
        handed = true;
        base = __shfl_sync(0xffffffffu, base, 0);
        for (int c = 0; c < nch; ++c) {
          const bool fs = gtop > gbot;
          const int give = fs ? min(kGroup, gtop - gbot)
                              : min(kGroup, sp > 2 * kGroup ? sp - kGroup : sp / 2);
          const uint2 *src = fs ? gs + gbot : stack;
          if (base + c < qcap) {
            if (lane >= 1)
              Q[(base + c) * kGroup + lane] = lane < give ? pack2(src[lane]) : kQFree;
            __threadfence();
            __syncwarp();
            if (lane == 0 && atomicExch(Q + (base + c) * kGroup, pack2(src[0])) != kQFree)
              atomicOr(&ctr->status, (unsigned)TL_ST_SPILL_OVF);  // a chunk was not free
          } else if (lane == 0) {
            atomicOr(&ctr->status, (unsigned)TL_ST_SPILL_OVF);
          }
          __syncwarp();
          if (fs) {
            gbot += give;
            if (gbot == gtop) gbot = gtop = 0;
          } else {  // the kept entries move to the bottom
            const int keep = sp - give;
            for (int e0 = 0; e0 < keep; e0 += 32) {
              uint2 v = make_uint2(0u, 0u);
              if (e0 + lane < keep) v = stack[give + e0 + lane];
              __syncwarp();
              if (e0 + lane < keep) stack[e0 + lane] = v;
              __syncwarp();
            }
            sp = keep;
          }
        }
      }
    }
    if (sp == 0) {
      int got = 0;  // 1: a frontier group; 2: a queue chunk
      unsigned long long idx = 0;
      uint2 item = make_uint2(0u, 0u);
      if (lane == 0) {
        if (holding) {
          if (handed) __threadfence();  // this item's hand-ons (q_tail) before its finish
          atomicAdd(&ctr->q_done, 1ull);
          holding = false;
        }
        handed = false;
        const unsigned long long i = atomicAdd(&ctr->q_head, 1ull);
        if (i < nf) {
          idx = i;
          got = 1;
        } else if (i - nf < qcap) {
          idx = i - nf;
          unsigned long long *slot = Q + idx * kGroup;
          long long spins = 0;
          unsigned ns = 32;
          bool waiting = false;
          while (true) {
            const unsigned long long v = atomicExch(slot, kQFree);
            if (v != kQFree) {
              item = make_uint2((unsigned)v, (unsigned)(v >> 32));
              got = 2;
              __threadfence();  // entry 0 seen: the chunk's other entries are written
              break;
            }
            if (!waiting) {  // working warps see that a warp waits for work
              waiting = true;
              atomicAdd(&ctr->hungry, 1u);
            }
            // finished items first, then hand-ons: equal means nothing was in
            // flight at the first read, so nothing more can come
            const unsigned long long done = *(volatile unsigned long long *)&ctr->q_done;
            __threadfence();
            const unsigned long long tail = *(volatile unsigned long long *)&ctr->q_tail;
            if (done >= nf + tail) break;
            if (*(volatile unsigned *)&ctr->status & (TL_ST_SPILL_OVF | TL_ST_TIMEOUT)) break;
            if (++spins > a.spin_limit) {
              atomicOr(&ctr->status, (unsigned)TL_ST_TIMEOUT);
              break;
            }
            __nanosleep(ns);
            if (ns < 1024) ns <<= 1;
          }
          if (waiting) atomicSub(&ctr->hungry, 1u);
        }
        // an index past the queue's end: its producer flagged the overflow
      }
      got = __shfl_sync(0xffffffffu, got, 0);
      if (!got) break;
      idx = __shfl_sync(0xffffffffu, idx, 0);
      if (got == 1) {  // up to 32 frontier pairs
        const unsigned long long f = idx * kGroup + (unsigned long long)lane;
        const bool have = f < n0;
        if (have) stack[lane] = __ldcg(src0 + f);
        sp = __popc(__ballot_sync(0xffffffffu, have));
      } else {  // entries 1..31 of the chunk: the written ones come first
        unsigned long long v = kQFree;
        if (lane >= 1) v = __ldcg(Q + idx * kGroup + lane);
        const unsigned mv = __ballot_sync(0xffffffffu, v != kQFree);
        if (v != kQFree) stack[lane] = make_uint2((unsigned)v, (unsigned)(v >> 32));
        if (lane == 0) stack[0] = item;
        sp = 1 + __popc(mv);
      }
      if (lane == 0) holding = true;
      __syncwarp();
      iters = 0;
    }
    ++iters;
    // one popped pair per lane
    const int npop = min(sp, P);
    sp -= npop;
    const bool active = lane < npop;
    const uint2 pr = active ? stack[sp + lane] : make_uint2(0u, 0u);
    __syncwarp();
    const bool bka = (pr.x & TL_FLAG) != 0u, bkb = (pr.y & TL_FLAG) != 0u;
    TLNode ra, rb;
    if (active) {
      ra = node_record(a.A, pr.x);
      rb = node_record(a.B, pr.y);
    }
    // a bucket pair taken from the frontier was tested when it was produced
    const bool pass = active && bka && bkb;
    int tested = 0;
#pragma unroll
    for (int combo = 0; combo < 4; ++combo) {
      const int ia = combo >> 1, ib = combo & 1;
      bool ok = false, leaf = false;
      uint2 o = make_uint2(0u, 0u);
      if (pass) {
        if (combo == 0) {
          const Kid ka = kid_of(ra, pr.x, 0), kb = kid_of(rb, pr.y, 0);
          ok = leaf = true;
          o = make_uint2(ka.pack, kb.pack);
        }
      } else if (active && !(bka && ia) && !(bkb && ib)) {
        const Kid ka = kid_of(ra, pr.x, ia), kb = kid_of(rb, pr.y, ib);
        ++tested;
        ok = tl_overlap(ka.box, kb.box);
        leaf = ka.bucket && kb.bucket;
        o = leaf ? make_uint2(ka.pack, kb.pack) : make_uint2(ka.sref, kb.sref);
      }
      const unsigned mpush = __ballot_sync(0xffffffffu, ok && !leaf);
      const unsigned mleaf = __ballot_sync(0xffffffffu, ok && leaf);
      if (sp + __popc(mpush) > D) handed = true;  // (warp-uniform)
      if (ok && !leaf) {
        const int slot = sp + __popc(mpush & lt);
        if (slot < D) {
          stack[slot] = o;
        } else {  // the stack is full: this pair goes to the queue as a chunk of one
          const unsigned long long qi = atomicAdd(&ctr->q_tail, 1ull);
          if (qi < qcap) {
            for (int k = 1; k < kGroup; ++k) Q[qi * kGroup + k] = kQFree;
            __threadfence();
            if (atomicExch(Q + qi * kGroup, pack2(o)) != kQFree)
              atomicOr(&ctr->status, (unsigned)TL_ST_SPILL_OVF);
          } else {
            atomicOr(&ctr->status, (unsigned)TL_ST_SPILL_OVF);
          }
        }
      }
      sp = min(sp + __popc(mpush), D);
      if (ok && leaf) ws.leafq[nq + __popc(mleaf & lt)] = o;
      nq += __popc(mleaf);
    }
    for (int off = 16; off; off >>= 1) tested += __shfl_xor_sync(0xffffffffu, tested, off);
    if (lane == 0) node_tests += (unsigned long long)tested;
    __syncwarp();
    if (nq >= 32) {
      spill_leaves(a, ws, nq, lane, lbase);
      nq = 0;
    }
  }
  if (nq) spill_leaves(a, ws, nq, lane, lbase);
  if (lane == 0 && node_tests) atomicAdd(&ctr->node_tests, node_tests);
}

// The narrow phase of the step's listed leaf pairs: each warp takes 32 of
// them at a time and flattens their photon pairs over its lanes.
template <bool FP64>
__global__ void __launch_bounds__(256) k_narrow(TravArgs a) {
  __shared__ WarpSmem wsm[8];
  __shared__ float sbin[TL_SBINS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  WarpSmem &ws = wsm[warp];
  for (int i = threadIdx.x; i < TL_SBINS; i += blockDim.x) sbin[i] = a.nk.sbin[i];
  __syncthreads();
  const unsigned long long listed = a.ctr->leaf_pairs - a.ctr->leaf_base;  // this part's
  const unsigned long long n = min(listed, a.leaf_cap);
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicMax(&a.ctr->max_part_leaves, listed);
  const unsigned long long stride = (unsigned long long)gridDim.x * (blockDim.x >> 5) * 32ull;
  unsigned long long tests = 0;
  int npend = 0;
  for (unsigned long long base = ((unsigned long long)blockIdx.x * (blockDim.x >> 5) + warp) * 32ull;
       base < n; base += stride) {
    const int m = (int)min(32ull, n - base);
    if (lane < m) ws.leafq[lane] = a.leaves[base + lane];
    __syncwarp();
    flush_leaves<FP64>(a, ws, m, lane, tests, npend, sbin);
  }
  if (!FP64 && npend > 0) decide_pending(a, ws, npend, lane, sbin);
  if (lane == 0 && tests) atomicAdd(&a.ctr->narrow_tests, tests);
}

// ------------------------------------------------------------ band re-test

__global__ void __launch_bounds__(256) k_band(TravArgs a) {
  const int lane = threadIdx.x & 31;
  const unsigned long long n = min(a.ctr->band, a.band_cap);
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  const unsigned long long nround = (n + 31ull) & ~31ull;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < nround;
       i += stride) {
    bool hit = false;
    uint2 q = make_uint2(0u, 0u);
    if (i < n) {
      q = a.band[i];
      hit = tl_exact_hit(a.mA, q.x, a.mB, q.y, a.ct, a.dt, a.kappa);
    }
    emit(hit, q.x, q.y, a.hits, a.hit_cap, &a.ctr->hits, &a.ctr->status, TL_ST_HIT_OVF, lane);
  }
}

// ------------------------------------------------------------ yield

// Sum over the step's hits of w_i w_j (FP64), the count and the order-free
// checksums.  Per-block partials are combined by the last block to finish,
// in a fixed order.
__global__ void __launch_bounds__(256) k_yield(TravArgs a, YieldPartial *partials) {
  __shared__ YieldPartial sp[8];
  __shared__ bool last;
  const unsigned long long n = min(a.ctr->hits, a.hit_cap);
  YieldPartial p = yield_zero();
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const uint2 h = a.hits[i];
    yield_hit(p, h.x, h.y, a.mA.w ? a.mA.w[h.x] : 1.0, a.mB.w ? a.mB.w[h.y] : 1.0);
  }
  const YieldPartial b = yield_block_reduce(p, sp);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = b;
    __threadfence();
    last = atomicAdd(&a.ctr->reduce_done, 1u) == gridDim.x - 1u;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  YieldPartial t = yield_zero();
  for (unsigned q = threadIdx.x; q < gridDim.x; q += blockDim.x) yield_add(t, yield_load_volatile(partials + q));
  const YieldPartial tot = yield_block_reduce(t, sp);
  if (threadIdx.x == 0) {
    a.ctr->count = tot.count;
    a.ctr->weighted = tot.weighted;
    a.ctr->hsum = tot.hsum;
    a.ctr->hxor = tot.hxor;
  }
}

// Per-instance yield: count and sum of w_i w_j of each instance's hits,
// accumulated into yields[2 * inst], yields[2 * inst + 1].
__global__ void __launch_bounds__(256) k_yield_inst(TravArgs a, const uint32_t *inst_of_a,
                                                    double *yields) {
  const unsigned long long n = min(a.ctr->hits, a.hit_cap);
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const uint2 h = a.hits[i];
    const double wi = a.mA.w ? a.mA.w[h.x] : 1.0, wj = a.mB.w ? a.mB.w[h.y] : 1.0;
    const uint32_t q = inst_of_a[h.x];
    atomicAdd(&yields[2 * q], 1.0);
    atomicAdd(&yields[2 * q + 1], wi * wj);
  }
}

// End of a step in graph mode: keep the step's status bits and add the
// step's yield and counters to the run's totals (acc may be NULL).
__global__ void k_step_finish(const TLCounters *ctr, unsigned *run_status, TLRunAcc *acc) {
  const unsigned st = ctr->status;
  if (st) atomicOr(run_status, st);
  if (acc) {
    acc->count += ctr->count;
    acc->weighted += ctr->weighted;
    acc->hsum += ctr->hsum;
    acc->hxor ^= ctr->hxor;
    acc->narrow_tests += ctr->narrow_tests;
    acc->node_tests += ctr->node_tests;
    acc->leaf_pairs += ctr->leaf_pairs;
    acc->band += ctr->band;
    if (ctr->hits > acc->max_hits) acc->max_hits = ctr->hits;
    if (ctr->band > acc->max_band) acc->max_band = ctr->band;
    if (ctr->q_tail > acc->max_handed) acc->max_handed = ctr->q_tail;
    if (ctr->max_part_leaves > acc->max_leaves) acc->max_leaves = ctr->max_part_leaves;
  }
}

// ------------------------------------------------------------ host launchers

size_t traverse_smem(int warps, int depth) {
  return sizeof(uint2) * (size_t)depth * warps + sizeof(WarpSmem) * (size_t)warps;
}

cudaError_t launch_step_init(TLCounters *ctr, uint2 *F0, uint32_t sa, uint32_t sb, int nonempty,
                             const unsigned *build_status, const unsigned *run_status,
                             cudaStream_t s) {
  k_step_init<<<1, 128, 0, s>>>(ctr, F0, sa, sb, nonempty, build_status, run_status);
  return cudaGetLastError();
}

cudaError_t launch_seed_cut(const TravArgs &a, const uint32_t *cutA, const unsigned *cntA,
                            uint32_t capA, const uint32_t *cutB, const unsigned *cntB,
                            uint32_t capB, uint2 *F0, unsigned cap, int blocks, cudaStream_t s) {
  k_seed_cut<<<blocks, 256, 0, s>>>(a, cutA, cntA, capA, cutB, cntB, capB, F0, cap);
  return cudaGetLastError();
}

cudaError_t launch_expand(const TravArgs &a, uint2 *F0, uint2 *F1, unsigned cap, unsigned target,
                          int max_levels, cudaStream_t s) {
  k_expand<<<1, 1024, 0, s>>>(a, F0, F1, cap, target, max_levels);
  return cudaGetLastError();
}

cudaError_t launch_widen(const TravArgs &a, uint2 *F0, uint2 *F1, unsigned cap, unsigned target,
                         int levels, int blocks, cudaStream_t s) {
  for (int l = 0; l < levels; ++l) {
    k_widen<<<blocks, 256, 0, s>>>(a, F0, F1, cap, target, l);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t traverse_config(int fp64, int warps, int depth, int *blocks_per_sm) {
  (void)fp64;  // the traversal is the same for both precisions (the narrow phase differs)
  const size_t smem = traverse_smem(warps, depth);
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_traverse, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem)))
    return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_traverse, warps * 32, smem);
}

cudaError_t launch_traverse(const TravArgs &a, const uint2 *F0, const uint2 *F1, const uint2 *list,
                            unsigned long long list_n, int from_frontier, int budget, int blocks,
                            int warps, cudaStream_t s, int part, int nparts) {
  // a warp only waits for work that warps holding items (running ones) hand
  // on, so no block needs another to be resident
  const size_t smem = traverse_smem(warps, a.stack_depth);
  k_traverse<<<blocks, warps * 32, smem, s>>>(a, F0, F1, list, list_n, from_frontier, budget,
                                              part, nparts);
  return cudaGetLastError();
}

// Before part p > 0 of a step: the leaf list starts again (at the count so
// far) and the work queue's counters are cleared for the next traversal.
__global__ void k_part_init(TLCounters *ctr) {
  ctr->leaf_base = ctr->leaf_pairs;
  ctr->q_head = ctr->q_done = ctr->q_tail = 0ull;
  ctr->hungry = 0u;
}

cudaError_t launch_part_init(TLCounters *ctr, cudaStream_t s) {
  k_part_init<<<1, 1, 0, s>>>(ctr);
  return cudaGetLastError();
}

cudaError_t launch_narrow(const TravArgs &a, int blocks, cudaStream_t s) {
  if (a.fp64) k_narrow<true><<<blocks, 256, 0, s>>>(a);
  else k_narrow<false><<<blocks, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_band(const TravArgs &a, int blocks, cudaStream_t s) {
  k_band<<<blocks, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_yield(const TravArgs &a, void *partials, int blocks, cudaStream_t s) {
  k_yield<<<blocks, 256, 0, s>>>(a, reinterpret_cast<YieldPartial *>(partials));
  return cudaGetLastError();
}

size_t partial_bytes() { return sizeof(YieldPartial); }

cudaError_t launch_seed_instances(TLCounters *ctr, uint2 *F0, const uint32_t *rootA,
                                  const uint32_t *rootB, int n_inst, cudaStream_t s) {
  k_seed_instances<<<(n_inst + 255) / 256, 256, 0, s>>>(ctr, F0, rootA, rootB, n_inst);
  return cudaGetLastError();
}

cudaError_t launch_yield_inst(const TravArgs &a, const uint32_t *inst_of_a, double *yields,
                              int blocks, cudaStream_t s) {
  k_yield_inst<<<blocks, 256, 0, s>>>(a, inst_of_a, yields);
  return cudaGetLastError();
}

cudaError_t launch_step_finish(const TLCounters *ctr, unsigned *run_status, TLRunAcc *acc,
                               cudaStream_t s) {
  k_step_finish<<<1, 1, 0, s>>>(ctr, run_status, acc);
  return cudaGetLastError();
}

}  // namespace tl
