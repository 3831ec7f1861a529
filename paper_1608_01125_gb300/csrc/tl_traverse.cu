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
// iteration a warp pops up to 8 pairs and tests the up-to-4 child
// combinations of each with one lane per combination; survivors are pushed
// (or, when both sides are leaf buckets, queued) with ballot/popc
// compaction.  Queued bucket pairs are flattened over the warp's lanes, one
// photon pair per lane, and given the narrow-phase test; hits leave with one
// atomic per warp.
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

__global__ void k_step_init(TLCounters *ctr, uint2 *F0, uint32_t superA, uint32_t superB,
                            int nonempty, const unsigned *build_status) {
  unsigned *w = reinterpret_cast<unsigned *>(ctr);
  for (int i = threadIdx.x; i < (int)(sizeof(TLCounters) / 4); i += blockDim.x) w[i] = 0u;
  if (threadIdx.x == 0) F0[0] = make_uint2(superA, superB);
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned bs = *build_status & (unsigned)TL_ST_TIMEOUT;
    ctr->status = bs;
    // after a failed build there is nothing valid to traverse
    ctr->counts[0] = (nonempty && !bs) ? 1u : 0u;
  }
}

// Several instances: the frontier starts from each instance's pair of
// subtree roots, so no pair of photons from different instances is tested.
__global__ void k_seed_instances(TLCounters *ctr, uint2 *F0, const uint32_t *rootA,
                                 const uint32_t *rootB, int n_inst) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n_inst || (ctr->status & TL_ST_TIMEOUT)) return;
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
  if (ctr->status & TL_ST_TIMEOUT) return;  // the build failed: nothing to traverse
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

// ------------------------------------------------------------ narrow phase

struct WarpSmem {
  uint2 leafq[64];
  int scan[32];
};

template <bool FP64>
__device__ __forceinline__ void flush_leaves(const TravArgs &a, WarpSmem &ws, int nq, int lane,
                                             unsigned long long &tests) {
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
      uint32_t oi = 0u, oj = 0u;
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
        const float4 da = __ldg(a.A.dir + fa + ia), db = __ldg(a.B.dir + fb + jb);
        oi = __float_as_uint(da.w);
        oj = __float_as_uint(db.w);
        if (FP64) {
          outcome = tl_exact_hit(a.mA, oi, a.mB, oj, a.ct, a.dt, a.kappa) ? TL_HIT : TL_MISS;
        } else {
          const float4 pa = __ldg(a.A.pos + fa + ia), pb = __ldg(a.B.pos + fb + jb);
          outcome = tl_narrow32(pa, da, pb, db, a.nk);
        }
      }
      emit(outcome == TL_HIT, oi, oj, a.hits, a.hit_cap, &a.ctr->hits, &a.ctr->status,
           TL_ST_HIT_OVF, lane);
      if (!FP64)
        emit(outcome == TL_BAND, oi, oj, a.band, a.band_cap, &a.ctr->band, &a.ctr->status,
             TL_ST_BAND_OVF, lane);
    }
    __syncwarp();
  }
  (void)lt;
}

// ------------------------------------------------------------ traversal

// Persistent warps share one work queue.  The frontier's items come first
// (indices below n0), then the queue's chunks of up to 8 node pairs each (64
// bytes): a warp that spends `budget` iterations on one item hands the rest of
// it (its whole stack) on as chunks, which idle warps take at once, popping 8
// pairs in their first iteration; a warp whose stack is full hands on the pair
// that does not fit as a chunk of one.  Unused and free entries hold a
// sentinel.  A writer fills a chunk's entries 1..7, fences, then swaps entry 0
// in; a taker swaps the sentinel back into entry 0 as it reads it (atomic
// exchange) and waits while it is still free and work is in flight.  The
// traversal ends when the chunks finished equal n0 plus the chunks handed on.
// Every wait is bounded by spin_limit (then TL_ST_TIMEOUT).
constexpr unsigned long long kQFree = 0xffffffffffffffffull;

__device__ __forceinline__ unsigned long long pack2(uint2 v) {
  return (unsigned long long)v.x | ((unsigned long long)v.y << 32);
}

// (Bounding the registers to 48 for five 256-thread blocks per SM spilled
// a little and ran the 2 x 1M traversal 2% slower.)
template <bool FP64>
__global__ void __launch_bounds__(512) k_traverse(TravArgs a, const uint2 *F0, const uint2 *F1,
                                                  const uint2 *list, unsigned long long list_n,
                                                  int from_frontier, int budget) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int D = a.stack_depth;
  uint2 *stack = reinterpret_cast<uint2 *>(smem_raw) + (size_t)warp * D;
  WarpSmem &ws = reinterpret_cast<WarpSmem *>(
      smem_raw + sizeof(uint2) * (size_t)D * (blockDim.x >> 5))[warp];
  TLCounters *ctr = a.ctr;
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
  unsigned long long *Q = a.queue;
  const unsigned long long qcap = a.queue_cap >> 3;  // chunks of 8 pairs
  const unsigned lt = (1u << lane) - 1u;
  int sp = 0, nq = 0, iters = 0;
  bool holding = false;  // this warp holds an item (counted in flight)
  bool handed = false;   // ... and has handed pieces of it on
  unsigned long long node_tests = 0, narrow_tests = 0, leaf_pairs = 0;
  while (true) {
    if (sp > 0 && budget > 0 && iters >= budget) {
      // this item is large: hand the rest of it (the whole stack) on as chunks;
      // they are counted before this item is counted finished
      const int nch = (sp + 7) >> 3;
      unsigned long long base = 0;
      if (lane == 0) base = atomicAdd(&ctr->q_tail, (unsigned long long)nch);
      handed = true;
      base = __shfl_sync(0xffffffffu, base, 0);
      for (int e = lane; e < nch * 8; e += 32) {  // entries 1..7 of every chunk
        if ((e & 7) != 0 && base + (e >> 3) < qcap)
          Q[(base + (e >> 3)) * 8 + (e & 7)] = e < sp ? pack2(stack[e]) : kQFree;
      }
      __threadfence();
      __syncwarp();
      for (int c = lane; c < nch; c += 32) {  // then entry 0: the chunk is ready
        if (base + c < qcap) {
          if (atomicExch(Q + (base + c) * 8, pack2(stack[c * 8])) != kQFree)
            atomicOr(&ctr->status, (unsigned)TL_ST_SPILL_OVF);  // a chunk was not free
        } else {
          atomicOr(&ctr->status, (unsigned)TL_ST_SPILL_OVF);
        }
      }
      __syncwarp();
      sp = 0;
    }
    if (sp == 0) {
      int got = 0;  // 1: a frontier item; 2: a queue chunk
      unsigned long long chunk = 0;
      uint2 item = make_uint2(0u, 0u);
      if (lane == 0) {
        if (holding) {
          if (handed) __threadfence();  // this item's hand-ons (q_tail) before its finish
          atomicAdd(&ctr->q_done, 1ull);
          holding = false;
        }
        handed = false;
        const unsigned long long i = atomicAdd(&ctr->q_head, 1ull);
        if (i < n0) {
          item = __ldcg(src0 + i);
          got = 1;
        } else if (i - n0 < qcap) {
          chunk = i - n0;
          unsigned long long *slot = Q + chunk * 8;
          long long spins = 0;
          unsigned ns = 32;
          while (true) {
            const unsigned long long v = atomicExch(slot, kQFree);
            if (v != kQFree) {
              item = make_uint2((unsigned)v, (unsigned)(v >> 32));
              got = 2;
              __threadfence();  // entry 0 seen: the chunk's other entries are written
              break;
            }
            // finished items first, then hand-ons: equal means nothing was in
            // flight at the first read, so nothing more can come
            const unsigned long long done = *(volatile unsigned long long *)&ctr->q_done;
            __threadfence();
            const unsigned long long tail = *(volatile unsigned long long *)&ctr->q_tail;
            if (done >= n0 + tail) break;
            if (*(volatile unsigned *)&ctr->status & (TL_ST_SPILL_OVF | TL_ST_TIMEOUT)) break;
            if (++spins > a.spin_limit) {
              atomicOr(&ctr->status, (unsigned)TL_ST_TIMEOUT);
              break;
            }
            __nanosleep(ns);
            if (ns < 1024) ns <<= 1;
          }
        }
        // an index past the queue's end: its producer flagged the overflow
      }
      got = __shfl_sync(0xffffffffu, got, 0);
      if (!got) break;
      sp = 1;
      if (got == 2) {  // entries 1..7 of the chunk: the written ones come first
        chunk = __shfl_sync(0xffffffffu, chunk, 0);
        unsigned long long v = kQFree;
        if (lane >= 1 && lane < 8) v = __ldcg(Q + chunk * 8 + lane);
        const unsigned mv = __ballot_sync(0xffffffffu, v != kQFree);
        if (v != kQFree) stack[lane] = make_uint2((unsigned)v, (unsigned)(v >> 32));
        sp = 1 + __popc(mv);
      }
      if (lane == 0) {
        stack[0] = item;
        holding = true;
      }
      __syncwarp();
      iters = 0;
    }
    ++iters;
    const int npop = min(sp, 8);
    sp -= npop;
    const int p = lane >> 2, combo = lane & 3;
    const bool active = p < npop;
    const uint2 pr = active ? stack[sp + p] : make_uint2(0u, 0u);
    __syncwarp();
    bool ok = false, leafleaf = false, tested = false;
    uint2 o = make_uint2(0u, 0u);
    if (active) {
      if ((pr.x & TL_FLAG) && (pr.y & TL_FLAG)) {
        if (combo == 0) {  // a bucket pair taken from the frontier
          const Side sa = side_of(a.A, pr.x, 0), sb = side_of(a.B, pr.y, 0);
          ok = leafleaf = true;
          o = make_uint2(pack_bucket(sa.first, sa.cnt), pack_bucket(sb.first, sb.cnt));
        }
      } else {
        Side sa, sb;
        if (child_pair(a.A, a.B, pr, combo, sa, sb)) {
          tested = true;
          ok = tl_overlap(sa.box, sb.box);
          leafleaf = sa.bucket && sb.bucket;
          o = leafleaf ? make_uint2(pack_bucket(sa.first, sa.cnt), pack_bucket(sb.first, sb.cnt))
                       : make_uint2(sa.sref, sb.sref);
        }
      }
    }
    const unsigned mtest = __ballot_sync(0xffffffffu, tested);
    if (lane == 0) node_tests += (unsigned long long)__popc(mtest);
    const unsigned mpush = __ballot_sync(0xffffffffu, ok && !leafleaf);
    const unsigned mleaf = __ballot_sync(0xffffffffu, ok && leafleaf);
    if (sp + __popc(mpush) > D) handed = true;  // (warp-uniform)
    if (ok && !leafleaf) {
      const int slot = sp + __popc(mpush & lt);
      if (slot < D) {
        stack[slot] = o;
      } else {  // the stack is full: this pair goes to the queue as a chunk of one
        const unsigned long long idx = atomicAdd(&ctr->q_tail, 1ull);
        if (idx < qcap) {
          for (int k = 1; k < 8; ++k) Q[idx * 8 + k] = kQFree;
          __threadfence();
          if (atomicExch(Q + idx * 8, pack2(o)) != kQFree)
            atomicOr(&ctr->status, (unsigned)TL_ST_SPILL_OVF);
        } else {
          atomicOr(&ctr->status, (unsigned)TL_ST_SPILL_OVF);
        }
      }
    }
    sp = min(sp + __popc(mpush), D);
    if (ok && leafleaf) ws.leafq[nq + __popc(mleaf & lt)] = o;
    nq += __popc(mleaf);
    __syncwarp();
    if (nq >= 32) {
      leaf_pairs += nq;
      flush_leaves<FP64>(a, ws, nq, lane, narrow_tests);
      nq = 0;
    }
  }
  if (nq) {
    leaf_pairs += nq;
    flush_leaves<FP64>(a, ws, nq, lane, narrow_tests);
  }
  if (lane == 0) {
    if (node_tests) atomicAdd(&ctr->node_tests, node_tests);
    if (narrow_tests) atomicAdd(&ctr->narrow_tests, narrow_tests);
    if (leaf_pairs) atomicAdd(&ctr->leaf_pairs, leaf_pairs);
  }
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
  }
}

// ------------------------------------------------------------ host launchers

size_t traverse_smem(int warps, int depth) {
  return sizeof(uint2) * (size_t)depth * warps + sizeof(WarpSmem) * (size_t)warps;
}

cudaError_t launch_step_init(TLCounters *ctr, uint2 *F0, uint32_t sa, uint32_t sb, int nonempty,
                             const unsigned *build_status, cudaStream_t s) {
  k_step_init<<<1, 128, 0, s>>>(ctr, F0, sa, sb, nonempty, build_status);
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

cudaError_t traverse_config(int fp64, int warps, int depth, int *blocks_per_sm) {
  size_t smem = traverse_smem(warps, depth);
  cudaError_t e;
  if (fp64) {
    if ((e = cudaFuncSetAttribute(k_traverse<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)))
      return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_traverse<true>,
                                                         warps * 32, smem);
  }
  if ((e = cudaFuncSetAttribute(k_traverse<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem)))
    return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_traverse<false>,
                                                       warps * 32, smem);
}

cudaError_t launch_traverse(const TravArgs &a, const uint2 *F0, const uint2 *F1, const uint2 *list,
                            unsigned long long list_n, int from_frontier, int budget, int blocks,
                            int warps, cudaStream_t s) {
  // a warp only waits for work that warps holding items (running ones) hand
  // on, so no block needs another to be resident
  const size_t smem = traverse_smem(warps, a.stack_depth);
  if (a.fp64)
    k_traverse<true><<<blocks, warps * 32, smem, s>>>(a, F0, F1, list, list_n, from_frontier,
                                                       budget);
  else
    k_traverse<false><<<blocks, warps * 32, smem, s>>>(a, F0, F1, list, list_n, from_frontier,
                                                        budget);
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
