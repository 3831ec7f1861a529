// tl_deplete.cu -- depletion with chronological order (Sec. 2.2, Sec. 3.1).
//
// Photons annihilate when they collide, so a collision only happens if both
// photons still exist; the collisions of a step are therefore taken in time
// order (Sec. 2.2 sorts them chronologically; Fig. ChronOrder shows why).  A
// macro-photon of weight w is a swarm of w photons handled one by one
// (Sec. 2.2), so a collision takes delta = min(rem_i, rem_j) from both; with
// unit weights the earliest remaining hit of a photon annihilates it.
//
// The order is (step, t*, i, j); calls come step by step, so inside a call it
// is (t*, i, j).  What a hit takes depends only on the earlier hits of its own
// two photons, and the order of the hits at one photon is (t*, j) for a photon
// of A and (t*, i) for one of B.  So no global sort is needed: a hit can be
// resolved as soon as it is the earliest unresolved hit at both of its
// photons, and every such hit of a round touches photons no other resolved
// hit of that round touches.  Each round, over the hits still open:
//   R1  hits whose photon is used up take 0; the others take part in an
//       atomicMin of their time key at both photons;
//   R2  among the hits holding that minimum, an atomicMin of the partner index
//       (only in rounds with a tie: R1's atomicMin returns the key it replaced,
//       and a hit that finds its own key there flags one; without a flag each
//       photon's minimum is held by one hit and R2 is skipped);
//   R3  a hit holding both minima at both photons is resolved; the others
//       clear the other round's slots of their photons and are appended to
//       the next round's list (the open hits are compacted once per round, so
//       a round costs what is still open, not the whole list).
// The globally earliest unresolved hit is always resolved, so a step of n
// hits needs at most n rounds.
//
// A call is one cooperative launch: the t* keys (fused with round 0's R1),
// every round and the final clear and sum run in one kernel whose phases are
// separated by a grid-wide barrier (every block is resident; each wait has an
// iteration limit after which the kernel sets an error flag and returns).  The
// list lengths, the round count and the results stay on the device: the
// asynchronous entry point leaves them in a caller-owned device record, the
// synchronous one reads that record back.  A call that fails after touching
// the photon slots marks them dirty on the device; the next call clears them
// first.
//
// Once few hits are left open (kTail), block 0 runs the remaining rounds
// alone, its phases separated by __syncthreads instead of grid barriers.
//
// Layout: a photon's slots of both round parities share one 32-byte record
// (one sector), and the photons' FP64 positions and directions are packed once
// per context into 64-byte records (two sectors per photon instead of six for
// the t* gather).
//
// t* is computed with the operations of the exact decision (FP64, explicit
// round-to-nearest), so the order is the one the FP64 definition gives.
#include "tl_ctx.h"

namespace {

constexpr unsigned long long kNoKey = ~0ull;
constexpr unsigned kNoIdx = ~0u;
constexpr int kThreads = 1024;
constexpr long long kTail = 2 * kThreads;  // open hits below which block 0 goes on alone

enum : uint8_t { kOpen = 0, kDone = 1 };
enum : int { kFlagBadInput = 1, kFlagRounds = 2, kFlagBarrier = 4 };

// Device control block of a call, zeroed before the launch.
struct DepCtl {
  unsigned cnt[2];  // entries of list[0], list[1]
  unsigned arrive;  // grid barrier: blocks arrived
  unsigned gen;     // grid barrier: generation
  int flag;         // kFlag* bits
  int tie[2];       // by round parity: some hit met its own time key at a photon in R1
  int pad;
};

}  // namespace

// A photon's slots: for each round parity, the time key of its earliest open
// hit and the smallest partner among its hits at that time (all ones: empty).
struct alignas(32) DepSlot {
  unsigned long long t[2];
  unsigned p[2];
  unsigned pad[2];
};

// A photon's FP64 position at t = 0 and direction, packed for the t* gather.
struct alignas(64) DepPhoton {
  double p[3], d[3], pad[2];
};

namespace {

struct DepArgs {
  long long na, nb;
  const DepPhoton *A, *B;
  double ct;
  const uint2 *hits;
  long long n;
  unsigned long long *key;
  uint8_t *state;
  double *delta;
  double *rem_a, *rem_b;
  DepSlot *sA, *sB;
  unsigned *list[2];  // open hits of the next round (indices into hits), by parity
  double *psum;       // one partial sum per block
  unsigned long long *pcnt;
  DepCtl *ctl;
  int *dirty;         // persistent: the photon slots need clearing
  trilens_deplete_out *out;
  long long spin;
};

// t* of photon i of A and photon j of B at c t_k = ct: the operations of the
// exact decision (Eq. CollDet's closest approach), infinity for parallel motion.
__device__ __forceinline__ double dep_tstar(const DepPhoton *A, uint32_t i, const DepPhoton *B,
                                            uint32_t j, double ct) {
  const double2 *qa = reinterpret_cast<const double2 *>(A + i);
  const double2 *qb = reinterpret_cast<const double2 *>(B + j);
  const double2 a0 = __ldg(qa), a1 = __ldg(qa + 1), a2 = __ldg(qa + 2);
  const double2 b0 = __ldg(qb), b1 = __ldg(qb + 1), b2 = __ldg(qb + 2);
  const double pxi = a0.x, pyi = a0.y, pzi = a1.x, dxi = a1.y, dyi = a2.x, dzi = a2.y;
  const double pxj = b0.x, pyj = b0.y, pzj = b1.x, dxj = b1.y, dyj = b2.x, dzj = b2.y;
  double vx = __dmul_rn(TL_C, __dsub_rn(dxi, dxj));
  double vy = __dmul_rn(TL_C, __dsub_rn(dyi, dyj));
  double vz = __dmul_rn(TL_C, __dsub_rn(dzi, dzj));
  double vv = __dadd_rn(__dadd_rn(__dmul_rn(vx, vx), __dmul_rn(vy, vy)), __dmul_rn(vz, vz));
  if (vv == 0.0) return __longlong_as_double(0x7ff0000000000000LL);
  double px = __dsub_rn(__dadd_rn(pxi, __dmul_rn(ct, dxi)), __dadd_rn(pxj, __dmul_rn(ct, dxj)));
  double py = __dsub_rn(__dadd_rn(pyi, __dmul_rn(ct, dyi)), __dadd_rn(pyj, __dmul_rn(ct, dyj)));
  double pz = __dsub_rn(__dadd_rn(pzi, __dmul_rn(ct, dzi)), __dadd_rn(pzj, __dmul_rn(ct, dzj)));
  double pv = __dadd_rn(__dadd_rn(__dmul_rn(px, vx), __dmul_rn(py, vy)), __dmul_rn(pz, vz));
  return __ddiv_rn(-pv, vv);
}

// x < y  <=>  time_key(x) < time_key(y) for non-NaN doubles; -0 and +0 equal
__device__ __forceinline__ unsigned long long time_key(double t) {
  if (t == 0.0) t = 0.0;
  const unsigned long long b = (unsigned long long)__double_as_longlong(t);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// Block reduction of (sum, count) into thread 0, in a fixed tree.
__device__ __forceinline__ void block_sum(double &s, unsigned long long &c, double *ss,
                                          unsigned long long *sc) {
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_down_sync(0xffffffffu, s, o);
    c += __shfl_down_sync(0xffffffffu, c, o);
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    ss[w] = s;
    sc[w] = c;
  }
  __syncthreads();
  if (w == 0) {
    s = lane < (int)(blockDim.x >> 5) ? ss[lane] : 0.0;
    c = lane < (int)(blockDim.x >> 5) ? sc[lane] : 0ull;
    for (int o = 16; o > 0; o >>= 1) {
      s += __shfl_down_sync(0xffffffffu, s, o);
      c += __shfl_down_sync(0xffffffffu, c, o);
    }
  }
}

// Grid-wide barrier of the cooperative launch.  Every thread makes its writes
// visible at device scope (a fence) before the block arrives; thread 0 then
// arrives on a counter, the last one to arrive resets it and advances the
// generation the others wait on, and every waiter fences again after it sees
// the new generation.  The wait is bounded: on a timeout (or when another
// block already gave up) the block sets kFlagBarrier, marks the slots dirty
// and the call returns false, after which the block leaves the kernel; the
// others then give up at their next barrier.
__device__ bool grid_sync(const DepArgs &g) {
  __shared__ int ok_s;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    DepCtl *ctl = g.ctl;
    volatile unsigned *gen = &ctl->gen;
    const unsigned g0 = *gen;
    __threadfence();
    if (atomicAdd(&ctl->arrive, 1u) == gridDim.x - 1) {
      atomicExch(&ctl->arrive, 0u);
      __threadfence();
      atomicAdd(&ctl->gen, 1u);
    } else {
      long long it = 0;
      while (*gen == g0) {
        if ((*(volatile int *)&ctl->flag & kFlagBarrier) || ++it > g.spin) {
          atomicOr(&ctl->flag, kFlagBarrier);
          atomicExch(g.dirty, 1);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// Block 0 records a call that ended early (every field but the status zero).
__device__ void record_failure(const DepArgs &g, long long status) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    g.out->transferred = 0.0;
    g.out->accepted = 0;
    g.out->rounds = 0;
    g.out->status = status;
  }
}

__device__ __forceinline__ void clear_slot(DepSlot *q) {
  uint4 *v = reinterpret_cast<uint4 *>(q);
  v[0] = make_uint4(~0u, ~0u, ~0u, ~0u);
  v[1] = make_uint4(~0u, ~0u, ~0u, ~0u);
}

__global__ void k_dep_pack(TLBeam A, TLBeam B, DepPhoton *pa, DepPhoton *pb) {
  const long long n = A.n > B.n ? A.n : B.n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    if (i < A.n) pa[i] = DepPhoton{{A.px[i], A.py[i], A.pz[i]}, {A.dx[i], A.dy[i], A.dz[i]}, {0, 0}};
    if (i < B.n) pb[i] = DepPhoton{{B.px[i], B.py[i], B.pz[i]}, {B.dx[i], B.dy[i], B.dz[i]}, {0, 0}};
  }
}

// Phase separation: grid-wide between the rounds every block shares, the
// block's own barrier once block 0 runs the tail alone.
template <bool kBlock>
__device__ __forceinline__ bool phase_sync(const DepArgs &g) {
  if (kBlock) {  // reads go through L2 (__ldcg): the block's writes first reach it
    __threadfence();
    __syncthreads();
    return true;
  }
  return grid_sync(g);
}

// Rounds from round r (R1 skipped for round 0: it ran with the t* keys) over
// the nr open hits of `cur` (nullptr: every hit), work items tid0, tid0 +
// stride, ...  Returns 0 when no hit is left open, 1 (grid mode only) when at
// most kTail are, -1 on a failed barrier, -2 when the rounds ran out.
template <bool kBlock>
__device__ int run_rounds(const DepArgs &g, long long &nr, const unsigned *&cur, long long &r,
                          long long tid0, long long stride) {
  const int lane = threadIdx.x & 31;
  DepCtl *ctl = g.ctl;
  for (;; ++r) {
    if (!kBlock && nr <= kTail) return 1;
    if (r > g.n) return -2;  // unreachable: every round resolves the earliest open hit
    const int b = (int)(r & 1), nb = b ^ 1;
    unsigned *cntn = b ? &ctl->cnt[0] : &ctl->cnt[1];
    unsigned *listn = b ? g.list[0] : g.list[1];
    int *tie = b ? &ctl->tie[1] : &ctl->tie[0];
    // the list written this round goes to list[nb]; its count held the list
    // of round r - 1, which every thread has finished reading; the same holds
    // for the other parity's tie flag.  Round 0's are zero from the launch's
    // start: a reset here would race with R3's appends when R2 is skipped (no
    // barrier between them), so only later rounds reset, before R1's barrier.
    if (tid0 == 0 && r > 0) {
      *cntn = 0;
      *(b ? &ctl->tie[0] : &ctl->tie[1]) = 0;
    }
    if (r > 0) {
      // R1
      for (long long i = tid0; i < nr; i += stride) {
        const unsigned e = __ldcg(cur + i);
        const uint2 h = g.hits[e];
        if (!(__ldcg(g.rem_a + h.x) > 0.0) || !(__ldcg(g.rem_b + h.y) > 0.0)) {
          g.state[e] = kDone;  // delta stays 0
          continue;
        }
        g.state[e] = kOpen;
        const unsigned long long k = __ldcg(g.key + e);
        if ((atomicMin(&g.sA[h.x].t[b], k) == k) | (atomicMin(&g.sB[h.y].t[b], k) == k))
          atomicOr(tie, 1);
      }
      if (!phase_sync<kBlock>(g)) return -1;
    }
    const bool ties = __ldcg(tie) != 0;
    // R2
    for (long long i = tid0; ties && i < nr; i += stride) {
      const unsigned e = cur ? __ldcg(cur + i) : (unsigned)i;
      if (__ldcg(g.state + e) != kOpen) continue;
      const uint2 h = g.hits[e];
      const unsigned long long k = __ldcg(g.key + e);
      if (__ldcg(&g.sA[h.x].t[b]) == k) atomicMin(&g.sA[h.x].p[b], h.y);
      if (__ldcg(&g.sB[h.y].t[b]) == k) atomicMin(&g.sB[h.y].p[b], h.x);
    }
    if (ties && !phase_sync<kBlock>(g)) return -1;
    // R3 (warp-uniform trip count, for the ballot of the compaction)
    for (long long i0 = tid0 - lane; i0 < nr; i0 += stride) {
      const long long i = i0 + lane;
      bool keep = false;
      unsigned e = 0;
      if (i < nr) {
        e = cur ? __ldcg(cur + i) : (unsigned)i;
        if (__ldcg(g.state + e) == kOpen) {
          const uint2 h = g.hits[e];
          const unsigned long long k = __ldcg(g.key + e);
          DepSlot *qa = g.sA + h.x, *qb = g.sB + h.y;
          const bool ready = __ldcg(&qa->t[b]) == k && __ldcg(&qb->t[b]) == k &&
                             (!ties || (__ldcg(&qa->p[b]) == h.y && __ldcg(&qb->p[b]) == h.x));
          qa->t[nb] = kNoKey;  // the next round's slots of both photons start empty
          qa->p[nb] = kNoIdx;
          qb->t[nb] = kNoKey;
          qb->p[nb] = kNoIdx;
          if (ready) {
            const double ra = __ldcg(g.rem_a + h.x), rb = __ldcg(g.rem_b + h.y);
            const double d = ra < rb ? ra : rb;
            g.rem_a[h.x] = __dsub_rn(ra, d);
            g.rem_b[h.y] = __dsub_rn(rb, d);
            g.delta[e] = d;
            g.state[e] = kDone;
          } else {
            keep = true;
          }
        }
      }
      const unsigned m = __ballot_sync(0xffffffffu, keep);
      if (m) {
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(cntn, (unsigned)__popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (keep) listn[base + __popc(m & ((1u << lane) - 1u))] = e;
      }
    }
    if (!phase_sync<kBlock>(g)) return -1;
    nr = (long long)__ldcg(cntn);
    cur = listn;
    if (nr == 0) return 0;
  }
}

// One depletion call.  Values that other threads wrote in an earlier phase
// are read with __ldcg (from L2), so no stale L1 line is seen.
__global__ void __launch_bounds__(kThreads, 1) k_deplete(DepArgs g) {
  const long long gtid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long gstride = (long long)gridDim.x * blockDim.x;
  DepCtl *ctl = g.ctl;

  // slots left dirty by a call that failed: every photon's slots back to empty
  if (__ldcg(g.dirty)) {
    for (long long q = gtid; q < g.na; q += gstride) clear_slot(g.sA + q);
    for (long long q = gtid; q < g.nb; q += gstride) clear_slot(g.sB + q);
    if (!grid_sync(g)) return record_failure(g, TRILENS_ERR_TIMEOUT);
    if (gtid == 0) atomicExch(g.dirty, 0);  // every block has read it
  }

  // t* keys, the input check and round 0's R1
  for (long long e = gtid; e < g.n; e += gstride) {
    const uint2 h = g.hits[e];
    g.delta[e] = 0.0;
    g.state[e] = kDone;
    if ((long long)h.x >= g.na || (long long)h.y >= g.nb) {
      atomicOr(&ctl->flag, kFlagBadInput);
      continue;
    }
    const double ra = g.rem_a[h.x], rb = g.rem_b[h.y];
    if (!(ra >= 0.0) || !(rb >= 0.0)) {
      atomicOr(&ctl->flag, kFlagBadInput);
      continue;
    }
    const unsigned long long k = time_key(dep_tstar(g.A, h.x, g.B, h.y, g.ct));
    g.key[e] = k;
    if (ra > 0.0 && rb > 0.0) {
      g.state[e] = kOpen;
      if ((atomicMin(&g.sA[h.x].t[0], k) == k) | (atomicMin(&g.sB[h.y].t[0], k) == k))
        atomicOr(&ctl->tie[0], 1);
    }
  }
  if (!grid_sync(g)) return record_failure(g, TRILENS_ERR_TIMEOUT);
  if (__ldcg(&ctl->flag) & kFlagBadInput) {  // nothing changed but delta
    if (gtid == 0) atomicExch(g.dirty, 1);
    return record_failure(g, TRILENS_ERR_INVALID);
  }

  long long nr = g.n;            // hits open at the start of round r
  const unsigned *cur = nullptr;  // their list (round 0: every hit, in order)
  long long r = 0;
  int st = run_rounds<false>(g, nr, cur, r, gtid, gstride);
  if (st == 1) {
    // the tail: block 0 alone; the others wait for it at the next barrier
    if (blockIdx.x == 0) {
      st = run_rounds<true>(g, nr, cur, r, threadIdx.x, blockDim.x);
      if (st == -2 && threadIdx.x == 0) atomicOr(&ctl->flag, kFlagRounds);
    }
    if (!grid_sync(g)) return record_failure(g, TRILENS_ERR_TIMEOUT);
    st = (__ldcg(&ctl->flag) & kFlagRounds) ? -2 : 0;
  }
  if (st == -1) return record_failure(g, TRILENS_ERR_TIMEOUT);
  if (st == -2) {
    if (gtid == 0) atomicExch(g.dirty, 1);
    return record_failure(g, TRILENS_ERR_CUDA);
  }

  // both parities' slots of every listed photon back to empty; the sum of
  // delta and the count of hits with delta > 0 over the block's contiguous range
  __shared__ double ss[kThreads / 32];
  __shared__ unsigned long long sc[kThreads / 32];
  {
    const long long lo = g.n * blockIdx.x / gridDim.x, hi = g.n * (blockIdx.x + 1) / gridDim.x;
    double s = 0.0;
    unsigned long long c = 0;
    for (long long e = lo + threadIdx.x; e < hi; e += blockDim.x) {
      const uint2 h = g.hits[e];
      clear_slot(g.sA + h.x);
      clear_slot(g.sB + h.y);
      const double d = __ldcg(g.delta + e);
      s = __dadd_rn(s, d);
      c += d > 0.0;
    }
    block_sum(s, c, ss, sc);
    if (threadIdx.x == 0) {
      g.psum[blockIdx.x] = s;
      g.pcnt[blockIdx.x] = c;
    }
  }
  if (!grid_sync(g)) return record_failure(g, TRILENS_ERR_TIMEOUT);
  if (blockIdx.x == 0) {
    __syncthreads();  // ss, sc reused
    double s = 0.0;
    unsigned long long c = 0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
      s = __dadd_rn(s, __ldcg(g.psum + k));
      c += __ldcg(g.pcnt + k);
    }
    block_sum(s, c, ss, sc);
    if (threadIdx.x == 0) {
      g.out->transferred = s;
      g.out->accepted = (int64_t)c;
      g.out->rounds = r + 1;
      // a block that gave up at the last barrier after it had been passed
      // left nothing undone; any earlier give-up stops block 0 before here
      g.out->status = TRILENS_OK;
    }
  }
}

}  // namespace

// Workspace of a context's depletion calls (allocated on first use).
struct DepState {
  int64_t na = 0, nb = 0;
  DepSlot *sA = nullptr, *sB = nullptr;
  DepPhoton *phA = nullptr, *phB = nullptr;
  long long cap = 0;
  unsigned long long *key = nullptr;
  uint8_t *state = nullptr;
  double *delta = nullptr;  // used when the caller passes no delta array
  unsigned *list[2]{};
  int max_blocks = 0;       // co-resident blocks of k_deplete
  double *psum = nullptr;
  unsigned long long *pcnt = nullptr;
  DepCtl *ctl = nullptr;
  int *dirty = nullptr;                    // device, persistent
  trilens_deplete_out *out = nullptr;      // device: the synchronous call's record
  trilens_deplete_out *out_host = nullptr;  // pinned
};

static void dep_free_hits(DepState *d) {
  cudaFree(d->key);
  cudaFree(d->state);
  cudaFree(d->delta);
  cudaFree(d->list[0]);
  cudaFree(d->list[1]);
  d->key = nullptr;
  d->state = nullptr;
  d->delta = nullptr;
  d->list[0] = d->list[1] = nullptr;
  d->cap = 0;
}

static void dep_free_bufs(DepState *d) {
  cudaFree(d->sA);
  cudaFree(d->sB);
  cudaFree(d->phA);
  cudaFree(d->phB);
  dep_free_hits(d);
  cudaFree(d->psum);
  cudaFree(d->pcnt);
  cudaFree(d->ctl);
  cudaFree(d->dirty);
  cudaFree(d->out);
  cudaFreeHost(d->out_host);
}

void deplete_free(trilens_ctx *c) {
  if (!c->dep) return;
  dep_free_bufs(c->dep);
  delete c->dep;
  c->dep = nullptr;
}

static int dep_prepare(trilens_ctx *c, int64_t n_hits) {
  if (!c->dep) {
    c->dep = new DepState();
    DepState &d = *c->dep;
    d.na = c->beam[0].n;
    d.nb = c->beam[1].n;
    CK(dalloc(&d.sA, (size_t)std::max<int64_t>(d.na, 1)));
    CK(dalloc(&d.sB, (size_t)std::max<int64_t>(d.nb, 1)));
    CK(cudaMemsetAsync(d.sA, 0xff, sizeof(DepSlot) * (size_t)d.na, c->stream));
    CK(cudaMemsetAsync(d.sB, 0xff, sizeof(DepSlot) * (size_t)d.nb, c->stream));
    CK(dalloc(&d.phA, (size_t)std::max<int64_t>(d.na, 1)));
    CK(dalloc(&d.phB, (size_t)std::max<int64_t>(d.nb, 1)));
    k_dep_pack<<<4 * std::max(c->n_sm, 1), 256, 0, c->stream>>>(c->beam[0], c->beam[1], d.phA,
                                                                 d.phB);
    CK(cudaGetLastError());
    int per_sm = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_deplete, kThreads, 0));
    if (per_sm < 1) return fail(c, TRILENS_ERR_CUDA, "deplete: the kernel does not fit an SM");
    d.max_blocks = std::min(per_sm, 2) * std::max(c->n_sm, 1);
    CK(dalloc(&d.psum, (size_t)d.max_blocks));
    CK(dalloc(&d.pcnt, (size_t)d.max_blocks));
    CK(dalloc(&d.ctl, 1));
    CK(dalloc(&d.dirty, 1));
    CK(cudaMemsetAsync(d.dirty, 0, sizeof(int), c->stream));
    CK(dalloc(&d.out, 1));
    CK(cudaMallocHost((void **)&d.out_host, sizeof(trilens_deplete_out)));
  }
  DepState &d = *c->dep;
  if (n_hits > d.cap) {
    const long long nc = std::min<long long>(
        std::max<long long>(n_hits + n_hits / 4 + 1024, 2 * d.cap), (1ll << 32) - 1);
    dep_free_hits(&d);
    CK(dalloc(&d.key, (size_t)nc));
    CK(dalloc(&d.state, (size_t)nc));
    CK(dalloc(&d.delta, (size_t)nc));
    CK(dalloc(&d.list[0], (size_t)nc));
    CK(dalloc(&d.list[1], (size_t)nc));
    d.cap = nc;
  }
  return TRILENS_OK;
}

// Enqueues one call on the context's stream; its record goes to `out` (device).
static int dep_launch(trilens_ctx *c, int64_t step, const uint32_t *hits, int64_t n_hits,
                      double *rem_a, double *rem_b, double *delta, trilens_deplete_out *out) {
  DepState &d = *c->dep;
  cudaStream_t s = c->stream;
  DepArgs g{};
  g.na = d.na;
  g.nb = d.nb;
  g.A = d.phA;
  g.B = d.phB;
  g.ct = TL_C * ((double)step * c->p.dt_fs);
  g.hits = reinterpret_cast<const uint2 *>(hits);
  g.n = n_hits;
  g.key = d.key;
  g.state = d.state;
  g.delta = delta ? delta : d.delta;
  g.rem_a = rem_a;
  g.rem_b = rem_b;
  g.sA = d.sA;
  g.sB = d.sB;
  g.list[0] = d.list[0];
  g.list[1] = d.list[1];
  g.psum = d.psum;
  g.pcnt = d.pcnt;
  g.ctl = d.ctl;
  g.dirty = d.dirty;
  g.out = out;
  g.spin = c->p.spin_limit;  // iterations of 64 ns sleeps per barrier wait
  const long long nblk = (n_hits + kThreads - 1) / kThreads;
  const int blocks = (int)std::min<long long>(nblk, d.max_blocks);
  CK(cudaMemsetAsync(d.ctl, 0, sizeof(DepCtl), s));
  void *args[] = {&g};
  CK(cudaLaunchCooperativeKernel((const void *)k_deplete, dim3(blocks), dim3(kThreads), args, 0,
                                 s));
  return TRILENS_OK;
}

static int dep_check_args(trilens_ctx *c, int64_t step, const uint32_t *hits, int64_t n_hits,
                          double *rem_a, double *rem_b) {
  if (!c || step < 0 || n_hits < 0 || n_hits >= (1ll << 32)) return TRILENS_ERR_INVALID;
  if (n_hits == 0) return TRILENS_OK;
  if (!hits || !rem_a || !rem_b)
    return fail(c, TRILENS_ERR_INVALID, "deplete: hits, rem_a and rem_b are required");
  if (cudaSetDevice(c->device) != cudaSuccess)
    return fail(c, TRILENS_ERR_CUDA, "deplete: cudaSetDevice failed");
  return dep_prepare(c, n_hits);
}

extern "C" int trilens_deplete_step(trilens_ctx *c, int64_t step, const uint32_t *hits,
                                    int64_t n_hits, double *rem_a, double *rem_b, double *delta,
                                    int64_t *n_accepted, double *transferred) {
  int rc = dep_check_args(c, step, hits, n_hits, rem_a, rem_b);
  if (rc != TRILENS_OK) return rc;
  if (n_accepted) *n_accepted = 0;
  if (transferred) *transferred = 0.0;
  if (n_hits == 0) return TRILENS_OK;
  DepState &d = *c->dep;
  rc = dep_launch(c, step, hits, n_hits, rem_a, rem_b, delta, d.out);
  if (rc != TRILENS_OK) return rc;
  CK(cudaMemcpyAsync(d.out_host, d.out, sizeof(trilens_deplete_out), cudaMemcpyDeviceToHost,
                     c->stream));
  CK(cudaStreamSynchronize(c->stream));
  const trilens_deplete_out o = *d.out_host;
  switch (o.status) {
    case TRILENS_OK:
      break;
    case TRILENS_ERR_INVALID:
      return fail(c, TRILENS_ERR_INVALID,
                  "deplete: a hit index is out of range or a remaining weight is negative or NaN");
    case TRILENS_ERR_TIMEOUT:
      return fail(c, TRILENS_ERR_TIMEOUT, "deplete: a grid barrier wait reached spin_limit=%lld",
                  (long long)c->p.spin_limit);
    default:
      return fail(c, TRILENS_ERR_CUDA, "deplete: hits still open after every round");
  }
  if (transferred) *transferred = o.transferred;
  if (n_accepted) *n_accepted = o.accepted;
  c->dep_rounds = o.rounds;
  return TRILENS_OK;
}

extern "C" int trilens_deplete_step_async(trilens_ctx *c, int64_t step, const uint32_t *hits,
                                          int64_t n_hits, double *rem_a, double *rem_b,
                                          double *delta, trilens_deplete_out *out) {
  if (!out || ((uintptr_t)out & 7u)) return TRILENS_ERR_INVALID;
  int rc = dep_check_args(c, step, hits, n_hits, rem_a, rem_b);
  if (rc != TRILENS_OK) return rc;
  if (n_hits == 0) {  // an all-zero record: nothing taken, status OK
    CK(cudaMemsetAsync(out, 0, sizeof(trilens_deplete_out), c->stream));
    return TRILENS_OK;
  }
  return dep_launch(c, step, hits, n_hits, rem_a, rem_b, delta, out);
}

extern "C" int trilens_deplete_rounds(trilens_ctx *c, int64_t *rounds) {
  if (!c || !rounds) return TRILENS_ERR_INVALID;
  *rounds = c->dep_rounds;
  return TRILENS_OK;
}
