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
// hit of that round touches.  Each round:
//   R1  hits whose photon is used up take 0; the others take part in an
//       atomicMin of their time key at both photons;
//   R2  among the hits holding that minimum, an atomicMin of the partner index;
//   R3  a hit holding both minima at both photons is resolved; the others
//       clear the other round's slots of their photons and are counted.
// The globally earliest unresolved hit is always resolved, so a step of n
// hits needs at most n rounds; the host runs rounds in batches of 8 and reads
// the count after each batch (rounds after the last one with open hits return
// at once).  No kernel waits on another block.
//
// t* is computed with the operations of the exact decision (FP64, explicit
// round-to-nearest), so the order is the one the FP64 definition gives.
#include "tl_ctx.h"

namespace {

constexpr unsigned long long kNoKey = ~0ull;
constexpr unsigned kNoIdx = ~0u;
constexpr int kThreads = 256;
constexpr int kRoundsPerBatch = 8;

enum : uint8_t { kOpen = 0, kDone = 1, kBad = 2 };

struct DepArgs {
  TLBeam A, B;
  double ct;
  const uint2 *hits;
  long long n;
  unsigned long long *key;
  uint8_t *state;
  double *delta;
  double *rem_a, *rem_b;
  unsigned long long *tA[2], *tB[2];
  unsigned *pA[2], *pB[2];
  int *ctr;  // [0], [1]: hits left open after a round (by round parity); [2]: bad input;
             // [3]: rounds that had open hits
};

// t* of input photons i of A and j of B at c t_k = ct: the operations of the
// exact decision (Eq. CollDet's closest approach), infinity for parallel motion.
__device__ __forceinline__ double dep_tstar(const TLBeam &A, uint32_t i, const TLBeam &B,
                                            uint32_t j, double ct) {
  const double dxi = A.dx[i], dyi = A.dy[i], dzi = A.dz[i];
  const double dxj = B.dx[j], dyj = B.dy[j], dzj = B.dz[j];
  double vx = __dmul_rn(TL_C, __dsub_rn(dxi, dxj));
  double vy = __dmul_rn(TL_C, __dsub_rn(dyi, dyj));
  double vz = __dmul_rn(TL_C, __dsub_rn(dzi, dzj));
  double vv = __dadd_rn(__dadd_rn(__dmul_rn(vx, vx), __dmul_rn(vy, vy)), __dmul_rn(vz, vz));
  if (vv == 0.0) return __longlong_as_double(0x7ff0000000000000LL);
  double px = __dsub_rn(__dadd_rn(A.px[i], __dmul_rn(ct, dxi)), __dadd_rn(B.px[j], __dmul_rn(ct, dxj)));
  double py = __dsub_rn(__dadd_rn(A.py[i], __dmul_rn(ct, dyi)), __dadd_rn(B.py[j], __dmul_rn(ct, dyj)));
  double pz = __dsub_rn(__dadd_rn(A.pz[i], __dmul_rn(ct, dzi)), __dadd_rn(B.pz[j], __dmul_rn(ct, dzj)));
  double pv = __dadd_rn(__dadd_rn(__dmul_rn(px, vx), __dmul_rn(py, vy)), __dmul_rn(pz, vz));
  return __ddiv_rn(-pv, vv);
}

// x < y  <=>  time_key(x) < time_key(y) for non-NaN doubles; -0 and +0 equal
__device__ __forceinline__ unsigned long long time_key(double t) {
  if (t == 0.0) t = 0.0;
  const unsigned long long b = (unsigned long long)__double_as_longlong(t);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__global__ void __launch_bounds__(kThreads) k_dep_init(DepArgs g) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    g.ctr[0] = 0;
    g.ctr[1] = 1;  // round 0 reads slot 1: non-zero, so it runs
  }
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < g.n;
       e += (long long)gridDim.x * blockDim.x) {
    const uint2 h = g.hits[e];
    g.delta[e] = 0.0;
    if ((long long)h.x >= g.A.n || (long long)h.y >= g.B.n || !(g.rem_a[h.x] >= 0.0) ||
        !(g.rem_b[h.y] >= 0.0)) {
      g.state[e] = kBad;
      atomicOr(&g.ctr[2], 1);
      continue;
    }
    g.key[e] = time_key(dep_tstar(g.A, h.x, g.B, h.y, g.ct));
    g.state[e] = kOpen;
  }
}

// R1: used-up photons; minimum time key at both photons
__global__ void __launch_bounds__(kThreads) k_dep_min_time(DepArgs g, int r, int round) {
  if (g.ctr[2]) return;  // bad input: no round changes anything
  const int prev = g.ctr[(r + 1) & 1];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    g.ctr[r & 1] = 0;
    if (prev) g.ctr[3] = round + 1;
  }
  if (prev == 0) return;
  const int b = r & 1;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < g.n;
       e += (long long)gridDim.x * blockDim.x) {
    if (g.state[e] != kOpen) continue;
    const uint2 h = g.hits[e];
    if (!(g.rem_a[h.x] > 0.0) || !(g.rem_b[h.y] > 0.0)) {
      g.state[e] = kDone;  // delta stays 0
      continue;
    }
    const unsigned long long k = g.key[e];
    atomicMin(&g.tA[b][h.x], k);
    atomicMin(&g.tB[b][h.y], k);
  }
}

// R2: among the hits at the minimum time of a photon, the smallest partner
__global__ void __launch_bounds__(kThreads) k_dep_min_partner(DepArgs g, int r) {
  if (g.ctr[2] || g.ctr[(r + 1) & 1] == 0) return;
  const int b = r & 1;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < g.n;
       e += (long long)gridDim.x * blockDim.x) {
    if (g.state[e] != kOpen) continue;
    const uint2 h = g.hits[e];
    const unsigned long long k = g.key[e];
    if (g.tA[b][h.x] == k) atomicMin(&g.pA[b][h.x], h.y);
    if (g.tB[b][h.y] == k) atomicMin(&g.pB[b][h.y], h.x);
  }
}

// R3: resolve the hits that are earliest at both photons
__global__ void __launch_bounds__(kThreads) k_dep_resolve(DepArgs g, int r) {
  if (g.ctr[2] || g.ctr[(r + 1) & 1] == 0) return;
  const int b = r & 1, nb = b ^ 1;
  int open = 0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < g.n;
       e += (long long)gridDim.x * blockDim.x) {
    if (g.state[e] != kOpen) continue;
    const uint2 h = g.hits[e];
    const unsigned long long k = g.key[e];
    g.tA[nb][h.x] = kNoKey;  // the next round's slots of both photons start empty
    g.pA[nb][h.x] = kNoIdx;
    g.tB[nb][h.y] = kNoKey;
    g.pB[nb][h.y] = kNoIdx;
    const bool ready = g.tA[b][h.x] == k && g.pA[b][h.x] == h.y && g.tB[b][h.y] == k &&
                       g.pB[b][h.y] == h.x;
    if (ready) {
      const double ra = g.rem_a[h.x], rb = g.rem_b[h.y];
      const double d = ra < rb ? ra : rb;
      g.rem_a[h.x] = __dsub_rn(ra, d);
      g.rem_b[h.y] = __dsub_rn(rb, d);
      g.delta[e] = d;
      g.state[e] = kDone;
    } else {
      ++open;
    }
  }
  for (int o = 16; o > 0; o >>= 1) open += __shfl_down_sync(0xffffffffu, open, o);
  if ((threadIdx.x & 31) == 0 && open) atomicAdd(&g.ctr[b], open);
}

// both rounds' slots of every photon of the list back to empty
__global__ void __launch_bounds__(kThreads) k_dep_clear(DepArgs g) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < g.n;
       e += (long long)gridDim.x * blockDim.x) {
    if (g.state[e] == kBad) continue;
    const uint2 h = g.hits[e];
    for (int b = 0; b < 2; ++b) {
      g.tA[b][h.x] = kNoKey;
      g.pA[b][h.x] = kNoIdx;
      g.tB[b][h.y] = kNoKey;
      g.pB[b][h.y] = kNoIdx;
    }
  }
}

// Sum of delta and number of hits with delta > 0: block k sums the k-th of
// gridDim.x contiguous ranges with a fixed reduction tree; k_dep_sum_final
// adds the partial sums in a fixed order, so the result is reproducible.
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

__global__ void __launch_bounds__(kThreads) k_dep_sum(const double *delta, long long n,
                                                      double *ps, unsigned long long *pc) {
  __shared__ double ss[kThreads / 32];
  __shared__ unsigned long long sc[kThreads / 32];
  const long long lo = n * blockIdx.x / gridDim.x, hi = n * (blockIdx.x + 1) / gridDim.x;
  double s = 0.0;
  unsigned long long c = 0;
  for (long long e = lo + threadIdx.x; e < hi; e += blockDim.x) {
    const double d = delta[e];
    s = __dadd_rn(s, d);
    c += d > 0.0;
  }
  block_sum(s, c, ss, sc);
  if (threadIdx.x == 0) {
    ps[blockIdx.x] = s;
    pc[blockIdx.x] = c;
  }
}

__global__ void __launch_bounds__(kThreads) k_dep_sum_final(const double *ps,
                                                            const unsigned long long *pc, int m,
                                                            double *out_s,
                                                            unsigned long long *out_c) {
  __shared__ double ss[kThreads / 32];
  __shared__ unsigned long long sc[kThreads / 32];
  double s = 0.0;
  unsigned long long c = 0;
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    s = __dadd_rn(s, ps[k]);
    c += pc[k];
  }
  block_sum(s, c, ss, sc);
  if (threadIdx.x == 0) {
    *out_s = s;
    *out_c = c;
  }
}

}  // namespace

// Workspace of a context's depletion calls (allocated on first use).
struct DepState {
  int64_t na = 0, nb = 0;
  unsigned long long *tA[2]{}, *tB[2]{};
  unsigned *pA[2]{}, *pB[2]{};
  long long cap = 0;
  unsigned long long *key = nullptr;
  uint8_t *state = nullptr;
  double *delta = nullptr;  // used when the caller passes no delta array
  int *ctr = nullptr;
  double *psum = nullptr;
  unsigned long long *pcnt = nullptr;
  double *out_s = nullptr;
  unsigned long long *out_c = nullptr;
  int part_cap = 0;
  int *ctr_host = nullptr;      // pinned: ctr[0..2]
  double *res_host = nullptr;   // pinned: sum, count bits
  bool dirty = true;            // photon slots must be cleared before use
};

static void dep_free_bufs(DepState *d) {
  for (int b = 0; b < 2; ++b) {
    cudaFree(d->tA[b]);
    cudaFree(d->tB[b]);
    cudaFree(d->pA[b]);
    cudaFree(d->pB[b]);
  }
  cudaFree(d->key);
  cudaFree(d->state);
  cudaFree(d->delta);
  cudaFree(d->ctr);
  cudaFree(d->psum);
  cudaFree(d->pcnt);
  cudaFree(d->out_s);
  cudaFree(d->out_c);
  cudaFreeHost(d->ctr_host);
  cudaFreeHost(d->res_host);
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
    for (int b = 0; b < 2; ++b) {
      CK(dalloc(&d.tA[b], (size_t)d.na));
      CK(dalloc(&d.pA[b], (size_t)d.na));
      CK(dalloc(&d.tB[b], (size_t)d.nb));
      CK(dalloc(&d.pB[b], (size_t)d.nb));
    }
    CK(dalloc(&d.ctr, 4));
    CK(cudaMemsetAsync(d.ctr, 0, 4 * sizeof(int), c->stream));
    d.part_cap = 4 * std::max(c->n_sm, 1);
    CK(dalloc(&d.psum, (size_t)d.part_cap));
    CK(dalloc(&d.pcnt, (size_t)d.part_cap));
    CK(dalloc(&d.out_s, 1));
    CK(dalloc(&d.out_c, 1));
    CK(cudaMallocHost((void **)&d.ctr_host, 4 * sizeof(int)));
    CK(cudaMallocHost((void **)&d.res_host, 2 * sizeof(double)));
  }
  DepState &d = *c->dep;
  if (d.dirty) {
    for (int b = 0; b < 2; ++b) {
      CK(cudaMemsetAsync(d.tA[b], 0xff, sizeof(unsigned long long) * (size_t)d.na, c->stream));
      CK(cudaMemsetAsync(d.pA[b], 0xff, sizeof(unsigned) * (size_t)d.na, c->stream));
      CK(cudaMemsetAsync(d.tB[b], 0xff, sizeof(unsigned long long) * (size_t)d.nb, c->stream));
      CK(cudaMemsetAsync(d.pB[b], 0xff, sizeof(unsigned) * (size_t)d.nb, c->stream));
    }
    d.dirty = false;
  }
  if (n_hits > d.cap) {
    const long long nc = std::max<long long>(n_hits + n_hits / 4 + 1024, 2 * d.cap);
    cudaFree(d.key);
    cudaFree(d.state);
    cudaFree(d.delta);
    d.key = nullptr;
    d.state = nullptr;
    d.delta = nullptr;
    d.cap = 0;
    CK(dalloc(&d.key, (size_t)nc));
    CK(dalloc(&d.state, (size_t)nc));
    CK(dalloc(&d.delta, (size_t)nc));
    d.cap = nc;
  }
  return TRILENS_OK;
}

static int dep_run(trilens_ctx *c, int64_t step, const uint32_t *hits, int64_t n_hits,
                   double *rem_a, double *rem_b, double *delta, int64_t *rounds_out,
                   int64_t *n_accepted, double *transferred) {
  DepState &d = *c->dep;
  cudaStream_t s = c->stream;
  DepArgs g{};
  g.A = c->beam[0];
  g.B = c->beam[1];
  g.ct = TL_C * ((double)step * c->p.dt_fs);
  g.hits = reinterpret_cast<const uint2 *>(hits);
  g.n = n_hits;
  g.key = d.key;
  g.state = d.state;
  g.delta = delta ? delta : d.delta;
  g.rem_a = rem_a;
  g.rem_b = rem_b;
  for (int b = 0; b < 2; ++b) {
    g.tA[b] = d.tA[b];
    g.tB[b] = d.tB[b];
    g.pA[b] = d.pA[b];
    g.pB[b] = d.pB[b];
  }
  g.ctr = d.ctr;
  const long long nblk = (n_hits + kThreads - 1) / kThreads;
  const int blocks = (int)std::min<long long>(nblk, 8ll * std::max(c->n_sm, 1));
  CK(cudaMemsetAsync(d.ctr, 0, 4 * sizeof(int), s));
  k_dep_init<<<blocks, kThreads, 0, s>>>(g);
  CK(cudaGetLastError());
  // rounds, in batches; at most n_hits rounds have work.  Bad input (found by
  // the init) stops every round kernel, and is reported after the first batch.
  int64_t r = 0;
  const int64_t max_rounds = n_hits + kRoundsPerBatch;
  for (;;) {
    for (int q = 0; q < kRoundsPerBatch; ++q, ++r) {
      k_dep_min_time<<<blocks, kThreads, 0, s>>>(g, (int)(r & 1), (int)std::min<int64_t>(r, 1 << 30));
      k_dep_min_partner<<<blocks, kThreads, 0, s>>>(g, (int)(r & 1));
      k_dep_resolve<<<blocks, kThreads, 0, s>>>(g, (int)(r & 1));
    }
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(d.ctr_host, d.ctr, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (d.ctr_host[2])
      return fail(c, TRILENS_ERR_INVALID,
                  "deplete: a hit index is out of range or a remaining weight is negative or NaN");
    if (d.ctr_host[(r - 1) & 1] == 0) break;
    if (r >= max_rounds) {
      d.dirty = true;
      return fail(c, TRILENS_ERR_CUDA, "deplete: %lld hits still open after %lld rounds",
                  (long long)d.ctr_host[(r - 1) & 1], (long long)r);
    }
  }
  k_dep_clear<<<blocks, kThreads, 0, s>>>(g);
  const int parts = (int)std::min<long long>(std::max<long long>(nblk, 1), d.part_cap);
  k_dep_sum<<<parts, kThreads, 0, s>>>(g.delta, n_hits, d.psum, d.pcnt);
  k_dep_sum_final<<<1, kThreads, 0, s>>>(d.psum, d.pcnt, parts, d.out_s, d.out_c);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(&d.res_host[0], d.out_s, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&d.res_host[1], d.out_c, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                     s));
  CK(cudaStreamSynchronize(s));
  if (transferred) *transferred = d.res_host[0];
  if (n_accepted) {
    unsigned long long cnt;
    memcpy(&cnt, &d.res_host[1], sizeof cnt);
    *n_accepted = (int64_t)cnt;
  }
  if (rounds_out) *rounds_out = d.ctr_host[3];
  return TRILENS_OK;
}

extern "C" int trilens_deplete_step(trilens_ctx *c, int64_t step, const uint32_t *hits,
                                    int64_t n_hits, double *rem_a, double *rem_b, double *delta,
                                    int64_t *n_accepted, double *transferred) {
  if (!c || step < 0 || n_hits < 0 || n_hits >= (1ll << 32)) return TRILENS_ERR_INVALID;
  if (n_accepted) *n_accepted = 0;
  if (transferred) *transferred = 0.0;
  if (n_hits == 0) return TRILENS_OK;
  if (!hits || !rem_a || !rem_b)
    return fail(c, TRILENS_ERR_INVALID, "deplete: hits, rem_a and rem_b are required");
  if (cudaSetDevice(c->device) != cudaSuccess)
    return fail(c, TRILENS_ERR_CUDA, "deplete: cudaSetDevice failed");
  int rc = dep_prepare(c, n_hits);
  if (rc != TRILENS_OK) return rc;
  int64_t rounds = 0;
  rc = dep_run(c, step, hits, n_hits, rem_a, rem_b, delta, &rounds, n_accepted, transferred);
  if (rc == TRILENS_OK) c->dep_rounds = rounds;
  else c->dep->dirty = true;  // clear every photon slot before the next call
  return rc;
}

extern "C" int trilens_deplete_rounds(trilens_ctx *c, int64_t *rounds) {
  if (!c || !rounds) return TRILENS_ERR_INVALID;
  *rounds = c->dep_rounds;
  return TRILENS_OK;
}
