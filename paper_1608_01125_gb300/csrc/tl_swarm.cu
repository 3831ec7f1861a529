// tl_swarm.cu -- the IP regime (Sec. 2.2): macro-photons split into swarms of
// real photons.
//
// A macro-photon (MP) of integer weight w stands for w real photons with its
// energy and direction spread as evenly as possible over its volume, taken as
// an axis-aligned cube of side h (one h per beam) centred on the MP: photon k
// sits at p0 + h u_k, u_k,d = frac(0.5 + k alpha_d) - 0.5, alpha = (1/g, 1/g^2,
// 1/g^3), g the real root > 1 of x^4 = x + 1 (Roberts' R_3 low-discrepancy
// sequence; u_0 = 0, so a weight-1 MP is its own photon).  The paper splits two
// MPs when they collide and builds an octree over each swarm for that
// collision; here the MPs that can collide at all during a run are marked
// first, their swarms are written out as real photons, and the real photons go
// through the exact path (Morton LBVH, dual traversal, FP64 decision), which
// finds every real-photon pair of every colliding MP pair at once.
//
//   k_swarm_mark      all MP pairs: can a photon of MP i meet a photon of MP j
//                     during the run's time window?  (s > 1 up to a relative
//                     1e-9, and the centres' closest approach within the window
//                     at most r_max + the swarms' half-diagonals, with margins
//                     for rounding; an FP32 pre-test rejects clear misses, FP64
//                     decides).  A superset of the pairs with real hits, so the
//                     hit set does not depend on it.
//   k_swarm_block_sums, k_swarm_scan_sums, k_swarm_offsets
//                     exclusive prefix sum of the marked MPs' weights.
//   k_swarm_expand    photon q of the expanded beam: its MP by binary search in
//                     the offsets, k = q - offset, position p0 + h u_k.
#include "tl_ctx.h"

namespace {

constexpr int kThreads = 256;
constexpr int kTile = 256;
constexpr int kMarkB = 1024;  // MPs of B per block of the marking
constexpr int kScanItems = 4;                     // per thread
constexpr int kScanBlock = kThreads * kScanItems;  // items per block

// 1/g, 1/g^2, 1/g^3 as the nearest doubles, g^4 = g + 1 (Roberts' R_3)
__constant__ double kR3[3] = {0.81917251339616448, 0.67104360670378926, 0.5497004779019703};

struct MarkArgs {
  TLBeam A, B;
  double T0, T1;   // the run's time window [fs]
  double lim2;     // (r_max + half-diagonals)^2 with margins [um^2]
  double s_floor;  // (2 m_e c^2) m_e c^2 (1 - 1e-9)
  uint8_t *mark_a, *mark_b;
};

// Block (x, y): 256 MPs of A (one per thread) against the y-th slice of kMarkB
// MPs of B, staged in shared memory 256 at a time.  A pair is skipped when both
// of its MPs are already marked (it could only set marks that are set); a stale
// mark read as 0 only costs a test.  Marks found in the block go to the staged
// copy too, so its other warps skip those MPs of B.  Each test first rejects pairs that are
// clearly apart in FP32 (margins 2x on the limit plus 4e-5 of the squared
// lengths involved, far above FP32 rounding), then decides in FP64.
__global__ void __launch_bounds__(kThreads) k_swarm_mark(MarkArgs g) {
  __shared__ double sp[3][kTile], sd[3][kTile], sE[kTile];
  __shared__ float sf[3][kTile];
  __shared__ volatile uint8_t sm[kTile];  // B's marks, also set here as they are found
  const long long i = blockIdx.x * (long long)kThreads + threadIdx.x;
  const bool live = i < g.A.n;
  double pi[3] = {0., 0., 0.}, di[3] = {0., 0., 0.}, Ei = 0.;
  float fi[3] = {0.f, 0.f, 0.f};
  bool known = false;
  if (live) {
    pi[0] = g.A.px[i]; pi[1] = g.A.py[i]; pi[2] = g.A.pz[i];
    di[0] = g.A.dx[i]; di[1] = g.A.dy[i]; di[2] = g.A.dz[i];
    fi[0] = (float)di[0]; fi[1] = (float)di[1]; fi[2] = (float)di[2];
    Ei = g.A.E[i];
    known = g.mark_a[i] != 0;
  }
  const double Tm = fmax(fabs(g.T0), fabs(g.T1));
  const float T0f = (float)g.T0, T1f = (float)g.T1, Tmf = (float)Tm;
  const float lim2f = 2.0f * (float)g.lim2;
  bool found = false;
  const long long jb = blockIdx.y * (long long)kMarkB;
  const long long je = min((long long)g.B.n, jb + kMarkB);
  for (long long j0 = jb; j0 < je; j0 += kTile) {
    __syncthreads();
    const long long jj = j0 + threadIdx.x;
    if (jj < je) {
      sp[0][threadIdx.x] = g.B.px[jj]; sp[1][threadIdx.x] = g.B.py[jj];
      sp[2][threadIdx.x] = g.B.pz[jj];
      sd[0][threadIdx.x] = g.B.dx[jj]; sd[1][threadIdx.x] = g.B.dy[jj];
      sd[2][threadIdx.x] = g.B.dz[jj];
      sf[0][threadIdx.x] = (float)sd[0][threadIdx.x];
      sf[1][threadIdx.x] = (float)sd[1][threadIdx.x];
      sf[2][threadIdx.x] = (float)sd[2][threadIdx.x];
      sE[threadIdx.x] = g.B.E[jj];
      sm[threadIdx.x] = g.mark_b[jj];
    }
    __syncthreads();
    const int m = (int)min((long long)kTile, je - j0);
    if (!live) continue;
    for (int t = 0; t < m; ++t) {
      if (known && sm[t]) continue;
      const double px = pi[0] - sp[0][t], py = pi[1] - sp[1][t], pz = pi[2] - sp[2][t];
      // FP32: reject pairs clearly apart.  Only when |v| >= 0.1 um/fs, so that the
      // rounding of the directions moves v by less than 1e-6 of itself; the
      // squared distance is then off by well under 1e-5 (|p|^2 + |v|^2 T^2).
      const float ux = (float)TL_C * (fi[0] - sf[0][t]);
      const float uy = (float)TL_C * (fi[1] - sf[1][t]);
      const float uz = (float)TL_C * (fi[2] - sf[2][t]);
      const float af = ux * ux + uy * uy + uz * uz;
      if (af >= 0.01f) {
        const float qx = (float)px, qy = (float)py, qz = (float)pz;
        const float bf = qx * ux + qy * uy + qz * uz;
        const float ppf = qx * qx + qy * qy + qz * qz;
        const float limf = lim2f + 4e-5f * (ppf + af * Tmf * Tmf);
        if (-bf <= af * T0f || -bf >= af * T1f) {
          const float T = (-bf <= af * T0f) ? T0f : T1f;
          const float ex = qx + T * ux, ey = qy + T * uy, ez = qz + T * uz;
          if (ex * ex + ey * ey + ez * ez > limf) continue;
        } else {
          const float cx = qy * uz - qz * uy, cy = qz * ux - qx * uz, cz = qx * uy - qy * ux;
          if (cx * cx + cy * cy + cz * cz > limf * af) continue;
        }
      }
      const double cs = di[0] * sd[0][t] + di[1] * sd[1][t] + di[2] * sd[2][t];
      if (!(Ei * sE[t] * (1.0 - cs) > g.s_floor)) continue;  // below threshold
      const double vx = TL_C * (di[0] - sd[0][t]);
      const double vy = TL_C * (di[1] - sd[1][t]);
      const double vz = TL_C * (di[2] - sd[2][t]);
      const double a = vx * vx + vy * vy + vz * vz;
      if (a == 0.0) continue;  // parallel: never a hit
      const double b = px * vx + py * vy + pz * vz;
      const double pp = px * px + py * py + pz * pz;
      const double lim = g.lim2 + 1e-13 * (pp + a * Tm * Tm);  // rounding of what follows
      bool cand;
      if (-b <= a * g.T0 || -b >= a * g.T1) {
        // closest approach at an end of the window
        const double T = (-b <= a * g.T0) ? g.T0 : g.T1;
        const double qx = px + T * vx, qy = py + T * vy, qz = pz + T * vz;
        cand = qx * qx + qy * qy + qz * qz <= lim;
      } else {
        // inside: distance^2 = |p x v|^2 / |v|^2
        const double cx = py * vz - pz * vy, cy = pz * vx - px * vz, cz = px * vy - py * vx;
        cand = cx * cx + cy * cy + cz * cz <= lim * a;
      }
      if (cand) {
        found = known = true;
        g.mark_b[j0 + t] = 1;
        sm[t] = 1;  // the block's other warps skip j from now on
      }
    }
  }
  if (found) g.mark_a[i] = 1;
}

__device__ __forceinline__ long long swarm_weight(const TLBeam &mp, const uint8_t *mark,
                                                  long long i, int *bad) {
  const double w = mp.w ? mp.w[i] : 1.0;
  if (!(w >= 1.0 && w < 4294967296.0 && w == floor(w))) {
    atomicOr(bad, 1);
    return 0;
  }
  return mark[i] ? (long long)w : 0;
}

__device__ __forceinline__ long long block_exclusive_scan(long long v, long long *total,
                                                          long long *ws) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  long long x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  if (w == 0) {
    long long s = lane < kThreads / 32 ? ws[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < kThreads / 32) ws[lane] = s;
  }
  __syncthreads();
  const long long before = (w ? ws[w - 1] : 0) + x - v;
  *total = ws[kThreads / 32 - 1];
  __syncthreads();
  return before;
}

__global__ void __launch_bounds__(kThreads) k_swarm_block_sums(TLBeam mp, const uint8_t *mark,
                                                               long long *bsum, int *bad) {
  __shared__ long long ws[kThreads / 32];
  const long long base = blockIdx.x * (long long)kScanBlock + threadIdx.x * kScanItems;
  long long s = 0;
  for (int q = 0; q < kScanItems; ++q)
    if (base + q < mp.n) s += swarm_weight(mp, mark, base + q, bad);
  long long tot;
  block_exclusive_scan(s, &tot, ws);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// one block: bsum[0..nb) -> exclusive prefix sums, bsum[nb] = total
__global__ void __launch_bounds__(kThreads) k_swarm_scan_sums(long long *bsum, long long nb) {
  __shared__ long long ws[kThreads / 32];
  long long carry = 0;
  for (long long c0 = 0; c0 < nb; c0 += kThreads) {
    const long long c = c0 + threadIdx.x;
    const long long v = c < nb ? bsum[c] : 0;
    long long tot;
    const long long ex = block_exclusive_scan(v, &tot, ws);
    if (c < nb) bsum[c] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) bsum[nb] = carry;
}

__global__ void __launch_bounds__(kThreads) k_swarm_offsets(TLBeam mp, const uint8_t *mark,
                                                            const long long *bsum, long long nb,
                                                            long long *offsets, int *bad) {
  __shared__ long long ws[kThreads / 32];
  const long long base = blockIdx.x * (long long)kScanBlock + threadIdx.x * kScanItems;
  long long v[kScanItems], s = 0;
  for (int q = 0; q < kScanItems; ++q) {
    v[q] = base + q < mp.n ? swarm_weight(mp, mark, base + q, bad) : 0;
    s += v[q];
  }
  long long tot;
  long long run = bsum[blockIdx.x] + block_exclusive_scan(s, &tot, ws);
  for (int q = 0; q < kScanItems; ++q) {
    if (base + q < mp.n) offsets[base + q] = run;
    run += v[q];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) offsets[mp.n] = bsum[nb];
}

struct ExpandArgs {
  TLBeam mp;
  double h;
  const long long *offsets;
  long long total;
  double *out[8];  // px py pz dx dy dz E w (w may be null)
  uint32_t *owner, *kof;
};

__global__ void __launch_bounds__(kThreads) k_swarm_expand(ExpandArgs g) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < g.total;
       q += (long long)gridDim.x * blockDim.x) {
    long long lo = 0, hi = g.mp.n;  // offsets[lo] <= q < offsets[hi]
    while (hi - lo > 1) {
      const long long mid = (lo + hi) >> 1;
      if (g.offsets[mid] <= q) lo = mid;
      else hi = mid;
    }
    const long long k = q - g.offsets[lo];
    double u[3];
    for (int d = 0; d < 3; ++d) {
      const double x = __dadd_rn(0.5, __dmul_rn((double)k, kR3[d]));
      u[d] = __dsub_rn(__dsub_rn(x, floor(x)), 0.5);
    }
    g.out[0][q] = __dadd_rn(g.mp.px[lo], __dmul_rn(g.h, u[0]));
    g.out[1][q] = __dadd_rn(g.mp.py[lo], __dmul_rn(g.h, u[1]));
    g.out[2][q] = __dadd_rn(g.mp.pz[lo], __dmul_rn(g.h, u[2]));
    g.out[3][q] = g.mp.dx[lo];
    g.out[4][q] = g.mp.dy[lo];
    g.out[5][q] = g.mp.dz[lo];
    g.out[6][q] = g.mp.E[lo];
    if (g.out[7]) g.out[7][q] = 1.0;
    g.owner[q] = (uint32_t)lo;
    g.kof[q] = (uint32_t)k;
  }
}

bool beam_valid(const trilens_beam *b) {
  if (!b || b->n < 0 || b->n >= (1ll << 32)) return false;
  if (b->n == 0) return true;
  return b->px && b->py && b->pz && b->dx && b->dy && b->dz && b->E;
}

TLBeam to_tl(const trilens_beam *b) {
  TLBeam t;
  t.n = b->n;
  t.px = b->px; t.py = b->py; t.pz = b->pz;
  t.dx = b->dx; t.dy = b->dy; t.dz = b->dz;
  t.E = b->E; t.w = b->w;
  return t;
}

int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  return n;
}

}  // namespace

extern "C" int trilens_swarm_mark(const trilens_beam *a, const trilens_beam *b, double h_a,
                                  double h_b, const trilens_params *p, int64_t first_step,
                                  int64_t steps, uint8_t *mark_a, uint8_t *mark_b,
                                  trilens_stream_t stream) {
  if (!beam_valid(a) || !beam_valid(b) || !p || !(p->dt_fs > 0.0) || !(p->kappa > 0.0) ||
      !(h_a >= 0.0) || !(h_b >= 0.0) || !(h_a < 1e30) || !(h_b < 1e30) || first_step < 0 ||
      steps < 1 || (a->n > 0 && !mark_a) || (b->n > 0 && !mark_b))
    return TRILENS_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  if (a->n > 0 && cudaMemsetAsync(mark_a, 0, (size_t)a->n, s) != cudaSuccess)
    return TRILENS_ERR_CUDA;
  if (b->n > 0 && cudaMemsetAsync(mark_b, 0, (size_t)b->n, s) != cudaSuccess)
    return TRILENS_ERR_CUDA;
  if (a->n == 0 || b->n == 0) return TRILENS_OK;
  MarkArgs g{};
  g.A = to_tl(a);
  g.B = to_tl(b);
  g.T0 = (double)first_step * p->dt_fs;
  g.T1 = (double)(first_step + steps) * p->dt_fs;
  const double rmax = 1e6 * sqrt(p->kappa * tl_sigma_max_bound() / TL_PI);
  const double reach = (rmax + 0.8660254037844387 * (h_a + h_b)) * (1.0 + 1e-6) + 1e-9;
  g.lim2 = reach * reach + 1e-9;
  g.s_floor = (2.0 * TL_MEC2) * TL_MEC2 * (1.0 - 1e-9);
  g.mark_a = mark_a;
  g.mark_b = mark_b;
  const dim3 grid((unsigned)((a->n + kThreads - 1) / kThreads),
                  (unsigned)((b->n + kMarkB - 1) / kMarkB));
  if (grid.y > 65535u) return TRILENS_ERR_INVALID;  // b->n above 2^26 MPs
  k_swarm_mark<<<grid, kThreads, 0, s>>>(g);
  return cudaGetLastError() == cudaSuccess ? TRILENS_OK : TRILENS_ERR_CUDA;
}

extern "C" int trilens_swarm_count(const trilens_beam *mp, const uint8_t *mark, int64_t *offsets,
                                   int64_t *total, trilens_stream_t stream) {
  if (!beam_valid(mp) || !offsets || !total || (mp->n > 0 && !mark)) return TRILENS_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  const long long n = mp->n;
  const long long nb = (n + kScanBlock - 1) / kScanBlock;
  long long *bsum = nullptr;
  int *bad = nullptr;
  int bad_h = 0;
  long long tot_h = 0;
  if (cudaMallocAsync((void **)&bsum, sizeof(long long) * (size_t)(nb + 1), s) != cudaSuccess)
    return TRILENS_ERR_NOMEM;
  int rc = TRILENS_OK;
  if (cudaMallocAsync((void **)&bad, sizeof(int), s) != cudaSuccess) {
    rc = TRILENS_ERR_NOMEM;
  } else if (cudaMemsetAsync(bad, 0, sizeof(int), s) != cudaSuccess) {
    rc = TRILENS_ERR_CUDA;
  } else {
    const TLBeam t = to_tl(mp);
    long long *off = reinterpret_cast<long long *>(offsets);
    if (nb > 0) k_swarm_block_sums<<<(unsigned)nb, kThreads, 0, s>>>(t, mark, bsum, bad);
    k_swarm_scan_sums<<<1, kThreads, 0, s>>>(bsum, nb);
    if (nb > 0) {
      k_swarm_offsets<<<(unsigned)nb, kThreads, 0, s>>>(t, mark, bsum, nb, off, bad);
    } else if (cudaMemsetAsync(off, 0, sizeof(long long), s) != cudaSuccess) {
      rc = TRILENS_ERR_CUDA;
    }
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&tot_h, bsum + nb, sizeof tot_h, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&bad_h, bad, sizeof bad_h, cudaMemcpyDeviceToHost, s) != cudaSuccess)
      rc = TRILENS_ERR_CUDA;
  }
  cudaFreeAsync(bsum, s);
  if (bad) cudaFreeAsync(bad, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return TRILENS_ERR_CUDA;
  if (rc != TRILENS_OK) return rc;
  if (bad_h) return TRILENS_ERR_INVALID;
  *total = tot_h;
  return TRILENS_OK;
}

extern "C" int trilens_swarm_expand(const trilens_beam *mp, double h, const int64_t *offsets,
                                    int64_t total, double *const *out, uint32_t *owner,
                                    uint32_t *index_in_swarm, trilens_stream_t stream) {
  if (!beam_valid(mp) || !offsets || total < 0 || !(h >= 0.0) || !(h < 1e30))
    return TRILENS_ERR_INVALID;
  if (total == 0) return TRILENS_OK;
  if (mp->n == 0 || !out || !owner || !index_in_swarm) return TRILENS_ERR_INVALID;
  for (int k = 0; k < 7; ++k)
    if (!out[k]) return TRILENS_ERR_INVALID;
  ExpandArgs g{};
  g.mp = to_tl(mp);
  g.h = h;
  g.offsets = reinterpret_cast<const long long *>(offsets);
  g.total = total;
  for (int k = 0; k < 8; ++k) g.out[k] = out[k];
  g.owner = owner;
  g.kof = index_in_swarm;
  const int n_sm = sm_count();
  if (n_sm == 0) return TRILENS_ERR_CUDA;
  const long long nblk = (total + kThreads - 1) / kThreads;
  const int blocks = (int)std::min<long long>(nblk, 8ll * n_sm);
  k_swarm_expand<<<blocks, kThreads, 0, (cudaStream_t)stream>>>(g);
  return cudaGetLastError() == cudaSuccess ? TRILENS_OK : TRILENS_ERR_CUDA;
}
