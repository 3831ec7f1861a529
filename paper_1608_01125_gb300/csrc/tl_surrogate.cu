// tl_surrogate.cu -- the statistical regime's node-pair level.
//
// The paper's ST regime treats macro-particles as continuous clouds and
// computes collision rates between whole clouds instead of testing single
// particles (Sec. 2.2).  Here the clouds are the hierarchy's nodes at level
// L (the first node on every path whose Morton prefix is at least L bits, or
// a leaf bucket): the dual traversal stops there and emits overlapping node
// pairs.  For each pair the kernels below gather 24 features (boxes, counts,
// weight sums and energy / direction moments from FP64 prefix sums over the
// Morton-ordered photons), a rate estimate of the ST form, and -- for
// training labels -- the exact yield of the pair, attributed hit by hit.
#include "tl_exact.cuh"
#include "tl_sur.h"

namespace tl {

__device__ __forceinline__ bool is_cut(const CutTree &T, uint32_t ref, int L) {
  return (ref & TL_FLAG) || T.nlev[ref] >= L;
}

__device__ __forceinline__ TLNode load_node(const TLNode *p) {
  const float4 *f = reinterpret_cast<const float4 *>(p);
  TLNode v;
  v.b0 = __ldg(f + 0);
  v.b1 = __ldg(f + 1);
  v.b2 = __ldg(f + 2);
  v.c = __ldg(reinterpret_cast<const int4 *>(f + 3));
  return v;
}

// box, first photon and count of the node a stack reference names
__device__ __forceinline__ void own(const CutTree &T, uint32_t ref, TLBox &box, uint32_t &first,
                                    uint32_t &cnt) {
  uint32_t parent, slot;
  if (ref & TL_FLAG) {
    parent = (ref & ~TL_FLAG) >> 1;
    slot = ref & 1u;
  } else {
    const uint32_t pn = T.parent_node[ref];
    parent = pn >> 1;
    slot = pn & 1u;
  }
  const TLNode v = load_node(T.nodes + parent);
  box = tl_child_box(v, (int)slot);
  cnt = (uint32_t)(slot ? v.c.w : v.c.z);
  const uint32_t cr = (uint32_t)(slot ? v.c.y : v.c.x);
  first = (ref & TL_FLAG) ? (cr & ~TL_FLAG) : T.nfirst[ref];
}

// child `slot` of inner node `ref`: box and stack reference
__device__ __forceinline__ void child(const CutTree &T, uint32_t ref, int slot, TLBox &box,
                                      uint32_t &cref) {
  const TLNode v = load_node(T.nodes + ref);
  box = tl_child_box(v, slot);
  const uint32_t cr = (uint32_t)(slot ? v.c.y : v.c.x);
  cref = (cr & TL_FLAG) ? (TL_FLAG | (ref << 1) | (uint32_t)slot) : cr;
}

// ------------------------------------------------------------ prefix moments

// per photon (sorted order): w, w lnE, w lnE^2, w dx, w dy, w dz; energy and
// direction from the Morton-ordered FP32 SoA (coalesced), only the weight
// gathered from the FP64 input
__device__ __forceinline__ void moments(const TLBeam &B, const float4 *pos, const float4 *dir,
                                        int64_t p, double m[6]) {
  const float4 d = dir[p];
  const double w = B.w ? B.w[__float_as_uint(d.w)] : 1.0;
  const double le = (double)logf(pos[p].w);
  m[0] = w;
  m[1] = w * le;
  m[2] = w * le * le;
  m[3] = w * (double)d.x;
  m[4] = w * (double)d.y;
  m[5] = w * (double)d.z;
}

constexpr int kScanBlock = 1024;

__global__ void __launch_bounds__(256) k_pre_blocks(TLBeam B, const float4 *pos,
                                                    const float4 *dir, int64_t n, double *bsum) {
  __shared__ double sh[8][6];
  double acc[6] = {0, 0, 0, 0, 0, 0};
  const int64_t b0 = (int64_t)blockIdx.x * kScanBlock;
  for (int64_t p = b0 + threadIdx.x; p < b0 + kScanBlock && p < n; p += blockDim.x) {
    double m[6];
    moments(B, pos, dir, p, m);
    for (int c = 0; c < 6; ++c) acc[c] += m[c];
  }
  for (int c = 0; c < 6; ++c)
    for (int off = 16; off; off >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], off);
  if ((threadIdx.x & 31) == 0)
    for (int c = 0; c < 6; ++c) sh[threadIdx.x >> 5][c] = acc[c];
  __syncthreads();
  if (threadIdx.x < 6) {
    double t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w][threadIdx.x];
    bsum[(int64_t)blockIdx.x * 6 + threadIdx.x] = t;
  }
}

// exclusive scan of the block sums in place (one block; sequential per thread chunk)
__global__ void k_pre_scan(double *bsum, int64_t nb) {
  __shared__ double part[1024][6];
  const int64_t per = (nb + blockDim.x - 1) / blockDim.x;
  const int64_t lo = threadIdx.x * per, hi = min(nb, lo + per);
  double run[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t b = lo; b < hi; ++b)
    for (int c = 0; c < 6; ++c) run[c] += bsum[b * 6 + c];
  for (int c = 0; c < 6; ++c) part[threadIdx.x][c] = run[c];
  __syncthreads();
  if (threadIdx.x < 6) {
    double t = 0;
    for (int q = 0; q < (int)blockDim.x; ++q) {
      const double v = part[q][threadIdx.x];
      part[q][threadIdx.x] = t;
      t += v;
    }
  }
  __syncthreads();
  for (int c = 0; c < 6; ++c) run[c] = part[threadIdx.x][c];
  for (int64_t b = lo; b < hi; ++b)
    for (int c = 0; c < 6; ++c) {
      const double v = bsum[b * 6 + c];
      bsum[b * 6 + c] = run[c];
      run[c] += v;
    }
}

// pre[c][p + 1] = sum over photons 0..p; pre[c][0] = 0
__global__ void __launch_bounds__(32) k_pre_fill(TLBeam B, const float4 *pos, const float4 *dir,
                                                 int64_t n, const double *boff, double *pre) {
  // one warp per block of kScanBlock photons, sequential in 32-photon chunks
  const int lane = threadIdx.x;
  const int64_t b0 = (int64_t)blockIdx.x * kScanBlock;
  double run[6];
  for (int c = 0; c < 6; ++c) run[c] = boff[(int64_t)blockIdx.x * 6 + c];
  if (blockIdx.x == 0 && lane == 0)
    for (int c = 0; c < 6; ++c) pre[(int64_t)c * (n + 1)] = 0.0;
  for (int64_t base = b0; base < b0 + kScanBlock && base < n; base += 32) {
    const int64_t p = base + lane;
    double m[6] = {0, 0, 0, 0, 0, 0};
    if (p < n) moments(B, pos, dir, p, m);
    for (int c = 0; c < 6; ++c) {
      double v = m[c];
      for (int off = 1; off < 32; off <<= 1) {
        const double t = __shfl_up_sync(0xffffffffu, v, off);
        if (lane >= off) v += t;
      }
      if (p < n) pre[(int64_t)c * (n + 1) + p + 1] = run[c] + v;
      run[c] += __shfl_sync(0xffffffffu, v, 31);
    }
  }
}

cudaError_t launch_prefix_moments(const TLBeam &B, const float4 *pos, const float4 *dir, int64_t n,
                                  double *bsum, double *pre, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
  k_pre_blocks<<<(unsigned)nb, 256, 0, s>>>(B, pos, dir, n, bsum);
  k_pre_scan<<<1, 1024, 0, s>>>(bsum, nb);
  k_pre_fill<<<(unsigned)nb, 32, 0, s>>>(B, pos, dir, n, bsum, pre);
  return cudaGetLastError();
}

// ------------------------------------------------------------ level-L cut traversal

__device__ __forceinline__ void append(bool pred, uint2 v, uint2 *buf, unsigned *cnt,
                                       unsigned cap, unsigned *status, int lane) {
  const unsigned m = __ballot_sync(0xffffffffu, pred);
  if (!m) return;
  unsigned base = 0;
  if (lane == 0) base = atomicAdd(cnt, (unsigned)__popc(m));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (pred) {
    const unsigned idx = base + __popc(m & ((1u << lane) - 1u));
    if (idx < cap) buf[idx] = v;
    else atomicOr(status, (unsigned)TL_ST_FRONT_OVF);
  }
}

// One breadth-first level: pairs whose both sides are cut nodes are emitted;
// otherwise the non-cut sides are split and the overlapping child pairs go
// to the next level.
__global__ void __launch_bounds__(256) k_cut_level(CutArgs a) {
  const unsigned nin = min(a.counts[0], a.cap);
  const int lane = threadIdx.x & 31;
  const unsigned nround = (nin + 31u) & ~31u;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < nround;
       i += gridDim.x * blockDim.x) {
    const bool valid = i < nin;
    const uint2 pr = valid ? a.in[i] : make_uint2(0u, 0u);
    const bool ca = valid && is_cut(a.A, pr.x, a.L), cb = valid && is_cut(a.B, pr.y, a.L);
    // emit finished pairs
    {
      const bool done = valid && ca && cb;
      const unsigned m = __ballot_sync(0xffffffffu, done);
      if (m) {
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(a.cut_count, (unsigned)__popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (done) {
          const unsigned idx = base + __popc(m & ((1u << lane) - 1u));
          if (idx < a.cut_cap) a.cut[idx] = make_uint4(pr.x, pr.y, 0u, 0u);
          else atomicOr(a.status, (unsigned)TL_ST_FRONT_OVF);
        }
      }
    }
    const bool split = valid && !(ca && cb);
    TLBox ba, bb;
    uint32_t fa = 0, na = 0, fb = 0, nb = 0;
    if (split && ca) own(a.A, pr.x, ba, fa, na);
    if (split && cb) own(a.B, pr.y, bb, fb, nb);
    for (int combo = 0; combo < 4; ++combo) {
      const int ia = combo >> 1, ib = combo & 1;
      bool ok = false;
      uint2 o = make_uint2(0u, 0u);
      if (split && !(ca && ia) && !(cb && ib)) {
        TLBox xa = ba, xb = bb;
        uint32_t ra = pr.x, rb = pr.y;
        if (!ca) child(a.A, pr.x, ia, xa, ra);
        if (!cb) child(a.B, pr.y, ib, xb, rb);
        ok = tl_overlap(xa, xb);
        o = make_uint2(ra, rb);
      }
      append(ok, o, a.out, a.counts + 1, a.cap, a.status, lane);
    }
  }
}

cudaError_t launch_cut_level(const CutArgs &a, int blocks, cudaStream_t s) {
  k_cut_level<<<blocks, 256, 0, s>>>(a);
  return cudaGetLastError();
}

// ------------------------------------------------------------ features

// The ST regime's rate for two clouds (Sec. 2.2, Eq. rate, Eq. reactivity).
// A cloud is a level-L node read as a box of uniform density moving rigidly
// with the mean velocity c dbar: its box at t_k is the node's swept box with
// the step's travel c dt dbar taken off, so that it sweeps the node's box
// over the step.  n_I n_II <sigma v> integrated over the overlap and the step:
//   N = W_A W_B (1e12 kappa sigma(sbar)) c |dbar_A - dbar_B|
//       * int_0^dt V_ov(t) dt / (V_A V_B),
// with the collision area 1e12 kappa sigma [um^2] and sbar from the
// geometric-mean energies and 1 - dbar_A . dbar_B.  V_ov(t) is the product of
// three piecewise-linear overlap lengths: the integral is exact, Simpson's
// rule on each piece between the times where an overlap length changes form.

__device__ __forceinline__ double st_len(double la, double ua, double va, double lb, double ub,
                                         double vb, double t) {
  const double hi = fmin(ua + va * t, ub + vb * t), lo = fmax(la + va * t, lb + vb * t);
  return hi > lo ? hi - lo : 0.0;
}

__device__ __forceinline__ double st_vol(const double *la, const double *ua, const double *va,
                                         const double *lb, const double *ub, const double *vb,
                                         double t) {
  return st_len(la[0], ua[0], va[0], lb[0], ub[0], vb[0], t) *
         st_len(la[1], ua[1], va[1], lb[1], ub[1], vb[1], t) *
         st_len(la[2], ua[2], va[2], lb[2], ub[2], vb[2], t);
}

__device__ double st_overlap_time_integral(const double *la, const double *ua, const double *va,
                                           const double *lb, const double *ub, const double *vb,
                                           double T) {
  double br[14];
  int nb = 0;
  br[nb++] = 0.0;
  br[nb++] = T;
  for (int q = 0; q < 3; ++q) {
    const double w = vb[q] - va[q];
    if (w == 0.0) continue;
    const double c4[4] = {(ua[q] - ub[q]) / w, (la[q] - lb[q]) / w, (ua[q] - lb[q]) / w,
                          (la[q] - ub[q]) / w};
    for (int r = 0; r < 4; ++r)
      if (c4[r] > 0.0 && c4[r] < T) br[nb++] = c4[r];
  }
  for (int i = 1; i < nb; ++i) {  // insertion sort of at most 14 times
    const double v = br[i];
    int j = i - 1;
    while (j >= 0 && br[j] > v) {
      br[j + 1] = br[j];
      --j;
    }
    br[j + 1] = v;
  }
  double I = 0.0, f0 = st_vol(la, ua, va, lb, ub, vb, br[0]);
  for (int i = 0; i + 1 < nb; ++i) {
    const double t0 = br[i], t1 = br[i + 1];
    const double f1 = st_vol(la, ua, va, lb, ub, vb, t1);
    if (t1 > t0) I += (t1 - t0) * (f0 + 4.0 * st_vol(la, ua, va, lb, ub, vb, 0.5 * (t0 + t1)) + f1) / 6.0;
    f0 = f1;
  }
  return I;
}

// 24 features per node pair, and the ST rate above (FP64 from the FP32 node
// boxes and the FP64 prefix moments).  L = c dt [um].
__global__ void __launch_bounds__(256) k_features(CutTree A, CutTree B, const uint4 *cut,
                                                  const unsigned *cut_count, unsigned cap,
                                                  float *feat, float *st, double L, double dt,
                                                  double kappa) {
  const unsigned n = min(*cut_count, cap);
  for (unsigned p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const uint4 c = cut[p];
    TLBox ba, bb;
    uint32_t fa, na, fb, nb;
    own(A, c.x, ba, fa, na);
    own(B, c.y, bb, fb, nb);
    double ma[6], mb[6];
    for (int q = 0; q < 6; ++q) {
      ma[q] = A.pre[(int64_t)q * (A.n + 1) + fa + na] - A.pre[(int64_t)q * (A.n + 1) + fa];
      mb[q] = B.pre[(int64_t)q * (B.n + 1) + fb + nb] - B.pre[(int64_t)q * (B.n + 1) + fb];
    }
    float *f = feat + (size_t)p * 24;
    const float cax = 0.5f * (ba.lx + ba.hx), cay = 0.5f * (ba.ly + ba.hy), caz = 0.5f * (ba.lz + ba.hz);
    const float cbx = 0.5f * (bb.lx + bb.hx), cby = 0.5f * (bb.ly + bb.hy), cbz = 0.5f * (bb.lz + bb.hz);
    f[0] = cbx - cax;
    f[1] = cby - cay;
    f[2] = cbz - caz;
    f[3] = 0.5f * (ba.hx - ba.lx);
    f[4] = 0.5f * (ba.hy - ba.ly);
    f[5] = 0.5f * (ba.hz - ba.lz);
    f[6] = 0.5f * (bb.hx - bb.lx);
    f[7] = 0.5f * (bb.hy - bb.ly);
    f[8] = 0.5f * (bb.hz - bb.lz);
    f[9] = logf((float)na);
    f[10] = logf((float)nb);
    const double swa = fmax(ma[0], 1e-300), swb = fmax(mb[0], 1e-300);
    f[11] = (float)log(swa);
    f[12] = (float)log(swb);
    const double mla = ma[1] / swa, mlb = mb[1] / swb;
    f[13] = (float)mla;
    f[14] = (float)mlb;
    f[15] = (float)sqrt(fmax(ma[2] / swa - mla * mla, 0.0));
    f[16] = (float)sqrt(fmax(mb[2] / swb - mlb * mlb, 0.0));
    const double dax = ma[3] / swa, day = ma[4] / swa, daz = ma[5] / swa;
    const double dbx = mb[3] / swb, dby = mb[4] / swb, dbz = mb[5] / swb;
    f[17] = (float)dax;
    f[18] = (float)day;
    f[19] = (float)daz;
    f[20] = (float)dbx;
    f[21] = (float)dby;
    f[22] = (float)dbz;
    const double omc = 1.0 - (dax * dbx + day * dby + daz * dbz);
    f[23] = (float)omc;
    // the ST rate
    const double sbar = exp(mla + mlb) * omc / (2.0 * TL_MEC2 * TL_MEC2);
    const double sig = tl_sigma64(sbar);
    const double loA[3] = {ba.lx, ba.ly, ba.lz}, hiA[3] = {ba.hx, ba.hy, ba.hz};
    const double loB[3] = {bb.lx, bb.ly, bb.lz}, hiB[3] = {bb.hx, bb.hy, bb.hz};
    const double dA[3] = {dax, day, daz}, dB[3] = {dbx, dby, dbz};
    double la[3], ua[3], va[3], lb[3], ub[3], vb[3], VA = 1.0, VB = 1.0, dv2 = 0.0;
    for (int q = 0; q < 3; ++q) {
      const double DA = L * dA[q], DB = L * dB[q];
      la[q] = loA[q] - fmin(0.0, DA);
      ua[q] = hiA[q] - fmax(0.0, DA);
      lb[q] = loB[q] - fmin(0.0, DB);
      ub[q] = hiB[q] - fmax(0.0, DB);
      va[q] = TL_C * dA[q];
      vb[q] = TL_C * dB[q];
      VA *= ua[q] - la[q];
      VB *= ub[q] - lb[q];
      dv2 += (va[q] - vb[q]) * (va[q] - vb[q]);
    }
    double rate = 0.0;
    if (sig > 0.0 && VA > 0.0 && VB > 0.0) {
      const double I = st_overlap_time_integral(la, ua, va, lb, ub, vb, dt);
      if (I > 0.0) rate = swa * swb * (1e12 * kappa * sig) * sqrt(dv2) * I / (VA * VB);
    }
    st[p] = (float)rate;
  }
}

cudaError_t launch_features(const CutTree &A, const CutTree &B, const uint4 *cut,
                            const unsigned *cut_count, unsigned cap, float *feat, float *st,
                            double dt, double kappa, int blocks, cudaStream_t s) {
  k_features<<<blocks, 256, 0, s>>>(A, B, cut, cut_count, cap, feat, st, TL_C * dt, dt, kappa);
  return cudaGetLastError();
}

// ------------------------------------------------------------ exact labels

// The level-L frontier of one tree: inner nodes at or past level L whose
// parent is not, and leaf buckets of inner nodes before level L.  Each gets
// an id; every photon learns the id of the frontier node that holds it.
__global__ void k_frontier_mark(CutTree T, int L, uint32_t *cid_node, uint32_t *cid_slot,
                                uint2 *flist, unsigned *fcount, unsigned fcap) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t ninner = T.n > 1 ? T.n - 1 : 0;
  if (i > ninner) return;  // inner nodes 0..n-2 and the super root (index n-1 or 0)
  const uint32_t node = (i == ninner) ? T.super : (uint32_t)i;
  if (node == T.super && i != ninner) return;
  const bool cut_here = node != T.super && T.nlev[node] >= L;
  if (cut_here) {
    TLBox b;
    uint32_t f, c;
    own(T, node, b, f, c);
    // a node of at most `bucket` photons is a leaf bucket or lies inside one:
    // buckets are frontier nodes through their parent's slot (below)
    if (c <= (uint32_t)T.bucket) return;
    const uint32_t pn = T.parent_node[node];
    const uint32_t parent = pn >> 1;
    const bool parent_cut = parent != T.super && T.nlev[parent] >= L;
    if (!parent_cut) {
      const unsigned id = atomicAdd(fcount, 1u);
      cid_node[node] = id;
      if (id < fcap) flist[id] = make_uint2(f, c);
    }
    return;
  }
  // not cut: its bucket children are frontier nodes -- unless the node is
  // itself a bucket or inside one (then its parent's slot names it)
  if (node != T.super) {
    TLBox b;
    uint32_t f, c;
    own(T, node, b, f, c);
    if (c <= (uint32_t)T.bucket) return;
  }
  const TLNode v = load_node(T.nodes + node);
  for (int slot = 0; slot < 2; ++slot) {
    const uint32_t cr = (uint32_t)(slot ? v.c.y : v.c.x);
    const uint32_t cnt = (uint32_t)(slot ? v.c.w : v.c.z);
    if ((cr & TL_FLAG) && cr != TL_NONE && cnt > 0) {
      const unsigned id = atomicAdd(fcount, 1u);
      cid_slot[2 * (size_t)node + slot] = id;
      if (id < fcap) flist[id] = make_uint2(cr & ~TL_FLAG, cnt);
    }
  }
}

// photon (sorted position) -> frontier id; one warp per frontier node
__global__ void k_frontier_fill(const uint2 *flist, const unsigned *fcount, unsigned fcap,
                                uint32_t *cut_of) {
  const unsigned nf = min(*fcount, fcap);
  const unsigned w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  for (unsigned f = w; f < nf; f += (gridDim.x * blockDim.x) >> 5) {
    const uint2 r = flist[f];
    for (uint32_t p = r.x + lane; p < r.x + r.y; p += 32) cut_of[p] = f;
  }
}

// input index -> sorted position
__global__ void k_inverse(const float4 *dir, int64_t n, uint32_t *inv) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p < n) inv[__float_as_uint(dir[p].w)] = (uint32_t)p;
}

__device__ __forceinline__ uint32_t cid_of(const CutTree &T, uint32_t ref, const uint32_t *cid_node,
                                           const uint32_t *cid_slot) {
  if (ref & TL_FLAG) return cid_slot[2 * (size_t)((ref & ~TL_FLAG) >> 1) + (ref & 1u)];
  return cid_node[ref];
}

__device__ __forceinline__ uint32_t hash64(unsigned long long k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  return (uint32_t)k;
}

// cut pair p: record (cidA, cidB) and insert key -> p into an open-addressing table
__global__ void k_pair_index(CutTree A, CutTree B, uint4 *cut, const unsigned *cut_count,
                             unsigned cap, const uint32_t *cnA, const uint32_t *csA,
                             const uint32_t *cnB, const uint32_t *csB, unsigned long long *hkey,
                             uint32_t *hval, unsigned hmask, unsigned *status) {
  const unsigned n = min(*cut_count, cap);
  for (unsigned p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    uint4 c = cut[p];
    c.z = cid_of(A, c.x, cnA, csA);
    c.w = cid_of(B, c.y, cnB, csB);
    cut[p] = c;
    const unsigned long long key = ((unsigned long long)c.z << 32) | c.w;
    uint32_t h = hash64(key) & hmask;
    bool placed = false;
    for (unsigned probe = 0; probe <= hmask; ++probe) {
      const unsigned long long prev = atomicCAS(&hkey[h], ~0ull, key);
      if (prev == ~0ull || prev == key) {
        hval[h] = p;
        placed = true;
        break;
      }
      h = (h + 1) & hmask;
    }
    if (!placed) atomicOr(status, (unsigned)TL_ST_FRONT_OVF);
  }
}

// every hit adds w_i w_j to the label of the node pair that holds it
__global__ void k_attribute(const uint2 *hits, const unsigned long long *nhits,
                            unsigned long long hcap, const TLBeam mA, const TLBeam mB,
                            const uint32_t *invA, const uint32_t *invB, const uint32_t *cutA,
                            const uint32_t *cutB, const unsigned long long *hkey,
                            const uint32_t *hval, unsigned hmask, double *label,
                            unsigned *status) {
  const unsigned long long n = min(*nhits, hcap);
  for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t < n;
       t += (unsigned long long)gridDim.x * blockDim.x) {
    const uint2 h = hits[t];
    const unsigned long long key =
        ((unsigned long long)cutA[invA[h.x]] << 32) | cutB[invB[h.y]];
    uint32_t s = hash64(key) & hmask;
    bool found = false;
    for (unsigned probe = 0; probe <= hmask; ++probe) {
      const unsigned long long k = hkey[s];
      if (k == key) {
        const double w = (mA.w ? mA.w[h.x] : 1.0) * (mB.w ? mB.w[h.y] : 1.0);
        atomicAdd(&label[hval[s]], w);
        found = true;
        break;
      }
      if (k == ~0ull) break;
      s = (s + 1) & hmask;
    }
    if (!found) atomicOr(status, (unsigned)TL_ST_FRONT_OVF);
  }
}

cudaError_t launch_labels_prep(const CutTree &T, int L, uint32_t *cid_node, uint32_t *cid_slot,
                               uint2 *flist, unsigned *fcount, unsigned fcap, uint32_t *cut_of,
                               uint32_t *inv, cudaStream_t s) {
  const int64_t ninner = T.n > 1 ? T.n - 1 : 0;
  k_frontier_mark<<<(unsigned)((ninner + 1 + 255) / 256), 256, 0, s>>>(T, L, cid_node, cid_slot,
                                                                       flist, fcount, fcap);
  k_frontier_fill<<<1024, 256, 0, s>>>(flist, fcount, fcap, cut_of);
  k_inverse<<<(unsigned)((T.n + 255) / 256), 256, 0, s>>>(T.dir, T.n, inv);
  return cudaGetLastError();
}

cudaError_t launch_pair_index(const CutTree &A, const CutTree &B, uint4 *cut,
                              const unsigned *cut_count, unsigned cap, const uint32_t *cnA,
                              const uint32_t *csA, const uint32_t *cnB, const uint32_t *csB,
                              unsigned long long *hkey, uint32_t *hval, unsigned hmask,
                              unsigned *status, int blocks, cudaStream_t s) {
  k_pair_index<<<blocks, 256, 0, s>>>(A, B, cut, cut_count, cap, cnA, csA, cnB, csB, hkey, hval,
                                      hmask, status);
  return cudaGetLastError();
}

cudaError_t launch_attribute(const uint2 *hits, const unsigned long long *nhits,
                             unsigned long long hcap, const TLBeam &mA, const TLBeam &mB,
                             const uint32_t *invA, const uint32_t *invB, const uint32_t *cutA,
                             const uint32_t *cutB, const unsigned long long *hkey,
                             const uint32_t *hval, unsigned hmask, double *label,
                             unsigned *status, int blocks, cudaStream_t s) {
  k_attribute<<<blocks, 256, 0, s>>>(hits, nhits, hcap, mA, mB, invA, invB, cutA, cutB, hkey, hval,
                                     hmask, label, status);
  return cudaGetLastError();
}

// ------------------------------------------------------------ surrogate estimate

// Pair yield from the network's (mu, s): the predicted mean (B + 1) e^mu over
// the baseline B = st_scale * st (the network is trained with a Poisson-type
// deviance whose minimiser is the conditional mean).  Pairs whose
// predicted standard deviation exceeds tau are flagged for the exact
// fallback (their refs copied out).
__global__ void k_estimate(const float *out, const float *st, float st_scale, const uint4 *cut,
                           const unsigned *cut_count, unsigned cap, float tau, double *pred,
                           uint2 *fb, unsigned *fb_count, unsigned fb_cap, uint8_t *flag) {
  const unsigned n = min(*cut_count, cap);
  const int lane = threadIdx.x & 31;
  const unsigned nround = (n + 31u) & ~31u;
  for (unsigned p = blockIdx.x * blockDim.x + threadIdx.x; p < nround;
       p += gridDim.x * blockDim.x) {
    bool fall = false;
    uint2 r = make_uint2(0u, 0u);
    if (p < n) {
      const float mu = out[2 * p], s = fminf(fmaxf(out[2 * p + 1], -12.f), 12.f);
      const float var = __expf(s);
      fall = sqrtf(var) > tau;
      // the predicted mean (B + 1) e^mu with baseline B = st_scale * st
      const double e = ((double)st_scale * (double)st[p] + 1.0) * exp(fmin((double)mu, 30.0));
      pred[p] = fall ? 0.0 : fmax(e, 0.0);
      if (flag) flag[p] = fall ? 1 : 0;
      const uint4 c = cut[p];
      r = make_uint2(c.x, c.y);
    }
    const unsigned m = __ballot_sync(0xffffffffu, fall);
    if (m) {
      unsigned base = 0;
      if (lane == 0) base = atomicAdd(fb_count, (unsigned)__popc(m));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (fall) {
        const unsigned idx = base + __popc(m & ((1u << lane) - 1u));
        if (idx < fb_cap) fb[idx] = r;
      }
    }
  }
}

cudaError_t launch_estimate(const float *out, const float *st, float st_scale, const uint4 *cut,
                            const unsigned *cut_count, unsigned cap, float tau, double *pred,
                            uint2 *fb, unsigned *fb_count, unsigned fb_cap, int blocks,
                            cudaStream_t s, uint8_t *flag) {
  k_estimate<<<blocks, 256, 0, s>>>(out, st, st_scale, cut, cut_count, cap, tau, pred, fb,
                                    fb_count, fb_cap, flag);
  return cudaGetLastError();
}

// ------------------------------------------------------------ helpers

__global__ void k_sur_misc(int op, const void *a, void *c, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
    if (op == 0) {
      const uint4 v = reinterpret_cast<const uint4 *>(a)[i];
      reinterpret_cast<uint2 *>(c)[i] = make_uint2(v.x, v.y);
    } else if (op == 1) {
      reinterpret_cast<float *>(c)[i] = (float)log1p(reinterpret_cast<const double *>(a)[i]);
    } else if (op == 2) {
      acc += reinterpret_cast<const double *>(a)[i];
    } else {
      acc += (double)reinterpret_cast<const float *>(a)[i];
    }
  }
  if (op >= 2) {
    for (int off = 16; off; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0 && acc != 0.0) atomicAdd(reinterpret_cast<double *>(c), acc);
  }
}

cudaError_t launch_sur_misc(int op, const void *a, const void *b, void *c, int64_t n,
                            cudaStream_t s) {
  (void)b;
  if (n <= 0) return cudaSuccess;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  k_sur_misc<<<(unsigned)blocks, 256, 0, s>>>(op, a, c, n);
  return cudaGetLastError();
}

}  // namespace tl
