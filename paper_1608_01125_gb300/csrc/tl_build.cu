// tl_build.cu -- per-step hierarchy build for one beam.
//
//   propagate   positions in closed form (FP64), FP32 SoA, Morton key of the
//               swept box's centre in the step's moment box, and the radix
//               sort's digit histogram (one pass over the FP64 input)
//   gather      SoA into Morton order
//   karras      inner nodes of the binary radix tree over the sorted keys
//               (Karras 2012, "Maximizing parallelism in the construction of
//               BVHs, octrees and k-d trees"), leaf buckets of <= B photons
//   refit       every node's box as the union of its photons' swept boxes
//               (Sec. 2.1: each box covers the travel of its photons during
//               the step) over its contiguous photon range: sparse tables per
//               tile and over tiles, no atomics and no waiting
#include "tl_common.cuh"

namespace tl {

// ---------------------------------------------------------------- bounds

__device__ __forceinline__ long long ord64(double x) {
  long long i = __double_as_longlong(x);
  return i >= 0 ? i : i ^ 0x7fffffffffffffffLL;
}

// One-time moments of a beam for the Morton box: per axis a the sums of p0,
// d, p0^2, p0 d and d^2 (15 FP64 values), in a fixed order (per-block sums,
// then one block over the blocks), so the box never depends on scheduling.
// The swept-box centre at step k is c = p0 + T d (T = c t_k + c dt / 2), so
// its mean and variance over the beam follow in closed form for every step.
constexpr int kMomentBlocks = 4 * 152;

__global__ void __launch_bounds__(256) k_beam_moments(TLBeam b, double *part) {
  double m[15];
  for (int q = 0; q < 15; ++q) m[q] = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < b.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double p[3] = {b.px[i], b.py[i], b.pz[i]}, d[3] = {b.dx[i], b.dy[i], b.dz[i]};
    for (int a = 0; a < 3; ++a) {
      m[a] += p[a];
      m[3 + a] += d[a];
      m[6 + a] += p[a] * p[a];
      m[9 + a] += p[a] * d[a];
      m[12 + a] += d[a] * d[a];
    }
  }
  __shared__ double sm[8][15];
  for (int q = 0; q < 15; ++q)
    for (int off = 16; off; off >>= 1) m[q] += __shfl_xor_sync(0xffffffffu, m[q], off);
  if ((threadIdx.x & 31) == 0)
    for (int q = 0; q < 15; ++q) sm[threadIdx.x >> 5][q] = m[q];
  __syncthreads();
  if (threadIdx.x < 15) {
    double t = 0.0;
    for (int w8 = 0; w8 < 8; ++w8) t += sm[w8][threadIdx.x];
    part[blockIdx.x * 15 + threadIdx.x] = t;
  }
}

__global__ void k_beam_moments_final(const double *part, int nparts, double *out) {
  if (threadIdx.x < 15) {
    double t = 0.0;
    for (int k = 0; k < nparts; ++k) t += part[k * 15 + threadIdx.x];
    out[threadIdx.x] = t;
  }
}

// out15: device, 15 doubles; scratch: device, 15 * kMomentBlocks doubles
cudaError_t launch_beam_moments(const TLBeam &b, double *out15, double *scratch, cudaStream_t s) {
  const int64_t nb = (b.n + 255) / 256;
  const int blocks = (int)(nb < 1 ? 1 : (nb < kMomentBlocks ? nb : kMomentBlocks));
  k_beam_moments<<<blocks, 256, 0, s>>>(b, scratch);
  k_beam_moments_final<<<1, 32, 0, s>>>(scratch, blocks, out15);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- instances

// Per-instance min and max of p0 and d (12 ordered int64 per instance, laid
// out as p0 min xyz, d min xyz, p0 max xyz, d max xyz).  A warp whose lanes share one instance reduces
// first and issues one atomic per quantity.
__global__ void k_inst_bounds(TLBeam b, const uint32_t *inst_of, long long *out) {
  const int lane = threadIdx.x & 31;
  for (int64_t i0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & ~31ll; i0 < b.n;
       i0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = i0 + lane;
    const bool valid = i < b.n;
    const uint32_t q = valid ? inst_of[i] : 0xffffffffu;
    const uint32_t q0 = __shfl_sync(0xffffffffu, q, 0);
    const bool uniform = __all_sync(0xffffffffu, !valid || q == q0);
    long long v[12];
    if (valid) {
      const double x[6] = {b.px[i], b.py[i], b.pz[i], b.dx[i], b.dy[i], b.dz[i]};
      for (int c = 0; c < 6; ++c) v[c] = v[6 + c] = ord64(x[c]);
    } else {
      for (int c = 0; c < 6; ++c) {
        v[c] = 0x7fffffffffffffffLL;
        v[6 + c] = -0x7fffffffffffffffLL - 1;
      }
    }
    if (uniform) {
      for (int c = 0; c < 6; ++c)
        for (int off = 16; off; off >>= 1) {
          v[c] = min(v[c], __shfl_xor_sync(0xffffffffu, v[c], off));
          v[6 + c] = max(v[6 + c], __shfl_xor_sync(0xffffffffu, v[6 + c], off));
        }
      if (lane == 0)
        for (int c = 0; c < 6; ++c) {
          atomicMin(&out[12 * (size_t)q0 + c], v[c]);
          atomicMax(&out[12 * (size_t)q0 + 6 + c], v[6 + c]);
        }
    } else if (valid) {
      for (int c = 0; c < 6; ++c) {
        atomicMin(&out[12 * (size_t)q + c], v[c]);
        atomicMax(&out[12 * (size_t)q + 6 + c], v[6 + c]);
      }
    }
  }
}

__global__ void k_inst_bounds_init(long long *out, int n_inst) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < 12 * n_inst) out[t] = (t % 12) < 6 ? 0x7fffffffffffffffLL : -0x7fffffffffffffffLL - 1;
}

__global__ void k_inst_bounds_decode(const long long *in, double *out, int n_inst) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < 12 * n_inst) {
    long long i = in[t];
    i = i >= 0 ? i : i ^ 0x7fffffffffffffffLL;
    out[t] = __longlong_as_double(i);
  }
}

// Morton quantisation box of every instance for the step with travel
// T = c t_k + L/2 to the swept segment's centre (lo, then scale per axis).
__global__ void k_inst_box(const double *bounds, int n_inst, double T, unsigned maxq,
                           float4 *box) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n_inst) return;
  const double *bd = bounds + 12 * (size_t)q;
  float lo[3], sc[3];
  for (int a = 0; a < 3; ++a) {
    const double l = bd[a] + T * bd[3 + a], h = bd[6 + a] + T * bd[9 + a];
    lo[a] = (float)l;
    sc[a] = h > l ? (float)((double)maxq / (h - l)) : 0.0f;
  }
  box[2 * q] = make_float4(lo[0], lo[1], lo[2], 0.f);
  box[2 * q + 1] = make_float4(sc[0], sc[1], sc[2], 0.f);
}

// Concatenate the instances' input arrays into one beam and record the
// instance of every photon.
__global__ void k_gather_instances(const InstSrc *src, int n_inst, int64_t n, double *const *dst,
                                   uint32_t *inst_of) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int lo = 0, hi = n_inst - 1;  // last instance whose offset <= i
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (src[mid].off <= i) lo = mid;
    else hi = mid - 1;
  }
  const InstSrc &s = src[lo];
  const int64_t j = i - s.off;
  for (int k = 0; k < 8; ++k) dst[k][i] = s.p[k] ? s.p[k][j] : 1.0;
  inst_of[i] = (uint32_t)lo;
}

cudaError_t launch_inst_bounds(const TLBeam &b, const uint32_t *inst_of, int n_inst,
                               long long *tmp, double *out, cudaStream_t s) {
  const int nt = 12 * n_inst;
  k_inst_bounds_init<<<(nt + 255) / 256, 256, 0, s>>>(tmp, n_inst);
  if (b.n > 0) {
    int64_t nb = (b.n + 255) / 256;
    k_inst_bounds<<<(int)(nb < 4096 ? nb : 4096), 256, 0, s>>>(b, inst_of, tmp);
  }
  k_inst_bounds_decode<<<(nt + 255) / 256, 256, 0, s>>>(tmp, out, n_inst);
  return cudaGetLastError();
}

cudaError_t launch_inst_box(const double *bounds, int n_inst, double T, int bits, float4 *box,
                            cudaStream_t s) {
  k_inst_box<<<(n_inst + 127) / 128, 128, 0, s>>>(bounds, n_inst, T, (1u << bits) - 1u, box);
  return cudaGetLastError();
}

cudaError_t launch_gather_instances(const InstSrc *src, int n_inst, int64_t n, double *const *dst,
                                    uint32_t *inst_of, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_gather_instances<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, n_inst, n, dst, inst_of);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- Morton

// spread the low 21 bits of x to every third bit (bit interleaving by masks)
__device__ __forceinline__ unsigned long long spread3(unsigned long long x) {
  x &= 0x1fffffull;
  x = (x | (x << 32)) & 0x1f00000000ffffull;
  x = (x | (x << 16)) & 0x1f0000ff0000ffull;
  x = (x | (x << 8)) & 0x100f00f00f00f00full;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}

__device__ __forceinline__ unsigned quant(float c, float lo, float scale, unsigned maxq) {
  float f = (c - lo) * scale;
  f = fminf(fmaxf(f, 0.0f), (float)maxq);
  return (unsigned)f;
}

// The step-invariant part of the unsorted FP32 SoA, written once per context:
// the direction rounded to FP32 with the photon's index in w (dir_u), and the
// energy in FP32 (pos_u's w; the propagation rewrites only x, y, z).  GB300's
// FP64 pipe is narrow, and these conversions were half of the propagation's
// FP64 instructions.
__global__ void __launch_bounds__(256) k_static_soa(TLBeam b, float4 *pos_u, float4 *dir_u) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < b.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    dir_u[i] = make_float4(__double2float_rn(b.dx[i]), __double2float_rn(b.dy[i]),
                           __double2float_rn(b.dz[i]), __int_as_float((int)i));
    pos_u[i] = make_float4(0.0f, 0.0f, 0.0f, __double2float_rn(b.E[i]));
  }
}

cudaError_t launch_static_soa(const TLBeam &b, BuildBufs &w, cudaStream_t s) {
  if (b.n <= 0) return cudaSuccess;
  const int64_t nb = (b.n + 255) / 256;
  k_static_soa<<<(unsigned)(nb < 8 * 152 ? nb : 8 * 152), 256, 0, s>>>(b, w.pos_u, w.dir_u);
  return cudaGetLastError();
}

// Propagate p = p0 + c t_k d in FP64 (closed form), round to the FP32 SoA,
// and key every photon by the Morton code of its swept box's centre in the
// box (lo, scale) -- with several instances, its instance's box, and the
// instance number above the Morton bits.  With passes > 0 also counts the
// 8-bit digits of every radix-sort pass (the sort's histogram) in shared
// memory, flushed once per block into the zeroed raw histogram.  A fixed
// grid of at most kPropBlocks blocks, grid-stride.
constexpr int kPropBlocks = 4 * 152;

__global__ void __launch_bounds__(256) k_propagate(TLBeam b, double ct, float halfL, float3 lo,
                                                   float3 scale, unsigned maxq, float4 *pos_u,
                                                   float4 *dir_u, unsigned long long *key,
                                                   uint32_t *val, const uint32_t *inst_of,
                                                   const float4 *inst_box, int inst_shift,
                                                   int passes, uint32_t *hist) {
  __shared__ uint32_t sh[8][256];
  if (passes > 0) {
    for (int t = threadIdx.x; t < 8 * 256; t += 256) (&sh[0][0])[t] = 0u;
    __syncthreads();
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < b.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long ikey = 0ull;
    float3 l3 = lo, s3 = scale;
    if (inst_of) {
      const uint32_t q = inst_of[i];
      const float4 bl = inst_box[2 * q], bs = inst_box[2 * q + 1];
      l3 = make_float3(bl.x, bl.y, bl.z);
      s3 = make_float3(bs.x, bs.y, bs.z);
      ikey = (unsigned long long)q << inst_shift;
    }
    const double dx = b.dx[i], dy = b.dy[i], dz = b.dz[i];
    const double Px = __dadd_rn(b.px[i], __dmul_rn(ct, dx));
    const double Py = __dadd_rn(b.py[i], __dmul_rn(ct, dy));
    const double Pz = __dadd_rn(b.pz[i], __dmul_rn(ct, dz));
    const float3 p = make_float3(__double2float_rn(Px), __double2float_rn(Py),
                                 __double2float_rn(Pz));
    const float4 d = dir_u[i];  // the FP32 direction, written once (k_static_soa)
    float *pu = reinterpret_cast<float *>(pos_u + i);  // x, y, z; w holds the energy
    *reinterpret_cast<float2 *>(pu) = make_float2(p.x, p.y);
    pu[2] = p.z;
    const unsigned qx = quant(fmaf(halfL, d.x, p.x), l3.x, s3.x, maxq),
                   qy = quant(fmaf(halfL, d.y, p.y), l3.y, s3.y, maxq),
                   qz = quant(fmaf(halfL, d.z, p.z), l3.z, s3.z, maxq);
    const unsigned long long k = ikey | (spread3(qx) << 2) | (spread3(qy) << 1) | spread3(qz);
    key[i] = k;
    val[i] = (uint32_t)i;
    for (int q = 0; q < passes; ++q) atomicAdd(&sh[q][(k >> (8 * q)) & 255u], 1u);
  }
  if (passes > 0) {
    __syncthreads();
    for (int t = threadIdx.x; t < passes * 256; t += 256) {
      const uint32_t v = (&sh[0][0])[t];
      if (v) atomicAdd(&hist[t], v);
    }
  }
}

cudaError_t launch_propagate(const TLBeam &b, double ct, float L, const float box_lo[3],
                             const float box_scale[3], int bits, BuildBufs &w,
                             const float4 *inst_box, int passes, cudaStream_t s) {
  if (b.n <= 0) return cudaSuccess;
  unsigned maxq = (1u << bits) - 1u;
  const int64_t nb = (b.n + 255) / 256;
  const int blocks = (int)(nb < kPropBlocks ? nb : kPropBlocks);
  k_propagate<<<blocks, 256, 0, s>>>(
      b, ct, 0.5f * L, make_float3(box_lo[0], box_lo[1], box_lo[2]),
      make_float3(box_scale[0], box_scale[1], box_scale[2]), maxq, w.pos_u, w.dir_u, w.key[0],
      w.val[0], w.inst_of, inst_box, 3 * bits, passes, w.sort_raw);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- gather

__global__ void __launch_bounds__(256) k_gather(int64_t n, const uint32_t *__restrict__ val,
                                                const float4 *__restrict__ pos_u,
                                                const float4 *__restrict__ dir_u,
                                                float4 *__restrict__ pos, float4 *__restrict__ dir,
                                                const unsigned *build_status) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n || (*build_status & TL_ST_TIMEOUT)) return;
  uint32_t src = val[i];
  pos[i] = pos_u[src];
  dir[i] = dir_u[src];
}

cudaError_t launch_gather(BuildBufs &w, int64_t n, int sel, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_gather<<<(int)((n + 255) / 256), 256, 0, s>>>(n, w.val[sel], w.pos_u, w.dir_u, w.pos, w.dir,
                                                  w.build_status);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- Karras

// common prefix length of sorted keys i and j (ki = key i); equal keys fall
// back to the indices (so every key is distinct); -1 outside [0, n).  32-bit
// indices: a beam holds fewer than 2^27 photons.
__device__ __forceinline__ int kdelta(const unsigned long long *__restrict__ key, int n, int i,
                                      unsigned long long ki, int j) {
  if ((unsigned)j >= (unsigned)n) return -1;
  const unsigned long long kj = __ldg(key + j);
  return ki != kj ? __clzll((long long)(ki ^ kj)) : 64 + __clz(i ^ j);
}

__device__ __forceinline__ void empty_box(float4 &b1, float4 &b2) {
  // box 1 of the super root: lo = +inf, hi = -inf never overlaps
  const float inf = __int_as_float(0x7f800000);
  b1.z = inf;
  b1.w = inf;
  b2 = make_float4(inf, -inf, -inf, -inf);
}

// With several instances (inst_root != NULL) a subtree never mixes instances
// below its instance's root: a node spanning two instances is never a leaf
// bucket, and the root of each instance's subtree (the first node on the path
// down that lies inside one instance) is recorded as a stack reference.
__global__ void __launch_bounds__(256) k_karras(const unsigned long long *__restrict__ key,
                                                int64_t n, int bucket, TLNode *nodes,
                                                uint32_t *parent_leaf, uint32_t *parent_node,
                                                const unsigned *build_status, uint32_t *inst_root,
                                                int inst_shift, uint32_t *nfirst,
                                                uint32_t *nlast, uint8_t *nlev, int key_bits) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (*build_status & TL_ST_TIMEOUT) return;  // keys unsorted: the build is abandoned
  const uint32_t super = (uint32_t)(n > 1 ? n - 1 : 0);
  const bool multi = inst_root != nullptr;
  if (i == 0) {
    // the super root: one child (the whole beam) in slot 0, slot 1 empty
    TLNode sr;
    sr.b0 = make_float4(0.f, 0.f, 0.f, 0.f);
    sr.b1 = make_float4(0.f, 0.f, 0.f, 0.f);
    empty_box(sr.b1, sr.b2);
    const bool one_inst = !multi || (key[0] >> inst_shift) == (key[n - 1] >> inst_shift);
    const bool root_bucket = n <= bucket && one_inst;
    int ref0 = root_bucket ? (int)(TL_FLAG | 0u) : 0;
    sr.c = make_int4(ref0, (int)TL_NONE, (int)n, 0);
    // boxes are written by the refit; write refs and the empty slot now
    nodes[super] = sr;
    if (n > 1) parent_node[0] = (super << 1) | 0u;
    else parent_leaf[0] = (super << 1) | 0u;
    if (multi && one_inst)
      inst_root[key[0] >> inst_shift] = root_bucket ? (TL_FLAG | (super << 1)) : 0u;
    nfirst[super] = 0u;
    nlast[super] = (uint32_t)(n - 1);
    nlev[super] = 0;
  }
  if (i >= n - 1) return;
  const int n32 = (int)n, i32 = (int)i;
  const unsigned long long ki = __ldg(key + i32);
  const int dl = kdelta(key, n32, i32, ki, i32 - 1), dr = kdelta(key, n32, i32, ki, i32 + 1);
  const int d = dr > dl ? 1 : -1;
  const int dmin = dr > dl ? dl : dr;
  int lmax = 2;
  while (kdelta(key, n32, i32, ki, i32 + lmax * d) > dmin) lmax <<= 1;
  int l = 0;
  for (int t = lmax >> 1; t >= 1; t >>= 1)
    if (kdelta(key, n32, i32, ki, i32 + (l + t) * d) > dmin) l += t;
  const int j32 = i32 + l * d;
  const int dnode = kdelta(key, n32, i32, ki, j32);
  int s = 0, t = l;
  do {
    t = (t + 1) >> 1;
    if (kdelta(key, n32, i32, ki, i32 + (s + t) * d) > dnode) s += t;
  } while (t > 1);
  const int64_t j = j32;
  int64_t gamma = i32 + s * d + (d < 0 ? -1 : 0);
  int64_t first = i < j ? i : j, last = i < j ? j : i;
  int64_t cl = gamma - first + 1, cr = last - gamma;
  bool lone = true, rone = true;  // child inside one instance
  if (multi) {
    const unsigned long long kf = key[first] >> inst_shift, kg = key[gamma] >> inst_shift,
                             kh = key[gamma + 1] >> inst_shift, kl = key[last] >> inst_shift;
    lone = kf == kg;
    rone = kh == kl;
    if (kf != kl) {  // this node spans instances: a one-instance child roots its instance
      if (lone) inst_root[kf] = cl <= bucket ? (TL_FLAG | ((uint32_t)i << 1)) : (uint32_t)gamma;
      if (rone)
        inst_root[kl] = cr <= bucket ? (TL_FLAG | ((uint32_t)i << 1) | 1u) : (uint32_t)(gamma + 1);
    }
  }
  nfirst[i] = (uint32_t)first;
  nlast[i] = (uint32_t)last;
  {
    const int lev = dnode - (64 - key_bits);  // equal keys: beyond key_bits
    nlev[i] = (uint8_t)(lev < 0 ? 0 : (lev > 255 ? 255 : lev));
  }
  int refl = (cl <= bucket && lone) ? (int)(TL_FLAG | (uint32_t)first) : (int)gamma;
  int refr = (cr <= bucket && rone) ? (int)(TL_FLAG | (uint32_t)(gamma + 1)) : (int)(gamma + 1);
  nodes[i].c = make_int4(refl, refr, (int)cl, (int)cr);
  if (first == gamma) parent_leaf[gamma] = ((uint32_t)i << 1) | 0u;
  else parent_node[gamma] = ((uint32_t)i << 1) | 0u;
  if (last == gamma + 1) parent_leaf[gamma + 1] = ((uint32_t)i << 1) | 1u;
  else parent_node[gamma + 1] = ((uint32_t)i << 1) | 1u;
}

cudaError_t launch_karras(BuildBufs &w, int64_t n, int sel, int bucket, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int64_t threads = n > 1 ? n - 1 : 1;
  k_karras<<<(int)((threads + 255) / 256), 256, 0, s>>>(w.key[sel], n, bucket, w.nodes,
                                                        w.parent_leaf, w.parent_node,
                                                        w.build_status, w.inst_root,
                                                        w.inst_shift, w.nfirst, w.nlast,
                                                        w.nlev, w.key_bits);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- refit

// Swept box of one photon in FP32 interval arithmetic with directed
// rounding.  The FP64 position of the definition lies within |P32| 2^-23 of
// P32 (and likewise the direction), the segment is P + lambda L d for
// lambda in [0, 1] with L in [L_lo, L_hi], and half = r_max / 2 plus margin.
__device__ __forceinline__ void seg_axis(float p, float dc, float Llo, float Lhi, float half,
                                         float &lo, float &hi) {
  const float ep = __fmaf_ru(fabsf(p), 1.1920928955078125e-7f, 1e-30f);
  const float plo = __fsub_rd(p, ep), phi = __fadd_ru(p, ep);
  const float ed = __fmaf_ru(fabsf(dc), 1.1920928955078125e-7f, 1e-30f);
  const float dlo = __fsub_rd(dc, ed), dhi = __fadd_ru(dc, ed);
  const float ldlo = dlo >= 0.f ? __fmul_rd(Llo, dlo) : __fmul_rd(Lhi, dlo);
  const float ldhi = dhi >= 0.f ? __fmul_ru(Lhi, dhi) : __fmul_ru(Llo, dhi);
  const float qlo = __fadd_rd(plo, ldlo), qhi = __fadd_ru(phi, ldhi);
  lo = __fsub_rd(fminf(plo, qlo), half);
  hi = __fadd_ru(fmaxf(phi, qhi), half);
}

// slot 0 = floats 0..5 of the record (b0, b1.xy), slot 1 = floats 6..11
// (b1.zw, b2): one 16-byte and one 8-byte store each
__device__ __forceinline__ void write_slot(TLNode *nodes, uint32_t node, uint32_t slot,
                                           const TLBox &b) {
  TLNode &r = nodes[node];
  if (slot == 0u) {
    r.b0 = make_float4(b.lx, b.ly, b.lz, b.hx);
    *reinterpret_cast<float2 *>(&r.b1.x) = make_float2(b.hy, b.hz);
  } else {
    *reinterpret_cast<float2 *>(&r.b1.z) = make_float2(b.lx, b.ly);
    r.b2 = make_float4(b.lz, b.hx, b.hy, b.hz);
  }
}

// Refit as range unions.  Every subtree of the Karras hierarchy holds a
// contiguous range [f, l] of the Morton-ordered photons, so its box is the
// union (FP32 min / max: exact, order-free) of the photons' swept boxes over
// that range, and every node can be finished on its own, with no bottom-up
// chain of waits:
//   k_refit_tile   one block per tile of kRTile photons: the tile's leaf boxes
//                  in a shared-memory sparse table (level j holds the unions of
//                  2^j consecutive boxes), so a range inside the tile is the
//                  union of two entries.  Writes every photon's box into its
//                  parent's slot, the box of every node whose range lies in
//                  the tile into its parent's slot, the prefix and suffix
//                  unions of every photon within its tile, and the tile box.
//   k_refit_super  one block per kRSuper tiles: the same table over tile boxes.
//   k_refit_cross  nodes whose range spans tiles: suffix of the first tile +
//                  the tiles in between (two table entries per super-tile
//                  end, plus whole super-tiles) + prefix of the last tile.
// A node's range: f = first photon (written by the emit), l = f + both child
// counts - 1.  A Karras node's index is one end of its range, so a node whose
// range lies in a tile has its index there too.
constexpr int kRTile = 256, kRTileLev = 8;  // levels 0..7 cover ranges of up to 256
constexpr int kRSuper = 512, kRSuperLog = 9;

struct Box6 {
  float v[6];  // lo xyz, hi xyz
};

__device__ __forceinline__ Box6 empty6() {
  const float inf = __int_as_float(0x7f800000);
  Box6 b;
  b.v[0] = b.v[1] = b.v[2] = inf;
  b.v[3] = b.v[4] = b.v[5] = -inf;
  return b;
}

__device__ __forceinline__ void join6(Box6 &a, const Box6 &b) {
  a.v[0] = fminf(a.v[0], b.v[0]);
  a.v[1] = fminf(a.v[1], b.v[1]);
  a.v[2] = fminf(a.v[2], b.v[2]);
  a.v[3] = fmaxf(a.v[3], b.v[3]);
  a.v[4] = fmaxf(a.v[4], b.v[4]);
  a.v[5] = fmaxf(a.v[5], b.v[5]);
}

__device__ __forceinline__ TLBox to_box(const Box6 &b) {
  TLBox t;
  t.lx = b.v[0];
  t.ly = b.v[1];
  t.lz = b.v[2];
  t.hx = b.v[3];
  t.hy = b.v[4];
  t.hz = b.v[5];
  return t;
}

// shared-memory sparse table: tab[(j * 6 + q) * W + i], W entries per level
template <int W>
__device__ __forceinline__ Box6 tab_get(const float *tab, int j, int i) {
  Box6 b;
#pragma unroll
  for (int q = 0; q < 6; ++q) b.v[q] = tab[(j * 6 + q) * W + i];
  return b;
}

// union over [a, b]: two entries of level j = floor(log2(b - a + 1)), capped
// at the table's top level LEV - 1 (two top-level entries still cover any
// range of up to 2^LEV boxes)
template <int W, int LEV>
__device__ __forceinline__ Box6 tab_query(const float *tab, int a, int b) {
  const int j = min(31 - __clz(b - a + 1), LEV - 1);
  Box6 r = tab_get<W>(tab, j, a);
  join6(r, tab_get<W>(tab, j, b - (1 << j) + 1));
  return r;
}

// fills levels 1..LOG of a W-wide table whose level 0 is in place
template <int W, int LOG>
__device__ __forceinline__ void tab_build(float *tab) {
  for (int j = 1; j <= LOG; ++j) {
    const int h = 1 << (j - 1);
    for (int i = threadIdx.x; i + (1 << j) <= W; i += blockDim.x) {
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        const float x = tab[((j - 1) * 6 + q) * W + i], y = tab[((j - 1) * 6 + q) * W + i + h];
        tab[(j * 6 + q) * W + i] = q < 3 ? fminf(x, y) : fmaxf(x, y);
      }
    }
    __syncthreads();
  }
}

__device__ __forceinline__ void put6(float *dst, const Box6 &b) {
  float2 *d2 = reinterpret_cast<float2 *>(dst);
  d2[0] = make_float2(b.v[0], b.v[1]);
  d2[1] = make_float2(b.v[2], b.v[3]);
  d2[2] = make_float2(b.v[4], b.v[5]);
}

__device__ __forceinline__ Box6 get6(const float *src) {
  const float2 *s2 = reinterpret_cast<const float2 *>(src);
  const float2 a = s2[0], b = s2[1], c = s2[2];
  Box6 r;
  r.v[0] = a.x;
  r.v[1] = a.y;
  r.v[2] = b.x;
  r.v[3] = b.y;
  r.v[4] = c.x;
  r.v[5] = c.y;
  return r;
}


__global__ void __launch_bounds__(kRTile) k_refit_tile(
    int64_t n, const float4 *__restrict__ pos, const float4 *__restrict__ dir, float Llo,
    float Lhi, float half, TLNode *nodes, const uint32_t *__restrict__ parent_leaf,
    const uint32_t *__restrict__ parent_node, const uint32_t *__restrict__ nfirst,
    const uint32_t *__restrict__ nlast, float *pre, float *suf, float *tilebox,
    unsigned *build_status) {
  extern __shared__ float tab[];  // kRTileLev levels x 6 x kRTile
  __shared__ unsigned abandoned;
  const int t = threadIdx.x;
  // one read for the whole block: other blocks of this kernel may set the flag
  if (t == 0) abandoned = *(volatile unsigned *)build_status & TL_ST_TIMEOUT;
  __syncthreads();
  if (abandoned) return;  // keys unsorted: the build is abandoned
  const int64_t base = blockIdx.x * (int64_t)kRTile;
  const int64_t p = base + t;
  const uint32_t super = (uint32_t)(n > 1 ? n - 1 : 0);
  const int cnt = n - base < kRTile ? (int)(n - base) : kRTile;
  // every global load first (they do not depend on the table)
  float4 ps = make_float4(0.f, 0.f, 0.f, 0.f), d = ps;
  uint32_t lref = 0u, nref = 0u;
  int64_t f = 0, l = -1;
  if (p < n) {
    ps = pos[p];
    d = dir[p];
    lref = parent_leaf[p];
  }
  const bool inner = p < (int64_t)super;  // the super root (index n - 1) has no parent
  if (inner) {
    f = nfirst[p];
    l = nlast[p];
    nref = parent_node[p];
  }
  Box6 b = empty6();
  if (p < n) {
    seg_axis(ps.x, d.x, Llo, Lhi, half, b.v[0], b.v[3]);
    seg_axis(ps.y, d.y, Llo, Lhi, half, b.v[1], b.v[4]);
    seg_axis(ps.z, d.z, Llo, Lhi, half, b.v[2], b.v[5]);
    if ((lref >> 1) <= super) write_slot(nodes, lref >> 1, lref & 1u, to_box(b));
    else atomicOr(build_status, (unsigned)TL_ST_BADTREE);
  }
#pragma unroll
  for (int q = 0; q < 6; ++q) tab[q * kRTile + t] = b.v[q];
  __syncthreads();
  tab_build<kRTile, kRTileLev - 1>(tab);
  if (p < n) {
    put6(pre + 6 * p, tab_query<kRTile, kRTileLev>(tab, 0, t));
    put6(suf + 6 * p, tab_query<kRTile, kRTileLev>(tab, t, cnt - 1));
  }
  if (t == 0) put6(tilebox + 6 * blockIdx.x, tab_query<kRTile, kRTileLev>(tab, 0, cnt - 1));
  // inner node p, if its range lies in the tile
  if (inner && f >= base && l < base + cnt) {
    if ((nref >> 1) <= super && f <= l)
      write_slot(nodes, nref >> 1, nref & 1u,
                 to_box(tab_query<kRTile, kRTileLev>(tab, (int)(f - base), (int)(l - base))));
    else atomicOr(build_status, (unsigned)TL_ST_BADTREE);
  }
}

// tables over tile boxes: stab[((s * (kRSuperLog + 1) + j) * kRSuper + i) * 6 + q]
__global__ void __launch_bounds__(kRSuper) k_refit_super(int64_t ntile, const float *tilebox,
                                                         float *stab,
                                                         const unsigned *build_status,
                                                         unsigned *cut_n) {
  extern __shared__ float tab[];  // (kRSuperLog + 1) levels x 6 x kRSuper
  if (blockIdx.x == 0 && threadIdx.x == 0 && cut_n) *cut_n = 0u;  // filled by k_refit_cross
  if (*build_status & TL_ST_TIMEOUT) return;
  const int64_t s = blockIdx.x, t0 = s * kRSuper;
  const int t = threadIdx.x;
  const Box6 b = t0 + t < ntile ? get6(tilebox + 6 * (t0 + t)) : empty6();
#pragma unroll
  for (int q = 0; q < 6; ++q) tab[q * kRSuper + t] = b.v[q];
  __syncthreads();
  tab_build<kRSuper, kRSuperLog>(tab);
  float *out = stab + s * (int64_t)(kRSuperLog + 1) * kRSuper * 6;
  for (int j = 0; j <= kRSuperLog; ++j)
    if (t + (1 << j) <= kRSuper) put6(out + ((int64_t)j * kRSuper + t) * 6, tab_get<kRSuper>(tab, j, t));
}

__device__ __forceinline__ Box6 super_query(const float *stab, int64_t s, int a, int b) {
  const float *tb = stab + s * (int64_t)(kRSuperLog + 1) * kRSuper * 6;
  const int j = 31 - __clz(b - a + 1);
  Box6 r = get6(tb + ((int64_t)j * kRSuper + a) * 6);
  join6(r, get6(tb + ((int64_t)j * kRSuper + b - (1 << j) + 1) * 6));
  return r;
}

// union of the tile boxes a..b (a <= b)
__device__ __forceinline__ Box6 tiles_union(const float *stab, int64_t a, int64_t b) {
  const int64_t s0 = a >> kRSuperLog, s1 = b >> kRSuperLog;
  const int a0 = (int)(a & (kRSuper - 1)), b1 = (int)(b & (kRSuper - 1));
  if (s0 == s1) return super_query(stab, s0, a0, b1);
  Box6 r = super_query(stab, s0, a0, kRSuper - 1);
  join6(r, super_query(stab, s1, 0, b1));
  for (int64_t s = s0 + 1; s < s1; ++s) join6(r, super_query(stab, s, 0, kRSuper - 1));
  return r;
}

// Also lists the traversal seeds: the children with at most cut_S photons of
// nodes with more (such a node spans tiles, as cut_S >= kRTile).
__global__ void __launch_bounds__(256) k_refit_cross(int64_t n, TLNode *nodes,
                                                     const uint32_t *__restrict__ parent_node,
                                                     const uint32_t *__restrict__ nfirst,
                                                     const uint32_t *__restrict__ nlast,
                                                     const float *pre, const float *suf,
                                                     const float *stab, unsigned *build_status,
                                                     uint32_t cut_S, uint32_t *cut,
                                                     unsigned *cut_n, uint32_t cut_cap) {
  if (*build_status & TL_ST_TIMEOUT) return;
  const uint32_t super = (uint32_t)(n > 1 ? n - 1 : 0);
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < (int64_t)super;
       x += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = nfirst[x], l = nlast[x];
    const int64_t t0 = f >> 8, t1 = l >> 8;
    if (t0 == t1) continue;  // finished by its tile
    if (f < 0 || l >= n || f > l) {
      atomicOr(build_status, (unsigned)TL_ST_BADTREE);
      continue;
    }
    if (cut_S && l - f + 1 > (int64_t)cut_S) {
      const int2 cnt = *(reinterpret_cast<const int2 *>(&nodes[x].c) + 1);  // child counts
      for (uint32_t sl = 0; sl < 2; ++sl)
        if ((uint32_t)(sl ? cnt.y : cnt.x) <= cut_S) {
          // a count above cut_cap (long chains of small siblings) tells the
          // traversal to start from the roots instead
          const unsigned k = atomicAdd(cut_n, 1u);
          if (k < cut_cap) cut[k] = ((uint32_t)x << 1) | sl;
        }
    }
    Box6 b = get6(suf + 6 * f);
    join6(b, get6(pre + 6 * l));
    if (t1 - t0 >= 2) join6(b, tiles_union(stab, t0 + 1, t1 - 1));
    const uint32_t ref = parent_node[x];
    if ((ref >> 1) <= super) write_slot(nodes, ref >> 1, ref & 1u, to_box(b));
    else atomicOr(build_status, (unsigned)TL_ST_BADTREE);
  }
}

int64_t refit_tiles(int64_t n) { return (n + kRTile - 1) / kRTile; }
int64_t refit_supers(int64_t n) { return (refit_tiles(n) + kRSuper - 1) / kRSuper; }
size_t refit_super_floats(int64_t n) {
  return (size_t)refit_supers(n) * (kRSuperLog + 1) * kRSuper * 6;
}

cudaError_t refit_prepare() {
  cudaError_t e = cudaFuncSetAttribute(k_refit_tile, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kRTileLev * 6 * kRTile * (int)sizeof(float));
  if (e) return e;
  return cudaFuncSetAttribute(k_refit_super, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (kRSuperLog + 1) * 6 * kRSuper * (int)sizeof(float));
}

cudaError_t launch_refit(BuildBufs &w, int64_t n, float Llo, float Lhi, float half, int n_sm,
                         cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t tiles = refit_tiles(n), supers = refit_supers(n);
  k_refit_tile<<<(unsigned)tiles, kRTile, kRTileLev * 6 * kRTile * sizeof(float), s>>>(
      n, w.pos, w.dir, Llo, Lhi, half, w.nodes, w.parent_leaf, w.parent_node, w.nfirst, w.nlast,
      w.rpre, w.rsuf, w.rtile, w.build_status);
  if (tiles > 1) {
    k_refit_super<<<(unsigned)supers, kRSuper, (kRSuperLog + 1) * 6 * kRSuper * sizeof(float),
                    s>>>(tiles, w.rtile, w.rsuper, w.build_status, w.cut_S ? w.cut_n : nullptr);
    const int64_t nb = (n + 255) / 256;
    const int blocks = (int)(nb < 8 * n_sm ? nb : 8 * n_sm);
    k_refit_cross<<<blocks, 256, 0, s>>>(n, w.nodes, w.parent_node, w.nfirst, w.nlast, w.rpre,
                                         w.rsuf,
                                         w.rsuper, w.build_status, w.cut_S, w.cut, w.cut_n,
                                         w.cut_cap);
  }
  return cudaGetLastError();
}

}  // namespace tl
