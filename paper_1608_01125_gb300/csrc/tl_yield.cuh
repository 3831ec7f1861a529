// tl_yield.cuh -- per-hit yield terms and their fixed-order block reduction,
// shared by the step's yield kernel and the allocation-free reduction.
//
// A step's yield (rate proportional to n_I n_II, Sec. 2.2) is reduced to the
// hit count, the FP64 sum of w_i w_j and two order-free checksums of the hit
// set: the sum (mod 2^64) and the xor of splitmix64((i << 32) | j).
#pragma once
#include "tl_common.cuh"

namespace tl {

struct YieldPartial {
  unsigned long long count;
  double weighted;
  unsigned long long hsum, hxor;
};

__device__ __forceinline__ YieldPartial yield_zero() { return {0ull, 0.0, 0ull, 0ull}; }

__device__ __forceinline__ void yield_add(YieldPartial &a, const YieldPartial &b) {
  a.count += b.count;
  a.weighted += b.weighted;
  a.hsum += b.hsum;
  a.hxor ^= b.hxor;
}

// one hit (i of beam A, j of beam B) with its weights
__device__ __forceinline__ void yield_hit(YieldPartial &p, uint32_t i, uint32_t j, double wi,
                                          double wj) {
  p.count += 1ull;
  p.weighted += wi * wj;
  const unsigned long long m = smix64(((unsigned long long)i << 32) | j);
  p.hsum += m;
  p.hxor ^= m;
}

// a partial read through a volatile pointer (written by another block)
__device__ __forceinline__ YieldPartial yield_load_volatile(const YieldPartial *q) {
  const volatile YieldPartial *v = q;
  YieldPartial o;
  o.count = v->count;
  o.weighted = v->weighted;
  o.hsum = v->hsum;
  o.hxor = v->hxor;
  return o;
}

// Fixed-order block reduction (warp xor-tree, then the warps in order); sp
// holds one partial per warp.  Every thread returns the block's total.
__device__ __forceinline__ YieldPartial yield_block_reduce(YieldPartial p, YieldPartial *sp) {
  for (int off = 16; off; off >>= 1) {
    YieldPartial o;
    o.count = __shfl_xor_sync(0xffffffffu, p.count, off);
    o.weighted = __shfl_xor_sync(0xffffffffu, p.weighted, off);
    o.hsum = __shfl_xor_sync(0xffffffffu, p.hsum, off);
    o.hxor = __shfl_xor_sync(0xffffffffu, p.hxor, off);
    yield_add(p, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sp[warp] = p;
  __syncthreads();
  YieldPartial b = sp[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) yield_add(b, sp[w]);
  __syncthreads();
  return b;
}

}  // namespace tl
