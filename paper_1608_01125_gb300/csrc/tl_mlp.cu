// tl_mlp.cu -- the surrogate network: 24 -> 128 -> 128 -> 128 -> 2, exact
// GELU between layers, BF16 weights and activations with FP32 accumulation.
//
// Forward and input-gradient passes run on the tensor cores (tcgen05.mma,
// accumulators in tensor memory): a block of 128 threads takes 128 rows at a
// time; each layer is one 128 x N x K tile product issued by one thread, its
// FP32 result is read back row per thread (tcgen05.ld), biased, activated and
// written as the next layer's BF16 operand.  Weight gradients (a reduction
// over the batch) run on the tensor cores too, with the batch as the
// reduction dimension (k_mlp_wgrad_tc); the optimiser on the CUDA cores.
//
// Outputs per row: mu and s (log variance) of a Gaussian over
// y = log1p(sum of w_i w_j of a node pair).  Loss 0.5 (s + (y - mu)^2 e^-s),
// s clamped to +-12, mean over the batch.
#include <cuda_bf16.h>

#include "tl_sur.h"
#include "tl_tc.cuh"
#include "trilens.h"

namespace tl {

constexpr int kIn = 24, kInP = 32, kH = 128, kOutP = 16;
// flat FP32 parameter vector: W1 (128x24), b1, W2 (128x128), b2, W3, b3, W4 (2x128), b4
constexpr int64_t kWgChunk = 512;  // batch rows per weight-gradient block
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kH * kIn, kOffW2 = kOffB1 + kH,
              kOffB2 = kOffW2 + kH * kH, kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH * kH,
              kOffW4 = kOffB3 + kH, kOffB4 = kOffW4 + 2 * kH, kParams = kOffB4 + 2;
static_assert(kParams == TRILENS_MLP_PARAMS, "parameter count");
constexpr float kSClamp = 12.0f;

struct MLPDev {
  const __nv_bfloat16 *W1;  // [128][32]  (columns 24..31 zero)
  const __nv_bfloat16 *W2;  // [128][128]
  const __nv_bfloat16 *W3;  // [128][128]
  const __nv_bfloat16 *W4;  // [16][128]  (rows 2..15 zero)
  const float *prm;         // FP32 parameters (biases are read from here)
  const float *norm;        // feature mean[24], 1/std[24]
};

__device__ __forceinline__ float gelu(float x) {
  return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_grad(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) +
         x * 0.39894228040143268f * __expf(-0.5f * x * x);
}

// ---------------------------------------------------------------- parameters

// FP32 master parameters -> padded BF16 weight matrices
__global__ void k_mlp_pack(const float *prm, __nv_bfloat16 *W1, __nv_bfloat16 *W2,
                           __nv_bfloat16 *W3, __nv_bfloat16 *W4) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < kH * kInP) {
    const int o = t / kInP, i = t % kInP;
    W1[t] = __float2bfloat16(i < kIn ? prm[kOffW1 + o * kIn + i] : 0.0f);
  }
  if (t < kH * kH) {
    W2[t] = __float2bfloat16(prm[kOffW2 + t]);
    W3[t] = __float2bfloat16(prm[kOffW3 + t]);
  }
  if (t < kOutP * kH) {
    const int o = t / kH;
    W4[t] = __float2bfloat16(o < 2 ? prm[kOffW4 + t] : 0.0f);
  }
}

// ---------------------------------------------------------------- forward

struct FwdSmem {
  __nv_bfloat16 W1[kH * kInP];
  __nv_bfloat16 W2[kH * kH];
  __nv_bfloat16 W3[kH * kH];
  __nv_bfloat16 W4[kOutP * kH];
  __nv_bfloat16 A[128 * kH];
  __nv_bfloat16 X[128 * kInP];
  float b[3][kH];
  float b4[2];
  uint64_t mbar;
  uint32_t tmem;
  int err;
};

template <class T>
__device__ __forceinline__ T *align1k(unsigned char *p) {
  return reinterpret_cast<T *>((reinterpret_cast<uintptr_t>(p) + 1023) & ~(uintptr_t)1023);
}

__device__ __forceinline__ void load_tile(__nv_bfloat16 *dst, const __nv_bfloat16 *src, int R,
                                          int K) {
  for (int idx = threadIdx.x; idx < R * K; idx += blockDim.x) {
    const int r = idx / K, k = idx - r * K;
    dst[core_idx(r, k, K)] = src[idx];
  }
}

// transposed: dst(n, k) = src[k][n] with src [K rows][N cols] row-major
__device__ __forceinline__ void load_tile_t(__nv_bfloat16 *dst, const __nv_bfloat16 *src, int N,
                                            int K, int src_rows) {
  for (int idx = threadIdx.x; idx < N * K; idx += blockDim.x) {
    const int n = idx / K, k = idx - n * K;
    dst[core_idx(n, k, K)] = k < src_rows ? src[k * N + n] : __float2bfloat16(0.0f);
  }
}

// write 8 consecutive values of row r (columns c..c+7) into a core tile
__device__ __forceinline__ void put8(__nv_bfloat16 *tile, int r, int c, int K, const float *v) {
  __align__(16) __nv_bfloat16 h[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) h[j] = __float2bfloat16(v[j]);
  *reinterpret_cast<uint4 *>(tile + core_idx(r, c, K)) = *reinterpret_cast<const uint4 *>(h);
}

// one layer's tensor-core product and its completion, with every wait bounded
__device__ __forceinline__ bool layer_mma(FwdSmem &S, uint32_t d, const void *A, const void *B,
                                          int K, int N, uint32_t &phase, long long spin) {
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (threadIdx.x == 0) {
    gemm_tile(d, A, B, K, N, false);
    mma_commit(&S.mbar);
  }
  const bool ok = mbar_wait(&S.mbar, phase, spin);
  phase ^= 1u;
  tc_fence_after();
  return ok;
}

// Forward pass over M rows of raw features x [M][24].  Inference writes out
// [M][2]; training (y != NULL) also stores the pre-activations Z1..Z3 (BF16),
// the loss gradient dout [M][2] (of the mean loss, scale inv_b) and adds the
// loss sum to *loss.  Loss kind 0: Gaussian NLL of y with (mu, s).  Kind 1
// (the surrogate's): y is the linear label Y, B = st_scale * st[row] the
// baseline, lam = (B + 1) e^mu the predicted mean; loss
// (lam - Y ln lam)/(B + 1) + 0.5 (s + r^2 e^-s), r = log1p(Y) - log1p(lam)
// with lam held fixed in r.
__global__ void __launch_bounds__(128, 1)
    k_mlp_forward(MLPDev P, const float *__restrict__ x, int64_t M, float *out, const float *y,
                  __nv_bfloat16 *Z1, __nv_bfloat16 *Z2, __nv_bfloat16 *Z3, float *dout,
                  float *loss, float inv_b, int *err, long long spin, int kind, const float *st,
                  float st_scale) {
  extern __shared__ unsigned char smem_raw[];
  FwdSmem &S = *align1k<FwdSmem>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5;
  load_tile(S.W1, P.W1, kH, kInP);
  load_tile(S.W2, P.W2, kH, kH);
  load_tile(S.W3, P.W3, kH, kH);
  load_tile(S.W4, P.W4, kOutP, kH);
  for (int j = tid; j < kH; j += blockDim.x) {
    S.b[0][j] = P.prm[kOffB1 + j];
    S.b[1][j] = P.prm[kOffB2 + j];
    S.b[2][j] = P.prm[kOffB3 + j];
  }
  if (tid < 2) S.b4[tid] = P.prm[kOffB4 + tid];
  if (tid == 0) {
    S.err = 0;
    mbar_init(&S.mbar, 1);
  }
  if (warp == 0) {
    tmem_alloc(&S.tmem, 128);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem;
  const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
  uint32_t phase = 0;
  float lsum = 0.0f;
  const int64_t ntiles = (M + 127) / 128;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t row = tile * 128 + tid;
    const bool valid = row < M;
    {  // normalised features -> BF16 operand
      float v[kInP];
#pragma unroll
      for (int k = 0; k < kInP; ++k) v[k] = 0.0f;
      if (valid)
        for (int k = 0; k < kIn; ++k) v[k] = (x[row * kIn + k] - P.norm[k]) * P.norm[kIn + k];
#pragma unroll
      for (int c = 0; c < kInP; c += 8) put8(S.X, tid, c, kInP, v + c);
    }
    bool ok = layer_mma(S, tmem, S.X, S.W1, kInP, kH, phase, spin);
    __nv_bfloat16 *Zs[3] = {Z1, Z2, Z3};
    const __nv_bfloat16 *Ws[3] = {S.W2, S.W3, S.W4};
    for (int l = 0; l < 3; ++l) {
      // epilogue of layer l+1: bias, (store Z), GELU -> next operand
#pragma unroll 1
      for (int c = 0; c < kH; c += 32) {
        uint32_t r[32];
        TL_TMEM_LD_X32(trow + (uint32_t)c, r);
        tmem_wait_ld();
        float z[32], h[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          z[j] = __uint_as_float(r[j]) + S.b[l][c + j];
          h[j] = gelu(z[j]);
        }
        if (y && valid) {
          __align__(16) __nv_bfloat16 zb[32];
#pragma unroll
          for (int j = 0; j < 32; ++j) zb[j] = __float2bfloat16(z[j]);
          uint4 *dst = reinterpret_cast<uint4 *>(Zs[l] + row * kH + c);
#pragma unroll
          for (int q = 0; q < 4; ++q) dst[q] = reinterpret_cast<const uint4 *>(zb)[q];
        }
#pragma unroll
        for (int q = 0; q < 32; q += 8) put8(S.A, tid, c + q, kH, h + q);
      }
      ok = layer_mma(S, tmem, S.A, Ws[l], kH, l < 2 ? kH : kOutP, phase, spin) && ok;
    }
    uint32_t r[16];
    TL_TMEM_LD_X16(trow, r);
    tmem_wait_ld();
    const float o0 = __uint_as_float(r[0]) + S.b4[0], o1 = __uint_as_float(r[1]) + S.b4[1];
    if (valid) {
      if (out) {
        out[2 * row] = o0;
        out[2 * row + 1] = o1;
      }
      if (y && kind == 0) {
        const float s = fminf(fmaxf(o1, -kSClamp), kSClamp);
        const float res = y[row] - o0, e = __expf(-s);
        lsum += 0.5f * (s + res * res * e);
        dout[2 * row] = -res * e * inv_b;
        dout[2 * row + 1] = (o1 > -kSClamp && o1 < kSClamp) ? 0.5f * (1.0f - res * res * e) * inv_b
                                                             : 0.0f;
      } else if (y) {
        const float Y = y[row], B1 = st_scale * st[row] + 1.0f;
        const float lam = B1 * __expf(fminf(o0, 30.0f));
        const float s = fminf(fmaxf(o1, -kSClamp), kSClamp), e = __expf(-s);
        const float r = log1pf(Y) - log1pf(lam);
        lsum += (lam - Y * __logf(lam)) / B1 + 0.5f * (s + r * r * e);
        dout[2 * row] = o0 < 30.0f ? (lam - Y) / B1 * inv_b : 0.0f;
        dout[2 * row + 1] = (o1 > -kSClamp && o1 < kSClamp) ? 0.5f * (1.0f - r * r * e) * inv_b
                                                             : 0.0f;
      }
    }
    if (!ok) S.err = 1;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  if (y) {
    for (int off = 16; off; off >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, off);
    if ((tid & 31) == 0) atomicAdd(loss, lsum);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 128);
  if (tid == 0 && S.err) atomicOr(err, 1);
}

// ---------------------------------------------------------------- input gradients

struct BwdSmem {
  __nv_bfloat16 W2T[kH * kH];
  __nv_bfloat16 W3T[kH * kH];
  __nv_bfloat16 W4T[kH * kOutP];
  __nv_bfloat16 A[128 * kH];
  uint64_t mbar;
  uint32_t tmem;
  int err;
};

__device__ __forceinline__ bool bwd_mma(BwdSmem &S, uint32_t d, const void *A, const void *B,
                                        int K, uint32_t &phase, long long spin) {
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (threadIdx.x == 0) {
    gemm_tile(d, A, B, K, kH, false);
    mma_commit(&S.mbar);
  }
  const bool ok = mbar_wait(&S.mbar, phase, spin);
  phase ^= 1u;
  tc_fence_after();
  return ok;
}

// dZ3 = (dout W4) gelu'(Z3), dZ2 = (dZ3 W3) gelu'(Z2), dZ1 = (dZ2 W2) gelu'(Z1):
// the products on the tensor cores with W^T as the B operand.
__global__ void __launch_bounds__(128, 1)
    k_mlp_dgrad(MLPDev P, const float *__restrict__ dout, const __nv_bfloat16 *Z1,
                const __nv_bfloat16 *Z2, const __nv_bfloat16 *Z3, __nv_bfloat16 *dZ1,
                __nv_bfloat16 *dZ2, __nv_bfloat16 *dZ3, int64_t M, int *err, long long spin) {
  extern __shared__ unsigned char smem_raw[];
  BwdSmem &S = *align1k<BwdSmem>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5;
  load_tile_t(S.W2T, P.W2, kH, kH, kH);
  load_tile_t(S.W3T, P.W3, kH, kH, kH);
  load_tile_t(S.W4T, P.W4, kH, kOutP, 2);
  if (tid == 0) {
    S.err = 0;
    mbar_init(&S.mbar, 1);
  }
  if (warp == 0) {
    tmem_alloc(&S.tmem, 128);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem;
  const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
  uint32_t phase = 0;
  const int64_t ntiles = (M + 127) / 128;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t row = tile * 128 + tid;
    const bool valid = row < M;
    {
      float v[kOutP];
#pragma unroll
      for (int k = 0; k < kOutP; ++k) v[k] = 0.0f;
      if (valid) {
        v[0] = dout[2 * row];
        v[1] = dout[2 * row + 1];
      }
      put8(S.A, tid, 0, kOutP, v);
      put8(S.A, tid, 8, kOutP, v + 8);
    }
    bool ok = bwd_mma(S, tmem, S.A, S.W4T, kOutP, phase, spin);
    const __nv_bfloat16 *Zs[3] = {Z3, Z2, Z1};
    __nv_bfloat16 *dZs[3] = {dZ3, dZ2, dZ1};
    const __nv_bfloat16 *Bs[2] = {S.W3T, S.W2T};
    for (int l = 0; l < 3; ++l) {
#pragma unroll 1
      for (int c = 0; c < kH; c += 32) {
        uint32_t r[32];
        TL_TMEM_LD_X32(trow + (uint32_t)c, r);
        tmem_wait_ld();
        float g[32];
        __align__(16) __nv_bfloat16 zb[32];
        if (valid) {
          const uint4 *src = reinterpret_cast<const uint4 *>(Zs[l] + row * kH + c);
#pragma unroll
          for (int q = 0; q < 4; ++q) reinterpret_cast<uint4 *>(zb)[q] = src[q];
        }
#pragma unroll
        for (int j = 0; j < 32; ++j)
          g[j] = valid ? __uint_as_float(r[j]) * gelu_grad(__bfloat162float(zb[j])) : 0.0f;
        if (valid) {
          __align__(16) __nv_bfloat16 gb[32];
#pragma unroll
          for (int j = 0; j < 32; ++j) gb[j] = __float2bfloat16(g[j]);
          uint4 *dst = reinterpret_cast<uint4 *>(dZs[l] + row * kH + c);
#pragma unroll
          for (int q = 0; q < 4; ++q) dst[q] = reinterpret_cast<const uint4 *>(gb)[q];
        }
        if (l < 2) {
#pragma unroll
          for (int q = 0; q < 32; q += 8) put8(S.A, tid, c + q, kH, g + q);
        }
      }
      if (l < 2) ok = bwd_mma(S, tmem, S.A, Bs[l], kH, phase, spin) && ok;
    }
    if (!ok) S.err = 1;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 128);
  if (tid == 0 && S.err) atomicOr(err, 1);
}

// ---------------------------------------------------------------- weight gradients

// Weight gradients on the tensor cores: dW[o][i] = sum_r G[r][o] H[r][i] is a
// 128 x N x K tile product with the batch rows as K.  A block reduces a range
// of rows, 128 at a time: it stages A = G^T (one output per tile row) and
// B = H^T (one input per tile row) as K-major core tiles, and one thread
// issues the MMAs into an FP32 accumulator in tensor memory that stays there
// for all of the block's rows; the block then writes its partial dW to its
// own slice of a partials buffer, and k_mlp_wsum adds the slices in block
// order, so the gradient (and training) is reproducible bit for bit.  H is
// what the forward products consumed: the
// BF16 normalised features (layer 1) or BF16 GELU(Z) (layers 2-4).  The bias
// gradient db[o] = sum_r G[r][o] is summed from the staged tile.  Layer 4 has
// 2 outputs, too few for a 128-row tile, so its product runs transposed:
// A = GELU(Z3)^T (the 128 inputs as tile rows), B = dout^T (2 outputs padded
// to 16), and the block writes dW4 transposed back.
struct WgSmem {
  __nv_bfloat16 A[128 * 128];
  __nv_bfloat16 B[128 * 128];
  uint64_t mbar;
  uint32_t tmem;
  int err;
};

// MODE 0: layer 1 (G = dZ1, H = features, N = 32); MODE 1: layers 2 and 3
// (G = dZ, H = GELU(Z), N = 128); MODE 2: layer 4 (transposed, N = 16).
template <int MODE>
__global__ void __launch_bounds__(128, 1)
    k_mlp_wgrad_tc(const __nv_bfloat16 *G, const float *dout, const __nv_bfloat16 *Z,
                   const float *x, const float *norm, int64_t M, int64_t chunk, float *dW,
                   float *db, int *err, long long spin) {
  constexpr int N = MODE == 0 ? kInP : (MODE == 1 ? kH : kOutP);
  extern __shared__ unsigned char smem_raw[];
  WgSmem &S = *align1k<WgSmem>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5;
  dW += (size_t)blockIdx.x * kParams;  // this block's slice of the partials
  db += (size_t)blockIdx.x * kParams;
  const int64_t r0 = blockIdx.x * chunk, r1 = min(M, r0 + chunk);
  if (tid == 0) {
    S.err = 0;
    mbar_init(&S.mbar, 1);
  }
  if (warp == 0) {
    tmem_alloc(&S.tmem, 128);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem;
  uint32_t phase = 0;
  bool ok = true;
  float bacc = 0.0f;  // bias gradient of output tid (MODE 0, 1) or tid < 2 (MODE 2)
  for (int64_t rb = r0; rb < r1; rb += 128) {
    // thread tid stages batch row k = tid of this chunk: column k of both tiles
    const int64_t row = rb + tid;
    const bool valid = row < r1;
    if (MODE == 2) {
      // A[i][k] = GELU(Z3[row][i]), B[o][k] = dout[row][o] (o < 2)
      for (int i = 0; i < kH; ++i)
        S.A[core_idx(i, tid, 128)] =
            __float2bfloat16(valid ? gelu(__bfloat162float(Z[row * kH + i])) : 0.0f);
      for (int o = 0; o < kOutP; ++o)
        S.B[core_idx(o, tid, 128)] = __float2bfloat16(valid && o < 2 ? dout[row * 2 + o] : 0.0f);
    } else {
      for (int o = 0; o < kH; ++o)
        S.A[core_idx(o, tid, 128)] = valid ? G[row * kH + o] : __float2bfloat16(0.0f);
      if (MODE == 0) {
        for (int i = 0; i < kInP; ++i)
          S.B[core_idx(i, tid, 128)] = __float2bfloat16(
              valid && i < kIn ? (x[row * kIn + i] - norm[i]) * norm[kIn + i] : 0.0f);
      } else {
        for (int i = 0; i < kH; ++i)
          S.B[core_idx(i, tid, 128)] =
              __float2bfloat16(valid ? gelu(__bfloat162float(Z[row * kH + i])) : 0.0f);
      }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
      gemm_tile(tmem, S.A, S.B, 128, N, rb > r0);
      mma_commit(&S.mbar);
    }
    // the bias gradient from the staged G while the tensor cores work
    if (MODE == 2) {
      if (tid < 2)
        for (int k = 0; k < 128; ++k) bacc += __bfloat162float(S.B[core_idx(tid, k, 128)]);
    } else {
      for (int k = 0; k < 128; ++k) bacc += __bfloat162float(S.A[core_idx(tid, k, 128)]);
    }
    ok = mbar_wait(&S.mbar, phase, spin) && ok;
    phase ^= 1u;
    tc_fence_after();
    __syncthreads();  // the tiles are free again
  }
  // the block's partial dW: thread tid holds accumulator row tid (warp w: rows 32w..)
  const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
  if (MODE == 2) {
    uint32_t r[16];
    TL_TMEM_LD_X16(trow, r);
    tmem_wait_ld();
    for (int o = 0; o < 2; ++o) dW[o * kH + tid] = __uint_as_float(r[o]);
    if (tid < 2) db[tid] = bacc;
  } else {
    constexpr int I = MODE == 0 ? kIn : kH;
#pragma unroll 1
    for (int c = 0; c < N; c += 32) {
      uint32_t r[32];
      TL_TMEM_LD_X32(trow + (uint32_t)c, r);
      tmem_wait_ld();
      for (int j = 0; j < 32; ++j)
        if (c + j < I) dW[tid * I + c + j] = __uint_as_float(r[j]);
    }
    db[tid] = bacc;
  }
  if (!ok) S.err = 1;
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 128);
  if (tid == 0 && S.err) atomicOr(err, 1);
}

// grad[p] = sum over the blocks b (in order) of part[b * kParams + p]: every
// block writes every parameter's entry of its slice
__global__ void __launch_bounds__(256) k_mlp_wsum(const float *part, int blocks, float *grad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kParams) return;
  float acc = 0.0f;
  for (int b = 0; b < blocks; ++b) acc += part[(size_t)b * kParams + p];
  grad[p] = acc;
}

// ---------------------------------------------------------------- optimiser

// AdamW on the flat FP32 parameters (bias-corrected moments, decoupled decay
// on weights only).
__global__ void k_adamw(float *prm, const float *grad, float *m, float *v, int n, float lr,
                        float b1, float b2, float eps, float wd, float c1, float c2) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const float g = grad[t];
  const float mt = b1 * m[t] + (1.0f - b1) * g;
  const float vt = b2 * v[t] + (1.0f - b2) * g * g;
  m[t] = mt;
  v[t] = vt;
  const bool is_bias = (t >= kOffB1 && t < kOffW2) || (t >= kOffB2 && t < kOffW3) ||
                       (t >= kOffB3 && t < kOffW4) || t >= kOffB4;
  float p = prm[t];
  if (!is_bias) p -= lr * wd * p;
  p -= lr * (mt / c1) / (sqrtf(vt / c2) + eps);
  prm[t] = p;
}

// ---------------------------------------------------------------- host side

size_t mlp_fwd_smem() { return sizeof(FwdSmem) + 1024; }
size_t mlp_bwd_smem() { return sizeof(BwdSmem) + 1024; }
size_t mlp_wg_smem() { return sizeof(WgSmem) + 1024; }

cudaError_t mlp_prepare() {
  cudaError_t e = cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)mlp_fwd_smem());
  if (e) return e;
  if ((e = cudaFuncSetAttribute(k_mlp_wgrad_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)mlp_wg_smem())))
    return e;
  if ((e = cudaFuncSetAttribute(k_mlp_wgrad_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)mlp_wg_smem())))
    return e;
  if ((e = cudaFuncSetAttribute(k_mlp_wgrad_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)mlp_wg_smem())))
    return e;
  return cudaFuncSetAttribute(k_mlp_dgrad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)mlp_bwd_smem());
}

cudaError_t mlp_pack(const float *prm, MLPWork &w, cudaStream_t s) {
  k_mlp_pack<<<(kH * kH + 255) / 256, 256, 0, s>>>(prm, w.W1, w.W2, w.W3, w.W4);
  return cudaGetLastError();
}

static MLPDev dev_of(const float *prm, const float *norm, const MLPWork &w) {
  MLPDev P;
  P.W1 = w.W1;
  P.W2 = w.W2;
  P.W3 = w.W3;
  P.W4 = w.W4;
  P.prm = prm;
  P.norm = norm;
  return P;
}

cudaError_t mlp_forward(const float *prm, const float *norm, const MLPWork &w, const float *x,
                        int64_t M, float *out, int blocks, long long spin, cudaStream_t s) {
  if (M <= 0) return cudaSuccess;
  const int64_t tiles = (M + 127) / 128;
  const int g = (int)(tiles < blocks ? tiles : blocks);
  k_mlp_forward<<<g, 128, mlp_fwd_smem(), s>>>(dev_of(prm, norm, w), x, M, out, nullptr, nullptr,
                                               nullptr, nullptr, nullptr, nullptr, 0.f, w.err,
                                               spin, 0, nullptr, 0.f);
  return cudaGetLastError();
}

// loss and gradient of the mean loss over M rows (w.grad, w.loss)
cudaError_t mlp_grad(const float *prm, const float *norm, const MLPWork &w, const float *x,
                     const float *y, int64_t M, int blocks, long long spin, cudaStream_t s,
                     int kind, const float *st, float st_scale) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(w.grad, 0, sizeof(float) * kParams, s))) return e;
  if ((e = cudaMemsetAsync(w.loss, 0, sizeof(float), s))) return e;
  if (M <= 0) return cudaSuccess;
  const int64_t tiles = (M + 127) / 128;
  const int g = (int)(tiles < blocks ? tiles : blocks);
  const MLPDev P = dev_of(prm, norm, w);
  k_mlp_forward<<<g, 128, mlp_fwd_smem(), s>>>(P, x, M, nullptr, y, w.Z[0], w.Z[1], w.Z[2],
                                               w.dout, w.loss, 1.0f / (float)M, w.err, spin, kind,
                                               st, st_scale);
  k_mlp_dgrad<<<g, 128, mlp_bwd_smem(), s>>>(P, w.dout, w.Z[0], w.Z[1], w.Z[2], w.dZ[0], w.dZ[1],
                                             w.dZ[2], M, w.err, spin);
  // weight gradients on the tensor cores: blocks of kWgChunk batch rows, each
  // into its own slice of w.wpart, then summed in block order
  if (M > w.cap) return cudaErrorInvalidValue;
  const int64_t chunk = kWgChunk;
  const unsigned gz = (unsigned)((M + chunk - 1) / chunk);
  float *G = w.wpart;
  const size_t sm = mlp_wg_smem();
  k_mlp_wgrad_tc<2><<<gz, 128, sm, s>>>(nullptr, w.dout, w.Z[2], nullptr, norm, M, chunk,
                                         G + kOffW4, G + kOffB4, w.err, spin);
  k_mlp_wgrad_tc<1><<<gz, 128, sm, s>>>(w.dZ[2], nullptr, w.Z[1], nullptr, norm, M, chunk,
                                         G + kOffW3, G + kOffB3, w.err, spin);
  k_mlp_wgrad_tc<1><<<gz, 128, sm, s>>>(w.dZ[1], nullptr, w.Z[0], nullptr, norm, M, chunk,
                                         G + kOffW2, G + kOffB2, w.err, spin);
  k_mlp_wgrad_tc<0><<<gz, 128, sm, s>>>(w.dZ[0], nullptr, nullptr, x, norm, M, chunk,
                                         G + kOffW1, G + kOffB1, w.err, spin);
  k_mlp_wsum<<<(kParams + 255) / 256, 256, 0, s>>>(w.wpart, (int)gz, w.grad);
  return cudaGetLastError();
}

cudaError_t mlp_adamw(float *prm, const float *grad, float *m, float *v, float lr, float wd,
                      int step, cudaStream_t s) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
  k_adamw<<<(kParams + 255) / 256, 256, 0, s>>>(prm, grad, m, v, kParams, lr, b1, b2, 1e-8f, wd,
                                                 c1, c2);
  return cudaGetLastError();
}

cudaError_t mlp_work_alloc(MLPWork &w, int64_t rows) {
  memset(&w, 0, sizeof(w));
  cudaError_t e;
  if ((e = cudaMalloc((void **)&w.W1, sizeof(__nv_bfloat16) * kH * kInP))) return e;
  if ((e = cudaMalloc((void **)&w.W2, sizeof(__nv_bfloat16) * kH * kH))) return e;
  if ((e = cudaMalloc((void **)&w.W3, sizeof(__nv_bfloat16) * kH * kH))) return e;
  if ((e = cudaMalloc((void **)&w.W4, sizeof(__nv_bfloat16) * kOutP * kH))) return e;
  if ((e = cudaMalloc((void **)&w.grad, sizeof(float) * kParams))) return e;
  if ((e = cudaMalloc((void **)&w.loss, sizeof(float)))) return e;
  if ((e = cudaMalloc((void **)&w.err, sizeof(int)))) return e;
  if ((e = cudaMemset(w.err, 0, sizeof(int)))) return e;
  w.cap = rows;
  if (rows > 0) {
    for (int l = 0; l < 3; ++l) {
      if ((e = cudaMalloc((void **)&w.Z[l], sizeof(__nv_bfloat16) * kH * rows))) return e;
      if ((e = cudaMalloc((void **)&w.dZ[l], sizeof(__nv_bfloat16) * kH * rows))) return e;
    }
    if ((e = cudaMalloc((void **)&w.dout, sizeof(float) * 2 * rows))) return e;
    const int64_t blocks = (rows + kWgChunk - 1) / kWgChunk;
    if ((e = cudaMalloc((void **)&w.wpart, sizeof(float) * kParams * (size_t)blocks))) return e;
  }
  return cudaSuccess;
}

void mlp_work_free(MLPWork &w) {
  cudaFree(w.W1);
  cudaFree(w.W2);
  cudaFree(w.W3);
  cudaFree(w.W4);
  cudaFree(w.grad);
  cudaFree(w.loss);
  cudaFree(w.err);
  for (int l = 0; l < 3; ++l) {
    cudaFree(w.Z[l]);
    cudaFree(w.dZ[l]);
  }
  cudaFree(w.dout);
  cudaFree(w.wpart);
  memset(&w, 0, sizeof(w));
}

}  // namespace tl

// ---------------------------------------------------------------- C ABI

static int mlp_blocks() {
  int dev = 0, sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev);
  return sm > 0 ? sm : 1;
}

extern "C" int trilens_mlp_forward(const float *params, const float *norm, const float *x,
                                   int64_t m, float *out, trilens_stream_t stream) {
  if (!params || !norm || m < 0 || (m > 0 && (!x || !out))) return TRILENS_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  tl::MLPWork w;
  if (tl::mlp_work_alloc(w, 0) || tl::mlp_prepare()) {
    tl::mlp_work_free(w);
    return TRILENS_ERR_CUDA;
  }
  int rc = TRILENS_OK;
  int herr = 0;
  if (tl::mlp_pack(params, w, s) ||
      tl::mlp_forward(params, norm, w, x, m, out, mlp_blocks(), 1ll << 24, s) ||
      cudaMemcpyAsync(&herr, w.err, sizeof(int), cudaMemcpyDeviceToHost, s) ||
      cudaStreamSynchronize(s))
    rc = TRILENS_ERR_CUDA;
  else if (herr)
    rc = TRILENS_ERR_TIMEOUT;
  tl::mlp_work_free(w);
  return rc;
}

extern "C" int trilens_mlp_grad(const float *params, const float *norm, const float *x,
                                const float *y, const float *st, float st_scale, int32_t loss_kind,
                                int64_t m, float *grad, float *loss, trilens_stream_t stream) {
  if (!params || !norm || !grad || !loss || m < 1 || !x || !y) return TRILENS_ERR_INVALID;
  if (loss_kind != 0 && (loss_kind != 1 || !st)) return TRILENS_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  tl::MLPWork w;
  if (tl::mlp_work_alloc(w, m) || tl::mlp_prepare()) {
    tl::mlp_work_free(w);
    return TRILENS_ERR_CUDA;
  }
  int rc = TRILENS_OK;
  int herr = 0;
  if (tl::mlp_pack(params, w, s) ||
      tl::mlp_grad(params, norm, w, x, y, m, mlp_blocks(), 1ll << 24, s, loss_kind, st, st_scale) ||
      cudaMemcpyAsync(grad, w.grad, sizeof(float) * tl::kParams, cudaMemcpyDeviceToDevice, s) ||
      cudaMemcpyAsync(loss, w.loss, sizeof(float), cudaMemcpyDeviceToDevice, s) ||
      cudaMemcpyAsync(&herr, w.err, sizeof(int), cudaMemcpyDeviceToHost, s) ||
      cudaStreamSynchronize(s))
    rc = TRILENS_ERR_CUDA;
  else if (herr)
    rc = TRILENS_ERR_TIMEOUT;
  tl::mlp_work_free(w);
  return rc;
}
