// tl_sur.h -- declarations shared by the surrogate translation units.
#pragma once
#include <cuda_bf16.h>

#include "tl_common.cuh"

namespace tl {

// one hierarchy as the level-L cut and the feature gather see it
struct CutTree {
  const TLNode *nodes;
  const uint32_t *parent_node;  // (parent << 1) | slot of every inner node
  const uint32_t *nfirst;       // first photon of every inner node's range
  const uint8_t *nlev;          // level of every inner node
  const float4 *dir;            // sorted SoA (w = input index)
  const double *pre;            // 6 prefix sums of n + 1 doubles each
  int64_t n;
  uint32_t super;
  int bucket;  // leaf bucket size: inner nodes of at most this many photons are buckets
};

// one breadth-first level of the cut traversal
struct CutArgs {
  CutTree A, B;
  int L;
  const uint2 *in;
  uint2 *out;
  unsigned *counts;  // [0] input count, [1] output count (of this level)
  unsigned cap;
  uint4 *cut;  // (refA, refB, frontier id A, frontier id B)
  unsigned *cut_count;
  unsigned cut_cap;
  unsigned *status;
};

// device workspace of the network
struct MLPWork {
  __nv_bfloat16 *W1, *W2, *W3, *W4;
  __nv_bfloat16 *Z[3], *dZ[3];
  float *dout;
  float *wpart;  // per-block partial weight gradients (rows / 512 slices of all parameters)
  float *grad;
  float *loss;
  int *err;
  int64_t cap;  // rows the training buffers hold
};

cudaError_t launch_prefix_moments(const TLBeam &B, const float4 *pos, const float4 *dir, int64_t n,
                                  double *bsum, double *pre, cudaStream_t s);
cudaError_t launch_cut_level(const CutArgs &a, int blocks, cudaStream_t s);
cudaError_t launch_features(const CutTree &A, const CutTree &B, const uint4 *cut,
                            const unsigned *cut_count, unsigned cap, float *feat, float *st,
                            double dt, double kappa, int blocks, cudaStream_t s);
cudaError_t launch_labels_prep(const CutTree &T, int L, uint32_t *cid_node, uint32_t *cid_slot,
                               uint2 *flist, unsigned *fcount, unsigned fcap, uint32_t *cut_of,
                               uint32_t *inv, cudaStream_t s);
cudaError_t launch_pair_index(const CutTree &A, const CutTree &B, uint4 *cut,
                              const unsigned *cut_count, unsigned cap, const uint32_t *cnA,
                              const uint32_t *csA, const uint32_t *cnB, const uint32_t *csB,
                              unsigned long long *hkey, uint32_t *hval, unsigned hmask,
                              unsigned *status, int blocks, cudaStream_t s);
cudaError_t launch_attribute(const uint2 *hits, const unsigned long long *nhits,
                             unsigned long long hcap, const TLBeam &mA, const TLBeam &mB,
                             const uint32_t *invA, const uint32_t *invB, const uint32_t *cutA,
                             const uint32_t *cutB, const unsigned long long *hkey,
                             const uint32_t *hval, unsigned hmask, double *label,
                             unsigned *status, int blocks, cudaStream_t s);
cudaError_t launch_estimate(const float *out, const float *st, float st_scale, const uint4 *cut,
                            const unsigned *cut_count, unsigned cap, float tau, double *pred,
                            uint2 *fb, unsigned *fb_count, unsigned fb_cap, int blocks,
                            cudaStream_t s, uint8_t *flag = nullptr);
// small helpers: op 0 copies cut refs (uint4 -> uint2), op 1 writes log1p of
// doubles as floats, op 2 / op 3 add n doubles / floats into *c (a double)
cudaError_t launch_sur_misc(int op, const void *a, const void *b, void *c, int64_t n,
                            cudaStream_t s);

cudaError_t mlp_prepare();
cudaError_t mlp_work_alloc(MLPWork &w, int64_t rows);
void mlp_work_free(MLPWork &w);
cudaError_t mlp_pack(const float *prm, MLPWork &w, cudaStream_t s);
cudaError_t mlp_forward(const float *prm, const float *norm, const MLPWork &w, const float *x,
                        int64_t M, float *out, int blocks, long long spin, cudaStream_t s);
cudaError_t mlp_grad(const float *prm, const float *norm, const MLPWork &w, const float *x,
                     const float *y, int64_t M, int blocks, long long spin, cudaStream_t s,
                     int kind, const float *st, float st_scale);
cudaError_t mlp_adamw(float *prm, const float *grad, float *m, float *v, float lr, float wd,
                      int step, cudaStream_t s);

}  // namespace tl
