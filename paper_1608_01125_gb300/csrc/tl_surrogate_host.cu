// tl_surrogate_host.cu -- the learned statistical regime, host side:
// level-L cut of the dual traversal, features, exact labels of node pairs,
// training of the network (tensor-core forward and input-gradient kernels,
// CUDA-core weight gradients, AdamW), and the surrogate step with the exact
// fallback for pairs whose predicted uncertainty is too large.
#include <math.h>

#include <algorithm>
#include <random>
#include <vector>

#include "tl_ctx.h"
#include "tl_sur.h"


constexpr int kBatch = 8192;
constexpr int kTauBins = 64;
// edges of the fallback-threshold bins of the calibration table: 2^(g/2 - 10)
static inline double tau_edge(int g) { return std::ldexp(1.0, -10) * std::pow(2.0, 0.5 * g); }

struct SurrogateState {
  // model
  float *prm = nullptr, *mom1 = nullptr, *mom2 = nullptr, *norm = nullptr;
  tl::MLPWork work{};
  bool trained = false;
  int level = -1;
  double calib = 1.0, st_calib = 1.0, st_only_calib = 1.0;
  // calibration by fallback threshold: cal_tau[g] is the calibration of the
  // training pairs whose predicted spread is at most kTauEdge(g) (the pairs the
  // network keeps at that threshold; the others are evaluated exactly)
  double cal_tau[64];
  int adam_step = 0;
  // per-step buffers
  double *pre[2]{}, *bsum[2]{};
  uint2 *lvl[2]{};
  unsigned lvl_cap = 0;
  unsigned *lcount = nullptr;  // device, per level
  uint4 *cut = nullptr;
  unsigned cut_cap = 0;
  unsigned *cut_count = nullptr;
  unsigned *status = nullptr;
  float *feat = nullptr, *st = nullptr, *out = nullptr;
  double *pred = nullptr, *scal = nullptr;
  uint2 *fb = nullptr, *seeds = nullptr;
  unsigned *fb_count = nullptr;
  // labels
  uint32_t *cid_node[2]{}, *cid_slot[2]{}, *cut_of[2]{}, *inv[2]{};
  uint2 *flist[2]{};
  unsigned *fcount = nullptr;
  unsigned fcap = 0;
  unsigned long long *hkey = nullptr;
  uint32_t *hval = nullptr;
  unsigned hmask = 0;
  double *label = nullptr;
  // training set
  float *tx = nullptr, *ty = nullptr, *tst = nullptr;
  double *tlab = nullptr;
  int64_t tn = 0, tcap = 0;
  double last_loss = 0.0;
  // cumulative surrogate totals
  double tot = 0.0;
};

static void sfree(SurrogateState *s) {
  cudaFree(s->prm);
  cudaFree(s->mom1);
  cudaFree(s->mom2);
  cudaFree(s->norm);
  tl::mlp_work_free(s->work);
  for (int k = 0; k < 2; ++k) {
    cudaFree(s->pre[k]);
    cudaFree(s->bsum[k]);
    cudaFree(s->lvl[k]);
    cudaFree(s->cid_node[k]);
    cudaFree(s->cid_slot[k]);
    cudaFree(s->cut_of[k]);
    cudaFree(s->inv[k]);
    cudaFree(s->flist[k]);
  }
  cudaFree(s->lcount);
  cudaFree(s->cut);
  cudaFree(s->cut_count);
  cudaFree(s->status);
  cudaFree(s->feat);
  cudaFree(s->st);
  cudaFree(s->out);
  cudaFree(s->pred);
  cudaFree(s->scal);
  cudaFree(s->fb);
  cudaFree(s->seeds);
  cudaFree(s->fb_count);
  cudaFree(s->fcount);
  cudaFree(s->hkey);
  cudaFree(s->hval);
  cudaFree(s->label);
  cudaFree(s->tx);
  cudaFree(s->ty);
  cudaFree(s->tst);
  cudaFree(s->tlab);
}

void surrogate_free(trilens_ctx *c) {
  if (c && c->sur) {
    sfree(c->sur);
    delete c->sur;
    c->sur = nullptr;
  }
}

static int cut_buffers(trilens_ctx *c, unsigned cap) {
  SurrogateState *s = c->sur;
  for (int k = 0; k < 2; ++k) {
    cudaFree(s->lvl[k]);
    s->lvl[k] = nullptr;
  }
  cudaFree(s->cut);
  cudaFree(s->feat);
  cudaFree(s->st);
  cudaFree(s->out);
  cudaFree(s->pred);
  cudaFree(s->fb);
  cudaFree(s->seeds);
  cudaFree(s->label);
  cudaFree(s->hkey);
  cudaFree(s->hval);
  s->cut = nullptr;
  s->cut_cap = cap;
  s->lvl_cap = 2 * cap;
  for (int k = 0; k < 2; ++k) CK(dalloc(&s->lvl[k], s->lvl_cap));
  CK(dalloc(&s->cut, cap));
  CK(dalloc(&s->feat, (size_t)cap * 24));
  CK(dalloc(&s->st, cap));
  CK(dalloc(&s->out, (size_t)cap * 2));
  CK(dalloc(&s->pred, cap));
  CK(dalloc(&s->fb, cap));
  CK(dalloc(&s->seeds, cap));
  CK(dalloc(&s->label, cap));
  unsigned hs = 1;
  while (hs < 2 * cap) hs <<= 1;
  s->hmask = hs - 1;
  CK(dalloc(&s->hkey, hs));
  CK(dalloc(&s->hval, hs));
  return TRILENS_OK;
}

static int ensure_state(trilens_ctx *c) {
  if (c->sur) return TRILENS_OK;
  c->sur = new SurrogateState();
  SurrogateState *s = c->sur;
  CK(tl::mlp_prepare());
  CK(dalloc(&s->prm, TRILENS_MLP_PARAMS));
  CK(dalloc(&s->mom1, TRILENS_MLP_PARAMS));
  CK(dalloc(&s->mom2, TRILENS_MLP_PARAMS));
  CK(dalloc(&s->norm, 48));
  CK(tl::mlp_work_alloc(s->work, kBatch));
  for (int k = 0; k < 2; ++k) {
    const int64_t n = std::max<int64_t>(c->beam[k].n, 1);
    CK(dalloc(&s->pre[k], (size_t)6 * (n + 1)));
    CK(dalloc(&s->bsum[k], (size_t)6 * ((n + 1023) / 1024 + 1)));
    CK(dalloc(&s->cid_node[k], (size_t)n));
    CK(dalloc(&s->cid_slot[k], (size_t)2 * n));
    CK(dalloc(&s->cut_of[k], (size_t)n));
    CK(dalloc(&s->inv[k], (size_t)n));
  }
  s->fcap = (unsigned)std::min<int64_t>(std::max(c->beam[0].n, c->beam[1].n) + 16, 1ll << 30);
  for (int k = 0; k < 2; ++k) CK(dalloc(&s->flist[k], s->fcap));
  CK(dalloc(&s->lcount, 256));
  CK(dalloc(&s->cut_count, 1));
  CK(dalloc(&s->status, 1));
  CK(dalloc(&s->fb_count, 1));
  CK(dalloc(&s->fcount, 2));
  CK(dalloc(&s->scal, 4));
  return cut_buffers(c, 1u << 20);
}

static tl::CutTree cut_tree(trilens_ctx *c, int k) {
  tl::CutTree t;
  t.nodes = c->w[k].nodes;
  t.parent_node = c->w[k].parent_node;
  t.nfirst = c->w[k].nfirst;
  t.nlev = c->w[k].nlev;
  t.dir = c->w[k].dir;
  t.pre = c->sur->pre[k];
  t.n = c->beam[k].n;
  t.super = (uint32_t)(t.n > 1 ? t.n - 1 : 0);
  t.bucket = c->p.leaf_bucket;
  return t;
}

// moments, level-L cut pairs and their features for the built step
static int sur_cut(trilens_ctx *c, int L, unsigned *ncut) {
  SurrogateState *s = c->sur;
  for (int attempt = 0; attempt < 6; ++attempt) {
    for (int k = 0; k < 2; ++k)
      CK(tl::launch_prefix_moments(c->beam[k], c->w[k].pos, c->w[k].dir, c->beam[k].n, s->bsum[k],
                                   s->pre[k], c->stream));
    CK(cudaMemsetAsync(s->lcount, 0, sizeof(unsigned) * 256, c->stream));
    CK(cudaMemsetAsync(s->cut_count, 0, sizeof(unsigned), c->stream));
    CK(cudaMemsetAsync(s->status, 0, sizeof(unsigned), c->stream));
    const uint2 root = make_uint2((uint32_t)(c->beam[0].n > 1 ? c->beam[0].n - 1 : 0),
                                  (uint32_t)(c->beam[1].n > 1 ? c->beam[1].n - 1 : 0));
    const unsigned one = (c->beam[0].n > 0 && c->beam[1].n > 0) ? 1u : 0u;
    CK(cudaMemcpyAsync(s->lvl[0], &root, sizeof(uint2), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(s->lcount, &one, sizeof(unsigned), cudaMemcpyHostToDevice, c->stream));
    tl::CutArgs a;
    a.A = cut_tree(c, 0);
    a.B = cut_tree(c, 1);
    a.L = L;
    a.cap = s->lvl_cap;
    a.cut = s->cut;
    a.cut_count = s->cut_count;
    a.cut_cap = s->cut_cap;
    a.status = s->status;
    int level = 0;
    unsigned left = one;
    while (left > 0 && level < 250) {
      for (int q = 0; q < 8 && level < 250; ++q, ++level) {
        a.in = s->lvl[level & 1];
        a.out = s->lvl[(level + 1) & 1];
        a.counts = s->lcount + level;
        CK(tl::launch_cut_level(a, 4 * c->n_sm, c->stream));
      }
      CK(cudaMemcpyAsync(&left, s->lcount + level, sizeof(unsigned), cudaMemcpyDeviceToHost,
                         c->stream));
      CK(cudaStreamSynchronize(c->stream));
    }
    unsigned st = 0;
    CK(cudaMemcpyAsync(ncut, s->cut_count, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&st, s->status, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(c->build_status_host, c->build_status, sizeof(unsigned),
                       cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    const unsigned bst = *c->build_status_host;
    if (bst & (TL_ST_TIMEOUT | TL_ST_BADTREE)) {  // the hierarchy of this step is invalid
      c->w[0].sort_epoch = c->w[1].sort_epoch = 0;
      CK(cudaMemsetAsync(c->build_status, 0, sizeof(unsigned), c->stream));
      CK(cudaStreamSynchronize(c->stream));
      if (bst & TL_ST_TIMEOUT)
        return fail(c, TRILENS_ERR_TIMEOUT, "a device wait of the build reached spin_limit");
      return fail(c, TRILENS_ERR_CUDA, "the refit met a node reference out of range (internal error)");
    }
    if (left > 0) return fail(c, TRILENS_ERR_STACK, "cut traversal did not finish");
    if (!(st & TL_ST_FRONT_OVF)) {
      CK(tl::launch_features(a.A, a.B, s->cut, s->cut_count, s->cut_cap, s->feat, s->st,
                             c->p.dt_fs, c->p.kappa, 4 * c->n_sm, c->stream));
      return TRILENS_OK;
    }
    int rc = cut_buffers(c, std::max(2 * s->cut_cap, *ncut + (*ncut >> 2) + 1024));
    if (rc) return rc;
  }
  return fail(c, TRILENS_ERR_STACK, "cut lists kept overflowing");
}

// ids of the level-L frontier nodes of both trees (every photon's id in
// cut_of, the input -> sorted map in inv) and of every cut pair (cut[p].z,
// cut[p].w), with the pairs' hash index
static int sur_ids(trilens_ctx *c, int L) {
  SurrogateState *s = c->sur;
  tl::CutTree A = cut_tree(c, 0), B = cut_tree(c, 1);
  CK(cudaMemsetAsync(s->fcount, 0, sizeof(unsigned) * 2, c->stream));
  CK(cudaMemsetAsync(s->status, 0, sizeof(unsigned), c->stream));
  for (int k = 0; k < 2; ++k) {
    if (c->beam[k].n <= 0) continue;
    CK(tl::launch_labels_prep(k ? B : A, L, s->cid_node[k], s->cid_slot[k], s->flist[k],
                              s->fcount + k, s->fcap, s->cut_of[k], s->inv[k], c->stream));
  }
  CK(cudaMemsetAsync(s->hkey, 0xff, sizeof(unsigned long long) * (s->hmask + 1ull), c->stream));
  CK(tl::launch_pair_index(A, B, s->cut, s->cut_count, s->cut_cap, s->cid_node[0], s->cid_slot[0],
                           s->cid_node[1], s->cid_slot[1], s->hkey, s->hval, s->hmask, s->status,
                           4 * c->n_sm, c->stream));
  return TRILENS_OK;
}

// exact yield of every cut pair (label[p]) for the built step; returns the
// step's exact total through *total
static int sur_labels(trilens_ctx *c, int L, double ct, unsigned ncut, double *total) {
  SurrogateState *s = c->sur;
  int rc0 = sur_ids(c, L);
  if (rc0) return rc0;
  // the cut pairs' node references seed the exact traversal
  CK(tl::launch_sur_misc(0, s->cut, nullptr, s->seeds, ncut, c->stream));
  int retries = 0;
  int rc = run_exact(c, ct, s->seeds, ncut, &retries);
  if (rc) return rc;
  *total = c->ctr_host->weighted;
  CK(cudaMemsetAsync(s->label, 0, sizeof(double) * std::max(ncut, 1u), c->stream));
  CK(tl::launch_attribute(c->hits, &c->ctr->hits, c->hit_cap, c->beam[0], c->beam[1], s->inv[0],
                          s->inv[1], s->cut_of[0], s->cut_of[1], s->hkey, s->hval, s->hmask,
                          s->label, s->status, 4 * c->n_sm, c->stream));
  unsigned st = 0;
  CK(cudaMemcpyAsync(&st, s->status, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (st & TL_ST_FRONT_OVF) return fail(c, TRILENS_ERR_STACK, "a hit outside the cut pairs");
  return TRILENS_OK;
}

static int append_samples(trilens_ctx *c, unsigned ncut) {
  SurrogateState *s = c->sur;
  if (s->tn + ncut > s->tcap) {
    const int64_t nc = std::max<int64_t>(2 * s->tcap, s->tn + ncut + 65536);
    float *tx, *ty, *tst;
    double *tlab;
    CK(dalloc(&tx, (size_t)nc * 24));
    CK(dalloc(&ty, (size_t)nc));
    CK(dalloc(&tst, (size_t)nc));
    CK(dalloc(&tlab, (size_t)nc));
    if (s->tn) {
      CK(cudaMemcpyAsync(tx, s->tx, sizeof(float) * 24 * s->tn, cudaMemcpyDeviceToDevice, c->stream));
      CK(cudaMemcpyAsync(ty, s->ty, sizeof(float) * s->tn, cudaMemcpyDeviceToDevice, c->stream));
      CK(cudaMemcpyAsync(tst, s->tst, sizeof(float) * s->tn, cudaMemcpyDeviceToDevice, c->stream));
      CK(cudaMemcpyAsync(tlab, s->tlab, sizeof(double) * s->tn, cudaMemcpyDeviceToDevice, c->stream));
      CK(cudaStreamSynchronize(c->stream));
    }
    cudaFree(s->tx);
    cudaFree(s->ty);
    cudaFree(s->tst);
    cudaFree(s->tlab);
    s->tx = tx;
    s->ty = ty;
    s->tst = tst;
    s->tlab = tlab;
    s->tcap = nc;
  }
  CK(cudaMemcpyAsync(s->tx + 24 * s->tn, s->feat, sizeof(float) * 24 * ncut, cudaMemcpyDeviceToDevice,
                     c->stream));
  CK(cudaMemcpyAsync(s->tst + s->tn, s->st, sizeof(float) * ncut, cudaMemcpyDeviceToDevice,
                     c->stream));
  CK(cudaMemcpyAsync(s->tlab + s->tn, s->label, sizeof(double) * ncut, cudaMemcpyDeviceToDevice,
                     c->stream));
  CK(tl::launch_sur_misc(1, s->label, nullptr, s->ty + s->tn, ncut, c->stream));  // log1p
  s->tn += ncut;
  return TRILENS_OK;
}

// sum of n doubles (op 2) or floats (op 3) into *host
static int dsum(trilens_ctx *c, int op, const void *x, int64_t n, double *host) {
  SurrogateState *s = c->sur;
  CK(cudaMemsetAsync(s->scal, 0, sizeof(double), c->stream));
  CK(tl::launch_sur_misc(op, x, nullptr, s->scal, n, c->stream));
  CK(cudaMemcpyAsync(host, s->scal, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return TRILENS_OK;
}

extern "C" {

int trilens_surrogate_collect(trilens_ctx *c, const int64_t *steps, int32_t n, int32_t level_L) {
  if (!c || !steps || n < 1 || level_L < 1 || level_L > 63) return TRILENS_ERR_INVALID;
  if (c->n_inst > 1) return fail(c, TRILENS_ERR_INVALID, "surrogate on a batch context");
  CK(cudaSetDevice(c->device));
  int rc = ensure_state(c);
  if (rc) return rc;
  SurrogateState *s = c->sur;
  if (s->level >= 0 && s->level != level_L && s->tn > 0)
    return fail(c, TRILENS_ERR_INVALID, "samples of another level are collected");
  s->level = level_L;
  const double keep_c = c->tot_count, keep_w = c->tot_weighted;
  for (int i = 0; i < n; ++i) {
    if ((rc = trilens_build(c, steps[i]))) return rc;
    unsigned ncut = 0;
    if ((rc = sur_cut(c, level_L, &ncut))) return rc;
    if (ncut == 0) continue;
    double total = 0.0;
    if ((rc = sur_labels(c, level_L, TL_C * ((double)steps[i] * c->p.dt_fs), ncut, &total)))
      return rc;
    if ((rc = append_samples(c, ncut))) return rc;
  }
  c->tot_count = keep_c;
  c->tot_weighted = keep_w;
  return TRILENS_OK;
}

int trilens_surrogate_fit(trilens_ctx *c, int32_t epochs, uint64_t seed) {
  if (!c || !c->sur || c->sur->tn < 1 || epochs < 1) return TRILENS_ERR_INVALID;
  CK(cudaSetDevice(c->device));
  SurrogateState *s = c->sur;
  const int64_t N = s->tn;
  // feature normalisation from the samples
  std::vector<float> hx((size_t)N * 24), hy((size_t)N), hst((size_t)N);
  std::vector<double> hlab((size_t)N);
  CK(cudaMemcpy(hx.data(), s->tx, sizeof(float) * 24 * N, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(hst.data(), s->tst, sizeof(float) * N, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(hlab.data(), s->tlab, sizeof(double) * N, cudaMemcpyDeviceToHost));
  // samples in random order; all of them train the network and fit the
  // scales (a random subset would not do: the yield is concentrated in a few
  // core pairs, so the ratio of sums over a subset is noisy)
  std::mt19937_64 rng(seed);
  std::vector<int64_t> perm((size_t)N);
  for (int64_t i = 0; i < N; ++i) perm[i] = i;
  std::shuffle(perm.begin(), perm.end(), rng);
  const int64_t Ntr = N;
  // the ST-form estimate's scale (from the training part), then the
  // network's target: the residual y = log1p(label) - log1p(scale * st)
  {
    double ls = 0, ss = 0;
    for (int64_t q = 0; q < Ntr; ++q) {
      ls += hlab[perm[q]];
      ss += hst[perm[q]];
    }
    s->st_calib = ss > 0 ? ls / ss : 1.0;
    for (int64_t i = 0; i < N; ++i) hy[i] = (float)hlab[i];  // the linear label
  }
  float hn[48];
  for (int k = 0; k < 24; ++k) {
    double m = 0, v = 0;
    for (int64_t i = 0; i < N; ++i) m += hx[i * 24 + k];
    m /= (double)N;
    for (int64_t i = 0; i < N; ++i) v += (hx[i * 24 + k] - m) * (hx[i * 24 + k] - m);
    v /= (double)N;
    hn[k] = (float)m;
    hn[24 + k] = v > 1e-20 ? (float)(1.0 / sqrt(v)) : 1.0f;
  }
  CK(cudaMemcpy(s->norm, hn, sizeof(hn), cudaMemcpyHostToDevice));
  // initial parameters (He initialisation; output bias at the target mean)
  std::normal_distribution<double> nd(0.0, 1.0);
  std::vector<float> p(TRILENS_MLP_PARAMS, 0.0f);
  auto fill = [&](int off, int rows, int cols) {
    const double sd = sqrt(2.0 / cols);
    for (int i = 0; i < rows * cols; ++i) p[off + i] = (float)(nd(rng) * sd);
  };
  fill(0, 128, 24);
  fill(128 * 24 + 128, 128, 128);
  fill(128 * 24 + 128 + 128 * 128 + 128, 128, 128);
  const int offW4 = 128 * 24 + 128 + 2 * (128 * 128 + 128);
  for (int i = 0; i < 2 * 128; ++i) p[offW4 + i] = (float)(nd(rng) * 0.01);
  {  // start at the calibrated baseline: mu = ln(sum Y / sum (B + 1))
    double ys = 0, bs = 0;
    for (int64_t q = 0; q < Ntr; ++q) {
      ys += hy[perm[q]];
      bs += s->st_calib * hst[perm[q]] + 1.0;
    }
    p[offW4 + 256] = (float)(ys > 0 && bs > 0 ? log(ys / bs) : 0.0);
    p[offW4 + 257] = 0.0f;
  }
  CK(cudaMemcpy(s->prm, p.data(), sizeof(float) * TRILENS_MLP_PARAMS, cudaMemcpyHostToDevice));
  CK(cudaMemset(s->mom1, 0, sizeof(float) * TRILENS_MLP_PARAMS));
  CK(cudaMemset(s->mom2, 0, sizeof(float) * TRILENS_MLP_PARAMS));
  s->adam_step = 0;
  // shuffled copy of the samples (training part first, held-out part last)
  std::vector<float> sx((size_t)N * 24), sy((size_t)N), sst((size_t)N);
  std::vector<double> slab((size_t)N);
  for (int64_t i = 0; i < N; ++i) {
    for (int k = 0; k < 24; ++k) sx[i * 24 + k] = hx[perm[i] * 24 + k];
    sy[i] = hy[perm[i]];
    sst[i] = hst[perm[i]];
    slab[i] = hlab[perm[i]];
  }
  float *dx = nullptr, *dy = nullptr, *dst = nullptr;
  double *dlab = nullptr;
  CK(dalloc(&dx, (size_t)N * 24));
  CK(dalloc(&dy, (size_t)N));
  CK(dalloc(&dst, (size_t)N));
  CK(dalloc(&dlab, (size_t)N));
  CK(cudaMemcpy(dx, sx.data(), sizeof(float) * 24 * N, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(dy, sy.data(), sizeof(float) * N, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(dst, sst.data(), sizeof(float) * N, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(dlab, slab.data(), sizeof(double) * N, cudaMemcpyHostToDevice));
  const int64_t nb = (Ntr + kBatch - 1) / kBatch;
  const int64_t total_steps = nb * epochs;
  const float lr0 = 2e-3f, lr1 = 5e-5f;
  int rc = TRILENS_OK;
  for (int e = 0; e < epochs && !rc; ++e) {
    double lsum = 0;
    for (int64_t b = 0; b < nb; ++b) {
      const int64_t r0 = b * kBatch, m = std::min<int64_t>(kBatch, Ntr - r0);
      const double t = (double)s->adam_step / (double)std::max<int64_t>(total_steps - 1, 1);
      const float lr = (float)(lr1 + 0.5 * (lr0 - lr1) * (1.0 + cos(3.14159265358979323846 * t)));
      if (tl::mlp_pack(s->prm, s->work, c->stream) ||
          tl::mlp_grad(s->prm, s->norm, s->work, dx + 24 * r0, dy + r0, m, c->n_sm,
                       c->p.spin_limit, c->stream, 1, dst + r0, (float)s->st_calib) ||
          tl::mlp_adamw(s->prm, s->work.grad, s->mom1, s->mom2, lr, 1e-4f, ++s->adam_step,
                        c->stream)) {
        rc = fail(c, TRILENS_ERR_CUDA, "training step failed");
        break;
      }
      if (b == nb - 1 || (b & 63) == 63) {
        float l = 0;
        cudaMemcpyAsync(&l, s->work.loss, sizeof(float), cudaMemcpyDeviceToHost, c->stream);
        cudaStreamSynchronize(c->stream);
        lsum = l / (double)m;
      }
    }
    s->last_loss = lsum;
  }
  int herr = 0;
  if (!rc) {
    CK(cudaMemcpy(&herr, s->work.err, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr) rc = fail(c, TRILENS_ERR_TIMEOUT, "a tensor-core wait ran out during training");
  }
  // calibration of the summed estimates on the samples (for the network,
  // whose objective has an intercept, it stays close to 1)
  const int64_t c0 = 0;
  double lab = 0, est = 0, stsum = 0;
  std::vector<double> bl(kTauBins + 1, 0.0), be(kTauBins + 1, 0.0);  // per spread bin
  std::vector<float> hout;
  std::vector<double> hpred, hlb;
  if (!rc && tl::mlp_pack(s->prm, s->work, c->stream)) rc = fail(c, TRILENS_ERR_CUDA, "pack");
  for (int64_t r0 = c0; !rc && r0 < N; r0 += s->cut_cap) {
    const int64_t m = std::min<int64_t>(s->cut_cap, N - r0);
    const unsigned mm = (unsigned)m;
    double a = 0, b = 0, d = 0;
    if (tl::mlp_forward(s->prm, s->norm, s->work, dx + 24 * r0, m, s->out, c->n_sm,
                        c->p.spin_limit, c->stream) ||
        cudaMemcpyAsync(s->cut_count, &mm, sizeof(unsigned), cudaMemcpyHostToDevice, c->stream) ||
        cudaMemsetAsync(s->fb_count, 0, sizeof(unsigned), c->stream) ||
        tl::launch_estimate(s->out, dst + r0, (float)s->st_calib, s->cut, s->cut_count,
                            s->cut_cap, 1e30f, s->pred, s->fb, s->fb_count, s->cut_cap,
                            4 * c->n_sm, c->stream)) {
      rc = fail(c, TRILENS_ERR_CUDA, "calibration pass failed");
      break;
    }
    if ((rc = dsum(c, 2, s->pred, m, &a)) || (rc = dsum(c, 2, dlab + r0, m, &b)) ||
        (rc = dsum(c, 3, dst + r0, m, &d)))
      break;
    est += a;
    lab += b;
    stsum += d;
    // the same sums split by predicted spread (in sample order: deterministic)
    hout.resize(2 * (size_t)m);
    hpred.resize((size_t)m);
    hlb.resize((size_t)m);
    if (cudaMemcpy(hout.data(), s->out, sizeof(float) * 2 * m, cudaMemcpyDeviceToHost) ||
        cudaMemcpy(hpred.data(), s->pred, sizeof(double) * m, cudaMemcpyDeviceToHost) ||
        cudaMemcpy(hlb.data(), dlab + r0, sizeof(double) * m, cudaMemcpyDeviceToHost)) {
      rc = fail(c, TRILENS_ERR_CUDA, "calibration copy failed");
      break;
    }
    for (int64_t q = 0; q < m; ++q) {
      const float sv = std::fmin(std::fmax(hout[2 * q + 1], -12.f), 12.f);
      const double spread = std::sqrt(std::exp((double)sv));
      int g = 0;
      while (g < kTauBins && spread > tau_edge(g)) ++g;  // bin kTauBins: above every edge
      bl[g] += hlb[q];
      be[g] += hpred[q];
    }
  }
  cudaFree(dx);
  cudaFree(dy);
  cudaFree(dst);
  cudaFree(dlab);
  if (rc) return rc;
  s->calib = est > 0 ? lab / est : 1.0;
  {  // the pairs with spread <= edge g: bins 0..g
    double cl = 0, ce = 0;
    for (int g = 0; g < kTauBins; ++g) {
      cl += bl[g];
      ce += be[g];
      s->cal_tau[g] = ce > 0 ? cl / ce : s->calib;
    }
  }
  // the ST-form estimator alone (the network keeps the baseline scale it was
  // trained with; over all samples the two agree)
  s->st_only_calib = stsum > 0 ? lab / stsum : s->st_calib;
  s->trained = true;
  return TRILENS_OK;
}

int trilens_surrogate_train(trilens_ctx *c, const int64_t *train_steps, int32_t n, int32_t level_L,
                            int32_t epochs, uint64_t seed) {
  int rc = trilens_surrogate_collect(c, train_steps, n, level_L);
  if (rc) return rc;
  return trilens_surrogate_fit(c, epochs, seed);
}

int trilens_surrogate_step(trilens_ctx *c, int64_t step, int32_t level_L, float tau,
                           double out[8]) {
  if (!c || !out || !c->sur || !c->sur->trained) return TRILENS_ERR_INVALID;
  if (step != c->built_step) return fail(c, TRILENS_ERR_INVALID, "step not built");
  if (level_L != c->sur->level) return fail(c, TRILENS_ERR_INVALID, "model trained at another L");
  CK(cudaSetDevice(c->device));
  SurrogateState *s = c->sur;
  cudaEvent_t e0, e1, e2;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventCreate(&e2));
  CK(cudaEventRecord(e0, c->stream));
  unsigned ncut = 0;
  int rc = sur_cut(c, level_L, &ncut);
  if (rc) return rc;
  CK(cudaEventRecord(e1, c->stream));
  CK(tl::mlp_pack(s->prm, s->work, c->stream));
  CK(tl::mlp_forward(s->prm, s->norm, s->work, s->feat, ncut, s->out, c->n_sm, c->p.spin_limit,
                     c->stream));
  CK(cudaMemsetAsync(s->fb_count, 0, sizeof(unsigned), c->stream));
  CK(tl::launch_estimate(s->out, s->st, (float)s->st_calib, s->cut, s->cut_count, s->cut_cap, tau,
                         s->pred, s->fb, s->fb_count, s->cut_cap, 4 * c->n_sm, c->stream));
  CK(cudaEventRecord(e2, c->stream));
  unsigned nfb = 0;
  CK(cudaMemcpyAsync(&nfb, s->fb_count, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
  double est = 0, st = 0;
  if ((rc = dsum(c, 2, s->pred, ncut, &est)) || (rc = dsum(c, 3, s->st, ncut, &st))) return rc;
  double fb_exact = 0;
  if (nfb > 0) {
    const double keep_c = c->tot_count, keep_w = c->tot_weighted;
    int retries = 0;
    if ((rc = run_exact(c, TL_C * ((double)step * c->p.dt_fs), s->fb, nfb, &retries))) return rc;
    fb_exact = c->ctr_host->weighted;
    c->tot_count = keep_c;
    c->tot_weighted = keep_w;
  }
  CK(cudaStreamSynchronize(c->stream));
  float ms_all = 0, ms_cut = 0;
  cudaEvent_t e3;
  CK(cudaEventCreate(&e3));
  CK(cudaEventRecord(e3, c->stream));
  CK(cudaEventSynchronize(e3));
  CK(cudaEventElapsedTime(&ms_all, e0, e3));
  CK(cudaEventElapsedTime(&ms_cut, e0, e1));
  float ms_mlp = 0;
  CK(cudaEventElapsedTime(&ms_mlp, e1, e2));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaEventDestroy(e2);
  cudaEventDestroy(e3);
  // the calibration of the pairs the network keeps at this threshold
  double cal = s->calib;
  for (int g = kTauBins - 1; g >= 0; --g)
    if (tau_edge(g) <= (double)tau) {
      if (g < kTauBins - 1) cal = s->cal_tau[g];
      break;
    }
  const double yield = cal * est + fb_exact;
  s->tot += yield;
  out[0] = yield;                 // surrogate estimate of the step's weighted yield
  out[1] = st;                    // the ST rate of the same pairs (no network, no scale)
  out[2] = (double)ncut;          // node pairs at level L
  out[3] = (double)nfb;           // pairs sent to the exact fallback
  out[4] = fb_exact;              // their exact yield
  out[5] = ms_all;                // device time of the whole surrogate path [ms]
  out[6] = ms_mlp;                // network + estimate [ms]
  out[7] = ms_cut;                // cut traversal + features [ms]
  return TRILENS_OK;
}

int trilens_surrogate_pairs(trilens_ctx *c, int64_t step, int32_t level_L, float tau,
                            trilens_sur_pairs *o) {
  if (!c || !o || o->cap < 0 || level_L < 1 || level_L > 63) return TRILENS_ERR_INVALID;
  if (c->n_inst > 1) return fail(c, TRILENS_ERR_INVALID, "surrogate on a batch context");
  if (step != c->built_step) return fail(c, TRILENS_ERR_INVALID, "step not built");
  const bool want_net = o->pred || o->fallback || o->net;
  if (want_net && (!c->sur || !c->sur->trained || c->sur->level != level_L))
    return fail(c, TRILENS_ERR_INVALID, "no surrogate model for level %d", level_L);
  CK(cudaSetDevice(c->device));
  int rc = ensure_state(c);
  if (rc) return rc;
  SurrogateState *s = c->sur;
  const double keep_c = c->tot_count, keep_w = c->tot_weighted;
  unsigned ncut = 0;
  if ((rc = sur_cut(c, level_L, &ncut))) return rc;
  o->n_pairs = ncut;
  o->fallback_exact = 0.0;
  if (ncut == 0) return TRILENS_OK;
  if (o->label) {
    double total = 0.0;
    if ((rc = sur_labels(c, level_L, TL_C * ((double)step * c->p.dt_fs), ncut, &total))) return rc;
  } else if ((rc = sur_ids(c, level_L))) {
    return rc;
  }
  uint8_t *flag = nullptr;
  if (want_net) {
    CK(dalloc(&flag, ncut));
    CK(tl::mlp_pack(s->prm, s->work, c->stream));
    CK(tl::mlp_forward(s->prm, s->norm, s->work, s->feat, ncut, s->out, c->n_sm,
                       c->p.spin_limit, c->stream));
    CK(cudaMemsetAsync(s->fb_count, 0, sizeof(unsigned), c->stream));
    CK(tl::launch_estimate(s->out, s->st, (float)s->st_calib, s->cut, s->cut_count, s->cut_cap,
                           tau, s->pred, s->fb, s->fb_count, s->cut_cap, 4 * c->n_sm, c->stream,
                           flag));
    unsigned nfb = 0;
    CK(cudaMemcpyAsync(&nfb, s->fb_count, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (nfb > 0) {
      int retries = 0;
      rc = run_exact(c, TL_C * ((double)step * c->p.dt_fs), s->fb, nfb, &retries);
      if (rc) {
        cudaFree(flag);
        return rc;
      }
      o->fallback_exact = c->ctr_host->weighted;
    }
  }
  CK(cudaStreamSynchronize(c->stream));
  const int64_t m = std::min<int64_t>(o->cap, ncut);
  int err = 0;
  if (m > 0) {
    std::vector<uint4> cut((size_t)m);
    err |= cudaMemcpy(cut.data(), s->cut, sizeof(uint4) * m, cudaMemcpyDeviceToHost);
    if (o->cloud)
      for (int64_t p = 0; p < m; ++p) {
        o->cloud[2 * p] = cut[p].z;
        o->cloud[2 * p + 1] = cut[p].w;
      }
    if (o->feat) err |= cudaMemcpy(o->feat, s->feat, sizeof(float) * 24 * m, cudaMemcpyDeviceToHost);
    if (o->st) err |= cudaMemcpy(o->st, s->st, sizeof(float) * m, cudaMemcpyDeviceToHost);
    if (o->label) err |= cudaMemcpy(o->label, s->label, sizeof(double) * m, cudaMemcpyDeviceToHost);
    if (o->pred) err |= cudaMemcpy(o->pred, s->pred, sizeof(double) * m, cudaMemcpyDeviceToHost);
    if (o->fallback) err |= cudaMemcpy(o->fallback, flag, m, cudaMemcpyDeviceToHost);
    if (o->net) err |= cudaMemcpy(o->net, s->out, sizeof(float) * 2 * m, cudaMemcpyDeviceToHost);
  }
  cudaFree(flag);
  uint32_t *cof[2] = {o->cloud_of_a, o->cloud_of_b};
  for (int k = 0; k < 2 && !err; ++k) {
    const int64_t n = c->beam[k].n;
    if (!cof[k] || n <= 0) continue;
    std::vector<uint32_t> cut_of((size_t)n), inv((size_t)n);
    err |= cudaMemcpy(cut_of.data(), s->cut_of[k], sizeof(uint32_t) * n, cudaMemcpyDeviceToHost);
    err |= cudaMemcpy(inv.data(), s->inv[k], sizeof(uint32_t) * n, cudaMemcpyDeviceToHost);
    for (int64_t i = 0; i < n && !err; ++i) cof[k][i] = cut_of[inv[i]];
  }
  c->tot_count = keep_c;
  c->tot_weighted = keep_w;
  return err ? fail(c, TRILENS_ERR_CUDA, "copying the cut pairs failed") : TRILENS_OK;
}

int trilens_surrogate_info(trilens_ctx *c, double out[6]) {
  if (!c || !out || !c->sur) return TRILENS_ERR_INVALID;
  out[0] = (double)c->sur->tn;
  out[1] = c->sur->last_loss;
  out[2] = c->sur->calib;
  out[3] = c->sur->st_only_calib;
  out[4] = (double)c->sur->level;
  out[5] = c->sur->tot;
  return TRILENS_OK;
}

int trilens_surrogate_dataset(trilens_ctx *c, float *x, double *label, float *st, int64_t cap,
                              int64_t *n) {
  if (!c || !n || cap < 0) return TRILENS_ERR_INVALID;
  *n = c->sur ? c->sur->tn : 0;
  if (!c->sur) return TRILENS_OK;
  CK(cudaSetDevice(c->device));
  const int64_t m = std::min<int64_t>(cap, c->sur->tn);
  if (m > 0) {
    if (x) CK(cudaMemcpy(x, c->sur->tx, sizeof(float) * 24 * m, cudaMemcpyDeviceToHost));
    if (label) CK(cudaMemcpy(label, c->sur->tlab, sizeof(double) * m, cudaMemcpyDeviceToHost));
    if (st) CK(cudaMemcpy(st, c->sur->tst, sizeof(float) * m, cudaMemcpyDeviceToHost));
  }
  return TRILENS_OK;
}

int trilens_surrogate_add_samples(trilens_ctx *c, const float *x, const double *label,
                                  const float *st, int64_t n, int32_t level_L) {
  if (!c || n < 0 || (n > 0 && (!x || !label || !st)) || level_L < 1 || level_L > 63)
    return TRILENS_ERR_INVALID;
  if (c->n_inst > 1) return fail(c, TRILENS_ERR_INVALID, "surrogate on a batch context");
  CK(cudaSetDevice(c->device));
  int rc = ensure_state(c);
  if (rc) return rc;
  SurrogateState *s = c->sur;
  if (s->level >= 0 && s->level != level_L && s->tn > 0)
    return fail(c, TRILENS_ERR_INVALID, "samples of another level are collected");
  s->level = level_L;
  for (int64_t r0 = 0; r0 < n; r0 += s->cut_cap) {
    const unsigned m = (unsigned)std::min<int64_t>(s->cut_cap, n - r0);
    CK(cudaMemcpy(s->feat, x + 24 * r0, sizeof(float) * 24 * m, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(s->st, st + r0, sizeof(float) * m, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(s->label, label + r0, sizeof(double) * m, cudaMemcpyHostToDevice));
    if ((rc = append_samples(c, m))) return rc;
  }
  CK(cudaStreamSynchronize(c->stream));
  return TRILENS_OK;
}

int surrogate_total(trilens_ctx *c, int level, double *out) {
  if (!c->sur || !c->sur->trained || c->sur->level != level)
    return fail(c, TRILENS_ERR_INVALID, "no surrogate model for level %d", level);
  *out = c->sur->tot;
  return TRILENS_OK;
}

// model file: magic, level, calibrations, then norm (48 FP32) and parameters
int trilens_surrogate_save(trilens_ctx *c, const char *path) {
  if (!c || !path || !c->sur || !c->sur->trained) return TRILENS_ERR_INVALID;
  CK(cudaSetDevice(c->device));
  SurrogateState *s = c->sur;
  std::vector<float> p(TRILENS_MLP_PARAMS), nrm(48);
  CK(cudaMemcpy(p.data(), s->prm, sizeof(float) * p.size(), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(nrm.data(), s->norm, sizeof(float) * 48, cudaMemcpyDeviceToHost));
  FILE *f = fopen(path, "wb");
  if (!f) return fail(c, TRILENS_ERR_INVALID, "cannot write %s", path);
  const char magic[8] = {'T', 'R', 'L', 'S', 'U', 'R', '0', '3'};
  const int32_t hdr[2] = {s->level, TRILENS_MLP_PARAMS};
  const double cal[3] = {s->calib, s->st_calib, s->st_only_calib};
  bool ok = fwrite(magic, 1, 8, f) == 8 && fwrite(hdr, sizeof(int32_t), 2, f) == 2 &&
            fwrite(cal, sizeof(double), 3, f) == 3 &&
            fwrite(s->cal_tau, sizeof(double), kTauBins, f) == (size_t)kTauBins &&
            fwrite(nrm.data(), sizeof(float), 48, f) == 48 &&
            fwrite(p.data(), sizeof(float), p.size(), f) == p.size();
  fclose(f);
  return ok ? TRILENS_OK : fail(c, TRILENS_ERR_INVALID, "short write to %s", path);
}

int trilens_surrogate_load(trilens_ctx *c, const char *path) {
  if (!c || !path) return TRILENS_ERR_INVALID;
  if (c->n_inst > 1) return fail(c, TRILENS_ERR_INVALID, "surrogate on a batch context");
  CK(cudaSetDevice(c->device));
  int rc = ensure_state(c);
  if (rc) return rc;
  SurrogateState *s = c->sur;
  FILE *f = fopen(path, "rb");
  if (!f) return fail(c, TRILENS_ERR_INVALID, "cannot read %s", path);
  char magic[8];
  int32_t hdr[2];
  double cal[3];
  std::vector<float> p(TRILENS_MLP_PARAMS), nrm(48);
  double tab[kTauBins];
  bool ok = fread(magic, 1, 8, f) == 8 &&
            (memcmp(magic, "TRLSUR03", 8) == 0 || memcmp(magic, "TRLSUR02", 8) == 0) &&
            fread(hdr, sizeof(int32_t), 2, f) == 2 && hdr[1] == TRILENS_MLP_PARAMS &&
            fread(cal, sizeof(double), 3, f) == 3;
  const bool has_tab = ok && magic[7] == '3';
  if (has_tab) ok = fread(tab, sizeof(double), kTauBins, f) == (size_t)kTauBins;
  ok = ok && fread(nrm.data(), sizeof(float), 48, f) == 48 &&
       fread(p.data(), sizeof(float), p.size(), f) == p.size();
  fclose(f);
  if (!ok) return fail(c, TRILENS_ERR_INVALID, "%s is not a surrogate model file", path);
  CK(cudaMemcpy(s->prm, p.data(), sizeof(float) * p.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(s->norm, nrm.data(), sizeof(float) * 48, cudaMemcpyHostToDevice));
  s->level = hdr[0];
  s->calib = cal[0];
  s->st_calib = cal[1];
  s->st_only_calib = cal[2];
  for (int g = 0; g < kTauBins; ++g) s->cal_tau[g] = has_tab ? tab[g] : cal[0];
  s->trained = true;
  return TRILENS_OK;
}

}  // extern "C"
