// tl_api.cu -- host runtime behind the C ABI declared in include/trilens.h:
// context and workspace, per-step build and collide sequencing on the
// caller's stream, device status checks and buffer regrowth.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "tl_ctx.h"
#include "trilens_debug.h"

namespace tl {
cudaError_t launch_step_init(TLCounters *ctr, uint2 *F0, uint32_t sa, uint32_t sb, int nonempty,
                             const unsigned *build_status, const unsigned *run_status,
                             cudaStream_t s);
cudaError_t launch_expand(const TravArgs &a, uint2 *F0, uint2 *F1, unsigned cap, unsigned target,
                          int max_levels, cudaStream_t s);
cudaError_t launch_seed_cut(const TravArgs &a, const uint32_t *cutA, const unsigned *cntA,
                            uint32_t capA, const uint32_t *cutB, const unsigned *cntB,
                            uint32_t capB, uint2 *F0, unsigned cap, int blocks, cudaStream_t s);
cudaError_t traverse_config(int fp64, int warps, int depth, int *blocks_per_sm);
cudaError_t launch_widen(const TravArgs &a, uint2 *F0, uint2 *F1, unsigned cap, unsigned target,
                         int levels, int blocks, cudaStream_t s);
cudaError_t launch_narrow(const TravArgs &a, int blocks, cudaStream_t s);
cudaError_t launch_traverse(const TravArgs &a, const uint2 *F0, const uint2 *F1, const uint2 *list,
                            unsigned long long list_n, int from_frontier, int budget, int blocks,
                            int warps, cudaStream_t s, int part, int nparts);
cudaError_t launch_part_init(TLCounters *ctr, cudaStream_t s);
cudaError_t launch_band(const TravArgs &a, int blocks, cudaStream_t s);
cudaError_t launch_yield(const TravArgs &a, void *partials, int blocks, cudaStream_t s);
size_t partial_bytes();
cudaError_t launch_seed_instances(TLCounters *ctr, uint2 *F0, const uint32_t *rootA,
                                  const uint32_t *rootB, int n_inst, cudaStream_t s);
cudaError_t launch_yield_inst(const TravArgs &a, const uint32_t *inst_of_a, double *yields,
                              int blocks, cudaStream_t s);
cudaError_t launch_pair_products(const TLBeam &a, const TLBeam &b, const uint32_t *hits,
                                 int64_t n_hits, unsigned long long seed, double *out, int n_sm,
                                 cudaStream_t s);
cudaError_t launch_step_finish(const TLCounters *ctr, unsigned *run_status, TLRunAcc *acc,
                               cudaStream_t s);
}  // namespace tl

enum {
  PH_PROP = 0, PH_SORT, PH_GATHER, PH_EMIT, PH_REFIT, PH_EXPAND, PH_TRAV, PH_BAND, PH_YIELD,
  PH_NARROW, PH_COUNT
};

// breadth-first levels that may widen the seed frontier of a large problem
// (each a launch that does nothing once the frontier holds widen_target pairs)
constexpr int kWidenLevels = 5;
// node pairs per traversal queue chunk and frontier item (tl_traverse.cu)
constexpr unsigned long long kQueueChunk = 32;
// the leaf-pair list never grows past 2^30 pairs (8 GiB): a step that lists
// more is done in parts, slices of its frontier, each listing at most that
constexpr unsigned long long kLeafListMax = 1ull << 30;

// after a step overflowed the leaf-pair list (the largest part listed need
// pairs): a larger list, or more parts
static int leaves_for(trilens_ctx *c, unsigned long long need) {
  if (need + need / 4 + 1024 <= kLeafListMax) return grow(c, &c->leaves, &c->leaf_cap, need);
  if (c->leaf_cap < kLeafListMax) {
    cudaFree(c->leaves);
    c->leaves = nullptr;
    c->leaf_cap = 0;
    CK(dalloc(&c->leaves, (size_t)kLeafListMax));
    c->leaf_cap = kLeafListMax;
  }
  const unsigned long long per = kLeafListMax / 2;  // room for uneven parts
  const unsigned long long more = (need + per - 1) / per;
  if ((unsigned long long)c->parts * more > 4096)
    return fail(c, TRILENS_ERR_STACK, "a step would need more than 4096 parts");
  c->parts = (int)(c->parts * more);
  return TRILENS_OK;
}

// the traversal and the narrow phase of a step, part by part
static int traverse_parts(trilens_ctx *c, const tl::TravArgs &a, const uint2 *seeds,
                          unsigned n_seeds) {
  for (int p = 0; p < c->parts; ++p) {
    if (p > 0) CK(tl::launch_part_init(c->ctr, c->stream));
    CK(tl::launch_traverse(a, c->front[0], c->front[1], seeds, seeds ? n_seeds : 0, seeds ? 0 : 1,
                           c->budget, c->trav_blocks, c->trav_warps, c->stream, p, c->parts));
    CK(tl::launch_narrow(a, 8 * c->n_sm, c->stream));
  }
  return TRILENS_OK;
}

// the frontier widening target: 64 pairs per resident traversal warp, two
// full items each; and the frontier buffers' capacity for every start
static void frontier_sizes(trilens_ctx *c, unsigned *target, unsigned *cap) {
  const long long warps = (long long)c->trav_blocks * c->trav_warps;
  *target = (unsigned)std::min<long long>(64ll * warps, 1 << 22);
  const unsigned long long need =
      std::max({(unsigned long long)c->n_inst + 4ull * c->front_target + 64,
                (unsigned long long)c->w[0].cut_cap * c->w[1].cut_cap + 64,
                4ull * *target + 64});
  *cap = (unsigned)std::min<unsigned long long>(need, 0xFFFFFFF0ull);
}

static void tmark(trilens_ctx *c, int ph, int k, int end) {
  if (!c->timing) return;
  cudaEventRecord(c->ev[ph][k][end], c->stream);
  if (end) c->ev_pending[ph][k] = true;
}

// add the elapsed time of every recorded phase (the stream is synchronised)
static void tcollect(trilens_ctx *c) {
  for (int ph = 0; ph < PH_COUNT; ++ph)
    for (int k = 0; k < 2; ++k)
      if (c->ev_pending[ph][k]) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->ev[ph][k][0], c->ev[ph][k][1]) == cudaSuccess)
          c->phase_ms[ph] += ms;
        c->ev_pending[ph][k] = false;
      }
}

// ---- host-side constants (plain double; used only for conservative bounds)

static double host_sigma(double s) {
  if (!(s > 1.0)) return 0.0;
  double b = sqrt((s - 1.0) / s);
  double lg = log((1.0 + b) * (1.0 + b) * s);
  return 0.5 * TL_PI * TL_RE * TL_RE / s * ((3.0 - b * b * b * b) * lg - 2.0 * b * (2.0 - b * b));
}

// s where Eq. BWcross peaks (golden-section search; sigma is unimodal)
static double host_sigma_peak_s() {
  double lo = 1.2, hi = 4.0, g = 0.5 * (sqrt(5.0) - 1.0);
  for (int it = 0; it < 200; ++it) {
    double x1 = hi - g * (hi - lo), x2 = lo + g * (hi - lo);
    if (host_sigma(x1) < host_sigma(x2)) lo = x1;
    else hi = x2;
  }
  return 0.5 * (lo + hi);
}

static double host_sigma_max() { return host_sigma(host_sigma_peak_s()); }

// an upper bound of Eq. BWcross over s (for conservative tests elsewhere)
double tl_sigma_max_bound() { return host_sigma_max() * (1.0 + 1e-6); }

static float round_up(double x) {
  float f = (float)x;
  if ((double)f < x) f = nextafterf(f, INFINITY);
  return f;
}
static float round_down(double x) {
  float f = (float)x;
  if ((double)f > x) f = nextafterf(f, -INFINITY);
  return f;
}

// constants of the FP32 narrow phase for a step of dt_fs and amplification kappa
TLNarrowConst tl_narrow_const(double dt_fs, double kappa) {
  const double u = ldexp(1.0, -24);
  const double sigma_max = host_sigma_max() * (1.0 + 1e-6);
  TLNarrowConst nk;
  nk.L = (float)(TL_C * dt_fs);
  nk.L_in = round_down((double)nk.L * (1.0 - 8.0 * u));
  nk.L_out = round_up((double)nk.L * (1.0 + 8.0 * u));
  nk.r2max = round_up(1e12 * kappa * sigma_max * (1.0 + 1e-5) / TL_PI);
  nk.kr = (float)(1e12 * kappa / TL_PI);
  nk.inv2mc4 = (float)(1.0 / (2.0 * TL_MEC2 * TL_MEC2));
  nk.pref = (float)(0.5 * TL_PI * TL_RE * TL_RE);
  // sure-miss radius per bin of s: sigma's largest value over the bin (at the
  // end nearer the peak, or the peak itself), with a relative margin
  const double s_peak = host_sigma_peak_s();
  nk.sbin[0] = 0.0f;
  for (int i = 1; i < TL_SBINS; ++i) {
    const int e = (i - 1) / TL_SBIN_OCT, k = (i - 1) % TL_SBIN_OCT;
    const double a = ldexp(1.0 + (double)k / TL_SBIN_OCT, e);
    const double b = ldexp(1.0 + (double)(k + 1) / TL_SBIN_OCT, e);
    double sig;
    if (i == TL_SBINS - 1) sig = host_sigma(a);  // [a, inf): sigma falls beyond the peak
    else if (b <= s_peak) sig = host_sigma(b);
    else if (a >= s_peak) sig = host_sigma(a);
    else sig = sigma_max;
    nk.sbin[i] = round_up(1e12 * kappa * std::min(sig * (1.0 + 1e-5), sigma_max) / TL_PI);
  }
  return nk;
}

static void free_beam(tl::BuildBufs &w) {
  cudaFree(w.pos_u);
  cudaFree(w.dir_u);
  cudaFree(w.pos);
  cudaFree(w.dir);
  cudaFree(w.key[0]);
  cudaFree(w.key[1]);
  cudaFree(w.val[0]);
  cudaFree(w.val[1]);
  cudaFree(w.nodes);
  cudaFree(w.parent_leaf);
  cudaFree(w.parent_node);
  cudaFree(w.rpre);
  cudaFree(w.rsuf);
  cudaFree(w.rtile);
  cudaFree(w.rsuper);
  cudaFree(w.cut);
  cudaFree(w.cut_n);
  cudaFree(w.nfirst);
  cudaFree(w.nlast);
  cudaFree(w.nlev);
  cudaFree(w.sort_status);
  cudaFree(w.sort_ep);
  cudaFree(w.sort_raw);
  cudaFree(w.sort_hist);
  cudaFree(w.sort_tile);
  memset(&w, 0, sizeof(w));
}

static int alloc_beam(trilens_ctx *c, tl::BuildBufs &w, int64_t n) {
  size_t m = (size_t)std::max<int64_t>(n, 1);
  CK(dalloc(&w.pos_u, m));
  CK(dalloc(&w.dir_u, m));
  CK(dalloc(&w.pos, m));
  CK(dalloc(&w.dir, m));
  CK(dalloc(&w.key[0], m));
  CK(dalloc(&w.key[1], m));
  CK(dalloc(&w.val[0], m));
  CK(dalloc(&w.val[1], m));
  CK(dalloc(&w.nodes, m));
  CK(dalloc(&w.parent_leaf, m));
  CK(dalloc(&w.parent_node, m));
  CK(dalloc(&w.rpre, 6 * m));
  CK(dalloc(&w.rsuf, 6 * m));
  CK(dalloc(&w.rtile, 6 * (size_t)tl::refit_tiles((int64_t)m)));
  CK(dalloc(&w.rsuper, tl::refit_super_floats((int64_t)m)));
  CK(dalloc(&w.nfirst, m));
  CK(dalloc(&w.nlast, m));
  CK(dalloc(&w.nlev, m));
  // traversal seeds for beams of 2^17 photons or more: about 256-512 cut nodes
  // (more where small siblings hang off long chains; past the capacity the
  // traversal starts from the roots)
  w.cut_S = n >= 131072 ? (uint32_t)(n >> 8) : 0u;
  w.cut_cap = w.cut_S ? (uint32_t)(8 * (n / w.cut_S) + 32) : 0u;
  w.cut_alloc = w.cut_cap;
  CK(dalloc(&w.cut, std::max<size_t>(w.cut_cap, 1)));
  CK(dalloc(&w.cut_n, 1));
  w.sort_tiles = (int64_t)((m + TL_SORT_TILE - 1) / TL_SORT_TILE);
  w.sort_epoch = 0;
  CK(dalloc(&w.sort_status, (size_t)w.sort_tiles * 256));
  CK(dalloc(&w.sort_ep, 9));
  CK(dalloc(&w.sort_raw, 8 * 256));
  CK(cudaMemsetAsync(w.sort_raw, 0, sizeof(uint32_t) * 8 * 256, c->stream));
  CK(dalloc(&w.sort_hist, 8 * 256));
  CK(dalloc(&w.sort_tile, 8));
  return TRILENS_OK;
}

// ---- C ABI

extern "C" {

const char *trilens_version(void) { return "trilens-gb300 0.1 (sm_103a)"; }

const char *trilens_status_str(int code) {
  switch (code) {
    case TRILENS_OK: return "ok";
    case TRILENS_ERR_INVALID: return "invalid argument";
    case TRILENS_ERR_CAPACITY: return "hit buffer too small";
    case TRILENS_ERR_CUDA: return "CUDA error";
    case TRILENS_ERR_TIMEOUT: return "device wait reached its spin limit";
    case TRILENS_ERR_STACK: return "traversal overflow after retries";
    case TRILENS_ERR_NOMEM: return "device allocation failed";
    default: return "unknown status";
  }
}

const char *trilens_last_error(trilens_ctx *c) { return c ? c->msg : "no context"; }

static bool beam_ok(const trilens_beam *b) {
  if (!b || b->n < 0 || b->n >= (1ll << 27)) return false;
  if (b->n == 0) return true;
  return b->px && b->py && b->pz && b->dx && b->dy && b->dz && b->E;
}

void trilens_destroy(trilens_ctx *c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  free_beam(c->w[0]);
  free_beam(c->w[1]);
  cudaFree(c->front[0]);
  cudaFree(c->front[1]);
  cudaFree(c->queue);
  cudaFree(c->run_acc);
  cudaFree(c->hits);
  cudaFree(c->band);
  cudaFree(c->leaves);
  cudaFree(c->spill);
  cudaFree(c->ctr);
  cudaFree(c->partials);
  cudaFree(c->build_status);
  surrogate_free(c);
  deplete_free(c);
  cudaFreeHost(c->ctr_host);
  cudaFreeHost(c->build_status_host);
  for (int k = 0; k < 2; ++k) {
    cudaFree(c->inst_of[k]);
    cudaFree(c->inst_root[k]);
    cudaFree(c->inst_bounds[k]);
    cudaFree(c->inst_box[k]);
    for (int a = 0; a < 8; ++a) cudaFree(c->owned[k][a]);
  }
  cudaFree(c->inst_tmp);
  cudaFree(c->run_status);
  cudaFreeHost(c->run_status_host);
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->side_stream) cudaStreamDestroy(c->side_stream);
  if (c->fork_ev) cudaEventDestroy(c->fork_ev);
  if (c->join_ev) cudaEventDestroy(c->join_ev);
  for (int ph = 0; ph < PH_COUNT; ++ph)
    for (int k = 0; k < 2; ++k)
      for (int e = 0; e < 2; ++e)
        if (c->ev[ph][k][e]) cudaEventDestroy(c->ev[ph][k][e]);
  delete c;
}

int trilens_create(trilens_ctx **out, const trilens_beam *a, const trilens_beam *b,
                   const trilens_params *p, trilens_stream_t stream) {
  if (!out) return TRILENS_ERR_INVALID;
  *out = nullptr;
  if (!beam_ok(a) || !beam_ok(b) || !p) return TRILENS_ERR_INVALID;
  if (!(p->dt_fs > 0.0) || !(p->kappa > 0.0) || !isfinite(p->dt_fs) || !isfinite(p->kappa))
    return TRILENS_ERR_INVALID;
  if (p->precision != TRILENS_FP64 && p->precision != TRILENS_FP32_BAND) return TRILENS_ERR_INVALID;
  if (p->leaf_bucket < 0 || p->leaf_bucket > 32) return TRILENS_ERR_INVALID;
  if (p->stack_depth != 0 && (p->stack_depth < 64 || p->stack_depth > 4096))
    return TRILENS_ERR_INVALID;
  if (p->block_shape < 0 || p->block_shape > TL_TRAV_MAX_WARPS) return TRILENS_ERR_INVALID;
  if (p->spin_limit < 0) return TRILENS_ERR_INVALID;

  trilens_ctx *c = new trilens_ctx();
  CK(cudaGetDevice(&c->device));
  c->stream = (cudaStream_t)stream;
  c->p = *p;
  if (c->p.leaf_bucket == 0) c->p.leaf_bucket = 4;
  if (c->p.stack_depth == 0) c->p.stack_depth = 512;
  if (c->p.block_shape == 0) c->p.block_shape = 4;
  if (c->p.spin_limit == 0) c->p.spin_limit = 1ll << 22;
  const trilens_beam *bs[2] = {a, b};
  for (int k = 0; k < 2; ++k) {
    TLBeam &t = c->beam[k];
    t.n = bs[k]->n;
    t.px = bs[k]->px; t.py = bs[k]->py; t.pz = bs[k]->pz;
    t.dx = bs[k]->dx; t.dy = bs[k]->dy; t.dz = bs[k]->dz;
    t.E = bs[k]->E; t.w = bs[k]->w;
  }
  int rc;
  // constants
  c->L64 = TL_C * c->p.dt_fs;
  c->sigma_max = host_sigma_max() * (1.0 + 1e-6);
  c->rmax = sqrt(1e12 * c->p.kappa * c->sigma_max / TL_PI) * (1.0 + 1e-6);
  c->L_lo = round_down(c->L64);
  c->L_hi = round_up(c->L64);
  c->half = round_up(0.5 * c->rmax * (1.0 + 1e-6) + 1e-9);
  c->nk = tl_narrow_const(c->p.dt_fs, c->p.kappa);
  // workspace
  CK(dalloc(&c->build_status, 1));
  CK(cudaMallocHost((void **)&c->build_status_host, sizeof(unsigned)));
  CK(cudaMemsetAsync(c->build_status, 0, sizeof(unsigned), c->stream));
  for (int k = 0; k < 2; ++k) {
    if ((rc = alloc_beam(c, c->w[k], c->beam[k].n))) {
      trilens_destroy(c);
      return rc;
    }
    c->w[k].build_status = c->build_status;
    // the step-invariant FP32 direction, index and energy, once
    CK(tl::launch_static_soa(c->beam[k], c->w[k], c->stream));
    int64_t n = std::max<int64_t>(c->beam[k].n, 2);
    int lg = 0;
    while ((1ll << lg) < n) ++lg;
    // Morton resolution: one bit per axis beyond one cell per photon (at 2 x 1M
    // head-on: 24-bit keys, 3 sort passes; 27 or 30 bits traverse as fast but
    // take 4 passes; 21 bits slow the traversal by a third)
    c->bits[k] = std::min(21, std::max(4, (lg + 2) / 3 + 1));
    c->key_bits[k] = 3 * c->bits[k];
    c->w[k].key_bits = c->key_bits[k];
    // one-time moments of p0 and d for the Morton box of every step
    double *mom = nullptr;
    CK(cudaMalloc((void **)&mom, sizeof(double) * 15 * (1 + 4 * 152)));
    cudaError_t me = tl::launch_beam_moments(c->beam[k], mom, mom + 15, c->stream);
    if (!me)
      me = cudaMemcpyAsync(c->moments[k], mom, sizeof(double) * 15, cudaMemcpyDeviceToHost,
                           c->stream);
    if (!me) me = cudaStreamSynchronize(c->stream);
    cudaFree(mom);
    CK(me);
  }
  CK(tl::sort_prepare());
  CK(tl::refit_prepare());
  int dev_sm = 0;
  CK(cudaDeviceGetAttribute(&dev_sm, cudaDevAttrMultiProcessorCount, c->device));
  c->n_sm = dev_sm;
  c->trav_warps = c->p.block_shape;
  int bps = 0;
  CK(tl::traverse_config(c->p.precision == TRILENS_FP64, c->trav_warps, c->p.stack_depth, &bps));
  if (bps < 1) {
    trilens_destroy(c);
    return TRILENS_ERR_INVALID;
  }
  c->trav_blocks = bps * c->n_sm;
  c->expand_blocks = 2 * c->n_sm;
  c->front_target = (unsigned)std::min<long long>(2ll * c->trav_blocks * c->trav_warps, 1 << 16);
  frontier_sizes(c, &c->widen_target, &c->front_cap);
  CK(dalloc(&c->front[0], c->front_cap));
  CK(dalloc(&c->front[1], c->front_cap));
  {
    const int rcq = alloc_queue(c, std::max<unsigned long long>(
                                       1 << 20, 2ull * c->trav_blocks * c->trav_warps *
                                                    (unsigned long long)c->p.stack_depth));
    if (rcq) {
      trilens_destroy(c);
      return rcq;
    }
  }
  if ((rc = alloc_spill(c, c->spill_per_warp, (unsigned long long)c->trav_blocks * c->trav_warps))) {
    trilens_destroy(c);
    return rc;
  }
  c->hit_cap = std::max<unsigned long long>(1 << 16, 2ull * (c->beam[0].n + c->beam[1].n));
  CK(dalloc(&c->hits, c->hit_cap));
  c->band_cap = std::max<unsigned long long>(1 << 16, (c->beam[0].n + c->beam[1].n) / 4);
  CK(dalloc(&c->band, c->band_cap));
  // the leaf-pair list: 16 per photon to start (a busy step of 2 x 1M
  // head-on lists ~2.6e7 with single-photon buckets), at most 2^29 (4 GiB)
  // before a step asks for more
  c->leaf_cap = std::min<unsigned long long>(
      std::max<unsigned long long>(1 << 20, 16ull * (c->beam[0].n + c->beam[1].n)), 1ull << 29);
  CK(dalloc(&c->leaves, c->leaf_cap));
  CK(dalloc(&c->ctr, 1));
  CK(cudaMallocHost((void **)&c->ctr_host, sizeof(TLCounters)));
  c->yield_blocks = 4 * c->n_sm;
  CK(cudaMalloc(&c->partials, tl::partial_bytes() * c->yield_blocks));
  CK(cudaStreamSynchronize(c->stream));
  *out = c;
  return TRILENS_OK;
}

int trilens_build(trilens_ctx *c, int64_t step) {
  if (!c) return TRILENS_ERR_INVALID;
  if (step < 0) return fail(c, TRILENS_ERR_INVALID, "step < 0");
  CK(cudaSetDevice(c->device));
  const double ct = TL_C * ((double)step * c->p.dt_fs);
  const double T = ct + 0.5 * c->L64;
  // the two beams' builds share nothing but the status word (set with
  // atomic OR): beam B's runs on a side stream, forked from the context's
  // stream and joined back before anything that reads the hierarchies (in a
  // captured run this is a fork and a join in the graph).  Per-phase timing
  // keeps them on one stream, one after the other.
  const bool fork = !c->timing && c->beam[0].n > 0 && c->beam[1].n > 0;
  if (fork) {
    if (!c->side_stream) CK(cudaStreamCreateWithFlags(&c->side_stream, cudaStreamNonBlocking));
    if (!c->fork_ev) CK(cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming));
    if (!c->join_ev) CK(cudaEventCreateWithFlags(&c->join_ev, cudaEventDisableTiming));
    CK(cudaEventRecord(c->fork_ev, c->stream));
    CK(cudaStreamWaitEvent(c->side_stream, c->fork_ev, 0));
  }
  for (int k = 0; k < 2; ++k) {
    const int64_t n = c->beam[k].n;
    if (n <= 0) continue;
    cudaStream_t st = (fork && k == 1) ? c->side_stream : c->stream;
    // Morton box of the step: per axis the mean of the swept boxes' centres
    // c = p0 + T d +- 5 standard deviations, in closed form from the beam's
    // moments (centres outside are clamped to the edge cells).  Unlike the
    // extreme centres, the moments of a large beam barely change from one
    // draw to the next, so neither do the cells a level of the hierarchy
    // stands for.  (Batches use each instance's own box, below.)
    float lo[3], scale[3];
    const double maxq = (double)((1u << c->bits[k]) - 1u);
    for (int a = 0; a < 3; ++a) {
      const double *m = c->moments[k], nn = (double)n;
      const double mean = (m[a] + T * m[3 + a]) / nn;
      const double msq = (m[6 + a] + 2.0 * T * m[9 + a] + T * T * m[12 + a]) / nn;
      const double h = 5.0 * std::sqrt(std::max(msq - mean * mean, 0.0));
      const float l = (float)(mean - h), u = (float)(mean + h);
      lo[a] = l;
      scale[a] = u > l ? (float)(maxq / ((double)u - (double)l)) : 0.0f;
    }
    tl::BuildBufs &w = c->w[k];
    tmark(c, PH_PROP, k, 0);
    if (c->n_inst > 1) {
      CK(tl::launch_inst_box(c->inst_bounds[k], c->n_inst, T, c->bits[k], c->inst_box[k],
                             st));
      CK(cudaMemsetAsync(c->inst_root[k], 0xff, sizeof(uint32_t) * c->n_inst, st));
    }
    CK(tl::launch_propagate(c->beam[k], ct, (float)c->L64, lo, scale, c->bits[k], w,
                            c->n_inst > 1 ? c->inst_box[k] : nullptr,
                            n > 1 ? (c->key_bits[k] + 7) / 8 : 0, st));
    tmark(c, PH_PROP, k, 1);
    tmark(c, PH_SORT, k, 0);
    CK(tl::launch_sort(w, n, c->key_bits[k], c->p.spin_limit, c->debug_stall_sort,
                       c->build_status, &c->sel[k], st));
    tmark(c, PH_SORT, k, 1);
    if (n <= 1) {  // no sort: copy the one photon (a longer beam is gathered by the sort)
      tmark(c, PH_GATHER, k, 0);
      CK(tl::launch_gather(w, n, c->sel[k], st));
      tmark(c, PH_GATHER, k, 1);
      c->phase_launches[PH_GATHER] += 1;
    }
    tmark(c, PH_EMIT, k, 0);
    CK(tl::launch_karras(w, n, c->sel[k], c->p.leaf_bucket, st));
    tmark(c, PH_EMIT, k, 1);
    tmark(c, PH_REFIT, k, 0);
    CK(tl::launch_refit(w, n, c->L_lo, c->L_hi, c->half, c->n_sm, st));
    tmark(c, PH_REFIT, k, 1);
    c->phase_launches[PH_PROP] += 1;
    c->phase_launches[PH_SORT] += n > 1 ? 1 + (c->key_bits[k] + 7) / 8 : 0;
    c->phase_launches[PH_EMIT] += 1;
    c->phase_launches[PH_REFIT] += tl::refit_tiles(n) > 1 ? 3 : 1;
  }
  if (fork) {
    CK(cudaEventRecord(c->join_ev, c->side_stream));
    CK(cudaStreamWaitEvent(c->stream, c->join_ev, 0));
  }
  c->built_step = step;
  return TRILENS_OK;
}

}  // extern "C"

// A step's (or a captured run's) failure from its traversal and build status
// words, or TRILENS_OK.  After a wait that expired or an invalid hierarchy the
// sort's status words are cleared before the next sort, the queue is reset to
// the sentinel (a traversal cut short may leave items in it) and the build
// status is cleared.
static int status_failure(trilens_ctx *c, unsigned trav_st, unsigned build_st) {
  if (!((trav_st | build_st) & (TL_ST_TIMEOUT | TL_ST_BADTREE))) return TRILENS_OK;
  c->w[0].sort_epoch = c->w[1].sort_epoch = 0;
  CK(cudaMemsetAsync(c->queue, 0xff, sizeof(uint2) * (size_t)c->queue_cap, c->stream));
  CK(cudaMemsetAsync(c->build_status, 0, sizeof(unsigned), c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (build_st & TL_ST_TIMEOUT)
    return fail(c, TRILENS_ERR_TIMEOUT,
                "a device wait reached spin_limit=%lld (the radix sort's look-back)",
                (long long)c->p.spin_limit);
  if (trav_st & TL_ST_TIMEOUT)
    return fail(c, TRILENS_ERR_TIMEOUT,
                "a device wait reached spin_limit=%lld (a traversal warp waiting for work)",
                (long long)c->p.spin_limit);
  return fail(c, TRILENS_ERR_CUDA,
              "the refit met a node reference out of range: the step's hierarchy is invalid "
              "(internal error)");
}

tl::TravArgs trav_args(trilens_ctx *c, double ct) {
  tl::TravArgs a;
  memset(&a, 0, sizeof(a));
  for (int k = 0; k < 2; ++k) {
    TLTree &t = k ? a.B : a.A;
    t.pos = c->w[k].pos;
    t.dir = c->w[k].dir;
    t.nodes = c->w[k].nodes;
    t.n = c->beam[k].n;
    t.super = (uint32_t)(t.n > 1 ? t.n - 1 : 0);
  }
  a.mA = c->beam[0];
  a.mB = c->beam[1];
  a.ct = ct;
  a.dt = c->p.dt_fs;
  a.kappa = c->p.kappa;
  a.nk = c->nk;
  a.fp64 = c->p.precision == TRILENS_FP64;
  a.ctr = c->ctr;
  a.hits = c->hits;
  a.hit_cap = c->hit_cap;
  a.band = c->band;
  a.band_cap = c->band_cap;
  a.leaves = c->leaves;
  a.leaf_cap = c->leaf_cap;
  a.queue = reinterpret_cast<unsigned long long *>(c->queue);
  a.queue_cap = c->queue_cap;
  a.spill = c->spill;
  a.spill_per_warp = c->spill_per_warp;
  a.spin_limit = c->p.spin_limit;
  a.stack_depth = c->p.stack_depth;
  a.leaf_bucket = c->p.leaf_bucket;
  a.build_status = c->build_status;
  return a;
}

int run_exact(trilens_ctx *c, double ct, const uint2 *seeds, unsigned n_seeds, int *retries_out) {
  const int nonempty = c->beam[0].n > 0 && c->beam[1].n > 0;
  int retries = 0;
  TLCounters &h = *c->ctr_host;
  while (true) {
    tl::TravArgs a = trav_args(c, ct);
    // large single problems start from the refit's cut lists; small ones and
    // batches expand their root pairs breadth first
    const bool use_cut = !seeds && c->n_inst <= 1 && c->w[0].cut_S && c->w[1].cut_S;
    tmark(c, PH_EXPAND, 0, 0);
    CK(tl::launch_step_init(c->ctr, c->front[0], a.A.super, a.B.super,
                            (c->n_inst > 1 || seeds || use_cut) ? 0 : nonempty, c->build_status,
                            nullptr, c->stream));
    if (use_cut) {
      CK(tl::launch_seed_cut(a, c->w[0].cut, c->w[0].cut_n, c->w[0].cut_cap, c->w[1].cut,
                             c->w[1].cut_n, c->w[1].cut_cap, c->front[0], c->front_cap,
                             2 * c->n_sm, c->stream));
      CK(tl::launch_widen(a, c->front[0], c->front[1], c->front_cap, c->widen_target,
                          kWidenLevels, 4 * c->n_sm, c->stream));
      c->phase_launches[PH_EXPAND] += kWidenLevels;
    } else if (!seeds) {
      if (c->n_inst > 1)
        CK(tl::launch_seed_instances(c->ctr, c->front[0], c->inst_root[0], c->inst_root[1],
                                     c->n_inst, c->stream));
      CK(tl::launch_expand(a, c->front[0], c->front[1], c->front_cap, c->front_target, kMaxLevels,
                           c->stream));
    }
    tmark(c, PH_EXPAND, 0, 1);
    c->phase_launches[PH_EXPAND] += seeds ? 1 : 2;
    if (c->parts == 1) {
      tmark(c, PH_TRAV, 0, 0);
      CK(tl::launch_traverse(a, c->front[0], c->front[1], seeds, seeds ? n_seeds : 0,
                             seeds ? 0 : 1, c->budget, c->trav_blocks, c->trav_warps, c->stream,
                             0, 1));
      tmark(c, PH_TRAV, 0, 1);
      tmark(c, PH_NARROW, 0, 0);
      CK(tl::launch_narrow(a, 8 * c->n_sm, c->stream));
      tmark(c, PH_NARROW, 0, 1);
    } else {  // parts: traversal and narrow phase timed together
      tmark(c, PH_TRAV, 0, 0);
      int rcp = traverse_parts(c, a, seeds, n_seeds);
      if (rcp) return rcp;
      tmark(c, PH_TRAV, 0, 1);
      c->phase_launches[PH_TRAV] += 2 * (c->parts - 1);
    }
    c->phase_launches[PH_TRAV] += 1;
    c->phase_launches[PH_NARROW] += 1;
    if (!a.fp64) {
      tmark(c, PH_BAND, 0, 0);
      CK(tl::launch_band(a, c->n_sm * 4, c->stream));
      tmark(c, PH_BAND, 0, 1);
      c->phase_launches[PH_BAND] += 1;
    }
    tmark(c, PH_YIELD, 0, 0);
    CK(tl::launch_yield(a, c->partials, c->yield_blocks, c->stream));
    tmark(c, PH_YIELD, 0, 1);
    c->phase_launches[PH_YIELD] += 1;
    CK(cudaMemcpyAsync(&h, c->ctr, sizeof(TLCounters), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(c->build_status_host, c->build_status, sizeof(unsigned),
                       cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    tcollect(c);
    const unsigned st = h.status | *c->build_status_host;
    if (int rf = status_failure(c, h.status, *c->build_status_host)) return rf;
    bool again = false;
    int rc;
    if (st & TL_ST_BAND_OVF) {
      if ((rc = grow(c, &c->band, &c->band_cap, h.band))) return rc;
      again = true;
    }
    if (st & TL_ST_HIT_OVF) {
      if ((rc = grow(c, &c->hits, &c->hit_cap, h.hits + (again ? h.band : 0)))) return rc;
      again = true;
    }
    if (st & TL_ST_SPILL_OVF) {  // the queue: larger, and every slot the sentinel again
      const unsigned long long need = kQueueChunk * (h.q_tail + h.q_tail / 4 + 1024);
      if ((rc = alloc_queue(c, std::max(need, 2 * c->queue_cap)))) return rc;
      again = true;
    }
    if (st & TL_ST_PRIV_OVF) {  // a warp's spill area: twice as large
      if ((rc = alloc_spill(c, 2 * c->spill_per_warp, c->spill_warps))) return rc;
      again = true;
    }
    if (st & TL_ST_LEAFQ) {  // the leaf-pair list: larger, or the step in more parts
      if ((rc = leaves_for(c, h.max_part_leaves))) return rc;
      again = true;
    }
    if (st & TL_ST_FRONT_OVF) return fail(c, TRILENS_ERR_STACK, "frontier overflow");
    if (!again) break;
    if (++retries > 8) return fail(c, TRILENS_ERR_STACK, "buffers kept overflowing");
  }
  if (retries_out) *retries_out = retries;
  return TRILENS_OK;
}

extern "C" {

int trilens_collide_step(trilens_ctx *c, int64_t step, uint32_t *hits, int64_t cap,
                         int64_t *n_hits) {
  if (!c) return TRILENS_ERR_INVALID;
  if (step != c->built_step) return fail(c, TRILENS_ERR_INVALID, "step %lld not built", (long long)step);
  if (cap < 0 || (hits == nullptr && cap > 0)) return fail(c, TRILENS_ERR_INVALID, "bad hit buffer");
  CK(cudaSetDevice(c->device));
  const double ct = TL_C * ((double)step * c->p.dt_fs);
  int retries = 0;
  const int rc = run_exact(c, ct, nullptr, 0, &retries);
  if (rc) return rc;
  TLCounters &h = *c->ctr_host;
  if (hits && (int64_t)h.count > cap) {
    // the step is not added to the cumulative yield: the caller repeats it
    // with a larger buffer (the hierarchies stay built)
    if (n_hits) *n_hits = (int64_t)h.count;
    return fail(c, TRILENS_ERR_CAPACITY, "need %llu hit slots", (unsigned long long)h.count);
  }
  trilens_step_stats &s = c->last;
  s.step = step;
  s.count = (int64_t)h.count;
  s.weighted = h.weighted;
  s.hsum = h.hsum;
  s.hxor = h.hxor;
  s.narrow_tests = (int64_t)h.narrow_tests;
  s.node_tests = (int64_t)h.node_tests;
  s.leaf_pairs = (int64_t)h.leaf_pairs;
  s.band = (int64_t)h.band;
  s.retries = retries;
  c->tot_count += (double)h.count;
  c->tot_weighted += h.weighted;
  if (n_hits) *n_hits = (int64_t)h.count;
  if (hits && cap > 0) {
    const unsigned long long ncopy = std::min<unsigned long long>(h.count, (unsigned long long)cap);
    if (ncopy)
      CK(cudaMemcpyAsync(hits, c->hits, sizeof(uint2) * ncopy, cudaMemcpyDeviceToDevice, c->stream));
  }
  return TRILENS_OK;
}

// ---- batches of independent instances ------------------------------------

static int ensure_graph(trilens_ctx *c);

static int batch_prepare(trilens_ctx *c, const trilens_beam *const src[2], int32_t n_inst) {
  // concatenate each side's instances into library-owned arrays
  std::vector<tl::InstSrc> tab(n_inst);
  int64_t tot[2] = {0, 0};
  for (int k = 0; k < 2; ++k)
    for (int q = 0; q < n_inst; ++q) tot[k] += src[k][q].n;
  for (int k = 0; k < 2; ++k) {
    int64_t off = 0;
    for (int q = 0; q < n_inst; ++q) {
      const trilens_beam &bq = src[k][q];
      const double *ps[8] = {bq.px, bq.py, bq.pz, bq.dx, bq.dy, bq.dz, bq.E, bq.w};
      for (int a = 0; a < 8; ++a) tab[q].p[a] = ps[a];
      tab[q].n = bq.n;
      tab[q].off = off;
      off += bq.n;
    }
    for (int a = 0; a < 8; ++a) CK(dalloc(&c->owned[k][a], (size_t)std::max<int64_t>(tot[k], 1)));
    CK(dalloc(&c->inst_of[k], (size_t)std::max<int64_t>(tot[k], 1)));
    tl::InstSrc *dtab = nullptr;
    double **dptr = nullptr;
    CK(cudaMalloc((void **)&dtab, sizeof(tl::InstSrc) * n_inst));
    CK(cudaMalloc((void **)&dptr, sizeof(double *) * 8));
    CK(cudaMemcpyAsync(dtab, tab.data(), sizeof(tl::InstSrc) * n_inst, cudaMemcpyHostToDevice,
                       c->stream));
    CK(cudaMemcpyAsync(dptr, c->owned[k], sizeof(double *) * 8, cudaMemcpyHostToDevice, c->stream));
    CK(tl::launch_gather_instances(dtab, n_inst, tot[k], dptr, c->inst_of[k], c->stream));
    CK(cudaStreamSynchronize(c->stream));
    cudaFree(dtab);
    cudaFree(dptr);
  }
  return TRILENS_OK;
}

int trilens_batch_create(trilens_ctx **out, const trilens_beam *a, const trilens_beam *b,
                         int32_t n_inst, const trilens_params *p, trilens_stream_t stream) {
  if (!out) return TRILENS_ERR_INVALID;
  *out = nullptr;
  if (!a || !b || !p || n_inst < 1 || n_inst > 65536) return TRILENS_ERR_INVALID;
  int64_t tot[2] = {0, 0}, nmax = 1;
  for (int q = 0; q < n_inst; ++q) {
    if (!beam_ok(&a[q]) || !beam_ok(&b[q])) return TRILENS_ERR_INVALID;
    tot[0] += a[q].n;
    tot[1] += b[q].n;
    nmax = std::max<int64_t>(nmax, std::max(a[q].n, b[q].n));
  }
  if (tot[0] >= (1ll << 27) || tot[1] >= (1ll << 27)) return TRILENS_ERR_INVALID;
  // a throwaway context holds the owned inputs while they are gathered
  trilens_ctx tmp;
  tmp.stream = (cudaStream_t)stream;
  trilens_ctx *c = &tmp;
  const trilens_beam *src[2] = {a, b};
  int rc = batch_prepare(c, src, n_inst);
  if (rc) return rc;
  trilens_beam cat[2];
  for (int k = 0; k < 2; ++k) {
    cat[k].n = tot[k];
    cat[k].px = tmp.owned[k][0]; cat[k].py = tmp.owned[k][1]; cat[k].pz = tmp.owned[k][2];
    cat[k].dx = tmp.owned[k][3]; cat[k].dy = tmp.owned[k][4]; cat[k].dz = tmp.owned[k][5];
    cat[k].E = tmp.owned[k][6]; cat[k].w = tmp.owned[k][7];
  }
  trilens_ctx *ctx = nullptr;
  rc = trilens_create(&ctx, &cat[0], &cat[1], p, stream);
  if (rc) {
    for (int k = 0; k < 2; ++k) {
      for (int q = 0; q < 8; ++q) cudaFree(tmp.owned[k][q]);
      cudaFree(tmp.inst_of[k]);
    }
    return rc;
  }
  c = ctx;
  for (int k = 0; k < 2; ++k) {
    for (int q = 0; q < 8; ++q) {
      c->owned[k][q] = tmp.owned[k][q];
      tmp.owned[k][q] = nullptr;
    }
    c->inst_of[k] = tmp.inst_of[k];
    tmp.inst_of[k] = nullptr;
    c->w[k].inst_of = c->inst_of[k];
  }
  c->n_inst = n_inst;
  for (int k = 0; k < 2; ++k) c->w[k].cut_S = 0;  // batches seed from instance roots
  int ib = 0;
  while ((1 << ib) < n_inst) ++ib;
  int lg = 0;
  while ((1ll << lg) < nmax) ++lg;
  const int bits = std::min((63 - ib) / 3, std::max(4, (lg + 2) / 3 + 3));
  CK(cudaMalloc((void **)&c->inst_tmp, sizeof(long long) * 12 * n_inst));
  for (int k = 0; k < 2; ++k) {
    c->bits[k] = bits;
    c->key_bits[k] = 3 * bits + ib;
    c->w[k].key_bits = c->key_bits[k];
    c->w[k].inst_shift = 3 * bits;
    CK(dalloc(&c->inst_root[k], (size_t)n_inst));
    c->w[k].inst_root = c->inst_root[k];
    CK(dalloc(&c->inst_bounds[k], (size_t)12 * n_inst));
    CK(dalloc(&c->inst_box[k], (size_t)2 * n_inst));
    CK(tl::launch_inst_bounds(c->beam[k], c->inst_of[k], n_inst, c->inst_tmp, c->inst_bounds[k],
                              c->stream));
  }
  if (c->front_cap < (unsigned)n_inst + 4 * c->front_target + 64) {
    c->front_cap = (unsigned)n_inst + 4 * c->front_target + 64;
    for (int k = 0; k < 2; ++k) {
      cudaFree(c->front[k]);
      CK(dalloc(&c->front[k], c->front_cap));
    }
  }
  if ((rc = ensure_graph(c))) return rc;
  CK(cudaStreamSynchronize(c->stream));
  *out = c;
  return TRILENS_OK;
}

// One step of a captured run: the collide sequence without host checks (the
// traversal needs none: its warps share a device work queue); every overflow
// is flagged in run_status, and the step's totals are added on the device.
static int graph_collide(trilens_ctx *c, int64_t step, double *yields) {
  const double ct = TL_C * ((double)step * c->p.dt_fs);
  const int nonempty = c->beam[0].n > 0 && c->beam[1].n > 0;
  tl::TravArgs a = trav_args(c, ct);
  const bool use_cut = c->n_inst <= 1 && c->w[0].cut_S && c->w[1].cut_S;
  CK(tl::launch_step_init(c->ctr, c->front[0], a.A.super, a.B.super,
                          (c->n_inst > 1 || use_cut) ? 0 : nonempty, c->build_status,
                          c->run_status, c->stream));
  if (use_cut) {
    CK(tl::launch_seed_cut(a, c->w[0].cut, c->w[0].cut_n, c->w[0].cut_cap, c->w[1].cut,
                           c->w[1].cut_n, c->w[1].cut_cap, c->front[0], c->front_cap,
                           2 * c->n_sm, c->stream));
    CK(tl::launch_widen(a, c->front[0], c->front[1], c->front_cap, c->widen_target, kWidenLevels,
                        4 * c->n_sm, c->stream));
  } else {
    if (c->n_inst > 1)
      CK(tl::launch_seed_instances(c->ctr, c->front[0], c->inst_root[0], c->inst_root[1],
                                   c->n_inst, c->stream));
    CK(tl::launch_expand(a, c->front[0], c->front[1], c->front_cap, c->front_target, kMaxLevels,
                         c->stream));
  }
  {
    const int rcp = traverse_parts(c, a, nullptr, 0);
    if (rcp) return rcp;
  }
  if (!a.fp64) CK(tl::launch_band(a, c->n_sm * 4, c->stream));
  CK(tl::launch_yield(a, c->partials, c->yield_blocks, c->stream));
  if (yields && c->n_inst > 1)
    CK(tl::launch_yield_inst(a, c->inst_of[0], yields, c->yield_blocks, c->stream));
  CK(tl::launch_step_finish(c->ctr, c->run_status, c->run_acc, c->stream));
  return TRILENS_OK;
}

static int capture_run(trilens_ctx *c, int64_t first, int64_t steps, double *yields) {
  if (c->gexec) {
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
  }
  const int timing = c->timing;
  c->timing = 0;
  cudaStream_t saved = c->stream;
  c->stream = c->cap_stream;
  CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
  int rc = TRILENS_OK;
  cudaError_t e = cudaMemsetAsync(c->run_status, 0, sizeof(unsigned), c->stream);
  if (e == cudaSuccess && c->run_acc)
    e = cudaMemsetAsync(c->run_acc, 0, sizeof(TLRunAcc), c->stream);
  if (e == cudaSuccess && yields && c->n_inst > 1)
    e = cudaMemsetAsync(yields, 0, sizeof(double) * 2 * c->n_inst, c->stream);
  if (e != cudaSuccess) rc = fail(c, TRILENS_ERR_CUDA, "capture: %s", cudaGetErrorString(e));
  for (int64_t k = first; rc == TRILENS_OK && k < first + steps; ++k) {
    rc = trilens_build(c, k);
    if (rc == TRILENS_OK) rc = graph_collide(c, k, yields);
  }
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(c->cap_stream, &g);
  c->stream = saved;
  c->timing = timing;
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return fail(c, TRILENS_ERR_CUDA, "end capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&c->gexec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(c, TRILENS_ERR_CUDA, "instantiate: %s", cudaGetErrorString(e));
  c->g_first = first;
  c->g_steps = steps;
  c->g_yields = yields;
  return TRILENS_OK;
}

// Capture (if needed) and replay a multi-step run; on an overflow grow the
// buffer and run again.
static int replay_run(trilens_ctx *c, int64_t first_step, int64_t steps, double *yields) {
  for (int attempt = 0; attempt < 8; ++attempt) {
    if (!c->gexec || c->g_first != first_step || c->g_steps != steps || c->g_yields != yields) {
      int rc = capture_run(c, first_step, steps, yields);
      if (rc) return rc;
    }
    CK(cudaGraphLaunch(c->gexec, c->stream));
    CK(cudaMemcpyAsync(c->run_status_host, c->run_status, sizeof(unsigned), cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaMemcpyAsync(c->build_status_host, c->build_status, sizeof(unsigned),
                       cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    const unsigned st = *c->run_status_host | *c->build_status_host;
    if (int rf = status_failure(c, *c->run_status_host, *c->build_status_host)) return rf;
    if (!(st & (TL_ST_HIT_OVF | TL_ST_BAND_OVF | TL_ST_SPILL_OVF | TL_ST_FRONT_OVF |
                TL_ST_PRIV_OVF | TL_ST_LEAFQ)))
      return TRILENS_OK;
    // grow what overflowed (to the largest size a step asked for) and capture again
    TLRunAcc m;
    CK(cudaMemcpyAsync(&m, c->run_acc, sizeof(TLRunAcc), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    int rc;
    if (st & TL_ST_HIT_OVF && (rc = grow(c, &c->hits, &c->hit_cap, m.max_hits + m.max_band)))
      return rc;
    if (st & TL_ST_BAND_OVF && (rc = grow(c, &c->band, &c->band_cap, m.max_band))) return rc;
    if (st & TL_ST_PRIV_OVF && (rc = alloc_spill(c, 2 * c->spill_per_warp, c->spill_warps)))
      return rc;
    if (st & TL_ST_LEAFQ && (rc = leaves_for(c, m.max_leaves))) return rc;
    if (st & TL_ST_SPILL_OVF) {  // the queue: larger, and every slot the sentinel again
      const unsigned long long need = kQueueChunk * (m.max_handed + m.max_handed / 4 + 1024);
      if ((rc = alloc_queue(c, std::max(need, 2 * c->queue_cap)))) return rc;
    }
    if (st & TL_ST_FRONT_OVF) return fail(c, TRILENS_ERR_STACK, "frontier overflow");
    if (c->gexec) {
      cudaGraphExecDestroy(c->gexec);
      c->gexec = nullptr;
    }
  }
  return fail(c, TRILENS_ERR_STACK, "captured run kept overflowing");
}

// graph resources of a context (a batch context makes them when created)
static int ensure_graph(trilens_ctx *c) {
  if (!c->cap_stream) CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  if (!c->run_status) CK(dalloc(&c->run_status, 1));
  if (!c->run_status_host) CK(cudaMallocHost((void **)&c->run_status_host, sizeof(unsigned)));
  if (!c->run_acc) CK(dalloc(&c->run_acc, 1));
  return TRILENS_OK;
}

int trilens_batch_run(trilens_ctx *c, int64_t first_step, int64_t steps, double *yields) {
  if (!c) return TRILENS_ERR_INVALID;
  if (first_step < 0 || steps < 1 || c->n_inst < 2 || !c->cap_stream)
    return fail(c, TRILENS_ERR_INVALID, "batch_run needs a batch context, first_step >= 0, steps >= 1");
  CK(cudaSetDevice(c->device));
  return replay_run(c, first_step, steps, yields);
}

int trilens_run(trilens_ctx *c, int64_t first_step, int64_t steps, trilens_step_stats *out) {
  if (!c) return TRILENS_ERR_INVALID;
  if (first_step < 0 || steps < 1 || c->n_inst > 1)
    return fail(c, TRILENS_ERR_INVALID, "run needs a single context, first_step >= 0, steps >= 1");
  CK(cudaSetDevice(c->device));
  int rc = ensure_graph(c);
  if (rc) return rc;
  if ((rc = replay_run(c, first_step, steps, nullptr))) return rc;
  TLRunAcc h;
  CK(cudaMemcpyAsync(&h, c->run_acc, sizeof(TLRunAcc), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->tot_count += (double)h.count;
  c->tot_weighted += h.weighted;
  if (out) {
    out->step = steps;
    out->count = (int64_t)h.count;
    out->weighted = h.weighted;
    out->hsum = h.hsum;
    out->hxor = h.hxor;
    out->narrow_tests = (int64_t)h.narrow_tests;
    out->node_tests = (int64_t)h.node_tests;
    out->leaf_pairs = (int64_t)h.leaf_pairs;
    out->band = (int64_t)h.band;
    out->retries = 0;
  }
  return TRILENS_OK;
}

int trilens_collide_batch(const trilens_beam *a, const trilens_beam *b, const trilens_params *p,
                          int32_t n_inst, int64_t steps, double *yields, trilens_stream_t stream) {
  if (!yields) return TRILENS_ERR_INVALID;
  trilens_ctx *c = nullptr;
  int rc = trilens_batch_create(&c, a, b, n_inst, p, stream);
  if (rc) return rc;
  rc = trilens_batch_run(c, 0, steps, yields);
  trilens_destroy(c);
  return rc;
}

// ---- tuning ---------------------------------------------------------------

static int apply_tuning(trilens_ctx *c, int bucket, int depth, int warps, int budget) {
  if (bucket < 1 || bucket > 32 || depth < 64 || depth > 4096 || warps < 1 ||
      warps > TL_TRAV_MAX_WARPS ||
      budget < 0)
    return fail(c, TRILENS_ERR_INVALID, "tuning out of range");
  int bps = 0;
  CK(tl::traverse_config(c->p.precision == TRILENS_FP64, warps, depth, &bps));
  if (bps < 1) return fail(c, TRILENS_ERR_INVALID, "traversal shape does not fit an SM");
  c->p.leaf_bucket = bucket;
  c->p.stack_depth = depth;
  c->p.block_shape = warps;
  c->trav_warps = warps;
  c->trav_blocks = bps * c->n_sm;
  c->budget = budget;
  c->front_target = (unsigned)std::min<long long>(2ll * c->trav_blocks * c->trav_warps, 1 << 16);
  unsigned need_front = 0;
  frontier_sizes(c, &c->widen_target, &need_front);
  if (need_front > c->front_cap) {
    c->front_cap = need_front;
    for (int k = 0; k < 2; ++k) {
      cudaFree(c->front[k]);
      c->front[k] = nullptr;
      CK(dalloc(&c->front[k], c->front_cap));
    }
  }
  const unsigned long long warps_now = (unsigned long long)c->trav_blocks * c->trav_warps;
  if (warps_now > c->spill_warps) {
    const int rcs = alloc_spill(c, c->spill_per_warp, warps_now);
    if (rcs) return rcs;
  }
  const unsigned long long need_queue =
      2ull * c->trav_blocks * c->trav_warps * (unsigned long long)depth;
  if (need_queue > c->queue_cap) {
    const int rcq = alloc_queue(c, need_queue);
    if (rcq) return rcq;
  }
  if (c->gexec) {  // a captured run holds the old shapes
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
  }
  c->built_step = -1;  // the leaf bucket changes the hierarchy: build again
  return TRILENS_OK;
}

int trilens_set_tuning(trilens_ctx *c, int32_t leaf_bucket, int32_t stack_depth,
                       int32_t block_shape, int32_t budget) {
  if (!c) return TRILENS_ERR_INVALID;
  CK(cudaSetDevice(c->device));
  return apply_tuning(c, leaf_bucket, stack_depth, block_shape, budget);
}

int trilens_get_tuning(trilens_ctx *c, int32_t out[4]) {
  if (!c || !out) return TRILENS_ERR_INVALID;
  out[0] = c->p.leaf_bucket;
  out[1] = c->p.stack_depth;
  out[2] = c->p.block_shape;
  out[3] = c->budget;
  return TRILENS_OK;
}

// key of a configuration class: sizes rounded to powers of two, precision,
// SM count
static void tuning_key(trilens_ctx *c, char *key, size_t len) {
  int la = 0, lb = 0;
  while ((1ll << la) < std::max<int64_t>(c->beam[0].n, 1)) ++la;
  while ((1ll << lb) < std::max<int64_t>(c->beam[1].n, 1)) ++lb;
  snprintf(key, len, "nA2^%d_nB2^%d_inst%d_prec%d_sm%d", la, lb, c->n_inst, c->p.precision,
           c->n_sm);
}

static bool cache_lookup(const char *path, const char *key, int v[4]) {
  if (!path) return false;
  FILE *f = fopen(path, "r");
  if (!f) return false;
  char line[512];
  bool found = false;
  while (!found && fgets(line, sizeof(line), f)) {
    char k[256];
    int a, b, cc, d;
    if (sscanf(line, " {\"key\": \"%255[^\"]\", \"leaf_bucket\": %d, \"stack_depth\": %d, "
                     "\"block_shape\": %d, \"budget\": %d", k, &a, &b, &cc, &d) == 5 &&
        strcmp(k, key) == 0) {
      v[0] = a; v[1] = b; v[2] = cc; v[3] = d;
      found = true;
    }
  }
  fclose(f);
  return found;
}

static void cache_store(const char *path, const char *key, const int v[4], double ms) {
  if (!path) return;
  // keep the other keys' lines, replace this key's
  std::vector<std::string> keep;
  if (FILE *f = fopen(path, "r")) {
    char line[512];
    while (fgets(line, sizeof(line), f)) {
      std::string l(line);
      if (l.find("\"key\"") != std::string::npos &&
          l.find(std::string("\"") + key + "\"") == std::string::npos) {
        while (!l.empty() && (l.back() == '\n' || l.back() == ',')) l.pop_back();
        keep.push_back(l);
      }
    }
    fclose(f);
  }
  char mine[512];
  snprintf(mine, sizeof(mine),
           " {\"key\": \"%s\", \"leaf_bucket\": %d, \"stack_depth\": %d, \"block_shape\": %d, "
           "\"budget\": %d, \"ms\": %.4f}",
           key, v[0], v[1], v[2], v[3], ms);
  keep.push_back(mine);
  std::string tmp = std::string(path) + ".tmp";
  FILE *f = fopen(tmp.c_str(), "w");
  if (!f) return;
  fprintf(f, "[\n");
  for (size_t i = 0; i < keep.size(); ++i)
    fprintf(f, "%s%s\n", keep[i].c_str(), i + 1 < keep.size() ? "," : "");
  fprintf(f, "]\n");
  fclose(f);
  rename(tmp.c_str(), path);
}

// time build + collide over the sample steps with the current tuning
// the faster of two timed passes over the sample steps (one pass is noisy
// enough to flip close choices)
static int time_steps(trilens_ctx *c, const int64_t *steps, int n, double *ms) {
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const double keep_count = c->tot_count, keep_w = c->tot_weighted;
  double best = 1e30;
  for (int rep = 0; rep < 2; ++rep) {
    CK(cudaEventRecord(e0, c->stream));
    for (int i = 0; i < n; ++i) {
      int rc = trilens_build(c, steps[i]);
      if (!rc) rc = trilens_collide_step(c, steps[i], nullptr, 0, nullptr);
      if (rc) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return rc;
      }
    }
    CK(cudaEventRecord(e1, c->stream));
    CK(cudaEventSynchronize(e1));
    float f = 0.f;
    CK(cudaEventElapsedTime(&f, e0, e1));
    best = std::min(best, (double)f);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->tot_count = keep_count;  // tuning runs do not count towards the yield
  c->tot_weighted = keep_w;
  *ms = best;
  return TRILENS_OK;
}

int trilens_autotune(trilens_ctx *c, const int64_t *steps, int32_t n_steps,
                     const char *cache_path, int32_t chosen[4]) {
  if (!c || !steps || n_steps < 1) return TRILENS_ERR_INVALID;
  CK(cudaSetDevice(c->device));
  char key[128];
  tuning_key(c, key, sizeof(key));
  int v[4];
  if (cache_lookup(cache_path, key, v)) {
    int rc = apply_tuning(c, v[0], v[1], v[2], v[3]);
    if (rc) return rc;
    if (chosen)
      for (int i = 0; i < 4; ++i) chosen[i] = v[i];
    return TRILENS_OK;
  }
  // coordinate descent over the four knobs, each swept with the others
  // fixed at the best so far (stack depth first: a shallow stack moves work
  // to the spill areas, which would bias the other sweeps); results never
  // depend on the knobs, only time does
  int best[4] = {c->p.leaf_bucket, c->p.stack_depth, c->p.block_shape, c->budget};
  static const int cand[4][5] = {{1, 2, 4, 8, 16}, {256, 512, 1024, 0, 0}, {2, 4, 8, 0, 0},
                                 {8, 16, 32, 64, 0}};
  static const int order[4] = {1, 0, 2, 3};
  double best_ms = 1e30;
  int rc = apply_tuning(c, best[0], best[1], best[2], best[3]);
  if (rc) return rc;
  if ((rc = time_steps(c, steps, n_steps, &best_ms))) return rc;  // warm-up
  if ((rc = time_steps(c, steps, n_steps, &best_ms))) return rc;
  for (int oi = 0; oi < 4; ++oi) {
    const int knob = order[oi];
    for (int j = 0; j < 5 && cand[knob][j]; ++j) {
      int t[4] = {best[0], best[1], best[2], best[3]};
      t[knob] = cand[knob][j];
      if (t[knob] == best[knob]) continue;
      if ((rc = apply_tuning(c, t[0], t[1], t[2], t[3]))) continue;  // shape does not fit
      double ms = 0;
      if ((rc = time_steps(c, steps, n_steps, &ms))) return rc;
      if (ms < best_ms) {
        best_ms = ms;
        for (int i = 0; i < 4; ++i) best[i] = t[i];
      }
    }
  }
  if ((rc = apply_tuning(c, best[0], best[1], best[2], best[3]))) return rc;
  cache_store(cache_path, key, best, best_ms);
  if (chosen)
    for (int i = 0; i < 4; ++i) chosen[i] = best[i];
  return TRILENS_OK;
}

int trilens_pair_products(const trilens_beam *a, const trilens_beam *b, const uint32_t *hits,
                          int64_t n_hits, uint64_t seed, double *out, trilens_stream_t stream) {
  if (!beam_ok(a) || !beam_ok(b) || n_hits < 0 || n_hits >= (1ll << 40)) return TRILENS_ERR_INVALID;
  if (n_hits == 0) return TRILENS_OK;
  if (!hits || !out || a->n == 0 || b->n == 0) return TRILENS_ERR_INVALID;
  int dev = 0, n_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return TRILENS_ERR_CUDA;
  TLBeam ta, tb;
  const trilens_beam *bs[2] = {a, b};
  TLBeam *ts[2] = {&ta, &tb};
  for (int k = 0; k < 2; ++k) {
    TLBeam &t = *ts[k];
    t.n = bs[k]->n;
    t.px = bs[k]->px; t.py = bs[k]->py; t.pz = bs[k]->pz;
    t.dx = bs[k]->dx; t.dy = bs[k]->dy; t.dz = bs[k]->dz;
    t.E = bs[k]->E; t.w = bs[k]->w;
  }
  if (tl::launch_pair_products(ta, tb, hits, n_hits, (unsigned long long)seed, out, n_sm,
                               (cudaStream_t)stream) != cudaSuccess)
    return TRILENS_ERR_CUDA;
  return TRILENS_OK;
}

int trilens_step_stats_get(trilens_ctx *c, trilens_step_stats *out) {
  if (!c || !out) return TRILENS_ERR_INVALID;
  *out = c->last;
  return TRILENS_OK;
}

int trilens_yield(trilens_ctx *c, int32_t mode, int32_t level_L, double *count,
                  double *weighted) {
  if (!c || !count || !weighted) return TRILENS_ERR_INVALID;
  if (mode == TRILENS_YIELD_SURROGATE) {
    *count = -1.0;
    return surrogate_total(c, level_L, weighted);
  }
  if (mode != TRILENS_YIELD_EXACT) return fail(c, TRILENS_ERR_INVALID, "yield mode %d", mode);
  *count = c->tot_count;
  *weighted = c->tot_weighted;
  return TRILENS_OK;
}

int trilens_reset_yield(trilens_ctx *c) {
  if (!c) return TRILENS_ERR_INVALID;
  c->tot_count = 0;
  c->tot_weighted = 0;
  return TRILENS_OK;
}

// Test hook (not in the public header): make the first tile of the next
// builds' first sort pass withhold its published counts so that the next tile's
// bounded wait expires.  Used to check that an expired wait becomes
// TRILENS_ERR_TIMEOUT instead of a hang.
int trilens_debug_stall_sort(trilens_ctx *c, int on) {
  if (!c) return TRILENS_ERR_INVALID;
  c->debug_stall_sort = on;
  return TRILENS_OK;
}

int trilens_debug_timing(trilens_ctx *c, int on) {
  if (!c) return TRILENS_ERR_INVALID;
  CK(cudaSetDevice(c->device));
  if (on && !c->ev[0][0][0])
    for (int ph = 0; ph < PH_COUNT; ++ph)
      for (int k = 0; k < 2; ++k)
        for (int e = 0; e < 2; ++e) CK(cudaEventCreate(&c->ev[ph][k][e]));
  c->timing = on ? 1 : 0;
  return TRILENS_OK;
}

int trilens_debug_phase_ms(trilens_ctx *c, double *out, int64_t *launches, int reset) {
  if (!c) return TRILENS_ERR_INVALID;
  for (int ph = 0; ph < PH_COUNT; ++ph) {
    if (out) out[ph] = c->phase_ms[ph];
    if (launches) launches[ph] = c->phase_launches[ph];
    if (reset) {
      c->phase_ms[ph] = 0.0;
      c->phase_launches[ph] = 0;
    }
  }
  return TRILENS_OK;
}

int trilens_debug_set_parts(trilens_ctx *c, int32_t parts) {
  if (!c || parts < 1 || parts > 4096) return TRILENS_ERR_INVALID;
  c->parts = parts;
  if (c->gexec) {  // a captured run holds the old part count
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
  }
  return TRILENS_OK;
}

int trilens_debug_set_spin_limit(trilens_ctx *c, int64_t limit) {
  if (!c || limit < 1) return TRILENS_ERR_INVALID;
  c->p.spin_limit = limit;
  return TRILENS_OK;
}

int trilens_debug_shrink_buffers(trilens_ctx *c, int64_t cap) {
  if (!c || cap < 1) return TRILENS_ERR_INVALID;
  CK(cudaSetDevice(c->device));
  CK(cudaStreamSynchronize(c->stream));
  if (c->gexec) {  // a captured run holds the old buffers
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
  }
  const unsigned long long n = (unsigned long long)cap;
  cudaFree(c->hits);
  cudaFree(c->band);
  cudaFree(c->leaves);
  c->hits = c->band = c->leaves = nullptr;
  c->hit_cap = c->band_cap = c->leaf_cap = n;
  CK(dalloc(&c->hits, n));
  CK(dalloc(&c->band, n));
  CK(dalloc(&c->leaves, n));
  {  // spill areas of cap entries per warp (at least 64)
    const int rcs = alloc_spill(c, (unsigned)std::max<int64_t>(64, std::min<int64_t>(cap, 1 << 20)),
                                c->spill_warps);
    if (rcs) return rcs;
  }
  const int rc = alloc_queue(c, n);
  if (rc) return rc;
  CK(cudaStreamSynchronize(c->stream));
  return TRILENS_OK;
}

int trilens_debug_set_key_bits(trilens_ctx *c, int32_t bits) {
  if (!c || c->n_inst > 1 || bits < 4 || bits > 21) return TRILENS_ERR_INVALID;
  for (int k = 0; k < 2; ++k) {
    c->bits[k] = bits;
    c->key_bits[k] = 3 * bits;
    c->w[k].key_bits = c->key_bits[k];
  }
  if (c->gexec) {  // a captured run holds the old pass count
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
  }
  c->built_step = -1;
  return TRILENS_OK;
}

int trilens_debug_set_cut_cap(trilens_ctx *c, int32_t cap) {
  if (!c) return TRILENS_ERR_INVALID;
  for (int k = 0; k < 2; ++k) {
    tl::BuildBufs &w = c->w[k];
    w.cut_cap = (cap <= 0 || (uint32_t)cap > w.cut_alloc) ? w.cut_alloc : (uint32_t)cap;
  }
  return TRILENS_OK;
}

}  // extern "C"
