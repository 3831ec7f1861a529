// tl_ctx.h -- the library context shared by the host translation units
// (private; the public interface is include/trilens.h).
#pragma once
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>

#include "tl_common.cuh"
#include "trilens.h"

struct SurrogateState;
struct DepState;

constexpr int kMaxLevels = 24;

struct trilens_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  trilens_params p{};
  TLBeam beam[2]{};
  // derived constants
  double L64 = 0, rmax = 0, sigma_max = 0;
  float L_lo = 0, L_hi = 0, half = 0;
  TLNarrowConst nk{};
  int bits[2]{}, key_bits[2]{};
  // per beam and axis: sums of p0, d, p0^2, p0 d, d^2 (one-time, fixed order)
  double moments[2][15]{};
  // build workspace
  tl::BuildBufs w[2]{};
  int sel[2]{};
  int64_t built_step = -1;
  // traversal workspace
  int n_sm = 0, trav_warps = 4, trav_blocks = 0, expand_blocks = 0;
  int budget = 16;  // traversal iterations per work item before it is handed on
  unsigned front_target = 0, front_cap = 0, widen_target = 0;
  uint2 *front[2]{};
  uint2 *queue = nullptr;  // traversal work queue (every free slot holds the sentinel)
  unsigned long long queue_cap = 0;
  uint2 *spill = nullptr;  // traversal warps' private spill areas
  unsigned spill_per_warp = 8192;
  unsigned long long spill_warps = 0;  // warps the areas are allocated for
  uint2 *hits = nullptr;
  unsigned long long hit_cap = 0;
  uint2 *band = nullptr;
  unsigned long long band_cap = 0;
  uint2 *leaves = nullptr;  // the step's overlapping leaf-bucket pairs
  unsigned long long leaf_cap = 0;
  int parts = 1;  // a step's traversal in this many slices of its frontier
  TLCounters *ctr = nullptr;
  TLCounters *ctr_host = nullptr;  // pinned
  void *partials = nullptr;
  int yield_blocks = 0;
  unsigned *build_status = nullptr;  // device status of the builds (sort waits)
  unsigned *build_status_host = nullptr;
  // results
  trilens_step_stats last{};
  double tot_count = 0, tot_weighted = 0;
  int debug_stall_sort = 0;
  // several independent instances (batch contexts)
  int n_inst = 1;
  uint32_t *inst_of[2]{};     // device, instance of every photon
  uint32_t *inst_root[2]{};   // device, subtree root (stack reference) per instance
  double *inst_bounds[2]{};   // device, 12 doubles per instance
  float4 *inst_box[2]{};      // device, Morton box of every instance for the current build
  long long *inst_tmp = nullptr;
  double *owned[2][8]{};      // concatenated inputs owned by a batch context
  // graph-captured multi-step runs (batch contexts)
  cudaStream_t cap_stream = nullptr;
  // beam B is built on side_stream, forked from and joined back into the
  // context's stream (the two builds are independent)
  cudaStream_t side_stream = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int64_t g_first = -1, g_steps = 0;
  double *g_yields = nullptr;
  TLRunAcc *run_acc = nullptr;       // device totals of a captured single-context run
  unsigned *run_status = nullptr;
  unsigned *run_status_host = nullptr;
  // per-phase timing (events on the context's stream) and launch counts
  int timing = 0;
  cudaEvent_t ev[10][2][2]{};   // [phase][beam or 0][start, end]
  bool ev_pending[10][2]{};
  double phase_ms[10]{};
  int64_t phase_launches[10]{};
  SurrogateState *sur = nullptr;  // learned statistical regime (tl_surrogate_host.cu)
  DepState *dep = nullptr;        // depletion workspace (tl_deplete.cu)
  int64_t dep_rounds = 0;         // rounds the last depletion call took
  char msg[512] = {0};
};


static inline int fail(trilens_ctx *c, int code, const char *fmt, ...) {
  if (c) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->msg, sizeof(c->msg), fmt, ap);
    va_end(ap);
  }
  return code;
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(c, e_ == cudaErrorMemoryAllocation ? TRILENS_ERR_NOMEM : TRILENS_ERR_CUDA, \
                  "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__);  \
  } while (0)

// ---- allocation helpers

template <class T>
static inline cudaError_t dalloc(T **p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  return cudaMalloc((void **)p, sizeof(T) * count);
}

// (re)allocate the traversal queue with cap slots, every slot the sentinel
// the traversal queue never grows past 2^30 node pairs (8 GiB): a step that
// asks for more fails with TRILENS_ERR_STACK (deeper stacks hand on less)
static inline int alloc_queue(trilens_ctx *c, unsigned long long cap) {
  if (cap > (1ull << 30))
    return fail(c, TRILENS_ERR_STACK, "the traversal queue would need %llu node pairs",
                (unsigned long long)cap);
  cudaFree(c->queue);
  c->queue = nullptr;
  c->queue_cap = 0;
  CK(dalloc(&c->queue, (size_t)cap));
  CK(cudaMemsetAsync(c->queue, 0xff, sizeof(uint2) * (size_t)cap, c->stream));
  c->queue_cap = cap;
  return TRILENS_OK;
}

// the traversal warps' private spill areas, for blocks x warps warps of
// per_warp entries each (at most 2^20 per warp)
static inline int alloc_spill(trilens_ctx *c, unsigned per_warp, unsigned long long warps) {
  if (per_warp > (1u << 20))
    return fail(c, TRILENS_ERR_STACK, "a traversal warp's spill area would need %u entries",
                per_warp);
  cudaFree(c->spill);
  c->spill = nullptr;
  c->spill_warps = 0;
  CK(dalloc(&c->spill, (size_t)per_warp * warps));
  c->spill_per_warp = per_warp;
  c->spill_warps = warps;
  return TRILENS_OK;
}

static inline int grow(trilens_ctx *c, uint2 **buf, unsigned long long *cap, unsigned long long need) {
  unsigned long long nc = std::max<unsigned long long>(need + need / 4 + 1024, *cap * 2);
  cudaFree(*buf);
  *buf = nullptr;
  *cap = 0;
  CK(dalloc(buf, (size_t)nc));
  *cap = nc;
  return TRILENS_OK;
}


// traversal arguments for the current build at time c t_k = ct
tl::TravArgs trav_args(trilens_ctx *c, double ct);
// exact collision of seed pairs (or, with seeds == NULL, of the whole
// hierarchies from the roots) for the built step; fills c->ctr_host
int run_exact(trilens_ctx *c, double ct, const uint2 *seeds, unsigned n_seeds, int *retries);
void surrogate_free(trilens_ctx *c);
void deplete_free(trilens_ctx *c);
double tl_sigma_max_bound();
TLNarrowConst tl_narrow_const(double dt_fs, double kappa);
extern "C" int surrogate_total(trilens_ctx *c, int level, double *out);
