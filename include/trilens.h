/*
 * trilens.h -- C ABI of the GB300 (sm_103a) Breit-Wheeler collision library.
 *
 * Two beams of photons (macro-photons) move on straight lines.  Each time
 * step the library builds, for each beam, a bounding-volume hierarchy over
 * the boxes swept by its photons during the step (Sec. 2.1: a BV grows by the
 * distance its particles travel in one step, so collisions are found before
 * they happen), traverses the two hierarchies against each other with the
 * axis-aligned overlap test (Eq. CollDet; depth-first descent, Sec. 2.2), and
 * tests the surviving photon pairs.  A pair (i in A, j in B) collides in step
 * k when
 *     s = E_i E_j (1 - cos Phi) / (2 m_e^2 c^4) > 1           (Eq. eq.Cond)
 *     t* = time of the pair's closest approach, 0 <= t* - t_k < dt
 *     d(t*)^2 < r^2 = kappa sigma(s) / pi,  sigma from Eq. BWcross
 * and contributes w_i w_j to the pair yield (Sec. 2.2: rates scale with
 * n_I n_II).  Decisions are those of the FP64 definition, bit for bit: in
 * TRILENS_FP32_BAND mode the FP32 fast path only decides pairs that its
 * rigorous error bound puts on one side; the rest are re-tested in FP64.
 *
 * Units: positions um, time fs, energies MeV, sigma m^2, c = 0.299792458 um/fs.
 *
 * Conventions shared by every call:
 *  - Return value: TRILENS_OK (0) or a negative TRILENS_ERR_* code; the last
 *    code and a message are kept per context (trilens_last_error).
 *  - Memory: "device" pointers are CUDA device memory on the context's
 *    device, "host" pointers are ordinary host memory.  The caller owns every
 *    array it passes and keeps input arrays alive and unchanged for the life
 *    of the context; the library owns all workspace it allocates.
 *  - Streams: work is enqueued on the stream given to trilens_create (a
 *    cudaStream_t; NULL = legacy default stream).  Calls that return host
 *    values synchronise that stream.
 *  - Photon indices in hit lists are the caller's input indices.
 */
#ifndef TRILENS_H
#define TRILENS_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *trilens_stream_t; /* == cudaStream_t */
typedef struct trilens_ctx trilens_ctx;       /* opaque, library-owned */

enum trilens_status {
  TRILENS_OK = 0,
  TRILENS_ERR_INVALID = -1,  /* bad argument, detected on the host */
  TRILENS_ERR_CAPACITY = -2, /* caller's hit buffer too small; *n_hits = size needed */
  TRILENS_ERR_CUDA = -3,     /* a CUDA runtime call failed */
  TRILENS_ERR_TIMEOUT = -4,  /* a bounded device wait reached spin_limit */
  TRILENS_ERR_STACK = -5,    /* traversal overflowed after the automatic retries */
  TRILENS_ERR_NOMEM = -6     /* device allocation failed */
};

enum trilens_precision {
  TRILENS_FP64 = 0,      /* every narrow-phase pair decided in FP64 */
  TRILENS_FP32_BAND = 1  /* FP32 decision with FP64 re-test of the band */
};

enum trilens_yield_mode { TRILENS_YIELD_EXACT = 0, TRILENS_YIELD_SURROGATE = 1 };

/* One beam: structure of arrays, FP64, device memory, length n.
 * p = position at t = 0 [um]; d = unit direction (used as given, never
 * renormalised); E = energy [MeV]; w = weight (real photons per
 * macro-photon), NULL means 1 for every photon.  Sec. 2.2 (macro-particles). */
typedef struct {
  int64_t n;
  const double *px, *py, *pz;
  const double *dx, *dy, *dz;
  const double *E;
  const double *w;
} trilens_beam;

/* Stepping and tuning parameters.  Tuning fields set to 0 pick defaults. */
typedef struct {
  double dt_fs;        /* time step [fs], > 0 */
  double kappa;        /* cross-section amplification, > 0 (r^2 = kappa sigma / pi) */
  int32_t precision;   /* enum trilens_precision */
  int32_t leaf_bucket; /* photons per hierarchy leaf, 1..32 (0: 4) */
  int32_t stack_depth; /* traversal stack entries per warp, 64..4096 (0: 512) */
  int32_t block_shape; /* traversal warps per block, 1..8 (0: 4) */
  int64_t spin_limit;  /* iteration limit of every device wait (0: 1<<22) */
} trilens_params;

/* Per-step counters of the last trilens_collide_step call. */
typedef struct {
  int64_t step;
  int64_t count;        /* |H_k|: colliding pairs found in the step */
  double weighted;      /* sum over H_k of w_i w_j (FP64) */
  uint64_t hsum;        /* sum of splitmix64((i << 32) | j) mod 2^64 over H_k */
  uint64_t hxor;        /* xor of the same (order-free checksum pair) */
  int64_t narrow_tests; /* photon pairs given the narrow-phase test */
  int64_t node_tests;   /* box-pair overlap tests during traversal */
  int64_t leaf_pairs;   /* overlapping leaf pairs */
  int64_t band;         /* pairs re-tested in FP64 (FP32_BAND mode) */
  int64_t retries;      /* internal buffer regrowths in this step */
} trilens_step_stats;

/* Create a context for beams a and b (both kept by pointer; arrays must stay
 * valid).  Allocates the workspace for both beams.  Returns INVALID for
 * n < 0, n >= 2^27, missing arrays, dt <= 0, kappa <= 0 or tuning fields out
 * of range; NOMEM if the workspace does not fit. */
int trilens_create(trilens_ctx **out, const trilens_beam *a, const trilens_beam *b,
                   const trilens_params *p, trilens_stream_t stream);

/* Build both hierarchies for step `step` (t_k = step * dt): propagate
 * positions in closed form p0 + c t_k d (FP64), form the FP32 swept boxes
 * (Sec. 2.1), Morton-sort them and emit the hierarchy (Sec. 2.1, 2.2).
 * Asynchronous.  INVALID if step < 0. */
int trilens_build(trilens_ctx *c, int64_t step);

/* Collide the hierarchies built for `step` (trilens_build must have been
 * called with the same step).  Adds the step's counters to the cumulative
 * yield.  If hits != NULL (device, 2*cap uint32: (i_A, j_B) pairs, order
 * unspecified), the step's pairs are written to it; if more than cap exist
 * the call writes nothing, adds nothing to the yield, returns CAPACITY and
 * stores the required size in *n_hits -- call it again for the same step
 * with a larger buffer (no rebuild needed).  n_hits (host) may be NULL.
 * Synchronises the stream (to check device status and regrow internal
 * buffers). */
int trilens_collide_step(trilens_ctx *c, int64_t step, uint32_t *hits, int64_t cap,
                         int64_t *n_hits);

/* Counters of the last collided step (host struct). */
int trilens_step_stats_get(trilens_ctx *c, trilens_step_stats *out);

/* Cumulative yield since creation or the last reset: number of colliding
 * pairs and sum of w_i w_j (host doubles).  mode EXACT returns the exact
 * totals (level_L ignored); mode SURROGATE returns, in *weighted, the sum of
 * trilens_surrogate_step estimates (level_L must be the model's) and sets
 * *count to -1 (the network estimates the weighted yield only). */
int trilens_yield(trilens_ctx *c, int32_t mode, int32_t level_L, double *count,
                  double *weighted);

/* Run time steps first_step .. first_step+steps-1 of a single (non-batch)
 * context -- trilens_build + trilens_collide_step for each, in step order --
 * as one captured CUDA graph on the context's stream, with no host round
 * trip between steps (each step's traversal is one launch whose warps share
 * a device work queue, so no step needs the host).  The graph is captured on the
 * first call and replayed while (first_step, steps) stay the same.  Adds the
 * run's yield to the cumulative yield; out (host, may be NULL) receives the
 * run's totals: step = steps, count, weighted, the checksums (hsum summed,
 * hxor xored over the steps) and the work counters.  Hit lists are not
 * returned.  On an internal overflow the buffer grows and the whole run is
 * repeated (the result is that of a complete run).  Synchronises the stream
 * at the end.  INVALID for a batch context, first_step < 0 or steps < 1;
 * TIMEOUT if a device wait ran out. */
int trilens_run(trilens_ctx *c, int64_t first_step, int64_t steps, trilens_step_stats *out);

/* The electron and the positron of each collision (Sec. 1, Eq. pTotal and
 * Eq. Lorentz).  hits: device, n_hits (i, j) uint32 pairs (i indexes beam a,
 * j beam b), e.g. a trilens_collide_step hit list.  For each, the photons'
 * total energy E and momentum P (MeV, c = 1) define the centre-of-mass (CoM)
 * frame, where each particle has energy M/2 (M^2 = E^2 - |P|^2) and momentum
 * p' = sqrt(M^2/4 - m_e^2); the electron flies along a random direction n
 * uniform on the sphere, the positron opposite, and both are boosted back to
 * the lab.  n is drawn from a counter-based splitmix64 stream keyed by
 * seed ^ ((i << 32) | j) (Marsaglia's method), so a hit's products depend
 * only on (seed, i, j).  out: device, n_hits x 8 doubles = electron (E, px,
 * py, pz), positron (E, px, py, pz) [MeV]; a hit whose indices are out of
 * range or whose pair is below threshold gets zeros.  FP64, every operation
 * rounded to nearest in a fixed order.  Asynchronous on `stream` (the current
 * device); allocates nothing.  INVALID for a bad beam, negative n_hits, or
 * NULL arrays with n_hits > 0. */
int trilens_pair_products(const trilens_beam *a, const trilens_beam *b, const uint32_t *hits,
                          int64_t n_hits, uint64_t seed, double *out, trilens_stream_t stream);

/* Depletion with chronological order (Sec. 2.2, Sec. 3.1, Fig. ChronOrder).
 * Photons annihilate when they collide, so a hit only produces pairs if both
 * photons still exist when it happens.  The hits of step `step` -- hits:
 * device, n_hits distinct (i, j) uint32 pairs as trilens_collide_step wrote
 * them -- are taken in the order of their closest-approach time t* (then i,
 * then j); t* is computed in FP64 with the operations of the exact decision.
 * A macro-photon of weight w stands for w photons handled one by one, so a
 * hit takes delta = min(rem_a[i], rem_b[j]) from both photons (with unit
 * weights: a photon's earliest remaining hit annihilates it).
 *
 * rem_a (n_a doubles) and rem_b (n_b doubles): device, caller-owned, what
 * each photon of the context's beams still holds; initialise them to the
 * weights (or 1) before the first step and pass them unchanged from step to
 * step, calling steps in increasing order, so that hits of earlier steps come
 * first.  They must be >= 0.  Updated in place.  delta: device, n_hits
 * doubles, what each hit took (in the order of `hits`), or NULL.  *n_accepted
 * (host, may be NULL): hits with delta > 0; *transferred (host, may be NULL):
 * the sum of delta, i.e. the pairs made (summed in a fixed order, so the
 * value is reproducible).
 *
 * Runs on the context's stream as one cooperative launch (every round inside
 * it, the open hits compacted after each round; a step needs as many rounds
 * as its longest chain of hits that wait on one another) and returns when the
 * step is done, after one 32-byte read-back.  Allocates its workspace on the
 * first call (96 bytes per photon of both beams, 25 per hit, growing with
 * n_hits).  TIMEOUT (rem_a, rem_b and delta then unspecified; the photon
 * slots are cleared on the device by the next call) if a grid-wide barrier
 * wait inside the launch reaches the context's spin_limit.  INVALID (nothing changed except delta, which
 * may hold zeros) for a NULL context, a negative step, n_hits < 0 or >= 2^32,
 * NULL hits/rem arrays with n_hits > 0, an index out of range or a negative
 * or NaN rem of a listed photon.  A pair listed twice is not supported. */
int trilens_deplete_step(trilens_ctx *c, int64_t step, const uint32_t *hits, int64_t n_hits,
                         double *rem_a, double *rem_b, double *delta, int64_t *n_accepted,
                         double *transferred);

/* Record of one asynchronous depletion call, written to device memory when the
 * call completes on the context's stream. */
typedef struct trilens_deplete_out {
  double transferred; /* the sum of delta: the pairs made */
  int64_t accepted;   /* hits with delta > 0 */
  int64_t rounds;     /* rounds that had open hits */
  int64_t status;     /* TRILENS_OK; TRILENS_ERR_INVALID (an index out of range or a
                         negative or NaN rem: nothing changed except delta);
                         TRILENS_ERR_TIMEOUT (a barrier wait reached spin_limit:
                         rem_a, rem_b and delta unspecified); the other fields are 0
                         unless the status is TRILENS_OK */
} trilens_deplete_out;

/* trilens_deplete_step without the wait: the call is enqueued on the context's
 * stream and returns; what the synchronous call returns on the host (and its
 * status) goes to `out` (device, caller-owned, 8-byte aligned, one record)
 * when the call completes.  Calls for consecutive steps may be enqueued back
 * to back, each with its own hit list, and `out` read once at the end.  A call
 * whose status is not OK leaves the photon slots marked for clearing; the next
 * call clears them first, on the device.  Same arguments and workspace as
 * trilens_deplete_step; n_hits == 0 writes an all-zero record (status OK).
 * INVALID (nothing enqueued) for the argument errors trilens_deplete_step
 * reports before it launches, or an unaligned or NULL out. */
int trilens_deplete_step_async(trilens_ctx *c, int64_t step, const uint32_t *hits,
                               int64_t n_hits, double *rem_a, double *rem_b, double *delta,
                               trilens_deplete_out *out);

/* Rounds that had open hits in the last successful trilens_deplete_step call
 * (the longest chain of hits waiting on one another). */
int trilens_deplete_rounds(trilens_ctx *c, int64_t *rounds);

/* IP regime (Sec. 2.2): macro-photons (MPs) of integer weight w split into
 * swarms of w real photons when they collide.  A swarm has its MP's energy
 * and direction; its photons are spread over the MP's volume, taken as an
 * axis-aligned cube of side h (one h per beam, um) centred on the MP: photon
 * k sits at p0 + h u_k, u_k,d = frac(0.5 + k alpha_d) - 0.5 with alpha =
 * (1/g, 1/g^2, 1/g^3), g^4 = g + 1 (Roberts' R_3 low-discrepancy sequence;
 * u_0 = 0, so a weight-1 MP is its own photon).  Every real-photon pair is
 * then decided like a pair of single photons.  Three calls write the real
 * photons of the MPs that can collide; the caller then runs the exact path
 * (trilens_create on the expanded beams, trilens_run / trilens_collide_step,
 * and trilens_deplete_step for annihilation of individual photons) and maps
 * each hit back to (MP, photon in swarm) with the owner / index arrays.
 *
 * trilens_swarm_mark: mark_a (n_a bytes) and mark_b (n_b bytes), device,
 * receive 1 for every MP that belongs to a pair which can collide in steps
 * [first_step, first_step + steps) of dt = p->dt_fs (with kappa = p->kappa),
 * else 0.  The test is conservative (s > 1 up to a relative 1e-9; the MP
 * centres' closest approach within the window at most the largest collision
 * radius plus both cubes' half-diagonals, with margins for rounding), so the
 * marked MPs hold every real-photon hit of the run.  FP64, all MP pairs,
 * asynchronous on `stream`.  INVALID for bad beams, h < 0, dt or kappa <= 0,
 * first_step < 0, steps < 1, or NULL marks of non-empty beams. */
int trilens_swarm_mark(const trilens_beam *a, const trilens_beam *b, double h_a, double h_b,
                       const trilens_params *p, int64_t first_step, int64_t steps,
                       uint8_t *mark_a, uint8_t *mark_b, trilens_stream_t stream);

/* offsets (device, n + 1 int64): offsets[i] = the sum of the weights of the
 * marked MPs before i, offsets[n] = *total (host) = the real photons of the
 * marked swarms.  Weights (mp->w, NULL = all 1) must be integers in
 * [1, 2^32): INVALID otherwise (offsets then undefined).  Returns after the
 * stream has done it; uses stream-ordered scratch (cudaMallocAsync). */
int trilens_swarm_count(const trilens_beam *mp, const uint8_t *mark, int64_t *offsets,
                        int64_t *total, trilens_stream_t stream);

/* Write the `total` real photons: out (host array of 8 device pointers, each
 * `total` doubles: px py pz dx dy dz E w; out[7] may be NULL, else all 1),
 * owner[q] = the MP of photon q and index_in_swarm[q] = its k (device uint32,
 * `total` each).  Photons come grouped by MP in MP order, k ascending.
 * Positions p0 + h u_k in FP64 (each product and sum rounded to nearest).
 * Asynchronous on `stream`; allocates nothing. */
int trilens_swarm_expand(const trilens_beam *mp, double h, const int64_t *offsets,
                         int64_t total, double *const *out, uint32_t *owner,
                         uint32_t *index_in_swarm, trilens_stream_t stream);

/* Zero the cumulative yield. */
int trilens_reset_yield(trilens_ctx *c);

/* Free the context and its workspace.  NULL is ignored. */
void trilens_destroy(trilens_ctx *c);

/* Message for a status code (static string). */
const char *trilens_status_str(int code);

/* Last error message recorded in a context (static until the next call). */
const char *trilens_last_error(trilens_ctx *c);

/* Library version string. */
const char *trilens_version(void);

/* ---- batches of independent instances ------------------------------------
 * Many independent beam crossings of uneven size (each one the problem above)
 * run as one problem: all instances' photons are concatenated per side, the
 * instance number is placed above the Morton bits of every photon's key so
 * that one sort and one hierarchy per side hold every instance as its own
 * subtree, and the traversal starts from each instance's pair of subtree
 * roots, so no pair of photons from different instances is ever tested.
 * dt and kappa are shared by all instances. */

/* Create a batch context from n_inst instances: a[q], b[q] are the two beams
 * of instance q (device arrays as in trilens_beam; copied into library-owned
 * concatenated arrays, so they need not outlive the call).  Photon indices of
 * the context (hit lists of trilens_collide_step) are positions in the
 * concatenation, instance by instance.  INVALID for n_inst outside
 * [1, 65536], a bad beam, or more than 2^27 photons per side. */
int trilens_batch_create(trilens_ctx **out, const trilens_beam *a, const trilens_beam *b,
                         int32_t n_inst, const trilens_params *p, trilens_stream_t stream);

/* Run time steps first_step .. first_step+steps-1 of every instance (build +
 * collide per step) as one captured CUDA graph, launched on the context's
 * stream; the graph is captured on the first call and replayed while
 * (first_step, steps, yields) stay the same.  yields (device, n_inst x 2
 * doubles) receives, per instance, the number of colliding pairs and the sum
 * of w_i w_j over the run.  Synchronises the stream at the end to check
 * device status; on an internal overflow it enlarges the buffer and runs the
 * graph again (the result is that of a complete run).  INVALID on a context
 * that trilens_batch_create did not make. */
int trilens_batch_run(trilens_ctx *c, int64_t first_step, int64_t steps, double *yields);

/* One call: trilens_batch_create, trilens_batch_run(0, steps), destroy. */
int trilens_collide_batch(const trilens_beam *a, const trilens_beam *b, const trilens_params *p,
                          int32_t n_inst, int64_t steps, double *yields, trilens_stream_t stream);

/* ---- tuning -----------------------------------------------------------------
 * The hit set never depends on these knobs; only the time does.
 *   leaf_bucket  photons per hierarchy leaf (1..32)
 *   stack_depth  traversal stack entries per warp in shared memory (64..4096; the
 *                rest of a warp's stack is its private spill area in global memory)
 *   block_shape  traversal warps per block (1..8)
 *   budget       traversal iterations a warp spends on one work item before it
 *                hands the rest on, as chunks of 8 node pairs, to the step's
 *                device work queue, where idle warps take them (0 = never;
 *                default 16) */

/* Set the knobs; the next trilens_collide_step needs a fresh trilens_build.
 * INVALID if a knob is out of range or the shape does not fit an SM. */
int trilens_set_tuning(trilens_ctx *c, int32_t leaf_bucket, int32_t stack_depth,
                       int32_t block_shape, int32_t budget);

/* Current knobs into out[4] (leaf_bucket, stack_depth, block_shape, budget). */
int trilens_get_tuning(trilens_ctx *c, int32_t out[4]);

/* Autotuner.  If cache_path (a JSON file; NULL = no cache) holds an entry for
 * this context's configuration class (beam sizes rounded to powers of two,
 * instance count, precision, SM count), apply it.  Otherwise time build +
 * collide of the n_steps sample steps while sweeping each knob in turn (the
 * others held at the best so far), apply the fastest, and record it in the
 * cache.  Tuning runs are not added to the yield.  chosen (host, 4 ints) may
 * be NULL.  Synchronises the stream. */
int trilens_autotune(trilens_ctx *c, const int64_t *steps, int32_t n_steps,
                     const char *cache_path, int32_t chosen[4]);

/* ---- surrogate network ------------------------------------------------------
 * The learned part of the statistical regime (the paper's ST regime estimates
 * collision rates of whole clouds, Sec. 2.2; here a network estimates the
 * pair yield of whole node pairs): 24 -> 128 -> 128 -> 128 -> 2 with exact
 * GELU, BF16 weights and activations, FP32 accumulation on the tensor cores.
 * Parameters are a flat FP32 device vector of TRILENS_MLP_PARAMS floats:
 * W1 (128x24), b1 (128), W2 (128x128), b2, W3 (128x128), b3, W4 (2x128), b4 (2),
 * each W row-major [out][in], layer z = W h + b.  norm (device, 48 floats) holds
 * the feature mean[24] and 1/std[24] applied to the raw features first.
 * Output per row: (mu, s), a Gaussian over the target y (for the surrogate,
 * the residual of log1p(pair yield) over log1p of the ST-rate baseline) with
 * log variance s; loss 0.5 (s + (y - mu)^2 e^-s), s clamped to +-12. */
#define TRILENS_MLP_PARAMS 36482

/* out (device, m x 2 FP32) = network(x) for x (device, m x 24 FP32 raw
 * features).  Synchronises the stream.  TIMEOUT if a tensor-core wait ran out. */
int trilens_mlp_forward(const float *params, const float *norm, const float *x, int64_t m,
                        float *out, trilens_stream_t stream);

/* grad (device, TRILENS_MLP_PARAMS FP32) = gradient of the MEAN loss over the
 * m rows of (x, y) (y: device, m FP32 targets); loss (device, 1 FP32) = the
 * SUM of the per-row losses.  loss_kind 0: the Gaussian NLL above (st
 * unused).  loss_kind 1 (what the surrogate trains): y is the linear label
 * Y, B = st_scale * st[row] a baseline (st: device, m FP32), lam = (B + 1)
 * e^mu the predicted mean, per-row loss (lam - Y ln lam)/(B + 1) +
 * 0.5 (s + r^2 e^-s) with r = log1p(Y) - log1p(lam), lam held fixed in r (its
 * gradient does not reach mu).  Synchronises the stream. */
int trilens_mlp_grad(const float *params, const float *norm, const float *x, const float *y,
                     const float *st, float st_scale, int32_t loss_kind, int64_t m, float *grad,
                     float *loss, trilens_stream_t stream);

/* ---- learned statistical regime ----------------------------------------------
 * The dual traversal stops at hierarchy level L: the first node on every path
 * whose Morton prefix is at least L bits long (or a leaf bucket), so every
 * photon lies in exactly one level-L node of its beam.  Overlapping level-L
 * node pairs get 24 features -- centre offset (3), half-extents of both boxes
 * (6), log counts (2), log weight sums (2), mean and std of ln E (4), mean
 * directions (6), 1 - dA.dB of the means (1) -- from FP64 prefix sums of the
 * weights and their energy and direction moments over the Morton-ordered
 * photons.  Training labels are the exact yields of the pairs (an exact
 * traversal seeded with the pairs; every hit is attributed to the pair that
 * holds its two photons).  Next to the features the kernels compute the
 * paper's ST rate of the pair (Eq. rate, n_I n_II <sigma v>, for the two
 * nodes read as boxes of uniform density moving with their mean velocities:
 * W_A W_B (1e12 kappa sigma(sbar)) c |dbar_A - dbar_B| times the time integral
 * of the boxes' overlap volume over the step, over V_A V_B; sbar from the
 * geometric-mean energies and the mean directions).  B, that rate times a
 * constant fitted on the training pairs, is the network's baseline: it
 * predicts each pair's mean yield (B + 1) e^mu over B
 * (trained with a Poisson-type deviance, whose minimiser is the conditional
 * mean; trilens_mlp_grad loss_kind 1), times a calibration scale fitted on
 * the training pairs; pairs whose predicted standard deviation of y
 * exceeds tau are evaluated exactly instead (the fallback), and the scale is
 * then the one fitted on the training pairs the network keeps at that tau
 * (a table over tau = 2^(g/2 - 10), g = 0..63; the largest edge <= tau). */

/* Build each listed step, collect its level-L pairs with features and exact
 * labels into the context's training set (steps are not added to the
 * yield).  INVALID for level_L outside [1, 63], n < 1, a batch context, or a
 * level different from samples already collected. */
int trilens_surrogate_collect(trilens_ctx *c, const int64_t *steps, int32_t n, int32_t level_L);

/* Train the network on the collected samples (feature normalisation from
 * the samples, He-initialised weights from `seed`, AdamW with cosine decay,
 * minibatches of 8192, `epochs` passes), then fit the calibration scales of
 * the network's estimate and of the ST rate on all the samples, and the
 * network's per fallback threshold (on the samples the network keeps). */
int trilens_surrogate_fit(trilens_ctx *c, int32_t epochs, uint64_t seed);

/* collect + fit. */
int trilens_surrogate_train(trilens_ctx *c, const int64_t *train_steps, int32_t n, int32_t level_L,
                            int32_t epochs, uint64_t seed);

/* Surrogate yield of the built step (trilens_build(step) first) with a model
 * trained or loaded for the same level_L.  out (host, 8 doubles): [0] the
 * estimated weighted yield (network part plus exact fallback), [1] the
 * ST rate of the same pairs summed (no network, no fitted scale;
 * trilens_surrogate_info [3] is the one scale fitted to it on the training
 * pairs), [2] level-L
 * pairs, [3] pairs sent to the fallback, [4] their exact yield, [5] device
 * milliseconds of the whole surrogate path, [6] of network + estimate, [7]
 * of the cut traversal + features.  Adds [0] to the cumulative surrogate
 * yield (trilens_yield with TRILENS_YIELD_SURROGATE). */
int trilens_surrogate_step(trilens_ctx *c, int64_t step, int32_t level_L, float tau,
                           double out[8]);

/* The level-L node pairs of the built step, for inspection and tests: what
 * the surrogate step sees (ST regime at the cut, Sec. 2.2).  Every array is
 * caller-owned host memory of the stated size, or NULL to skip it; arrays
 * per pair hold the first min(cap, n_pairs) pairs.
 *   cloud       2 x cap uint32: the pair's cut node in beam A and in beam B
 *               (ids 0 .. of the level-L frontier of each tree)
 *   feat        24 x cap FP32 features (see trilens_surrogate_dataset)
 *   st          cap FP32: the ST rate of the pair -- the expected number of
 *               pairs of Eq. rate for the two nodes as uniform boxes moving
 *               with their mean velocities over the step (no fitted scale)
 *   label       cap FP64: the pair's exact yield, sum of w_i w_j over its hits
 *   pred        cap FP64: the network's estimate (0 where the pair falls back)
 *   fallback    cap bytes: 1 where the predicted spread exceeds tau
 *   net         2 x cap FP32: the network's outputs (mu, log variance)
 *   cloud_of_a  n_a uint32: the cut node of every input photon of beam A
 *   cloud_of_b  n_b uint32: the same for beam B
 * n_pairs receives the number of pairs; fallback_exact the exact yield of the
 * pairs that fall back (computed when pred, fallback or net is requested,
 * which needs a model trained at level_L).  The cumulative yields are left
 * unchanged.  INVALID for a step that is not built, a bad level, or a
 * missing model. */
typedef struct {
  int64_t cap;
  int64_t n_pairs;
  uint32_t *cloud;
  float *feat;
  float *st;
  double *label;
  double *pred;
  uint8_t *fallback;
  float *net;
  uint32_t *cloud_of_a;
  uint32_t *cloud_of_b;
  double fallback_exact;
} trilens_sur_pairs;
int trilens_surrogate_pairs(trilens_ctx *c, int64_t step, int32_t level_L, float tau,
                            trilens_sur_pairs *out);

/* [0] samples collected, [1] last training loss, [2] network calibration,
 * [3] the single scale of the ST rate fitted on the samples (sum of labels
 * over sum of ST rates), [4] level L, [5] cumulative surrogate yield. */
int trilens_surrogate_info(trilens_ctx *c, double out[6]);

/* Copy the training set to host arrays of capacity cap: x (cap x 24 FP32
 * features), label (cap FP64 exact pair yields), st (cap FP32 ST rates, no
 * fitted scale); any may be NULL.  *n receives the number of samples. */
int trilens_surrogate_dataset(trilens_ctx *c, float *x, double *label, float *st, int64_t cap,
                              int64_t *n);

/* Append samples (host arrays as trilens_surrogate_dataset returns them)
 * to the context's training set, e.g. pairs collected in other contexts
 * (other seeds).  INVALID on a level mismatch. */
int trilens_surrogate_add_samples(trilens_ctx *c, const float *x, const double *label,
                                  const float *st, int64_t n, int32_t level_L);

/* Save / load the model (level, calibrations and the table by fallback
 * threshold, feature normalisation and parameters) as a little-endian binary
 * file ("TRLSUR03"; an older "TRLSUR02" file without the table loads with
 * one scale for every threshold). */
int trilens_surrogate_save(trilens_ctx *c, const char *path);
int trilens_surrogate_load(trilens_ctx *c, const char *path);

/* Largest hit list trilens_yield_reduce_noalloc accepts (2^28 pairs). */
#define TRILENS_NOALLOC_MAX_HITS (1ll << 28)

/* Yield reduction that allocates no device memory.  The paper has no
 * counterpart; this is a service for callers that cannot call cudaMalloc
 * (code that runs inside another framework's memory pool or under a fixed
 * memory budget, or that must not change the device's allocation state).
 *
 * Reduces a hit list -- hits: device, 2 * n_hits uint32 (i_A, j_B) pairs as
 * written by trilens_collide_step -- with the weights w_a, w_b (device FP64
 * arrays indexed by i_A and j_B; NULL means weight 1) to the four values
 * trilens_collide_step reports for a step: out_result (device, 32 bytes) =
 * { uint64 count, double sum of w_i w_j, uint64 checksum sum, uint64
 * checksum xor } (see trilens_step_stats).  Count and checksums are
 * bit-identical to the step's; the weighted sum equals it up to rounding
 * (the terms are added in another order).  Asynchronous on `stream`.
 * hits and out_result must be 8-byte aligned (TRILENS_ERR_INVALID
 * otherwise, before anything is launched).
 *
 * Scratch lives in a fixed 128 KiB device array inside the library (held on
 * every GPU that loads it until the process exits), so n_hits is limited to
 * TRILENS_NOALLOC_MAX_HITS; larger lists, negative n_hits or NULL pointers
 * give TRILENS_ERR_INVALID without launching anything.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current, so make it before any stream capture.  All calls share
 * the array: calls that overlap on the GPU (other streams, other threads)
 * race and must be serialised by the caller. */
int trilens_yield_reduce_noalloc(const uint32_t *hits, int64_t n_hits, const double *w_a,
                                 const double *w_b, void *out_result, trilens_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* TRILENS_H */
