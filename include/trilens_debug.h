/*
 * trilens_debug.h -- fault-injection hooks of the trilens library, for tests.
 *
 * They make the library's bounded device waits expire on purpose, on the
 * host's request, so that tests can check that an expired wait is reported
 * as TRILENS_ERR_TIMEOUT and the context stays usable -- without faulting or
 * hanging a GPU.  The paper describes no such mechanism; it is part of the
 * library's own error handling (every device wait carries an iteration
 * limit).
 */
#ifndef TRILENS_DEBUG_H
#define TRILENS_DEBUG_H
#include <stdint.h>
#include "trilens.h"

#ifdef __cplusplus
extern "C" {
#endif

/* on != 0: in the next builds, the first tile of the radix sort's first pass
 * withholds its published digit counts, so the second tile's look-back wait
 * runs to the spin limit, records a timeout and continues.  The following
 * trilens_collide_step then returns TRILENS_ERR_TIMEOUT.  on = 0 restores
 * normal operation.  INVALID for a NULL context. */
int trilens_debug_stall_sort(trilens_ctx *c, int on);

/* Do the traversal and narrow phase of every following step in `parts`
 * slices of its frontier (1..4096), as the library does by itself when a
 * step's leaf-pair list would exceed its largest size (2^30 pairs).  The hit
 * set never depends on it.  INVALID for a NULL context or parts outside
 * 1..4096. */
int trilens_debug_set_parts(trilens_ctx *c, int32_t parts);

/* Replace the context's spin limit (iterations of every bounded device wait,
 * >= 1).  INVALID for a NULL context or limit < 1. */
int trilens_debug_set_spin_limit(trilens_ctx *c, int64_t limit);

/* Morton resolution of a single context's keys: bits per axis (4..21; the
 * default is a few bits beyond one cell per photon).  The hit set never
 * depends on it (the hierarchy only prunes); tests use it to check that, and
 * to time the sort (ceil(3 bits / 8) digit passes) against tree quality.
 * The next collisions need a fresh build.  INVALID for a NULL or batch
 * context or bits outside 4..21. */
int trilens_debug_set_key_bits(trilens_ctx *c, int32_t bits);

/* Capacity of the traversal-seed lists the refit writes (children with at
 * most n/64 photons of nodes with more; normally a few hundred).  cap
 * below the list's length makes the next collisions start from the root pair
 * instead -- the path taken when a list overflows -- so tests can check that
 * both starts give the same hits.  cap <= 0 restores the allocated capacity.
 * INVALID for a NULL context. */
int trilens_debug_set_cut_cap(trilens_ctx *c, int32_t cap);

/* Replace the internal hit, band, leaf-pair and hand-on buffers with buffers of cap
 * pairs each (>= 1), so that the next collisions overflow them and exercise
 * the regrow-and-repeat path.  Synchronises the stream.  INVALID for a NULL
 * context or cap < 1. */
int trilens_debug_shrink_buffers(trilens_ctx *c, int64_t cap);

/* Evaluate the device FP64 functions of the exact decision element-wise:
 * which = 0: sigma(x) of Eq. BWcross [m^2] (0 for x <= 1); which = 1: the
 * natural log of x (x >= 1 finite; the only arguments the decision uses).
 * x and out are device arrays of n doubles; asynchronous on `stream`.
 * INVALID for n < 0, NULL arrays with n > 0 or another `which`. */
int trilens_debug_eval64(const double *x, double *out, int64_t n, int32_t which,
                         trilens_stream_t stream);

/* Per-phase device time.  on != 0 records CUDA events around every kernel
 * phase on the context's stream (cheap, but adds event records).  The
 * phases, in order: 0 propagate+Morton, 1 radix sort, 2 gather, 3 hierarchy
 * emit, 4 refit, 5 frontier (seeds, expansion, widening), 6 dual traversal
 * (listing the overlapping leaf-bucket pairs), 7 FP64 band re-test, 8 yield
 * reduction, 9 FP32 narrow phase of the listed leaf pairs. */
int trilens_debug_timing(trilens_ctx *c, int on);

/* Copy the accumulated milliseconds of the 10 phases into out[0..9], the
 * launches of each phase into launches[0..9] (either may be NULL), then zero
 * them if reset != 0.  Accumulated at each trilens_collide_step (which
 * synchronises). */
int trilens_debug_phase_ms(trilens_ctx *c, double *out, int64_t *launches, int reset);

/* Random stress of the FP32 narrow phase's error band (the precision
 * pattern's guarantee that the FP32 path returns exactly the FP64 hit set of
 * Eq. BWcross / Eq. eq.Cond and the closest-approach test).  Draws n_pairs
 * seeded photon pairs near a boundary of the decision and decides each with
 * the FP32 narrow phase and with the FP64 definition.  Pair q belongs to
 * category q mod 8:
 *   0-3  distance at closest approach d^2 = r^2 (1 +- 2^-e), e in 1..50
 *   4    closest-approach time t* = +-2^-e dt (the window's start)
 *   5    t* = dt (1 +- 2^-e) (the window's end)
 *   6    invariant s = 1 +- 2^-e (the threshold), e in 1..52
 *   7    d^2 uniform in [0, 4 r_max^2), t* in [-0.1 dt, 1.1 dt) (the quick
 *        miss's margin 2.5 r^2, with r^2 bounded over the pair's bin of s)
 * with a random time step 0..63, beam axes at a random angle, 5 mrad spread,
 * and the meeting point anywhere within +-100 um.  counts (device,
 * TRILENS_STRESS_CATEGORIES x TRILENS_STRESS_FIELDS uint64, accumulated: zero
 * it first) receives per category: pairs, FP64 hits, FP32 sure hits, FP32
 * sure misses, FP32 band, sure hits FP64 rejects, sure misses FP64 accepts.
 * The first n_sample pairs (<= n_pairs) are written to sample (device,
 * n_sample x TRILENS_STRESS_SAMPLE doubles: p0 (3), direction (3) and energy
 * of photon i, the same of photon j, the step k, the FP64 decision (0/1) and
 * the FP32 outcome (0 miss, 1 hit, 2 band)).  Asynchronous on `stream`.
 * INVALID for negative sizes, dt_fs or kappa not positive, NULL counts, or
 * n_sample > n_pairs. */
#define TRILENS_STRESS_CATEGORIES 8
#define TRILENS_STRESS_FIELDS 7
#define TRILENS_STRESS_SAMPLE 17
int trilens_debug_band_stress(uint64_t seed, int64_t n_pairs, double dt_fs, double kappa,
                              unsigned long long *counts, double *sample, int64_t n_sample,
                              trilens_stream_t stream);

/* The FP32 narrow phase's sure-miss radii per bin of the invariant s (host
 * only, no GPU): bin 0 holds s < 1; bin 1 + 8 e + k holds s in
 * [2^e (1 + k/8), 2^e (1 + (k+1)/8)) for e = 0..23, the last bin also every
 * larger s.  out (host, n >= TRILENS_NARROW_BINS floats) receives for each bin
 * an upper bound [um^2] on r^2 = 1e12 kappa sigma(s) / pi (Eq. BWcross) over
 * the bin, as the narrow phase of a context with these dt_fs and kappa uses
 * it; *r2max (host, may be NULL) the bound over every s.  Returns the number of
 * bins, or INVALID for non-positive dt_fs or kappa, a NULL out or n too small. */
#define TRILENS_NARROW_BINS 193
int trilens_debug_narrow_bins(double dt_fs, double kappa, float *out, int32_t n, float *r2max);

#ifdef __cplusplus
}
#endif
#endif
