/*
 * oracle.h -- FP64 CPU oracle for Breit-Wheeler collision detection between
 * two photon beams.  TEST INFRASTRUCTURE ONLY: the tests, the smoke check and
 * the benchmark's CPU-baseline leg call it; the product path never does.
 *
 * It shares no code with the CUDA path.  Every function is the plain
 * definition, evaluated in IEEE double with no FMA contraction
 * (compile with -ffp-contract=off), in the operation order written here.
 *
 * Units: um, fs, MeV; cross sections in m^2.
 */
#ifndef TRILENS_ORACLE_H
#define TRILENS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int64_t n;
  const double *px, *py, *pz; /* position at t = 0 [um] */
  const double *dx, *dy, *dz; /* unit direction */
  const double *E;            /* energy [MeV] */
  const double *w;            /* weight (real photons per macro-photon) */
} oracle_beam;

typedef struct {
  int64_t count;    /* |H_k|, hits found (may exceed the caller's capacity) */
  double weighted;  /* sum over hits of w_i * w_j */
  uint64_t hsum;    /* sum of splitmix64((i << 32) | j) mod 2^64 */
  uint64_t hxor;    /* xor of the same */
  int64_t tests;    /* photon pairs given the full narrow-phase test */
  int64_t node_tests; /* box-pair overlap tests (tree only) */
} oracle_result;

/* natural log by argument reduction to [sqrt(1/2), sqrt(2)) and the odd
 * atanh series ln m = 2 (f + f^3/3 + ... + f^23/23), f = (m-1)/(m+1) */
double oracle_ln(double x);
/* Eq. BWcross: total Breit-Wheeler cross section [m^2]; 0 for s <= 1 */
double oracle_sigma(double s);
/* the invariant s of the text below Eq. BWcross */
double oracle_s(double E1, double E2, double cos_phi);
/* maximum of oracle_sigma over s (golden-section search) */
double oracle_sigma_max(void);
/* the full per-pair decision for step k (positions propagated in closed form) */
int oracle_pair_hit(const oracle_beam *a, int64_t i, const oracle_beam *b, int64_t j,
                    int64_t step, double dt, double kappa);
/* the same decision with the pieces it computed (for diagnostics/tests) */
int oracle_pair_detail(const oracle_beam *a, int64_t i, const oracle_beam *b, int64_t j,
                       int64_t step, double dt, double kappa, double out[6]);
uint64_t oracle_splitmix64(uint64_t x);

/* Pair products of collisions (Sec. 1, Eq. pTotal and Eq. Lorentz): for each
 * hit (hits[2k] = i in a, hits[2k+1] = j in b) the electron and the positron
 * made from photons i and j.  The photons' total energy E and momentum P
 * (units of MeV, c = 1) fix the centre-of-mass (CoM) frame; there each
 * particle has energy M/2 (M^2 = E^2 - P^2 = 2 E_i E_j (1 - cos)) and momentum
 * p' = sqrt(M^2/4 - m^2), the electron along a random unit vector n and the
 * positron opposite; both are boosted back to the lab.  n is uniform on the
 * sphere: Marsaglia (1972) from uniforms of splitmix64 (the counter-based
 * stream of key = seed ^ ((i << 32) | j), draws splitmix64(key + t), t = 0, 1,
 * ...).  out[8k .. 8k+7] = electron (E, px, py, pz), positron (E, px, py, pz)
 * [MeV].  Returns 0, or -1 if a hit's pair is below threshold. */
int oracle_pair_products(const oracle_beam *a, const oracle_beam *b, const uint32_t *hits,
                         int64_t n_hits, uint64_t seed, double *out);
/* the same CoM direction draw, exposed for tests: n[3] for (seed, i, j) */
void oracle_com_direction(uint64_t seed, uint32_t i, uint32_t j, double n[3]);

/* Depletion with chronological order (Sec. 2.2, Sec. 3.1, Fig. ChronOrder).
 * A photon annihilates when it collides, so a collision can only happen if
 * neither photon was used up by an earlier one; the collisions of a step are
 * therefore taken in time order.  With macro-photons of weight w (Sec. 2.2:
 * a swarm of w photons handled individually) a collision takes
 * delta = min(rem_i, rem_j) from both, the number of photon pairs the two
 * swarms can still form; with unit weights that is "the earliest hit of a
 * photon annihilates it".  Each beam then loses exactly the pairs made
 * (Eq. for n_I(t), n_II(t): n_I(0) - n(t)).
 *
 * oracle_hit_times: the closest-approach time t* (relative to t_k) of each
 * hit (i, j) of step k, by the same definition as oracle_pair_hit; returns
 * -1 if a listed pair is not a hit of that step (its t* is still written).
 *
 * oracle_deplete: the hits, each with its step, taken in (step, t*, i, j)
 * lexicographic order; rem_a[na] and rem_b[nb] hold what each photon still
 * holds (updated in place), delta[k] receives what hit k took.  Returns 0,
 * -1 for an index out of range (nothing changed), -2 out of memory. */
int oracle_hit_times(const oracle_beam *a, const oracle_beam *b, int64_t step, double dt,
                     double kappa, const uint32_t *hits, int64_t n_hits, double *tstar);
int oracle_deplete(int64_t n_hits, const int64_t *step, const double *tstar,
                   const uint32_t *hits, double *rem_a, int64_t na, double *rem_b, int64_t nb,
                   double *delta);

/* IP regime (Sec. 2.2): a macro-photon of integer weight w is a swarm of w
 * real photons with its energy and direction, "positioned as homogeneously as
 * possible over the volume of the MP".  The volume is an axis-aligned cube of
 * side h (one h per beam) centred on the MP; photon k of the swarm sits at
 * p0 + h u_k, u_k,d = frac(0.5 + k alpha_d) - 0.5 with alpha = (1/g, 1/g^2,
 * 1/g^3), g the real root > 1 of x^4 = x + 1 (Roberts' R_3 low-discrepancy
 * sequence), so u_0 = 0 and a weight-1 MP is its own photon.
 *
 * oracle_swarm_offset: u_k.
 * oracle_ip_bruteforce: every real-photon pair (photon k of MP i of a, photon
 * l of MP j of b) decided as oracle_pair_hit decides a pair of photons, with
 * p0 = MP position + h u; hits written as (i, k, j, l) uint32 quadruples in
 * lexicographic order, at most cap of them; *count is the true number.
 * Returns -1 if a weight is not an integer in [1, 2^32), -2 out of memory. */
void oracle_swarm_offset(uint64_t k, double u[3]);
int oracle_ip_bruteforce(const oracle_beam *a, const oracle_beam *b, double h_a, double h_b,
                         int64_t step, double dt, double kappa, uint32_t *hits, int64_t cap,
                         int64_t *count);

/* Statistical (ST) regime at a cut of the hierarchy (Sec. 2.2, Eq. rate,
 * Eq. reactivity).  Clouds are sets of photons: cloud_a[i] is the cloud
 * (0 .. n_cloud_a - 1) of photon i of a, likewise for b.  For each pair p of
 * clouds (pairs[2p] of a, pairs[2p + 1] of b) at step k: the 24 node-pair
 * features feat[24p .. 24p + 23] -- centre of B's swept box minus A's (3),
 * half-extents of A's (3) and B's (3) swept boxes, ln count of A and B, ln of
 * the weight sums, weighted mean of ln E of A and B, weighted spread of ln E
 * of A and B, weighted mean direction of A (3) and B (3), 1 - dbar_A . dbar_B
 * -- with the swept box of a cloud the AABB of its photons' segments over
 * the step, each widened by half the largest collision radius; and st[p], the
 * expected number of pairs of Eq. rate for the two clouds as uniform boxes
 * moving with their mean velocities (details in oracle.c).  Returns 0, -1
 * for a membership or pair out of range or an empty cloud, -2 out of memory. */
int oracle_cloud_pairs(const oracle_beam *a, const oracle_beam *b, int64_t step, double dt,
                       double kappa, const uint32_t *cloud_a, int64_t n_cloud_a,
                       const uint32_t *cloud_b, int64_t n_cloud_b, const uint32_t *pairs,
                       int64_t n_pairs, double *feat, double *st);
/* the exact integral over [0, T] of the overlap volume of box A ([la, ua]
 * moving with va) and box B ([lb, ub] moving with vb) */
double oracle_overlap_integral(const double la[3], const double ua[3], const double va[3],
                               const double lb[3], const double ub[3], const double vb[3],
                               double T);

/* All pairs.  Hits (i, j) written as uint32 pairs in lexicographic order,
 * at most cap of them; res->count is the true number. */
int oracle_bruteforce(const oracle_beam *a, const oracle_beam *b, int64_t step, double dt,
                      double kappa, uint32_t *hits, int64_t cap, oracle_result *res);
/* Paper's k-d hierarchy (median cuts, cycling axis) per beam over swept
 * boxes, dual depth-first traversal; same output contract as brute force.
 * nthreads > 1 splits the traversal over subtrees of beam A. */
int oracle_tree(const oracle_beam *a, const oracle_beam *b, int64_t step, double dt,
                double kappa, int leaf_size, int nthreads, uint32_t *hits, int64_t cap,
                oracle_result *res);

#ifdef __cplusplus
}
#endif
#endif
