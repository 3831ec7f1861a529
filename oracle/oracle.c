/*
 * oracle.c -- FP64 CPU oracle (TEST INFRASTRUCTURE ONLY; see oracle.h).
 *
 * Plain definitions, slow on purpose, no blocking or fusion beyond what the
 * definition states.  Build with:  gcc -O2 -ffp-contract=off -fPIC -shared
 * (contraction off so that every a*b+c is two rounded operations, on x86-64
 * and on aarch64 alike).
 *
 * What is computed, and where the paper defines it:
 *   - sigma(s): Eq. BWcross (Sec. 1), with beta = sqrt(1 - 1/s).  Evaluated
 *     in the algebraically equal form
 *        (pi/2) r_e^2 (1/s) [ (3 - b^4) ln((1+b)^2 s) - 2 b (2 - b^2) ],
 *     using (1+b)/(1-b) = (1+b)^2 / (1-b^2) = (1+b)^2 s, which avoids the
 *     1 - b cancellation near b -> 1.
 *   - s and the threshold s > 1: the definition below Eq. BWcross and
 *     Eq. eq.Cond (Sec. 1); sigma is zero at and below threshold.
 *   - the collision criterion (reading of the method stated in the design
 *     notes): time-synchronous closest approach of the two straight-line
 *     photons within the step, t* in [0, dt), hit iff d^2 < r^2 with
 *     r^2 = kappa sigma / pi (sigma in m^2 -> r in um via 1e12).
 *   - the hierarchy: the k-d tree of Sec. 2.1 (binary, each cut balances the
 *     particle counts, the cut axis cycles x, y, z), over boxes that include
 *     the distance travelled in the step (Sec. 2.1), tested pairwise with the
 *     axis-aligned overlap test Eq. CollDet, traversed depth first (Sec. 2.2).
 *     The tree only prunes; its hit set must equal brute force.
 *   - yield: weights multiply (Sec. 2.2, rate proportional to n_I n_II).
 *   - checksum: splitmix64 (Steele, Lea, Flood 2014; Vigna's published
 *     constants) of the packed pair, summed mod 2^64 and xor-ed.
 */
#include "oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* CODATA 2018; c exact */
#define O_C 0.299792458              /* um / fs */
#define O_RE 2.8179403262e-15        /* classical electron radius [m] */
#define O_MEC2 0.51099895000         /* electron rest energy [MeV] */
#define O_PI 3.14159265358979323846

/* ln 2 split: the high part has 32 significant bits so e * hi is exact */
#define O_LN2_HI 0.6931471803691238
#define O_LN2_LO 1.9082149292705877e-10
#define O_SQRT_HALF 0.70710678118654752440

double oracle_ln(double x) {
  if (x != x || x < 0.0) return NAN;
  if (x == 0.0) return -INFINITY;
  if (isinf(x)) return x;
  int e;
  double m = frexp(x, &e); /* x = m 2^e, m in [1/2, 1), exact */
  if (m < O_SQRT_HALF) {
    m = m * 2.0;
    e = e - 1;
  }
  /* m in [sqrt(1/2), sqrt(2)); f in (-0.1716, 0.1716) */
  double f = (m - 1.0) / (m + 1.0);
  double z = f * f;
  /* ln m = 2 atanh f = 2 f sum_k z^k / (2k + 1), k = 0..11; the first
   * omitted term is below 2^-60 relative */
  double p = 1.0 / 23.0;
  p = p * z + 1.0 / 21.0;
  p = p * z + 1.0 / 19.0;
  p = p * z + 1.0 / 17.0;
  p = p * z + 1.0 / 15.0;
  p = p * z + 1.0 / 13.0;
  p = p * z + 1.0 / 11.0;
  p = p * z + 1.0 / 9.0;
  p = p * z + 1.0 / 7.0;
  p = p * z + 1.0 / 5.0;
  p = p * z + 1.0 / 3.0;
  p = p * z + 1.0;
  double lnm = (2.0 * f) * p;
  double de = (double)e;
  return de * O_LN2_HI + (de * O_LN2_LO + lnm);
}

double oracle_sigma(double s) {
  if (!(s > 1.0)) return 0.0; /* threshold, Eq. eq.Cond */
  double inv = 1.0 / s;       /* = 1 - beta^2 */
  double b = sqrt((s - 1.0) / s);
  double b2 = b * b;
  double opb = 1.0 + b;
  double lg = oracle_ln((opb * opb) * s); /* ln((1+b)/(1-b)) */
  double br = (3.0 - b2 * b2) * lg - (2.0 * b) * (2.0 - b2);
  double pref = ((0.5 * O_PI) * O_RE) * O_RE;
  return (pref * inv) * br;
}

double oracle_s(double E1, double E2, double cos_phi) {
  return ((E1 * E2) * (1.0 - cos_phi)) / ((2.0 * O_MEC2) * O_MEC2);
}

double oracle_sigma_max(void) {
  /* golden-section search for the single maximum, which lies in (1.2, 4) */
  double lo = 1.2, hi = 4.0, g = 0.5 * (sqrt(5.0) - 1.0);
  double x1 = hi - g * (hi - lo), x2 = lo + g * (hi - lo);
  double f1 = oracle_sigma(x1), f2 = oracle_sigma(x2);
  for (int it = 0; it < 200; ++it) {
    if (f1 < f2) {
      lo = x1; x1 = x2; f1 = f2;
      x2 = lo + g * (hi - lo); f2 = oracle_sigma(x2);
    } else {
      hi = x2; x2 = x1; f2 = f1;
      x1 = hi - g * (hi - lo); f1 = oracle_sigma(x1);
    }
  }
  return f1 > f2 ? f1 : f2;
}

uint64_t oracle_splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* ---- the per-pair definition ------------------------------------------ */

/* position at t = step * dt, closed form p0 + (c t) d */
static inline void pos_at(const oracle_beam *bm, int64_t i, double ct, double P[3]) {
  P[0] = bm->px[i] + ct * bm->dx[i];
  P[1] = bm->py[i] + ct * bm->dy[i];
  P[2] = bm->pz[i] + ct * bm->dz[i];
}

/* out (optional): s, sigma, r2, tstar, d2, vv */
static int decide(const double Pi[3], const double di[3], double Ei, const double Pj[3],
                  const double dj[3], double Ej, double dt, double kappa, double *out) {
  double cs = di[0] * dj[0] + di[1] * dj[1] + di[2] * dj[2];
  double s = oracle_s(Ei, Ej, cs);
  if (out) { out[0] = s; out[1] = 0.0; out[2] = 0.0; out[3] = NAN; out[4] = NAN; out[5] = NAN; }
  if (!(s > 1.0)) return 0;
  double vx = O_C * (di[0] - dj[0]);
  double vy = O_C * (di[1] - dj[1]);
  double vz = O_C * (di[2] - dj[2]);
  double vv = vx * vx + vy * vy + vz * vz;
  if (out) out[5] = vv;
  if (vv == 0.0) return 0;
  double px = Pi[0] - Pj[0], py = Pi[1] - Pj[1], pz = Pi[2] - Pj[2];
  double pv = px * vx + py * vy + pz * vz;
  double ts = -pv / vv;
  if (out) out[3] = ts;
  else if (!(ts >= 0.0) || !(ts < dt)) return 0; /* same predicate, decided early */
  double qx = px + ts * vx, qy = py + ts * vy, qz = pz + ts * vz;
  double d2 = qx * qx + qy * qy + qz * qz;
  double sg = oracle_sigma(s);
  double r2 = ((1e12 * kappa) * sg) / O_PI;
  if (out) { out[1] = sg; out[2] = r2; out[4] = d2; }
  if (!(ts >= 0.0) || !(ts < dt)) return 0; /* half-open window [0, dt) */
  return d2 < r2;
}

int oracle_pair_detail(const oracle_beam *a, int64_t i, const oracle_beam *b, int64_t j,
                       int64_t step, double dt, double kappa, double out[6]) {
  double ct = O_C * ((double)step * dt);
  double Pi[3], Pj[3];
  pos_at(a, i, ct, Pi);
  pos_at(b, j, ct, Pj);
  double di[3] = {a->dx[i], a->dy[i], a->dz[i]};
  double dj[3] = {b->dx[j], b->dy[j], b->dz[j]};
  return decide(Pi, di, a->E[i], Pj, dj, b->E[j], dt, kappa, out);
}

int oracle_pair_hit(const oracle_beam *a, int64_t i, const oracle_beam *b, int64_t j,
                    int64_t step, double dt, double kappa) {
  return oracle_pair_detail(a, i, b, j, step, dt, kappa, NULL);
}

/* ---- result accumulation ---------------------------------------------- */

typedef struct {
  uint64_t *key;
  int64_t n, cap;
  int64_t tests, node_tests;
} hitvec;

static int hv_push(hitvec *h, uint64_t k) {
  if (h->n == h->cap) {
    int64_t nc = h->cap ? 2 * h->cap : 1024;
    uint64_t *p = (uint64_t *)realloc(h->key, (size_t)nc * sizeof(uint64_t));
    if (!p) return -1;
    h->key = p;
    h->cap = nc;
  }
  h->key[h->n++] = k;
  return 0;
}

static int cmp_u64(const void *x, const void *y) {
  uint64_t a = *(const uint64_t *)x, b = *(const uint64_t *)y;
  return a < b ? -1 : (a > b);
}

/* sort, write (i, j) pairs up to cap, fill the result in lexicographic order */
static void finish(hitvec *h, const oracle_beam *a, const oracle_beam *b, uint32_t *hits,
                   int64_t cap, oracle_result *res) {
  qsort(h->key, (size_t)h->n, sizeof(uint64_t), cmp_u64);
  res->count = h->n;
  res->weighted = 0.0;
  res->hsum = 0;
  res->hxor = 0;
  for (int64_t k = 0; k < h->n; ++k) {
    uint64_t key = h->key[k];
    uint32_t i = (uint32_t)(key >> 32), j = (uint32_t)(key & 0xffffffffu);
    double wi = a->w ? a->w[i] : 1.0, wj = b->w ? b->w[j] : 1.0;
    res->weighted += wi * wj;
    uint64_t hm = oracle_splitmix64(key);
    res->hsum += hm;
    res->hxor ^= hm;
    if (hits && k < cap) {
      hits[2 * k] = i;
      hits[2 * k + 1] = j;
    }
  }
  res->tests = h->tests;
  res->node_tests = h->node_tests;
}

/* ---- positions of one beam at one step -------------------------------- */

typedef struct {
  int64_t n;
  double *P;  /* 3n, xyz interleaved */
  double *d;  /* 3n */
  const double *E;
} posed;

static int pose(const oracle_beam *bm, int64_t step, double dt, posed *o) {
  o->n = bm->n;
  o->P = (double *)malloc((size_t)(bm->n > 0 ? bm->n : 1) * 3 * sizeof(double));
  o->d = (double *)malloc((size_t)(bm->n > 0 ? bm->n : 1) * 3 * sizeof(double));
  if (!o->P || !o->d) return -1;
  double ct = O_C * ((double)step * dt);
  for (int64_t i = 0; i < bm->n; ++i) {
    pos_at(bm, i, ct, o->P + 3 * i);
    o->d[3 * i] = bm->dx[i];
    o->d[3 * i + 1] = bm->dy[i];
    o->d[3 * i + 2] = bm->dz[i];
  }
  o->E = bm->E;
  return 0;
}

static void unpose(posed *o) {
  free(o->P);
  free(o->d);
}

int oracle_bruteforce(const oracle_beam *a, const oracle_beam *b, int64_t step, double dt,
                      double kappa, uint32_t *hits, int64_t cap, oracle_result *res) {
  posed A, B;
  if (pose(a, step, dt, &A) || pose(b, step, dt, &B)) return -1;
  hitvec h = {0};
  for (int64_t i = 0; i < a->n; ++i)
    for (int64_t j = 0; j < b->n; ++j)
      if (decide(A.P + 3 * i, A.d + 3 * i, A.E[i], B.P + 3 * j, B.d + 3 * j, B.E[j], dt, kappa,
                 NULL))
        if (hv_push(&h, ((uint64_t)i << 32) | (uint64_t)j)) return -1;
  h.tests = a->n * b->n;
  finish(&h, a, b, hits, cap, res);
  free(h.key);
  unpose(&A);
  unpose(&B);
  return 0;
}

/* ---- the k-d hierarchy (Sec. 2.1) -------------------------------------- */

typedef struct {
  double lo[3], hi[3];
  int64_t left, right; /* children, -1 for a leaf */
  int64_t first, count; /* leaf: particles idx[first .. first+count) */
} kdnode;

typedef struct {
  kdnode *node;
  int64_t nn;
  int64_t *idx;     /* particle array sorted by leaf affiliation */
  double *lo, *hi;  /* per-particle swept box, 3n each */
  double *cen;      /* per-particle box centre, 3n */
  int leaf_size;
} kdtree;

static void swap_i64(int64_t *a, int64_t *b) {
  int64_t t = *a;
  *a = *b;
  *b = t;
}

/* place the k-th smallest (by cen[axis], ties by index) at idx[k] */
static void select_kth(int64_t *idx, int64_t lo, int64_t hi, int64_t k, const double *cen,
                       int axis) {
  while (hi - lo > 1) {
    int64_t mid = lo + (hi - lo) / 2;
    /* median of three as pivot */
    int64_t c3[3] = {idx[lo], idx[mid], idx[hi - 1]};
    for (int x = 0; x < 3; ++x)
      for (int y = x + 1; y < 3; ++y) {
        double vx = cen[3 * c3[x] + axis], vy = cen[3 * c3[y] + axis];
        if (vy < vx || (vy == vx && c3[y] < c3[x])) swap_i64(&c3[x], &c3[y]);
      }
    int64_t piv = c3[1];
    double pv = cen[3 * piv + axis];
    /* three-way partition around (pv, piv) */
    int64_t l = lo, r = hi - 1, m = lo;
    while (m <= r) {
      int64_t q = idx[m];
      double v = cen[3 * q + axis];
      int less = v < pv || (v == pv && q < piv);
      int greater = v > pv || (v == pv && q > piv);
      if (less) {
        swap_i64(&idx[l], &idx[m]);
        ++l;
        ++m;
      } else if (greater) {
        swap_i64(&idx[m], &idx[r]);
        --r;
      } else {
        ++m;
      }
    }
    if (k < l)
      hi = l;
    else if (k > r)
      lo = r + 1;
    else
      return;
  }
}

static int64_t kd_build_rec(kdtree *t, int64_t first, int64_t count, int depth) {
  int64_t me = t->nn++;
  kdnode *nd = &t->node[me];
  for (int c = 0; c < 3; ++c) {
    nd->lo[c] = INFINITY;
    nd->hi[c] = -INFINITY;
  }
  for (int64_t k = first; k < first + count; ++k) {
    int64_t p = t->idx[k];
    for (int c = 0; c < 3; ++c) {
      if (t->lo[3 * p + c] < nd->lo[c]) nd->lo[c] = t->lo[3 * p + c];
      if (t->hi[3 * p + c] > nd->hi[c]) nd->hi[c] = t->hi[3 * p + c];
    }
  }
  nd->first = first;
  nd->count = count;
  if (count <= t->leaf_size) {
    nd->left = nd->right = -1;
    return me;
  }
  int axis = depth % 3; /* the cut direction cycles after each cut */
  int64_t half = count / 2; /* balance the particle counts */
  select_kth(t->idx, first, first + count, first + half, t->cen, axis);
  int64_t l = kd_build_rec(t, first, half, depth + 1);
  int64_t r = kd_build_rec(t, first + half, count - half, depth + 1);
  t->node[me].left = l;
  t->node[me].right = r;
  return me;
}

static int kd_build(kdtree *t, const posed *p, double L, double h, int leaf_size) {
  int64_t n = p->n;
  size_t n1 = (size_t)(n > 0 ? n : 1);
  t->idx = (int64_t *)malloc(n1 * sizeof(int64_t));
  t->lo = (double *)malloc(n1 * 3 * sizeof(double));
  t->hi = (double *)malloc(n1 * 3 * sizeof(double));
  t->cen = (double *)malloc(n1 * 3 * sizeof(double));
  t->node = (kdnode *)malloc(n1 * 2 * sizeof(kdnode));
  t->leaf_size = leaf_size < 1 ? 1 : leaf_size;
  t->nn = 0;
  if (!t->idx || !t->lo || !t->hi || !t->cen || !t->node) return -1;
  for (int64_t i = 0; i < n; ++i) {
    t->idx[i] = i;
    for (int c = 0; c < 3; ++c) {
      double s0 = p->P[3 * i + c];
      double s1 = s0 + L * p->d[3 * i + c]; /* end of the step's travel */
      double mn = s0 < s1 ? s0 : s1, mx = s0 < s1 ? s1 : s0;
      t->lo[3 * i + c] = mn - h;
      t->hi[3 * i + c] = mx + h;
      t->cen[3 * i + c] = 0.5 * (mn + mx);
    }
  }
  if (n > 0) kd_build_rec(t, 0, n, 0);
  return 0;
}

static void kd_free(kdtree *t) {
  free(t->idx);
  free(t->lo);
  free(t->hi);
  free(t->cen);
  free(t->node);
}

/* Eq. CollDet with closed boxes (the symmetric six comparisons) */
static inline int overlap(const kdnode *x, const kdnode *y) {
  return x->lo[0] <= y->hi[0] && y->lo[0] <= x->hi[0] && x->lo[1] <= y->hi[1] &&
         y->lo[1] <= x->hi[1] && x->lo[2] <= y->hi[2] && y->lo[2] <= x->hi[2];
}

typedef struct {
  const kdtree *ta, *tb;
  const posed *A, *B;
  double dt, kappa;
  hitvec h;
  int err;
} trav;

static void visit(trav *w, int64_t ia, int64_t ib) {
  const kdnode *na = &w->ta->node[ia], *nb = &w->tb->node[ib];
  w->h.node_tests++;
  if (!overlap(na, nb)) return;
  int la = na->left < 0, lb = nb->left < 0;
  if (la && lb) {
    for (int64_t x = na->first; x < na->first + na->count; ++x) {
      int64_t i = w->ta->idx[x];
      for (int64_t y = nb->first; y < nb->first + nb->count; ++y) {
        int64_t j = w->tb->idx[y];
        w->h.tests++;
        if (decide(w->A->P + 3 * i, w->A->d + 3 * i, w->A->E[i], w->B->P + 3 * j,
                   w->B->d + 3 * j, w->B->E[j], w->dt, w->kappa, NULL))
          if (hv_push(&w->h, ((uint64_t)i << 32) | (uint64_t)j)) w->err = 1;
      }
    }
    return;
  }
  /* descend the side that is not a leaf; of two inner nodes the larger */
  if (la || (!lb && nb->count > na->count)) {
    visit(w, ia, nb->left);
    visit(w, ia, nb->right);
  } else {
    visit(w, na->left, ib);
    visit(w, na->right, ib);
  }
}

typedef struct {
  trav *w;
  const int64_t *roots;
  int64_t nroots;
  int tid, nthreads;
} job;

static void *run_job(void *arg) {
  job *j = (job *)arg;
  for (int64_t k = j->tid; k < j->nroots; k += j->nthreads) visit(j->w, j->roots[k], 0);
  return NULL;
}

int oracle_tree(const oracle_beam *a, const oracle_beam *b, int64_t step, double dt,
                double kappa, int leaf_size, int nthreads, uint32_t *hits, int64_t cap,
                oracle_result *res) {
  posed A, B;
  if (pose(a, step, dt, &A) || pose(b, step, dt, &B)) return -1;
  /* inflate each swept box by half the largest collision radius, with a
   * relative and an absolute margin far above FP64 rounding */
  double smax = oracle_sigma_max() * (1.0 + 1e-6);
  double rmax = sqrt(((1e12 * kappa) * smax) / O_PI) * (1.0 + 1e-6);
  double h = 0.5 * rmax + 1e-9;
  double L = O_C * dt;
  kdtree ta, tb;
  if (kd_build(&ta, &A, L, h, leaf_size) || kd_build(&tb, &B, L, h, leaf_size)) return -1;
  hitvec all = {0};
  int err = 0;
  if (a->n > 0 && b->n > 0) {
    if (nthreads <= 1) {
      trav w = {&ta, &tb, &A, &B, dt, kappa, {0}, 0};
      visit(&w, 0, 0);
      all = w.h;
      err = w.err;
    } else {
      /* subtrees of A at the first level with >= 8 nthreads nodes */
      int64_t cap_r = 16 * (int64_t)nthreads + 2, nr = 1;
      int64_t *roots = (int64_t *)malloc((size_t)cap_r * 2 * sizeof(int64_t));
      int64_t *next = roots + cap_r;
      roots[0] = 0;
      while (nr < 8 * nthreads) {
        int64_t nn = 0, grew = 0;
        for (int64_t k = 0; k < nr; ++k) {
          const kdnode *nd = &ta.node[roots[k]];
          if (nd->left >= 0 && nn + 2 <= cap_r) {
            next[nn++] = nd->left;
            next[nn++] = nd->right;
            grew = 1;
          } else {
            next[nn++] = roots[k];
          }
        }
        memcpy(roots, next, (size_t)nn * sizeof(int64_t));
        nr = nn;
        if (!grew || nn + 2 > cap_r) break;
      }
      trav *ws = (trav *)calloc((size_t)nthreads, sizeof(trav));
      job *js = (job *)calloc((size_t)nthreads, sizeof(job));
      pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
      for (int t = 0; t < nthreads; ++t) {
        ws[t] = (trav){&ta, &tb, &A, &B, dt, kappa, {0}, 0};
        js[t] = (job){&ws[t], roots, nr, t, nthreads};
        pthread_create(&th[t], NULL, run_job, &js[t]);
      }
      for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
      for (int t = 0; t < nthreads; ++t) {
        for (int64_t k = 0; k < ws[t].h.n; ++k)
          if (hv_push(&all, ws[t].h.key[k])) err = 1;
        all.tests += ws[t].h.tests;
        all.node_tests += ws[t].h.node_tests;
        err |= ws[t].err;
        free(ws[t].h.key);
      }
      free(ws);
      free(js);
      free(th);
      free(roots);
    }
  }
  finish(&all, a, b, hits, cap, res);
  free(all.key);
  kd_free(&ta);
  kd_free(&tb);
  unpose(&A);
  unpose(&B);
  return err ? -1 : 0;
}

/* ---- pair products (Sec. 1: Eq. pTotal, Eq. Lorentz) ----------------------- */

/* uniform double in [0, 1) from the top 53 bits of a splitmix64 output */
static double unit_draw(uint64_t key, uint64_t t) {
  return (double)(oracle_splitmix64(key + t) >> 11) * (1.0 / 9007199254740992.0);
}

/* Marsaglia (1972): x1, x2 uniform in (-1, 1) until S = x1^2 + x2^2 is in
 * (0, 1); then n = (2 x1 sqrt(1 - S), 2 x2 sqrt(1 - S), 1 - 2 S) is uniform on
 * the unit sphere.  At most 64 tries (then n = z; never reached in practice). */
void oracle_com_direction(uint64_t seed, uint32_t i, uint32_t j, double n[3]) {
  const uint64_t key = seed ^ (((uint64_t)i << 32) | (uint64_t)j);
  for (uint64_t t = 0; t < 128; t += 2) {
    const double x1 = 2.0 * unit_draw(key, t) - 1.0;
    const double x2 = 2.0 * unit_draw(key, t + 1) - 1.0;
    const double S = x1 * x1 + x2 * x2;
    if (S < 1.0 && S > 0.0) {
      const double r = sqrt(1.0 - S);
      n[0] = 2.0 * x1 * r;
      n[1] = 2.0 * x2 * r;
      n[2] = 1.0 - 2.0 * S;
      return;
    }
  }
  n[0] = 0.0;
  n[1] = 0.0;
  n[2] = 1.0;
}

/* Lorentz boost of the four-momentum (e, q) by velocity beta (|beta| < 1,
 * gamma given): e' = gamma (e + beta.q), q' = q + beta (gamma^2/(gamma+1)
 * beta.q + gamma e) */
static void boost(const double beta[3], double gamma, double e, const double q[3],
                  double out[4]) {
  const double bq = beta[0] * q[0] + beta[1] * q[1] + beta[2] * q[2];
  const double k = gamma * gamma / (gamma + 1.0) * bq + gamma * e;
  out[0] = gamma * (e + bq);
  out[1] = q[0] + beta[0] * k;
  out[2] = q[1] + beta[1] * k;
  out[3] = q[2] + beta[2] * k;
}

int oracle_pair_products(const oracle_beam *a, const oracle_beam *b, const uint32_t *hits,
                         int64_t n_hits, uint64_t seed, double *out) {
  int rc = 0;
  for (int64_t k = 0; k < n_hits; ++k) {
    const uint32_t i = hits[2 * k], j = hits[2 * k + 1];
    const double E1 = a->E[i], E2 = b->E[j];
    const double d1[3] = {a->dx[i], a->dy[i], a->dz[i]}, d2[3] = {b->dx[j], b->dy[j], b->dz[j]};
    const double E = E1 + E2;
    const double P[3] = {E1 * d1[0] + E2 * d2[0], E1 * d1[1] + E2 * d2[1],
                         E1 * d1[2] + E2 * d2[2]};
    const double cs = d1[0] * d2[0] + d1[1] * d2[1] + d1[2] * d2[2];
    const double M2 = 2.0 * (E1 * E2) * (1.0 - cs); /* invariant mass squared */
    const double m = O_MEC2;
    double *o = out + 8 * k;
    if (!(M2 > 4.0 * m * m)) { /* below threshold: no pair */
      for (int q = 0; q < 8; ++q) o[q] = 0.0;
      rc = -1;
      continue;
    }
    const double M = sqrt(M2);
    const double ep = 0.5 * M;                 /* CoM energy of each particle */
    const double pp = sqrt(0.25 * M2 - m * m); /* CoM momentum (Eq. pTotal) */
    double n[3];
    oracle_com_direction(seed, i, j, n);
    const double beta[3] = {P[0] / E, P[1] / E, P[2] / E};
    const double gamma = E / M;
    const double qe[3] = {pp * n[0], pp * n[1], pp * n[2]};
    const double qp[3] = {-qe[0], -qe[1], -qe[2]};
    boost(beta, gamma, ep, qe, o);
    boost(beta, gamma, ep, qp, o + 4);
  }
  return rc;
}

/* ---- depletion with chronological order (Sec. 2.2, Sec. 3.1) ----------- */

int oracle_hit_times(const oracle_beam *a, const oracle_beam *b, int64_t step, double dt,
                     double kappa, const uint32_t *hits, int64_t n_hits, double *tstar) {
  int rc = 0;
  for (int64_t k = 0; k < n_hits; ++k) {
    double out[6];
    const int hit = oracle_pair_detail(a, hits[2 * k], b, hits[2 * k + 1], step, dt, kappa, out);
    tstar[k] = out[3];
    if (!hit) rc = -1;
  }
  return rc;
}

typedef struct {
  int64_t step;
  double t;
  uint32_t i, j;
  int64_t k; /* position in the caller's list */
} dep_item;

/* (step, t*, i, j) lexicographic; equal t* (also -0 and +0) fall to i, then j */
static int cmp_dep(const void *x, const void *y) {
  const dep_item *p = (const dep_item *)x, *q = (const dep_item *)y;
  if (p->step != q->step) return p->step < q->step ? -1 : 1;
  if (p->t < q->t) return -1;
  if (q->t < p->t) return 1;
  if (p->i != q->i) return p->i < q->i ? -1 : 1;
  if (p->j != q->j) return p->j < q->j ? -1 : 1;
  return 0;
}

int oracle_deplete(int64_t n_hits, const int64_t *step, const double *tstar,
                   const uint32_t *hits, double *rem_a, int64_t na, double *rem_b, int64_t nb,
                   double *delta) {
  dep_item *it = (dep_item *)malloc(sizeof(dep_item) * (size_t)(n_hits > 0 ? n_hits : 1));
  if (!it) return -2;
  for (int64_t k = 0; k < n_hits; ++k) {
    it[k].step = step[k];
    it[k].t = tstar[k];
    it[k].i = hits[2 * k];
    it[k].j = hits[2 * k + 1];
    it[k].k = k;
    if ((int64_t)it[k].i >= na || (int64_t)it[k].j >= nb) {
      free(it);
      return -1;
    }
  }
  qsort(it, (size_t)n_hits, sizeof(dep_item), cmp_dep);
  /* in time order: the collision takes what both photons still hold */
  for (int64_t q = 0; q < n_hits; ++q) {
    const uint32_t i = it[q].i, j = it[q].j;
    const double d = rem_a[i] < rem_b[j] ? rem_a[i] : rem_b[j];
    rem_a[i] = rem_a[i] - d;
    rem_b[j] = rem_b[j] - d;
    delta[it[q].k] = d;
  }
  free(it);
  return 0;
}

/* ---- IP regime: macro-photons split into swarms of real photons (Sec. 2.2) */

/* 1/g, 1/g^2, 1/g^3 with g the real root > 1 of x^4 = x + 1 (Roberts' R_3
 * low-discrepancy sequence), as the nearest doubles */
static const double O_R3[3] = {0.81917251339616448, 0.67104360670378926, 0.5497004779019703};

void oracle_swarm_offset(uint64_t k, double u[3]) {
  for (int d = 0; d < 3; ++d) {
    const double x = 0.5 + (double)k * O_R3[d];
    u[d] = (x - floor(x)) - 0.5;
  }
}

static int weight_ok(double w) { return w >= 1.0 && w < 4294967296.0 && w == floor(w); }

typedef struct {
  uint32_t i, k, j, l;
} ip_hit;

static int cmp_ip(const void *x, const void *y) {
  const ip_hit *p = (const ip_hit *)x, *q = (const ip_hit *)y;
  if (p->i != q->i) return p->i < q->i ? -1 : 1;
  if (p->k != q->k) return p->k < q->k ? -1 : 1;
  if (p->j != q->j) return p->j < q->j ? -1 : 1;
  if (p->l != q->l) return p->l < q->l ? -1 : 1;
  return 0;
}

int oracle_ip_bruteforce(const oracle_beam *a, const oracle_beam *b, double h_a, double h_b,
                         int64_t step, double dt, double kappa, uint32_t *hits, int64_t cap,
                         int64_t *count) {
  for (int64_t i = 0; i < a->n; ++i)
    if (!weight_ok(a->w[i])) return -1;
  for (int64_t j = 0; j < b->n; ++j)
    if (!weight_ok(b->w[j])) return -1;
  const double ct = O_C * ((double)step * dt);
  ip_hit *hv = NULL;
  int64_t n = 0, hcap = 0;
  for (int64_t i = 0; i < a->n; ++i) {
    const double di[3] = {a->dx[i], a->dy[i], a->dz[i]};
    for (int64_t j = 0; j < b->n; ++j) {
      const double dj[3] = {b->dx[j], b->dy[j], b->dz[j]};
      /* every photon of a swarm has its MP's energy and direction: the same s */
      const double cs = di[0] * dj[0] + di[1] * dj[1] + di[2] * dj[2];
      if (!(oracle_s(a->E[i], b->E[j], cs) > 1.0)) continue;
      for (uint64_t k = 0; k < (uint64_t)a->w[i]; ++k) {
        double u[3], Pi[3];
        oracle_swarm_offset(k, u);
        Pi[0] = (a->px[i] + h_a * u[0]) + ct * di[0];
        Pi[1] = (a->py[i] + h_a * u[1]) + ct * di[1];
        Pi[2] = (a->pz[i] + h_a * u[2]) + ct * di[2];
        for (uint64_t l = 0; l < (uint64_t)b->w[j]; ++l) {
          double v[3], Pj[3];
          oracle_swarm_offset(l, v);
          Pj[0] = (b->px[j] + h_b * v[0]) + ct * dj[0];
          Pj[1] = (b->py[j] + h_b * v[1]) + ct * dj[1];
          Pj[2] = (b->pz[j] + h_b * v[2]) + ct * dj[2];
          if (!decide(Pi, di, a->E[i], Pj, dj, b->E[j], dt, kappa, NULL)) continue;
          if (n == hcap) {
            int64_t nc = hcap ? 2 * hcap : 1024;
            ip_hit *p = (ip_hit *)realloc(hv, (size_t)nc * sizeof(ip_hit));
            if (!p) {
              free(hv);
              return -2;
            }
            hv = p;
            hcap = nc;
          }
          hv[n].i = (uint32_t)i;
          hv[n].k = (uint32_t)k;
          hv[n].j = (uint32_t)j;
          hv[n].l = (uint32_t)l;
          ++n;
        }
      }
    }
  }
  qsort(hv, (size_t)n, sizeof(ip_hit), cmp_ip);
  for (int64_t q = 0; q < n && q < cap; ++q) {
    hits[4 * q] = hv[q].i;
    hits[4 * q + 1] = hv[q].k;
    hits[4 * q + 2] = hv[q].j;
    hits[4 * q + 3] = hv[q].l;
  }
  *count = n;
  free(hv);
  return 0;
}

/* ------------------------------------------------------------------------
 * Statistical (ST) regime at a cut of the hierarchy (Sec. 2.2, Eq. rate and
 * Eq. reactivity).  A cloud is a set of photons (a node of the cut, given as
 * a photon -> cloud membership).  Per cloud X at step k:
 *   W_X = sum w;  mean and spread of ln E with weights w;  mean direction
 *   dbar_X = sum w d / W_X (not renormalised);  swept box S_X = the AABB of
 *   the photons' segments from P(t_k) to P(t_k) + c dt d, each widened by
 *   h = r_max / 2 (half the largest collision radius) on every side.
 * The cloud is read as a box of uniform density moving rigidly with c dbar:
 * its box at t_k is S_X with the step's travel c dt dbar taken off (per axis
 * [lo - min(0, D), hi - max(0, D)], D = c dt dbar_a), volume V_X, so that the
 * box swept by it over the step is S_X again.  Eq. rate, n_I n_II <sigma v>
 * per unit volume with n = W / V, integrated over the clouds' overlap and the
 * step, gives the expected number of pairs
 *   N = W_A W_B (1e12 kappa sigma(sbar)) |v_rel| int_0^dt V_ov(t) dt / (V_A V_B)
 * with the collision area pi r^2 = 1e12 kappa sigma [um^2] of the collision
 * criterion, the reactivity taken at the clouds' mean momenta: sbar from the
 * geometric-mean energies exp(<ln E>) and 1 - dbar_A . dbar_B, and
 * v_rel = c |dbar_A - dbar_B| the speed at which the criterion's cylinder
 * sweeps (the printed <sigma v> = 2 pi sigma c is garbled; for head-on clouds
 * c(1 - cos) and |v_A - v_B| are both 2c).  V_ov(t) is a product of three
 * piecewise-linear overlap lengths, so its integral is taken exactly: split
 * [0, dt] where an overlap length changes form, Simpson's rule on each piece
 * (exact for the cubic there).
 * ------------------------------------------------------------------------ */

typedef struct {
  int64_t count;
  double W, wl, wl2, wd[3];
  double lo[3], hi[3];
} o_cloud;

static int o_clouds(const oracle_beam *bm, int64_t step, double dt, double kappa,
                    const uint32_t *cloud, int64_t n_cloud, o_cloud *out) {
  const double h = 0.5 * 1e6 * sqrt(kappa * oracle_sigma_max() / O_PI);
  const double ct = O_C * ((double)step * dt), L = O_C * dt;
  for (int64_t c = 0; c < n_cloud; ++c) {
    memset(&out[c], 0, sizeof(o_cloud));
    for (int a = 0; a < 3; ++a) {
      out[c].lo[a] = INFINITY;
      out[c].hi[a] = -INFINITY;
    }
  }
  for (int64_t i = 0; i < bm->n; ++i) {
    const uint32_t c = cloud[i];
    if ((int64_t)c >= n_cloud) return -1;
    o_cloud *q = &out[c];
    const double w = bm->w ? bm->w[i] : 1.0;
    const double le = log(bm->E[i]);
    const double p0[3] = {bm->px[i], bm->py[i], bm->pz[i]};
    const double d[3] = {bm->dx[i], bm->dy[i], bm->dz[i]};
    q->count += 1;
    q->W += w;
    q->wl += w * le;
    q->wl2 += w * le * le;
    for (int a = 0; a < 3; ++a) {
      q->wd[a] += w * d[a];
      const double P = p0[a] + ct * d[a];   /* position at t_k */
      const double Q = P + L * d[a];        /* and at t_k + dt */
      const double lo = (P < Q ? P : Q) - h, hi = (P < Q ? Q : P) + h;
      if (lo < q->lo[a]) q->lo[a] = lo;
      if (hi > q->hi[a]) q->hi[a] = hi;
    }
  }
  return 0;
}

/* overlap length at time t of [la + va t, ua + va t] and [lb + vb t, ub + vb t] */
static double o_olap(double la, double ua, double va, double lb, double ub, double vb, double t) {
  const double hi = fmin(ua + va * t, ub + vb * t), lo = fmax(la + va * t, lb + vb * t);
  return hi > lo ? hi - lo : 0.0;
}

static double o_vol_ov(const double la[3], const double ua[3], const double va[3],
                       const double lb[3], const double ub[3], const double vb[3], double t) {
  double v = 1.0;
  for (int a = 0; a < 3; ++a) v *= o_olap(la[a], ua[a], va[a], lb[a], ub[a], vb[a], t);
  return v;
}

static int o_cmp_double(const void *x, const void *y) {
  const double a = *(const double *)x, b = *(const double *)y;
  return (a > b) - (a < b);
}

/* exact integral over [0, T] of the overlap volume of two moving boxes */
double oracle_overlap_integral(const double la[3], const double ua[3], const double va[3],
                               const double lb[3], const double ub[3], const double vb[3],
                               double T) {
  double br[14];
  int nb = 0;
  br[nb++] = 0.0;
  br[nb++] = T;
  for (int a = 0; a < 3; ++a) {
    const double w = vb[a] - va[a];
    if (w == 0.0) continue;
    /* times where an end of B passes an end of A */
    const double cand[4] = {(ua[a] - ub[a]) / w, (la[a] - lb[a]) / w, (ua[a] - lb[a]) / w,
                            (la[a] - ub[a]) / w};
    for (int q = 0; q < 4; ++q)
      if (cand[q] > 0.0 && cand[q] < T) br[nb++] = cand[q];
  }
  qsort(br, (size_t)nb, sizeof(double), o_cmp_double);
  double I = 0.0;
  for (int q = 0; q + 1 < nb; ++q) {
    const double t0 = br[q], t1 = br[q + 1];
    if (!(t1 > t0)) continue;
    const double f0 = o_vol_ov(la, ua, va, lb, ub, vb, t0);
    const double fm = o_vol_ov(la, ua, va, lb, ub, vb, 0.5 * (t0 + t1));
    const double f1 = o_vol_ov(la, ua, va, lb, ub, vb, t1);
    I += (t1 - t0) * (f0 + 4.0 * fm + f1) / 6.0;
  }
  return I;
}

int oracle_cloud_pairs(const oracle_beam *a, const oracle_beam *b, int64_t step, double dt,
                       double kappa, const uint32_t *cloud_a, int64_t n_cloud_a,
                       const uint32_t *cloud_b, int64_t n_cloud_b, const uint32_t *pairs,
                       int64_t n_pairs, double *feat, double *st) {
  o_cloud *ca = (o_cloud *)malloc(sizeof(o_cloud) * (size_t)(n_cloud_a > 0 ? n_cloud_a : 1));
  o_cloud *cb = (o_cloud *)malloc(sizeof(o_cloud) * (size_t)(n_cloud_b > 0 ? n_cloud_b : 1));
  if (!ca || !cb) {
    free(ca);
    free(cb);
    return -2;
  }
  int rc = 0;
  if (o_clouds(a, step, dt, kappa, cloud_a, n_cloud_a, ca) ||
      o_clouds(b, step, dt, kappa, cloud_b, n_cloud_b, cb))
    rc = -1;
  const double L = O_C * dt;
  for (int64_t p = 0; p < n_pairs && !rc; ++p) {
    const uint32_t ia = pairs[2 * p], ib = pairs[2 * p + 1];
    if ((int64_t)ia >= n_cloud_a || (int64_t)ib >= n_cloud_b || ca[ia].count == 0 ||
        cb[ib].count == 0) {
      rc = -1;
      break;
    }
    const o_cloud *A = &ca[ia], *B = &cb[ib];
    double *f = feat + 24 * p;
    for (int q = 0; q < 3; ++q) {
      f[q] = 0.5 * (B->lo[q] + B->hi[q]) - 0.5 * (A->lo[q] + A->hi[q]);
      f[3 + q] = 0.5 * (A->hi[q] - A->lo[q]);
      f[6 + q] = 0.5 * (B->hi[q] - B->lo[q]);
    }
    f[9] = log((double)A->count);
    f[10] = log((double)B->count);
    f[11] = log(A->W);
    f[12] = log(B->W);
    const double mla = A->wl / A->W, mlb = B->wl / B->W;
    f[13] = mla;
    f[14] = mlb;
    f[15] = sqrt(fmax(A->wl2 / A->W - mla * mla, 0.0));
    f[16] = sqrt(fmax(B->wl2 / B->W - mlb * mlb, 0.0));
    double da[3], db[3];
    for (int q = 0; q < 3; ++q) {
      da[q] = A->wd[q] / A->W;
      db[q] = B->wd[q] / B->W;
      f[17 + q] = da[q];
      f[20 + q] = db[q];
    }
    const double omc = 1.0 - (da[0] * db[0] + da[1] * db[1] + da[2] * db[2]);
    f[23] = omc;
    /* the ST rate */
    const double sbar = exp(mla + mlb) * omc / (2.0 * O_MEC2 * O_MEC2);
    const double sig = oracle_sigma(sbar);
    double la[3], ua[3], va[3], lb[3], ub[3], vb[3], VA = 1.0, VB = 1.0, dv2 = 0.0;
    for (int q = 0; q < 3; ++q) {
      const double DA = L * da[q], DB = L * db[q];
      la[q] = A->lo[q] - fmin(0.0, DA);
      ua[q] = A->hi[q] - fmax(0.0, DA);
      lb[q] = B->lo[q] - fmin(0.0, DB);
      ub[q] = B->hi[q] - fmax(0.0, DB);
      va[q] = O_C * da[q];
      vb[q] = O_C * db[q];
      VA *= ua[q] - la[q];
      VB *= ub[q] - lb[q];
      dv2 += (va[q] - vb[q]) * (va[q] - vb[q]);
    }
    const double I = oracle_overlap_integral(la, ua, va, lb, ub, vb, dt);
    st[p] = (sig > 0.0 && I > 0.0)
                ? A->W * B->W * (1e12 * kappa * sig) * sqrt(dv2) * I / (VA * VB)
                : 0.0;
  }
  free(ca);
  free(cb);
  return rc;
}
