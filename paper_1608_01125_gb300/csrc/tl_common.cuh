// tl_common.cuh -- types shared by the library's CUDA translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define TL_C 0.299792458            /* um / fs, exact */
#define TL_RE 2.8179403262e-15      /* classical electron radius [m], CODATA 2018 */
#define TL_MEC2 0.51099895000       /* electron rest energy [MeV], CODATA 2018 */
#define TL_PI 3.14159265358979323846

// most warps per block of the traversal kernel (its launch bounds)
#define TL_TRAV_MAX_WARPS 8

// keys per radix-sort tile (threads 256 x items 8); the look-back status
// array holds 256 words per tile
#define TL_SORT_TILE 2048

// Child / stack references.  Bit 31 clear: an inner node index.  Bit 31 set:
// in a node's child slot, FLAG | first photon of a leaf bucket; on a stack,
// FLAG | (parent << 1 | slot) naming the bucket through its parent's slot.
#define TL_FLAG 0x80000000u
#define TL_NONE 0xFFFFFFFFu

// One inner node of a hierarchy: the boxes of both children (box 0 in
// b0.xyz/b0.w,b1.xy; box 1 in b1.zw,b2), child references and the photon
// count under each child.  64 bytes, one line pair per pop.
struct __align__(16) TLNode {
  float4 b0;  // lo0.x lo0.y lo0.z hi0.x
  float4 b1;  // hi0.y hi0.z lo1.x lo1.y
  float4 b2;  // lo1.z hi1.x hi1.y hi1.z
  int4 c;     // child0 child1 cnt0 cnt1
};

struct TLBox {
  float lx, ly, lz, hx, hy, hz;
};

__device__ __forceinline__ TLBox tl_child_box(const TLNode &n, int slot) {
  TLBox b;
  if (slot == 0) {
    b.lx = n.b0.x; b.ly = n.b0.y; b.lz = n.b0.z; b.hx = n.b0.w; b.hy = n.b1.x; b.hz = n.b1.y;
  } else {
    b.lx = n.b1.z; b.ly = n.b1.w; b.lz = n.b2.x; b.hx = n.b2.y; b.hy = n.b2.z; b.hz = n.b2.w;
  }
  return b;
}

// Eq. CollDet with closed boxes: the symmetric six comparisons.
__device__ __forceinline__ bool tl_overlap(const TLBox &a, const TLBox &b) {
  return a.lx <= b.hx && b.lx <= a.hx && a.ly <= b.hy && b.ly <= a.hy && a.lz <= b.hz &&
         b.lz <= a.hz;
}

// splitmix64 (Steele, Lea, Flood 2014; Vigna's published constants): the
// hit-set checksum and the counter-based stream of the pair products
__device__ __forceinline__ unsigned long long smix64(unsigned long long x) {
  unsigned long long z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// device status bits (OR-ed into TLCounters::status)
enum {
  TL_ST_HIT_OVF = 1,
  TL_ST_BAND_OVF = 2,
  TL_ST_SPILL_OVF = 4,  // the traversal queue overflowed (or a slot was not free)
  TL_ST_FRONT_OVF = 8,
  TL_ST_TIMEOUT = 16,
  TL_ST_LEAFQ = 32,    // the leaf-pair list overflowed
  TL_ST_PRIV_OVF = 64,  // a traversal warp's private spill area overflowed
  TL_ST_BADTREE = 128   // the refit met a node reference out of range (an internal error)
};

// Per-step device counters; zeroed by the step's init kernel.
struct TLCounters {
  unsigned long long hits;         // colliding pairs found (may exceed capacity)
  unsigned long long band;         // FP32 band pairs queued for FP64
  unsigned long long q_tail;       // traversal queue: chunks reserved (items handed on)
  unsigned long long narrow_tests; // photon pairs tested
  unsigned long long node_tests;   // box pair tests
  unsigned long long leaf_pairs;   // overlapping bucket pairs
  unsigned int counts[32];         // frontier size after each expansion level
  unsigned int frozen;             // frontier expansion finished
  unsigned int final_level;        // level whose frontier the traversal reads
  unsigned int widen_done;         // blocks finished in the frontier's widening level
  unsigned int status;             // TL_ST_* bits
  unsigned int reduce_done;        // blocks finished in the yield reduction
  unsigned int hungry;             // traversal warps waiting for a handed-on chunk
  unsigned long long q_head;       // traversal items taken (the frontier's, then the queue's)
  unsigned long long q_done;       // traversal items finished
  // results of the yield reduction for this step
  unsigned long long count;
  double weighted;
  unsigned long long hsum, hxor;
  // a step done in parts (slices of its frontier): the leaf-pair count at
  // the start of the current part, and the largest part's leaf pairs
  unsigned long long leaf_base;
  unsigned long long max_part_leaves;
};

// Totals of a captured multi-step run (accumulated on the device, step by
// step, in step order).
struct TLRunAcc {
  unsigned long long count;
  double weighted;
  unsigned long long hsum, hxor;
  unsigned long long narrow_tests, node_tests, leaf_pairs, band;
  unsigned long long max_hits, max_band, max_handed;  // largest per-step list and queue sizes
  unsigned long long max_leaves;
};

// FP64 input beam on the device.
struct TLBeam {
  const double *px, *py, *pz, *dx, *dy, *dz, *E, *w;
  int64_t n;
};

// Per-beam hierarchy produced by the build.
struct TLTree {
  const float4 *pos;    // sorted: x y z E (FP32)
  const float4 *dir;    // sorted: dx dy dz, w = input index (int bits)
  const TLNode *nodes;  // n - 1 inner nodes, then the super root at index n - 1
  uint32_t super;       // index of the super root (max(n - 1, 0))
  int64_t n;
};

// Conservative constants of the FP32 narrow phase (see tl_narrow.cuh).
// Bins of the invariant s for the narrow phase's sure-miss radius: bin 0
// holds s < 1 (below threshold); bin 1 + 8 e + k holds s in
// [2^e (1 + k/8), 2^e (1 + (k+1)/8)) for e = 0..23; the last bin also holds
// every larger s.  A bin's index is read off the FP32 bits of s exactly.
constexpr int TL_SBIN_OCT = 8;
constexpr int TL_SBIN_EMAX = 24;
constexpr int TL_SBINS = 1 + TL_SBIN_OCT * TL_SBIN_EMAX;

__device__ __forceinline__ int tl_sbin(float s) {
  if (s < 1.0f) return 0;
  const unsigned b = __float_as_uint(s);
  const int i = 1 + ((int)(b >> 23) - 127) * TL_SBIN_OCT + (int)((b >> 20) & 7u);
  return i < TL_SBINS - 1 ? i : TL_SBINS - 1;
}

struct TLNarrowConst {
  float L;        // c dt [um], rounded to nearest
  float L_in;     // L (1 - 8u): t* surely inside when tau + err < L_in
  float L_out;    // L (1 + 8u): surely outside when tau - err >= L_out
  float r2max;    // upper bound on r^2 over all s [um^2]
  float kr;       // 1e12 kappa / pi in FP32
  float inv2mc4;  // 1 / (2 m_e^2 c^4) [MeV^-2]
  float pref;     // (pi/2) r_e^2 [m^2]
  // per bin of s (tl_sbin): an upper bound on r^2 = 1e12 kappa sigma(s) / pi
  // over the bin [um^2] (sigma rises up to its peak near s = 1.97, then falls)
  float sbin[TL_SBINS];
};

// Build-time launch helpers (defined in the .cu files).
namespace tl {
// one instance's input arrays (px py pz dx dy dz E w; w may be NULL) and
// its first photon in the concatenated beam
struct InstSrc {
  const double *p[8];
  long long n, off;
};
cudaError_t launch_inst_bounds(const TLBeam &b, const uint32_t *inst_of, int n_inst,
                               long long *tmp, double *out, cudaStream_t s);
cudaError_t launch_inst_box(const double *bounds, int n_inst, double T, int bits, float4 *box,
                            cudaStream_t s);
cudaError_t launch_gather_instances(const InstSrc *src, int n_inst, int64_t n, double *const *dst,
                                    uint32_t *inst_of, cudaStream_t s);
struct BuildBufs {
  float4 *pos_u, *dir_u;      // unsorted SoA32
  float4 *pos, *dir;          // sorted SoA32
  unsigned long long *key[2];
  uint32_t *val[2];
  TLNode *nodes;
  uint32_t *parent_leaf, *parent_node;
  float *rpre, *rsuf;  // per photon: union of the swept boxes from its tile's start / to its end
  float *rtile;        // per refit tile: union of its photons' swept boxes
  float *rsuper;       // sparse tables over the tile boxes, one per super-tile
  // traversal seeds: the children with at most cut_S photons of the nodes with
  // more, as (node << 1) | slot, written by the refit (cut_S = 0: none)
  uint32_t *cut;
  unsigned *cut_n;
  uint32_t cut_S, cut_cap, cut_alloc;
  // sort scratch
  uint32_t *sort_status;  // tiles * 256 per pass
  uint32_t *sort_raw;     // 8 * 256 digit counts of the keys (zero between sorts)
  uint32_t *sort_hist;    // 8 * 256 digit offsets (exclusive scan of sort_raw)
  uint32_t *sort_tile;    // 8 tile counters
  int64_t sort_tiles;
  int sort_epoch;  // 0: the status words must be cleared before the next sort
  uint32_t *sort_ep;  // device: epochs of the passes of the current sort, and the last one

  unsigned *build_status;  // shared status word of the context's builds
  // several independent instances in one beam (NULL / 0 for a single one)
  const uint32_t *inst_of;  // instance of each input photon
  uint32_t *inst_root;      // per instance: stack reference of its subtree root
  int inst_shift;           // bit position of the instance number in the key
  // per inner node: first photon of its range and its level (Morton prefix
  // length in bits below the key's top bit), for the level-L cut
  uint32_t *nfirst;
  uint32_t *nlast;   // last photon of every inner node's range (and the super root's)
  uint8_t *nlev;
  int key_bits;
};

// Arguments of the traversal kernels (tl_traverse.cu).
struct TravArgs {
  TLTree A, B;        // FP32 hierarchies
  TLBeam mA, mB;      // FP64 input beams
  double ct, dt, kappa;
  TLNarrowConst nk;
  int fp64;           // 1: every photon pair decided by the FP64 definition
  TLCounters *ctr;
  uint2 *hits;
  unsigned long long hit_cap;
  uint2 *band;
  unsigned long long band_cap;
  uint2 *leaves;  // overlapping leaf-bucket pairs (packed first | (count - 1) << 27)
  unsigned long long leaf_cap;
  unsigned long long *queue;  // traversal work queue: chunks of 32 (ref A, ref B) pairs
  unsigned long long queue_cap;  // in pairs
  uint2 *spill;                  // per traversal warp: the bottom of its stack
  unsigned spill_per_warp;       // entries per warp
  int stack_depth;
  int leaf_bucket;               // photons per leaf bucket at most
  const unsigned *build_status;  // build errors (a timed-out sort) skip the traversal
  long long spin_limit;          // iteration limit of a warp's wait for queued work
};

cudaError_t launch_propagate(const TLBeam &b, double ct, float L, const float box_lo[3],
                             const float box_scale[3], int bits, BuildBufs &w,
                             const float4 *inst_box, int passes, cudaStream_t s);
cudaError_t launch_static_soa(const TLBeam &b, BuildBufs &w, cudaStream_t s);
cudaError_t launch_beam_moments(const TLBeam &b, double *out15, double *scratch, cudaStream_t s);
cudaError_t sort_prepare();
cudaError_t launch_sort(BuildBufs &w, int64_t n, int key_bits, long long spin_limit,
                        int debug_stall, unsigned int *status, int *out_sel, cudaStream_t s);
cudaError_t launch_gather(BuildBufs &w, int64_t n, int sel, cudaStream_t s);
cudaError_t launch_karras(BuildBufs &w, int64_t n, int sel, int bucket, cudaStream_t s);
cudaError_t launch_refit(BuildBufs &w, int64_t n, float Llo, float Lhi, float half, int n_sm,
                         cudaStream_t s);
int64_t refit_tiles(int64_t n);
size_t refit_super_floats(int64_t n);
cudaError_t refit_prepare();
}  // namespace tl
