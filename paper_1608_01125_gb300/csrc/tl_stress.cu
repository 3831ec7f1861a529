// tl_stress.cu -- random stress of the FP32 narrow phase's error band.
//
// The FP32 narrow phase (tl_narrow.cuh) may only return a sure hit or a sure
// miss where the FP64 definition (tl_exact.cuh) decides the same way; every
// other pair must go to the FP64 band.  This entry point draws seeded photon
// pairs that sit on or near a boundary of the decision -- the distance at
// closest approach against the collision radius (d = r(1 +- 2^-e)), the
// closest-approach time against both ends of the half-open window [0, dt),
// the invariant s against the threshold s = 1 (Eq. eq.Cond), and the quick
// miss's 2.5 r_max^2 margin -- decides each both ways and counts the FP32
// sure decisions that disagree with FP64.
//
// A pair is drawn from a counter-based splitmix64 stream keyed by (seed,
// pair index), so any pair can be re-drawn; the first n_sample pairs are
// written out so that the CPU oracle can decide them too.
#include <math.h>

#include "tl_common.cuh"
#include "tl_ctx.h"
#include "tl_exact.cuh"
#include "tl_narrow.cuh"
#include "trilens.h"
#include "trilens_debug.h"

namespace {

constexpr int kCats = TRILENS_STRESS_CATEGORIES;
constexpr int kFields = TRILENS_STRESS_FIELDS;
constexpr int kThreads = 256;

struct Draw {
  unsigned long long key;
  unsigned t;
  __device__ double u() { return (double)(smix64(key + (t++)) >> 11) * 0x1p-53; }
  // 2^-e with e uniform in [lo, hi], with a random sign
  __device__ double tiny(int lo, int hi) {
    const int e = lo + (int)(u() * (double)(hi - lo + 1));
    const double v = ldexp(1.0, -(e > hi ? hi : e));
    return u() < 0.5 ? -v : v;
  }
  __device__ double normal() {  // Box-Muller
    const double a = u(), b = u();
    return sqrt(-2.0 * log(fmax(a, 1e-300))) * cos(2.0 * TL_PI * b);
  }
};

__device__ void unit(double &x, double &y, double &z) {
  const double n = sqrt(x * x + y * y + z * z);
  x /= n;
  y /= n;
  z /= n;
}

__global__ void __launch_bounds__(kThreads) k_band_stress(unsigned long long base, int64_t q0,
                                                          int64_t n, double dt, double kappa,
                                                          TLNarrowConst nk,
                                                          unsigned long long *counts,
                                                          double *sample, int64_t n_sample) {
  __shared__ unsigned long long sc[kCats * kFields];
  __shared__ float sbin[TL_SBINS];
  for (int t = threadIdx.x; t < kCats * kFields; t += kThreads) sc[t] = 0ull;
  for (int t = threadIdx.x; t < TL_SBINS; t += kThreads) sbin[t] = nk.sbin[t];
  __syncthreads();
  const double two_m2 = (2.0 * TL_MEC2) * TL_MEC2;
  for (int64_t q = q0 + blockIdx.x * (int64_t)kThreads + threadIdx.x; q < q0 + n;
       q += (int64_t)gridDim.x * kThreads) {
    Draw g{base + ((unsigned long long)q << 7), 0u};
    const int cat = (int)(q & (kCats - 1));
    const int k = (int)(g.u() * 64.0);
    // beam axes: A along +z, B at angle alpha from head-on (rotation about y);
    // each photon 5 mrad off its axis
    const double al = g.u() * TL_PI;
    double dxi = 5e-3 * g.normal(), dyi = 5e-3 * g.normal(), dzi = 1.0;
    unit(dxi, dyi, dzi);
    const double bx0 = 5e-3 * g.normal(), by0 = 5e-3 * g.normal(), bz0 = -1.0;
    double dxj = cos(al) * bx0 - sin(al) * bz0, dyj = by0, dzj = sin(al) * bx0 + cos(al) * bz0;
    unit(dxj, dyj, dzj);
    const double omc = 1.0 - (dxi * dxj + dyi * dyj + dzi * dzj);
    // energies: s on the threshold (category 6) or log-uniform in [1.001, 1e4]
    const double Ei = exp(log(0.2) + g.u() * log(500.0));
    const double st = cat == 6 ? 1.0 + g.tiny(1, 52) : 1.001 * exp(g.u() * log(1e4));
    const double Ej = st * two_m2 / (Ei * fmax(omc, 1e-300));
    const double sig = tl_sigma64(tl_s64(Ei, Ej, 1.0 - omc));
    const double r2 = 1e12 * kappa * sig / TL_PI;
    // closest-approach time within the step and squared distance there
    double t;
    if (cat == 4) t = g.tiny(1, 52) * dt;
    else if (cat == 5) t = dt * (1.0 + g.tiny(1, 52));
    else if (cat == 7) t = (-0.1 + 1.2 * g.u()) * dt;
    else t = g.u() * dt;
    double d2;
    if (cat < 4) d2 = r2 * (1.0 + g.tiny(1, 50));
    else if (cat == 7) d2 = 4.0 * g.u() * (double)nk.r2max;  // spans 2.5 r^2 bound of every s
    else d2 = 0.9 * g.u() * r2;
    // meeting point M anywhere within +-100 um; offset q perpendicular to the
    // relative velocity, so that the two photons are closest at t
    const double Mx = 200.0 * (g.u() - 0.5), My = 200.0 * (g.u() - 0.5), Mz = 200.0 * (g.u() - 0.5);
    double vx = dxi - dxj, vy = dyi - dyj, vz = dzi - dzj;
    const double vn = sqrt(vx * vx + vy * vy + vz * vz);
    double ex = g.normal(), ey = g.normal(), ez = g.normal();
    if (vn > 0.0) {
      vx /= vn;
      vy /= vn;
      vz /= vn;
      const double gv = ex * vx + ey * vy + ez * vz;
      ex -= gv * vx;
      ey -= gv * vy;
      ez -= gv * vz;
    }
    unit(ex, ey, ez);
    const double qd = sqrt(fmax(d2, 0.0));
    const double T = TL_C * ((double)k * dt + t);
    const double pxi = Mx + 0.5 * qd * ex - T * dxi, pyi = My + 0.5 * qd * ey - T * dyi,
                 pzi = Mz + 0.5 * qd * ez - T * dzi;
    const double pxj = Mx - 0.5 * qd * ex - T * dxj, pyj = My - 0.5 * qd * ey - T * dyj,
                 pzj = Mz - 0.5 * qd * ez - T * dzj;
    const double ct = TL_C * ((double)k * dt);
    const bool hit = tl_exact_decide(pxi, pyi, pzi, dxi, dyi, dzi, Ei, pxj, pyj, pzj, dxj, dyj, dzj,
                                     Ej, ct, dt, kappa);
    // the FP32 records the build writes: positions at t_k rounded once from FP64
    const float4 pa = make_float4(__double2float_rn(__dadd_rn(pxi, __dmul_rn(ct, dxi))),
                                  __double2float_rn(__dadd_rn(pyi, __dmul_rn(ct, dyi))),
                                  __double2float_rn(__dadd_rn(pzi, __dmul_rn(ct, dzi))),
                                  __double2float_rn(Ei));
    const float4 pb = make_float4(__double2float_rn(__dadd_rn(pxj, __dmul_rn(ct, dxj))),
                                  __double2float_rn(__dadd_rn(pyj, __dmul_rn(ct, dyj))),
                                  __double2float_rn(__dadd_rn(pzj, __dmul_rn(ct, dzj))),
                                  __double2float_rn(Ej));
    const float4 da = make_float4(__double2float_rn(dxi), __double2float_rn(dyi),
                                  __double2float_rn(dzi), 0.0f);
    const float4 db = make_float4(__double2float_rn(dxj), __double2float_rn(dyj),
                                  __double2float_rn(dzj), 0.0f);
    const int r32 = tl_narrow32(pa, da, pb, db, nk, sbin);
    unsigned long long *c = sc + cat * kFields;
    atomicAdd(c + 0, 1ull);
    if (hit) atomicAdd(c + 1, 1ull);
    if (r32 == TL_HIT) atomicAdd(c + 2, 1ull);
    if (r32 == TL_MISS) atomicAdd(c + 3, 1ull);
    if (r32 == TL_BAND) atomicAdd(c + 4, 1ull);
    if (r32 == TL_HIT && !hit) atomicAdd(c + 5, 1ull);
    if (r32 == TL_MISS && hit) atomicAdd(c + 6, 1ull);
    if (q < n_sample && sample) {
      double *o = sample + q * TRILENS_STRESS_SAMPLE;
      const double v[TRILENS_STRESS_SAMPLE] = {pxi, pyi, pzi, dxi, dyi, dzi, Ei, pxj, pyj,
                                               pzj, dxj, dyj, dzj, Ej, (double)k,
                                               hit ? 1.0 : 0.0, (double)r32};
      for (int f = 0; f < TRILENS_STRESS_SAMPLE; ++f) o[f] = v[f];
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < kCats * kFields; t += kThreads)
    if (sc[t]) atomicAdd(counts + t, sc[t]);
}

}  // namespace

extern "C" int trilens_debug_band_stress(uint64_t seed, int64_t n_pairs, double dt_fs,
                                         double kappa, unsigned long long *counts, double *sample,
                                         int64_t n_sample, trilens_stream_t stream) {
  if (n_pairs < 0 || !counts || !(dt_fs > 0.0) || !(kappa > 0.0) || n_sample < 0 ||
      (n_sample > 0 && !sample) || n_sample > n_pairs)
    return TRILENS_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  const TLNarrowConst nk = tl_narrow_const(dt_fs, kappa);
  const unsigned long long base = seed * 0x9E3779B97F4A7C15ull;
  int dev = 0, nsm = 152;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  // chunks of 2^26 pairs keep every launch short
  for (int64_t q0 = 0; q0 < n_pairs; q0 += (1ll << 26)) {
    const int64_t m = n_pairs - q0 < (1ll << 26) ? n_pairs - q0 : (1ll << 26);
    k_band_stress<<<8 * nsm, kThreads, 0, s>>>(base, q0, m, dt_fs, kappa, nk, counts, sample,
                                               n_sample);
    if (cudaGetLastError() != cudaSuccess) return TRILENS_ERR_CUDA;
  }
  return TRILENS_OK;
}

static_assert(TRILENS_NARROW_BINS == TL_SBINS, "the bin count of the ABI and of the kernels");

extern "C" int trilens_debug_narrow_bins(double dt_fs, double kappa, float *out, int32_t n,
                                         float *r2max) {
  if (!(dt_fs > 0.0) || !(kappa > 0.0) || !out || n < TL_SBINS) return TRILENS_ERR_INVALID;
  const TLNarrowConst nk = tl_narrow_const(dt_fs, kappa);
  for (int i = 0; i < TL_SBINS; ++i) out[i] = nk.sbin[i];
  if (r2max) *r2max = nk.r2max;
  return TL_SBINS;
}
