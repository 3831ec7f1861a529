// tl_narrow.cuh -- FP32 narrow phase with a rigorous error band.
//
// For a photon pair the FP32 path computes the same quantities as the FP64
// definition (tl_exact.cuh) -- s, the closest-approach parameter
// tau = c t* = -(dP . dD)/|dD|^2 with dD = d_i - d_j, the offset
// q = dP + tau dD, d^2 = |q|^2 and r^2 = 1e12 kappa sigma(s)/pi -- together
// with bounds on how far each FP32 value can be from the FP64 one.  It
// returns a decision only when the bound puts the pair on one side of every
// test; otherwise the pair goes to the FP64 re-test.  So the FP32 path
// returns exactly the FP64 hit set.
//
// Error model (u = 2^-24, first order, then every bound doubled so that
// second-order terms, the rounding of the bound's own evaluation and the FP64
// definition's ~1e-16 relative error are covered):
//   inputs  P32 = P64 (1+e), |e| <= u per coordinate; d32, E32 likewise
//   dP      |d dP|  <= 2u SA,           SA = sum_c |Pa_c| + |Pb_c|
//   dD      |d dD|  <= 4u
//   q       |dq|    <= 2u SA + 4u (|q|/|dD| + |tau|) + 7.02u |tau||dD| + 4.01u |q|
//   d^2     |d d2|  <= 2|q| dq + dq^2 + 3.01u d2
//   tau     |dtau|  <= 2u SA/|dD| + 4u |q|/|dD|^2 + 12u |tau|/|dD| + 7.02u |tau| + 3.01u |q|/|dD|
//   s       |ds|    <= 9u s + 6u E_i E_j / (2 m^2 c^4)   (cos error <= 5u absolute)
//   sigma   relative: evaluation terms (logf within 1 ulp, sqrtf and the
//           divisions correctly rounded) plus |g(s)| ds/s with the
//           logarithmic slope |g| = |s sigma'/sigma| <= s/(s-1) + 1.
#pragma once
#include "tl_common.cuh"

enum { TL_MISS = 0, TL_HIT = 1, TL_BAND = 2 };

// The test's prefix: the threshold and the quick miss, with the quantities
// the rest of the test uses.  early >= 0 is the outcome the prefix already
// decides (a sure miss, or the band for nearly parallel pairs).
struct TLNarrowPre {
  float s, es;
  bool above;
  float dd, rdd, tau, d2, SA, r2ub;
  int early;
};

// sbin: the table k.sbin (a copy in shared memory: its lookups diverge)
__device__ __forceinline__ TLNarrowPre tl_narrow32_pre(const float4 pa, const float4 da,
                                                       const float4 pb, const float4 db,
                                                       const TLNarrowConst &k,
                                                       const float *sbin) {
  const float u = 5.9604644775390625e-8f;  // 2^-24
  TLNarrowPre r;
  r.early = -1;
  // --- threshold (Eq. eq.Cond) -------------------------------------------
  const float cs = fmaf(da.x, db.x, fmaf(da.y, db.y, da.z * db.z));
  const float omc = 1.0f - cs;
  const float eek = (pa.w * pb.w) * k.inv2mc4;
  r.s = eek * omc;
  r.es = 2.0f * (9.0f * u * r.s + 6.0f * u * eek);
  const float thr = 9.5367431640625e-7f;  // 2^-20
  if (r.s + r.es <= 1.0f - thr) {  // surely s64 <= 1 (covers parallel pairs)
    r.early = TL_MISS;
    return r;
  }
  r.above = (r.s - r.es) >= 1.0f + thr;

  // --- closest approach -----------------------------------------------------
  const float dpx = pa.x - pb.x, dpy = pa.y - pb.y, dpz = pa.z - pb.z;
  const float ddx = da.x - db.x, ddy = da.y - db.y, ddz = da.z - db.z;
  r.dd = fmaf(ddx, ddx, fmaf(ddy, ddy, ddz * ddz));
  if (!(r.dd > 1e-20f)) {  // nearly parallel yet maybe above threshold
    r.early = TL_BAND;
    return r;
  }
  const float pd = fmaf(dpx, ddx, fmaf(dpy, ddy, dpz * ddz));
  r.rdd = __frcp_rn(r.dd);
  r.tau = -pd * r.rdd;
  const float qx = fmaf(r.tau, ddx, dpx), qy = fmaf(r.tau, ddy, dpy), qz = fmaf(r.tau, ddz, dpz);
  r.d2 = fmaf(qx, qx, fmaf(qy, qy, qz * qz));

  r.SA = (fabsf(pa.x) + fabsf(pb.x)) + (fabsf(pa.y) + fabsf(pb.y)) + (fabsf(pa.z) + fabsf(pb.z));
  // The largest radius^2 of any s the FP64 invariant can take: s64 lies in
  // [s - es, s + es], which meets at most two adjacent bins of s when es is
  // small (else every s counts).
  const int b0 = tl_sbin(__fsub_rd(r.s, r.es)), b1 = tl_sbin(__fadd_ru(r.s, r.es));
  r.r2ub = b1 - b0 <= 1 ? fmaxf(sbin[b0], sbin[b1]) : k.r2max;
  // Quick miss, before the bounds: if |dD|^2 >= 2^-30, SA <= 2^18 |q| and
  // either |tau| <= 2^10 and |q|^2 >= 2^-12, or |tau| <= 4 and |q|^2 >= 2^-26,
  // every term of dq below is a small fraction of |q| (2u SA <= |q|/32,
  // 4u |q|/|dD| <= |q|/128, 4u |tau| <= |q|/64, 7.1u |tau||dD| <= |q|/18), so
  // dq <= 0.23 |q| and ed2 <= 0.5 d2: d2 >= 2.5 r2ub then puts the FP64
  // distance beyond the radius of every s the pair can have.
  const float at = fabsf(r.tau);
  const float floor2 = at <= 4.0f ? 0x1p-26f : 0x1p-12f;
  if (r.dd >= 0x1p-30f && at <= 1024.0f && r.d2 >= fmaxf(2.5f * r.r2ub, floor2) &&
      r.SA * r.SA <= 0x1p36f * r.d2)
    r.early = TL_MISS;
  return r;
}

// true when the prefix alone makes the pair a sure miss (exactly when
// tl_narrow32 returns TL_MISS before its error bounds)
__device__ __forceinline__ bool tl_narrow32_quick_miss(const float4 pa, const float4 da,
                                                       const float4 pb, const float4 db,
                                                       const TLNarrowConst &k,
                                                       const float *sbin) {
  return tl_narrow32_pre(pa, da, pb, db, k, sbin).early == TL_MISS;
}

__device__ __forceinline__ int tl_narrow32(const float4 pa, const float4 da, const float4 pb,
                                           const float4 db, const TLNarrowConst &k,
                                           const float *sbin) {
  const float u = 5.9604644775390625e-8f;  // 2^-24
  const TLNarrowPre pre = tl_narrow32_pre(pa, da, pb, db, k, sbin);
  if (pre.early >= 0) return pre.early;
  const float s = pre.s, es = pre.es, dd = pre.dd, rdd = pre.rdd, tau = pre.tau, d2 = pre.d2;
  const float SA = pre.SA;
  const bool above = pre.above;
  const float nq = sqrtf(d2);
  // over-estimates of 1/|dD| and |dD| for the bounds: rsqrtf is within 2 ulp
  // (4u relative) of 1/sqrt(dd), so 1 + 8u covers it and the product's rounding
  const float rnd = rsqrtf(dd) * (1.0f + 8.0f * u);
  const float nd = dd * rnd;
  const float at = fabsf(tau);
  const float dq =
      2.0f * (2.0f * u * SA + 4.0f * u * (nq * rnd + at) + 7.1f * u * at * nd + 4.1f * u * nq);
  const float ed2 = 2.0f * nq * dq + dq * dq + 2.0f * 3.1f * u * d2;
  const float et = 2.0f * (2.0f * u * SA * rnd + 4.0f * u * nq * rdd + 12.0f * u * at * rnd +
                           7.1f * u * at + 3.1f * u * nq * rnd);

  // window 0 <= t* < dt (half open)
  if (tau + et < 0.0f || tau - et >= k.L_out) return TL_MISS;
  const bool win_in = (tau - et > 0.0f) && (tau + et < k.L_in);
  // farther than the largest radius of any s the pair can have
  if (d2 - ed2 >= pre.r2ub) return TL_MISS;
  if (!above) return TL_BAND;  // too close to threshold for the FP32 sigma

  // --- sigma(s) (Eq. BWcross) in FP32 with its bound -------------------------
  const float inv = 1.0f / s;
  const float b2 = (s - 1.0f) * inv;
  const float b = sqrtf(b2);
  const float opb = 1.0f + b;
  const float lg = logf((opb * opb) * s);
  const float t1 = (3.0f - b2 * b2) * lg;
  const float t2 = (2.0f * b) * (2.0f - b2);
  const float br = t1 - t2;
  const float sig = (k.pref * inv) * br;
  const float ebr = 6.0f * u * fabsf(t1) + 27.0f * u + 6.0f * u * fabsf(lg) +
                    8.5f * u * fabsf(t2) + u * fabsf(br);
  const float sm1 = s - es - 1.0f;  // lower bound of s - 1 (> 0 here)
  const float xs = es / sm1;        // relative size of the s error near threshold
  if (!(xs < 0.5f) || !(br > 0.0f)) return TL_BAND;
  const float g = s / sm1 + 1.0f;
  const float er = 2.0f * (ebr / br + 5.0f * u + g * (es / s));
  const float r2 = sig * k.kr;
  if (d2 - ed2 >= r2 * (1.0f + er)) return TL_MISS;
  if (win_in && d2 + ed2 < r2 * (1.0f - er)) return TL_HIT;
  return TL_BAND;
}
