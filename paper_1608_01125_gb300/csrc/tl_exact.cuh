// tl_exact.cuh -- the FP64 collision decision on the device.
//
// This is the reference decision of the library: every hit the library
// reports is a pair this function accepts, evaluated with explicit
// round-to-nearest FP64 intrinsics in a fixed order (no contraction), so the
// result does not depend on the compiler's FMA choices.
//
//   s     = (E_i E_j)(1 - cos Phi) / ((2 m_e c^2) m_e c^2)      (text below Eq. BWcross)
//   s > 1 required                                               (Eq. eq.Cond)
//   sigma = (pi/2) r_e^2 (1/s) [(3 - b^4) ln((1+b)^2 s) - 2b(2 - b^2)],
//           b = sqrt((s-1)/s)                                    (Eq. BWcross; (1+b)/(1-b) = (1+b)^2 s)
//   P     = p0 + (c t_k) d                                       (straight lines, Sec. 2.1)
//   v     = c (d_i - d_j),  t* = -(dP . v)/(v . v), 0 <= t* < dt
//   hit  <=> |dP + t* v|^2 < 1e12 kappa sigma / pi
#pragma once
#include "tl_common.cuh"

// Natural log for finite x >= 1 (the only arguments used here):
// x = m 2^e with m in [sqrt(1/2), sqrt(2)), ln m = 2 atanh f, f = (m-1)/(m+1),
// summed as the odd power series up to f^23 by Horner in z = f^2.
__device__ __forceinline__ double tl_ln64(double x) {
  long long bits = __double_as_longlong(x);
  int e = (int)((bits >> 52) & 0x7ff) - 1022;  // x = m 2^e, m in [1/2, 1)
  double m = __longlong_as_double((bits & 0x800fffffffffffffLL) | 0x3fe0000000000000LL);
  if (m < 0.70710678118654752440) {
    m = __dmul_rn(m, 2.0);
    e = e - 1;
  }
  double f = __ddiv_rn(__dsub_rn(m, 1.0), __dadd_rn(m, 1.0));
  double z = __dmul_rn(f, f);
  double p = 1.0 / 23.0;
  p = __dadd_rn(__dmul_rn(p, z), 1.0 / 21.0);
  p = __dadd_rn(__dmul_rn(p, z), 1.0 / 19.0);
  p = __dadd_rn(__dmul_rn(p, z), 1.0 / 17.0);
  p = __dadd_rn(__dmul_rn(p, z), 1.0 / 15.0);
  p = __dadd_rn(__dmul_rn(p, z), 1.0 / 13.0);
  p = __dadd_rn(__dmul_rn(p, z), 1.0 / 11.0);
  p = __dadd_rn(__dmul_rn(p, z), 1.0 / 9.0);
  p = __dadd_rn(__dmul_rn(p, z), 1.0 / 7.0);
  p = __dadd_rn(__dmul_rn(p, z), 1.0 / 5.0);
  p = __dadd_rn(__dmul_rn(p, z), 1.0 / 3.0);
  p = __dadd_rn(__dmul_rn(p, z), 1.0);
  double lnm = __dmul_rn(__dmul_rn(2.0, f), p);
  double de = (double)e;
  // ln 2 split so that e * hi is exact (hi has 32 significant bits)
  return __dadd_rn(__dmul_rn(de, 0.6931471803691238),
                   __dadd_rn(__dmul_rn(de, 1.9082149292705877e-10), lnm));
}

// Eq. BWcross [m^2]; zero at and below threshold.
__device__ __forceinline__ double tl_sigma64(double s) {
  if (!(s > 1.0)) return 0.0;
  double inv = __ddiv_rn(1.0, s);
  double b = __dsqrt_rn(__ddiv_rn(__dsub_rn(s, 1.0), s));
  double b2 = __dmul_rn(b, b);
  double opb = __dadd_rn(1.0, b);
  double lg = tl_ln64(__dmul_rn(__dmul_rn(opb, opb), s));
  double br = __dsub_rn(__dmul_rn(__dsub_rn(3.0, __dmul_rn(b2, b2)), lg),
                        __dmul_rn(__dmul_rn(2.0, b), __dsub_rn(2.0, b2)));
  const double pref = ((0.5 * TL_PI) * TL_RE) * TL_RE;
  return __dmul_rn(__dmul_rn(pref, inv), br);
}

__device__ __forceinline__ double tl_s64(double Ei, double Ej, double cs) {
  return __ddiv_rn(__dmul_rn(__dmul_rn(Ei, Ej), __dsub_rn(1.0, cs)), (2.0 * TL_MEC2) * TL_MEC2);
}

// The decision for one photon pair given by value: positions at t = 0,
// unit directions and energies of photon i (beam A) and photon j (beam B),
// at the step with ct = c * (k * dt).
__device__ __forceinline__ bool tl_exact_decide(double p0xi, double p0yi, double p0zi, double dxi,
                                                double dyi, double dzi, double Ei, double p0xj,
                                                double p0yj, double p0zj, double dxj, double dyj,
                                                double dzj, double Ej, double ct, double dt,
                                                double kappa) {
  double cs = __dadd_rn(__dadd_rn(__dmul_rn(dxi, dxj), __dmul_rn(dyi, dyj)), __dmul_rn(dzi, dzj));
  double s = tl_s64(Ei, Ej, cs);
  if (!(s > 1.0)) return false;
  double vx = __dmul_rn(TL_C, __dsub_rn(dxi, dxj));
  double vy = __dmul_rn(TL_C, __dsub_rn(dyi, dyj));
  double vz = __dmul_rn(TL_C, __dsub_rn(dzi, dzj));
  double vv = __dadd_rn(__dadd_rn(__dmul_rn(vx, vx), __dmul_rn(vy, vy)), __dmul_rn(vz, vz));
  if (vv == 0.0) return false;
  double px = __dsub_rn(__dadd_rn(p0xi, __dmul_rn(ct, dxi)), __dadd_rn(p0xj, __dmul_rn(ct, dxj)));
  double py = __dsub_rn(__dadd_rn(p0yi, __dmul_rn(ct, dyi)), __dadd_rn(p0yj, __dmul_rn(ct, dyj)));
  double pz = __dsub_rn(__dadd_rn(p0zi, __dmul_rn(ct, dzi)), __dadd_rn(p0zj, __dmul_rn(ct, dzj)));
  double pv = __dadd_rn(__dadd_rn(__dmul_rn(px, vx), __dmul_rn(py, vy)), __dmul_rn(pz, vz));
  double ts = __ddiv_rn(-pv, vv);
  if (!(ts >= 0.0) || !(ts < dt)) return false;  // half-open window [0, dt)
  double qx = __dadd_rn(px, __dmul_rn(ts, vx));
  double qy = __dadd_rn(py, __dmul_rn(ts, vy));
  double qz = __dadd_rn(pz, __dmul_rn(ts, vz));
  double d2 = __dadd_rn(__dadd_rn(__dmul_rn(qx, qx), __dmul_rn(qy, qy)), __dmul_rn(qz, qz));
  double r2 = __ddiv_rn(__dmul_rn(__dmul_rn(1e12, kappa), tl_sigma64(s)), TL_PI);
  return d2 < r2;
}

// The decision for input photons i of A and j of B at the step with
// ct = c * (k * dt).
__device__ __forceinline__ bool tl_exact_hit(const TLBeam &A, uint32_t i, const TLBeam &B,
                                             uint32_t j, double ct, double dt, double kappa) {
  return tl_exact_decide(A.px[i], A.py[i], A.pz[i], A.dx[i], A.dy[i], A.dz[i], A.E[i], B.px[j],
                         B.py[j], B.pz[j], B.dx[j], B.dy[j], B.dz[j], B.E[j], ct, dt, kappa);
}
