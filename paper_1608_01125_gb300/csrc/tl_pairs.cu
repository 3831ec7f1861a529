// tl_pairs.cu -- the electron and positron of each collision (Sec. 1,
// Eq. pTotal and Eq. Lorentz).
//
// For a colliding pair (i of beam A, j of beam B) the photons' total energy E
// and momentum P (MeV, c = 1) fix the centre-of-mass (CoM) frame.  There each
// created particle has energy M/2, M^2 = E^2 - |P|^2 = 2 E_i E_j (1 - cos), and
// momentum p' = sqrt(M^2/4 - m^2) (Eq. pTotal); the electron flies along a
// random unit vector n, the positron opposite.  Both four-momenta are boosted
// back to the lab with the CoM velocity beta = P / E, gamma = E / M:
//   e_lab = gamma (e + beta.q),  q_lab = q + beta (gamma^2/(gamma+1) beta.q + gamma e),
// which is the paper's velocity addition (Eq. Lorentz) applied to momenta.
// n is uniform on the sphere (Marsaglia 1972: x1, x2 uniform in (-1, 1) until
// S = x1^2 + x2^2 lies in (0, 1); n = (2 x1 sqrt(1-S), 2 x2 sqrt(1-S), 1 - 2S)),
// its uniforms drawn from splitmix64 as a counter-based stream: key = seed ^
// ((i << 32) | j), draw t = top 53 bits of splitmix64(key + t) / 2^53.
// Everything is FP64 with explicit round-to-nearest operations in a fixed
// order (no contraction), so the result does not depend on the compiler.
#include "tl_common.cuh"

namespace tl {

__device__ __forceinline__ double unit_draw(unsigned long long key, unsigned long long t) {
  return __dmul_rn((double)(smix64(key + t) >> 11), 1.0 / 9007199254740992.0);
}

__device__ __forceinline__ void com_direction(unsigned long long seed, uint32_t i, uint32_t j,
                                              double n[3]) {
  const unsigned long long key = seed ^ (((unsigned long long)i << 32) | (unsigned long long)j);
  for (unsigned long long t = 0; t < 128; t += 2) {
    const double x1 = __dsub_rn(__dmul_rn(2.0, unit_draw(key, t)), 1.0);
    const double x2 = __dsub_rn(__dmul_rn(2.0, unit_draw(key, t + 1)), 1.0);
    const double S = __dadd_rn(__dmul_rn(x1, x1), __dmul_rn(x2, x2));
    if (S < 1.0 && S > 0.0) {
      const double r = __dsqrt_rn(__dsub_rn(1.0, S));
      n[0] = __dmul_rn(__dmul_rn(2.0, x1), r);
      n[1] = __dmul_rn(__dmul_rn(2.0, x2), r);
      n[2] = __dsub_rn(1.0, __dmul_rn(2.0, S));
      return;
    }
  }
  n[0] = 0.0;  // 64 rejections in a row: not reached in practice
  n[1] = 0.0;
  n[2] = 1.0;
}

__device__ __forceinline__ void boost(const double beta[3], double gamma, double e,
                                      const double q[3], double *out) {
  const double bq =
      __dadd_rn(__dadd_rn(__dmul_rn(beta[0], q[0]), __dmul_rn(beta[1], q[1])),
                __dmul_rn(beta[2], q[2]));
  const double k = __dadd_rn(__dmul_rn(__ddiv_rn(__dmul_rn(gamma, gamma), __dadd_rn(gamma, 1.0)),
                                       bq),
                             __dmul_rn(gamma, e));
  out[0] = __dmul_rn(gamma, __dadd_rn(e, bq));
  out[1] = __dadd_rn(q[0], __dmul_rn(beta[0], k));
  out[2] = __dadd_rn(q[1], __dmul_rn(beta[1], k));
  out[3] = __dadd_rn(q[2], __dmul_rn(beta[2], k));
}

// One hit per thread (grid-stride).  A hit whose indices are out of range or
// whose pair is below threshold gets eight zeros.
__global__ void __launch_bounds__(256) k_pair_products(TLBeam a, TLBeam b, const uint2 *hits,
                                                       int64_t n_hits, unsigned long long seed,
                                                       double *out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_hits;
       k += (int64_t)gridDim.x * blockDim.x) {
    const uint2 h = hits[k];
    double *o = out + 8 * k;
    double r[8] = {0., 0., 0., 0., 0., 0., 0., 0.};
    if ((int64_t)h.x < a.n && (int64_t)h.y < b.n) {
      const double E1 = a.E[h.x], E2 = b.E[h.y];
      const double d1[3] = {a.dx[h.x], a.dy[h.x], a.dz[h.x]};
      const double d2[3] = {b.dx[h.y], b.dy[h.y], b.dz[h.y]};
      const double E = __dadd_rn(E1, E2);
      double P[3];
      for (int c = 0; c < 3; ++c) P[c] = __dadd_rn(__dmul_rn(E1, d1[c]), __dmul_rn(E2, d2[c]));
      const double cs = __dadd_rn(__dadd_rn(__dmul_rn(d1[0], d2[0]), __dmul_rn(d1[1], d2[1])),
                                  __dmul_rn(d1[2], d2[2]));
      const double M2 = __dmul_rn(__dmul_rn(2.0, __dmul_rn(E1, E2)), __dsub_rn(1.0, cs));
      const double m = TL_MEC2;
      if (M2 > __dmul_rn(__dmul_rn(4.0, m), m)) {
        const double M = __dsqrt_rn(M2);
        const double ep = __dmul_rn(0.5, M);                                     // CoM energy
        const double pp = __dsqrt_rn(__dsub_rn(__dmul_rn(0.25, M2), __dmul_rn(m, m)));  // p'
        double n[3];
        com_direction(seed, h.x, h.y, n);
        const double beta[3] = {__ddiv_rn(P[0], E), __ddiv_rn(P[1], E), __ddiv_rn(P[2], E)};
        const double gamma = __ddiv_rn(E, M);
        const double qe[3] = {__dmul_rn(pp, n[0]), __dmul_rn(pp, n[1]), __dmul_rn(pp, n[2])};
        const double qp[3] = {-qe[0], -qe[1], -qe[2]};
        boost(beta, gamma, ep, qe, r);
        boost(beta, gamma, ep, qp, r + 4);
      }
    }
    double2 *o2 = reinterpret_cast<double2 *>(o);
    o2[0] = make_double2(r[0], r[1]);
    o2[1] = make_double2(r[2], r[3]);
    o2[2] = make_double2(r[4], r[5]);
    o2[3] = make_double2(r[6], r[7]);
  }
}

cudaError_t launch_pair_products(const TLBeam &a, const TLBeam &b, const uint32_t *hits,
                                 int64_t n_hits, unsigned long long seed, double *out, int n_sm,
                                 cudaStream_t s) {
  if (n_hits <= 0) return cudaSuccess;
  const int64_t nb = (n_hits + 255) / 256;
  const int blocks = (int)(nb < 8 * n_sm ? nb : 8 * n_sm);
  k_pair_products<<<blocks, 256, 0, s>>>(a, b, reinterpret_cast<const uint2 *>(hits), n_hits,
                                         seed, out);
  return cudaGetLastError();
}

}  // namespace tl
