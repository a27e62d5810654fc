// Derivatives shared by the adjoint kernels: the MWB increment's partials,
// the cotangent of the equilibrium (Eqs. 10-11) with respect to the node
// state, and the change of variables to the moments of Eqs. (3)-(5).
#pragma once

#include "device_common.cuh"
#include "pclb_internal.h"

namespace pclb {

// 1/x for the partials below: the hardware approximation in FP32 (relative
// error ~1 ulp), two Newton steps on it in FP64 (recip_newton).
__device__ __forceinline__ float recip_fast(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ double recip_fast(double x) { return recip_newton(x); }

// 1/x for the cotangent factors: FP32 by the hardware approximation and one
// Newton-Raphson step r + r (1 - x r); FP64 the correctly rounded quotient.
__device__ __forceinline__ float recip1(float x) {
  const float r = recip_fast(x);
  return fmaf(r, fmaf(-x, r, 1.0f), r);
}
__device__ __forceinline__ double recip1(double x) { return 1.0 / x; }

template <class T>
__device__ __forceinline__ T smallest_normal();
template <>
__device__ __forceinline__ float smallest_normal<float>() { return 1.17549435e-38f; }
template <>
__device__ __forceinline__ double smallest_normal<double>() { return 2.2250738585072014e-308; }

// Partial derivatives of M = a D + K h(D, Dp), h = |D|(D - Dp)/(|D| + |Dp|),
// with respect to D and Dp.  With n = |D| + |Dp|, a' = |D|/n, b' = |Dp|/n and
// s = sign(D) sign(Dp):
//   h_D = a'(1 + b') - s b'^2,   h_Dp = -(1 + s) a'^2,
// both 0 when n = 0 (sign(0) = 0: the derivative on the active branch).  The
// pair is unchanged when D and Dp change sign together.
template <class T>
__device__ __forceinline__ void mwb_partials(T a, T K, T D, T Dp, T& MD, T& MDp) {
  const T aD = abs(D), aP = abs(Dp), n = aD + aP;
  const T rn = n >= smallest_normal<T>() ? recip_fast(n) : T(0);
  const T ar = aD * rn, br = aP * rn;
  // s: the sign of the product D Dp is exact even where the product
  // underflows; s = 0 when either factor is 0
  const T s = min(aD, aP) > T(0) ? copysign(T(1), D * Dp) : T(0);
  const T Ka = K * ar;
  MD = fma(K, fma(br, fma(-s, br, ar), ar), a);   // a + K (ar + br (ar - s br))
  MDp = -(T(1) + s) * (Ka * ar);
}
// FP64: the same, with the zero tests and the sign of D Dp taken on the bit
// patterns by integer instructions (GB300 runs FP64 arithmetic at 1/64 of the
// FP32 rate; integer compares keep it free for the products).
template <>
__device__ __forceinline__ void mwb_partials<double>(double a, double K, double D, double Dp, double& MD,
                                                     double& MDp) {
  const long long bD = __double_as_longlong(D), bP = __double_as_longlong(Dp);
  const double aD = fabs(D), aP = fabs(Dp), n = aD + aP;
  // n >= 2^-1022 (n is non-negative: its high word orders like the value)
  const double rn = __double2hiint(n) >= 0x00100000 ? recip_fast(n) : 0.0;
  const double ar = aD * rn, br = aP * rn;
  // |D| > 0 and |Dp| > 0: a nonzero magnitude (sign bit cleared); the sign of
  // D Dp from the sign bits
  const bool nz = ((bD & 0x7fffffffffffffffll) != 0) && ((bP & 0x7fffffffffffffffll) != 0);
  const double s = nz ? ((bD ^ bP) < 0 ? -1.0 : 1.0) : 0.0;
  const double Ka = K * ar;
  MD = fma(K, fma(br, fma(-s, br, ar), ar), a);   // a + K (ar + br (ar - s br))
  MDp = -(1.0 + s) * (Ka * ar);
}

// The terms of one pair of opposite velocities (v, -v) of a shell in the sums
// of eq_cotangent below, added to Ak, Bxk, Byk, Ck, Dk; lp, lm: the
// cotangents of f^eq at v and -v.
template <class T>
__device__ __forceinline__ void pair_terms(T vx, T vy, T uxE, T uyE, T s, T a0, T a1, T lp, T lm, T& Ak, T& Bxk,
                                           T& Byk, T& Ck, T& Dk) {
  const T x = vx * uxE + vy * uyE;
  const T x2 = x * x;
  const T Pe = a0 + x2 * (T(0.5) * a1 + x2 * T(1.0 / 24.0));   // P(+-x) = Pe +- Po
  const T Po = x * (a1 + x2 * T(1.0 / 6.0));
  const T Xe = a1 + x2 * T(0.5);                                // P_x(+-x) = Xe +- Xo
  const T Xo = x * (a1 + x2 * T(1.0 / 6.0));
  const T Se = T(-0.5) + T(0.25) * s - T(0.25) * x2;           // P_s(+-x) = Se -+ x/2
  const T ls = lp + lm, ld = lp - lm;
  Ak += ls * Pe + ld * Po;
  const T lpx = ld * Xe + ls * Xo;        // lp Px(x) - lm Px(-x)
  Bxk += lpx * vx;
  Byk += lpx * vy;
  Ck += ls * Se - ld * T(0.5) * x;
  Dk += x * (ls * Xo + ld * Xe);          // lp x Px(x) + lm (-x) Px(-x)
}

// G = sum_q lam(q) d f^eq_q / d(rho, u_x, u_y, E) at the given state (Eq. 10,
// weights Eq. 11).  With P(x) the polynomial of Eq. (10), P_x, P_s its
// derivatives in x = v.u/E and s = u^2/E:
//   G_rho = sum lam F P,  G_u = rho sum lam F (P_x v + 2 P_s u) / E,
//   G_E = rho sum lam (F' P - F (x P_x + s P_s) / E).
// Opposite velocities of a shell (x and -x) share the even and odd parts of
// P, P_x and P_s.
template <class T, class LamFn>
__device__ __forceinline__ void eq_cotangent(T rho, T ux, T uy, T E, const DvmConst<T>& d, LamFn lam,
                                             T G[4]) {
  T F[5], Fd[5];
  T Fs = T(0), Fds = T(0);
#pragma unroll
  for (int k = 1; k <= 4; ++k) {
    const T* c = d.Fc[k];
    F[k] = E * (c[0] + E * (c[1] + E * (c[2] + E * c[3])));
    Fd[k] = c[0] + E * (T(2) * c[1] + E * (T(3) * c[2] + E * T(4) * c[3]));
    Fs += F[k];
    Fds += Fd[k];
  }
  F[0] = T(1) - d.B0 * Fs;
  Fd[0] = -d.B0 * Fds;
  const T invE = recip1(E);
  const T s = (ux * ux + uy * uy) * invE;
  const T a1 = T(1) - T(0.5) * s;
  const T a0 = a1 + T(0.125) * s * s;
  const T uxE = ux * invE, uyE = uy * invE;
  // rest velocity: x = 0
  const T l0 = lam(0);
  T A = l0 * F[0] * a0, Bx = 0, By = 0, Cs = l0 * F[0] * (T(-0.5) + T(0.25) * s), Dx = 0;
  T Fq = l0 * Fd[0] * a0;
  constexpr int half = kNDirs / 2;
#pragma unroll
  for (int k = 1; k <= 4; ++k) {
    T Ak = 0, Bxk = 0, Byk = 0, Ck = 0, Dk = 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const int q = 1 + (k - 1) * kNDirs + i;
      pair_terms<T>(d.vx[q], d.vy[q], uxE, uyE, s, a0, a1, lam(q), lam(q + half), Ak, Bxk, Byk, Ck, Dk);
    }
    A += F[k] * Ak;
    Bx += F[k] * Bxk;
    By += F[k] * Byk;
    Cs += F[k] * Ck;
    Dx += F[k] * Dk;
    Fq += Fd[k] * Ak;
  }
  G[0] = A;
  G[1] = rho * (Bx + T(2) * ux * Cs) * invE;
  G[2] = rho * (By + T(2) * uy * Cs) * invE;
  G[3] = rho * (Fq - (Dx + s * Cs) * invE);
}

// Cotangent in (rho, u, E) -> cotangent in m = (rho, j_x, j_y, e).
template <class T>
__device__ __forceinline__ void to_moment_cotangent(T rho, T ux, T uy, T E, const T G[4], T g[4]) {
  const T inv = recip1(rho);
  g[0] = G[0] - (ux * G[1] + uy * G[2]) * inv + (T(0.5) * (ux * ux + uy * uy) - E) * G[3] * inv;
  g[1] = (G[1] - ux * G[3]) * inv;
  g[2] = (G[2] - uy * G[3]) * inv;
  g[3] = G[3] * inv;
}

// The FP32 pair kernel over tiles a0 .. a0 + na - 1 and b0 .. (nx blocks in
// r), all theta tiles (adjoint_f32x2.cu); tmap_fn, tmap_ln: descriptors of f
// and lam with one tile per box, for its node phase.  walls: the tiles may
// include wall tiles (radial tile 0 or r0 >= n_r - 33); false only for a
// launch of interior tiles, which then runs the instance without wall code.
cudaError_t launch_adjoint_pairs_f32(const CUtensorMap* tmap_f, const CUtensorMap* tmap_l, const CUtensorMap* tmap_fn,
                                     const CUtensorMap* tmap_ln, const float* f,
                                     const float* lam_in, float* lam_out, const EqParams<float>* ghost,
                                     const float* gwall, const float* gdir, int a0, int na, int b0, int nx,
                                     bool walls, const StepParams& p, const DvmConst<float>& d, cudaStream_t s);

}  // namespace pclb
