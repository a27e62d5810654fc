// Derivatives shared by the adjoint kernels: the MWB increment's partials,
// the cotangent of the equilibrium (Eqs. 10-11) with respect to the node
// state, and the change of variables to the moments of Eqs. (3)-(5).
#pragma once

#include "device_common.cuh"
#include "pclb_internal.h"

namespace pclb {

template <class T>
__device__ __forceinline__ T sgn(T x) { return T((x > T(0)) - (x < T(0))); }

// Partial derivatives of M = a D + K h(D, Dp) with respect to D and Dp.
template <class T>
__device__ __forceinline__ void mwb_partials(T a, T K, T D, T Dp, T& MD, T& MDp) {
  const T aD = abs(D), aP = abs(Dp), n = aD + aP;
  T hD = T(0), hP = T(0);
  if (n > T(0)) {
    const T inv2 = T(1) / (n * n);
    hD = (sgn(D) * (D - Dp) * aP + aD * n) * inv2;
    hP = -aD * (aD + D * sgn(Dp)) * inv2;
  }
  MD = a + K * hD;
  MDp = K * hP;
}

// G = sum_q lam(q) d f^eq_q / d(rho, u_x, u_y, E) at the given state (Eq. 10,
// weights Eq. 11).
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
  const T invE = T(1) / E;
  const T s = (ux * ux + uy * uy) * invE;
  const T a1 = T(1) - T(0.5) * s;
  const T a0 = a1 + T(0.125) * s * s;
  T A = 0, Bx = 0, By = 0, Cs = 0, Dx = 0, Fq = 0;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const int qb = k == 0 ? 0 : 1 + (k - 1) * kNDirs;
    const int qe = k == 0 ? 1 : qb + kNDirs;
#pragma unroll 1
    for (int q = qb; q < qe; ++q) {
      const T vx = d.vx[q], vy = d.vy[q];
      const T x = (vx * ux + vy * uy) * invE;
      const T x2 = x * x;
      const T P = a0 + x * (a1 + x * (T(0.5) * a1 + x * (T(1.0 / 6.0) + x * T(1.0 / 24.0))));
      const T Px = a1 * (T(1) + x) + x2 * (T(0.5) + x * T(1.0 / 6.0));
      const T Ps = T(-0.5) + T(0.25) * s - T(0.5) * x - T(0.25) * x2;
      const T l = lam(q);
      const T lF = l * F[k];
      A += lF * P;
      Bx += lF * Px * vx;
      By += lF * Px * vy;
      Cs += lF * Ps;
      Dx += lF * x * Px;
      Fq += l * Fd[k] * P;
    }
  }
  G[0] = A;
  G[1] = rho * (Bx + T(2) * ux * Cs) * invE;
  G[2] = rho * (By + T(2) * uy * Cs) * invE;
  G[3] = rho * (Fq - (Dx + s * Cs) * invE);
}

// Cotangent in (rho, u, E) -> cotangent in m = (rho, j_x, j_y, e).
template <class T>
__device__ __forceinline__ void to_moment_cotangent(T rho, T ux, T uy, T E, const T G[4], T g[4]) {
  const T inv = T(1) / rho;
  g[0] = G[0] - (ux * G[1] + uy * G[2]) * inv + (T(0.5) * (ux * ux + uy * uy) - E) * G[3] * inv;
  g[1] = (G[1] - ux * G[3]) * inv;
  g[2] = (G[2] - uy * G[3]) * inv;
  g[3] = G[3] * inv;
}

}  // namespace pclb
