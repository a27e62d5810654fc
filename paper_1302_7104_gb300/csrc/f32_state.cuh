// FP32 path: float-float node state, equilibrium factors and the
// equilibrium of Eq. (10), shared by the step and the field kernels.
#pragma once

#include "device_common.cuh"

namespace pclb {

constexpr int kHalf = kNDirs / 2;   // opposite-direction pairs per shell

__device__ __forceinline__ ff ff_of(float x) { return ff{x, 0.f}; }

// Float-float macroscopic state of a node.
struct State32 {
  ff rho, ux, uy, E;
  bool ok;
};

// Per-node factors of the equilibrium used by the update loop.
struct Eq32 {
  float w[5];              // rho F_k(E)
  float a0, a1, a1h;       // Eq. (10) polynomial coefficients
  float yh[kHalf], yl[kHalf];  // c_i . u / E for the first direction of each pair (float-float)
};

// Moments of one node (Eqs. 3-5) from f[q * stride], then the temperature
// recovery E = (e - |j|^2/(2 rho)) / rho in float-float.  Within a shell the
// eight values are summed in float over opposite-direction pairs; shells 2 and
// 3 (speeds 2.92 and 2.99, weights of opposite sign) are first added direction
// by direction so that their large contributions cancel before rounding, and
// shell 3 enters once more with the speed differences; the shell totals are
// combined with error-free transformations.
template <class Stride>
__device__ __forceinline__ void shell_sums(const float* f, Stride stride, const DvmConst<float>& d,
                                           int k, int k_add, float& S, float& X, float& Xl, float& Y,
                                           float& Yl) {
  S = 0.f; X = 0.f; Xl = 0.f; Y = 0.f; Yl = 0.f;
#pragma unroll
  for (int i = 0; i < kHalf; ++i) {
    const int q = 1 + (k - 1) * kNDirs + i;
    float fa = f[q * stride], fb = f[(q + kHalf) * stride];
    if (k_add > 0) {
      const int qa = 1 + (k_add - 1) * kNDirs + i;
      fa += f[qa * stride];
      fb += f[(qa + kHalf) * stride];
    }
    S += fa + fb;
    const float dd = fa - fb;   // the pair has opposite unit vectors
    X = fmaf(d.cx[q], dd, X);
    Xl = fmaf(d.cx_lo[q], dd, Xl);
    Y = fmaf(d.cy[q], dd, Y);
    Yl = fmaf(d.cy_lo[q], dd, Yl);
  }
}

template <class Stride>
__device__ __forceinline__ State32 state32(const float* f, Stride stride, const DvmConst<float>& d) {
  ff rho = ff_of(f[0]), jx = ff_of(0.f), jy = ff_of(0.f), e = ff_of(0.f);
  // (shell, shell added to it, speed, v^2/2): 1; 2+3 with v_2; 3 with v_3 - v_2; 4
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    const int k = g == 0 ? 1 : (g == 1 ? 2 : (g == 2 ? 3 : 4));
    const int k_add = g == 1 ? 3 : 0;
    float S, X, Xl, Y, Yl;
    shell_sums(f, stride, d, k, k_add, S, X, Xl, Y, Yl);
    ff sp, hv;
    if (g == 2) {
      sp = ff{d.dv23, d.dv23_lo};
      hv = ff{d.dh23, d.dh23_lo};
    } else {
      sp = ff{d.speed[k], d.speed_lo[k]};
      hv = ff{d.half_v2[k], d.half_v2_lo[k]};
    }
    if (g != 2) rho = ff_add(rho, ff_of(S));
    jx = ff_add(jx, ff_mul(sp, ff{X, Xl}));
    jy = ff_add(jy, ff_mul(sp, ff{Y, Yl}));
    e = ff_add(e, ff_mul(hv, ff_of(S)));
  }
  State32 s;
  const ff inv = ff_recip(rho);
  s.rho = rho;
  s.ux = ff_mul(jx, inv);
  s.uy = ff_mul(jy, inv);
  const ff ke = ff_add(ff_mul(jx, s.ux), ff_mul(jy, s.uy));      // |j|^2 / rho
  s.E = ff_mul(ff_add(e, ff_scale(ke, -0.5f)), inv);
  s.ok = (rho.hi > 0.f) && (s.E.hi > 0.f) && isfinite(e.hi) && isfinite(jx.hi) && isfinite(jy.hi);
  return s;
}

// Weights and polynomial factors of Eq. (10) for a node state.
__device__ __forceinline__ Eq32 eq32(const State32& s, const DvmConst<float>& d) {
  Eq32 q;
  ff sum = ff_of(0.f);
#pragma unroll
  for (int k = 1; k <= 4; ++k) {
    ff a{d.Fc[k][3], d.Fc_lo[k][3]};
#pragma unroll
    for (int n = 2; n >= 0; --n) a = ff_mul_add(a, s.E, ff{d.Fc[k][n], d.Fc_lo[k][n]});
    a = ff_mul(a, s.E);                  // F_k(E)
    sum = ff_add(sum, a);
    const ff wk = ff_mul(s.rho, a);
    q.w[k] = wk.hi + wk.lo;
  }
  const ff f0 = ff_add(ff_of(1.f), ff_mul(ff_of(-d.B0), sum));   // F_0 = 1 - B0 sum F_k
  const ff w0 = ff_mul(s.rho, f0);
  q.w[0] = w0.hi + w0.lo;
  const ff invE = ff_recip(s.E);
  const ff uxE = ff_mul(s.ux, invE), uyE = ff_mul(s.uy, invE);
  const ff u2E = ff_add(ff_mul(s.ux, uxE), ff_mul(s.uy, uyE));   // u^2 / E
  const ff a1 = ff_add(ff_of(1.f), ff_scale(u2E, -0.5f));
  const ff a0 = ff_add(a1, ff_scale(ff_mul(u2E, u2E), 0.125f));
  q.a1 = a1.hi + a1.lo;
  q.a0 = a0.hi + a0.lo;
  q.a1h = 0.5f * q.a1;
#pragma unroll
  for (int i = 0; i < kHalf; ++i) {
    const int qq = 1 + i;   // direction i of shell 1: unit vector (cx, cy)
    const ff y = ff_add(ff_mul(ff{d.cx[qq], d.cx_lo[qq]}, uxE), ff_mul(ff{d.cy[qq], d.cy_lo[qq]}, uyE));
    q.yh[i] = y.hi;
    q.yl[i] = y.lo;
  }
  return q;
}

// v_k c_i . u / E rounded once: x = s (y_hi + y_lo) with s = (s_hi + s_lo).
__device__ __forceinline__ float x_of(float sh, float sl, float yh, float yl) {
  return fmaf(sh, yh, fmaf(sh, yl, sl * yh));
}

// Equilibrium of label q (direction i of shell k, sign +1 for the first of the
// pair) from the node factors; used for ghost nodes.
__device__ __forceinline__ float feq32(const Eq32& e, const DvmConst<float>& d, int k, int i, float sign) {
  if (k == 0) return e.w[0] * e.a0;
  const float x = sign * x_of(d.speed[k], d.speed_lo[k], e.yh[i], e.yl[i]);
  const float x2 = x * x;
  const float ev = fmaf(x2, fmaf(x2, 1.0f / 24.0f, e.a1h), e.a0);
  const float od = x * fmaf(x2, 1.0f / 6.0f, e.a1);
  return e.w[k] * (ev + od);
}


// Node state from given fields (rho, Cartesian u, E = T).
__device__ __forceinline__ State32 state32_from_fields(float rho, float ux, float uy, float E) {
  State32 s;
  s.rho = ff_of(rho);
  s.ux = ff_of(ux);
  s.uy = ff_of(uy);
  s.E = ff_of(E);
  s.ok = rho > 0.f && E > 0.f;
  return s;
}

// Node state (rho, u_x, u_y, E) in double for the global diagnostics, from the
// FP32 path's float-float moments or the FP64 path's plain sums.
__device__ __forceinline__ void node_state_double(const float* f, size_t plane, const DvmConst<float>& d,
                                                  double& rho, double& ux, double& uy, double& E) {
  const State32 m = state32(f, plane, d);
  rho = (double)m.rho.hi + m.rho.lo;
  ux = (double)m.ux.hi + m.ux.lo;
  uy = (double)m.uy.hi + m.uy.lo;
  E = (double)m.E.hi + m.E.lo;
}
__device__ __forceinline__ void node_state_double(const double* f, size_t plane, const DvmConst<double>& d,
                                                  double& rho, double& ux, double& uy, double& E) {
  const NodeState<double> m = node_moments(f, plane, d);
  rho = m.rho; ux = m.ux; uy = m.uy; E = m.E;
}

}  // namespace pclb
