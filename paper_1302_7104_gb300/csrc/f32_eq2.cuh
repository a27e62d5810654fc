// FP32 path: the node state and equilibrium factors of two radially adjacent
// nodes in packed FP32x2 float-float arithmetic (Eqs. 10-11), shared by the
// step and the set-state kernel.
#pragma once

#include "device_common.cuh"
#include "f32_state.cuh"
#include "f32x2.cuh"

namespace pclb {

// Unit vectors of the first direction of each opposite pair, i = 0..3 of the
// octagon (Eq. 2), as float-float pairs: (1,0), (s,s), (0,1), (-s,s), s = 1/sqrt 2.
constexpr float kS = 0.7071067690849304f;
constexpr float kSl = 1.2101617152815436e-08f;

struct State2 {
  ff2 rho, ux, uy, E;
};

__device__ __forceinline__ ff2 ffc(float hi, float lo) { return ff2{bc2(hi), bc2(lo)}; }

struct Eq2 {
  f2 w[5];                  // rho F_k(E)
  f2 a0, a1, a1h;           // Eq. (10) polynomial coefficients
  f2 yh[kHalf], yl[kHalf];  // c_i . u / E, float-float
};

__device__ __forceinline__ Eq2 eq2(const State2& s, const DvmConst<float>& d) {
  Eq2 q;
  ff2 sum = ff2_of(bc2(0.f));
#pragma unroll
  for (int k = 1; k <= 4; ++k) {
    ff2 a = ffc(d.Fc[k][3], d.Fc_lo[k][3]);
#pragma unroll
    for (int n = 2; n >= 0; --n) a = ff2_mul_add(a, s.E, ffc(d.Fc[k][n], d.Fc_lo[k][n]));
    a = ff2_mul(a, s.E);                               // F_k(E)
    sum = ff2_add(sum, a);
    q.w[k] = ff2_round(ff2_mul(s.rho, a));
  }
  const ff2 f0 = ff2_add(ff2_of(bc2(1.f)), ff2_mul(ff2_of(bc2(-d.B0)), sum));   // F_0
  q.w[0] = ff2_round(ff2_mul(s.rho, f0));
  const ff2 invE = ff2_recip(s.E);
  const ff2 uxE = ff2_mul(s.ux, invE), uyE = ff2_mul(s.uy, invE);
  const ff2 u2E = ff2_add(ff2_mul(s.ux, uxE), ff2_mul(s.uy, uyE));   // u^2 / E
  const ff2 a1 = ff2_add(ff2_of(bc2(1.f)), ff2_scale(u2E, -0.5f));
  const ff2 a0 = ff2_add(a1, ff2_scale(ff2_mul(u2E, u2E), 0.125f));
  q.a1 = ff2_round(a1);
  q.a0 = ff2_round(a0);
  q.a1h = mul2(bc2(0.5f), q.a1);
  const ff2 sq = ffc(kS, kSl);
  const ff2 y1 = ff2_mul(sq, ff2_add(uxE, uyE));
  const ff2 y3 = ff2_mul(sq, ff2_add(uyE, ff2{neg2(uxE.hi), neg2(uxE.lo)}));
  q.yh[0] = uxE.hi; q.yl[0] = uxE.lo;
  q.yh[1] = y1.hi;  q.yl[1] = y1.lo;
  q.yh[2] = uyE.hi; q.yl[2] = uyE.lo;
  q.yh[3] = y3.hi;  q.yl[3] = y3.lo;
  return q;
}

// Equilibrium (Eq. 10) of direction i of a shell (speed sh + sl, weight wk =
// rho F_k) and of its opposite direction: with x = v.u/E, P(+x) = ev + od and
// P(-x) = ev - od share the even and odd parts of the polynomial; the pair
// is formed as w ev +- w od with fused multiply-adds.
__device__ __forceinline__ void feq_pair2(const Eq2& eq, f2 sh, f2 sl, int i, f2 wk, f2& fp, f2& fm) {
  const f2 x = fma2(sh, eq.yh[i], fma2(sh, eq.yl[i], mul2(sl, eq.yh[i])));
  const f2 x2 = mul2(x, x);
  const f2 ev = fma2(x2, fma2(x2, bc2(1.0f / 24.0f), eq.a1h), eq.a0);
  const f2 od = mul2(x, fma2(x2, bc2(1.0f / 6.0f), eq.a1));
  const f2 wev = mul2(wk, ev);                     // w (ev +- od) with one rounding after w ev
  fp = fma2(wk, od, wev);
  fm = fma2(neg2(wk), od, wev);
}

}  // namespace pclb
