// Device helpers: TMA / mbarrier wrappers (inline PTX for sm_103a), the
// per-node moments with the double-precision temperature recovery, the
// equilibrium of Eq. (10) and the Modified Warming-Beam increment of Eq. (28).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "pclb_internal.h"

namespace pclb {

// ---------------------------------------------------------------------------
// Shared-memory barrier and tensor-copy primitives.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Make the initialised barrier visible to the asynchronous (TMA) proxy.
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Wait for the barrier phase with a time limit.  Returns false (and the
// caller reports PCLB_FLAG_TIMEOUT) if the copies did not land within
// limit_ns; the wait never spins forever.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_timer_ns() - t0 > limit_ns) return false;
  }
}

// 3-D tiled TMA load of one box into shared memory, completing on bar.
// The innermost coordinate x must be a multiple of 16 bytes / element size.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_prefetch_desc(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// ---------------------------------------------------------------------------
// Error-free transformations used by the compensated moment sums.
// ---------------------------------------------------------------------------
// a + b = s + e exactly (Knuth's two-sum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// a * b = p + e exactly (via fused multiply-add).
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}

// Macroscopic state of a node as the step needs it.
template <class T>
struct NodeState {
  T rho, ux, uy, E;
  double rho_d, E_d;  // rho and E as recovered in double (weights use these)
  bool ok;            // rho > 0, E > 0, all finite
};

// ---------------------------------------------------------------------------
// Moments of one node, Eqs. (3)-(5).  f[q * stride] for q = 0..Q-1.
// FP32: shell sums in float, then a compensated (two-sum / two-product)
// combination across the five shells; (hi, lo) pairs are merged in double and
// T = (e - |j|^2 / (2 rho)) / rho is recovered in double.
// FP64: plain double sums.
// ---------------------------------------------------------------------------
// 1/n by the Newton-Raphson iteration r <- r (2 - n r) from the hardware's
// approximate reciprocal (rcp.approx.ftz.f64: relative error <= 1e-6,
// measured 9.9e-7 over 6.7e7 arguments); each step squares the relative
// error.  Two steps reach the correctly rounded quotient in every argument
// measured; one step leaves <= 1e-12 (measured 9.9e-13).  n must be a
// positive normal number.
__device__ __forceinline__ double recip_newton(double n) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(n));
  double e = fma(-n, r, 1.0);
  r = fma(r, e, r);
  e = fma(-n, r, 1.0);
  return fma(r, e, r);
}
__device__ __forceinline__ double recip_newton1(double n) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(n));
  return fma(r, fma(-n, r, 1.0), r);
}

__device__ __forceinline__ double recip_refined(double x) {
  // Newton-Raphson step y1 = y0 (2 - x y0) on a single-precision seed.
  double y0 = (double)__frcp_rn((float)x);
  return y0 * (2.0 - x * y0);
}

// The stride type is int for shared-memory windows and size_t for global
// arrays (planes of large grids exceed 2^31 elements in total).
template <class Stride>
__device__ __forceinline__ NodeState<float> node_moments(const float* f, Stride stride,
                                                         const DvmConst<float>& d) {
  float S[5], X[5], Y[5];
  S[0] = f[0];
#pragma unroll
  for (int k = 1; k <= 4; ++k) {
    float s = 0.f, x = 0.f, y = 0.f;
#pragma unroll
    for (int i = 0; i < kNDirs; ++i) {
      const int q = 1 + (k - 1) * kNDirs + i;
      const float v = f[q * stride];
      s += v;
      x = fmaf(d.cx[q], v, x);
      y = fmaf(d.cy[q], v, y);
    }
    S[k] = s; X[k] = x; Y[k] = y;
  }
  // rho = S0 + .. + S4, jx = sum v_k X_k, jy = sum v_k Y_k, e = sum v_k^2/2 S_k
  float rh = S[0], rl = 0.f;
  float xh = 0.f, xl = 0.f, yh = 0.f, yl = 0.f, eh = 0.f, el = 0.f;
#pragma unroll
  for (int k = 1; k <= 4; ++k) {
    float s, e, p, pe;
    two_sum(rh, S[k], s, e); rh = s; rl += e;
    two_prod(d.speed[k], X[k], p, pe); two_sum(xh, p, s, e); xh = s; xl += e + pe;
    two_prod(d.speed[k], Y[k], p, pe); two_sum(yh, p, s, e); yh = s; yl += e + pe;
    two_prod(d.half_v2[k], S[k], p, pe); two_sum(eh, p, s, e); eh = s; el += e + pe;
  }
  const double rho = (double)rh + (double)rl;
  const double jx = (double)xh + (double)xl;
  const double jy = (double)yh + (double)yl;
  const double e = (double)eh + (double)el;
  const double inv = recip_refined(rho);
  const double ux = jx * inv, uy = jy * inv;
  const double E = (e - 0.5 * (jx * ux + jy * uy)) * inv;
  NodeState<float> st;
  st.rho = (float)rho; st.ux = (float)ux; st.uy = (float)uy; st.E = (float)E;
  st.rho_d = rho; st.E_d = E;
  st.ok = (rho > 0.0) && (E > 0.0) && isfinite(e) && isfinite(jx) && isfinite(jy);
  return st;
}

template <class Stride>
__device__ __forceinline__ NodeState<double> node_moments(const double* f, Stride stride,
                                                          const DvmConst<double>& d) {
  double s0 = 0.0, sx = 0.0, sy = 0.0, se = 0.0;
#pragma unroll
  for (int q = 0; q < kQ; ++q) {
    const double v = f[q * stride];
    s0 += v;
    sx = fma(d.vx[q], v, sx);
    sy = fma(d.vy[q], v, sy);
    se = fma(d.half_v2[d.shell[q]], v, se);
  }
  const double inv = 1.0 / s0;
  const double ux = sx * inv, uy = sy * inv;
  const double E = (se - 0.5 * (sx * ux + sy * uy)) * inv;
  NodeState<double> st;
  st.rho = s0; st.ux = ux; st.uy = uy; st.E = E;
  st.rho_d = s0; st.E_d = E;
  st.ok = (s0 > 0.0) && (E > 0.0) && isfinite(se) && isfinite(sx) && isfinite(sy);
  return st;
}

// ---------------------------------------------------------------------------
// Equilibrium, Eq. (10), factored per node:
//   f^eq_q = rho F_k(E) [a0 + x (a1 + x (a1/2 + x (1/6 + x/24)))],
//   x = v_q . u / E,  a1 = 1 - u^2/(2E),  a0 = a1 + u^4/(8E^2).
// ---------------------------------------------------------------------------
template <class T>
struct EqParams {
  T w[5];        // rho F_k(E), k = 0..4
  T a0, a1, a1h; // polynomial coefficients
  T uxE, uyE;    // u / E
};

// ---- float-float helpers (an unevaluated sum hi + lo of two floats) --------
struct ff {
  float hi, lo;
};
__device__ __forceinline__ ff ff_from(double x) {
  ff r;
  r.hi = (float)x;
  r.lo = (float)(x - (double)r.hi);
  return r;
}
// a * b + c with every operand a float-float pair (Horner step).  Uses the
// error-free product (via fma) and sum above; relative error ~ 2^-44.
__device__ __forceinline__ ff ff_mul_add(ff a, ff b, ff c) {
  float p, pe, s, se;
  two_prod(a.hi, b.hi, p, pe);
  pe = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, pe));
  two_sum(p, c.hi, s, se);
  const float lo = se + (pe + c.lo);
  ff r;
  r.hi = __fadd_rn(s, lo);
  r.lo = __fsub_rn(lo, __fsub_rn(r.hi, s));
  return r;
}
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  float p, e;
  two_prod(a.hi, b.hi, p, e);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  ff r;
  r.hi = __fadd_rn(p, e);
  r.lo = __fsub_rn(e, __fsub_rn(r.hi, p));
  return r;
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  float s, se;
  two_sum(a.hi, b.hi, s, se);
  const float lo = se + (a.lo + b.lo);
  ff r;
  r.hi = __fadd_rn(s, lo);
  r.lo = __fsub_rn(lo, __fsub_rn(r.hi, s));
  return r;
}

__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_scale(ff a, float s) { return ff{a.hi * s, a.lo * s}; }  // s a power of 2
// 1 / a: single-precision seed refined by one Newton step on the float-float value.
__device__ __forceinline__ ff ff_recip(ff a) {
  const float r0 = __frcp_rn(a.hi);
  const float e = fmaf(-a.hi, r0, 1.0f) - a.lo * r0;   // 1 - a r0
  ff r;
  r.hi = r0;
  r.lo = r0 * e;
  const float s = __fadd_rn(r.hi, r.lo);
  r.lo = __fsub_rn(r.lo, __fsub_rn(s, r.hi));
  r.hi = s;
  return r;
}

// Weights rho F_k(E) of Eqs. (11a)-(11b).  The polynomial in E cancels
// heavily (|terms| ~ 15 |F_k| for the octagon speeds), so the FP32 path
// evaluates it in float-float from the double-precision rho and E and rounds
// only the final products; FP64 uses plain double Horner.
__device__ __forceinline__ void shell_weights(double rho, double E, const DvmConst<float>& d, float w[5]) {
  const ff e = ff_from(E), r = ff_from(rho);
  ff sum;
  sum.hi = 0.f;
  sum.lo = 0.f;
#pragma unroll
  for (int k = 1; k <= 4; ++k) {
    ff a = {d.Fc[k][3], d.Fc_lo[k][3]};
#pragma unroll
    for (int n = 2; n >= 0; --n) a = ff_mul_add(a, e, ff{d.Fc[k][n], d.Fc_lo[k][n]});
    a = ff_mul(a, e);
    sum = ff_add(sum, a);
    const ff wk = ff_mul(r, a);
    w[k] = wk.hi + wk.lo;
  }
  // F_0 = 1 - B0 sum F_k
  ff b0s = ff_mul(ff{-d.B0, 0.f}, sum);
  ff f0 = ff_add(ff{1.f, 0.f}, b0s);
  const ff w0 = ff_mul(r, f0);
  w[0] = w0.hi + w0.lo;
}

__device__ __forceinline__ void shell_weights(double rho, double E, const DvmConst<double>& d, double w[5]) {
  double Fsum = 0.0;
#pragma unroll
  for (int k = 1; k <= 4; ++k) {
    const double F = E * (d.Fc[k][0] + E * (d.Fc[k][1] + E * (d.Fc[k][2] + E * d.Fc[k][3])));
    w[k] = rho * F;
    Fsum += F;
  }
  w[0] = rho * (1.0 - d.B0 * Fsum);
}

template <class T>
__device__ __forceinline__ EqParams<T> eq_params(double rho, T ux, T uy, double E, const DvmConst<T>& d) {
  EqParams<T> p;
  shell_weights(rho, E, d, p.w);
  const T Ef = (T)E;
  const T invE = T(1) / Ef;
  const T u2E = (ux * ux + uy * uy) * invE;   // u^2 / E
  p.a1 = T(1) - T(0.5) * u2E;
  p.a0 = p.a1 + T(0.125) * u2E * u2E;
  p.a1h = T(0.5) * p.a1;
  p.uxE = ux * invE;
  p.uyE = uy * invE;
  return p;
}

template <class T>
__device__ __forceinline__ T feq_q(const EqParams<T>& p, T vx, T vy, int k) {
  const T x = vx * p.uxE + vy * p.uyE;
  const T poly = p.a0 + x * (p.a1 + x * (p.a1h + x * (T(1.0 / 6.0) + x * T(1.0 / 24.0))));
  return p.w[k] * poly;
}

// ---------------------------------------------------------------------------
// Convection increments in upwind form, as the step kernels evaluate them.
// With the upstream values u1 = psi_{j-s}, u2 = psi_{j-2s} (s = sign of C,
// s = +1 for C >= 0), D = psi_j - u1, Dp = u1 - u2, the downwind neighbour
// d1 = psi_{j+s}, a = |C| and K = a (1 - a):
//   MWB (Eq. 28)          a D + K h,  h = |D| (D - Dp) / (|D| + |Dp|)
//                         (h = 0 when D = Dp = 0): the paper's bracket
//                         [C + C(1-|C|)(1-S(eta))(1-eta)/2] delta wherever
//                         eta = Dp / D is defined, its continuous extension
//                         elsewhere;
//   Warming-Beam (Eq. 25) a D + K (D - Dp) / 2;
//   Lax-Wendroff          a D + K (Dd - D) / 2,   Dd = d1 - psi_j;
//   2nd-order upwind      a D + a (D - Dp) / 2   (forward Euler with Eq. 23).
// ---------------------------------------------------------------------------

}  // namespace pclb
