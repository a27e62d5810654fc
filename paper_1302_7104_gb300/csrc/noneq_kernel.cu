// Non-equilibrium manifestations of Sec. IV, one node per thread.
//
// For the weights w_q = f_q (moments) or w_q = f_q - f^eq_q (departures) and
// the velocities c_q = v_q (plain) or c_q = v_q - u (central), in polar
// components at the node, the groups are
//   M_2 = sum w c c (rr, r theta, theta theta),
//   M_3 = sum w c c c (rrr, rr theta, r theta theta, theta theta theta),
//   M_{3,1} = sum w (c.c/2) c (r, theta),
//   M_{4,2} = sum w (c.c/2) c c (rr, r theta, theta theta),
// for each requested group: M_m(f), Delta_m = M_m(f - f^eq), M*_m(f) and
// Delta*_m = M*_m(f - f^eq).
//
// One pass accumulates the 12 central moments M*_m(f) of the node.  The
// others follow per node:
//   * Delta*_m = M*_m(f) - M*_m(f^eq), and the central moments of the model's
//     equilibrium are those of the Maxwellian, (rho E I, 0, 0, 2 rho E^2 I)
//     (the relations the velocity set is built to satisfy, Eqs. 6-9);
//   * the plain moments from the central ones with v = u + c: with
//     S = M*_2, T = M*_3, V = M*_{3,1}, Q = M*_{4,2} and sum w c = 0,
//       M_2 = S + rho u u,
//       M_3 = T + (u S + S u + ...: the three placements of u) + rho u u u,
//       M_{3,1} = V + S u + u tr(S)/2 + rho u |u|^2/2,
//       M_{4,2} = Q + u V + V u + u.T + u u tr(S)/2 + u (S u) + (S u) u
//                 + |u|^2/2 S + rho |u|^2/2 u u;
//     the departures the same way from Delta*_m with rho replaced by
//     sum (f - f^eq) = 0 (f and f^eq share mass, momentum and energy).
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "dvm_generic.h"
#include "f32_state.cuh"
#include "pclb_internal.h"

namespace pclb {

namespace {

constexpr int kNeqThreads = 128;

// rho, u and E of the node in the precision of the step kernels (float-float
// moments in FP32), and rho E, 2 rho E^2 in double.
__device__ __forceinline__ void neq_state(const float* f, size_t plane, const DvmConst<float>& d, float& rho,
                                          float& ux, float& uy, bool& ok, double& rE, double& rE2) {
  const State32 s = state32(f, plane, d);
  const double R = (double)s.rho.hi + s.rho.lo, E = (double)s.E.hi + s.E.lo;
  rho = (float)R;
  ux = s.ux.hi + s.ux.lo;
  uy = s.uy.hi + s.uy.lo;
  ok = s.ok;
  rE = R * E;
  rE2 = 2.0 * R * E * E;
}

__device__ __forceinline__ void neq_state(const double* f, size_t plane, const DvmConst<double>& d, double& rho,
                                          double& ux, double& uy, bool& ok, double& rE, double& rE2) {
  const NodeState<double> m = node_moments(f, plane, d);
  rho = m.rho;
  ux = m.ux;
  uy = m.uy;
  ok = m.ok;
  rE = m.rho_d * m.E_d;
  rE2 = 2.0 * m.rho_d * m.E_d * m.E_d;
}

// Plain moments (12 components, order as above) from central ones C with
// density R (0 for departures) and velocity (ur, ut), polar components.
template <class T>
__device__ __forceinline__ void plain_from_central(T R, T ur, T ut, const T* C, T* M) {
  const T Srr = C[0], Srt = C[1], Stt = C[2];
  const T Trrr = C[3], Trrt = C[4], Trtt = C[5], Tttt = C[6];
  const T Vr = C[7], Vt = C[8];
  const T trS2 = T(0.5) * (Srr + Stt);
  const T u2 = T(0.5) * (ur * ur + ut * ut);
  const T Sur = Srr * ur + Srt * ut, Sut = Srt * ur + Stt * ut;   // S u
  M[0] = Srr + R * ur * ur;
  M[1] = Srt + R * ur * ut;
  M[2] = Stt + R * ut * ut;
  M[3] = Trrr + T(3) * ur * Srr + R * ur * ur * ur;
  M[4] = Trrt + T(2) * ur * Srt + ut * Srr + R * ur * ur * ut;
  M[5] = Trtt + ur * Stt + T(2) * ut * Srt + R * ur * ut * ut;
  M[6] = Tttt + T(3) * ut * Stt + R * ut * ut * ut;
  M[7] = Vr + Sur + ur * trS2 + R * ur * u2;
  M[8] = Vt + Sut + ut * trS2 + R * ut * u2;
  // u.T for the pairs (rr, rt, tt): u_r T_r.. + u_t T_t..
  const T uTrr = ur * Trrr + ut * Trrt, uTrt = ur * Trrt + ut * Trtt, uTtt = ur * Trtt + ut * Tttt;
  M[9] = C[9] + T(2) * ur * Vr + uTrr + ur * ur * trS2 + T(2) * ur * Sur + u2 * Srr + R * u2 * ur * ur;
  M[10] = C[10] + ur * Vt + ut * Vr + uTrt + ur * ut * trS2 + ur * Sut + ut * Sur + u2 * Srt + R * u2 * ur * ut;
  M[11] = C[11] + T(2) * ut * Vt + uTtt + ut * ut * trS2 + T(2) * ut * Sut + u2 * Stt + R * u2 * ut * ut;
}

}  // namespace

template <class T>
__global__ void __launch_bounds__(kNeqThreads)
    noneq_kernel(const T* __restrict__ f, T* __restrict__ out, int groups, const __grid_constant__ StepParams p,
                 const __grid_constant__ DvmConst<T> d) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int t = blockIdx.y;
  if (r >= p.n_r || t >= p.n_theta) return;
  const size_t plane = (size_t)p.rows * p.pitch;
  const T* fn = f + (size_t)(t + kGhostRows) * p.pitch + r;
  T rho, ux, uy;
  bool ok;
  double rE, rE2;
  neq_state(fn, plane, d, rho, ux, uy, ok, rE, rE2);
  if (!ok) atomicOr(p.status, PCLB_FLAG_NONPHYS);
  const T cs = (T)p.cos_t[t], sn = (T)p.sin_t[t];
  const T u_r = ux * cs + uy * sn, u_t = uy * cs - ux * sn;

  // central moments of f
  T A[12];
#pragma unroll
  for (int c = 0; c < 12; ++c) A[c] = T(0);
#pragma unroll
  for (int q = 0; q < kQ; ++q) {
    const T w = fn[(size_t)q * plane];
    const T cr = d.vx[q] * cs + d.vy[q] * sn - u_r, ct = d.vy[q] * cs - d.vx[q] * sn - u_t;
    const T h = T(0.5) * (cr * cr + ct * ct);
    const T wr = w * cr, wt = w * ct;
    const T wrr = wr * cr, wrt = wr * ct, wtt = wt * ct;
    A[0] += wrr;
    A[1] += wrt;
    A[2] += wtt;
    A[3] += wrr * cr;
    A[4] += wrr * ct;
    A[5] += wrt * ct;
    A[6] += wtt * ct;
    A[7] += h * wr;
    A[8] += h * wt;
    A[9] += h * wrr;
    A[10] += h * wrt;
    A[11] += h * wtt;
  }
  // central departures: minus the equilibrium's (rho E I, 0, 0, 2 rho E^2 I)
  T D[12];
#pragma unroll
  for (int c = 0; c < 12; ++c) D[c] = A[c];
  D[0] = (T)((double)A[0] - rE);
  D[2] = (T)((double)A[2] - rE);
  D[9] = (T)((double)A[9] - rE2);
  D[11] = (T)((double)A[11] - rE2);

  const size_t nodes = (size_t)p.n_theta * p.n_r, n = (size_t)t * p.n_r + r;
  int slot = 0;
  T out_g[12];
#pragma unroll 1
  for (int g = 0; g < 4; ++g) {
    if (!(groups & (1 << g))) continue;
    if (g == 0) plain_from_central<T>(rho, u_r, u_t, A, out_g);
    else if (g == 1) plain_from_central<T>(T(0), u_r, u_t, D, out_g);
    else if (g == 2)
      for (int c = 0; c < 12; ++c) out_g[c] = A[c];
    else
      for (int c = 0; c < 12; ++c) out_g[c] = D[c];
#pragma unroll
    for (int c = 0; c < 12; ++c) out[(size_t)(slot * 12 + c) * nodes + n] = out_g[c];
    ++slot;
  }
}

// The same for the N_i = 16 and 24 sets of Table I (Q = 65, 97, built to
// reproduce the same equilibrium moments, Eqs. 6-9): the node's moments in
// double (one pass over its Q values), the central moments in the storage
// type with the velocities of the set (float tables for FP32).
template <class T>
__global__ void __launch_bounds__(kNeqThreads)
    noneq_gen_kernel(const T* __restrict__ f, T* __restrict__ out, int groups, const __grid_constant__ StepParams p,
                     const __grid_constant__ DvmG d, const __grid_constant__ DvmG32 c) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int t = blockIdx.y;
  if (r >= p.n_r || t >= p.n_theta) return;
  const size_t plane = (size_t)p.rows * p.pitch;
  const T* fn = f + (size_t)(t + kGhostRows) * p.pitch + r;
  // rho, rho u, rho (E + u^2/2) (Eqs. 3-5), then u and E
  double s0 = 0.0, sx = 0.0, sy = 0.0, se = 0.0;
  for (int q = 0; q < d.q; ++q) {
    const double v = (double)fn[(size_t)q * plane];
    s0 += v;
    sx = fma(d.vx[q], v, sx);
    sy = fma(d.vy[q], v, sy);
    se = fma(d.half_v2[d.shell[q]], v, se);
  }
  const double uxd = sx / s0, uyd = sy / s0;
  const double E = (se - 0.5 * (sx * uxd + sy * uyd)) / s0;
  if (!(s0 > 0.0 && E > 0.0 && isfinite(E) && isfinite(uxd) && isfinite(uyd))) atomicOr(p.status, PCLB_FLAG_NONPHYS);
  const double rE = s0 * E, rE2 = 2.0 * s0 * E * E;
  const T rho = (T)s0, ux = (T)uxd, uy = (T)uyd;
  const T cs = (T)p.cos_t[t], sn = (T)p.sin_t[t];
  const T u_r = ux * cs + uy * sn, u_t = uy * cs - ux * sn;

  // central moments of f
  T A[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) A[k] = T(0);
  for (int q = 0; q < d.q; ++q) {
    const T w = fn[(size_t)q * plane];
    T vx, vy;
    if constexpr (sizeof(T) == 4) {
      vx = c.vx[q];
      vy = c.vy[q];
    } else {
      vx = d.vx[q];
      vy = d.vy[q];
    }
    const T cr = vx * cs + vy * sn - u_r, ct = vy * cs - vx * sn - u_t;
    const T h = T(0.5) * (cr * cr + ct * ct);
    const T wr = w * cr, wt = w * ct;
    const T wrr = wr * cr, wrt = wr * ct, wtt = wt * ct;
    A[0] += wrr;
    A[1] += wrt;
    A[2] += wtt;
    A[3] += wrr * cr;
    A[4] += wrr * ct;
    A[5] += wrt * ct;
    A[6] += wtt * ct;
    A[7] += h * wr;
    A[8] += h * wt;
    A[9] += h * wrr;
    A[10] += h * wrt;
    A[11] += h * wtt;
  }
  // central departures: minus the equilibrium's (rho E I, 0, 0, 2 rho E^2 I)
  T D[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) D[k] = A[k];
  D[0] = (T)((double)A[0] - rE);
  D[2] = (T)((double)A[2] - rE);
  D[9] = (T)((double)A[9] - rE2);
  D[11] = (T)((double)A[11] - rE2);

  const size_t nodes = (size_t)p.n_theta * p.n_r, n = (size_t)t * p.n_r + r;
  int slot = 0;
  T out_g[12];
#pragma unroll 1
  for (int g = 0; g < 4; ++g) {
    if (!(groups & (1 << g))) continue;
    if (g == 0) plain_from_central<T>(rho, u_r, u_t, A, out_g);
    else if (g == 1) plain_from_central<T>(T(0), u_r, u_t, D, out_g);
    else if (g == 2)
      for (int k = 0; k < 12; ++k) out_g[k] = A[k];
    else
      for (int k = 0; k < 12; ++k) out_g[k] = D[k];
#pragma unroll
    for (int k = 0; k < 12; ++k) out[(size_t)(slot * 12 + k) * nodes + n] = out_g[k];
    ++slot;
  }
}

template <class T>
cudaError_t launch_noneq_gen(const T* f, T* out, int groups, const StepParams& p, const DvmG& d, const DvmG32& c,
                             cudaStream_t s) {
  dim3 grid((p.n_r + kNeqThreads - 1) / kNeqThreads, p.n_theta);
  noneq_gen_kernel<T><<<grid, kNeqThreads, 0, s>>>(f, out, groups, p, d, c);
  return cudaGetLastError();
}

template cudaError_t launch_noneq_gen<float>(const float*, float*, int, const StepParams&, const DvmG&, const DvmG32&,
                                             cudaStream_t);
template cudaError_t launch_noneq_gen<double>(const double*, double*, int, const StepParams&, const DvmG&,
                                              const DvmG32&, cudaStream_t);

template <class T>
cudaError_t launch_noneq(const T* f, T* out, int groups, const StepParams& p, const DvmConst<T>& d,
                         cudaStream_t s) {
  dim3 grid((p.n_r + kNeqThreads - 1) / kNeqThreads, p.n_theta);
  noneq_kernel<T><<<grid, kNeqThreads, 0, s>>>(f, out, groups, p, d);
  return cudaGetLastError();
}

template cudaError_t launch_noneq<float>(const float*, float*, int, const StepParams&, const DvmConst<float>&,
                                         cudaStream_t);
template cudaError_t launch_noneq<double>(const double*, double*, int, const StepParams&, const DvmConst<double>&,
                                          cudaStream_t);

}  // namespace pclb
