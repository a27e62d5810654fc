// Non-equilibrium manifestations of Sec. IV, one node per thread.
//
// For the weights w_q = f_q (moments) or w_q = f_q - f^eq_q (departures) and
// the velocities c_q = v_q (plain) or c_q = v_q - u (central), in polar
// components at the node, the kernel forms
//   M_2 = sum w c c (rr, r theta, theta theta),
//   M_3 = sum w c c c (rrr, rr theta, r theta theta, theta theta theta),
//   M_{3,1} = sum w (c.c/2) c (r, theta),
//   M_{4,2} = sum w (c.c/2) c c (rr, r theta, theta theta),
// for each requested group: M_m(f), Delta_m = M_m(f - f^eq), M*_m(f) and
// Delta*_m = M*_m(f - f^eq).  f^eq is the equilibrium of Eq. (10) at the
// node's own moments (Eqs. 3-5), evaluated exactly as the step kernels do.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "f32_state.cuh"
#include "pclb_internal.h"

namespace pclb {

namespace {

constexpr int kNeqThreads = 128;

// Node state and equilibrium factors in the precision of the step kernels.
__device__ __forceinline__ void neq_state(const float* f, size_t plane, const DvmConst<float>& d, float& rho,
                                          float& ux, float& uy, bool& ok, Eq32& e) {
  const State32 s = state32(f, plane, d);
  e = eq32(s, d);
  rho = s.rho.hi + s.rho.lo;
  ux = s.ux.hi + s.ux.lo;
  uy = s.uy.hi + s.uy.lo;
  ok = s.ok;
}
// label q = 1 + (k - 1) N_i + i: shell k, direction i (q = 0: rest)
__device__ __forceinline__ float neq_feq(const Eq32& e, const DvmConst<float>& d, int q) {
  if (q == 0) return feq32(e, d, 0, 0, 1.f);
  const int k = 1 + (q - 1) / kNDirs, i = (q - 1) % kNDirs;
  return i < kHalf ? feq32(e, d, k, i, 1.f) : feq32(e, d, k, i - kHalf, -1.f);
}

__device__ __forceinline__ void neq_state(const double* f, size_t plane, const DvmConst<double>& d, double& rho,
                                          double& ux, double& uy, bool& ok, EqParams<double>& e) {
  const NodeState<double> m = node_moments(f, plane, d);
  e = eq_params<double>(m.rho_d, m.ux, m.uy, m.E_d, d);
  rho = m.rho;
  ux = m.ux;
  uy = m.uy;
  ok = m.ok;
}
__device__ __forceinline__ double neq_feq(const EqParams<double>& e, const DvmConst<double>& d, int q) {
  return feq_q<double>(e, d.vx[q], d.vy[q], q == 0 ? 0 : 1 + (q - 1) / kNDirs);
}

template <class T>
struct NeqEq;
template <>
struct NeqEq<float> {
  using type = Eq32;
};
template <>
struct NeqEq<double> {
  using type = EqParams<double>;
};

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
  typename NeqEq<T>::type e;
  neq_state(fn, plane, d, rho, ux, uy, ok, e);
  if (!ok) atomicOr(p.status, PCLB_FLAG_NONPHYS);
  const T cs = (T)p.cos_t[t], sn = (T)p.sin_t[t];
  const T u_r = ux * cs + uy * sn, u_t = uy * cs - ux * sn;

  T m[4][12];
#pragma unroll
  for (int g = 0; g < 4; ++g)
#pragma unroll
    for (int c = 0; c < 12; ++c) m[g][c] = T(0);
#pragma unroll
  for (int q = 0; q < kQ; ++q) {
    const T fq = fn[(size_t)q * plane];
    const T dq = fq - neq_feq(e, d, q);
    const T vr = d.vx[q] * cs + d.vy[q] * sn, vt = d.vy[q] * cs - d.vx[q] * sn;
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      if (!(groups & (1 << g))) continue;
      const T w = (g == 1 || g == 3) ? dq : fq;
      const T cr = g >= 2 ? vr - u_r : vr, ct = g >= 2 ? vt - u_t : vt;
      const T h = T(0.5) * (cr * cr + ct * ct);
      const T wr = w * cr, wt = w * ct;
      m[g][0] += wr * cr;
      m[g][1] += wr * ct;
      m[g][2] += wt * ct;
      m[g][3] += wr * cr * cr;
      m[g][4] += wr * cr * ct;
      m[g][5] += wr * ct * ct;
      m[g][6] += wt * ct * ct;
      m[g][7] += h * wr;
      m[g][8] += h * wt;
      m[g][9] += h * wr * cr;
      m[g][10] += h * wr * ct;
      m[g][11] += h * wt * ct;
    }
  }
  const size_t nodes = (size_t)p.n_theta * p.n_r, n = (size_t)t * p.n_r + r;
  int slot = 0;
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    if (!(groups & (1 << g))) continue;
#pragma unroll
    for (int c = 0; c < 12; ++c) out[(size_t)(slot * 12 + c) * nodes + n] = m[g][c];
    ++slot;
  }
}

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
