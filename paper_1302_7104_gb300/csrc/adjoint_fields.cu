// Adjoints of the two maps between fields and distributions:
//   * moments (Eqs. 3-5 as returned by pclb_moments): lam_q = sum over the
//     fields of g_field d field / d f_q, with d rho/d f_q = 1,
//     d u_r/d f_q = (v_r,q - u_r)/rho, d u_theta/d f_q = (v_theta,q - u_theta)/rho,
//     d T/d f_q = (|v_q - u|^2/2 - T)/rho;
//   * the equilibrium initialisation f = f^eq(rho, u, T) (Eq. 10): the field
//     gradients are the equilibrium cotangent rotated to polar components.
#include <cuda_runtime.h>

#include "adjoint_common.cuh"
#include "device_common.cuh"
#include "pclb_internal.h"

namespace pclb {

template <class T>
__device__ __forceinline__ void store_ghosted(T* f, const StepParams& p, const DvmConst<T>& d, int q, int t,
                                              int r, T v) {
  const size_t plane = (size_t)p.rows * p.pitch;
  f[(size_t)q * plane + (size_t)(t + kGhostRows) * p.pitch + r] = v;
  if (t >= p.n_theta - 2) f[(size_t)d.recv_lo[q] * plane + (size_t)(t - (p.n_theta - 2)) * p.pitch + r] = v;
  if (t < 2) f[(size_t)d.recv_hi[q] * plane + (size_t)(p.n_theta + kGhostRows + t) * p.pitch + r] = v;
}

template <class T>
__global__ void moments_vjp_kernel(const T* __restrict__ f, const T* g_rho, const T* g_ur, const T* g_ut,
                                   const T* g_T, T* __restrict__ lam, const __grid_constant__ StepParams p, const __grid_constant__ DvmConst<T> d) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int t = blockIdx.y;
  if (r >= p.n_r || t >= p.n_theta) return;
  const size_t plane = (size_t)p.rows * p.pitch;
  const NodeState<T> m = node_moments(f + (size_t)(t + kGhostRows) * p.pitch + r, plane, d);
  const size_t n = (size_t)t * p.n_r + r;
  const T c = (T)p.cos_t[t], s = (T)p.sin_t[t];
  const T gr = g_rho ? g_rho[n] : T(0), gu = g_ur ? g_ur[n] : T(0), gv = g_ut ? g_ut[n] : T(0),
          gT = g_T ? g_T[n] : T(0);
  const T inv = T(1) / m.rho;
  const T ur = m.ux * c + m.uy * s, ut = m.uy * c - m.ux * s;
  for (int q = 0; q < kQ; ++q) {
    const T vx = d.vx[q], vy = d.vy[q];
    const T vr = vx * c + vy * s, vt = vy * c - vx * s;
    const T cx = vx - m.ux, cy = vy - m.uy;
    const T l = gr + (gu * (vr - ur) + gv * (vt - ut) + gT * (T(0.5) * (cx * cx + cy * cy) - m.E)) * inv;
    store_ghosted<T>(lam, p, d, q, t, r, l);
  }
}

template <class T>
__global__ void set_state_vjp_kernel(const T* __restrict__ rho, const T* __restrict__ u_r,
                                     const T* __restrict__ u_t, const T* __restrict__ temp,
                                     const T* __restrict__ lam, T* g_rho, T* g_ur, T* g_ut, T* g_T,
                                     const __grid_constant__ StepParams p, const __grid_constant__ DvmConst<T> d) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int t = blockIdx.y;
  if (r >= p.n_r || t >= p.n_theta) return;
  const size_t n = (size_t)t * p.n_r + r;
  const size_t plane = (size_t)p.rows * p.pitch;
  const T c = (T)p.cos_t[t], s = (T)p.sin_t[t];
  const T ux = u_r[n] * c - u_t[n] * s, uy = u_r[n] * s + u_t[n] * c;
  const T* lp = lam + (size_t)(t + kGhostRows) * p.pitch + r;
  T G[4];
  eq_cotangent<T>(rho[n], ux, uy, temp[n], d, [&](int q) -> T { return lp[(size_t)q * plane]; }, G);
  if (g_rho) g_rho[n] = G[0];
  if (g_ur) g_ur[n] = G[1] * c + G[2] * s;
  if (g_ut) g_ut[n] = G[2] * c - G[1] * s;
  if (g_T) g_T[n] = G[3];   // E = T for gamma = 2
}

constexpr int kVjpThreads = 128;

template <class T>
cudaError_t launch_moments_vjp(const T* f, const T* gr, const T* gu, const T* gv, const T* gT, T* lam,
                               const StepParams& p, const DvmConst<T>& d, cudaStream_t s) {
  dim3 grid((p.n_r + kVjpThreads - 1) / kVjpThreads, p.n_theta);
  moments_vjp_kernel<T><<<grid, kVjpThreads, 0, s>>>(f, gr, gu, gv, gT, lam, p, d);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_set_state_vjp(const T* rho, const T* ur, const T* ut, const T* temp, const T* lam, T* gr,
                                 T* gu, T* gv, T* gT, const StepParams& p, const DvmConst<T>& d, cudaStream_t s) {
  dim3 grid((p.n_r + kVjpThreads - 1) / kVjpThreads, p.n_theta);
  set_state_vjp_kernel<T><<<grid, kVjpThreads, 0, s>>>(rho, ur, ut, temp, lam, gr, gu, gv, gT, p, d);
  return cudaGetLastError();
}

#define PCLB_VJP_INSTANTIATE(T)                                                                          \
  template cudaError_t launch_moments_vjp<T>(const T*, const T*, const T*, const T*, const T*, T*,      \
                                             const StepParams&, const DvmConst<T>&, cudaStream_t);      \
  template cudaError_t launch_set_state_vjp<T>(const T*, const T*, const T*, const T*, const T*, T*, T*, \
                                               T*, T*, const StepParams&, const DvmConst<T>&, cudaStream_t);
PCLB_VJP_INSTANTIATE(float)
PCLB_VJP_INSTANTIATE(double)

}  // namespace pclb
