// Per-node kernels around the step: equilibrium initialisation (f = f^eq of
// given fields, Eq. 10), macroscopic fields out (Eqs. 3-5), copies between
// the packed [Q][n_theta][n_r] layout and the stored layout (with azimuthal
// ghost rows and padded rows), and the global diagnostics reduction.
#include <cuda_runtime.h>
#include <float.h>

#include "device_common.cuh"
#include "f32_eq2.cuh"
#include "f32_state.cuh"
#include "pclb_internal.h"

namespace pclb {

// Write value v of label q at interior row t, column r of the stored layout,
// together with its copies in the azimuthal ghost rows (Eq. 40).
template <class T>
__device__ __forceinline__ void store_with_ghosts(T* f, const StepParams& p, const DvmConst<T>& d,
                                                  int q, int t, int r, T v) {
  const size_t plane = (size_t)p.rows * p.pitch;
  f[(size_t)q * plane + (size_t)(t + kGhostRows) * p.pitch + r] = v;
  if (t >= p.n_theta - 2)
    f[(size_t)d.recv_lo[q] * plane + (size_t)(t - (p.n_theta - 2)) * p.pitch + r] = v;
  if (t < 2) f[(size_t)d.recv_hi[q] * plane + (size_t)(p.n_theta + kGhostRows + t) * p.pitch + r] = v;
}

template <class T>
__global__ void set_state_kernel(T* __restrict__ f, const T* __restrict__ rho, const T* __restrict__ u_r,
                                 const T* __restrict__ u_t, const T* __restrict__ temp,
                                 const __grid_constant__ StepParams p, const __grid_constant__ DvmConst<T> d,
                                 int t_begin) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int t = blockIdx.y + t_begin;
  if (r >= p.n_r || t >= p.n_theta) return;
  const size_t n = (size_t)t * p.n_r + r;
  const T c = (T)p.cos_t[t], s = (T)p.sin_t[t];
  const T R = rho[n], ur = u_r[n], ut = u_t[n], E = temp[n];  // E = T for gamma = 2
  if (!(R > T(0) && E > T(0))) atomicOr(p.status, PCLB_FLAG_NONPHYS);
  const T ux = ur * c - ut * s, uy = ur * s + ut * c;
  const EqParams<T> e = eq_params<T>((double)R, ux, uy, (double)E, d);
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const int q_begin = k == 0 ? 0 : 1 + (k - 1) * kNDirs;
    const int q_end = k == 0 ? 1 : q_begin + kNDirs;
    for (int q = q_begin; q < q_end; ++q)
      store_with_ghosts<T>(f, p, d, q, t, r, feq_q<T>(e, d.vx[q], d.vy[q], k));
  }
}


// FP32 path: two radially adjacent nodes per thread in packed FP32x2
// arithmetic, with the step's float-float equilibrium (eq2, feq_pair2) of the
// given fields; the velocity is rotated to Cartesian components in
// float-float (no FP64 arithmetic), values are stored in pairs.
constexpr int kSetThreads32 = 128;   // 256 nodes of a row per block

__global__ void __launch_bounds__(kSetThreads32)
    set_state_f32_kernel(float* __restrict__ f, const float* __restrict__ rho, const float* __restrict__ u_r,
                         const float* __restrict__ u_t, const float* __restrict__ temp,
                         const __grid_constant__ StepParams p, const __grid_constant__ DvmConst<float> d,
                         int t_begin) {
  const int r = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int t = blockIdx.y + t_begin;
  if (r >= p.n_r || t >= p.n_theta) return;
  const bool v1 = r + 1 < p.n_r;             // the second node exists
  const size_t n = (size_t)t * p.n_r + r;
  auto field = [&](const float* a) { return mk2(a[n], v1 ? a[n + 1] : a[n]); };
  const f2 R = field(rho), E = field(temp);   // E = T for gamma = 2
  if (!(R.x > 0.f && E.x > 0.f && R.y > 0.f && E.y > 0.f)) atomicOr(p.status, PCLB_FLAG_NONPHYS);
  const float4 cs = p.cs_ff[t];
  const ff2 c = ffc(cs.x, cs.y), s = ffc(cs.z, cs.w);
  const ff2 ur = ff2_of(field(u_r)), ut = ff2_of(field(u_t));
  State2 st;
  st.rho = ff2_of(R);
  st.E = ff2_of(E);
  const ff2 uts = ff2_mul(ut, s);
  st.ux = ff2_add(ff2_mul(ur, c), ff2{neg2(uts.hi), neg2(uts.lo)});
  st.uy = ff2_add(ff2_mul(ur, s), ff2_mul(ut, c));
  const Eq2 eq = eq2(st, d);

  const size_t plane = (size_t)p.rows * p.pitch;
  float* row = f + (size_t)(t + kGhostRows) * p.pitch + r;
  float* lo = t >= p.n_theta - 2 ? f + (size_t)(t - (p.n_theta - 2)) * p.pitch + r : nullptr;
  float* hi = t < 2 ? f + (size_t)(p.n_theta + kGhostRows + t) * p.pitch + r : nullptr;
  // label q at this row, and at the azimuthal ghost rows it feeds (Eq. 40)
  auto put = [&](int q, f2 v) {
    auto one = [&](float* base) {
      if (v1)
        *reinterpret_cast<float2*>(base) = v;   // r even, pitch even: 8-byte aligned
      else
        base[0] = v.x;
    };
    one(row + (size_t)q * plane);
    if (lo) one(lo + (size_t)d.recv_lo[q] * plane);
    if (hi) one(hi + (size_t)d.recv_hi[q] * plane);
  };
  put(0, mul2(eq.w[0], eq.a0));
#pragma unroll
  for (int k = 1; k <= 4; ++k) {
    const f2 sh = bc2(d.speed[k]), sl = bc2(d.speed_lo[k]);
#pragma unroll
    for (int i = 0; i < kHalf; ++i) {
      const int q = 1 + (k - 1) * kNDirs + i;
      f2 fp, fm;
      feq_pair2(eq, sh, sl, i, eq.w[k], fp, fm);
      put(q, fp);
      put(q + kHalf, fm);
    }
  }
}

__global__ void moments_f32_kernel(const float* __restrict__ f, float* rho, float* u_r, float* u_t,
                                   float* temp, const __grid_constant__ StepParams p,
                                   const __grid_constant__ DvmConst<float> d, int t_begin) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int t = blockIdx.y + t_begin;
  if (r >= p.n_r || t >= p.n_theta) return;
  const size_t plane = (size_t)p.rows * p.pitch;
  const State32 m = state32(f + (size_t)(t + kGhostRows) * p.pitch + r, plane, d);
  const size_t n = (size_t)t * p.n_r + r;
  // polar components in float-float, rounded once (no FP64 arithmetic)
  const float4 cs = p.cs_ff[t];
  const ff c{cs.x, cs.y}, s{cs.z, cs.w};
  if (rho) rho[n] = m.rho.hi + m.rho.lo;
  if (u_r) u_r[n] = ff_add(ff_mul(m.ux, c), ff_mul(m.uy, s)).hi;
  if (u_t) u_t[n] = ff_add(ff_mul(m.uy, c), ff_neg(ff_mul(m.ux, s))).hi;
  if (temp) temp[n] = m.E.hi + m.E.lo;
}

template <class T>
__global__ void moments_kernel(const T* __restrict__ f, T* rho, T* u_r, T* u_t, T* temp,
                               const __grid_constant__ StepParams p, const __grid_constant__ DvmConst<T> d,
                               int t_begin) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int t = blockIdx.y + t_begin;
  if (r >= p.n_r || t >= p.n_theta) return;
  const size_t plane = (size_t)p.rows * p.pitch;
  const NodeState<T> m = node_moments(f + (size_t)(t + kGhostRows) * p.pitch + r, plane, d);
  const size_t n = (size_t)t * p.n_r + r;
  const T c = (T)p.cos_t[t], s = (T)p.sin_t[t];
  if (rho) rho[n] = m.rho;
  if (u_r) u_r[n] = m.ux * c + m.uy * s;
  if (u_t) u_t[n] = m.uy * c - m.ux * s;
  if (temp) temp[n] = m.E;
}

template <class T>
__global__ void pack_kernel(const T* __restrict__ f, T* __restrict__ out, const __grid_constant__ StepParams p) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int t = blockIdx.y, q = blockIdx.z;
  if (r >= p.n_r) return;
  out[((size_t)q * p.n_theta + t) * p.n_r + r] =
      f[(size_t)q * p.rows * p.pitch + (size_t)(t + kGhostRows) * p.pitch + r];
}

template <class T>
__global__ void unpack_kernel(const T* __restrict__ in, T* __restrict__ f, const __grid_constant__ StepParams p,
                              const __grid_constant__ DvmConst<T> d) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int t = blockIdx.y, q = blockIdx.z;
  if (r >= p.n_r) return;
  store_with_ghosts<T>(f, p, d, q, t, r, in[((size_t)q * p.n_theta + t) * p.n_r + r]);
}

// Global integrals with weight r dr dtheta, in double.  Each block reduces a
// fixed grid-stride subset in a fixed order, so results are reproducible.
template <class T>
__global__ void diag_partial_kernel(const T* __restrict__ f, double* partials, const __grid_constant__ StepParams p,
                                    const __grid_constant__ DvmConst<T> d, double dr, double dth, double r_in) {
  const size_t plane = (size_t)p.rows * p.pitch;
  const size_t n_nodes = (size_t)p.n_r * p.n_theta;
  double acc[4] = {0, 0, 0, 0};
  double mn[2] = {DBL_MAX, DBL_MAX};
  for (size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x; n < n_nodes;
       n += (size_t)gridDim.x * blockDim.x) {
    const int t = (int)(n / p.n_r), r = (int)(n % p.n_r);
    double rho, ux, uy, E;
    node_state_double(f + (size_t)(t + kGhostRows) * p.pitch + r, plane, d, rho, ux, uy, E);
    const double w = (r_in + r * dr) * dr * dth;
    acc[0] += w * rho;
    acc[1] += w * rho * ux;
    acc[2] += w * rho * uy;
    acc[3] += w * rho * (E + 0.5 * (ux * ux + uy * uy));
    mn[0] = fmin(mn[0], rho);
    mn[1] = fmin(mn[1], E);
  }
  __shared__ double red[6][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double v[6] = {acc[0], acc[1], acc[2], acc[3], mn[0], mn[1]};
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    for (int off = 16; off > 0; off >>= 1) {
      const double o = __shfl_down_sync(0xffffffffu, v[i], off);
      v[i] = i < 4 ? v[i] + o : fmin(v[i], o);
    }
    if (lane == 0) red[i][warp] = v[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = blockDim.x / 32;
    for (int i = 0; i < 6; ++i) {
      double s = red[i][0];
      for (int w = 1; w < nw; ++w) s = i < 4 ? s + red[i][w] : fmin(s, red[i][w]);
      partials[(size_t)blockIdx.x * 8 + i] = s;
    }
  }
}

__global__ void diag_final_kernel(const double* partials, int n_blocks, double* out, double n_nodes) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s[6] = {0, 0, 0, 0, DBL_MAX, DBL_MAX};
  for (int b = 0; b < n_blocks; ++b)
    for (int i = 0; i < 6; ++i)
      s[i] = i < 4 ? s[i] + partials[(size_t)b * 8 + i] : fmin(s[i], partials[(size_t)b * 8 + i]);
  for (int i = 0; i < 6; ++i) out[i] = s[i];
  out[6] = n_nodes;
  out[7] = 0.0;
}

// ---------------------------------------------------------------------------
// Launchers.
// ---------------------------------------------------------------------------
constexpr int kRowThreads = 128;

// Rows [t_begin, t_end) of the grid (t_end < 0: to the last row); the field
// arrays are always indexed with the full [n_theta][n_r] layout.
template <class T>
cudaError_t launch_set_state(T* f, const T* rho, const T* ur, const T* ut, const T* temp,
                             const StepParams& p, const DvmConst<T>& d, cudaStream_t s, int t_begin, int t_end) {
  if (t_end < 0) t_end = p.n_theta;
  if (t_begin < 0 || t_end <= t_begin) return cudaSuccess;
  if constexpr (sizeof(T) == 4) {
    const dim3 grid((p.n_r + 2 * kSetThreads32 - 1) / (2 * kSetThreads32), t_end - t_begin);
    set_state_f32_kernel<<<grid, kSetThreads32, 0, s>>>(f, rho, ur, ut, temp, p, d, t_begin);
  } else {
    const dim3 grid((p.n_r + kRowThreads - 1) / kRowThreads, t_end - t_begin);
    set_state_kernel<T><<<grid, kRowThreads, 0, s>>>(f, rho, ur, ut, temp, p, d, t_begin);
  }
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_moments(const T* f, T* rho, T* ur, T* ut, T* temp, const StepParams& p,
                           const DvmConst<T>& d, cudaStream_t s, int t_begin, int t_end) {
  if (t_end < 0) t_end = p.n_theta;
  if (t_begin < 0 || t_end <= t_begin) return cudaSuccess;
  dim3 grid((p.n_r + kRowThreads - 1) / kRowThreads, t_end - t_begin);
  if constexpr (sizeof(T) == 4)
    moments_f32_kernel<<<grid, kRowThreads, 0, s>>>(f, rho, ur, ut, temp, p, d, t_begin);
  else
    moments_kernel<T><<<grid, kRowThreads, 0, s>>>(f, rho, ur, ut, temp, p, d, t_begin);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_pack(const T* f, T* out, const StepParams& p, cudaStream_t s) {
  dim3 grid((p.n_r + kRowThreads - 1) / kRowThreads, p.n_theta, kQ);
  pack_kernel<T><<<grid, kRowThreads, 0, s>>>(f, out, p);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_unpack(const T* in, T* f, const StepParams& p, const DvmConst<T>& d, cudaStream_t s) {
  dim3 grid((p.n_r + kRowThreads - 1) / kRowThreads, p.n_theta, kQ);
  unpack_kernel<T><<<grid, kRowThreads, 0, s>>>(in, f, p, d);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_diagnostics(const T* f, double* partials, double* out, const StepParams& p,
                               const DvmConst<T>& d, double dr, double dth, double r_in,
                               cudaStream_t s) {
  diag_partial_kernel<T><<<kDiagBlocks, 256, 0, s>>>(f, partials, p, d, dr, dth, r_in);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  diag_final_kernel<<<1, 32, 0, s>>>(partials, kDiagBlocks, out, (double)p.n_r * p.n_theta);
  return cudaGetLastError();
}

#define PCLB_INSTANTIATE(T)                                                                         \
  template cudaError_t launch_set_state<T>(T*, const T*, const T*, const T*, const T*,             \
                                           const StepParams&, const DvmConst<T>&, cudaStream_t,    \
                                           int, int);                                              \
  template cudaError_t launch_moments<T>(const T*, T*, T*, T*, T*, const StepParams&,              \
                                         const DvmConst<T>&, cudaStream_t, int, int);              \
  template cudaError_t launch_pack<T>(const T*, T*, const StepParams&, cudaStream_t);              \
  template cudaError_t launch_unpack<T>(const T*, T*, const StepParams&, const DvmConst<T>&,       \
                                        cudaStream_t);                                             \
  template cudaError_t launch_diagnostics<T>(const T*, double*, double*, const StepParams&,        \
                                             const DvmConst<T>&, double, double, double,           \
                                             cudaStream_t);
PCLB_INSTANTIATE(float)
PCLB_INSTANTIATE(double)

}  // namespace pclb
