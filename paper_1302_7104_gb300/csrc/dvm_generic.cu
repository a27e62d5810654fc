// The FP64 step and the field kernels (both precisions) for the larger
// velocity sets of Table I, N_i = 16 and 24 directions per shell (Q = 65,
// 97): the same model (Eqs. 2-5, 10-11, 19 or 18, 28 or the other convection
// schemes, 38-40), one thread per node, stencil values read from global
// memory (L1/L2), the moments, the temperature and the equilibrium factors in
// double.  These sets serve the paper's velocity-set comparison; their FP32
// step is the tiled kernel of dvm_tiled32.cu, the tuned TMA kernels cover
// N_i = 8.
//
// Radial ghost nodes (Sec. II C 1) are formed once per wall row by
// gen_ghost_kernel into a small buffer [side][layer][n_theta][Q] (f = f^eq of
// the extrapolated or prescribed state, plus the wall node's departure from
// equilibrium for non-equilibrium ghosts); the azimuthal ghost rows (Eq. 40)
// are stored rows, written by the producer of the seam rows with the label
// rotation, as in the rest of the library.
#include <cfloat>
#include <cmath>
#include <cstddef>
#include <cuda_runtime.h>

#include "dvm_generic.h"
#include "f32_state.cuh"
#include "pclb_internal.h"

namespace pclb {

namespace {

constexpr int kGenThreads = 128;

struct GenEq {
  double w[5];              // rho F_k(E) (Eq. 11); w[0] = rho (1 - B0 sum_k F_k)
  double a0, a1, a1h;       // coefficients of the polynomial of Eq. (10)
  double uxE, uyE;          // u / E
};

struct GenState {
  double rho, ux, uy, E;
  bool ok;
};

// Velocity and temperature from the sums rho, rho u, rho (E + u^2/2).
__device__ __forceinline__ GenState gen_state_of(double s0, double sx, double sy, double se) {
  GenState m;
  m.rho = s0;
  m.ux = sx / s0;
  m.uy = sy / s0;
  m.E = (se - 0.5 * (sx * m.ux + sy * m.uy)) / s0;
  m.ok = s0 > 0.0 && m.E > 0.0 && isfinite(m.E) && isfinite(m.ux) && isfinite(m.uy);
  return m;
}

// Moments (Eqs. 3-5): rho = sum f, rho u = sum f v, rho (E + u^2/2) = sum f v^2/2.
template <class T>
__device__ GenState gen_moments_node(const T* f, size_t plane, const DvmG& d) {
  double s0 = 0.0, sx = 0.0, sy = 0.0, se = 0.0;
  for (int q = 0; q < d.q; ++q) {
    const double v = (double)f[(size_t)q * plane];
    s0 += v;
    sx = fma(d.vx[q], v, sx);
    sy = fma(d.vy[q], v, sy);
    se = fma(d.half_v2[d.shell[q]], v, se);
  }
  return gen_state_of(s0, sx, sy, se);
}

__device__ GenEq gen_eq(double rho, double ux, double uy, double E, const DvmG& d) {
  GenEq e;
  double Fs = 0.0;
  for (int k = 1; k <= 4; ++k) {
    const double F = E * (d.Fc[k][0] + E * (d.Fc[k][1] + E * (d.Fc[k][2] + E * d.Fc[k][3])));
    e.w[k] = rho * F;
    Fs += F;
  }
  e.w[0] = rho * (1.0 - d.B0 * Fs);
  const double u2E = (ux * ux + uy * uy) / E;
  e.a1 = 1.0 - 0.5 * u2E;
  e.a0 = e.a1 + 0.125 * u2E * u2E;
  e.a1h = 0.5 * e.a1;
  e.uxE = ux / E;
  e.uyE = uy / E;
  return e;
}

__device__ __forceinline__ double gen_feq(const GenEq& e, const DvmG& d, int q) {
  const double x = d.vx[q] * e.uxE + d.vy[q] * e.uyE;
  return e.w[d.shell[q]] * (e.a0 + x * (e.a1 + x * (e.a1h + x * (1.0 / 6.0 + x * (1.0 / 24.0)))));
}

// The equilibrium factors in the arithmetic type C of the per-velocity work
// (float for FP32 storage, double for FP64), rounded from the double ones.
template <class C>
struct GenEqC {
  C w[5], a0, a1, a1h, uxE, uyE;
};

template <class C>
__device__ __forceinline__ GenEqC<C> gen_eq_c(const GenEq& e) {
  GenEqC<C> c;
  for (int k = 0; k < 5; ++k) c.w[k] = (C)e.w[k];
  c.a0 = (C)e.a0; c.a1 = (C)e.a1; c.a1h = (C)e.a1h; c.uxE = (C)e.uxE; c.uyE = (C)e.uyE;
  return c;
}

// f^eq of velocity (vx, vy) of shell k, Eq. (10), as even and odd parts in x
// = v.u/E: P(x) = ev + od, P(-x) = ev - od (the opposite velocity).
template <class C>
__device__ __forceinline__ void gen_feq_pair(const GenEqC<C>& e, C vx, C vy, int k, C& fp, C& fm) {
  const C x = vx * e.uxE + vy * e.uyE, x2 = x * x;
  const C ev = e.a0 + x2 * (e.a1h + x2 * C(1.0 / 24.0));
  const C od = x * (e.a1 + x2 * C(1.0 / 6.0));
  fp = e.w[k] * (ev + od);
  fm = e.w[k] * (ev - od);
}

// Convection increment in upwind form from a = |C|, K = a (1 - a), the node
// value f0, its upwind neighbours u1, u2 and (Lax-Wendroff) the downwind one d1.
// The limiter ratio |D| / (|D| + |Dp|) with the correctly rounded quotient
// (0 when the sum is below the smallest normal number).
template <int SCH>
__device__ __forceinline__ double gen_convect(double a, double K, double f0, double u1, double u2, double d1) {
  const double D = f0 - u1, Dp = u1 - u2;
  if (SCH == PCLB_SCHEME_MWB) {
    const double den = fabs(D) + fabs(Dp);
    const double h = den >= DBL_MIN ? fabs(D) * (D - Dp) / den : 0.0;
    return a * D + K * h;
  }
  if (SCH == PCLB_SCHEME_WB) return a * D + 0.5 * K * (D - Dp);
  if (SCH == PCLB_SCHEME_UPWIND2) return a * D + 0.5 * a * (D - Dp);
  return a * D + 0.5 * K * ((d1 - f0) - D);
}

// Store of label q at interior node (t, r), and of the azimuthal ghost rows
// of the receiving labels when t is a seam row (Eq. 40).
template <class T>
__device__ __forceinline__ void gen_store(T* f, const StepParams& p, const DvmG& d, int q, int t, int r, T v) {
  const size_t plane = (size_t)p.rows * p.pitch;
  f[(size_t)q * plane + (size_t)(t + kGhostRows) * p.pitch + r] = v;
  if (t >= p.n_theta - 2)
    f[(size_t)d.recv_lo[q] * plane + (size_t)(t - (p.n_theta - 2)) * p.pitch + r] = v;
  if (t < 2) f[(size_t)d.recv_hi[q] * plane + (size_t)(p.n_theta + kGhostRows + t) * p.pitch + r] = v;
}

// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(kGenThreads)
    gen_set_state_kernel(T* __restrict__ f, const T* __restrict__ rho, const T* __restrict__ u_r,
                         const T* __restrict__ u_t, const T* __restrict__ temp, const __grid_constant__ StepParams p,
                         const __grid_constant__ DvmG d) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int t = blockIdx.y;
  if (r >= p.n_r) return;
  const size_t n = (size_t)t * p.n_r + r;
  const double c = p.cos_t[t], s = p.sin_t[t];
  const double R = (double)rho[n], ur = (double)u_r[n], ut = (double)u_t[n], E = (double)temp[n];  // E = T
  if (!(R > 0.0 && E > 0.0)) atomicOr(p.status, PCLB_FLAG_NONPHYS);
  const GenEq e = gen_eq(R, ur * c - ut * s, ur * s + ut * c, E, d);
  for (int q = 0; q < d.q; ++q) gen_store<T>(f, p, d, q, t, r, (T)gen_feq(e, d, q));
}

template <class T>
__global__ void __launch_bounds__(kGenThreads)
    gen_moments_kernel(const T* __restrict__ f, T* rho, T* u_r, T* u_t, T* temp, const __grid_constant__ StepParams p,
                       const __grid_constant__ DvmG d) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int t = blockIdx.y;
  if (r >= p.n_r) return;
  const size_t plane = (size_t)p.rows * p.pitch;
  const GenState m = gen_moments_node(f + (size_t)(t + kGhostRows) * p.pitch + r, plane, d);
  const size_t n = (size_t)t * p.n_r + r;
  const double c = p.cos_t[t], s = p.sin_t[t];
  if (rho) rho[n] = (T)m.rho;
  if (u_r) u_r[n] = (T)(m.ux * c + m.uy * s);
  if (u_t) u_t[n] = (T)(m.uy * c - m.ux * s);
  if (temp) temp[n] = (T)m.E;
}

template <class T>
__global__ void __launch_bounds__(kGenThreads)
    gen_pack_kernel(const T* __restrict__ f, T* __restrict__ out, const __grid_constant__ StepParams p) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int t = blockIdx.y, q = blockIdx.z;
  if (r >= p.n_r) return;
  out[((size_t)q * p.n_theta + t) * p.n_r + r] = f[(size_t)q * p.rows * p.pitch + (size_t)(t + kGhostRows) * p.pitch + r];
}

template <class T>
__global__ void __launch_bounds__(kGenThreads)
    gen_unpack_kernel(const T* __restrict__ in, T* __restrict__ f, const __grid_constant__ StepParams p,
                      const __grid_constant__ DvmG d) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int t = blockIdx.y, q = blockIdx.z;
  if (r >= p.n_r) return;
  gen_store<T>(f, p, d, q, t, r, in[((size_t)q * p.n_theta + t) * p.n_r + r]);
}

// Radial ghost layers of wall `side` at row t: layer l sits at r = -1 - l
// (inner) or n_r + l (outer).  Eq. (39) applied twice to the wall node a and
// the next node b: g0 = 2a - b, g1 = 2 g0 - a, for the components the
// boundary kind extrapolates; the others prescribed.
template <class T>
__global__ void __launch_bounds__(kGenThreads)
    gen_ghost_kernel(const T* __restrict__ f, T* __restrict__ ghost, const __grid_constant__ StepParams p,
                     const __grid_constant__ DvmG d) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int side = blockIdx.y;
  if (t >= p.n_theta) return;
  const size_t plane = (size_t)p.rows * p.pitch;
  const int ra = side == 0 ? 0 : p.n_r - 1, step = side == 0 ? 1 : -1;
  const T* fa = f + (size_t)(t + kGhostRows) * p.pitch + ra;
  const GenState a = gen_moments_node(fa, plane, d);
  const GenState b = gen_moments_node(fa + step, plane, d);
  double g[2][4];
  g[0][0] = 2.0 * a.rho - b.rho;  g[1][0] = 2.0 * g[0][0] - a.rho;
  g[0][1] = 2.0 * a.ux - b.ux;    g[1][1] = 2.0 * g[0][1] - a.ux;
  g[0][2] = 2.0 * a.uy - b.uy;    g[1][2] = 2.0 * g[0][2] - a.uy;
  g[0][3] = 2.0 * a.E - b.E;      g[1][3] = 2.0 * g[0][3] - a.E;
  const int kind = p.bc_kind[side] & ~PCLB_BC_NEQ;
  const bool neq = (p.bc_kind[side] & PCLB_BC_NEQ) != 0;
  if (kind != PCLB_BC_EXTRAP) {
    const double c = p.cos_t[t], s = p.sin_t[t];
    for (int l = 0; l < 2; ++l) {
      const double* v = p.bc_vals + (size_t)((side * 2 + l) * 4) * p.n_theta + t;
      const double ur = v[1 * p.n_theta], ut = v[2 * p.n_theta];
      g[l][1] = ur * c - ut * s;
      g[l][2] = ur * s + ut * c;
      if (kind == PCLB_BC_DIRICHLET) {
        g[l][0] = v[0];
        g[l][3] = v[3 * p.n_theta];
      }
    }
  }
  bool ok = a.ok && b.ok;
  const GenEq ea = gen_eq(a.rho, a.ux, a.uy, a.E, d);
  for (int l = 0; l < 2; ++l) {
    ok = ok && g[l][0] > 0.0 && g[l][3] > 0.0;
    const GenEq e = gen_eq(g[l][0], g[l][1], g[l][2], g[l][3], d);
    T* out = ghost + ((size_t)(side * 2 + l) * p.n_theta + t) * d.q;
    for (int q = 0; q < d.q; ++q) {
      double v = gen_feq(e, d, q);
      if (neq) v += (double)fa[(size_t)q * plane] - gen_feq(ea, d, q);
      out[q] = (T)v;
    }
  }
  if (!ok) atomicOr(p.status, PCLB_FLAG_NONPHYS);
}

// One FP64 step (Eq. 38) at node (t, r): moments and equilibrium factors in
// double, then per pair of opposite velocities (sharing the Courant entry
// and the even and odd parts of the equilibrium polynomial) the relaxation
// (decay d = exp(-dt/tau) or 1 - dt/tau) minus the convection increments in r
// and theta.
template <int SCH>
__global__ void __launch_bounds__(kGenThreads)
    gen_step_kernel(const double* __restrict__ f, double* __restrict__ f_out, const double* __restrict__ ghost,
                    const __grid_constant__ StepParams p, const __grid_constant__ DvmG d) {
  using T = double;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int t = blockIdx.y;
  if (r >= p.n_r) return;
  const size_t plane = (size_t)p.rows * p.pitch;
  const int srow = t + kGhostRows;
  const T* fn = f + (size_t)srow * p.pitch + r;
  const GenState m = gen_moments_node(fn, plane, d);
  const GenEqC<T> e = gen_eq_c<T>(gen_eq(m.rho, m.ux, m.uy, m.E, d));
  if (!m.ok) atomicOr(p.status, PCLB_FLAG_NONPHYS);
  const T decay = (T)p.decay;
  // value of label q (plane fq) at radial index rr of row t (a ghost layer
  // outside the grid)
  auto fr = [&](const T* fq, int q, int rr) -> T {
    if (rr < 0) return ghost[((size_t)(0 * 2 + (-1 - rr)) * p.n_theta + t) * d.q + q];
    if (rr >= p.n_r) return ghost[((size_t)(1 * 2 + (rr - p.n_r)) * p.n_theta + t) * d.q + q];
    return fq[rr - r];
  };
  // value of plane fq at stored row srow + dt_rows of column r
  const ptrdiff_t pitch = p.pitch;
  auto ft = [&](const T* fq, int dt_rows) -> T { return fq[dt_rows * pitch]; };
  // label q at this node and at the azimuthal ghost rows it feeds (Eq. 40)
  T* out_row = f_out + (size_t)srow * p.pitch + r;
  T* out_lo = t >= p.n_theta - 2 ? f_out + (size_t)(t - (p.n_theta - 2)) * p.pitch + r : nullptr;
  T* out_hi = t < 2 ? f_out + (size_t)(p.n_theta + kGhostRows + t) * p.pitch + r : nullptr;
  auto put = [&](int q, T v) {
    out_row[(size_t)q * plane] = v;
    if (out_lo) out_lo[(size_t)d.recv_lo[q] * plane] = v;
    if (out_hi) out_hi[(size_t)d.recv_hi[q] * plane] = v;
  };
  {
    const T f0 = fn[0];
    const T fe = e.w[0] * e.a0;
    put(0, fe + (f0 - fe) * decay);
  }
  const int half = d.n_dirs / 2, npairs = 2 * d.n_dirs;
  const T inv_r = (T)p.inv_r[r];
  const bool lw = SCH == PCLB_SCHEME_LW;
  for (int k = 1; k <= 4; ++k)
    for (int i = 0; i < half; ++i) {
      const int q1 = 1 + (k - 1) * d.n_dirs + i, q2 = q1 + half;
      const double* ce = p.courant64 + ((size_t)srow * npairs + (k - 1) * half + i) * 4;
      const T ar = ce[0], kr = ce[1], at = ce[2] * inv_r;
      const int fl = (int)ce[3];
      const T kt = at - at * at;
      const int sr = (fl & 1) ? 1 : -1;   // v_r < 0 for q1: upwind at larger r
      const int st = (fl & 2) ? 1 : -1;   // v_theta < 0 for q1: upwind at larger theta
      T fe[2];
      gen_feq_pair<T>(e, d.vx[q1], d.vy[q1], k, fe[0], fe[1]);
      for (int L = 0; L < 2; ++L) {
        const int q = L ? q2 : q1, s_r = L ? -sr : sr, s_t = L ? -st : st;
        const T* fq = fn + (size_t)q * plane;
        const T a = fq[0];
        const T cr = gen_convect<SCH>(ar, kr, a, fr(fq, q, r + s_r), fr(fq, q, r + 2 * s_r),
                                      lw ? fr(fq, q, r - s_r) : T(0));
        const T ct = gen_convect<SCH>(at, kt, a, ft(fq, s_t), ft(fq, 2 * s_t), lw ? ft(fq, -s_t) : T(0));
        put(q, fe[L] + (a - fe[L]) * decay - cr - ct);
      }
    }
}

// Global integrals with weight r dr dtheta (as pclb_diagnostics): per block a
// fixed grid-stride subset in a fixed order, then one thread sums the blocks.
template <class T>
__global__ void __launch_bounds__(kGenThreads)
    gen_diag_partial_kernel(const T* __restrict__ f, double* partials, const __grid_constant__ StepParams p,
                            const __grid_constant__ DvmG d, double dr, double dth, double r_in) {
  const size_t plane = (size_t)p.rows * p.pitch;
  const size_t n_nodes = (size_t)p.n_r * p.n_theta;
  double v[6] = {0, 0, 0, 0, DBL_MAX, DBL_MAX};
  for (size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x; n < n_nodes; n += (size_t)gridDim.x * blockDim.x) {
    const int t = (int)(n / p.n_r), r = (int)(n % p.n_r);
    const GenState m = gen_moments_node(f + (size_t)(t + kGhostRows) * p.pitch + r, plane, d);
    const double w = (r_in + r * dr) * dr * dth;
    v[0] += w * m.rho;
    v[1] += w * m.rho * m.ux;
    v[2] += w * m.rho * m.uy;
    v[3] += w * m.rho * (m.E + 0.5 * (m.ux * m.ux + m.uy * m.uy));
    v[4] = fmin(v[4], m.rho);
    v[5] = fmin(v[5], m.E);
  }
  __shared__ double red[6][kGenThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = 0; i < 6; ++i) {
    for (int off = 16; off > 0; off >>= 1) {
      const double o = __shfl_down_sync(0xffffffffu, v[i], off);
      v[i] = i < 4 ? v[i] + o : fmin(v[i], o);
    }
    if (lane == 0) red[i][warp] = v[i];
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int i = 0; i < 6; ++i) {
      double s = red[i][0];
      for (int w = 1; w < kGenThreads / 32; ++w) s = i < 4 ? s + red[i][w] : fmin(s, red[i][w]);
      partials[(size_t)blockIdx.x * 8 + i] = s;
    }
}

__global__ void gen_diag_final_kernel(const double* partials, int n_blocks, double* out, double n_nodes) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s[6] = {0, 0, 0, 0, DBL_MAX, DBL_MAX};
  for (int b = 0; b < n_blocks; ++b)
    for (int i = 0; i < 6; ++i)
      s[i] = i < 4 ? s[i] + partials[(size_t)b * 8 + i] : fmin(s[i], partials[(size_t)b * 8 + i]);
  for (int i = 0; i < 6; ++i) out[i] = s[i];
  out[6] = n_nodes;
  out[7] = 0.0;
}

template <int SCH>
cudaError_t gen_step_scheme(const double* f, double* f_out, double* ghost, const StepParams& p, const DvmG& d,
                            cudaStream_t s) {
  // one thread per wall row, in warps, so that the rows spread over the SMs
  gen_ghost_kernel<double><<<dim3((p.n_theta + 31) / 32, 2), 32, 0, s>>>(f, ghost, p, d);
  gen_step_kernel<SCH><<<dim3((p.n_r + kGenThreads - 1) / kGenThreads, p.n_theta), kGenThreads, 0, s>>>(
      f, f_out, ghost, p, d);
  return cudaGetLastError();
}

}  // namespace

template <class T>
cudaError_t gen_launch_set_state(T* f, const T* rho, const T* ur, const T* ut, const T* temp, const StepParams& p,
                                 const DvmG& d, cudaStream_t s) {
  gen_set_state_kernel<T><<<dim3((p.n_r + kGenThreads - 1) / kGenThreads, p.n_theta), kGenThreads, 0, s>>>(
      f, rho, ur, ut, temp, p, d);
  return cudaGetLastError();
}

template <class T>
cudaError_t gen_launch_moments(const T* f, T* rho, T* ur, T* ut, T* temp, const StepParams& p, const DvmG& d,
                               cudaStream_t s) {
  gen_moments_kernel<T><<<dim3((p.n_r + kGenThreads - 1) / kGenThreads, p.n_theta), kGenThreads, 0, s>>>(
      f, rho, ur, ut, temp, p, d);
  return cudaGetLastError();
}

template <class T>
cudaError_t gen_launch_pack(const T* f, T* out, const StepParams& p, const DvmG& d, cudaStream_t s) {
  gen_pack_kernel<T><<<dim3((p.n_r + kGenThreads - 1) / kGenThreads, p.n_theta, d.q), kGenThreads, 0, s>>>(f, out, p);
  return cudaGetLastError();
}

template <class T>
cudaError_t gen_launch_unpack(const T* in, T* f, const StepParams& p, const DvmG& d, cudaStream_t s) {
  gen_unpack_kernel<T><<<dim3((p.n_r + kGenThreads - 1) / kGenThreads, p.n_theta, d.q), kGenThreads, 0, s>>>(
      in, f, p, d);
  return cudaGetLastError();
}

cudaError_t gen_launch_step_f64(const double* f, double* f_out, double* ghost, const StepParams& p, const DvmG& d,
                                cudaStream_t s) {
  switch (p.scheme) {
    case PCLB_SCHEME_WB: return gen_step_scheme<PCLB_SCHEME_WB>(f, f_out, ghost, p, d, s);
    case PCLB_SCHEME_LW: return gen_step_scheme<PCLB_SCHEME_LW>(f, f_out, ghost, p, d, s);
    case PCLB_SCHEME_UPWIND2: return gen_step_scheme<PCLB_SCHEME_UPWIND2>(f, f_out, ghost, p, d, s);
    default: return gen_step_scheme<PCLB_SCHEME_MWB>(f, f_out, ghost, p, d, s);
  }
}

void fill_dvm_generic32(DvmG32& c, const pclb_dvm& d, const DvmG& g) {
  const int nd = d.n_dirs;
  c = DvmG32{};
  auto split = [](double x, float& hi, float& lo) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
  };
  for (int k = 0; k < 5; ++k) {
    split(d.speeds[k], c.sph[k], c.spl[k]);
    split(g.half_v2[k], c.hvh[k], c.hvl[k]);
    for (int n = 0; n < 4; ++n) split(g.Fc[k][n], c.Fch[k][n], c.Fcl[k][n]);
  }
  split(d.speeds[3] - d.speeds[2], c.dv23h, c.dv23l);
  split(g.half_v2[3] - g.half_v2[2], c.dh23h, c.dh23l);
  split(g.B0, c.B0h, c.B0l);
  for (int i = 0; i < nd / 2; ++i) {
    const double phi = 2.0 * M_PI * i / nd;
    const double u[2] = {std::cos(phi), std::sin(phi)};
    float* hi[2] = {c.cxh, c.cyh};
    float* lo[2] = {c.cxl, c.cyl};
    for (int j = 0; j < 2; ++j) {
      hi[j][i] = (float)u[j];
      lo[j][i] = (float)(u[j] - (double)hi[j][i]);
    }
  }
  // the same velocities as DvmG (opposite directions exactly antisymmetric)
  for (int k = 1; k <= 4; ++k)
    for (int i = 0; i < nd; ++i) {
      const int q = 1 + (k - 1) * nd + i;
      const int ib = i % (nd / 2);
      const double phi = 2.0 * M_PI * ib / nd, sgn = i < nd / 2 ? 1.0 : -1.0;
      c.vx[q] = (float)(d.speeds[k] * sgn * std::cos(phi));
      c.vy[q] = (float)(d.speeds[k] * sgn * std::sin(phi));
    }
}

template <class T>
cudaError_t gen_launch_diagnostics(const T* f, double* partials, double* out, const StepParams& p, const DvmG& d,
                                   double dr, double dth, double r_in, cudaStream_t s) {
  gen_diag_partial_kernel<T><<<kDiagBlocks, kGenThreads, 0, s>>>(f, partials, p, d, dr, dth, r_in);
  gen_diag_final_kernel<<<1, 32, 0, s>>>(partials, kDiagBlocks, out, (double)p.n_r * p.n_theta);
  return cudaGetLastError();
}

#define PCLB_GEN_INSTANTIATE(T)                                                                               \
  template cudaError_t gen_launch_set_state<T>(T*, const T*, const T*, const T*, const T*, const StepParams&, \
                                               const DvmG&, cudaStream_t);                                    \
  template cudaError_t gen_launch_moments<T>(const T*, T*, T*, T*, T*, const StepParams&, const DvmG&,        \
                                             cudaStream_t);                                                   \
  template cudaError_t gen_launch_pack<T>(const T*, T*, const StepParams&, const DvmG&, cudaStream_t);        \
  template cudaError_t gen_launch_unpack<T>(const T*, T*, const StepParams&, const DvmG&, cudaStream_t);      \
  template cudaError_t gen_launch_diagnostics<T>(const T*, double*, double*, const StepParams&, const DvmG&,  \
                                                 double, double, double, cudaStream_t);
PCLB_GEN_INSTANTIATE(float)
PCLB_GEN_INSTANTIATE(double)

}  // namespace pclb
