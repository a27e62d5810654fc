// Fused FP32 time step of the polar-coordinate FDLB model (Eq. 38), the hot
// kernel of the library.
//
// Work per CTA: a tile of 32 (r) x 16 (theta) nodes.  One thread issues 33
// TMA box copies (one per velocity plane) of the window [r0-4, r0+36) x
// [t0-2, t0+18) into shared memory; meanwhile the threads tabulate, for each
// opposite-direction velocity pair and tile row, |C_r|, |C_r|(1-|C_r|),
// |v_theta| dt/dtheta and the upwind signs.  Each thread then owns two
// radially adjacent nodes of one row:
//   * moments (Eqs. 3-5) with compensated sums, temperature recovery and the
//     weights rho F_k(E) (Eqs. 11a-b) in float-float arithmetic, so that the
//     rounded equilibrium keeps the collision invariants of the exact one;
//   * radial ghost columns for wall tiles (Eq. 39, f = f^eq), in shared memory;
//   * for every pair (q, q') of opposite velocities in a shell: v_q.u/E from
//     float-float constants, the even / odd parts of the equilibrium
//     polynomial (Eq. 10) shared by q and q', then per velocity the relaxation
//     (Eq. 19) minus the MWB increments (Eq. 28) in r and theta, stored with
//     8-byte stores, plus the azimuthal ghost rows of the seam (Eq. 40).
#include <cuda.h>
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "f32_state.cuh"
#include "pclb_internal.h"

namespace pclb {

namespace {

constexpr int kPairs = 4 * kHalf;                    // 16
constexpr int kPlaneF = kWinR * kWinT;               // floats per plane window
constexpr int kPlanesBytes = kQ * kPlaneF * 4;       // 105600
constexpr int kTabBytes = kPairs * kTileT * 16;      // one float4 per (pair, row)
constexpr int kSmemF32 = kPlanesBytes + kTabBytes + 128;
constexpr uint64_t kWaitNs = 2000000000ull;

// Ghost columns of one wall for tile row `row` (window row index), Sec. II C 1.
__device__ void ghost_columns_f32(float* sm, int row, int side, int cw, int t, const StepParams& p,
                                  const DvmConst<float>& d) {
  const int step = side == 0 ? 1 : -1;
  const State32 a = state32(sm + row * kWinR + cw, kPlaneF, d);
  const State32 b = state32(sm + row * kWinR + cw + step, kPlaneF, d);
  State32 g[2];
  // Eq. (39), applied twice: g0 = 2a - b, g1 = 2 g0 - a = 3a - 2b.
  g[0].rho = ff_add(ff_scale(a.rho, 2.f), ff_neg(b.rho));
  g[0].E = ff_add(ff_scale(a.E, 2.f), ff_neg(b.E));
  g[0].ux = ff_add(ff_scale(a.ux, 2.f), ff_neg(b.ux));
  g[0].uy = ff_add(ff_scale(a.uy, 2.f), ff_neg(b.uy));
  g[1].rho = ff_add(ff_scale(g[0].rho, 2.f), ff_neg(a.rho));
  g[1].E = ff_add(ff_scale(g[0].E, 2.f), ff_neg(a.E));
  g[1].ux = ff_add(ff_scale(g[0].ux, 2.f), ff_neg(a.ux));
  g[1].uy = ff_add(ff_scale(g[0].uy, 2.f), ff_neg(a.uy));
  const int kind = p.bc_kind[side];
  if (kind != PCLB_BC_EXTRAP) {
    const double c = p.cos_t[t], s = p.sin_t[t];
    for (int layer = 0; layer < 2; ++layer) {
      const double* v = p.bc_vals + (size_t)((side * 2 + layer) * 4) * p.n_theta + t;
      const double ur = v[1 * p.n_theta], ut = v[2 * p.n_theta];
      g[layer].ux = ff_from(ur * c - ut * s);
      g[layer].uy = ff_from(ur * s + ut * c);
      if (kind == PCLB_BC_DIRICHLET) {
        g[layer].rho = ff_from(v[0]);
        g[layer].E = ff_from(v[3 * p.n_theta]);
      }
    }
  }
  bool ok = a.ok && b.ok;
  for (int layer = 0; layer < 2; ++layer) {
    ok = ok && g[layer].rho.hi > 0.f && g[layer].E.hi > 0.f;
    const int col = cw - step * (1 + layer);
    if (col < 0 || col >= kWinR) continue;
    const Eq32 e = eq32(g[layer], d);
    float* gp = sm + row * kWinR + col;
    gp[0] = feq32(e, d, 0, 0, 1.f);
#pragma unroll
    for (int k = 1; k <= 4; ++k)
#pragma unroll
      for (int i = 0; i < kHalf; ++i) {
        const int q = 1 + (k - 1) * kNDirs + i;
        gp[q * kPlaneF] = feq32(e, d, k, i, 1.f);
        gp[(q + kHalf) * kPlaneF] = feq32(e, d, k, i, -1.f);
      }
  }
  if (!ok) atomicOr(p.status, PCLB_FLAG_NONPHYS);
}

// MWB increment in upwind form (see device_common.cuh); rcp.approx is enough
// for the limiter ratio in single precision.
__device__ __forceinline__ float mwb32(float a, float K, float D, float Dp) {
  const float den = fmaxf(fabsf(D) + fabsf(Dp), 1e-30f);
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(den));
  const float h = fabsf(D) * (D - Dp) * r;
  return fmaf(a, D, K * h);
}

}  // namespace

__global__ void __launch_bounds__(kStepThreads, 2)
    step_kernel_f32(const __grid_constant__ CUtensorMap tmap_in, float* __restrict__ f_out,
                    const StepParams p, const DvmConst<float> d) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* sm = reinterpret_cast<float*>(smem_raw);
  float4* tab = reinterpret_cast<float4*>(smem_raw + kPlanesBytes);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + kPlanesBytes + kTabBytes);

  const int r0 = blockIdx.x * kTileR;
  const int t0 = blockIdx.y * kTileT;
  const int tid = threadIdx.x;

  if (tid == 0) {
    tma_prefetch_desc(&tmap_in);
    mbar_init(bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (tid == 0) {
    mbar_arrive_expect_tx(bar, (uint32_t)kPlanesBytes);
#pragma unroll 1
    for (int q = 0; q < kQ; ++q) tma_load_3d(sm + q * kPlaneF, &tmap_in, r0 - kLeft, t0, q, bar);
  }

  // Courant table, one (pair, row) entry per thread, while the copies land.
  {
    const int pair = tid / kTileT, rl = tid % kTileT;
    const int k = 1 + pair / kHalf, i = pair % kHalf;
    const int q = 1 + (k - 1) * kNDirs + i;
    const int t = min(t0 + rl, p.n_theta - 1);
    const double c = p.cos_t[t], s = p.sin_t[t];
    const double vx = (double)d.vx[q] + (double)d.vx_lo[q], vy = (double)d.vy[q] + (double)d.vy_lo[q];
    const double vr = vx * c + vy * s, vt = vy * c - vx * s;
    const float ar = (float)(fabs(vr) * p.dt_dr);
    const float aw = (float)(fabs(vt) * p.dt_dth);
    const int flags = (vr < 0.0 ? 1 : 0) | (vt < 0.0 ? 2 : 0);
    tab[pair * kTileT + rl] = make_float4(ar, ar - ar * ar, aw, __int_as_float(flags));
  }

  if (!mbar_wait_bounded(bar, 0, kWaitNs)) {
    if (tid == 0) atomicOr(p.status, PCLB_FLAG_TIMEOUT);
    mbar_wait_bounded(bar, 0, kWaitNs);
    return;
  }
  __syncthreads();   // table visible

  // ---- per-thread nodes: row rl, radial cells j2 and j2 + 1 -----------------
  const int warp = tid >> 5, lane = tid & 31;
  const int rl = 2 * warp + (lane >> 4);          // tile row 0..15
  const int j2 = 2 * (lane & 15);                  // even radial offset 0..30
  const int row = rl + 2;                          // window row
  const int col = kLeft + j2;                      // window column of the first node
  const int t = t0 + rl;
  const int r = r0 + j2;
  const bool row_ok = t < p.n_theta;
  const bool v0 = row_ok && r < p.n_r, v1 = row_ok && r + 1 < p.n_r;

  Eq32 eq[2];
  bool ok = true;
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const bool valid = c == 0 ? v0 : v1;
    State32 s;
    if (valid) {
      s = state32(sm + row * kWinR + col + c, kPlaneF, d);
      ok = ok && s.ok;
    } else {
      s.rho = ff_of(1.f); s.ux = ff_of(0.f); s.uy = ff_of(0.f); s.E = ff_of(1.f); s.ok = true;
    }
    eq[c] = eq32(s, d);
  }
  if (!ok) atomicOr(p.status, PCLB_FLAG_NONPHYS);

  // ---- radial ghost columns ------------------------------------------------
  if (r0 == 0 && warp == 0 && lane < kTileT && t0 + lane < p.n_theta)
    ghost_columns_f32(sm, 2 + lane, 0, kLeft, t0 + lane, p, d);
  const int cw_out = p.n_r - 1 - r0 + kLeft;
  if (cw_out <= kLeft + kTileR && warp == 1 && lane < kTileT && t0 + lane < p.n_theta)
    ghost_columns_f32(sm, 2 + lane, 1, cw_out, t0 + lane, p, d);
  __syncthreads();

  // ---- update ----------------------------------------------------------------
  const float inv_r0 = v0 ? (float)p.inv_r[r] : 1.f;
  const float inv_r1 = v1 ? (float)p.inv_r[r + 1] : 1.f;
  const float decay = (float)p.decay;
  const size_t plane_out = (size_t)p.rows * p.pitch;
  float* out_row = f_out + (size_t)(t + kGhostRows) * p.pitch + r;
  const bool lo_ghost = row_ok && t >= p.n_theta - 2;
  const bool hi_ghost = row_ok && t < 2;
  float* out_lo = f_out + (size_t)max(t - (p.n_theta - 2), 0) * p.pitch + r;
  float* out_hi = f_out + (size_t)(p.n_theta + kGhostRows + t) * p.pitch + r;
  const float* win = sm + row * kWinR + col;

  auto store = [&](int q, float o0, float o1) {
    if (v1) {
      *reinterpret_cast<float2*>(out_row + (size_t)q * plane_out) = make_float2(o0, o1);
      if (lo_ghost) *reinterpret_cast<float2*>(out_lo + (size_t)d.recv_lo[q] * plane_out) = make_float2(o0, o1);
      if (hi_ghost) *reinterpret_cast<float2*>(out_hi + (size_t)d.recv_hi[q] * plane_out) = make_float2(o0, o1);
    } else if (v0) {
      out_row[(size_t)q * plane_out] = o0;
      if (lo_ghost) out_lo[(size_t)d.recv_lo[q] * plane_out] = o0;
      if (hi_ghost) out_hi[(size_t)d.recv_hi[q] * plane_out] = o0;
    }
  };

  // rest velocity: no convection
  {
    const float2 f0 = *reinterpret_cast<const float2*>(win);
    const float e0 = eq[0].w[0] * eq[0].a0, e1 = eq[1].w[0] * eq[1].a0;
    store(0, fmaf(f0.x - e0, decay, e0), fmaf(f0.y - e1, decay, e1));
  }

  // One velocity of a pair: sr = +1 if the upwind side is at larger r, st the
  // same for theta (in rows); fe0, fe1 its equilibrium at the two nodes.
  auto update = [&](int q, int sr, int st, float ar, float kr, float at0, float kt0, float at1,
                    float kt1, float fe0, float fe1) {
    const float* w = win + q * kPlaneF;
    const float2 C = *reinterpret_cast<const float2*>(w);
    const float2 S = *reinterpret_cast<const float2*>(w + 2 * sr);      // (j-2, j-1) or (j+2, j+3)
    const float2 T1 = *reinterpret_cast<const float2*>(w + st * kWinR);
    const float2 T2 = *reinterpret_cast<const float2*>(w + 2 * st * kWinR);
    // upwind neighbours in r of the two nodes
    const float u1a = sr < 0 ? S.y : C.y, u1b = sr < 0 ? C.x : S.x;
    const float u2a = S.x, u2b = S.y;
    const float mr0 = mwb32(ar, kr, C.x - u1a, u1a - u2a);
    const float mr1 = mwb32(ar, kr, C.y - u1b, u1b - u2b);
    const float mt0 = mwb32(at0, kt0, C.x - T1.x, T1.x - T2.x);
    const float mt1 = mwb32(at1, kt1, C.y - T1.y, T1.y - T2.y);
    const float o0 = fmaf(C.x - fe0, decay, fe0) - mr0 - mt0;
    const float o1 = fmaf(C.y - fe1, decay, fe1) - mr1 - mt1;
    store(q, o0, o1);
  };

  // Shells run as a loop (keeps the unrolled body small enough for the
  // instruction cache); the four direction pairs of a shell are unrolled.
#pragma unroll 1
  for (int k = 1; k <= 4; ++k) {
    const float sh = d.speed[k], sl = d.speed_lo[k];
    const float wk0 = k == 1 ? eq[0].w[1] : (k == 2 ? eq[0].w[2] : (k == 3 ? eq[0].w[3] : eq[0].w[4]));
    const float wk1 = k == 1 ? eq[1].w[1] : (k == 2 ? eq[1].w[2] : (k == 3 ? eq[1].w[3] : eq[1].w[4]));
    const int qb = 1 + (k - 1) * kNDirs;
#pragma unroll
    for (int i = 0; i < kHalf; ++i) {
      const int q = qb + i;
      const float4 tb = tab[((k - 1) * kHalf + i) * kTileT + rl];
      const int fl = __float_as_int(tb.w);
      const int sr = (fl & 1) ? 1 : -1;            // v_r < 0: upwind at larger r
      const int st = (fl & 2) ? 1 : -1;            // v_theta < 0: upwind at larger theta
      const float at0 = tb.z * inv_r0, at1 = tb.z * inv_r1;
      const float kt0 = fmaf(-at0, at0, at0), kt1 = fmaf(-at1, at1, at1);
      // equilibrium of the pair at both nodes: P(+x) = ev + od, P(-x) = ev - od
      float fp[2], fm[2];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const float x = x_of(sh, sl, eq[c].yh[i], eq[c].yl[i]);
        const float x2 = x * x;
        const float ev = fmaf(x2, fmaf(x2, 1.0f / 24.0f, eq[c].a1h), eq[c].a0);
        const float od = x * fmaf(x2, 1.0f / 6.0f, eq[c].a1);
        const float wk = c == 0 ? wk0 : wk1;
        fp[c] = wk * (ev + od);
        fm[c] = wk * (ev - od);
      }
      update(q, sr, st, tb.x, tb.y, at0, kt0, at1, kt1, fp[0], fp[1]);
      update(q + kHalf, -sr, -st, tb.x, tb.y, at0, kt0, at1, kt1, fm[0], fm[1]);
    }
  }
}

cudaError_t launch_step_f32(const CUtensorMap* tmap_in, float* f_out, const StepParams& p,
                            const DvmConst<float>& d, cudaStream_t stream) {
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(step_kernel_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemF32);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  dim3 grid((p.n_r + kTileR - 1) / kTileR, (p.n_theta + kTileT - 1) / kTileT);
  step_kernel_f32<<<grid, kStepThreads, kSmemF32, stream>>>(*tmap_in, f_out, p, d);
  return cudaGetLastError();
}

}  // namespace pclb
