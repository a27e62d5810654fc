// FP32 step for the larger velocity sets of Table I (N_i = 16 and 24
// directions per shell, Q = 65 and 97), tiled like the octagon's kernel: the
// same model (Eqs. 2-5, 10-11, 19 or 18, 28 or the other convection schemes,
// 38-40), 32 (r) x 16 (theta) nodes per block, two radially adjacent nodes
// per thread in packed FP32x2 arithmetic.  A window of all Q planes would not
// fit in shared memory, so:
//   * each thread first forms the moments of its two nodes (Eqs. 3-5) from
//     global memory, in float-float (float shell sums over opposite-direction
//     pairs with float-float unit vectors, shells 2 and 3 added direction by
//     direction first, the shell totals combined with error-free
//     transformations), then the temperature and the equilibrium factors
//     (Eqs. 10-11) in float-float, rounded to float once;
//   * the pairs of opposite velocities (q, q + N_i/2) of each shell then
//     stream, two pairs per stage, through a ring of four shared-memory
//     stages filled by TMA (each plane's window over [r0-4, r0+36) x
//     [t0-2, t0+18)), the copies of the
//     first pairs landing while the moments are formed (and finding the
//     tile's lines in L2);
//   * per pair, the relaxation (Eq. 19 or 18) minus the convection increments
//     in r and theta, summed first and added once, with the float Courant
//     table of the pair; streaming stores, plus the azimuthal ghost rows of
//     the seam (Eq. 40).
// The radial ghost nodes (Sec. II C 1) come from a small per-wall buffer that
// a ghost kernel (one thread per wall row, float-float as the node state)
// writes before the step; tiles at a wall copy them into the window's ghost
// columns once each pair's planes have landed.
#include <cuda.h>
#include <cuda_runtime.h>

#include <atomic>

#include "device_common.cuh"
#include "dvm_generic.h"
#include "f32x2.cuh"
#include "pclb_internal.h"

namespace pclb {

namespace {

constexpr int kTThreads = 16 * kTileT32;            // 256: two nodes each
constexpr int kTPlane = kWinR * (kTileT32 + 4);     // floats per plane window (800)
constexpr int kTStages = 4;                         // ring depth (stages in flight)
constexpr int kTPPS = 2;                            // pairs per stage: one wait and one barrier per two pairs
constexpr int kGhostThreads = 32;                   // ghost kernel: one thread per wall row
static_assert((kTPlane * 4) % 128 == 0, "TMA destinations must stay 128-byte aligned");

template <int ND>
struct TiledSize {
  static constexpr int Q = 1 + 4 * ND, H = ND / 2, NP = 4 * H;   // labels, pairs per shell, pairs
  static constexpr int ring_bytes = kTStages * kTPPS * 2 * kTPlane * 4;
  static constexpr int tab_bytes = NP * kTileT32 * 16;           // one float4 per (pair, row)
  static constexpr int smem = ring_bytes + tab_bytes + 8 * kTStages + 64;
};

__device__ __forceinline__ f2 ldg2(const float* p) { return __ldg(reinterpret_cast<const float2*>(p)); }
__device__ __forceinline__ f2 lds2(const float* p) { return *reinterpret_cast<const float2*>(p); }

__device__ __forceinline__ float rcp_approx_t(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// |D| (D - Dp) / (|D| + |Dp|) of both nodes (0 when D = Dp = 0), Eq. (28) in upwind form.
__device__ __forceinline__ f2 limiter2_t(f2 D, f2 Dp) {
  const f2 aD = abs2(D);
  const f2 den = add2(aD, abs2(Dp));
  const f2 rr = mk2(rcp_approx_t(fmaxf(den.x, 1e-30f)), rcp_approx_t(fmaxf(den.y, 1e-30f)));
  return mul2(mul2(aD, rr), sub2(D, Dp));
}

// Equilibrium factors of two nodes, rounded to float.
struct TEq {
  f2 w[5];              // rho F_k(E)
  f2 a0, a1, a1h;       // Eq. (10) polynomial coefficients
  f2 uxE, uyE;          // u / E
};

// Moments (Eqs. 3-5) of two nodes in float-float: density, velocity and
// temperature.  ld(q) returns the two nodes' f_q.
template <int ND, class LD>
__device__ __forceinline__ void tiled_moments(LD ld, const DvmG32& c, ff2& rho, ff2& ux, ff2& uy, ff2& E) {
  constexpr int H = ND / 2;
  rho = ff2_of(ld(0));
  ff2 jx = ff2_of(bc2(0.f)), jy = jx, e = jx;
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    const int k = g == 0 ? 1 : (g == 1 ? 2 : (g == 2 ? 3 : 4));   // g = 1: shells 2 + 3; g = 2: shell 3
    f2 S = bc2(0.f), X = S, Xl = S, Y = S, Yl = S;
#pragma unroll
    for (int i = 0; i < H; ++i) {
      const int q = 1 + (k - 1) * ND + i;
      f2 fa = ld(q), fb = ld(q + H);
      if (g == 1) {
        fa = add2(fa, ld(q + ND));
        fb = add2(fb, ld(q + ND + H));
      }
      S = add2(S, add2(fa, fb));
      const f2 dd = sub2(fa, fb);   // the pair has opposite unit vectors
      X = fma2(bc2(c.cxh[i]), dd, X);
      Xl = fma2(bc2(c.cxl[i]), dd, Xl);
      Y = fma2(bc2(c.cyh[i]), dd, Y);
      Yl = fma2(bc2(c.cyl[i]), dd, Yl);
    }
    const ff2 sp = g == 2 ? ff2{bc2(c.dv23h), bc2(c.dv23l)} : ff2{bc2(c.sph[k]), bc2(c.spl[k])};
    const ff2 hv = g == 2 ? ff2{bc2(c.dh23h), bc2(c.dh23l)} : ff2{bc2(c.hvh[k]), bc2(c.hvl[k])};
    if (g != 2) rho = ff2_add(rho, ff2_of(S));
    jx = ff2_add(jx, ff2_mul(sp, ff2{X, Xl}));
    jy = ff2_add(jy, ff2_mul(sp, ff2{Y, Yl}));
    e = ff2_add(e, ff2_mul(hv, ff2_of(S)));
  }
  const ff2 inv = ff2_recip(rho);
  ux = ff2_mul(jx, inv);
  uy = ff2_mul(jy, inv);
  const ff2 ke = ff2_add(ff2_mul(jx, ux), ff2_mul(jy, uy));   // |j|^2 / rho
  E = ff2_mul(ff2_add(e, ff2_scale(ke, -0.5f)), inv);
}

// Equilibrium factors (Eqs. 10-11) of two states in float-float, rounded to
// float once.
__device__ __forceinline__ TEq tiled_factors(const ff2& rho, const ff2& ux, const ff2& uy, const ff2& E,
                                             const DvmG32& c) {
  TEq q;
  ff2 sum = ff2_of(bc2(0.f));
#pragma unroll
  for (int k = 1; k <= 4; ++k) {
    ff2 a{bc2(c.Fch[k][3]), bc2(c.Fcl[k][3])};
#pragma unroll
    for (int n = 2; n >= 0; --n) a = ff2_mul_add(a, E, ff2{bc2(c.Fch[k][n]), bc2(c.Fcl[k][n])});
    a = ff2_mul(a, E);   // F_k(E)
    sum = ff2_add(sum, a);
    q.w[k] = ff2_round(ff2_mul(rho, a));
  }
  q.w[0] = ff2_round(ff2_mul(rho, ff2_add(ff2_of(bc2(1.f)), ff2_mul(ff2{bc2(-c.B0h), bc2(-c.B0l)}, sum))));
  const ff2 invE = ff2_recip(E);
  const ff2 uxE = ff2_mul(ux, invE), uyE = ff2_mul(uy, invE);
  const ff2 u2E = ff2_add(ff2_mul(ux, uxE), ff2_mul(uy, uyE));   // u^2 / E
  const ff2 a1 = ff2_add(ff2_of(bc2(1.f)), ff2_scale(u2E, -0.5f));
  const ff2 a0 = ff2_add(a1, ff2_scale(ff2_mul(u2E, u2E), 0.125f));
  q.a1 = ff2_round(a1);
  q.a0 = ff2_round(a0);
  q.a1h = mul2(bc2(0.5f), q.a1);
  q.uxE = ff2_round(uxE);
  q.uyE = ff2_round(uyE);
  return q;
}

__device__ __forceinline__ bool phys_x(const ff2& rho, const ff2& ux, const ff2& uy, const ff2& E) {
  return rho.hi.x > 0.f && E.hi.x > 0.f && isfinite(E.hi.x) && isfinite(ux.hi.x) && isfinite(uy.hi.x);
}
__device__ __forceinline__ bool phys_y(const ff2& rho, const ff2& ux, const ff2& uy, const ff2& E) {
  return rho.hi.y > 0.f && E.hi.y > 0.f && isfinite(E.hi.y) && isfinite(ux.hi.y) && isfinite(uy.hi.y);
}

// Moments and equilibrium factors of the two radially adjacent nodes at fn
// (global, planes `plane` apart); the physical flags in ok0, ok1.
template <int ND>
__device__ __forceinline__ TEq tiled_state(const float* fn, size_t plane, const DvmG32& c, bool& ok0, bool& ok1) {
  ff2 rho, ux, uy, E;
  tiled_moments<ND>([&](int q) { return ldg2(fn + (size_t)q * plane); }, c, rho, ux, uy, E);
  ok0 = phys_x(rho, ux, uy, E);
  ok1 = phys_y(rho, ux, uy, E);
  return tiled_factors(rho, ux, uy, E, c);
}

// The pair of equilibria f^eq(+-v) of both states (Eq. 10): P(+-x) = ev +- od
// with x = v.u/E, times w.
__device__ __forceinline__ void tiled_feq_pair(const TEq& e, f2 w, float vx, float vy, f2& fp, f2& fm) {
  const f2 x = fma2(bc2(vx), e.uxE, mul2(bc2(vy), e.uyE));
  const f2 x2 = mul2(x, x);
  const f2 ev = fma2(x2, fma2(x2, bc2(1.0f / 24.0f), e.a1h), e.a0);
  const f2 od = mul2(x, fma2(x2, bc2(1.0f / 6.0f), e.a1));
  const f2 wev = mul2(w, ev);
  fp = fma2(w, od, wev);
  fm = fma2(neg2(w), od, wev);
}

// (v, v) as a float-float pair from a double.
__device__ __forceinline__ ff2 ff2_from_double(double v) {
  const float h = (float)v;
  return ff2{bc2(h), bc2((float)(v - (double)h))};
}

// Radial ghost layers of wall `side` at row t into ghost [side][layer][n_theta][Q]
// (Sec. II C 1): Eq. (39) applied twice to the wall node a and the next node
// b, g0 = 2a - b and g1 = 2 g0 - a = 3a - 2b, for the components the boundary
// kind extrapolates, the others prescribed; the ghost distribution is the
// equilibrium of that state, plus the wall node's departure from equilibrium
// for non-equilibrium ghosts.  All in float-float and float, as the step's
// node state: the two layers are the two halves of the packed arithmetic.
template <int ND>
__global__ void __launch_bounds__(kGhostThreads)
    tiled_ghost_f32(const float* __restrict__ f, float* __restrict__ ghost, const __grid_constant__ StepParams p,
                    const __grid_constant__ DvmG d, const __grid_constant__ DvmG32 c) {
  constexpr int Q = 1 + 4 * ND, H = ND / 2;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int side = blockIdx.y;
  if (t >= p.n_theta) return;
  const size_t plane = (size_t)p.rows * p.pitch;
  const int ra = side == 0 ? 0 : p.n_r - 1, rb = side == 0 ? 1 : p.n_r - 2;
  const float* fa = f + (size_t)(t + kGhostRows) * p.pitch + ra;
  const float* fb = f + (size_t)(t + kGhostRows) * p.pitch + rb;
  // node a in the low half, node b in the high half
  ff2 m[4];
  tiled_moments<ND>([&](int q) { return mk2(__ldg(fa + (size_t)q * plane), __ldg(fb + (size_t)q * plane)); }, c,
                    m[0], m[1], m[2], m[3]);
  bool ok = phys_x(m[0], m[1], m[2], m[3]) && phys_y(m[0], m[1], m[2], m[3]);
  const TEq ea = tiled_factors(m[0], m[1], m[2], m[3], c);
  ff2 g[4];   // (g0, g1) of rho, u_x, u_y, E
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const ff2 A{bc2(m[i].hi.x), bc2(m[i].lo.x)}, B{bc2(m[i].hi.y), bc2(m[i].lo.y)};
    g[i] = ff2_add(ff2_mul(A, ff2{mk2(2.f, 3.f), bc2(0.f)}), ff2_mul(B, ff2{mk2(-1.f, -2.f), bc2(0.f)}));
  }
  const int kind = p.bc_kind[side] & ~PCLB_BC_NEQ;
  const bool neq = (p.bc_kind[side] & PCLB_BC_NEQ) != 0;
  if (kind != PCLB_BC_EXTRAP) {
    const double cs = p.cos_t[t], sn = p.sin_t[t];
    ff2 v[4];
    for (int l = 0; l < 2; ++l) {
      const double* bv = p.bc_vals + (size_t)((side * 2 + l) * 4) * p.n_theta + t;
      const double ur = bv[1 * p.n_theta], ut = bv[2 * p.n_theta];
      const double x[4] = {bv[0], ur * cs - ut * sn, ur * sn + ut * cs, bv[3 * p.n_theta]};
      for (int i = 0; i < 4; ++i) {
        const ff2 y = ff2_from_double(x[i]);
        if (l == 0) v[i] = y; else { v[i].hi.y = y.hi.y; v[i].lo.y = y.lo.y; }
      }
    }
    g[1] = v[1];
    g[2] = v[2];
    if (kind == PCLB_BC_DIRICHLET) {
      g[0] = v[0];
      g[3] = v[3];
    }
  }
  ok = ok && g[0].hi.x > 0.f && g[3].hi.x > 0.f && g[0].hi.y > 0.f && g[3].hi.y > 0.f;
  if (!ok) atomicOr(p.status, PCLB_FLAG_NONPHYS);
  const TEq eg = tiled_factors(g[0], g[1], g[2], g[3], c);
  float* out0 = ghost + ((size_t)(side * 2 + 0) * p.n_theta + t) * Q;
  float* out1 = ghost + ((size_t)(side * 2 + 1) * p.n_theta + t) * Q;
  {
    f2 v = mul2(eg.w[0], eg.a0);
    if (neq) v = add2(v, bc2(fa[0] - ea.w[0].x * ea.a0.x));
    out0[0] = v.x;
    out1[0] = v.y;
  }
#pragma unroll 1
  for (int pr = 0; pr < 4 * H; ++pr) {
    const int k = 1 + pr / H, q1 = 1 + (k - 1) * ND + pr % H, q2 = q1 + H;
    const f2 wg = k == 1 ? eg.w[1] : (k == 2 ? eg.w[2] : (k == 3 ? eg.w[3] : eg.w[4]));
    f2 gp, gm;
    tiled_feq_pair(eg, wg, c.vx[q1], c.vy[q1], gp, gm);
    if (neq) {
      const f2 wa = k == 1 ? ea.w[1] : (k == 2 ? ea.w[2] : (k == 3 ? ea.w[3] : ea.w[4]));
      f2 ap, am;
      tiled_feq_pair(ea, wa, c.vx[q1], c.vy[q1], ap, am);
      gp = add2(gp, bc2(fa[(size_t)q1 * plane] - ap.x));
      gm = add2(gm, bc2(fa[(size_t)q2 * plane] - am.x));
    }
    out0[q1] = gp.x;
    out1[q1] = gp.y;
    out0[q2] = gm.x;
    out1[q2] = gm.y;
  }
}

// One label of a pair at the thread's two nodes with its upwind offsets as
// constants (SU: columns, SV: rows): the relaxation minus the convection
// increments in r and theta, summed first and added once.  The two rows of a
// warp share the offsets nearly everywhere (a label's upwind side changes at
// a few theta rows only), so the dispatch below is uniform in practice.
template <int SCH, int SU, int SV, class Store>
__device__ __forceinline__ void tupd(const float* w, f2 nar, f2 nkr, f2 nat, f2 nkt, f2 fe, f2 decay, int q, Store& store) {
  const f2 C = lds2(w);
  const f2 S = lds2(w + 2 * SU);
  const f2 T1 = lds2(w + SV * kWinR);
  const f2 T2 = lds2(w + 2 * SV * kWinR);
  const f2 u1 = SU < 0 ? mk2(S.y, C.x) : mk2(C.y, S.x);
  const f2 Dr = sub2(C, u1), Dt = sub2(C, T1);
  f2 dc = mul2(nar, Dr);
  dc = fma2(nat, Dt, dc);
  if constexpr (SCH == PCLB_SCHEME_MWB) {
    dc = fma2(nkr, limiter2_t(Dr, sub2(u1, S)), dc);
    dc = fma2(nkt, limiter2_t(Dt, sub2(T1, T2)), dc);
  } else if constexpr (SCH == PCLB_SCHEME_WB) {
    dc = fma2(mul2(bc2(0.5f), nkr), sub2(Dr, sub2(u1, S)), dc);
    dc = fma2(mul2(bc2(0.5f), nkt), sub2(Dt, sub2(T1, T2)), dc);
  } else if constexpr (SCH == PCLB_SCHEME_UPWIND2) {
    dc = fma2(mul2(bc2(0.5f), nar), sub2(Dr, sub2(u1, S)), dc);
    dc = fma2(mul2(bc2(0.5f), nat), sub2(Dt, sub2(T1, T2)), dc);
  } else {
    const f2 X = lds2(w - 2 * SU);
    const f2 d1 = SU < 0 ? mk2(C.y, X.x) : mk2(X.y, C.x);
    const f2 Td = lds2(w - SV * kWinR);
    dc = fma2(mul2(bc2(0.5f), nkr), sub2(sub2(d1, C), Dr), dc);
    dc = fma2(mul2(bc2(0.5f), nkt), sub2(sub2(Td, C), Dt), dc);
  }
  store(q, add2(fma2(sub2(C, fe), decay, fe), dc));
}

// Three CTAs per SM (at most 85 registers; a few bytes spill in some
// instantiations): 12% faster than two CTAs at 124 registers.
template <int ND, int SCH>
__global__ void __launch_bounds__(kTThreads, 3)
    tiled_step_f32(const __grid_constant__ CUtensorMap tmap, const float* __restrict__ f, float* __restrict__ f_out,
                   const float* __restrict__ ghost, const __grid_constant__ StepParams p,
                   const __grid_constant__ DvmG d, const __grid_constant__ DvmG32 c) {
  using TS = TiledSize<ND>;
  constexpr int H = TS::H, NP = TS::NP, Q = TS::Q;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* ring = reinterpret_cast<float*>(smem_raw);
  float4* tab = reinterpret_cast<float4*>(smem_raw + TS::ring_bytes);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + TS::ring_bytes + TS::tab_bytes);

  const int r0 = blockIdx.x * kTileR;
  const int t0 = blockIdx.y * kTileT32;
  const int tid = threadIdx.x;

  // the planes of the kTPPS pairs of stage group sg into stage s (thread 0)
  auto issue = [&](int sg, int s) {
    float* st = ring + s * kTPPS * 2 * kTPlane;
    mbar_arrive_expect_tx(&full[s], (uint32_t)(kTPPS * 2 * kTPlane * 4));
    for (int pp = 0; pp < kTPPS; ++pp) {
      const int pr = sg * kTPPS + pp;
      const int q1 = 1 + (pr / H) * ND + pr % H;
      tma_load_3d(st + pp * 2 * kTPlane, &tmap, r0 - kLeft, t0, q1, &full[s]);
      tma_load_3d(st + pp * 2 * kTPlane + kTPlane, &tmap, r0 - kLeft, t0, q1 + H, &full[s]);
    }
  };
  constexpr int NS = NP / kTPPS;
  static_assert(NP % kTPPS == 0, "whole stages");
  if (tid == 0) {
    tma_prefetch_desc(&tmap);
    for (int s = 0; s < kTStages; ++s) mbar_init(&full[s], 1);
    mbar_fence_init();
    for (int s = 0; s < kTStages && s < NS; ++s) issue(s, s);
  }
  for (int i = tid; i < NP * kTileT32; i += kTThreads) {   // Courant entries: [pair][row]
    const int pr = i / kTileT32, rl = i % kTileT32;
    const int t = min(t0 + rl, p.n_theta - 1);
    tab[i] = p.courant[(size_t)(t + kGhostRows) * NP + pr];
  }
  __syncthreads();   // barriers initialised, table visible

  const int warp = tid >> 5, lane = tid & 31;
  const int rl = 2 * warp + (lane >> 4);       // tile row 0..15
  const int j2 = 2 * (lane & 15);               // even radial offset 0..30
  const int t = t0 + rl, r = r0 + j2;
  const bool row_ok = t < p.n_theta;
  const bool v0 = row_ok && r < p.n_r, v1 = row_ok && r + 1 < p.n_r;
  const size_t plane = (size_t)p.rows * p.pitch;
  // rows past the grid read the last row (their results are not stored);
  // columns past n_r read the row's padding (r + 1 < pitch)
  const int srow = min(t, p.n_theta - 1) + kGhostRows;
  const float* fn = f + (size_t)srow * p.pitch + r;

  TEq eq;
  f2 f0;
  {
    bool ok0, ok1;
    f0 = ldg2(fn);
    eq = tiled_state<ND>(fn, plane, c, ok0, ok1);
    if ((v0 && !ok0) || (v1 && !ok1)) atomicOr(p.status, PCLB_FLAG_NONPHYS);
    // lanes without a valid node: any finite factors (never stored)
    if (!v0 || !ok0) { for (int k = 0; k < 5; ++k) eq.w[k].x = 0.f; eq.a0.x = 1.f; eq.a1.x = 1.f; eq.a1h.x = 0.5f; eq.uxE.x = 0.f; eq.uyE.x = 0.f; }
    if (!v1 || !ok1) { for (int k = 0; k < 5; ++k) eq.w[k].y = 0.f; eq.a0.y = 1.f; eq.a1.y = 1.f; eq.a1h.y = 0.5f; eq.uxE.y = 0.f; eq.uyE.y = 0.f; }
  }

  const f2 invr = mk2(v0 ? p.inv_r_f[r] : 1.f, v1 ? p.inv_r_f[r + 1] : 1.f);
  const f2 decay = bc2((float)p.decay);
  float* out_row = f_out + (size_t)(t + kGhostRows) * p.pitch + r;
  const bool lo_ghost = row_ok && t >= p.n_theta - 2;
  const bool hi_ghost = row_ok && t < 2;
  float* out_lo = f_out + (size_t)max(t - (p.n_theta - 2), 0) * p.pitch + r;
  float* out_hi = f_out + (size_t)(p.n_theta + kGhostRows + t) * p.pitch + r;
  const bool plain_tile = r0 + kTileR <= p.n_r && t0 >= 2 && t0 + kTileT32 <= p.n_theta - 2;
  auto store = [&](int q, f2 o) {
    if (plain_tile) {
      __stcs(reinterpret_cast<float2*>(out_row + (size_t)q * plane), o);
    } else if (v1) {
      *reinterpret_cast<float2*>(out_row + (size_t)q * plane) = o;
      if (lo_ghost) *reinterpret_cast<float2*>(out_lo + (size_t)d.recv_lo[q] * plane) = o;
      if (hi_ghost) *reinterpret_cast<float2*>(out_hi + (size_t)d.recv_hi[q] * plane) = o;
    } else if (v0) {
      out_row[(size_t)q * plane] = o.x;
      if (lo_ghost) out_lo[(size_t)d.recv_lo[q] * plane] = o.x;
      if (hi_ghost) out_hi[(size_t)d.recv_hi[q] * plane] = o.x;
    }
  };
  {  // rest velocity: no convection
    const f2 e0 = mul2(eq.w[0], eq.a0);
    store(0, fma2(sub2(f0, e0), decay, e0));
  }

  // wall tiles: ghost columns of both walls (inner: window columns kLeft - 1,
  // kLeft - 2; outer: cw_out + 1, cw_out + 2) for the tile rows
  const int cw_out = p.n_r - 1 - r0 + kLeft;
  const bool inner = r0 == 0, outer = cw_out <= kLeft + kTileR;
  const int row = rl + 2, col = kLeft + j2;
  bool ok = true;
#pragma unroll 1
  for (int sg = 0; sg < NS; ++sg) {
    const int s = sg % kTStages;
    if (ok) ok = p.wait_ns != 0 && mbar_wait_bounded(&full[s], (uint32_t)((sg / kTStages) & 1), p.wait_ns);
    float* stg = ring + s * kTPPS * 2 * kTPlane;
    if (inner || outer) {
      // per pair: 2 walls x 2 labels x 2 layers x 16 rows
      for (int it = tid; it < kTPPS * 128 && ok; it += kTThreads) {
        const int P = it >> 7, side = (it >> 6) & 1, L = (it >> 5) & 1, layer = (it >> 4) & 1, rr = it & 15;
        const int pr = sg * kTPPS + P;
        const int q1 = 1 + (pr / H) * ND + pr % H, q2 = q1 + H;
        const int tt = t0 + rr;
        if ((side == 0 ? inner : outer) && tt < p.n_theta) {
          const int cg = side == 0 ? kLeft - 1 - layer : cw_out + 1 + layer;
          if (cg >= 0 && cg < kWinR)
            stg[P * 2 * kTPlane + L * kTPlane + (rr + 2) * kWinR + cg] =
                ghost[((size_t)(side * 2 + layer) * p.n_theta + tt) * Q + (L ? q2 : q1)];
        }
      }
      __syncthreads();
    }
    if (ok) {
#pragma unroll
      for (int pp = 0; pp < kTPPS; ++pp) {
        const int pr = sg * kTPPS + pp;
        const int k = 1 + pr / H, i = pr % H;
        const int q1 = 1 + (k - 1) * ND + i, q2 = q1 + H;
        const float4 tb = tab[pr * kTileT32 + rl];
        const int fl = __float_as_int(tb.w);
        const f2 nar = bc2(-tb.x), nkr = bc2(-tb.y);
        const f2 nat = mul2(bc2(-tb.z), invr);
        const f2 nkt = fma2(nat, nat, nat);           // -(a - a^2) with a = -nat
        // equilibrium of the pair (Eq. 10): P(+-x) = ev +- od, x = v.u/E
        const f2 wk = k == 1 ? eq.w[1] : (k == 2 ? eq.w[2] : (k == 3 ? eq.w[3] : eq.w[4]));
        f2 fe[2];
        tiled_feq_pair(eq, wk, c.vx[q1], c.vy[q1], fe[0], fe[1]);
        const float* w0 = stg + pp * 2 * kTPlane + row * kWinR + col;
        const float* w1 = w0 + kTPlane;
        // bit 0: q1's upwind side at larger r; bit 1: at larger theta (q2 the opposite)
        switch (fl & 3) {
          case 0:
            tupd<SCH, -1, -1>(w0, nar, nkr, nat, nkt, fe[0], decay, q1, store);
            tupd<SCH, 1, 1>(w1, nar, nkr, nat, nkt, fe[1], decay, q2, store);
            break;
          case 1:
            tupd<SCH, 1, -1>(w0, nar, nkr, nat, nkt, fe[0], decay, q1, store);
            tupd<SCH, -1, 1>(w1, nar, nkr, nat, nkt, fe[1], decay, q2, store);
            break;
          case 2:
            tupd<SCH, -1, 1>(w0, nar, nkr, nat, nkt, fe[0], decay, q1, store);
            tupd<SCH, 1, -1>(w1, nar, nkr, nat, nkt, fe[1], decay, q2, store);
            break;
          default:
            tupd<SCH, 1, 1>(w0, nar, nkr, nat, nkt, fe[0], decay, q1, store);
            tupd<SCH, -1, -1>(w1, nar, nkr, nat, nkt, fe[1], decay, q2, store);
            break;
        }
      }
    }
    // the stage is read by every thread before it is refilled; a copy that
    // did not land in time stops the tile
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicOr(p.status, PCLB_FLAG_TIMEOUT);
        for (int gg = sg; gg < sg + kTStages && gg < NS; ++gg)
          mbar_wait_bounded(&full[gg % kTStages], (uint32_t)((gg / kTStages) & 1), kDefaultWaitNs);
      }
      return;
    }
    if (tid == 0 && sg + kTStages < NS) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(sg + kTStages, s);
    }
  }
}

template <int ND, int SCH>
cudaError_t launch_tiled(const CUtensorMap* tmap, const float* f, float* f_out, const float* ghost, const StepParams& p,
                         const DvmG& d, const DvmG32& c, cudaStream_t s) {
  static std::atomic<unsigned long long> configured{0};
  constexpr int smem = TiledSize<ND>::smem;
  {
    const cudaError_t e = set_smem_once(tiled_step_f32<ND, SCH>, smem, configured);
    if (e != cudaSuccess) return e;
  }
  const dim3 grid((p.n_r + kTileR - 1) / kTileR, (p.n_theta + kTileT32 - 1) / kTileT32);
  tiled_step_f32<ND, SCH><<<grid, kTThreads, smem, s>>>(*tmap, f, f_out, ghost, p, d, c);
  return cudaGetLastError();
}

template <int ND>
cudaError_t launch_tiled_nd(const CUtensorMap* tmap, const float* f, float* f_out, const float* ghost,
                            const StepParams& p, const DvmG& d, const DvmG32& c, cudaStream_t s) {
  switch (p.scheme) {
    case PCLB_SCHEME_WB: return launch_tiled<ND, PCLB_SCHEME_WB>(tmap, f, f_out, ghost, p, d, c, s);
    case PCLB_SCHEME_LW: return launch_tiled<ND, PCLB_SCHEME_LW>(tmap, f, f_out, ghost, p, d, c, s);
    case PCLB_SCHEME_UPWIND2: return launch_tiled<ND, PCLB_SCHEME_UPWIND2>(tmap, f, f_out, ghost, p, d, c, s);
    default: return launch_tiled<ND, PCLB_SCHEME_MWB>(tmap, f, f_out, ghost, p, d, c, s);
  }
}

}  // namespace

// One FP32 step of the N_i = 16 or 24 set: the radial ghost layers, then the
// tiled kernel over the whole grid (the same stream orders them).  tmap describes f (box kWinR x
// (kTileT32 + 4) x 1, Q planes).
cudaError_t gen_tiled_step_f32(const CUtensorMap* tmap, const float* f, float* f_out, float* ghost,
                               const StepParams& p, const DvmG& d, const DvmG32& c, cudaStream_t s) {
  const dim3 ggrid((p.n_theta + kGhostThreads - 1) / kGhostThreads, 2);
  if (d.n_dirs == 16) {
    tiled_ghost_f32<16><<<ggrid, kGhostThreads, 0, s>>>(f, ghost, p, d, c);
    const cudaError_t e = cudaGetLastError();
    return e != cudaSuccess ? e : launch_tiled_nd<16>(tmap, f, f_out, ghost, p, d, c, s);
  }
  tiled_ghost_f32<24><<<ggrid, kGhostThreads, 0, s>>>(f, ghost, p, d, c);
  const cudaError_t e = cudaGetLastError();
  return e != cudaSuccess ? e : launch_tiled_nd<24>(tmap, f, f_out, ghost, p, d, c, s);
}

}  // namespace pclb
