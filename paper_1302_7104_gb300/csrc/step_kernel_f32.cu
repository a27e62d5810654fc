// Fused FP32 time step of the polar-coordinate FDLB model (Eq. 38), the hot
// kernel of the library.
//
// Work per CTA: a tile of 32 (r) x 16 (theta) nodes, 256 threads.  One thread
// issues 33 TMA box copies (one per velocity plane) of the window
// [r0-4, r0+36) x [t0-2, t0+18) into shared memory, in four groups with a
// barrier each (rest + shell 1, shells 2, 3, 4), while the others copy the
// tile's rows of the host-computed Courant table.  Each thread then owns two
// radially adjacent nodes of one row and processes them together with packed
// FP32x2 arithmetic:
//   * moments (Eqs. 3-5), temperature recovery and the weights rho F_k(E)
//     (Eqs. 11a-b) in float-float arithmetic, so that the rounded equilibrium
//     keeps the collision invariants of the exact one;
//   * radial ghost columns for tiles at a wall (Eq. 39, f = f^eq), computed in
//     shared memory;
//   * for every pair (q, q') of opposite velocities of a shell: v_q.u/E from
//     float-float constants, the even and odd parts of the equilibrium
//     polynomial (Eq. 10) shared by q and q'; then per velocity the relaxation
//     (Eq. 19) minus the MWB increments (Eq. 28) in r and theta, stored with
//     8-byte streaming stores, plus the azimuthal ghost rows of the seam
//     (Eq. 40).  The convection increments -M_r - M_theta are summed first
//     and added once to the relaxed value, so that they cost one rounding at
//     the magnitude of f instead of four (this halves the FP32 path's drift
//     from the FP64 one over long runs).
#include <cuda.h>
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "f32_eq2.cuh"
#include "f32_state.cuh"
#include "f32x2.cuh"
#include "pclb_internal.h"

namespace pclb {

namespace {

constexpr int kPairs = 4 * kHalf;                    // 16
constexpr int kPlaneF = kWinR * (kTileT32 + 4);      // floats per plane window
constexpr int kPlanesBytes = kQ * kPlaneF * 4;       // 105600
constexpr int kTabBytes = kPairs * kTileT32 * 16;    // one float4 per (pair, row)
constexpr int kSmemF32 = kPlanesBytes + kTabBytes + 128;
// every plane window is a TMA destination: 128-byte aligned (a tile height
// whose window breaks this faults with a misaligned address)
static_assert((kPlaneF * 4) % 128 == 0 && kPlanesBytes % 16 == 0, "TMA destinations must stay 128-byte aligned");
constexpr int kGroups = 4;
__device__ __forceinline__ int group_first(int g) { return g == 0 ? 0 : 1 + g * kNDirs; }
__device__ __forceinline__ int group_planes(int g) { return g == 0 ? 1 + kNDirs : kNDirs; }

__device__ __forceinline__ f2 ld2(const float* p) { return *reinterpret_cast<const float2*>(p); }

// Sums over one shell (plus, optionally, a second shell added direction by
// direction) of f, c_x f and c_y f for both nodes, with the octagon's exact
// unit vectors as float-float constants.
template <int K, int KADD>
__device__ __forceinline__ void shell_sums2(const float* f, f2& S, f2& X, f2& Xl, f2& Y, f2& Yl) {
  S = bc2(0.f); X = bc2(0.f); Xl = bc2(0.f); Y = bc2(0.f); Yl = bc2(0.f);
#pragma unroll
  for (int i = 0; i < kHalf; ++i) {
    const int q = 1 + (K - 1) * kNDirs + i;
    f2 fa = ld2(f + q * kPlaneF), fb = ld2(f + (q + kHalf) * kPlaneF);
    if (KADD > 0) {
      const int qa = 1 + (KADD - 1) * kNDirs + i;
      fa = add2(fa, ld2(f + qa * kPlaneF));
      fb = add2(fb, ld2(f + (qa + kHalf) * kPlaneF));
    }
    S = add2(S, add2(fa, fb));
    const f2 dd = sub2(fa, fb);
    if (i == 0) {
      X = add2(X, dd);
    } else if (i == 2) {
      Y = add2(Y, dd);
    } else {
      const float sx = i == 1 ? 1.f : -1.f;
      X = fma2(bc2(sx * kS), dd, X);
      Xl = fma2(bc2(sx * kSl), dd, Xl);
      Y = fma2(bc2(kS), dd, Y);
      Yl = fma2(bc2(kSl), dd, Yl);
    }
  }
}

// Moments (Eqs. 3-5) and temperature recovery of the two nodes.  ready(g)
// is called before plane group g (the rest plane and shell 1, then shells 2,
// 3, 4) is first read, so the sums start while later groups still land.
template <class Ready>
__device__ __forceinline__ State2 state2(const float* f, const DvmConst<float>& d, Ready ready) {
  ready(0);
  ff2 rho = ff2_of(ld2(f)), jx = ff2_of(bc2(0.f)), jy = jx, e = jx;
  f2 S, X, Xl, Y, Yl;
  // shell 1
  shell_sums2<1, 0>(f, S, X, Xl, Y, Yl);
  rho = ff2_add(rho, ff2_of(S));
  jx = ff2_add(jx, ff2_mul(ffc(d.speed[1], d.speed_lo[1]), ff2{X, Xl}));
  jy = ff2_add(jy, ff2_mul(ffc(d.speed[1], d.speed_lo[1]), ff2{Y, Yl}));
  e = ff2_add(e, ff2_mul(ffc(d.half_v2[1], d.half_v2_lo[1]), ff2_of(S)));
  // shells 2 + 3 direction by direction, with the speed and v^2/2 of shell 2
  ready(1);
  ready(2);
  shell_sums2<2, 3>(f, S, X, Xl, Y, Yl);
  rho = ff2_add(rho, ff2_of(S));
  jx = ff2_add(jx, ff2_mul(ffc(d.speed[2], d.speed_lo[2]), ff2{X, Xl}));
  jy = ff2_add(jy, ff2_mul(ffc(d.speed[2], d.speed_lo[2]), ff2{Y, Yl}));
  e = ff2_add(e, ff2_mul(ffc(d.half_v2[2], d.half_v2_lo[2]), ff2_of(S)));
  // shell 3 again with the differences v_3 - v_2, (v_3^2 - v_2^2)/2
  shell_sums2<3, 0>(f, S, X, Xl, Y, Yl);
  jx = ff2_add(jx, ff2_mul(ffc(d.dv23, d.dv23_lo), ff2{X, Xl}));
  jy = ff2_add(jy, ff2_mul(ffc(d.dv23, d.dv23_lo), ff2{Y, Yl}));
  e = ff2_add(e, ff2_mul(ffc(d.dh23, d.dh23_lo), ff2_of(S)));
  // shell 4
  ready(3);
  shell_sums2<4, 0>(f, S, X, Xl, Y, Yl);
  rho = ff2_add(rho, ff2_of(S));
  jx = ff2_add(jx, ff2_mul(ffc(d.speed[4], d.speed_lo[4]), ff2{X, Xl}));
  jy = ff2_add(jy, ff2_mul(ffc(d.speed[4], d.speed_lo[4]), ff2{Y, Yl}));
  e = ff2_add(e, ff2_mul(ffc(d.half_v2[4], d.half_v2_lo[4]), ff2_of(S)));

  State2 s;
  const ff2 inv = ff2_recip(rho);
  s.rho = rho;
  s.ux = ff2_mul(jx, inv);
  s.uy = ff2_mul(jy, inv);
  const ff2 ke = ff2_add(ff2_mul(jx, s.ux), ff2_mul(jy, s.uy));    // |j|^2 / rho
  s.E = ff2_mul(ff2_add(e, ff2_scale(ke, -0.5f)), inv);
  return s;
}

// Ghost columns of one wall for tile row `row` (window row index), Sec. II C 1.
__device__ __noinline__ void ghost_columns_f32(float* sm, int row, int side, int cw, int t,
                                               const StepParams& p, const DvmConst<float>& d) {
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
  const int kind = p.bc_kind[side] & ~PCLB_BC_NEQ;
  const bool neq = (p.bc_kind[side] & PCLB_BC_NEQ) != 0;
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
  // equilibrium of the wall node, for the departure it hands to its ghosts
  Eq32 ea{};
  if (neq) ea = eq32(a, d);
  const float* fa = sm + row * kWinR + cw;
  for (int layer = 0; layer < 2; ++layer) {
    ok = ok && g[layer].rho.hi > 0.f && g[layer].E.hi > 0.f;
    const int col = cw - step * (1 + layer);
    if (col < 0 || col >= kWinR) continue;
    const Eq32 e = eq32(g[layer], d);
    float* gp = sm + row * kWinR + col;
    gp[0] = feq32(e, d, 0, 0, 1.f) + (neq ? fa[0] - feq32(ea, d, 0, 0, 1.f) : 0.f);
#pragma unroll 1
    for (int k = 1; k <= 4; ++k)
#pragma unroll
      for (int i = 0; i < kHalf; ++i) {
        const int q = 1 + (k - 1) * kNDirs + i;
        float v1 = feq32(e, d, k, i, 1.f), v2 = feq32(e, d, k, i, -1.f);
        if (neq) {
          v1 += fa[q * kPlaneF] - feq32(ea, d, k, i, 1.f);
          v2 += fa[(q + kHalf) * kPlaneF] - feq32(ea, d, k, i, -1.f);
        }
        gp[q * kPlaneF] = v1;
        gp[(q + kHalf) * kPlaneF] = v2;
      }
  }
  if (!ok) atomicOr(p.status, PCLB_FLAG_NONPHYS);
}

__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Limiter part of the MWB increment of both nodes, |D| (D - Dp) / (|D| + |Dp|)
// (0 when D = Dp = 0), Eq. (28) in upwind form.
__device__ __forceinline__ f2 limiter2(f2 D, f2 Dp) {
  const f2 aD = abs2(D);
  const f2 den = add2(aD, abs2(Dp));
  const f2 rr = mk2(rcp_approx(fmaxf(den.x, 1e-30f)), rcp_approx(fmaxf(den.y, 1e-30f)));
  return mul2(mul2(aD, rr), sub2(D, Dp));
}

}  // namespace

template <int SCH>
__global__ void __launch_bounds__(kStepThreads32, kCtasPerSm32)
    step_kernel_f32(const __grid_constant__ CUtensorMap tmap_in, float* __restrict__ f_out,
                    const __grid_constant__ StepParams p, const __grid_constant__ DvmConst<float> d, int ty0) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* sm = reinterpret_cast<float*>(smem_raw);
  float4* tab = reinterpret_cast<float4*>(smem_raw + kPlanesBytes);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + kPlanesBytes + kTabBytes);

  const int r0 = blockIdx.x * kTileR;
  const int t0 = (blockIdx.y + ty0) * kTileT32;   // ty0: first tile row of the launch
  const int tid = threadIdx.x;

  // Thread 0 initialises the barriers and issues the copies at once; the
  // block barrier below (after the table fill) makes the initialised
  // barriers visible to the other threads before their first wait.
  if (tid == 0) {
    tma_prefetch_desc(&tmap_in);
    for (int g = 0; g < kGroups; ++g) mbar_init(&bar[g], 1);
    mbar_fence_init();
#pragma unroll 1
    for (int g = 0; g < kGroups; ++g) {
      const int q0 = group_first(g), n = group_planes(g);
      mbar_arrive_expect_tx(&bar[g], (uint32_t)(n * kPlaneF * 4));
#pragma unroll 1
      for (int q = q0; q < q0 + n; ++q) tma_load_3d(sm + q * kPlaneF, &tmap_in, r0 - kLeft, t0, q, &bar[g]);
    }
  }
  {  // Courant entries of the tile rows: table layout [pair][row]
    const int pair = tid / kTileT32, rl = tid % kTileT32;
    const int t = min(t0 + rl, p.n_theta - 1);
    tab[pair * kTileT32 + rl] = p.courant[(size_t)(t + kGhostRows) * kPairs + pair];
  }
  __syncthreads();   // table visible (while the copies are still landing)
  bool ok = true;

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
  const float* win = sm + row * kWinR + col;

  Eq2 eq;
  {
    auto ready = [&](int g) {
      if (ok) ok = p.wait_ns != 0 && mbar_wait_bounded(&bar[g], 0, p.wait_ns);   // 0: give up at once
    };
    State2 s = state2(win, d, ready);
    const bool ok0 = s.rho.hi.x > 0.f && s.E.hi.x > 0.f && isfinite(s.E.hi.x) && isfinite(s.ux.hi.x) &&
                     isfinite(s.uy.hi.x);
    const bool ok1 = s.rho.hi.y > 0.f && s.E.hi.y > 0.f && isfinite(s.E.hi.y) && isfinite(s.ux.hi.y) &&
                     isfinite(s.uy.hi.y);
    if (ok && ((v0 && !ok0) || (v1 && !ok1))) atomicOr(p.status, PCLB_FLAG_NONPHYS);
    // keep lanes without a valid node finite (their results are never stored)
    if (!v0) { s.rho.hi.x = 1.f; s.rho.lo.x = 0.f; s.E.hi.x = 1.f; s.E.lo.x = 0.f;
               s.ux.hi.x = 0.f; s.ux.lo.x = 0.f; s.uy.hi.x = 0.f; s.uy.lo.x = 0.f; }
    if (!v1) { s.rho.hi.y = 1.f; s.rho.lo.y = 0.f; s.E.hi.y = 1.f; s.E.lo.y = 0.f;
               s.ux.hi.y = 0.f; s.ux.lo.y = 0.f; s.uy.hi.y = 0.f; s.uy.lo.y = 0.f; }
    eq = eq2(s, d);
  }

  // ---- radial ghost columns (tiles at a wall only) ----------------------------
  const int cw_out = p.n_r - 1 - r0 + kLeft;
  if (r0 == 0 || cw_out <= kLeft + kTileR) {
    if (ok && r0 == 0 && warp == 0 && lane < kTileT32 && t0 + lane < p.n_theta)
      ghost_columns_f32(sm, 2 + lane, 0, kLeft, t0 + lane, p, d);
    if (ok && cw_out <= kLeft + kTileR && warp == 1 && lane < kTileT32 && t0 + lane < p.n_theta)
      ghost_columns_f32(sm, 2 + lane, 1, cw_out, t0 + lane, p, d);
    if (__syncthreads_or(!ok)) {   // ghost columns visible; a copy that timed out stops the tile
      if (tid == 0) {
        atomicOr(p.status, PCLB_FLAG_TIMEOUT);
        for (int g = 0; g < kGroups; ++g) mbar_wait_bounded(&bar[g], 0, kDefaultWaitNs);
      }
      return;
    }
  } else if (!ok) {
    // a copy did not land in time: report it, give the copies a bounded time
    // to finish, and leave (no barrier follows in this tile)
    atomicOr(p.status, PCLB_FLAG_TIMEOUT);
    for (int g = 0; g < kGroups; ++g) mbar_wait_bounded(&bar[g], 0, kDefaultWaitNs);
    return;
  }

  // ---- update ----------------------------------------------------------------
  const f2 invr = mk2(v0 ? p.inv_r_f[r] : 1.f, v1 ? p.inv_r_f[r + 1] : 1.f);
  const f2 decay = bc2((float)p.decay);
  const size_t plane_out = (size_t)p.rows * p.pitch;
  float* out_row = f_out + (size_t)(t + kGhostRows) * p.pitch + r;
  // tiles away from the radial walls and the seam take the plain store
  const bool plain_tile = r0 + kTileR <= p.n_r && t0 >= 2 && t0 + kTileT32 <= p.n_theta - 2;
  auto store = [&](int q, f2 o) {
    if (plain_tile) {
      __stcs(reinterpret_cast<float2*>(out_row + (size_t)q * plane_out), o);   // not read again before the next step
      return;
    }
    // seam and ragged tiles: the seam rows' ghost copies, formed here so
    // that plain tiles keep no registers for them
    const bool lo_ghost = row_ok && t >= p.n_theta - 2;
    const bool hi_ghost = row_ok && t < 2;
    float* out_lo = f_out + (size_t)max(t - (p.n_theta - 2), 0) * p.pitch + r;
    float* out_hi = f_out + (size_t)(p.n_theta + kGhostRows + t) * p.pitch + r;
    if (v1) {
      *reinterpret_cast<float2*>(out_row + (size_t)q * plane_out) = o;
      if (lo_ghost) *reinterpret_cast<float2*>(out_lo + (size_t)d.recv_lo[q] * plane_out) = o;
      if (hi_ghost) *reinterpret_cast<float2*>(out_hi + (size_t)d.recv_hi[q] * plane_out) = o;
    } else if (v0) {
      out_row[(size_t)q * plane_out] = o.x;
      if (lo_ghost) out_lo[(size_t)d.recv_lo[q] * plane_out] = o.x;
      if (hi_ghost) out_hi[(size_t)d.recv_hi[q] * plane_out] = o.x;
    }
  };

  {  // rest velocity: no convection
    const f2 f0 = ld2(win);
    const f2 e0 = mul2(eq.w[0], eq.a0);
    store(0, fma2(sub2(f0, e0), decay, e0));
  }

  // One velocity of a pair.  sr = +1 if its upwind neighbour in r is at
  // larger r, st the same for theta (rows); fe is its equilibrium.
  // nar, nkr, nat, nkt: the negated a = |C| and K = |C|(1 - |C|) in r and
  // theta.  Increments in upwind form (D, Dp the upwind differences):
  // MWB a D + K h(D, Dp); WB a D + K (D - Dp)/2; LW a D + K (Dd - D)/2 with
  // Dd the downwind difference; second-order upwind a D + a (D - Dp)/2.
  auto update = [&](int q, int sr, int st, f2 nar, f2 nkr, f2 nat, f2 nkt, f2 fe) {
    const float* w = win + q * kPlaneF;
    const f2 C = ld2(w);
    const f2 S = ld2(w + 2 * sr);                 // (j-2, j-1) or (j+2, j+3)
    const f2 T1 = ld2(w + st * kWinR);
    const f2 T2 = ld2(w + 2 * st * kWinR);
    const f2 u1 = sr < 0 ? mk2(S.y, C.x) : mk2(C.y, S.x);   // first upwind neighbours
    const f2 Dr = sub2(C, u1), Dt = sub2(C, T1);
    // the convection increments summed first (small), then added once to
    // the relaxed value (one rounding at the magnitude of f for them)
    f2 dc = mul2(nar, Dr);
    dc = fma2(nat, Dt, dc);
    if constexpr (SCH == PCLB_SCHEME_MWB) {
      dc = fma2(nkr, limiter2(Dr, sub2(u1, S)), dc);
      dc = fma2(nkt, limiter2(Dt, sub2(T1, T2)), dc);
    } else if constexpr (SCH == PCLB_SCHEME_WB) {
      dc = fma2(mul2(bc2(0.5f), nkr), sub2(Dr, sub2(u1, S)), dc);
      dc = fma2(mul2(bc2(0.5f), nkt), sub2(Dt, sub2(T1, T2)), dc);
    } else if constexpr (SCH == PCLB_SCHEME_UPWIND2) {
      dc = fma2(mul2(bc2(0.5f), nar), sub2(Dr, sub2(u1, S)), dc);
      dc = fma2(mul2(bc2(0.5f), nat), sub2(Dt, sub2(T1, T2)), dc);
    } else {
      const f2 X = ld2(w - 2 * sr);               // the pair on the downwind side
      const f2 d1 = sr < 0 ? mk2(C.y, X.x) : mk2(X.y, C.x);   // first downwind neighbours
      const f2 Td = ld2(w - st * kWinR);
      dc = fma2(mul2(bc2(0.5f), nkr), sub2(sub2(d1, C), Dr), dc);
      dc = fma2(mul2(bc2(0.5f), nkt), sub2(sub2(Td, C), Dt), dc);
    }
    store(q, add2(fma2(sub2(C, fe), decay, fe), dc));
  };

  // Shells run as a loop (keeps the hot body small for the instruction
  // cache); the four direction pairs of a shell are unrolled.
#pragma unroll 1
  for (int k = 1; k <= 4; ++k) {
    const f2 sh = bc2(d.speed[k]), sl = bc2(d.speed_lo[k]);
    const f2 wk = k == 1 ? eq.w[1] : (k == 2 ? eq.w[2] : (k == 3 ? eq.w[3] : eq.w[4]));
    const int qb = 1 + (k - 1) * kNDirs;
#pragma unroll
    for (int i = 0; i < kHalf; ++i) {
      const int q = qb + i;
      const float4 tb = tab[((k - 1) * kHalf + i) * kTileT32 + rl];
      const int fl = __float_as_int(tb.w);
      const int sr = (fl & 1) ? 1 : -1;            // v_r < 0: upwind at larger r
      const int st = (fl & 2) ? 1 : -1;            // v_theta < 0: upwind at larger theta
      const f2 nar = bc2(-tb.x), nkr = bc2(-tb.y);
      const f2 nat = mul2(bc2(-tb.z), invr);
      const f2 nkt = fma2(nat, nat, nat);            // -(a - a^2) with a = -nat
      f2 fp, fm;   // equilibrium of the pair
      feq_pair2(eq, sh, sl, i, wk, fp, fm);
      update(q, sr, st, nar, nkr, nat, nkt, fp);
      update(q + kHalf, -sr, -st, nar, nkr, nat, nkt, fm);
    }
  }
}

template <int SCH>
static cudaError_t launch_scheme_f32(const CUtensorMap* tmap_in, float* f_out, const StepParams& p,
                                     const DvmConst<float>& d, cudaStream_t stream, int ty_begin, int ty_end) {
  static std::atomic<unsigned long long> configured{0};   // per instantiation and device
  {
    const cudaError_t e = set_smem_once(step_kernel_f32<SCH>, kSmemF32, configured);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((p.n_r + kTileR - 1) / kTileR, ty_end - ty_begin);
  step_kernel_f32<SCH><<<grid, kStepThreads32, kSmemF32, stream>>>(*tmap_in, f_out, p, d, ty_begin);
  return cudaGetLastError();
}

// Tile rows [ty_begin, ty_end) of the grid (ty_end < 0: to the last tile row);
// an empty range launches nothing.
cudaError_t launch_step_f32(const CUtensorMap* tmap_in, float* f_out, const StepParams& p,
                            const DvmConst<float>& d, cudaStream_t stream, int ty_begin, int ty_end) {
  if (ty_end < 0) ty_end = (p.n_theta + kTileT32 - 1) / kTileT32;
  if (ty_begin < 0 || ty_end <= ty_begin) return cudaSuccess;
  switch (p.scheme) {
    case PCLB_SCHEME_WB: return launch_scheme_f32<PCLB_SCHEME_WB>(tmap_in, f_out, p, d, stream, ty_begin, ty_end);
    case PCLB_SCHEME_LW: return launch_scheme_f32<PCLB_SCHEME_LW>(tmap_in, f_out, p, d, stream, ty_begin, ty_end);
    case PCLB_SCHEME_UPWIND2:
      return launch_scheme_f32<PCLB_SCHEME_UPWIND2>(tmap_in, f_out, p, d, stream, ty_begin, ty_end);
    default: return launch_scheme_f32<PCLB_SCHEME_MWB>(tmap_in, f_out, p, d, stream, ty_begin, ty_end);
  }
}

}  // namespace pclb
