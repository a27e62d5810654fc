// FP32 adjoint step, lam^n = J(f^n)^T lam^{n+1} (the transpose of Eq. 38
// with the boundary nodes of Sec. II C), with two radially adjacent nodes per
// thread in packed FP32x2 arithmetic.  The mathematics and the two-phase
// structure are those of the scalar pair kernel (adjoint_kernel.cu, which
// keeps the FP64 path); only the data layout per thread differs:
//   * tile 32 (r) x 16 (theta), 256 threads; thread (row, 2j) owns the nodes
//     (2j, 2j + 1) of its row;
//   * the node cotangent g of both nodes (Eqs. 3-5, 10-11 differentiated)
//     from f^n and lam^{n+1} read from global memory, float-float moments
//     rounded once, then the equilibrium cotangent in packed float;
//   * the pairs of opposite velocities stream their f and lam windows over
//     [r0-4, r0+36) x [t0-2, t0+18) through a 2-stage TMA ring; per pair,
//     phase (A) forms lam(n) dM(n)/dD and lam(n) dM(n)/dDp of every node whose
//     upwind stencil reaches the tile (MWB, Eq. 28, in r and in theta), 8-byte
//     shared-memory stores of both nodes; one barrier; phase (B) gathers the
//     products of the nodes that read each tile node and stores lam^n.
// Shared memory ~70 KB and at most 80 registers: three CTAs per SM.
#include <cuda.h>
#include <cuda_runtime.h>

#include <atomic>

#include "adjoint_common.cuh"
#include "device_common.cuh"
#include "f32_state.cuh"
#include "f32x2.cuh"
#include "pclb_internal.h"

namespace pclb {

namespace {

constexpr int kTT = kAdjRows32;                 // tile rows
constexpr int kAThr = 16 * kTT;                 // two nodes per thread
constexpr int kAPl = kWinR * (kTT + 4);         // floats per plane window
constexpr int kANP = 4 * kNDirs / 2;            // pairs of opposite velocities
constexpr int kAS = 2;                          // ring stages
constexpr int kRC = kTileR + 4;                 // radial product columns -2 .. 33
// products of one label: radial A, B [kTT][kRC], azimuthal A, B [kTT + 4][kTileR]
constexpr int kAR = 0, kBR = kTT * kRC;
constexpr int kAT = 2 * kTT * kRC, kBT = kAT + (kTT + 4) * kTileR;
constexpr int kProd = kBT + (kTT + 4) * kTileR;
constexpr int kRingBytes = kAS * 4 * kAPl * 4;  // [stage][f q1, f q2, lam q1, lam q2][plane]
constexpr int kProdBytes = 2 * 2 * kProd * 4;   // [buffer][label][products]
constexpr int kInvrBytes = kTileR * 4;
constexpr int kTabBytes = (kTT + 4) * kANP * 16;
constexpr int kASmem = kRingBytes + kProdBytes + kInvrBytes + kTabBytes + 8 * kAS;
static_assert(kTT == 16 && kAThr == 256, "thread layout: 8 warps of two 16-thread rows");
static_assert((kAPl * 4) % 128 == 0, "TMA destinations must stay 128-byte aligned");
static_assert(kProdBytes % 16 == 0 && (kRingBytes + kProdBytes + kInvrBytes) % 16 == 0, "float4 table alignment");
static_assert(kRC % 2 == 0 && kAT % 2 == 0 && kBT % 2 == 0 && kProd % 2 == 0, "8-byte product slots");

__device__ __forceinline__ f2 lds2(const float* p) { return *reinterpret_cast<const float2*>(p); }
__device__ __forceinline__ void sts2(float* p, f2 v) { *reinterpret_cast<float2*>(p) = v; }
__device__ __forceinline__ f2 ldg2(const float* p) { return __ldg(reinterpret_cast<const float2*>(p)); }

// mwb_partials of two nodes: MD = a + K (ar + br (ar - s br)), MDp = -(1 + s)
// K ar^2 with ar, br = |D|, |Dp| / (|D| + |Dp|) (0 when the sum is below the
// smallest normal) and s the sign of D Dp (0 when either is 0).
__device__ __forceinline__ void mwb_partials2(f2 a, f2 K, f2 D, f2 Dp, f2& MD, f2& MDp) {
  const f2 aD = abs2(D), aP = abs2(Dp), n = add2(aD, aP);
  const f2 rn = mk2(n.x >= smallest_normal<float>() ? recip_fast(n.x) : 0.f,
                    n.y >= smallest_normal<float>() ? recip_fast(n.y) : 0.f);
  const f2 ar = mul2(aD, rn), br = mul2(aP, rn);
  const f2 pr = mul2(D, Dp);
  const f2 s = mk2(fminf(aD.x, aP.x) > 0.f ? copysignf(1.f, pr.x) : 0.f,
                   fminf(aD.y, aP.y) > 0.f ? copysignf(1.f, pr.y) : 0.f);
  const f2 Ka = mul2(K, ar);
  MD = fma2(K, fma2(br, fma2(neg2(s), br, ar), ar), a);
  MDp = mul2(neg2(add2(bc2(1.f), s)), mul2(Ka, ar));
}

// Float-float moments (Eqs. 3-5) and temperature of two nodes, as state32:
// float shell sums over opposite-direction pairs, shells 2 and 3 added
// direction by direction first, shell totals combined with error-free
// transformations.  ld(q) returns both nodes' f_q.
template <class LD>
__device__ __forceinline__ void state_pair(LD ld, const DvmConst<float>& d, f2& rho_o, f2& ux_o, f2& uy_o, f2& E_o,
                                           bool& ok0, bool& ok1) {
  ff2 rho = ff2_of(ld(0)), jx = ff2_of(bc2(0.f)), jy = jx, e = jx;
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    const int k = g == 0 ? 1 : (g == 1 ? 2 : (g == 2 ? 3 : 4));
    f2 S = bc2(0.f), X = S, Xl = S, Y = S, Yl = S;
#pragma unroll
    for (int i = 0; i < kHalf; ++i) {
      const int q = 1 + (k - 1) * kNDirs + i;
      f2 fa = ld(q), fb = ld(q + kHalf);
      if (g == 1) {
        const int qa = 1 + 2 * kNDirs + i;   // shell 3 added to shell 2
        fa = add2(fa, ld(qa));
        fb = add2(fb, ld(qa + kHalf));
      }
      S = add2(S, add2(fa, fb));
      const f2 dd = sub2(fa, fb);   // the pair has opposite unit vectors
      X = fma2(bc2(d.cx[q]), dd, X);
      Xl = fma2(bc2(d.cx_lo[q]), dd, Xl);
      Y = fma2(bc2(d.cy[q]), dd, Y);
      Yl = fma2(bc2(d.cy_lo[q]), dd, Yl);
    }
    const ff2 sp = g == 2 ? ff2{bc2(d.dv23), bc2(d.dv23_lo)} : ff2{bc2(d.speed[k]), bc2(d.speed_lo[k])};
    const ff2 hv = g == 2 ? ff2{bc2(d.dh23), bc2(d.dh23_lo)} : ff2{bc2(d.half_v2[k]), bc2(d.half_v2_lo[k])};
    if (g != 2) rho = ff2_add(rho, ff2_of(S));
    jx = ff2_add(jx, ff2_mul(sp, ff2{X, Xl}));
    jy = ff2_add(jy, ff2_mul(sp, ff2{Y, Yl}));
    e = ff2_add(e, ff2_mul(hv, ff2_of(S)));
  }
  const ff2 inv = ff2_recip(rho);
  const ff2 ux = ff2_mul(jx, inv), uy = ff2_mul(jy, inv);
  const ff2 ke = ff2_add(ff2_mul(jx, ux), ff2_mul(jy, uy));   // |j|^2 / rho
  const ff2 E = ff2_mul(ff2_add(e, ff2_scale(ke, -0.5f)), inv);
  ok0 = rho.hi.x > 0.f && E.hi.x > 0.f && isfinite(e.hi.x) && isfinite(jx.hi.x) && isfinite(jy.hi.x);
  ok1 = rho.hi.y > 0.f && E.hi.y > 0.f && isfinite(e.hi.y) && isfinite(jx.hi.y) && isfinite(jy.hi.y);
  rho_o = ff2_round(rho);
  ux_o = ff2_round(ux);
  uy_o = ff2_round(uy);
  E_o = ff2_round(E);
}

__device__ __forceinline__ f2 recip1_2(f2 x) {
  const f2 r = mk2(recip_fast(x.x), recip_fast(x.y));
  return fma2(r, fma2(neg2(x), r, bc2(1.f)), r);
}

// eq_cotangent of two nodes: G = sum_q lam_q d f^eq_q / d(rho, u_x, u_y, E)
// (Eq. 10 with the weights of Eq. 11), opposite velocities of a shell
// sharing the even and odd parts of P, P_x and P_s.
template <class LamFn>
__device__ __forceinline__ void eq_cotangent2(f2 rho, f2 ux, f2 uy, f2 E, const DvmConst<float>& d, LamFn lam,
                                              f2 G[4]) {
  f2 F[5], Fd[5];
  f2 Fs = bc2(0.f), Fds = bc2(0.f);
#pragma unroll
  for (int k = 1; k <= 4; ++k) {
    const float* c = d.Fc[k];
    F[k] = mul2(E, fma2(E, fma2(E, fma2(E, bc2(c[3]), bc2(c[2])), bc2(c[1])), bc2(c[0])));
    Fd[k] = fma2(E, fma2(E, fma2(mul2(E, bc2(4.f)), bc2(c[3]), bc2(3.f * c[2])), bc2(2.f * c[1])), bc2(c[0]));
    Fs = add2(Fs, F[k]);
    Fds = add2(Fds, Fd[k]);
  }
  F[0] = fma2(bc2(-d.B0), Fs, bc2(1.f));
  Fd[0] = mul2(bc2(-d.B0), Fds);
  const f2 invE = recip1_2(E);
  const f2 s = mul2(fma2(ux, ux, mul2(uy, uy)), invE);
  const f2 a1 = fma2(bc2(-0.5f), s, bc2(1.f));
  const f2 a0 = fma2(mul2(bc2(0.125f), s), s, a1);
  const f2 uxE = mul2(ux, invE), uyE = mul2(uy, invE);
  const f2 l0 = lam(0);
  const f2 l0F0 = mul2(l0, F[0]);
  f2 A = mul2(l0F0, a0), Bx = bc2(0.f), By = bc2(0.f);
  f2 Cs = mul2(l0F0, fma2(bc2(0.25f), s, bc2(-0.5f))), Dx = bc2(0.f);
  f2 Fq = mul2(mul2(l0, Fd[0]), a0);
  const f2 a1h = mul2(bc2(0.5f), a1);
#pragma unroll
  for (int k = 1; k <= 4; ++k) {
    f2 Ak = bc2(0.f), Bxk = Ak, Byk = Ak, Ck = Ak, Dk = Ak;
#pragma unroll
    for (int i = 0; i < kHalf; ++i) {
      const int q = 1 + (k - 1) * kNDirs + i;
      const f2 vx = bc2(d.vx[q]), vy = bc2(d.vy[q]);
      const f2 x = fma2(vx, uxE, mul2(vy, uyE));
      const f2 x2 = mul2(x, x);
      const f2 Pe = fma2(x2, fma2(x2, bc2(1.0f / 24.0f), a1h), a0);   // P(+-x) = Pe +- Po
      const f2 Xo = mul2(x, fma2(x2, bc2(1.0f / 6.0f), a1));          // odd part of P and of P_x
      const f2 Xe = fma2(x2, bc2(0.5f), a1);                           // even part of P_x
      const f2 Se = fma2(bc2(-0.25f), x2, fma2(bc2(0.25f), s, bc2(-0.5f)));   // P_s(+-x) = Se -+ x/2
      const f2 lp = lam(q), lm = lam(q + kHalf);
      const f2 ls = add2(lp, lm), ld = sub2(lp, lm);
      Ak = fma2(ls, Pe, fma2(ld, Xo, Ak));
      const f2 lpx = fma2(ld, Xe, mul2(ls, Xo));                     // lp P_x(x) - lm P_x(-x)
      Bxk = fma2(lpx, vx, Bxk);
      Byk = fma2(lpx, vy, Byk);
      Ck = fma2(ls, Se, fma2(mul2(ld, bc2(-0.5f)), x, Ck));
      Dk = fma2(x, fma2(ls, Xo, mul2(ld, Xe)), Dk);                  // lp x P_x(x) + lm (-x) P_x(-x)
    }
    A = fma2(F[k], Ak, A);
    Bx = fma2(F[k], Bxk, Bx);
    By = fma2(F[k], Byk, By);
    Cs = fma2(F[k], Ck, Cs);
    Dx = fma2(F[k], Dk, Dx);
    Fq = fma2(Fd[k], Ak, Fq);
  }
  G[0] = A;
  const f2 rE = mul2(rho, invE);
  G[1] = mul2(rE, fma2(mul2(bc2(2.f), ux), Cs, Bx));
  G[2] = mul2(rE, fma2(mul2(bc2(2.f), uy), Cs, By));
  G[3] = mul2(rho, sub2(Fq, mul2(fma2(s, Cs, Dx), invE)));
}

// Cotangent in (rho, u, E) to the cotangent in m = (rho, j_x, j_y, e).
__device__ __forceinline__ void to_moment_cotangent2(f2 rho, f2 ux, f2 uy, f2 E, const f2 G[4], f2 g[4]) {
  const f2 inv = recip1_2(rho);
  const f2 uG = fma2(ux, G[1], mul2(uy, G[2]));
  const f2 k = sub2(mul2(bc2(0.5f), fma2(ux, ux, mul2(uy, uy))), E);
  g[0] = add2(sub2(G[0], mul2(uG, inv)), mul2(mul2(k, G[3]), inv));
  g[1] = mul2(fma2(neg2(ux), G[3], G[1]), inv);
  g[2] = mul2(fma2(neg2(uy), G[3], G[2]), inv);
  g[3] = mul2(G[3], inv);
}

__global__ void __launch_bounds__(kAThr, 3)
    adjoint_pair_f32x2(const __grid_constant__ CUtensorMap tmap_f, const __grid_constant__ CUtensorMap tmap_l,
                       const float* __restrict__ f, const float* __restrict__ lam_in, float* __restrict__ lam_out,
                       const EqParams<float>* __restrict__ ghost, const float* __restrict__ gwall, int a0, int na,
                       int b0, const __grid_constant__ StepParams p, const __grid_constant__ DvmConst<float> d) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* ring = reinterpret_cast<float*>(smem_raw);
  float* prod = reinterpret_cast<float*>(smem_raw + kRingBytes);
  float* invr = reinterpret_cast<float*>(smem_raw + kRingBytes + kProdBytes);
  float4* ctab = reinterpret_cast<float4*>(smem_raw + kRingBytes + kProdBytes + kInvrBytes);   // [kTT + 4][kANP]
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + kRingBytes + kProdBytes + kInvrBytes + kTabBytes);

  // radial tile: blocks 0 .. na - 1 take tiles a0 .., the rest tiles b0 ..
  const int tx = (int)blockIdx.x < na ? a0 + (int)blockIdx.x : b0 + (int)blockIdx.x - na;
  const int r0 = tx * kTileR;
  const int t0 = blockIdx.y * kTT;
  const int tid = threadIdx.x;

  auto issue_pair = [&](int pr, int s) {
    const int k = 1 + pr / kHalf;
    const int q1 = 1 + (k - 1) * kNDirs + pr % kHalf, q2 = q1 + kHalf;
    float* st = ring + s * 4 * kAPl;
    mbar_arrive_expect_tx(&bar[s], (uint32_t)(4 * kAPl * 4));
    tma_load_3d(st, &tmap_f, r0 - kLeft, t0, q1, &bar[s]);
    tma_load_3d(st + kAPl, &tmap_f, r0 - kLeft, t0, q2, &bar[s]);
    tma_load_3d(st + 2 * kAPl, &tmap_l, r0 - kLeft, t0, q1, &bar[s]);
    tma_load_3d(st + 3 * kAPl, &tmap_l, r0 - kLeft, t0, q2, &bar[s]);
  };
  if (tid == 0) {
    tma_prefetch_desc(&tmap_f);
    tma_prefetch_desc(&tmap_l);
    for (int s = 0; s < kAS; ++s) mbar_init(&bar[s], 1);
    mbar_fence_init();
  }
  if (tid < kTileR) invr[tid] = r0 + tid < p.n_r ? p.inv_r_f[r0 + tid] : 1.f;
  // Courant entries of the stored rows t0 .. t0 + kTT + 3 (theta rows t0 - 2 .. t0 + kTT + 1)
  for (int i = tid; i < (kTT + 4) * kANP; i += kAThr) {
    const int srow = t0 + i / kANP, pr = i % kANP;
    ctab[i] = srow < p.rows ? p.courant[(size_t)srow * kANP + pr] : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __syncthreads();
  // bits 2..6 of the tile rows' flags: bit 1 (v_theta < 0 for q1) of the rows
  // -2 .. +2 around them, the rows whose azimuthal stencils reach the node
  for (int i = tid; i < kTT * kANP; i += kAThr) {
    const int w = 2 + i / kANP, pr = i % kANP;
    int m = 0;
#pragma unroll
    for (int o = 0; o < 5; ++o) m |= ((__float_as_int(ctab[(w - 2 + o) * kANP + pr].w) >> 1) & 1) << o;
    ctab[w * kANP + pr].w = __int_as_float(__float_as_int(ctab[w * kANP + pr].w) | (m << 2));
  }
  __syncthreads();
  if (tid == 0)
    for (int s = 0; s < kAS && s < kANP; ++s) issue_pair(s, s);

  // ---- this thread's two nodes ---------------------------------------------
  const int warp = tid >> 5, lane = tid & 31;
  const int rl = 2 * warp + (lane >> 4);       // tile row
  const int j2 = 2 * (lane & 15);              // even radial offset
  const int t = t0 + rl, r = r0 + j2;
  const bool row_ok = t < p.n_theta;
  const bool v0 = row_ok && r < p.n_r, v1 = row_ok && r + 1 < p.n_r;
  const int srow = min(t, p.n_theta - 1) + kGhostRows;   // rows past the grid read the last row
  const size_t plane_out = (size_t)p.rows * p.pitch;
  const f2 decay = bc2((float)p.decay);
  f2 gs[4] = {bc2(0.f), bc2(0.f), bc2(0.f), bc2(0.f)};
  const size_t off = (size_t)srow * p.pitch + r;
  {
    // (1 - d) g of both nodes from global memory, while the first pairs'
    // windows land (their copies then mostly hit L2); columns past n_r read
    // the row's padding (r + 1 < pitch), their results are never stored
    f2 rho, ux, uy, E;
    bool ok0, ok1;
    state_pair([&](int q) { return ldg2(f + off + (size_t)q * plane_out); }, d, rho, ux, uy, E, ok0, ok1);
    if ((v0 && !ok0) || (v1 && !ok1)) atomicOr(p.status, PCLB_FLAG_NONPHYS);
    f2 G[4], g[4];
    eq_cotangent2(rho, ux, uy, E, d, [&](int q) { return ldg2(lam_in + off + (size_t)q * plane_out); }, G);
    to_moment_cotangent2(rho, ux, uy, E, G, g);
    const f2 omd = sub2(bc2(1.f), decay);
#pragma unroll
    for (int j = 0; j < 4; ++j) gs[j] = mul2(omd, g[j]);
    // the cotangent the ghost nodes return to the two nodes next to each wall
    if (row_ok && (r < 2 || r + 3 >= p.n_r)) {
      auto wall = [&](int rr) {
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
        auto add = [&](int side, int node) {
          const float4 w = *reinterpret_cast<const float4*>(gwall + ((size_t)(side * 2 + node) * p.n_theta + t) * 4);
          a.x += w.x; a.y += w.y; a.z += w.z; a.w += w.w;
        };
        if (rr == 0) add(0, 0);
        if (rr == 1) add(0, 1);
        if (rr == p.n_r - 1) add(1, 0);
        if (rr == p.n_r - 2) add(1, 1);
        return a;
      };
      const float4 w0 = wall(r), w1 = wall(r + 1);
      gs[0] = add2(gs[0], mk2(w0.x, w1.x));
      gs[1] = add2(gs[1], mk2(w0.y, w1.y));
      gs[2] = add2(gs[2], mk2(w0.z, w1.z));
      gs[3] = add2(gs[3], mk2(w0.w, w1.w));
    }
  }
  const int row = rl + 2;                      // window row of this thread's nodes
  const int o_node = row * kWinR + kLeft + j2;  // first node in a window plane
  const int p_rad = rl * kRC + j2 + 2;          // its radial product slot
  const int p_az = kAT + row * kTileR + j2;     // its azimuthal product slot
  const f2 my_invr = lds2(invr + j2);
  float* out_row = lam_out + (size_t)srow * p.pitch + r;
  const bool lo_ghost = row_ok && t >= p.n_theta - 2;
  const bool hi_ghost = row_ok && t < 2;
  float* out_lo = lam_out + (size_t)max(t - (p.n_theta - 2), 0) * p.pitch + r;
  float* out_hi = lam_out + (size_t)(p.n_theta + kGhostRows + t) * p.pitch + r;
  const bool plain_tile = r0 + kTileR <= p.n_r && t0 >= 2 && t0 + kTT <= p.n_theta - 2;
  auto store = [&](int q, f2 o) {
    if (plain_tile) {
      __stcs(reinterpret_cast<float2*>(out_row + (size_t)q * plane_out), o);
    } else if (v1) {
      *reinterpret_cast<float2*>(out_row + (size_t)q * plane_out) = o;
      if (lo_ghost) *reinterpret_cast<float2*>(out_lo + (size_t)d.recv_lo[q] * plane_out) = o;
      if (hi_ghost) *reinterpret_cast<float2*>(out_hi + (size_t)d.recv_hi[q] * plane_out) = o;
    } else if (v0) {
      out_row[(size_t)q * plane_out] = o.x;
      if (lo_ghost) out_lo[(size_t)d.recv_lo[q] * plane_out] = o.x;
      if (hi_ghost) out_hi[(size_t)d.recv_hi[q] * plane_out] = o.x;
    }
  };
  // rest velocity: no convection
  store(0, add2(fma2(decay, ldg2(lam_in + off), gs[0]), mul2(gs[3], bc2(d.half_v2[0]))));

  // wall tiles: the ghost states of the rows this thread fills (threads 0..15
  // the inner wall, 32..47 the outer wall, one tile row each)
  const int cw_out = p.n_r - 1 - r0 + kLeft;
  const bool inner = r0 == 0, outer = cw_out <= kLeft + kTileR;
  const bool wall_tile = inner || outer;
  const int gside = tid >> 5, grow = tid & 31;
  const bool fills = wall_tile && tid < 64 && grow < kTT && t0 + grow < p.n_theta && (gside == 0 ? inner : outer);
  const EqParams<float>* eg = ghost + (size_t)(gside * 2) * p.n_theta + t0 + grow;   // layer l at + l n_theta

  bool ok = true;
  int brk = kANP;                                // the pair at which a wait timed out
#pragma unroll 1
  for (int pair = 0; pair < kANP; ++pair) {
    const int k = 1 + pair / kHalf;
    const int q1 = 1 + (k - 1) * kNDirs + pair % kHalf;
    const int q2 = q1 + kHalf;                     // opposite velocity
    const int s = pair % kAS;
    float* st = ring + s * 4 * kAPl;
    float* pb = prod + (pair & 1) * 2 * kProd;     // this pair's products: [label][...]
    if (ok) ok = p.wait_ns != 0 && mbar_wait_bounded(&bar[s], (uint32_t)((pair / kAS) & 1), p.wait_ns);
    if (wall_tile) {
      // radial ghost columns of this pair's f planes (f = f^eq of the ghost states)
      if (fills && ok) {
        float* fw = st + (2 + grow) * kWinR;
        const int c0 = gside == 0 ? kLeft : cw_out, stp = gside == 0 ? 1 : -1;
        for (int l = 0; l < 2; ++l) {
          const int c = c0 - stp * (1 + l);
          if (c < 0 || c >= kWinR) continue;
          const EqParams<float> e = eg[(size_t)l * p.n_theta];
          fw[c] = feq_q<float>(e, d.vx[q1], d.vy[q1], k);
          fw[kAPl + c] = feq_q<float>(e, d.vx[q2], d.vy[q2], k);
        }
      }
      __syncthreads();
    }

    // (A) products lam(n) M_D(n), lam(n) M_Dp(n)
    const float* sf = st;                          // f q1, f q2 at + kAPl
    const float* sl = st + 2 * kAPl;               // lam q1, lam q2 at + kAPl
    const float4 ce = ctab[row * kANP + pair];
    const int fl_c = __float_as_int(ce.w);
    const int ur = (fl_c & 1) ? 1 : -1;            // q1 reads n + 1, n + 2 in r
    const int vt = (fl_c & 2) ? kWinR : -kWinR;    // q1 reads the rows above (+) or below (-)
    const f2 a_r = bc2(ce.x), k_r = bc2(ce.y);
    const f2 a_t = mul2(bc2(ce.z), my_invr), k_t = fma2(neg2(a_t), a_t, a_t);
    f2 lam_c[2];
#pragma unroll
    for (int L = 0; L < 2; ++L) {
      const int u = L ? -ur : ur, v = L ? -vt : vt;
      const float* w = sf + L * kAPl + o_node;
      const f2 C = lds2(w);
      const f2 S2 = lds2(w + 2 * u);               // f(n + 2u) of both nodes
      const f2 u1 = u > 0 ? mk2(C.y, S2.x) : mk2(S2.y, C.x);   // f(n + u)
      f2 MD, MP;
      mwb_partials2(a_r, k_r, sub2(C, u1), sub2(u1, S2), MD, MP);
      const f2 lam = lds2(sl + L * kAPl + o_node);
      lam_c[L] = lam;
      float* P = pb + L * kProd;
      sts2(P + kAR + p_rad, mul2(lam, MD));
      sts2(P + kBR + p_rad, mul2(lam, MP));
      const f2 T1 = lds2(w + v), T2 = lds2(w + 2 * v);
      mwb_partials2(a_t, k_t, sub2(C, T1), sub2(T1, T2), MD, MP);
      sts2(P + p_az, mul2(lam, MD));
      sts2(P + p_az + (kBT - kAT), mul2(lam, MP));
    }
    if (tid < 64) {
      // halo rows (window rows 0, 1, kTT + 2, kTT + 3), the label whose
      // upwind side points into the tile: rows below it are read by the
      // label with its upwind side at +theta
      const int hrow = tid >> 4, jj = 2 * (tid & 15);
      const int rr = hrow < 2 ? hrow : kTT + hrow;
      const float4 eh = ctab[rr * kANP + pair];
      const bool q1_up_pos = (__float_as_int(eh.w) & 2) != 0;
      const int L = (hrow < 2) == q1_up_pos ? 0 : 1;
      const int v = hrow < 2 ? kWinR : -kWinR;
      const f2 ath = mul2(bc2(eh.z), lds2(invr + jj)), kth = fma2(neg2(ath), ath, ath);
      const int o = rr * kWinR + kLeft + jj;
      const float* w = sf + L * kAPl + o;
      const f2 C = lds2(w), T1 = lds2(w + v), T2 = lds2(w + 2 * v);
      f2 MD, MP;
      mwb_partials2(ath, kth, sub2(C, T1), sub2(T1, T2), MD, MP);
      const f2 lam = lds2(sl + L * kAPl + o);
      float* P = pb + L * kProd + kAT + rr * kTileR + jj;
      sts2(P, mul2(lam, MD));
      sts2(P + (kBT - kAT), mul2(lam, MP));
    } else if (tid < 96) {
      // halo columns: per tile row and label the two columns whose upwind
      // stencils reach the tile, -2, -1 (upwind at larger r) or 32, 33
      const int h = tid - 64, hr = h >> 1, L = h & 1;
      const float4 eh = ctab[(hr + 2) * kANP + pair];
      const int uh = (__float_as_int(eh.w) & 1) ? 1 : -1, u = L ? -uh : uh;
      const int c = u > 0 ? -2 : kTileR;
      const int o = (hr + 2) * kWinR + kLeft + c;
      const float* w = sf + L * kAPl + o;
      const f2 C = lds2(w), S2 = lds2(w + 2 * u);
      const f2 u1 = u > 0 ? mk2(C.y, S2.x) : mk2(S2.y, C.x);
      f2 MD, MP;
      mwb_partials2(bc2(eh.x), bc2(eh.y), sub2(C, u1), sub2(u1, S2), MD, MP);
      const f2 lam = lds2(sl + L * kAPl + o);
      float* P = pb + L * kProd + hr * kRC + c + 2;
      sts2(P + kAR, mul2(lam, MD));
      sts2(P + kBR, mul2(lam, MP));
    }
    if (__syncthreads_or(!ok)) {
      brk = pair;
      break;
    }
    // the stage of this pair is free: the planes of pair + kAS start now
    if (tid == 0 && pair + kAS < kANP) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue_pair(pair + kAS, s);
    }

    // (B) gather at both nodes: node n = c + j u_n reads f(n), f(n + u_n),
    // f(n + 2 u_n), so dM(n)/df(c) collects M_D of n = c, M_Dp - M_D of
    // n = c - u and -M_Dp of n = c - 2u
    if (v0 || v1) {
      f2 acc[2];
#pragma unroll
      for (int L = 0; L < 2; ++L) {
        const float* P = pb + L * kProd;
        const int u = L ? -ur : ur;
        const f2 A0 = lds2(P + kAR + p_rad), B0 = lds2(P + kBR + p_rad);
        const f2 An = lds2(P + kAR + p_rad - 2 * u), Bn = lds2(P + kBR + p_rad - 2 * u);
        // A(c - u), B(c - u), B(c - 2u) of both nodes
        const f2 Au = u > 0 ? mk2(An.y, A0.x) : mk2(A0.y, An.x);
        const f2 Bu = u > 0 ? mk2(Bn.y, B0.x) : mk2(B0.y, Bn.x);
        acc[L] = sub2(add2(sub2(A0, Au), Bu), Bn);
      }
      const int tneg = fl_c >> 2;                  // bit o: row o - 2 has v_theta < 0 for q1
      constexpr int DB = kBT - kAT;
      if (tneg == 0 || tneg == 31) {
        const int V = tneg == 0 ? kTileR : -kTileR;   // q1's readers at +V, +2V; q2's at -V, -2V
#pragma unroll
        for (int L = 0; L < 2; ++L) {
          const int W = L ? -V : V;
          const float* P = pb + L * kProd + p_az;
          acc[L] = add2(acc[L], sub2(sub2(add2(lds2(P), lds2(P + DB + W)), lds2(P + W)), lds2(P + DB + 2 * W)));
        }
      } else {
#pragma unroll
        for (int L = 0; L < 2; ++L) {
          const float* P = pb + L * kProd + p_az;
          const int neg = L ? (tneg ^ 0x1f) : tneg;   // the partner has the opposite velocity
          f2 a = lds2(P);
          if (neg & 2) a = add2(a, sub2(lds2(P + DB - kTileR), lds2(P - kTileR)));
          if (!(neg & 8)) a = add2(a, sub2(lds2(P + DB + kTileR), lds2(P + kTileR)));
          if (neg & 1) a = sub2(a, lds2(P + DB - 2 * kTileR));
          if (!(neg & 16)) a = sub2(a, lds2(P + DB + 2 * kTileR));
          acc[L] = add2(acc[L], a);
        }
      }
      const f2 A = fma2(gs[3], bc2(d.half_v2[k]), gs[0]);
      const f2 B = fma2(gs[1], bc2(d.vx[q1]), mul2(gs[2], bc2(d.vy[q1])));
      store(q1, sub2(fma2(decay, lam_c[0], add2(A, B)), acc[0]));
      store(q2, sub2(fma2(decay, lam_c[1], sub2(A, B)), acc[1]));
    }
  }
  if (brk < kANP && tid == 0) {
    // a copy did not land in time: report it, give the copies still in
    // flight (the last one issued into each stage) a bounded time to finish
    atomicOr(p.status, PCLB_FLAG_TIMEOUT);
    const int issued = brk + kAS < kANP ? brk + kAS : kANP;
    for (int s = 0; s < kAS && s < issued; ++s) {
      const int last = s + ((issued - 1 - s) / kAS) * kAS;
      mbar_wait_bounded(&bar[s], (uint32_t)((last / kAS) & 1), kDefaultWaitNs);
    }
  }
}

}  // namespace

cudaError_t launch_adjoint_pairs_f32(const CUtensorMap* tmap_f, const CUtensorMap* tmap_l, const float* f,
                                     const float* lam_in, float* lam_out, const EqParams<float>* ghost,
                                     const float* gwall, int a0, int na, int b0, int nx, const StepParams& p,
                                     const DvmConst<float>& d, cudaStream_t s) {
  static std::atomic<unsigned long long> configured{0};
  {
    const cudaError_t e = set_smem_once(adjoint_pair_f32x2, kASmem, configured);
    if (e != cudaSuccess) return e;
  }
  const dim3 grid((unsigned)nx, (unsigned)((p.n_theta + kTT - 1) / kTT));
  adjoint_pair_f32x2<<<grid, kAThr, kASmem, s>>>(*tmap_f, *tmap_l, f, lam_in, lam_out, ghost, gwall, a0, na, b0, p,
                                                 d);
  return cudaGetLastError();
}

}  // namespace pclb
