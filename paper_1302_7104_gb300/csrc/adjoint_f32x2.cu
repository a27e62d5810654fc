// FP32 adjoint step, lam^n = J(f^n)^T lam^{n+1} (the transpose of Eq. 38
// with the boundary nodes of Sec. II C), with two radially adjacent nodes per
// thread in packed FP32x2 arithmetic.  The mathematics and the two-phase
// structure are those of the scalar pair kernel (adjoint_kernel.cu, which
// keeps the FP64 path); only the data layout per thread differs:
//   * tile 32 (r) x 16 (theta), 256 threads; thread (row, 2j) owns the nodes
//     (2j, 2j + 1) of its row;
//   * the node cotangent g of both nodes (Eqs. 3-5, 10-11 differentiated):
//     the tile's nodes of all 33 f planes, then of all 33 lam planes, stream
//     through 30 tile-sized slots (two halves of fifteen, one TMA barrier
//     each) laid over the pair ring and the product buffers, which are free
//     until the pairs start; the moments in float-float, rounded once, then
//     the equilibrium cotangent in packed float;
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
constexpr int kASmem = kRingBytes + kProdBytes + kInvrBytes + kTabBytes + 8 * (kAS + 2);
// node phase: 66 plane windows (f then lam) in groups of six through 12 slots
// node phase: 66 tile boxes (32 x 16 nodes of one plane, f then lam) in
// groups of fifteen through 30 slots laid over the pair ring and the product
// buffers, which are free until the pairs start.  Even groups use slots
// 15..29 (product buffers), odd groups slots 0..14 (the pair ring's stages
// and the start of the product buffers): the last group (six planes) is
// even, so the pair ring is free for the first two pairs once group 3 has
// been read.
constexpr int kNPl = kTileR * kTT;               // floats per node-phase box
constexpr int kPGroup = 15, kPBoxes = 2 * kQ, kPGroups = (kPBoxes + kPGroup - 1) / kPGroup;
static_assert(2 * kPGroup * kNPl * 4 <= kRingBytes + kProdBytes, "node-phase slots inside ring and products");
static_assert(kPGroups == 5 && kPGroup * kNPl * 4 >= kRingBytes, "the last group is even; odd groups cover the ring");
static_assert((kNPl * 4) % 128 == 0, "TMA destinations must stay 128-byte aligned");
__host__ __device__ constexpr int node_group_size(int g) {
  return (g + 1) * kPGroup <= kPBoxes ? kPGroup : kPBoxes - g * kPGroup;
}
__host__ __device__ constexpr int node_slot(int b) { return (b / kPGroup) % 2 == 0 ? kPGroup + b % kPGroup : b % kPGroup; }
static_assert(kTT == 16 && kAThr == 256, "thread layout: 8 warps of two 16-thread rows");
static_assert((kAPl * 4) % 128 == 0, "TMA destinations must stay 128-byte aligned");
static_assert(kProdBytes % 16 == 0 && (kRingBytes + kProdBytes + kInvrBytes) % 16 == 0, "float4 table alignment");
static_assert(kRC % 2 == 0 && kAT % 2 == 0 && kBT % 2 == 0 && kProd % 2 == 0, "8-byte product slots");

__device__ __forceinline__ f2 lds2(const float* p) { return *reinterpret_cast<const float2*>(p); }
__device__ __forceinline__ void sts2(float* p, f2 v) { *reinterpret_cast<float2*>(p) = v; }

// mwb_partials of two nodes: MD = a + K (ar + br (ar - s br)), MDp = -(1 + s)
// K ar^2 with ar, br = |D|, |Dp| / max(|D| + |Dp|, smallest normal) (both 0
// when D = Dp = 0) and s the sign of D Dp (0 when either is 0).  The scalar
// form takes ar = br = 0 for a subnormal sum and tests min(|D|, |Dp|) > 0
// for s; the maximum and the clamped product below save compares and
// selects per node and differ only where |D| or |Dp| is subnormal.
__device__ __forceinline__ void mwb_partials2(f2 a, f2 K, f2 D, f2 Dp, f2& MD, f2& MDp) {
  const f2 aD = abs2(D), aP = abs2(Dp), n = add2(aD, aP);
  const f2 rn = mk2(recip_fast(fmaxf(n.x, smallest_normal<float>())), recip_fast(fmaxf(n.y, smallest_normal<float>())));
  const f2 ar = mul2(aD, rn), br = mul2(aP, rn);
  const f2 pr = mul2(D, Dp);
  // s = sign(D Dp), 0 when either is 0: min(|D|, |Dp|) scaled by 2^126 and
  // clamped to 1 carries the zero test (the sign of a product is exact even
  // where it underflows)
  const f2 zb = mul2(mk2(fminf(aD.x, aP.x), fminf(aD.y, aP.y)), bc2(8.507059173023462e37f));
  const f2 s = mk2(copysignf(fminf(zb.x, 1.f), pr.x), copysignf(fminf(zb.y, 1.f), pr.y));
  const f2 Ka = mul2(K, ar);
  MD = fma2(K, fma2(br, fma2(neg2(s), br, ar), ar), a);
  MDp = mul2(neg2(add2(bc2(1.f), s)), mul2(Ka, ar));
}

// Streaming order of the node phase: box b < 33 is f plane pro_f_plane(b),
// box 33 + c lam plane pro_l_plane(c).  f: the rest plane; shell 1 by pairs
// of opposite directions; shells 2 and 3 direction by direction (2, its
// opposite, 3, its opposite); shell 4 by pairs.  lam: the rest plane, then
// every shell by pairs of opposite directions.
__host__ __device__ constexpr int pro_f_plane(int b) {
  return b == 0 ? 0
         : b <= 8 ? 1 + (b - 1) / 2 + 4 * ((b - 1) % 2)
         : b <= 24 ? 9 + (b - 9) / 4 + 4 * ((b - 9) % 4)
                   : 25 + (b - 25) / 2 + 4 * ((b - 25) % 2);
}
__host__ __device__ constexpr int pro_l_plane(int c) {
  return c == 0 ? 0 : 1 + kNDirs * ((c - 1) / kNDirs) + ((c - 1) % kNDirs) / 2 + kHalf * ((c - 1) % 2);
}
static_assert(pro_f_plane(2) == 5 && pro_f_plane(11) == 17 && pro_f_plane(12) == 21 && pro_f_plane(13) == 10 &&
                  pro_f_plane(26) == 29 && pro_f_plane(32) == 32 && pro_l_plane(2) == 5 && pro_l_plane(9) == 9 &&
                  pro_l_plane(32) == 32,
              "node-phase plane order");

// Running sums of the node phase for two nodes.
struct NodeAcc {
  // moments (Eqs. 3-5) in float-float, float sums of the current shell group
  // and of shell 3 alone, plane values waiting for the rest of their unit
  ff2 rho, jx, jy, e;
  f2 S, X, Xl, Y, Yl, S3, X3, X3l, Y3, Y3l, pa, pb, pc;
  // the state rounded to float, and the factors of the equilibrium cotangent
  f2 rh, ux, uy, E;
  bool ok0, ok1;
  f2 F[5], Fd[5], invE, s, a0, a1, a1h, uxE, uyE;
  // G = sum_q lam_q d f^eq_q / d(rho, u, E): totals and the current shell
  f2 A, Bx, By, Cs, Dx, Fq, Ak, Bxk, Byk, Ck, Dk, lp, l0;
};

__device__ __forceinline__ f2 recip1_2(f2 x) {
  const f2 r = mk2(recip_fast(x.x), recip_fast(x.y));
  return fma2(r, fma2(neg2(x), r, bc2(1.f)), r);
}

// Temperature recovery E = (e - |j|^2 / (2 rho)) / rho in float-float, the
// state rounded once, then the weights F_k(E), F'_k(E) (Eq. 11) and the
// polynomial coefficients of Eq. (10) for the cotangent.
__device__ __forceinline__ void node_state(NodeAcc& a, const DvmConst<float>& d) {
  const ff2 inv = ff2_recip(a.rho);
  const ff2 ux = ff2_mul(a.jx, inv), uy = ff2_mul(a.jy, inv);
  const ff2 ke = ff2_add(ff2_mul(a.jx, ux), ff2_mul(a.jy, uy));   // |j|^2 / rho
  const ff2 E = ff2_mul(ff2_add(a.e, ff2_scale(ke, -0.5f)), inv);
  a.ok0 = a.rho.hi.x > 0.f && E.hi.x > 0.f && isfinite(a.e.hi.x) && isfinite(a.jx.hi.x) && isfinite(a.jy.hi.x);
  a.ok1 = a.rho.hi.y > 0.f && E.hi.y > 0.f && isfinite(a.e.hi.y) && isfinite(a.jx.hi.y) && isfinite(a.jy.hi.y);
  a.rh = ff2_round(a.rho);
  a.ux = ff2_round(ux);
  a.uy = ff2_round(uy);
  a.E = ff2_round(E);
  f2 Fs = bc2(0.f), Fds = bc2(0.f);
#pragma unroll
  for (int k = 1; k <= 4; ++k) {
    const float* c = d.Fc[k];
    a.F[k] = mul2(a.E, fma2(a.E, fma2(a.E, fma2(a.E, bc2(c[3]), bc2(c[2])), bc2(c[1])), bc2(c[0])));
    a.Fd[k] = fma2(a.E, fma2(a.E, fma2(mul2(a.E, bc2(4.f)), bc2(c[3]), bc2(3.f * c[2])), bc2(2.f * c[1])), bc2(c[0]));
    Fs = add2(Fs, a.F[k]);
    Fds = add2(Fds, a.Fd[k]);
  }
  a.F[0] = fma2(bc2(-d.B0), Fs, bc2(1.f));
  a.Fd[0] = mul2(bc2(-d.B0), Fds);
  a.invE = recip1_2(a.E);
  a.s = mul2(fma2(a.ux, a.ux, mul2(a.uy, a.uy)), a.invE);
  a.a1 = fma2(bc2(-0.5f), a.s, bc2(1.f));
  a.a0 = fma2(mul2(bc2(0.125f), a.s), a.s, a.a1);
  a.uxE = mul2(a.ux, a.invE);
  a.uyE = mul2(a.uy, a.invE);
  a.a1h = mul2(bc2(0.5f), a.a1);
}

// Box B of the node phase, with v the two nodes' values of its plane.
template <int B>
__device__ __forceinline__ void node_box(NodeAcc& a, f2 v, const DvmConst<float>& d) {
  if constexpr (B == 0) {
    a.rho = ff2_of(v);
    a.jx = a.jy = a.e = ff2_of(bc2(0.f));
    a.S = a.X = a.Xl = a.Y = a.Yl = bc2(0.f);
    a.S3 = a.X3 = a.X3l = a.Y3 = a.Y3l = bc2(0.f);
  } else if constexpr (B <= 8 || (B >= 25 && B < kQ)) {
    // shell 1 or 4: f_a + f_b and (f_a - f_b) c_i of each pair of opposite directions
    constexpr int base = B <= 8 ? 1 : 25, j = B - base, q = base + j / 2;
    if constexpr (j % 2 == 0) {
      a.pa = v;
    } else {
      a.S = add2(a.S, add2(a.pa, v));
      const f2 dd = sub2(a.pa, v);
      a.X = fma2(bc2(d.cx[q]), dd, a.X);
      a.Xl = fma2(bc2(d.cx_lo[q]), dd, a.Xl);
      a.Y = fma2(bc2(d.cy[q]), dd, a.Y);
      a.Yl = fma2(bc2(d.cy_lo[q]), dd, a.Yl);
    }
    if constexpr (B == 8 || B == kQ - 1) {
      constexpr int k = B == 8 ? 1 : 4;
      const ff2 sp{bc2(d.speed[k]), bc2(d.speed_lo[k])}, hv{bc2(d.half_v2[k]), bc2(d.half_v2_lo[k])};
      a.rho = ff2_add(a.rho, ff2_of(a.S));
      a.jx = ff2_add(a.jx, ff2_mul(sp, ff2{a.X, a.Xl}));
      a.jy = ff2_add(a.jy, ff2_mul(sp, ff2{a.Y, a.Yl}));
      a.e = ff2_add(a.e, ff2_mul(hv, ff2_of(a.S)));
      a.S = a.X = a.Xl = a.Y = a.Yl = bc2(0.f);
    }
    if constexpr (B == kQ - 1) node_state(a, d);
  } else if constexpr (B < 25) {
    // shells 2 and 3 direction by direction: (f2_a + f3_a) +- (f2_b + f3_b)
    // with the speed of shell 2, and shell 3 alone for the speed difference
    constexpr int i = (B - 9) / 4, j = (B - 9) % 4, q = 9 + i, q3 = 17 + i;
    if constexpr (j == 0) {
      a.pa = v;
    } else if constexpr (j == 1) {
      a.pb = v;
    } else if constexpr (j == 2) {
      a.pc = v;
    } else {
      const f2 fa = add2(a.pa, a.pc), fb = add2(a.pb, v);
      a.S = add2(a.S, add2(fa, fb));
      const f2 dd = sub2(fa, fb);
      a.X = fma2(bc2(d.cx[q]), dd, a.X);
      a.Xl = fma2(bc2(d.cx_lo[q]), dd, a.Xl);
      a.Y = fma2(bc2(d.cy[q]), dd, a.Y);
      a.Yl = fma2(bc2(d.cy_lo[q]), dd, a.Yl);
      a.S3 = add2(a.S3, add2(a.pc, v));
      const f2 d3 = sub2(a.pc, v);
      a.X3 = fma2(bc2(d.cx[q3]), d3, a.X3);
      a.X3l = fma2(bc2(d.cx_lo[q3]), d3, a.X3l);
      a.Y3 = fma2(bc2(d.cy[q3]), d3, a.Y3);
      a.Y3l = fma2(bc2(d.cy_lo[q3]), d3, a.Y3l);
    }
    if constexpr (B == 24) {
      const ff2 sp{bc2(d.speed[2]), bc2(d.speed_lo[2])}, hv{bc2(d.half_v2[2]), bc2(d.half_v2_lo[2])};
      a.rho = ff2_add(a.rho, ff2_of(a.S));
      a.jx = ff2_add(a.jx, ff2_mul(sp, ff2{a.X, a.Xl}));
      a.jy = ff2_add(a.jy, ff2_mul(sp, ff2{a.Y, a.Yl}));
      a.e = ff2_add(a.e, ff2_mul(hv, ff2_of(a.S)));
      const ff2 dv{bc2(d.dv23), bc2(d.dv23_lo)}, dh{bc2(d.dh23), bc2(d.dh23_lo)};
      a.jx = ff2_add(a.jx, ff2_mul(dv, ff2{a.X3, a.X3l}));
      a.jy = ff2_add(a.jy, ff2_mul(dv, ff2{a.Y3, a.Y3l}));
      a.e = ff2_add(a.e, ff2_mul(dh, ff2_of(a.S3)));
      a.S = a.X = a.Xl = a.Y = a.Yl = bc2(0.f);
    }
  } else {
    constexpr int c = B - kQ;   // lam plane pro_l_plane(c)
    if constexpr (c == 0) {
      // rest velocity: x = 0
      a.l0 = v;
      const f2 l0F0 = mul2(v, a.F[0]);
      a.A = mul2(l0F0, a.a0);
      a.Bx = a.By = a.Dx = bc2(0.f);
      a.Cs = mul2(l0F0, fma2(bc2(0.25f), a.s, bc2(-0.5f)));
      a.Fq = mul2(mul2(v, a.Fd[0]), a.a0);
      a.Ak = a.Bxk = a.Byk = a.Ck = a.Dk = bc2(0.f);
    } else if constexpr ((c - 1) % 2 == 0) {
      a.lp = v;
    } else {
      // the pair (v, -v) of direction i of shell k shares the even and odd
      // parts of P, P_x and P_s (x = v.u/E, s = u^2/E)
      constexpr int k = 1 + (c - 1) / kNDirs, q = pro_l_plane(c - 1);
      const f2 vx = bc2(d.vx[q]), vy = bc2(d.vy[q]);
      const f2 x = fma2(vx, a.uxE, mul2(vy, a.uyE));
      const f2 x2 = mul2(x, x);
      const f2 Pe = fma2(x2, fma2(x2, bc2(1.0f / 24.0f), a.a1h), a.a0);   // P(+-x) = Pe +- Po
      const f2 Xo = mul2(x, fma2(x2, bc2(1.0f / 6.0f), a.a1));            // odd part of P and of P_x
      const f2 Xe = fma2(x2, bc2(0.5f), a.a1);                             // even part of P_x
      const f2 Se = fma2(bc2(-0.25f), x2, fma2(bc2(0.25f), a.s, bc2(-0.5f)));   // P_s(+-x) = Se -+ x/2
      const f2 ls = add2(a.lp, v), ld = sub2(a.lp, v);
      a.Ak = fma2(ls, Pe, fma2(ld, Xo, a.Ak));
      const f2 lpx = fma2(ld, Xe, mul2(ls, Xo));                       // lp P_x(x) - lm P_x(-x)
      a.Bxk = fma2(lpx, vx, a.Bxk);
      a.Byk = fma2(lpx, vy, a.Byk);
      a.Ck = fma2(ls, Se, fma2(mul2(ld, bc2(-0.5f)), x, a.Ck));
      a.Dk = fma2(x, fma2(ls, Xo, mul2(ld, Xe)), a.Dk);                // lp x P_x(x) + lm (-x) P_x(-x)
      if constexpr (c % kNDirs == 0) {
        a.A = fma2(a.F[k], a.Ak, a.A);
        a.Bx = fma2(a.F[k], a.Bxk, a.Bx);
        a.By = fma2(a.F[k], a.Byk, a.By);
        a.Cs = fma2(a.F[k], a.Ck, a.Cs);
        a.Dx = fma2(a.F[k], a.Dk, a.Dx);
        a.Fq = fma2(a.Fd[k], a.Ak, a.Fq);
        a.Ak = a.Bxk = a.Byk = a.Ck = a.Dk = bc2(0.f);
      }
    }
  }
}

template <int B, int J, int N>
__device__ __forceinline__ void node_group_boxes(NodeAcc& a, const float* pring, int o, const DvmConst<float>& d) {
  node_box<B + J>(a, lds2(pring + node_slot(B + J) * kNPl + o), d);
  if constexpr (J + 1 < N) node_group_boxes<B, J + 1, N>(a, pring, o, d);
}

// Groups G .. of the node phase: wait for the group's half of the slots,
// accumulate its planes, release the half (the group two ahead refills it;
// after the last odd group, the first two pairs take the ring).  Returns the
// group whose copies did not land in time, or kPGroups.
template <int G, class Refill, class Prime>
__device__ __forceinline__ int node_groups(NodeAcc& a, const float* pring, int o, uint64_t* pbar, uint64_t wait_ns,
                                           const DvmConst<float>& d, Refill refill, Prime prime) {
  const bool ok = wait_ns != 0 && mbar_wait_bounded(&pbar[G % 2], (uint32_t)((G / 2) & 1), wait_ns);
  if (ok) node_group_boxes<G * kPGroup, 0, node_group_size(G)>(a, pring, o, d);
  if (__syncthreads_or(!ok)) return G;
  if (threadIdx.x == 0 && (G + 2 < kPGroups || G == kPGroups - 2)) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (G + 2 < kPGroups)
      refill(G + 2);
    else
      prime();
  }
  if constexpr (G + 1 < kPGroups) return node_groups<G + 1>(a, pring, o, pbar, wait_ns, d, refill, prime);
  return kPGroups;
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

// Phase (A) for one label at this thread's two nodes, its upwind offsets U
// (columns) and V (window rows) as constants: the products of the MWB
// partials in r and theta; returns lam of the two nodes.
template <int U, int V>
__device__ __forceinline__ f2 products_label(const float* w, const float* wl, float* P, int p_rad, int p_az, f2 a_r,
                                             f2 k_r, f2 a_t, f2 k_t) {
  const f2 C = lds2(w);
  const f2 S2 = lds2(w + 2 * U);                            // f(n + 2u) of both nodes
  const f2 u1 = U > 0 ? mk2(C.y, S2.x) : mk2(S2.y, C.x);     // f(n + u)
  f2 MD, MP;
  mwb_partials2(a_r, k_r, sub2(C, u1), sub2(u1, S2), MD, MP);
  const f2 lam = lds2(wl);
  sts2(P + kAR + p_rad, mul2(lam, MD));
  sts2(P + kBR + p_rad, mul2(lam, MP));
  const f2 T1 = lds2(w + V), T2 = lds2(w + 2 * V);
  mwb_partials2(a_t, k_t, sub2(C, T1), sub2(T1, T2), MD, MP);
  sts2(P + p_az, mul2(lam, MD));
  sts2(P + p_az + (kBT - kAT), mul2(lam, MP));
  return lam;
}

// Phase (A) for both labels of a pair: q1's upwind offsets UR, VT, q2's the
// opposite ones.
template <int UR, int VT>
__device__ __forceinline__ void products_pair(const float* sf, const float* sl, float* pb, int o, int p_rad, int p_az,
                                              f2 a_r, f2 k_r, f2 a_t, f2 k_t, f2 lam_c[2]) {
  lam_c[0] = products_label<UR, VT>(sf + o, sl + o, pb, p_rad, p_az, a_r, k_r, a_t, k_t);
  lam_c[1] = products_label<-UR, -VT>(sf + kAPl + o, sl + kAPl + o, pb + kProd, p_rad, p_az, a_r, k_r, a_t, k_t);
}

// Products of one halo row (window row rr) at the node pair jj, jj + 1, for
// the label whose upwind side points into the tile: V = +row for the rows
// below the tile, -row for those above.
template <int V>
__device__ __forceinline__ void halo_row(const float* sf, const float* sl, float* pb, const float4* ctab,
                                         const float* invr, int pair, int rr, int jj) {
  const float4 eh = ctab[rr * kANP + pair];
  const bool q1_up_pos = (__float_as_int(eh.w) & 2) != 0;
  const int L = (V > 0) == q1_up_pos ? 0 : 1;
  const f2 ath = mul2(bc2(eh.z), lds2(invr + jj)), kth = fma2(neg2(ath), ath, ath);
  const int o = rr * kWinR + kLeft + jj;
  const float* w = sf + L * kAPl + o;
  const f2 C = lds2(w), T1 = lds2(w + V), T2 = lds2(w + 2 * V);
  f2 MD, MP;
  mwb_partials2(ath, kth, sub2(C, T1), sub2(T1, T2), MD, MP);
  const f2 lam = lds2(sl + L * kAPl + o);
  float* P = pb + L * kProd + kAT + rr * kTileR + jj;
  sts2(P, mul2(lam, MD));
  sts2(P + (kBT - kAT), mul2(lam, MP));
}

// Radial gather of one label at the two nodes (upwind offset U): A(c) -
// A(c - u) + B(c - u) - B(c - 2u).
template <int U>
__device__ __forceinline__ f2 gather_radial2(const float* P, int p_rad) {
  const f2 A0 = lds2(P + kAR + p_rad), B0 = lds2(P + kBR + p_rad);
  const f2 An = lds2(P + kAR + p_rad - 2 * U), Bn = lds2(P + kBR + p_rad - 2 * U);
  const f2 Au = U > 0 ? mk2(An.y, A0.x) : mk2(A0.y, An.x);
  const f2 Bu = U > 0 ? mk2(Bn.y, B0.x) : mk2(B0.y, Bn.x);
  return sub2(add2(sub2(A0, Au), Bu), Bn);
}

// Azimuthal gather of one label where the rows -2 .. +2 around the node all
// have their upwind side on one side: the readers of the node at +W, +2W.
template <int W>
__device__ __forceinline__ f2 gather_az2(const float* P) {
  constexpr int DB = kBT - kAT;
  return sub2(sub2(add2(lds2(P), lds2(P + DB + W)), lds2(P + W)), lds2(P + DB + 2 * W));
}

// WALLS: the launch may contain wall tiles (the tiles of radial index 0 and
// those within 33 columns of n_r); the interior launch is the instance
// without any wall code.
template <bool WALLS>
__global__ void __launch_bounds__(kAThr, 3)
    adjoint_pair_f32x2(const __grid_constant__ CUtensorMap tmap_f, const __grid_constant__ CUtensorMap tmap_l,
                       const __grid_constant__ CUtensorMap tmap_fn, const __grid_constant__ CUtensorMap tmap_ln,
                       const float* __restrict__ f, const float* __restrict__ lam_in, float* __restrict__ lam_out,
                       const EqParams<float>* __restrict__ ghost, const float* __restrict__ gwall,
                       const float* __restrict__ gdir, int a0, int na,
                       int b0, const __grid_constant__ StepParams p, const __grid_constant__ DvmConst<float> d) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* ring = reinterpret_cast<float*>(smem_raw);
  float* prod = reinterpret_cast<float*>(smem_raw + kRingBytes);
  float* invr = reinterpret_cast<float*>(smem_raw + kRingBytes + kProdBytes);
  float4* ctab = reinterpret_cast<float4*>(smem_raw + kRingBytes + kProdBytes + kInvrBytes);   // [kTT + 4][kANP]
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + kRingBytes + kProdBytes + kInvrBytes + kTabBytes);
  uint64_t* pbar = bar + kAS;                   // the node phase's two halves

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
  // node-phase group g (boxes 6g .. 6g + 5) into its half of the ring
  auto issue_group = [&](int g) {
    const int nb = node_group_size(g);
    mbar_arrive_expect_tx(&pbar[g % 2], (uint32_t)(nb * kNPl * 4));
    for (int j = 0; j < nb; ++j) {
      const int b = g * kPGroup + j;
      float* dst = ring + node_slot(b) * kNPl;
      if (b < kQ)
        tma_load_3d(dst, &tmap_fn, r0, t0 + kGhostRows, pro_f_plane(b), &pbar[g % 2]);
      else
        tma_load_3d(dst, &tmap_ln, r0, t0 + kGhostRows, pro_l_plane(b - kQ), &pbar[g % 2]);
    }
  };
  if (tid == 0) {
    tma_prefetch_desc(&tmap_f);
    tma_prefetch_desc(&tmap_l);
    tma_prefetch_desc(&tmap_fn);
    tma_prefetch_desc(&tmap_ln);
    for (int s = 0; s < kAS + 2; ++s) mbar_init(&bar[s], 1);
    mbar_fence_init();
    issue_group(0);
    issue_group(1);
  }
  auto prime_pairs = [&]() {
    for (int s = 0; s < kAS && s < kANP; ++s) issue_pair(s, s);
  };
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

  // ---- this thread's two nodes ---------------------------------------------
  const int warp = tid >> 5, lane = tid & 31;
  const int rl = 2 * warp + (lane >> 4);       // tile row
  const int j2 = 2 * (lane & 15);              // even radial offset
  const int t = t0 + rl, r = r0 + j2;
  const bool row_ok = t < p.n_theta;
  const bool v0 = row_ok && r < p.n_r, v1 = row_ok && r + 1 < p.n_r;
  const int srow = t + kGhostRows;
  const size_t plane_out = (size_t)p.rows * p.pitch;
  const f2 decay = bc2((float)p.decay);
  const int row = rl + 2;                       // window row of this thread's nodes
  const int o_node = row * kWinR + kLeft + j2;  // first node in a window plane
  f2 gs[4];
  f2 lam0;                                      // lam of the rest velocity
  {
    // (1 - d) g of both nodes; rows past the grid see the ghost rows or the
    // copies' zero fill, columns past n_r zero fill: never stored
    NodeAcc a;
    const int bad = node_groups<0>(a, ring, rl * kTileR + j2, pbar, p.wait_ns, d, issue_group, prime_pairs);
    if (bad < kPGroups) {
      // a copy did not land in time: report it and give the copies still in
      // flight (the failed group, the one after it, and the first two pairs
      // once they were issued) a bounded time to finish before the block exits
      if (tid == 0) {
        atomicOr(p.status, PCLB_FLAG_TIMEOUT);
        mbar_wait_bounded(&pbar[bad % 2], (uint32_t)((bad / 2) & 1), kDefaultWaitNs);
        if (bad + 1 < kPGroups) mbar_wait_bounded(&pbar[(bad + 1) % 2], (uint32_t)(((bad + 1) / 2) & 1), kDefaultWaitNs);
        if (bad == kPGroups - 1)
          for (int s = 0; s < kAS && s < kANP; ++s) mbar_wait_bounded(&bar[s], 0u, kDefaultWaitNs);
      }
      return;
    }
    if ((v0 && !a.ok0) || (v1 && !a.ok1)) atomicOr(p.status, PCLB_FLAG_NONPHYS);
    f2 G[4], g[4];
    G[0] = a.A;
    const f2 rE = mul2(a.rh, a.invE);
    G[1] = mul2(rE, fma2(mul2(bc2(2.f), a.ux), a.Cs, a.Bx));
    G[2] = mul2(rE, fma2(mul2(bc2(2.f), a.uy), a.Cs, a.By));
    G[3] = mul2(a.rh, sub2(a.Fq, mul2(fma2(a.s, a.Cs, a.Dx), a.invE)));
    to_moment_cotangent2(a.rh, a.ux, a.uy, a.E, G, g);
    lam0 = a.l0;
    const f2 omd = sub2(bc2(1.f), decay);
#pragma unroll
    for (int j = 0; j < 4; ++j) gs[j] = mul2(omd, g[j]);
    // the cotangent the ghost nodes return to the two nodes next to each wall
    if (WALLS && row_ok && (r < 2 || r + 3 >= p.n_r)) {
      auto wall = [&](int rr) {
        float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
        auto add = [&](int side, int node) {
          const float4 x = *reinterpret_cast<const float4*>(gwall + ((size_t)(side * 2 + node) * p.n_theta + t) * 4);
          w.x += x.x; w.y += x.y; w.z += x.z; w.w += x.w;
        };
        if (rr == 0) add(0, 0);
        if (rr == 1) add(0, 1);
        if (rr == p.n_r - 1) add(1, 0);
        if (rr == p.n_r - 2) add(1, 1);
        return w;
      };
      const float4 w0 = wall(r), w1 = wall(r + 1);
      gs[0] = add2(gs[0], mk2(w0.x, w1.x));
      gs[1] = add2(gs[1], mk2(w0.y, w1.y));
      gs[2] = add2(gs[2], mk2(w0.z, w1.z));
      gs[3] = add2(gs[3], mk2(w0.w, w1.w));
    }
  }
  const int p_rad = rl * kRC + j2 + 2;          // its radial product slot
  const int p_az = kAT + row * kTileR + j2;     // its azimuthal product slot
  const f2 my_invr = lds2(invr + j2);
  float* out_row = lam_out + (size_t)srow * p.pitch + r;
  const bool plain_tile = r0 + kTileR <= p.n_r && t0 >= 2 && t0 + kTT <= p.n_theta - 2;
  auto store = [&](int q, f2 o) {
    if (plain_tile) {
      __stcs(reinterpret_cast<float2*>(out_row + (size_t)q * plane_out), o);
      return;
    }
    // seam and ragged tiles: the seam rows' ghost copies, formed here so
    // that plain tiles keep no registers for them
    const bool lo_ghost = row_ok && t >= p.n_theta - 2;
    const bool hi_ghost = row_ok && t < 2;
    float* out_lo = lam_out + (size_t)max(t - (p.n_theta - 2), 0) * p.pitch + r;
    float* out_hi = lam_out + (size_t)(p.n_theta + kGhostRows + t) * p.pitch + r;
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
  // rest velocity: no convection
  store(0, add2(fma2(decay, lam0, gs[0]), mul2(gs[3], bc2(d.half_v2[0]))));

  // wall tiles: the ghost states of the rows this thread fills (threads 0..15
  // the inner wall, 32..47 the outer wall, one tile row each)
  const int cw_out = p.n_r - 1 - r0 + kLeft;
  const bool inner = r0 == 0, outer = cw_out <= kLeft + kTileR;
  const bool wall_tile = WALLS && (inner || outer);
  const int gside = tid >> 5, grow = tid & 31;
  const bool fills = wall_tile && tid < 64 && grow < kTT && t0 + grow < p.n_theta && (gside == 0 ? inner : outer);
  const EqParams<float>* eg = ghost + (size_t)(gside * 3) * p.n_theta + t0 + grow;   // layer l at + l n_theta
  const bool gneq = (p.bc_kind[gside & 1] & PCLB_BC_NEQ) != 0;   // its ghosts carry the wall node's departure

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
      // radial ghost columns of this pair's f planes (f = f^eq of the ghost
      // states, plus the wall node's departure for non-equilibrium ghosts)
      if (fills && ok) {
        float* fw = st + (2 + grow) * kWinR;
        const int c0 = gside == 0 ? kLeft : cw_out, stp = gside == 0 ? 1 : -1;
        float dep1 = 0.f, dep2 = 0.f;   // the wall node's departure f_q - f^eq_q
        if (gneq) {
          const EqParams<float> ea = eg[(size_t)2 * p.n_theta];
          dep1 = fw[c0] - feq_q<float>(ea, d.vx[q1], d.vy[q1], k);
          dep2 = fw[kAPl + c0] - feq_q<float>(ea, d.vx[q2], d.vy[q2], k);
        }
        for (int l = 0; l < 2; ++l) {
          const int c = c0 - stp * (1 + l);
          if (c < 0 || c >= kWinR) continue;
          const EqParams<float> e = eg[(size_t)l * p.n_theta];
          fw[c] = feq_q<float>(e, d.vx[q1], d.vy[q1], k) + dep1;
          fw[kAPl + c] = feq_q<float>(e, d.vx[q2], d.vy[q2], k) + dep2;
        }
      }
      __syncthreads();
    }

    // (A) products lam(n) M_D(n), lam(n) M_Dp(n)
    const float* sf = st;                          // f q1, f q2 at + kAPl
    const float* sl = st + 2 * kAPl;               // lam q1, lam q2 at + kAPl
    const float4 ce = ctab[row * kANP + pair];
    const int fl_c = __float_as_int(ce.w);
    const f2 a_r = bc2(ce.x), k_r = bc2(ce.y);
    const f2 a_t = mul2(bc2(ce.z), my_invr), k_t = fma2(neg2(a_t), a_t, a_t);
    f2 lam_c[2];
    // bit 0: q1 reads n + 1, n + 2 in r; bit 1: q1 reads the rows above.  The
    // two rows of a warp nearly always agree (a label's upwind side changes
    // at a few theta rows only), so the branch is uniform in practice.
    switch (fl_c & 3) {
      case 0: products_pair<-1, -kWinR>(sf, sl, pb, o_node, p_rad, p_az, a_r, k_r, a_t, k_t, lam_c); break;
      case 1: products_pair<1, -kWinR>(sf, sl, pb, o_node, p_rad, p_az, a_r, k_r, a_t, k_t, lam_c); break;
      case 2: products_pair<-1, kWinR>(sf, sl, pb, o_node, p_rad, p_az, a_r, k_r, a_t, k_t, lam_c); break;
      default: products_pair<1, kWinR>(sf, sl, pb, o_node, p_rad, p_az, a_r, k_r, a_t, k_t, lam_c); break;
    }
    if (tid < 64) {
      // halo rows (window rows 0, 1, kTT + 2, kTT + 3), the label whose
      // upwind side points into the tile: warp 0 the rows below the tile
      // (read by the label with its upwind side at +theta), warp 1 the rows
      // above it
      if (tid < 32)
        halo_row<kWinR>(sf, sl, pb, ctab, invr, pair, tid >> 4, 2 * (tid & 15));
      else
        halo_row<-kWinR>(sf, sl, pb, ctab, invr, pair, kTT + 2 + ((tid >> 4) & 1), 2 * (tid & 15));
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
      if (fl_c & 1) {
        acc[0] = gather_radial2<1>(pb, p_rad);
        acc[1] = gather_radial2<-1>(pb + kProd, p_rad);
      } else {
        acc[0] = gather_radial2<-1>(pb, p_rad);
        acc[1] = gather_radial2<1>(pb + kProd, p_rad);
      }
      const int tneg = fl_c >> 2;                  // bit o: row o - 2 has v_theta < 0 for q1
      constexpr int DB = kBT - kAT;
      if (tneg == 0) {
        // q1's readers at +V, +2V, q2's at -V, -2V (V = one row)
        acc[0] = add2(acc[0], gather_az2<kTileR>(pb + p_az));
        acc[1] = add2(acc[1], gather_az2<-kTileR>(pb + kProd + p_az));
      } else if (tneg == 31) {
        acc[0] = add2(acc[0], gather_az2<-kTileR>(pb + p_az));
        acc[1] = add2(acc[1], gather_az2<kTileR>(pb + kProd + p_az));
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
      f2 o1 = sub2(fma2(decay, lam_c[0], add2(A, B)), acc[0]);
      f2 o2 = sub2(fma2(decay, lam_c[1], sub2(A, B)), acc[1]);
      if (wall_tile) {
        // non-equilibrium ghosts hand their cotangent straight to f_q of the wall node
        for (int sd = 0; sd < 2; ++sd) {
          if (!(p.bc_kind[sd] & PCLB_BC_NEQ)) continue;
          const int rw = sd == 0 ? 0 : p.n_r - 1;
          const float* gd = gdir + ((size_t)sd * p.n_theta + t) * kQ;
          if (r == rw) { o1.x += gd[q1]; o2.x += gd[q2]; }
          if (r + 1 == rw) { o1.y += gd[q1]; o2.y += gd[q2]; }
        }
      }
      store(q1, o1);
      store(q2, o2);
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

template <bool WALLS>
cudaError_t launch_pairs(const CUtensorMap* tmap_f, const CUtensorMap* tmap_l, const CUtensorMap* tmap_fn,
                                const CUtensorMap* tmap_ln, const float* f, const float* lam_in, float* lam_out,
                                const EqParams<float>* ghost, const float* gwall, const float* gdir, int a0, int na,
                                int b0, int nx, const StepParams& p, const DvmConst<float>& d, cudaStream_t s) {
  static std::atomic<unsigned long long> configured{0};   // per instance and device
  {
    const cudaError_t e = set_smem_once(adjoint_pair_f32x2<WALLS>, kASmem, configured);
    if (e != cudaSuccess) return e;
  }
  const dim3 grid((unsigned)nx, (unsigned)((p.n_theta + kTT - 1) / kTT));
  adjoint_pair_f32x2<WALLS><<<grid, kAThr, kASmem, s>>>(*tmap_f, *tmap_l, *tmap_fn, *tmap_ln, f, lam_in, lam_out,
                                                        ghost, gwall, gdir, a0, na, b0, p, d);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_adjoint_pairs_f32(const CUtensorMap* tmap_f, const CUtensorMap* tmap_l, const CUtensorMap* tmap_fn,
                                     const CUtensorMap* tmap_ln, const float* f,
                                     const float* lam_in, float* lam_out, const EqParams<float>* ghost,
                                     const float* gwall, const float* gdir, int a0, int na, int b0, int nx,
                                     bool walls, const StepParams& p, const DvmConst<float>& d, cudaStream_t s) {
  return walls ? launch_pairs<true>(tmap_f, tmap_l, tmap_fn, tmap_ln, f, lam_in, lam_out, ghost, gwall, gdir, a0, na,
                                    b0, nx, p, d, s)
               : launch_pairs<false>(tmap_f, tmap_l, tmap_fn, tmap_ln, f, lam_in, lam_out, ghost, gwall, gdir, a0,
                                     na, b0, nx, p, d, s);
}

}  // namespace pclb
