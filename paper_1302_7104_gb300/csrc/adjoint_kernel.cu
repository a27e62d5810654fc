// Reverse-mode adjoint of one time step (Eq. 38 with the boundary nodes of
// Sec. II C): given the state f^n and the cotangent lam^{n+1} of f^{n+1},
// computes lam^n = J(f^n)^T lam^{n+1}.
//
// With m = (rho, j_x, j_y, e) the moments (linear in f, psi_q = (1, v_x, v_y,
// |v|^2/2)), the step is F_q(c) = (1-d) f^eq_q(m(c)) + d f_q(c) - M^r_q(c) -
// M^theta_q(c), d = exp(-dt/tau) (Eq. 19), M the MWB increments (Eq. 28)
// M = a D + K h(D, Dp), h = |D|(D - Dp)/(|D| + |Dp|), a = |C|, K = |C|(1-|C|),
// D, Dp the upwind differences of the node.  Hence, per node c and label q,
//   lam^n_q(c) = d lam_q(c) + (1-d) psi_q . g(c)
//              - sum over the nodes n whose stencil reads f_q(c) of
//                lam_q(n) dM_q(n)/df_q(c)                    (r and theta)
//              + psi_q . g_wall(c)  for the two nodes next to a wall,
// with g(c) = (dm/d(rho,u,E))^T sum_q' lam_q'(c) df^eq_q'/d(rho,u,E), and
// g_wall the cotangent that flows back from the radial ghost nodes through
// f^eq of the extrapolated state (Eq. 39).  |x| is differentiated as
// sign(x) with sign(0) = 0 (the switch function on its active branch); at
// D = Dp = 0 the derivative of h is 0.
//
// One CTA: 32 (r) x TT (theta) nodes, one node per thread; the windows of f
// and lam over [r0-4, r0+36) x [t0-2, t0+TT+2) for all 33 labels are staged
// in shared memory by TMA.  Velocities are processed in pairs of opposite
// labels, each in two phases: (A) every node whose upwind stencil can reach
// the tile forms lam(n) dM(n)/dD and lam(n) dM(n)/dDp once, in r and in
// theta, into shared memory; (B) every tile node gathers the products of the
// nodes that read it.  One barrier per pair separates the phases; the
// products live in two alternating buffers.
#include <cuda.h>
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "adjoint_common.cuh"
#include "ghost_cols.cuh"
#include "f32_state.cuh"
#include "pclb_internal.h"

namespace pclb {

template <class T>
struct AdjTile;
template <>
struct AdjTile<float> {
  static constexpr int TT = kAdjRows32;
};
template <>
struct AdjTile<double> {
  static constexpr int TT = kAdjRows64;
};

// Courant entry of one pair of opposite velocities at one theta row:
// (|C_r|, |C_r|(1 - |C_r|), |v_theta| dt / dtheta, flags) with flag bit 0 set
// when v_r < 0 and bit 1 when v_theta < 0 for the first label of the pair.
template <class T>
struct alignas(4 * sizeof(T)) CourEntry {
  T a_r, k_r, a_w;
  int fl;
};

template <class T>
struct AdjSize {
  static constexpr int TT = AdjTile<T>::TT;
  static constexpr int plane = kWinR * (TT + 4);
  static constexpr int npairs = 4 * kNDirs / 2;
  // products of one label: radial A, B over TT rows x 36 columns (tile
  // columns -2 .. 33), azimuthal A, B over TT + 4 rows (-2 .. TT + 1) x 32
  static constexpr int rcols = kTileR + 4;
  static constexpr int prod = 2 * TT * rcols + 2 * (TT + 4) * kTileR;
  static constexpr int win_bytes = 2 * kQ * plane * (int)sizeof(T);
  static constexpr int prod_bytes = 2 * 2 * prod * (int)sizeof(T);  // 2 buffers x 2 labels
  static constexpr int gw_bytes = 2 * 2 * TT * 4 * (int)sizeof(T);
  static constexpr int invr_bytes = kTileR * (int)sizeof(T);
  static constexpr int tab_bytes = (TT + 4) * npairs * (int)sizeof(CourEntry<T>);
  static constexpr int smem = win_bytes + prod_bytes + gw_bytes + invr_bytes + tab_bytes + 128;
};

namespace {

constexpr uint64_t kAdjWaitNs = 2000000000ull;

template <class T>
struct Cour {
  T a_r, k_r, a_w;
  int up_r, up_t;   // upwind offsets in r (columns) and theta (rows): -1 or +1
};

__device__ __forceinline__ void courant_entry(const StepParams& p, int row, int pair, float& ar, float& kr,
                                              float& aw, int& fl) {
  const float4 e = p.courant[(size_t)row * (4 * kNDirs / 2) + pair];
  ar = e.x; kr = e.y; aw = e.z; fl = __float_as_int(e.w);
}
__device__ __forceinline__ void courant_entry(const StepParams& p, int row, int pair, double& ar, double& kr,
                                              double& aw, int& fl) {
  const double* e = p.courant64 + ((size_t)row * (4 * kNDirs / 2) + pair) * 4;
  ar = e[0]; kr = e[1]; aw = e[2]; fl = (int)e[3];
}

// Courant data of label q at stored row `row` (ghost rows included), from
// the table of opposite-velocity pairs.
template <class T>
__device__ __forceinline__ Cour<T> courant(const StepParams& p, const DvmConst<T>& d, int q, int row) {
  Cour<T> c;
  if (q == 0) {
    c.a_r = T(0); c.k_r = T(0); c.a_w = T(0); c.up_r = -1; c.up_t = -1;
    return c;
  }
  const int k = d.shell[q];
  const int i = (q - 1) % kNDirs;
  const bool second = i >= kNDirs / 2;
  const int pair = (k - 1) * (kNDirs / 2) + (second ? i - kNDirs / 2 : i);
  int fl;
  courant_entry(p, row, pair, c.a_r, c.k_r, c.a_w, fl);
  const bool vr_neg = ((fl & 1) != 0) != second;   // the partner has the opposite velocity
  const bool vt_neg = ((fl & 2) != 0) != second;
  c.up_r = vr_neg ? 1 : -1;
  c.up_t = vt_neg ? 1 : -1;
  return c;
}

// (rho, u_x, u_y, E) of one node for the cotangent of the equilibrium:
// float-float moments rounded to float in FP32, double in FP64.
__device__ __forceinline__ void adj_node_state(const float* f, int plane, const DvmConst<float>& d, float& rho,
                                               float& ux, float& uy, float& E, bool& ok) {
  const State32 m = state32(f, plane, d);
  rho = m.rho.hi + m.rho.lo;
  ux = m.ux.hi + m.ux.lo;
  uy = m.uy.hi + m.uy.lo;
  E = m.E.hi + m.E.lo;
  ok = m.ok;
}
__device__ __forceinline__ void adj_node_state(const double* f, int plane, const DvmConst<double>& d, double& rho,
                                               double& ux, double& uy, double& E, bool& ok) {
  const NodeState<double> m = node_moments(f, plane, d);
  rho = m.rho; ux = m.ux; uy = m.uy; E = m.E; ok = m.ok;
}

}  // namespace

template <class T>
__global__ void __launch_bounds__(AdjTile<T>::TT * 32, 1)
    adjoint_kernel(const __grid_constant__ CUtensorMap tmap_f, const __grid_constant__ CUtensorMap tmap_l,
                   T* __restrict__ lam_out, const __grid_constant__ StepParams p, const __grid_constant__ DvmConst<T> d) {
  constexpr int TT = AdjTile<T>::TT;
  constexpr int PLANE = AdjSize<T>::plane;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* sf = reinterpret_cast<T*>(smem_raw);
  T* sl = sf + kQ * PLANE;
  T* prod = sl + kQ * PLANE;                        // [buffer][label][products]
  T* gw = prod + 2 * 2 * AdjSize<T>::prod;          // [side][node][TT][4]
  T* invr = gw + 2 * 2 * TT * 4;                    // 1/r of the tile columns
  CourEntry<T>* ctab = reinterpret_cast<CourEntry<T>*>(invr + kTileR);   // [TT + 4][npairs]
  uint64_t* bar = reinterpret_cast<uint64_t*>(ctab + (TT + 4) * AdjSize<T>::npairs);   // [0] f, [1] lam

  const int r0 = blockIdx.x * kTileR;
  const int t0 = blockIdx.y * TT;
  const int tid = threadIdx.x;
  const int lane = tid & 31, rowl = tid >> 5;

  if (tid == 0) {
    tma_prefetch_desc(&tmap_f);
    tma_prefetch_desc(&tmap_l);
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
  }
  for (int i = tid; i < 2 * 2 * TT * 4; i += blockDim.x) gw[i] = T(0);
  if (tid < kTileR) invr[tid] = r0 + tid < p.n_r ? (T)p.inv_r[r0 + tid] : T(1);
  // Courant entries of the stored rows t0 .. t0 + TT + 3 (theta rows t0 - 2 .. t0 + TT + 1)
  for (int i = tid; i < (TT + 4) * AdjSize<T>::npairs; i += blockDim.x) {
    const int srow = t0 + i / AdjSize<T>::npairs, pair = i % AdjSize<T>::npairs;
    CourEntry<T> e{T(0), T(0), T(0), 0};
    if (srow < p.rows) courant_entry(p, srow, pair, e.a_r, e.k_r, e.a_w, e.fl);
    ctab[i] = e;
  }
  __syncthreads();
  if (tid == 0) {
    mbar_arrive_expect_tx(&bar[0], (uint32_t)(kQ * PLANE * sizeof(T)));
    mbar_arrive_expect_tx(&bar[1], (uint32_t)(kQ * PLANE * sizeof(T)));
#pragma unroll 1
    for (int q = 0; q < kQ; ++q) tma_load_3d(sf + q * PLANE, &tmap_f, r0 - kLeft, t0, q, &bar[0]);
#pragma unroll 1
    for (int q = 0; q < kQ; ++q) tma_load_3d(sl + q * PLANE, &tmap_l, r0 - kLeft, t0, q, &bar[1]);
  }
  // f first (moments, ghost columns); lam is awaited before it is first read
  const bool f_ok = mbar_wait_bounded(&bar[0], 0, kAdjWaitNs);
  if (__syncthreads_or(!f_ok)) {
    if (tid == 0) {
      atomicOr(p.status, PCLB_FLAG_TIMEOUT);
      mbar_wait_bounded(&bar[0], 0, kAdjWaitNs);
      mbar_wait_bounded(&bar[1], 0, kAdjWaitNs);
    }
    return;
  }

  // ---- radial ghost columns of f, exactly as the forward step ---------------
  const int cw_out = p.n_r - 1 - r0 + kLeft;
  const bool inner = r0 == 0;
  const bool outer = cw_out <= kLeft + kTileR;
  if (inner && rowl == 0 && lane < TT && t0 + lane < p.n_theta)
    fill_ghost_columns<T, PLANE>(sf, 2 + lane, 0, kLeft, t0 + lane, p, d);
  if (outer && rowl == 1 && lane < TT && t0 + lane < p.n_theta)
    fill_ghost_columns<T, PLANE>(sf, 2 + lane, 1, cw_out, t0 + lane, p, d);
  __syncthreads();

  // this thread's node moments (f only), while lam is still landing
  const int row = 2 + rowl;
  const int col = kLeft + lane;
  const int t = t0 + rowl;
  const int r = r0 + lane;
  const bool valid = r < p.n_r && t < p.n_theta;
  const int srow = t + kGhostRows;
  T n_rho = T(1), n_ux = T(0), n_uy = T(0), n_E = T(1);
  if (valid) {
    bool ok;
    adj_node_state(sf + row * kWinR + col, PLANE, d, n_rho, n_ux, n_uy, n_E, ok);
    if (!ok) atomicOr(p.status, PCLB_FLAG_NONPHYS);
  }
  const bool l_ok = mbar_wait_bounded(&bar[1], 0, kAdjWaitNs);
  if (__syncthreads_or(!l_ok)) {
    if (tid == 0) {
      atomicOr(p.status, PCLB_FLAG_TIMEOUT);
      mbar_wait_bounded(&bar[1], 0, kAdjWaitNs);
    }
    return;
  }

  // ---- cotangent returned by the ghost nodes to the two wall nodes ---------
  auto wall_feedback = [&](int side, int rl) {
    const int row = 2 + rl;
    const int srow = t0 + rl + kGhostRows;             // stored row of this theta node
    const int t = t0 + rl;
    const int step = side == 0 ? 1 : -1;
    const int ca = side == 0 ? kLeft : cw_out;          // wall node column
    const int cb = ca + step;                           // next node inward
    const int outward = -step;                          // upwind offset that reads the ghosts
    const NodeState<T> a = node_moments(sf + row * kWinR + ca, PLANE, d);
    const NodeState<T> b = node_moments(sf + row * kWinR + cb, PLANE, d);
    const int kind = p.bc_kind[side] & ~PCLB_BC_NEQ;
    T st[2][4];   // ghost states (rho, ux, uy, E), layers 0 and 1
    st[0][0] = T(2) * a.rho - b.rho;  st[1][0] = T(2) * st[0][0] - a.rho;
    st[0][1] = T(2) * a.ux - b.ux;    st[1][1] = T(2) * st[0][1] - a.ux;
    st[0][2] = T(2) * a.uy - b.uy;    st[1][2] = T(2) * st[0][2] - a.uy;
    st[0][3] = T(2) * a.E - b.E;      st[1][3] = T(2) * st[0][3] - a.E;
    if (kind != PCLB_BC_EXTRAP) {
      const double c = p.cos_t[t], s = p.sin_t[t];
      for (int l = 0; l < 2; ++l) {
        const double* v = p.bc_vals + (size_t)((side * 2 + l) * 4) * p.n_theta + t;
        st[l][1] = (T)(v[1 * p.n_theta] * c - v[2 * p.n_theta] * s);
        st[l][2] = (T)(v[1 * p.n_theta] * s + v[2 * p.n_theta] * c);
        if (kind == PCLB_BC_DIRICHLET) {
          st[l][0] = (T)v[0];
          st[l][3] = (T)v[3 * p.n_theta];
        }
      }
    }
    T Gl[2][4];
    for (int l = 0; l < 2; ++l) {
      // cotangent of ghost value f_q(layer l) = -sum_n lam_q(n) dM_q(n)/d f_q(ghost l)
      auto ghost_lam = [&](int q) -> T {
        const Cour<T> c = courant<T>(p, d, q, srow);
        if (c.up_r != outward) return T(0);
        const T* fp = sf + q * PLANE + row * kWinR;
        const T* lp = sl + q * PLANE + row * kWinR;
        T MDa, MPa, MDb, MPb;
        mwb_partials<T>(c.a_r, c.k_r, fp[ca] - fp[ca + outward], fp[ca + outward] - fp[ca + 2 * outward],
                        MDa, MPa);
        mwb_partials<T>(c.a_r, c.k_r, fp[cb] - fp[cb + outward], fp[cb + outward] - fp[cb + 2 * outward],
                        MDb, MPb);
        if (l == 0) return lp[ca] * (MDa - MPa) + lp[cb] * MPb;
        return lp[ca] * MPa;
      };
      eq_cotangent<T>(st[l][0], st[l][1], st[l][2], st[l][3], d, ghost_lam, Gl[l]);
    }
    // back through the extrapolation g0 = 2a - b, g1 = 3a - 2b (extrapolated components only)
    const bool ext_rho_E = kind != PCLB_BC_DIRICHLET;
    const bool ext_u = kind == PCLB_BC_EXTRAP;
    T Ga[4], Gb[4];
    for (int j = 0; j < 4; ++j) {
      const bool ext = (j == 0 || j == 3) ? ext_rho_E : ext_u;
      Ga[j] = ext ? T(2) * Gl[0][j] + T(3) * Gl[1][j] : T(0);
      Gb[j] = ext ? -Gl[0][j] - T(2) * Gl[1][j] : T(0);
    }
    T ga[4], gb[4];
    to_moment_cotangent<T>(a.rho, a.ux, a.uy, a.E, Ga, ga);
    to_moment_cotangent<T>(b.rho, b.ux, b.uy, b.E, Gb, gb);
    for (int j = 0; j < 4; ++j) {
      gw[((side * 2 + 0) * TT + rl) * 4 + j] = ga[j];
      gw[((side * 2 + 1) * TT + rl) * 4 + j] = gb[j];
    }
  };
  if (inner && rowl == 0 && lane < TT && t0 + lane < p.n_theta) wall_feedback(0, lane);
  if (outer && rowl == 1 && lane < TT && t0 + lane < p.n_theta) wall_feedback(1, lane);

  // ---- this thread's node: cotangent of its equilibrium ----------------------
  T g[4] = {T(0), T(0), T(0), T(0)};
  if (valid) {
    T G[4];
    eq_cotangent<T>(n_rho, n_ux, n_uy, n_E, d, [&](int q) -> T { return sl[q * PLANE + row * kWinR + col]; }, G);
    to_moment_cotangent<T>(n_rho, n_ux, n_uy, n_E, G, g);
  }
  __syncthreads();   // wall feedback ready
  // gs = (1 - d) g + g_wall: every label receives psi_q . gs
  const T decay = (T)p.decay;
  T gs[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    T w = T(0);
    if (inner && r == 0) w += gw[((0 * 2 + 0) * TT + rowl) * 4 + j];
    if (inner && r == 1) w += gw[((0 * 2 + 1) * TT + rowl) * 4 + j];
    if (outer && r == p.n_r - 1) w += gw[((1 * 2 + 0) * TT + rowl) * 4 + j];
    if (outer && r == p.n_r - 2) w += gw[((1 * 2 + 1) * TT + rowl) * 4 + j];
    gs[j] = (T(1) - decay) * g[j] + w;
  }

  const size_t plane_out = (size_t)p.rows * p.pitch;
  const int win = row * kWinR + col;
  auto store = [&](int q, T v) {
    lam_out[(size_t)q * plane_out + (size_t)srow * p.pitch + r] = v;
    if (t >= p.n_theta - 2)
      lam_out[(size_t)d.recv_lo[q] * plane_out + (size_t)(t - (p.n_theta - 2)) * p.pitch + r] = v;
    if (t < 2) lam_out[(size_t)d.recv_hi[q] * plane_out + (size_t)(p.n_theta + kGhostRows + t) * p.pitch + r] = v;
  };
  // rest velocity: no convection
  if (valid) store(0, decay * sl[win] + gs[0] + gs[3] * d.half_v2[0]);

  constexpr int NP = AdjSize<T>::npairs, RC = AdjSize<T>::rcols, PROD = AdjSize<T>::prod;
  // offsets inside one label's products
  constexpr int AR = 0, BR = TT * RC, AT = 2 * TT * RC, BT = 2 * TT * RC + (TT + 4) * kTileR;
#pragma unroll 1
  for (int pair = 0; pair < NP; ++pair) {
    const int k = 1 + pair / (kNDirs / 2);
    const int q1 = 1 + (k - 1) * kNDirs + pair % (kNDirs / 2);
    const int q2 = q1 + kNDirs / 2;                      // opposite velocity
    T* pb = prod + (pair & 1) * 2 * PROD;                // this pair's buffer: [label][products]

    // (A) products lam(n) M_D(n), lam(n) M_Dp(n) of every node that can reach the
    // tile.  Warp w forms those of tile row w at its 32 columns (both labels),
    // lanes 0..3 the two halo columns of each label on its upwind side, and
    // warps 0..3 the halo rows -2, -1, TT, TT + 1 for the label whose upwind
    // side points into the tile.
    {
      const CourEntry<T> e = ctab[row * NP + pair];
      auto radial = [&](int L, int uL, int c) {
        const int o = row * kWinR + c + kLeft;
        const T* fw = sf + (L ? q2 : q1) * PLANE + o;
        T MD, MP;
        mwb_partials<T>(e.a_r, e.k_r, fw[0] - fw[uL], fw[uL] - fw[2 * uL], MD, MP);
        const T lam = sl[(L ? q2 : q1) * PLANE + o];
        pb[L * PROD + AR + rowl * RC + c + 2] = lam * MD;
        pb[L * PROD + BR + rowl * RC + c + 2] = lam * MP;
      };
      auto azimuthal = [&](int L, int uL, int rr, T at, T kt) {
        const int o = rr * kWinR + lane + kLeft;
        const T* fw = sf + (L ? q2 : q1) * PLANE + o;
        T MD, MP;
        mwb_partials<T>(at, kt, fw[0] - fw[uL * kWinR], fw[uL * kWinR] - fw[2 * uL * kWinR], MD, MP);
        const T lam = sl[(L ? q2 : q1) * PLANE + o];
        pb[L * PROD + AT + rr * kTileR + lane] = lam * MD;
        pb[L * PROD + BT + rr * kTileR + lane] = lam * MP;
      };
      const int u = (e.fl & 1) ? 1 : -1;                 // radial upwind offset of q1 in this row
      const int un = (e.fl & 2) ? 1 : -1;                // azimuthal upwind offset of q1 in this row
      radial(0, u, lane);
      radial(1, -u, lane);
      const T at = e.a_w * invr[lane], kt = at - at * at;
      azimuthal(0, un, row, at, kt);
      azimuthal(1, -un, row, at, kt);
      if (rowl < 4) {
        // halo rows: warps 0..3 take window rows 0, 1, TT + 2, TT + 3
        const int rr = rowl < 2 ? rowl : TT + rowl;
        const CourEntry<T> eh = ctab[rr * NP + pair];
        const int unh = (eh.fl & 2) ? 1 : -1;
        const int need = rr < 2 ? 1 : -1;
        const T ath = eh.a_w * invr[lane], kth = ath - ath * ath;
        azimuthal(unh == need ? 0 : 1, need, rr, ath, kth);
      }
      // halo columns: 4 per tile row (label, column); the warps after the first
      // four take them, or warp 0 as well when the tile has too few rows.
      // Upwind at larger r (+1) reads the tile from columns -2, -1, at
      // smaller r from 32, 33.
      constexpr int HW = (4 * TT + 31) / 32;
      constexpr bool kSep = TT >= 4 + HW;
      if (kSep ? (rowl >= 4 && rowl < 4 + HW) : rowl < HW) {
        const int h = (kSep ? rowl - 4 : rowl) * 32 + lane;
        if (h < 4 * TT) {
          const int hr = h >> 2, L = (h >> 1) & 1, j = h & 1;
          const CourEntry<T> eh = ctab[(hr + 2) * NP + pair];
          const int uh = (eh.fl & 1) ? 1 : -1, uL = L ? -uh : uh;
          const int c = uL == 1 ? j - 2 : kTileR + j;
          const int o = (hr + 2) * kWinR + c + kLeft;
          const T* fw = sf + (L ? q2 : q1) * PLANE + o;
          T MD, MP;
          mwb_partials<T>(eh.a_r, eh.k_r, fw[0] - fw[uL], fw[uL] - fw[2 * uL], MD, MP);
          const T lam = sl[(L ? q2 : q1) * PLANE + o];
          pb[L * PROD + AR + hr * RC + c + 2] = lam * MD;
          pb[L * PROD + BR + hr * RC + c + 2] = lam * MP;
        }
      }
    }
    __syncthreads();

    // (B) gather at this node: node n = c + j u_n reads f(n), f(n + u_n),
    // f(n + 2 u_n), so dM(n)/df(n) = M_D, dM(n)/df(n + u_n) = M_Dp - M_D,
    // dM(n)/df(n + 2 u_n) = -M_Dp.
    if (valid) {
      const CourEntry<T>* cr = ctab + rowl * NP + pair;  // rows rowl - 2 .. rowl + 2 at stride NP
      const int u = (cr[2 * NP].fl & 1) ? 1 : -1;
      int tneg = 0;                                       // bit o: row o - 2 has v_theta < 0 for q1
#pragma unroll
      for (int o = 0; o < 5; ++o) tneg |= ((cr[o * NP].fl >> 1) & 1) << o;
      const T A = gs[0] + gs[3] * d.half_v2[k];
      const T B = gs[1] * d.vx[q1] + gs[2] * d.vy[q1];
#pragma unroll
      for (int L = 0; L < 2; ++L) {
        const T* P = pb + L * PROD;
        const int uL = L ? -u : u;
        const int neg = L ? (tneg ^ 0x1f) : tneg;        // the partner has the opposite velocity
        const int cc = lane + 2;
        T acc = P[AR + rowl * RC + cc] - P[AR + rowl * RC + cc - uL] + P[BR + rowl * RC + cc - uL] -
                P[BR + rowl * RC + cc - 2 * uL];
        const int rr = rowl + 2;
        acc += P[AT + rr * kTileR + lane];
        if (neg & 2) acc += P[BT + (rr - 1) * kTileR + lane] - P[AT + (rr - 1) * kTileR + lane];
        if (!(neg & 8)) acc += P[BT + (rr + 1) * kTileR + lane] - P[AT + (rr + 1) * kTileR + lane];
        if (neg & 1) acc -= P[BT + (rr - 2) * kTileR + lane];
        if (!(neg & 16)) acc -= P[BT + (rr + 2) * kTileR + lane];
        const int q = L ? q2 : q1;
        store(q, decay * sl[q * PLANE + win] + (L ? A - B : A + B) - acc);
      }
    }
  }
}

template <class T>
cudaError_t launch_adjoint(const CUtensorMap* tmap_f, const CUtensorMap* tmap_l, T* lam_out, const StepParams& p,
                           const DvmConst<T>& d, cudaStream_t stream) {
  static bool configured = false;
  constexpr int smem = AdjSize<T>::smem;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(adjoint_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  constexpr int TT = AdjTile<T>::TT;
  dim3 grid((p.n_r + kTileR - 1) / kTileR, (p.n_theta + TT - 1) / TT);
  adjoint_kernel<T><<<grid, TT * 32, smem, stream>>>(*tmap_f, *tmap_l, lam_out, p, d);
  return cudaGetLastError();
}

template cudaError_t launch_adjoint<float>(const CUtensorMap*, const CUtensorMap*, float*, const StepParams&,
                                           const DvmConst<float>&, cudaStream_t);
template cudaError_t launch_adjoint<double>(const CUtensorMap*, const CUtensorMap*, double*, const StepParams&,
                                            const DvmConst<double>&, cudaStream_t);

}  // namespace pclb
