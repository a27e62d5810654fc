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
// in shared memory by TMA.
#include <cuda.h>
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "adjoint_common.cuh"
#include "ghost_cols.cuh"
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
  static constexpr int win_bytes = 2 * kQ * plane * (int)sizeof(T);
  static constexpr int gw_bytes = 2 * 2 * TT * 4 * (int)sizeof(T);
  static constexpr int tab_bytes = (TT + 4) * npairs * (int)sizeof(CourEntry<T>);
  static constexpr int smem = win_bytes + gw_bytes + tab_bytes + 128;
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

// Sum over the nodes n whose MWB increments (Eq. 28) in r and theta read
// f_q(c) of lam_q(n) dM_q(n)/df_q(c), for one label at this node c.  f and l
// point at c in the label's f and lam windows; ur is the radial upwind offset
// (+-1 column); at[o], kt[o] are a = |C_theta| and K = a(1 - a) of the theta
// rows o - 2 (o = 0..4) at this radius, and bit o of vt_neg is set when row
// o - 2 takes its upwind neighbour at the next row (v_theta < 0).  The node
// n = c + j u_n reads f(n), f(n + u_n), f(n + 2 u_n) with D = f(n) - f(n + u_n),
// Dp = f(n + u_n) - f(n + 2 u_n), so
//   dM(n)/df(n) = M_D,  dM(n)/df(n + u_n) = M_Dp - M_D,  dM(n)/df(n + 2 u_n) = -M_Dp.
template <class T>
__device__ __forceinline__ T adjoint_stencil(const T* f, const T* l, int ur, T ar, T kr, const T* at, const T* kt,
                                             int vt_neg) {
  const T f0 = f[0];
  // radial: the nodes c, c - u, c - 2u
  const T fm2 = f[-2 * ur], fm1 = f[-ur], fp1 = f[ur], fp2 = f[2 * ur];
  const T dm2 = fm2 - fm1, dm1 = fm1 - f0, d0 = f0 - fp1, d1 = fp1 - fp2;
  T MD0, MP0, MD1, MP1, MD2, MP2;
  mwb_partials<T>(ar, kr, d0, d1, MD0, MP0);
  mwb_partials<T>(ar, kr, dm1, d0, MD1, MP1);
  mwb_partials<T>(ar, kr, dm2, dm1, MD2, MP2);
  T acc = l[0] * MD0 + l[-ur] * (MP1 - MD1) - l[-2 * ur] * MP2;
  // azimuthal: rows -2..2 of this column, e_j = f(row j) - f(row j + 1)
  constexpr int S = kWinR;
  const T gm2 = f[-2 * S], gm1 = f[-S], gp1 = f[S], gp2 = f[2 * S];
  const T em2 = gm2 - gm1, em1 = gm1 - f0, e0 = f0 - gp1, e1 = gp1 - gp2;
  T MD, MP;
  if (vt_neg & 4)
    mwb_partials<T>(at[2], kt[2], e0, e1, MD, MP);     // this node, upwind at row +1
  else
    mwb_partials<T>(at[2], kt[2], em1, em2, MD, MP);   // upwind at row -1 (signs flipped)
  acc += l[0] * MD;
  if (vt_neg & 2) {          // row -1 reads this node as its first upwind neighbour
    mwb_partials<T>(at[1], kt[1], em1, e0, MD, MP);
    acc += l[-S] * (MP - MD);
  }
  if (!(vt_neg & 8)) {       // row +1, likewise
    mwb_partials<T>(at[3], kt[3], e0, em1, MD, MP);
    acc += l[S] * (MP - MD);
  }
  if (vt_neg & 1) {          // row -2 reads this node as its second upwind neighbour
    mwb_partials<T>(at[0], kt[0], em2, em1, MD, MP);
    acc -= l[-2 * S] * MP;
  }
  if (!(vt_neg & 16)) {      // row +2, likewise
    mwb_partials<T>(at[4], kt[4], e1, e0, MD, MP);
    acc -= l[2 * S] * MP;
  }
  return acc;
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
  T* gw = sl + kQ * PLANE;                          // [side][node][TT][4]
  CourEntry<T>* ctab = reinterpret_cast<CourEntry<T>*>(gw + 2 * 2 * TT * 4);   // [TT + 4][npairs]
  uint64_t* bar = reinterpret_cast<uint64_t*>(ctab + (TT + 4) * AdjSize<T>::npairs);

  const int r0 = blockIdx.x * kTileR;
  const int t0 = blockIdx.y * TT;
  const int tid = threadIdx.x;
  const int lane = tid & 31, rowl = tid >> 5;

  if (tid == 0) {
    tma_prefetch_desc(&tmap_f);
    tma_prefetch_desc(&tmap_l);
    mbar_init(bar, 1);
    mbar_fence_init();
  }
  for (int i = tid; i < 2 * 2 * TT * 4; i += blockDim.x) gw[i] = T(0);
  // Courant entries of the stored rows t0 .. t0 + TT + 3 (theta rows t0 - 2 .. t0 + TT + 1)
  for (int i = tid; i < (TT + 4) * AdjSize<T>::npairs; i += blockDim.x) {
    const int srow = t0 + i / AdjSize<T>::npairs, pair = i % AdjSize<T>::npairs;
    CourEntry<T> e{T(0), T(0), T(0), 0};
    if (srow < p.rows) courant_entry(p, srow, pair, e.a_r, e.k_r, e.a_w, e.fl);
    ctab[i] = e;
  }
  __syncthreads();
  if (tid == 0) {
    mbar_arrive_expect_tx(bar, (uint32_t)(2 * kQ * PLANE * sizeof(T)));
#pragma unroll 1
    for (int q = 0; q < kQ; ++q) {
      tma_load_3d(sf + q * PLANE, &tmap_f, r0 - kLeft, t0, q, bar);
      tma_load_3d(sl + q * PLANE, &tmap_l, r0 - kLeft, t0, q, bar);
    }
  }
  if (!mbar_wait_bounded(bar, 0, kAdjWaitNs)) {
    if (tid == 0) atomicOr(p.status, PCLB_FLAG_TIMEOUT);
    mbar_wait_bounded(bar, 0, kAdjWaitNs);
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
    const int kind = p.bc_kind[side];
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

  // ---- this thread's node ----------------------------------------------------
  const int row = 2 + rowl;
  const int col = kLeft + lane;
  const int t = t0 + rowl;
  const int r = r0 + lane;
  const bool valid = r < p.n_r && t < p.n_theta;
  const int srow = t + kGhostRows;

  T g[4] = {T(0), T(0), T(0), T(0)};
  if (valid) {
    const NodeState<T> m = node_moments(sf + row * kWinR + col, PLANE, d);
    if (!m.ok) atomicOr(p.status, PCLB_FLAG_NONPHYS);
    T G[4];
    eq_cotangent<T>(m.rho, m.ux, m.uy, m.E, d,
                    [&](int q) -> T { return sl[q * PLANE + row * kWinR + col]; }, G);
    to_moment_cotangent<T>(m.rho, m.ux, m.uy, m.E, G, g);
  }
  __syncthreads();   // wall feedback ready
  if (!valid) return;
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

  const T inv_r = (T)p.inv_r[r];
  const size_t plane_out = (size_t)p.rows * p.pitch;
  const int win = row * kWinR + col;
  auto store = [&](int q, T v) {
    lam_out[(size_t)q * plane_out + (size_t)srow * p.pitch + r] = v;
    if (t >= p.n_theta - 2)
      lam_out[(size_t)d.recv_lo[q] * plane_out + (size_t)(t - (p.n_theta - 2)) * p.pitch + r] = v;
    if (t < 2) lam_out[(size_t)d.recv_hi[q] * plane_out + (size_t)(p.n_theta + kGhostRows + t) * p.pitch + r] = v;
  };
  // rest velocity: no convection
  store(0, decay * sl[win] + gs[0] + gs[3] * d.half_v2[0]);

  const CourEntry<T>* crow = ctab + rowl * AdjSize<T>::npairs;   // stored row srow - 2
#pragma unroll 1
  for (int pair = 0; pair < AdjSize<T>::npairs; ++pair) {
    const int k = 1 + pair / (kNDirs / 2);
    const int q = 1 + (k - 1) * kNDirs + pair % (kNDirs / 2);
    const int q2 = q + kNDirs / 2;                       // opposite velocity
    // theta Courant numbers of the five rows o = -2..2 at this radius; flag
    // bits of the first label (the second has the opposite signs)
    T at[5], kt[5];
    int vt_neg = 0;
#pragma unroll
    for (int o = 0; o < 5; ++o) {
      const CourEntry<T> e = crow[o * AdjSize<T>::npairs + pair];
      at[o] = e.a_w * inv_r;
      kt[o] = at[o] - at[o] * at[o];
      vt_neg |= ((e.fl >> 1) & 1) << o;
    }
    const CourEntry<T> e0 = crow[2 * AdjSize<T>::npairs + pair];
    const int ur = (e0.fl & 1) ? 1 : -1;          // radial upwind offset of the first label
    const T A = gs[0] + gs[3] * d.half_v2[k];
    const T B = gs[1] * d.vx[q] + gs[2] * d.vy[q];
    const T* f1 = sf + q * PLANE + win;
    const T* l1 = sl + q * PLANE + win;
    const T* f2 = sf + q2 * PLANE + win;
    const T* l2 = sl + q2 * PLANE + win;
    const T c1 = adjoint_stencil<T>(f1, l1, ur, e0.a_r, e0.k_r, at, kt, vt_neg);
    const T c2 = adjoint_stencil<T>(f2, l2, -ur, e0.a_r, e0.k_r, at, kt, vt_neg ^ 0x1f);
    store(q, decay * l1[0] + A + B - c1);
    store(q2, decay * l2[0] + A - B - c2);
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
