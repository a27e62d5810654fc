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

template <class T>
struct AdjSize {
  static constexpr int plane = kWinR * (AdjTile<T>::TT + 4);
  static constexpr int smem = 2 * kQ * plane * (int)sizeof(T) + 2 * 2 * AdjTile<T>::TT * 4 * (int)sizeof(T) + 128;
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

}  // namespace

template <class T>
__global__ void __launch_bounds__(AdjTile<T>::TT * 32, 1)
    adjoint_kernel(const __grid_constant__ CUtensorMap tmap_f, const __grid_constant__ CUtensorMap tmap_l,
                   T* __restrict__ lam_out, const StepParams p, const DvmConst<T> d) {
  constexpr int TT = AdjTile<T>::TT;
  constexpr int PLANE = AdjSize<T>::plane;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* sf = reinterpret_cast<T*>(smem_raw);
  T* sl = sf + kQ * PLANE;
  T* gw = sl + kQ * PLANE;                          // [side][node][TT][4]
  uint64_t* bar = reinterpret_cast<uint64_t*>(gw + 2 * 2 * TT * 4);

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
  T gwl[4] = {T(0), T(0), T(0), T(0)};
  if (valid) {
    for (int j = 0; j < 4; ++j) {
      if (inner && r == 0) gwl[j] += gw[((0 * 2 + 0) * TT + rowl) * 4 + j];
      if (inner && r == 1) gwl[j] += gw[((0 * 2 + 1) * TT + rowl) * 4 + j];
      if (outer && r == p.n_r - 1) gwl[j] += gw[((1 * 2 + 0) * TT + rowl) * 4 + j];
      if (outer && r == p.n_r - 2) gwl[j] += gw[((1 * 2 + 1) * TT + rowl) * 4 + j];
    }
  }
  if (!valid) return;

  const T decay = (T)p.decay;
  const T inv_r = (T)p.inv_r[r];
  const size_t plane_out = (size_t)p.rows * p.pitch;
#pragma unroll 1
  for (int q = 0; q < kQ; ++q) {
    const T* fp = sf + q * PLANE;
    const T* lp = sl + q * PLANE;
    const int k = d.shell[q];
    const T vx = d.vx[q], vy = d.vy[q], hq = d.half_v2[k];
    const T psi_g = g[0] + g[1] * vx + g[2] * vy + g[3] * hq;
    const T psi_w = gwl[0] + gwl[1] * vx + gwl[2] * vy + gwl[3] * hq;
    T out = decay * lp[row * kWinR + col] + (T(1) - decay) * psi_g + psi_w;
    if (q != 0) {
      // radial gather: nodes n = c, c - u, c - 2u of this row (same Courant numbers)
      const Cour<T> cr = courant<T>(p, d, q, srow);
      const int u = cr.up_r;
      const T* fr = fp + row * kWinR;
      const T* lr = lp + row * kWinR;
      T MD0, MP0, MD1, MP1, MD2, MP2;
      mwb_partials<T>(cr.a_r, cr.k_r, fr[col] - fr[col + u], fr[col + u] - fr[col + 2 * u], MD0, MP0);
      mwb_partials<T>(cr.a_r, cr.k_r, fr[col - u] - fr[col], fr[col] - fr[col + u], MD1, MP1);
      mwb_partials<T>(cr.a_r, cr.k_r, fr[col - 2 * u] - fr[col - u], fr[col - u] - fr[col], MD2, MP2);
      out -= lr[col] * MD0 + lr[col - u] * (MP1 - MD1) - lr[col - 2 * u] * MP2;
      // azimuthal gather: each neighbour row n has its own upwind side
      const T* fc = fp + col;
      const T* lc = lp + col;
      {
        const int un = cr.up_t;
        const T at = cr.a_w * inv_r, kt = at - at * at;
        T MD, MP;
        mwb_partials<T>(at, kt, fc[row * kWinR] - fc[(row + un) * kWinR],
                        fc[(row + un) * kWinR] - fc[(row + 2 * un) * kWinR], MD, MP);
        out -= lc[row * kWinR] * MD;
      }
#pragma unroll
      for (int o = -2; o <= 2; ++o) {
        if (o == 0) continue;
        const int n = row + o;
        const Cour<T> cn = courant<T>(p, d, q, srow + o);
        const int un = cn.up_t;
        // this node is the first (o = -un) or second (o = -2 un) upwind neighbour of n
        if (o != -un && o != -2 * un) continue;
        const T at = cn.a_w * inv_r, kt = at - at * at;
        T MD, MP;
        mwb_partials<T>(at, kt, fc[n * kWinR] - fc[(n + un) * kWinR],
                        fc[(n + un) * kWinR] - fc[(n + 2 * un) * kWinR], MD, MP);
        if (o == -un)
          out -= lc[n * kWinR] * (MP - MD);
        else
          out += lc[n * kWinR] * MP;
      }
    }
    T* dst = lam_out + (size_t)q * plane_out + r;
    dst[(size_t)srow * p.pitch] = out;
    if (t >= p.n_theta - 2)
      lam_out[(size_t)d.recv_lo[q] * plane_out + (size_t)(t - (p.n_theta - 2)) * p.pitch + r] = out;
    if (t < 2) lam_out[(size_t)d.recv_hi[q] * plane_out + (size_t)(p.n_theta + kGhostRows + t) * p.pitch + r] = out;
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
