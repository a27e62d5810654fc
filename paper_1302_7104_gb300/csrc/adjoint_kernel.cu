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
// Two kernels:
//   * adjoint_wall_kernel, one warp per wall and row: the ghost states
//     (Eq. 39 or prescribed) and the cotangent g_wall they return, written to
//     small global buffers;
//   * adjoint_pair_kernel, tiles of 32 (r) x TT (theta) nodes, one node per
//     thread.  Each thread first forms g of its node from f^n and lam^{n+1}
//     read from global memory (a reduction over the 33 labels).  Then the
//     velocities, in pairs of opposite labels, stream their f and lam windows
//     over [r0-4, r0+36) x [t0-2, t0+TT+2) through a ring of shared-memory
//     stages filled by TMA while earlier pairs compute.  Each pair runs in two
//     phases: (A) every node whose upwind stencil can reach the tile forms
//     lam(n) dM(n)/dD and lam(n) dM(n)/dDp once, in r and in theta; (B) every
//     tile node gathers the products of the nodes that read it and adds
//     d lam + psi . ((1-d) g + g_wall).  One barrier per pair separates the
//     phases; a stage is refilled as soon as its pair's phase (A) is done.
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
struct AdjTile<double> {
  static constexpr int TT = kAdjRows64;
  static constexpr int min_blocks = 3;   // at most 85 registers
};

// Courant entry of one pair of opposite velocities at one theta row:
// (|C_r|, |C_r|(1 - |C_r|), |v_theta| dt / dtheta, flags) with flag bit 0 set
// when v_r < 0 and bit 1 when v_theta < 0 for the first label of the pair.
template <class T>
struct alignas(4 * sizeof(T)) CourEntry {
  T a_r, k_r, a_w;
  int fl;
};

constexpr int kAdjStages = 2;   // ring depth of the pair-streaming kernel (2 measured best of 1..4)
static_assert(sizeof(EqParams<float>) == 10 * sizeof(float) && sizeof(EqParams<double>) == 10 * sizeof(double),
              "ghost-state scratch holds 10 values per EqParams");

template <class T>
struct AdjSize {
  static constexpr int TT = AdjTile<T>::TT;
  static constexpr int threads = 32 * TT;
  static constexpr int plane = kWinR * (TT + 4);
  static constexpr int npairs = 4 * kNDirs / 2;
  // products of one label: radial A, B over TT rows x 36 columns (tile
  // columns -2 .. 33), azimuthal A, B over TT + 4 rows (-2 .. TT + 1) x 32
  static constexpr int rcols = kTileR + 4;
  static constexpr int prod = 2 * TT * rcols + 2 * (TT + 4) * kTileR;
  static constexpr int ring_bytes = kAdjStages * 4 * plane * (int)sizeof(T);   // f, f', lam, lam' per stage
  static constexpr int prod_bytes = 2 * 2 * prod * (int)sizeof(T);             // 2 buffers x 2 labels
  static constexpr int invr_bytes = kTileR * (int)sizeof(T);
  static constexpr int tab_bytes = (TT + 4) * npairs * (int)sizeof(CourEntry<T>);
  static constexpr int smem = ring_bytes + prod_bytes + invr_bytes + tab_bytes + 128;
  // the ring's planes are TMA destinations: 128-byte aligned
  static_assert((plane * (int)sizeof(T)) % 128 == 0, "TMA destinations must stay 128-byte aligned");
};

namespace {


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

// (rho, u_x, u_y, E) of one node for the cotangent of the equilibrium (FP64;
// the FP32 pair kernel forms the state of its two nodes in float-float).
__device__ __forceinline__ void adj_node_state(const double* f, int plane, const DvmConst<double>& d, double& rho,
                                               double& ux, double& uy, double& E, bool& ok) {
  const NodeState<double> m = node_moments(f, plane, d);
  rho = m.rho; ux = m.ux; uy = m.uy; E = m.E; ok = m.ok;
}


// ---- the pair-streaming kernel's stencil pieces ------------------------------
// Products of both labels of a pair at one node in one direction: q1 has its
// upwind side at offset U, q2 (the opposite velocity) at -U.  sf, sl: the
// pair's f and lam planes (q2 at +PLANE); o: the node in a plane; pr: its
// product slot (M_D products; the M_Dp ones at +DB, q2's at +PROD).
template <class T, int U, int PLANE, int PROD, int DB>
__device__ __forceinline__ void radial_pair(const T* sf, const T* sl, T* pb, int o, int pr, T a, T K, T lam[2]) {
  T MD, MP;
  const T* f1 = sf + o;
  mwb_partials<T>(a, K, f1[0] - f1[U], f1[U] - f1[2 * U], MD, MP);
  lam[0] = sl[o];
  pb[pr] = lam[0] * MD;
  pb[pr + DB] = lam[0] * MP;
  const T* f2 = sf + PLANE + o;
  mwb_partials<T>(a, K, f2[0] - f2[-U], f2[-U] - f2[-2 * U], MD, MP);
  lam[1] = sl[PLANE + o];
  pb[PROD + pr] = lam[1] * MD;
  pb[PROD + pr + DB] = lam[1] * MP;
}

template <class T, int U, int PLANE, int PROD, int DB>
__device__ __forceinline__ void azimuthal_pair(const T* sf, const T lam[2], T* pb, int o, int pa, T a, T K) {
  T MD, MP;
  const T* f1 = sf + o;
  mwb_partials<T>(a, K, f1[0] - f1[U], f1[U] - f1[2 * U], MD, MP);
  pb[pa] = lam[0] * MD;
  pb[pa + DB] = lam[0] * MP;
  const T* f2 = sf + PLANE + o;
  mwb_partials<T>(a, K, f2[0] - f2[-U], f2[-U] - f2[-2 * U], MD, MP);
  pb[PROD + pa] = lam[1] * MD;
  pb[PROD + pa + DB] = lam[1] * MP;
}

// One label at one halo node, upwind side at offset U.
template <class T, int U>
__device__ __forceinline__ void azimuthal_one(const T* fw, const T* lw, T* pa, int DB, T a, T K) {
  T MD, MP;
  mwb_partials<T>(a, K, fw[0] - fw[U], fw[U] - fw[2 * U], MD, MP);
  const T lam = lw[0];
  pa[0] = lam * MD;
  pa[DB] = lam * MP;
}

// Gather of the radial products at one node: the node n = c + j u reads f(n),
// f(n + u), f(n + 2 u), so dM(n)/df(c) collects M_D of n = c, M_Dp - M_D of
// n = c - u and -M_Dp of n = c - 2u (u = U for q1, -U for q2).
template <class T, int U, int PROD, int DB>
__device__ __forceinline__ void gather_radial(const T* pb, int pr, T acc[2]) {
  acc[0] = pb[pr] - pb[pr - U] + pb[pr + DB - U] - pb[pr + DB - 2 * U];
  const T* p2 = pb + PROD;
  acc[1] = p2[pr] - p2[pr + U] + p2[pr + DB + U] - p2[pr + DB + 2 * U];
}

// Azimuthal gather when the rows -2 .. +2 around the node all have q1's
// upwind side on the same side: the readers of the node sit at +V, +2V for
// q1 and at -V, -2V for q2 (V = +-row stride).
template <class T, int V, int PROD, int DB>
__device__ __forceinline__ void gather_azimuthal(const T* pb, int pa, T acc[2]) {
  acc[0] += pb[pa] + pb[pa + DB + V] - pb[pa + V] - pb[pa + DB + 2 * V];
  const T* p2 = pb + PROD;
  acc[1] += p2[pa] + p2[pa + DB - V] - p2[pa - V] - p2[pa + DB - 2 * V];
}

// The same where the upwind side changes within the five rows: bit o of neg
// set when row o - 2 has v_theta < 0 for q1 (its reader of row 0 is then the
// row below it).
template <class T, int PROD, int DB>
__device__ __forceinline__ void gather_azimuthal_mixed(const T* pb, int pa, int tneg, T acc[2]) {
#pragma unroll
  for (int L = 0; L < 2; ++L) {
    const T* P = pb + L * PROD;
    const int neg = L ? (tneg ^ 0x1f) : tneg;          // the partner has the opposite velocity
    T a = P[pa];
    if (neg & 2) a += P[pa + DB - kTileR] - P[pa - kTileR];
    if (!(neg & 8)) a += P[pa + DB + kTileR] - P[pa + kTileR];
    if (neg & 1) a -= P[pa + DB - 2 * kTileR];
    if (!(neg & 16)) a -= P[pa + DB + 2 * kTileR];
    acc[L] += a;
  }
}

// f^eq_q of a node state (rho and E in double as the step evaluates them).
template <class T>
__device__ __forceinline__ T adj_feq(const EqParams<T>& e, const DvmConst<T>& d, int q) {
  return feq_q<T>(e, d.vx[q], d.vy[q], d.shell[q]);
}

}  // namespace

// ---------------------------------------------------------------------------
// Walls: one warp per side s (0 inner, 1 outer) and row t.  It forms the
// equilibrium parameters of the two ghost layers (Eq. 39, or the prescribed
// states) and the cotangent g_wall that the ghosts return to the wall node
// (node 0) and the next node inward (node 1); lanes 0..15 take one pair of
// opposite velocities each, a warp reduction sums them.
// ghost [side][layer][n_theta] EqParams; gwall [side][node][n_theta][4].
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(128)
    adjoint_wall_kernel(const T* __restrict__ f, const T* __restrict__ lam, EqParams<T>* __restrict__ ghost,
                        T* __restrict__ gwall, T* __restrict__ gdir, const __grid_constant__ StepParams p,
                        const __grid_constant__ DvmConst<T> d) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int side = warp & 1, t = warp >> 1;
  if (t >= p.n_theta) return;                          // uniform across the warp
  const int plane = p.rows * p.pitch;
  const int srow = t + kGhostRows;
  const int step = side == 0 ? 1 : -1;                // towards the interior
  const int out = -step;                              // the upwind offset that reads the ghosts
  const int ra = side == 0 ? 0 : p.n_r - 1;
  const T* fa = f + (size_t)srow * p.pitch + ra;
  const T* fb = fa + step;
  const T* la = lam + (size_t)srow * p.pitch + ra;
  const T* lb = la + step;
  const NodeState<T> a = node_moments(fa, plane, d);
  const NodeState<T> b = node_moments(fb, plane, d);
  const int kind = p.bc_kind[side] & ~PCLB_BC_NEQ;
  double grho[2], gE[2];
  T gux[2], guy[2];
  grho[0] = 2.0 * a.rho_d - b.rho_d;  grho[1] = 2.0 * grho[0] - a.rho_d;   // Eq. (39), applied twice
  gE[0] = 2.0 * a.E_d - b.E_d;        gE[1] = 2.0 * gE[0] - a.E_d;
  gux[0] = T(2) * a.ux - b.ux;        gux[1] = T(2) * gux[0] - a.ux;
  guy[0] = T(2) * a.uy - b.uy;        guy[1] = T(2) * guy[0] - a.uy;
  if (kind != PCLB_BC_EXTRAP) {
    const double c = p.cos_t[t], s = p.sin_t[t];
    for (int l = 0; l < 2; ++l) {
      const double* v = p.bc_vals + (size_t)((side * 2 + l) * 4) * p.n_theta + t;
      gux[l] = (T)(v[1 * p.n_theta] * c - v[2 * p.n_theta] * s);
      guy[l] = (T)(v[1 * p.n_theta] * s + v[2 * p.n_theta] * c);
      if (kind == PCLB_BC_DIRICHLET) {
        grho[l] = v[0];
        gE[l] = v[3 * p.n_theta];
      }
    }
  }
  const EqParams<T> e0 = eq_params<T>(grho[0], gux[0], guy[0], gE[0], d);
  const EqParams<T> e1 = eq_params<T>(grho[1], gux[1], guy[1], gE[1], d);
  const bool neq = (p.bc_kind[side] & PCLB_BC_NEQ) != 0;
  // non-equilibrium ghosts also carry the wall node's departure f_q(a) -
  // f^eq_q(a): its equilibrium parameters go to the third slot (zero for
  // other walls, whose pair kernels do not read it; neq is uniform across
  // the warp, which serves one side)
  EqParams<T> ea{};
  if (neq) ea = eq_params<T>(a.rho_d, a.ux, a.uy, a.E_d, d);
  if (lane == 0) {
    if (!(grho[0] > 0.0 && grho[1] > 0.0 && gE[0] > 0.0 && gE[1] > 0.0)) atomicOr(p.status, PCLB_FLAG_NONPHYS);
    ghost[(size_t)(side * 3 + 0) * p.n_theta + t] = e0;
    ghost[(size_t)(side * 3 + 1) * p.n_theta + t] = e1;
    ghost[(size_t)(side * 3 + 2) * p.n_theta + t] = ea;
    gdir[((size_t)side * p.n_theta + t) * kQ] = T(0);   // the rest velocity reads no ghost
  }
  // per layer: the sums A, Bx, By, Cs, Dx, Fq of eq_cotangent over this
  // lane's pair; layer 2: those at the wall node's own state for the
  // departure of non-equilibrium ghosts
  T c[3][6];
#pragma unroll
  for (int l = 0; l < 3; ++l)
#pragma unroll
    for (int j = 0; j < 6; ++j) c[l][j] = T(0);
  constexpr int half = kNDirs / 2;
  if (lane < 4 * half) {
    const int k = 1 + lane / half;
    const int q1 = 1 + (k - 1) * kNDirs + lane % half;
    // cotangent of the ghost values f_q(layer l) = -sum_n lam_q(n) dM_q(n)/df_q(ghost l):
    // the wall node a reads (a, g0, g1), the next node b reads (b, a, g0)
    T lg[2][2];                                        // [label][layer]
#pragma unroll
    for (int L = 0; L < 2; ++L) {
      const int q = q1 + L * half;
      const Cour<T> cr = courant<T>(p, d, q, srow);
      lg[L][0] = lg[L][1] = T(0);
      if (cr.up_r == out) {
        const T f_a = fa[(size_t)q * plane], f_b = fb[(size_t)q * plane];
        // the ghost values as the step forms them (plus the departure f_q(a)
        // - f^eq_q(a) for non-equilibrium ghosts)
        const T dep = neq ? f_a - adj_feq<T>(ea, d, q) : T(0);
        const T g0 = adj_feq<T>(e0, d, q) + dep, g1 = adj_feq<T>(e1, d, q) + dep;
        T MDa, MPa, MDb, MPb;
        mwb_partials<T>(cr.a_r, cr.k_r, f_a - g0, g0 - g1, MDa, MPa);
        mwb_partials<T>(cr.a_r, cr.k_r, f_b - f_a, f_a - g0, MDb, MPb);
        const T lam_a = la[(size_t)q * plane], lam_b = lb[(size_t)q * plane];
        lg[L][0] = lam_a * (MDa - MPa) + lam_b * MPb;
        lg[L][1] = lam_a * MPa;
      }
    }
    // the ghost values' cotangents flow, for non-equilibrium ghosts, straight
    // to f_q(a) (coefficient 1) and, with the opposite sign, through f^eq_q(a)
    gdir[((size_t)side * p.n_theta + t) * kQ + q1] = lg[0][0] + lg[0][1];
    gdir[((size_t)side * p.n_theta + t) * kQ + q1 + half] = lg[1][0] + lg[1][1];
    const T lneq[2] = {neq ? -(lg[0][0] + lg[0][1]) : T(0), neq ? -(lg[1][0] + lg[1][1]) : T(0)};
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      if (l == 2 && !neq) break;                      // the departure's terms: non-equilibrium ghosts only
      const T E = l < 2 ? (T)gE[l] : a.E, ux = l < 2 ? gux[l] : a.ux, uy = l < 2 ? guy[l] : a.uy;
      const T lp = l < 2 ? lg[0][l] : lneq[0], lm = l < 2 ? lg[1][l] : lneq[1];
      const T* cf = d.Fc[k];
      const T F = E * (cf[0] + E * (cf[1] + E * (cf[2] + E * cf[3])));
      const T Fd = cf[0] + E * (T(2) * cf[1] + E * (T(3) * cf[2] + E * T(4) * cf[3]));
      const T invE = recip1(E);
      const T s = (ux * ux + uy * uy) * invE;
      const T a1 = T(1) - T(0.5) * s;
      const T a0 = a1 + T(0.125) * s * s;
      T Ak = 0, Bxk = 0, Byk = 0, Ck = 0, Dk = 0;
      pair_terms<T>(d.vx[q1], d.vy[q1], ux * invE, uy * invE, s, a0, a1, lp, lm, Ak, Bxk, Byk, Ck, Dk);
      c[l][0] = F * Ak; c[l][1] = F * Bxk; c[l][2] = F * Byk; c[l][3] = F * Ck; c[l][4] = F * Dk; c[l][5] = Fd * Ak;
    }
  }
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    if (l == 2 && !neq) break;
#pragma unroll
    for (int j = 0; j < 6; ++j)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) c[l][j] += __shfl_xor_sync(0xffffffffu, c[l][j], o);
  }
  if (lane != 0) return;
  T Gl[3][4];
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    // G of eq_cotangent at the ghost state, and at the wall node's state for
    // the departure (the rest velocity returns nothing)
    if (l == 2 && !neq) {
      Gl[2][0] = Gl[2][1] = Gl[2][2] = Gl[2][3] = T(0);
      break;
    }
    const T rho = l < 2 ? (T)grho[l] : a.rho, E = l < 2 ? (T)gE[l] : a.E;
    const T ux = l < 2 ? gux[l] : a.ux, uy = l < 2 ? guy[l] : a.uy;
    const T invE = recip1(E);
    const T s = (ux * ux + uy * uy) * invE;
    Gl[l][0] = c[l][0];
    Gl[l][1] = rho * (c[l][1] + T(2) * ux * c[l][3]) * invE;
    Gl[l][2] = rho * (c[l][2] + T(2) * uy * c[l][3]) * invE;
    Gl[l][3] = rho * (c[l][5] - (c[l][4] + s * c[l][3]) * invE);
  }
  // back through the extrapolation g0 = 2a - b, g1 = 3a - 2b (extrapolated components only)
  const bool ext_rho_E = kind != PCLB_BC_DIRICHLET;
  const bool ext_u = kind == PCLB_BC_EXTRAP;
  T Ga[4], Gb[4];
  for (int j = 0; j < 4; ++j) {
    const bool ext = (j == 0 || j == 3) ? ext_rho_E : ext_u;
    Ga[j] = (ext ? T(2) * Gl[0][j] + T(3) * Gl[1][j] : T(0)) + (neq ? Gl[2][j] : T(0));
    Gb[j] = ext ? -Gl[0][j] - T(2) * Gl[1][j] : T(0);
  }
  T ga[4], gb[4];
  to_moment_cotangent<T>(a.rho, a.ux, a.uy, a.E, Ga, ga);
  to_moment_cotangent<T>(b.rho, b.ux, b.uy, b.E, Gb, gb);
  for (int j = 0; j < 4; ++j) {
    gwall[((size_t)(side * 2 + 0) * p.n_theta + t) * 4 + j] = ga[j];
    gwall[((size_t)(side * 2 + 1) * p.n_theta + t) * 4 + j] = gb[j];
  }
}

// ---------------------------------------------------------------------------
// Pair-streaming part.
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(AdjSize<T>::threads, AdjTile<T>::min_blocks)
    adjoint_pair_kernel(const __grid_constant__ CUtensorMap tmap_f, const __grid_constant__ CUtensorMap tmap_l,
                        const T* __restrict__ f, const T* __restrict__ lam_in, T* __restrict__ lam_out,
                        const EqParams<T>* __restrict__ ghost, const T* __restrict__ gwall,
                        const T* __restrict__ gdir, int a0, int na, int b0, const __grid_constant__ StepParams p,
                        const __grid_constant__ DvmConst<T> d) {
  constexpr int TT = AdjTile<T>::TT;
  constexpr int PLANE = AdjSize<T>::plane;
  constexpr int NP = AdjSize<T>::npairs, RC = AdjSize<T>::rcols, PROD = AdjSize<T>::prod;
  constexpr int S = kAdjStages;
  // offsets inside one label's products
  constexpr int AR = 0, BR = TT * RC, AT = 2 * TT * RC, BT = 2 * TT * RC + (TT + 4) * kTileR;
  constexpr uint32_t kStageBytes = (uint32_t)(4 * PLANE * sizeof(T));
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* ring = reinterpret_cast<T*>(smem_raw);                 // [stage][f q1, f q2, lam q1, lam q2][PLANE]
  T* prod = ring + S * 4 * PLANE;                             // [buffer][label][products]
  T* invr = prod + 2 * 2 * PROD;                              // 1/r of the tile columns
  CourEntry<T>* ctab = reinterpret_cast<CourEntry<T>*>(invr + kTileR);   // [TT + 4][NP]
  uint64_t* bar = reinterpret_cast<uint64_t*>(ctab + (TT + 4) * NP);     // [S]

  // radial tile: blocks 0 .. na - 1 take tiles a0 .., the rest tiles b0 ..
  const int tx = (int)blockIdx.x < na ? a0 + (int)blockIdx.x : b0 + (int)blockIdx.x - na;
  const int r0 = tx * kTileR;
  const int t0 = blockIdx.y * TT;
  const int tid = threadIdx.x;
  const int lane = tid & 31, rowl = tid >> 5;

  // the planes of pair pr (labels q1, q1 + N_i/2) into stage s (thread 0)
  auto issue_pair = [&](int pr, int s) {
    const int k = 1 + pr / (kNDirs / 2);
    const int q1 = 1 + (k - 1) * kNDirs + pr % (kNDirs / 2), q2 = q1 + kNDirs / 2;
    T* st = ring + s * 4 * PLANE;
    mbar_arrive_expect_tx(&bar[s], kStageBytes);
    tma_load_3d(st, &tmap_f, r0 - kLeft, t0, q1, &bar[s]);
    tma_load_3d(st + PLANE, &tmap_f, r0 - kLeft, t0, q2, &bar[s]);
    tma_load_3d(st + 2 * PLANE, &tmap_l, r0 - kLeft, t0, q1, &bar[s]);
    tma_load_3d(st + 3 * PLANE, &tmap_l, r0 - kLeft, t0, q2, &bar[s]);
  };
  if (tid == 0) {
    tma_prefetch_desc(&tmap_f);
    tma_prefetch_desc(&tmap_l);
    for (int s = 0; s < S; ++s) mbar_init(&bar[s], 1);
    mbar_fence_init();
  }
  if (tid < kTileR) invr[tid] = r0 + tid < p.n_r ? (T)p.inv_r[r0 + tid] : T(1);
  // Courant entries of the stored rows t0 .. t0 + TT + 3 (theta rows t0 - 2 .. t0 + TT + 1)
  for (int i = tid; i < (TT + 4) * NP; i += blockDim.x) {
    const int srow = t0 + i / NP, pr = i % NP;
    CourEntry<T> e{T(0), T(0), T(0), 0};
    if (srow < p.rows) courant_entry(p, srow, pr, e.a_r, e.k_r, e.a_w, e.fl);
    ctab[i] = e;
  }
  __syncthreads();
  // bits 2..6 of the tile rows' flags: bit 1 (v_theta < 0 for q1) of the rows
  // -2 .. +2 around them, the rows whose azimuthal stencils reach the node
  for (int i = tid; i < TT * NP; i += blockDim.x) {
    const int w = 2 + i / NP, pr = i % NP;
    int m = 0;
#pragma unroll
    for (int o = 0; o < 5; ++o) m |= ((ctab[(w - 2 + o) * NP + pr].fl >> 1) & 1) << o;
    ctab[w * NP + pr].fl |= m << 2;
  }
  __syncthreads();
  if (tid == 0)
    for (int s = 0; s < S && s < NP; ++s) issue_pair(s, s);

  // ---- this thread's node -----------------------------------------------------
  const int row = 2 + rowl;
  const int col = kLeft + lane;
  const int t = t0 + rowl;
  const int r = r0 + lane;
  const bool valid = r < p.n_r && t < p.n_theta;
  const int srow = t + kGhostRows;
  const size_t plane_out = (size_t)p.rows * p.pitch;
  const T decay = (T)p.decay;
  T gs[4] = {T(0), T(0), T(0), T(0)};
  if (valid) {
    // (1 - d) g of this node, read from global memory while the first pairs'
    // windows land (the TMA copies then mostly hit L2)
    const int plane = p.rows * p.pitch;
    const size_t off = (size_t)srow * p.pitch + r;
    const T* ln = lam_in + off;
    T rho, ux, uy, E;
    bool nok;
    adj_node_state(f + off, plane, d, rho, ux, uy, E, nok);
    if (!nok) atomicOr(p.status, PCLB_FLAG_NONPHYS);
    T G[4], g[4];
    eq_cotangent<T>(rho, ux, uy, E, d, [&](int q) -> T { return ln[(size_t)q * plane]; }, G);
    to_moment_cotangent<T>(rho, ux, uy, E, G, g);
#pragma unroll
    for (int j = 0; j < 4; ++j) gs[j] = (T(1) - decay) * g[j];
    // the cotangent the ghost nodes return to the two nodes next to each wall
    auto add_wall = [&](int side, int node) {
#pragma unroll
      for (int j = 0; j < 4; ++j) gs[j] += gwall[((size_t)(side * 2 + node) * p.n_theta + t) * 4 + j];
    };
    if (r == 0) add_wall(0, 0);
    if (r == 1) add_wall(0, 1);
    if (r == p.n_r - 1) add_wall(1, 0);
    if (r == p.n_r - 2) add_wall(1, 1);
  }
  const int o_node = row * kWinR + col;                 // this node in a window plane
  const int p_rad = AR + rowl * RC + lane + 2;          // its radial product slot
  const int p_az = AT + row * kTileR + lane;            // its azimuthal product slot
  const T my_invr = invr[lane];
  auto store = [&](int q, T v) {
    lam_out[(size_t)q * plane_out + (size_t)srow * p.pitch + r] = v;
    if (t >= p.n_theta - 2)
      lam_out[(size_t)d.recv_lo[q] * plane_out + (size_t)(t - (p.n_theta - 2)) * p.pitch + r] = v;
    if (t < 2) lam_out[(size_t)d.recv_hi[q] * plane_out + (size_t)(p.n_theta + kGhostRows + t) * p.pitch + r] = v;
  };
  // rest velocity: no convection
  if (valid) store(0, decay * lam_in[(size_t)srow * p.pitch + r] + gs[0] + gs[3] * d.half_v2[0]);

  // wall tiles: the ghost states of the rows this thread fills (warp 0: inner, warp 1: outer)
  const int cw_out = p.n_r - 1 - r0 + kLeft;
  const bool inner = r0 == 0, outer = cw_out <= kLeft + kTileR;
  const bool wall_tile = inner || outer;
  const int gside = rowl == 0 ? 0 : 1;
  const bool fills = wall_tile && rowl < 2 && lane < TT && t0 + lane < p.n_theta && (gside == 0 ? inner : outer);
  const EqParams<T>* eg = ghost + (size_t)(gside * 3) * p.n_theta + t0 + lane;   // layer l at + l n_theta
  const bool gneq = (p.bc_kind[gside] & PCLB_BC_NEQ) != 0;   // its ghosts carry the wall node's departure

  bool ok = true;
  int brk = NP;                                         // the pair at which a wait timed out
#pragma unroll 1
  for (int pair = 0; pair < NP; ++pair) {
    const int k = 1 + pair / (kNDirs / 2);
    const int q1 = 1 + (k - 1) * kNDirs + pair % (kNDirs / 2);
    const int q2 = q1 + kNDirs / 2;                      // opposite velocity
    const int s = pair % S;
    const T* st = ring + s * 4 * PLANE;
    T* pb = prod + (pair & 1) * 2 * PROD;                // this pair's products: [label][...]
    if (ok) ok = p.wait_ns != 0 && mbar_wait_bounded(&bar[s], (uint32_t)((pair / S) & 1), p.wait_ns);
    if (wall_tile) {
      // radial ghost columns of this pair's f planes (f = f^eq of the ghost
      // states, plus the wall node's departure for non-equilibrium ghosts)
      if (fills && ok) {
        T* fw = const_cast<T*>(st) + (2 + lane) * kWinR;
        const int c0 = gside == 0 ? kLeft : cw_out, stp = gside == 0 ? 1 : -1;
        T dep1 = T(0), dep2 = T(0);
        if (gneq) {
          const EqParams<T> ea = eg[(size_t)2 * p.n_theta];
          dep1 = fw[c0] - adj_feq<T>(ea, d, q1);
          dep2 = fw[PLANE + c0] - adj_feq<T>(ea, d, q2);
        }
        for (int l = 0; l < 2; ++l) {
          const int c = c0 - stp * (1 + l);
          if (c < 0 || c >= kWinR) continue;
          const EqParams<T> e = eg[(size_t)l * p.n_theta];
          fw[c] = adj_feq<T>(e, d, q1) + dep1;
          fw[PLANE + c] = adj_feq<T>(e, d, q2) + dep2;
        }
      }
      __syncthreads();
    }

    // (A) products lam(n) M_D(n), lam(n) M_Dp(n) of every node that can reach the
    // tile.  Warp w forms those of tile row w at its 32 columns (both labels),
    // warps 0..3 the halo rows -2, -1, TT, TT + 1 for the label whose upwind
    // side points into the tile, and the next warps the halo columns.  The
    // upwind sides are uniform across a warp (one row), so each warp takes a
    // branch in which the stencil offsets are constants.
    const T* sfp = st;                                    // f q1, f q2 at +PLANE
    const T* slp = st + 2 * PLANE;                        // lam q1, lam q2 at +PLANE
    const CourEntry<T> e = ctab[row * NP + pair];
    const int fl_c = e.fl;                                // flags of this node's row
    T lam_c[2];                                           // lam^{n+1} of both labels at this node
    if (fl_c & 1)
      radial_pair<T, 1, PLANE, PROD, BR - AR>(sfp, slp, pb, o_node, p_rad, e.a_r, e.k_r, lam_c);
    else
      radial_pair<T, -1, PLANE, PROD, BR - AR>(sfp, slp, pb, o_node, p_rad, e.a_r, e.k_r, lam_c);
    {
      const T at = e.a_w * my_invr, kt = at - at * at;
      if (fl_c & 2)
        azimuthal_pair<T, kWinR, PLANE, PROD, BT - AT>(sfp, lam_c, pb, o_node, p_az, at, kt);
      else
        azimuthal_pair<T, -kWinR, PLANE, PROD, BT - AT>(sfp, lam_c, pb, o_node, p_az, at, kt);
    }
    if (rowl < 4) {
      // halo rows: warps 0..3 take window rows 0, 1, TT + 2, TT + 3; rows
      // above the tile are read by labels whose upwind side is +theta
      const int rr = rowl < 2 ? rowl : TT + rowl;
      const CourEntry<T> eh = ctab[rr * NP + pair];
      const bool q1_up_pos = (eh.fl & 2) != 0;
      const T ath = eh.a_w * my_invr, kth = ath - ath * ath;
      const int o = rr * kWinR + col;
      if (rowl < 2)
        azimuthal_one<T, kWinR>(sfp + (q1_up_pos ? 0 : PLANE) + o, slp + (q1_up_pos ? 0 : PLANE) + o,
                                pb + (q1_up_pos ? 0 : PROD) + AT + rr * kTileR + lane, BT - AT, ath, kth);
      else
        azimuthal_one<T, -kWinR>(sfp + (q1_up_pos ? PLANE : 0) + o, slp + (q1_up_pos ? PLANE : 0) + o,
                                 pb + (q1_up_pos ? PROD : 0) + AT + rr * kTileR + lane, BT - AT, ath, kth);
    }
    {
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
          const T* fw = sfp + L * PLANE + o;
          T MD, MP;
          mwb_partials<T>(eh.a_r, eh.k_r, fw[0] - fw[uL], fw[uL] - fw[2 * uL], MD, MP);
          const T lam = slp[L * PLANE + o];
          pb[L * PROD + AR + hr * RC + c + 2] = lam * MD;
          pb[L * PROD + BR + hr * RC + c + 2] = lam * MP;
        }
      }
    }
    if (__syncthreads_or(!ok)) {
      brk = pair;
      break;
    }
    // the stage of this pair is free: the planes of pair + S start now
    if (tid == 0 && pair + S < NP) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue_pair(pair + S, s);
    }

    // (B) gather at this node: node n = c + j u_n reads f(n), f(n + u_n),
    // f(n + 2 u_n), so dM(n)/df(n) = M_D, dM(n)/df(n + u_n) = M_Dp - M_D,
    // dM(n)/df(n + 2 u_n) = -M_Dp.
    if (valid) {
      T acc[2];
      if (fl_c & 1)
        gather_radial<T, 1, PROD, BR - AR>(pb, p_rad, acc);
      else
        gather_radial<T, -1, PROD, BR - AR>(pb, p_rad, acc);
      const int tneg = fl_c >> 2;                        // bit o: row o - 2 has v_theta < 0 for q1
      if (tneg == 0)
        gather_azimuthal<T, kTileR, PROD, BT - AT>(pb, p_az, acc);
      else if (tneg == 31)
        gather_azimuthal<T, -kTileR, PROD, BT - AT>(pb, p_az, acc);
      else
        gather_azimuthal_mixed<T, PROD, BT - AT>(pb, p_az, tneg, acc);
      const T A = gs[0] + gs[3] * d.half_v2[k];
      const T B = gs[1] * d.vx[q1] + gs[2] * d.vy[q1];
      T o1 = decay * lam_c[0] + (A + B) - acc[0], o2 = decay * lam_c[1] + (A - B) - acc[1];
      if (wall_tile) {
        // non-equilibrium ghosts hand their cotangent straight to f_q of the wall node
        for (int sd = 0; sd < 2; ++sd)
          if ((p.bc_kind[sd] & PCLB_BC_NEQ) && r == (sd == 0 ? 0 : p.n_r - 1)) {
            o1 += gdir[((size_t)sd * p.n_theta + t) * kQ + q1];
            o2 += gdir[((size_t)sd * p.n_theta + t) * kQ + q2];
          }
      }
      store(q1, o1);
      store(q2, o2);
    }
  }
  if (brk < NP && tid == 0) {
    // a copy did not land in time: report it, give the copies still in
    // flight (the last one issued into each stage) a bounded time to finish
    atomicOr(p.status, PCLB_FLAG_TIMEOUT);
    const int issued = brk + S < NP ? brk + S : NP;
    for (int s = 0; s < S && s < issued; ++s) {
      const int last = s + ((issued - 1 - s) / S) * S;
      mbar_wait_bounded(&bar[s], (uint32_t)((last / S) & 1), kDefaultWaitNs);
    }
  }
}

// The tiles that read the wall kernel's output (ghost columns, g_wall) are
// tile 0 and the tiles with r0 >= n_r - 33; they run on the side stream after
// the wall kernel while the interior tiles run on the main stream.
template <class T>
cudaError_t launch_adjoint(const CUtensorMap* tmap_f, const CUtensorMap* tmap_l, const CUtensorMap* tmap_fn,
                           const CUtensorMap* tmap_ln, const T* f, const T* lam_in,
                           T* lam_out, const AdjScratch& ws, const StepParams& p, const DvmConst<T>& d,
                           cudaStream_t stream, cudaStream_t side, cudaEvent_t ev_fork, cudaEvent_t ev_join) {
  EqParams<T>* ghost = reinterpret_cast<EqParams<T>*>(ws.ghost);
  T* gwall = reinterpret_cast<T*>(ws.gwall);
  const int nt = (p.n_r + kTileR - 1) / kTileR;
  const int t_hi = p.n_r - 33 > 0 ? (p.n_r - 33 + kTileR - 1) / kTileR : 0;   // first tile with r0 >= n_r - 33
  const int b0 = t_hi > 1 ? t_hi : 1;
  const int n_interior = t_hi > 1 ? t_hi - 1 : 0;                              // tiles 1 .. t_hi - 1
  cudaError_t e = cudaEventRecord(ev_fork, stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(side, ev_fork, 0);
  if (e != cudaSuccess) return e;
  // per-label cotangents of non-equilibrium ghosts: [side][n_theta][Q] after gwall
  T* gdir = reinterpret_cast<T*>(ws.gwall + (((size_t)16 * p.n_theta * sizeof(T) + 255) & ~(size_t)255));
  adjoint_wall_kernel<T><<<(2 * p.n_theta + 3) / 4, 128, 0, side>>>(f, lam_in, ghost, gwall, gdir, p, d);
  if constexpr (sizeof(T) == 4) {
    // FP32: the packed two-nodes-per-thread pair kernel (adjoint_f32x2.cu)
    e = cudaGetLastError();
    if (e == cudaSuccess)
      e = launch_adjoint_pairs_f32(tmap_f, tmap_l, tmap_fn, tmap_ln, f, lam_in, lam_out, ghost, gwall, gdir, 0, 1, b0,
                                   1 + (nt - b0), true, p, d, side);
    // tiles 1 .. t_hi - 1 have r0 > 0 and r0 < n_r - 33: no wall tile among them
    if (e == cudaSuccess && n_interior > 0)
      e = launch_adjoint_pairs_f32(tmap_f, tmap_l, tmap_fn, tmap_ln, f, lam_in, lam_out, ghost, gwall, gdir, 1, n_interior,
                                   0, n_interior, false, p, d, stream);
  } else {
    static std::atomic<unsigned long long> configured{0};
    constexpr int smem = AdjSize<T>::smem;
    e = set_smem_once(adjoint_pair_kernel<T>, smem, configured);
    if (e != cudaSuccess) return e;
    constexpr int TT = AdjTile<T>::TT;
    const unsigned gy = (unsigned)((p.n_theta + TT - 1) / TT);
    adjoint_pair_kernel<T><<<dim3(1 + (nt - b0), gy), AdjSize<T>::threads, smem, side>>>(
        *tmap_f, *tmap_l, f, lam_in, lam_out, ghost, gwall, gdir, 0, 1, b0, p, d);
    if (n_interior > 0)
      adjoint_pair_kernel<T><<<dim3(n_interior, gy), AdjSize<T>::threads, smem, stream>>>(
          *tmap_f, *tmap_l, f, lam_in, lam_out, ghost, gwall, gdir, 1, n_interior, 0, p, d);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return e;
  e = cudaEventRecord(ev_join, side);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, ev_join, 0);
  return e;
}

size_t adjoint_scratch_bytes(int n_theta, int elem) {
  // ghost: 2 x 3 EqParams (10 values) per row (two ghost layers and the wall
  // node); gwall: 2 x 2 x 4 per row; the non-equilibrium ghosts' per-label
  // cotangents: 2 x Q per row
  const size_t b = (size_t)6 * n_theta * 10 * elem, c = (size_t)16 * n_theta * elem;
  const size_t g = (size_t)2 * n_theta * kQ * elem;
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  return up(b) + up(c) + up(g);
}

AdjScratch adjoint_scratch(unsigned char* base, int n_theta, int elem) {
  AdjScratch s;
  s.ghost = base;
  s.gwall = base + (((size_t)6 * n_theta * 10 * elem + 255) & ~(size_t)255);
  return s;
}

template cudaError_t launch_adjoint<float>(const CUtensorMap*, const CUtensorMap*, const CUtensorMap*,
                                           const CUtensorMap*, const float*, const float*, float*,
                                           const AdjScratch&, const StepParams&, const DvmConst<float>&, cudaStream_t,
                                           cudaStream_t, cudaEvent_t, cudaEvent_t);
template cudaError_t launch_adjoint<double>(const CUtensorMap*, const CUtensorMap*, const CUtensorMap*,
                                            const CUtensorMap*, const double*, const double*,
                                            double*, const AdjScratch&, const StepParams&, const DvmConst<double>&,
                                            cudaStream_t, cudaStream_t, cudaEvent_t, cudaEvent_t);

}  // namespace pclb
