// Radial ghost columns of a shared-memory window (generic precision), Sec. II C 1.
#pragma once

#include "device_common.cuh"
#include "pclb_internal.h"

namespace pclb {

// Compute one wall's two ghost columns for the tile row `row` (window row
// index) from the window itself.  side 0: inner wall, ghost columns kLeft-1
// (layer 0) and kLeft-2 (layer 1) from wall node column kLeft and the next
// column.  side 1: outer wall at window column cw = n_r - 1 - r0 + kLeft,
// ghosts at cw+1 (layer 0) and cw+2 (layer 1).
template <class T, int PLANE>
__device__ void fill_ghost_columns(T* sm, int row, int side, int cw, int t, const StepParams& p,
                                   const DvmConst<T>& d) {
  const int step = side == 0 ? 1 : -1;               // towards the interior
  const T* fa = sm + row * kWinR + cw;                // wall node (i_r = 1 or N_r)
  const T* fb = sm + row * kWinR + cw + step;         // next node inward
  NodeState<T> a = node_moments(fa, PLANE, d);
  NodeState<T> b = node_moments(fb, PLANE, d);
  double rho[2], E[2];
  T ux[2], uy[2];
  rho[0] = 2.0 * a.rho_d - b.rho_d;  rho[1] = 2.0 * rho[0] - a.rho_d;   // Eq. (39), applied twice
  E[0] = 2.0 * a.E_d - b.E_d;        E[1] = 2.0 * E[0] - a.E_d;
  ux[0] = T(2) * a.ux - b.ux;        ux[1] = T(2) * ux[0] - a.ux;
  uy[0] = T(2) * a.uy - b.uy;        uy[1] = T(2) * uy[0] - a.uy;
  const int kind = p.bc_kind[side] & ~PCLB_BC_NEQ;
  const bool neq = (p.bc_kind[side] & PCLB_BC_NEQ) != 0;
  if (kind != PCLB_BC_EXTRAP) {
    const double c = p.cos_t[t], s = p.sin_t[t];
    for (int layer = 0; layer < 2; ++layer) {
      const double* v = p.bc_vals + (size_t)((side * 2 + layer) * 4) * p.n_theta + t;
      const double ur = v[1 * p.n_theta], ut = v[2 * p.n_theta];
      ux[layer] = (T)(ur * c - ut * s);
      uy[layer] = (T)(ur * s + ut * c);
      if (kind == PCLB_BC_DIRICHLET) {
        rho[layer] = v[0];
        E[layer] = v[3 * p.n_theta];
      }
    }
  }
  bool ok = a.ok && b.ok;
  // equilibrium of the wall node, for the departure it hands to its ghosts
  const EqParams<T> ea = eq_params<T>(a.rho_d, a.ux, a.uy, a.E_d, d);
  for (int layer = 0; layer < 2; ++layer) {
    ok = ok && rho[layer] > 0.0 && E[layer] > 0.0;
    const int col = cw - step * (1 + layer);
    if (col < 0 || col >= kWinR) continue;
    EqParams<T> e = eq_params<T>(rho[layer], ux[layer], uy[layer], E[layer], d);
    T* g = sm + row * kWinR + col;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const int q_begin = k == 0 ? 0 : 1 + (k - 1) * kNDirs;
      const int q_end = k == 0 ? 1 : q_begin + kNDirs;
#pragma unroll 1
      for (int q = q_begin; q < q_end; ++q) {
        T v = feq_q<T>(e, d.vx[q], d.vy[q], k);
        if (neq) v += fa[q * PLANE] - feq_q<T>(ea, d.vx[q], d.vy[q], k);
        g[q * PLANE] = v;
      }
    }
  }
  if (!ok) atomicOr(p.status, PCLB_FLAG_NONPHYS);
}

}  // namespace pclb
