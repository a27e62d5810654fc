// Fused time step of the polar-coordinate FDLB model: one launch advances
// every node by the combined scheme of Eq. (38).
//
// Tile work (one CTA = kTileR x kTileT interior nodes):
//   1. one thread issues 33 TMA box copies (one per velocity plane) of the
//      window [r0-4, r0+36) x [t0-2, t0+18) into shared memory, completing on
//      one mbarrier (bounded wait);
//   2. every thread computes the moments (Eqs. 3-5) of its two nodes and
//      factors their equilibrium (Eqs. 10-11);
//   3. CTAs whose window covers a wall compute the radial ghost columns in
//      shared memory: moments of the two wall nodes, Eq. (39) extrapolation
//      (or prescribed values), f = f^eq (Sec. II C 1) -- ghosts never touch
//      global memory;
//   4. for every velocity: relaxation (Eq. 19) minus the MWB increments
//      (Eq. 28) in r and theta read from the window, stored straight to the
//      output; rows next to the azimuthal seam are also written into the
//      output's ghost rows (Eq. 40, label rotated by N_f) so the next step's
//      window is one contiguous box.
#include <cuda.h>
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "ghost_cols.cuh"
#include "pclb_internal.h"

namespace pclb {

constexpr int kPlane = kWinR * kWinT;   // elements per velocity plane in shared memory
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s

template <class T>
constexpr int step_smem_bytes() {
  return kQ * kPlane * (int)sizeof(T) + 128;   // planes + barrier slot
}

template <class T, int SCH>
__global__ void __launch_bounds__(kStepThreads, (sizeof(T) == 4 ? 2 : 1))
    step_kernel(const __grid_constant__ CUtensorMap tmap_in, T* __restrict__ f_out,
                const __grid_constant__ StepParams p, const __grid_constant__ DvmConst<T> d) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + kQ * kPlane * sizeof(T));

  const int r0 = blockIdx.x * kTileR;
  const int t0 = blockIdx.y * kTileT;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;

  if (threadIdx.x == 0) {
    tma_prefetch_desc(&tmap_in);
    mbar_init(bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(bar, (uint32_t)(kQ * kPlane * sizeof(T)));
    // Window rows [t0-2, t0+18) are stored rows [t0, t0+20) (two ghost rows first).
#pragma unroll 1
    for (int q = 0; q < kQ; ++q) tma_load_3d(sm + q * kPlane, &tmap_in, r0 - kLeft, t0, q, bar);
  }
  if (!mbar_wait_bounded(bar, 0, kWaitLimitNs)) {
    if (threadIdx.x == 0) atomicOr(p.status, PCLB_FLAG_TIMEOUT);
    // give the copies one more bounded chance to land before the CTA exits
    mbar_wait_bounded(bar, 0, kWaitLimitNs);
    return;
  }

  // ---- 2. moments and equilibrium factors of this thread's two nodes ------
  const int r = r0 + lane;
  const int col = kLeft + lane;
  int row[2], t[2];
  bool valid[2];
  T cs[2], sn[2];
  EqParams<T> eq[2];
  bool ok = true;
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    row[c] = 2 + warp + 8 * c;
    t[c] = t0 + warp + 8 * c;
    valid[c] = (r < p.n_r) && (t[c] < p.n_theta);
    cs[c] = valid[c] ? (T)p.cos_t[t[c]] : T(1);
    sn[c] = valid[c] ? (T)p.sin_t[t[c]] : T(0);
    NodeState<T> m;
    if (valid[c]) {
      m = node_moments(sm + row[c] * kWinR + col, kPlane, d);
      ok = ok && m.ok;
    } else {
      m.rho = T(1); m.ux = T(0); m.uy = T(0); m.E = T(1); m.ok = true;
      m.rho_d = 1.0; m.E_d = 1.0;
    }
    eq[c] = eq_params<T>(m.rho_d, m.ux, m.uy, m.E_d, d);
  }
  if (!ok) atomicOr(p.status, PCLB_FLAG_NONPHYS);

  // ---- 3. radial ghost columns (inside the window only) -------------------
  if (r0 == 0 && warp == 0 && lane < kTileT) {
    const int tt = t0 + lane;
    if (tt < p.n_theta) fill_ghost_columns<T, kPlane>(sm, 2 + lane, 0, kLeft, tt, p, d);
  }
  const int cw_out = p.n_r - 1 - r0 + kLeft;   // window column of the outer wall node
  if (cw_out + 1 <= kLeft + kTileR + 1 && warp == 1 && lane < kTileT) {
    const int tt = t0 + lane;
    if (tt < p.n_theta) fill_ghost_columns<T, kPlane>(sm, 2 + lane, 1, cw_out, tt, p, d);
  }
  __syncthreads();

  // ---- 4. relaxation minus MWB increments, per velocity -------------------
  const T inv_r = (r < p.n_r) ? (T)p.inv_r[r] : T(1);
  const T dt_dr = (T)p.dt_dr;
  const T dt_dth_r = (T)p.dt_dth * inv_r;
  const T decay = (T)p.decay;
  const size_t plane_out = (size_t)p.rows * p.pitch;
  // Shells are unrolled so that the weight rho F_k is a register, not an
  // indexed array; directions within a shell run as a loop.
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const int q_begin = k == 0 ? 0 : 1 + (k - 1) * kNDirs;
    const int q_end = k == 0 ? 1 : q_begin + kNDirs;
#pragma unroll 1
    for (int q = q_begin; q < q_end; ++q) {
      const T vx = d.vx[q], vy = d.vy[q];
      const T* base = sm + q * kPlane + col;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        if (!valid[c]) continue;
        const T vr = vx * cs[c] + vy * sn[c];
        const T vt = vy * cs[c] - vx * sn[c];
        const int sr = vr >= T(0) ? -1 : 1;            // upwind neighbour in r
        const int st = vt >= T(0) ? -kWinR : kWinR;    // upwind neighbour in theta
        const T* fp = base + row[c] * kWinR;
        const T f0 = fp[0];
        const T mr = convect<SCH>(vr * dt_dr, f0, fp[sr], fp[2 * sr], SCH == PCLB_SCHEME_LW ? fp[-sr] : T(0));
        const T mt = convect<SCH>(vt * dt_dth_r, f0, fp[st], fp[2 * st], SCH == PCLB_SCHEME_LW ? fp[-st] : T(0));
        const T fe = feq_q<T>(eq[c], vx, vy, k);
        const T out = fe + (f0 - fe) * decay - mr - mt;
        T* dst = f_out + (size_t)q * plane_out + r;
        dst[(size_t)(t[c] + kGhostRows) * p.pitch] = out;
        if (t[c] >= p.n_theta - 2)   // also the low ghost rows (theta <= 0) of the receiving label
          f_out[(size_t)d.recv_lo[q] * plane_out + (size_t)(t[c] - (p.n_theta - 2)) * p.pitch + r] = out;
        if (t[c] < 2)                // and the high ghost rows (theta > 2 pi n_f / n_dirs)
          f_out[(size_t)d.recv_hi[q] * plane_out + (size_t)(p.n_theta + kGhostRows + t[c]) * p.pitch + r] = out;
      }
    }
  }
}

template <class T, int SCH>
static cudaError_t launch_scheme(const CUtensorMap* tmap_in, T* f_out, const StepParams& p, const DvmConst<T>& d,
                                 cudaStream_t stream) {
  static bool configured = false;   // one-time attribute set per instantiation
  const int smem = step_smem_bytes<T>();
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(step_kernel<T, SCH>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  dim3 grid((p.n_r + kTileR - 1) / kTileR, (p.n_theta + kTileT - 1) / kTileT);
  step_kernel<T, SCH><<<grid, kStepThreads, smem, stream>>>(*tmap_in, f_out, p, d);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_step(const CUtensorMap* tmap_in, T* f_out, const StepParams& p,
                        const DvmConst<T>& d, cudaStream_t stream) {
  switch (p.scheme) {
    case PCLB_SCHEME_WB: return launch_scheme<T, PCLB_SCHEME_WB>(tmap_in, f_out, p, d, stream);
    case PCLB_SCHEME_LW: return launch_scheme<T, PCLB_SCHEME_LW>(tmap_in, f_out, p, d, stream);
    case PCLB_SCHEME_UPWIND2: return launch_scheme<T, PCLB_SCHEME_UPWIND2>(tmap_in, f_out, p, d, stream);
    default: return launch_scheme<T, PCLB_SCHEME_MWB>(tmap_in, f_out, p, d, stream);
  }
}

template cudaError_t launch_step<double>(const CUtensorMap*, double*, const StepParams&,
                                         const DvmConst<double>&, cudaStream_t);

}  // namespace pclb
