// Fused time step of the polar-coordinate FDLB model: one launch advances
// every node by the combined scheme of Eq. (38).
//
// Tile work (one CTA = kTileR x kTileT interior nodes):
//   1. one thread issues 33 TMA box copies (one per velocity plane) of the
//      window [r0-4, r0+36) x [t0-2, t0+18) into shared memory, completing on
//      one mbarrier (bounded wait);
//   2. every thread computes the moments (Eqs. 3-5) of its node(s) and
//      factors their equilibrium (Eqs. 10-11);
//   3. CTAs whose window covers a wall compute the radial ghost columns in
//      shared memory: moments of the two wall nodes, Eq. (39) extrapolation
//      (or prescribed values), f = f^eq (Sec. II C 1) -- ghosts never touch
//      global memory;
//   4. for every pair of opposite velocities (sharing their Courant entry,
//      staged per tile row in shared memory, and the even and odd parts of
//      the equilibrium polynomial): relaxation (Eq. 19) minus the convection
//      increments (Eq. 28 or the compared schemes) in r and theta read from
//      the window, stored straight to the output; rows next to the azimuthal
//      seam are also written into the output's ghost rows (Eq. 40, label
//      rotated by N_f) so the next step's window is one contiguous box.
#include <cuda.h>
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "ghost_cols.cuh"
#include "pclb_internal.h"

namespace pclb {

constexpr int kPlane = kWinR * kWinT;   // elements per velocity plane in shared memory

constexpr int kPairs64 = 4 * kNDirs / 2;   // pairs of opposite velocities
constexpr int kThreads64 = 512;            // 16 warps: one node per thread
constexpr int kWarps64 = kThreads64 / 32;
constexpr int kNodes64 = kTileT / kWarps64;   // nodes per thread (rows w, w + kWarps64, ..)
static_assert(kTileT % kWarps64 == 0 && kPairs64 * kTileT <= 2 * kThreads64, "tile / thread mapping");

// every plane window is a TMA destination: 128-byte aligned
static_assert((kPlane * 4) % 128 == 0, "TMA destinations must stay 128-byte aligned");

template <class T>
constexpr int step_smem_bytes() {
  // planes, Courant table [pair][row] of 4 values, barrier slot
  return kQ * kPlane * (int)sizeof(T) + kPairs64 * kTileT * 4 * (int)sizeof(T) + 128;
}

// Convection increment (upwind form, see device_common.cuh) from
// a = |C| and K = a (1 - a) given by the Courant table.
// Limiter part of the MWB increment, h = |D| (D - Dp) / (|D| + |Dp|), 0 when
// D = Dp = 0.  One Newton step on the reciprocal: h then carries a relative
// error <= 1e-12, i.e. K h <= 2.5e-13 |D| (K <= 1/4) in the update.
__device__ __forceinline__ double mwb_h(double D, double Dp) {
  const double den = fabs(D) + fabs(Dp);
  // den >= 2^-1022 (the smallest normal number), tested on the high word of
  // the non-negative den with an integer compare (keeps the FP64 pipe free)
  return __double2hiint(den) >= 0x00100000 ? fabs(D) * (D - Dp) * recip_newton1(den) : 0.0;
}

template <int SCH>
__device__ __forceinline__ double convect_aK(double a, double K, double f0, double u1, double u2, double d1) {
  const double D = f0 - u1, Dp = u1 - u2;
  if (SCH == PCLB_SCHEME_MWB) return a * D + K * mwb_h(D, Dp);
  if (SCH == PCLB_SCHEME_WB) return a * D + 0.5 * K * (D - Dp);
  if (SCH == PCLB_SCHEME_UPWIND2) return a * D + 0.5 * a * (D - Dp);
  return a * D + 0.5 * K * ((d1 - f0) - D);
}

template <class T, int SCH>
__global__ void __launch_bounds__(kThreads64, 1)
    step_kernel(const __grid_constant__ CUtensorMap tmap_in, T* __restrict__ f_out,
                const __grid_constant__ StepParams p, const __grid_constant__ DvmConst<T> d, int ty0) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  T* tab = sm + kQ * kPlane;                           // [pair][row][a_r, k_r, a_w, flags]
  uint64_t* bar = reinterpret_cast<uint64_t*>(tab + kPairs64 * kTileT * 4);

  const int r0 = blockIdx.x * kTileR;
  const int t0 = (blockIdx.y + ty0) * kTileT;   // ty0: first tile row of the launch
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
  // Courant entries of the tile rows (from the FP64 table of the context)
  for (int i = threadIdx.x; i < kPairs64 * kTileT; i += kThreads64) {
    const int pair = i / kTileT, rl = i % kTileT;
    const int tt = min(t0 + rl, p.n_theta - 1);
    const double* e = p.courant64 + ((size_t)(tt + kGhostRows) * kPairs64 + pair) * 4;
#pragma unroll
    for (int j = 0; j < 4; ++j) tab[(pair * kTileT + rl) * 4 + j] = (T)e[j];
  }
  // The whole block gives the tile up if any thread's wait ran out (a block
  // barrier follows below, so the decision must be uniform); thread 0 then
  // gives the copies one more bounded chance to land before the block exits.
  if (__syncthreads_or(p.wait_ns == 0 || !mbar_wait_bounded(bar, 0, p.wait_ns))) {   // 0: give up at once
    if (threadIdx.x == 0) {
      atomicOr(p.status, PCLB_FLAG_TIMEOUT);
      mbar_wait_bounded(bar, 0, kDefaultWaitNs);
    }
    return;
  }

  // ---- 2. moments and equilibrium factors of this thread's two nodes ------
  const int r = r0 + lane;
  const int col = kLeft + lane;
  int row[kNodes64], t[kNodes64];
  bool valid[kNodes64];
  EqParams<T> eq[kNodes64];
  bool ok = true;
#pragma unroll
  for (int c = 0; c < kNodes64; ++c) {
    row[c] = 2 + warp + kWarps64 * c;
    t[c] = t0 + warp + kWarps64 * c;
    valid[c] = (r < p.n_r) && (t[c] < p.n_theta);
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

  // ---- 4. relaxation minus MWB increments, per pair of opposite velocities --
  const T inv_r = (r < p.n_r) ? (T)p.inv_r[r] : T(1);
  const T decay = (T)p.decay, omd = T(1) - decay;
  const size_t plane_out = (size_t)p.rows * p.pitch;
  auto store = [&](int q, int c, T out) {
    T* dst = f_out + (size_t)q * plane_out + r;
    dst[(size_t)(t[c] + kGhostRows) * p.pitch] = out;
    if (t[c] >= p.n_theta - 2)   // also the low ghost rows (theta <= 0) of the receiving label
      f_out[(size_t)d.recv_lo[q] * plane_out + (size_t)(t[c] - (p.n_theta - 2)) * p.pitch + r] = out;
    if (t[c] < 2)                // and the high ghost rows (theta > 2 pi n_f / n_dirs)
      f_out[(size_t)d.recv_hi[q] * plane_out + (size_t)(p.n_theta + kGhostRows + t[c]) * p.pitch + r] = out;
  };
#pragma unroll
  for (int c = 0; c < kNodes64; ++c) {   // rest velocity: no convection
    if (!valid[c]) continue;
    const T f0 = sm[row[c] * kWinR + col];
    const T fe = eq[c].w[0] * eq[c].a0;
    store(0, c, fe + (f0 - fe) * decay);
  }
  // Shells are unrolled so that the weight rho F_k is a register; the four
  // pairs (q, q + N_i/2) of a shell run as a loop and share their Courant
  // entry and the even and odd parts of the equilibrium polynomial.
#pragma unroll
  for (int k = 1; k <= 4; ++k) {
#pragma unroll 1
    for (int i = 0; i < kNDirs / 2; ++i) {
      const int pair = (k - 1) * (kNDirs / 2) + i;
      const int q1 = 1 + (k - 1) * kNDirs + i, q2 = q1 + kNDirs / 2;
      const T vx = d.vx[q1], vy = d.vy[q1];
#pragma unroll
      for (int c = 0; c < kNodes64; ++c) {
        if (!valid[c]) continue;
        const T* e = tab + (pair * kTileT + warp + kWarps64 * c) * 4;
        const T ar = e[0], kr = e[1], at = e[2] * inv_r, kt = at - at * at;
        const int fl = (int)e[3];
        const int sr = (fl & 1) ? 1 : -1;               // v_r < 0 for q1: upwind at larger r
        const int st = (fl & 2) ? kWinR : -kWinR;       // v_theta < 0 for q1: upwind at larger theta
        // equilibrium of the pair: P(+x) = ev + od, P(-x) = ev - od (Eq. 10)
        const T x = vx * eq[c].uxE + vy * eq[c].uyE, x2 = x * x;
        const T ev = eq[c].a0 + x2 * (eq[c].a1h + x2 * T(1.0 / 24.0));
        const T od = x * (eq[c].a1 + x2 * T(1.0 / 6.0));
        const T fe1 = SCH == PCLB_SCHEME_MWB ? T(0) : eq[c].w[k] * (ev + od);
        const T fe2 = SCH == PCLB_SCHEME_MWB ? T(0) : eq[c].w[k] * (ev - od);
        const T* fp1 = sm + q1 * kPlane + row[c] * kWinR + col;
        const T* fp2 = sm + q2 * kPlane + row[c] * kWinR + col;
        const bool lw = SCH == PCLB_SCHEME_LW;
        const T a = fp1[0], b = fp2[0];
        T o1, o2;
        if constexpr (SCH == PCLB_SCHEME_MWB) {
          // relaxation minus a D + K h in r and theta, as one chain of fused
          // multiply-adds
          // (1 - d) f^eq + d f0 = (1 - d) rho F_k P + d f0
          const T wd = omd * eq[c].w[k];
          auto mwb = [&](T f0, T P, const T* fp, int s_r, int s_t) {
            const T u1 = fp[s_r], v1 = fp[s_t];
            const T Dr = f0 - u1, Dt = f0 - v1;
            T o = fma(wd, P, decay * f0);
            o = fma(-ar, Dr, o);
            o = fma(-kr, mwb_h(Dr, u1 - fp[2 * s_r]), o);
            o = fma(-at, Dt, o);
            return fma(-kt, mwb_h(Dt, v1 - fp[2 * s_t]), o);
          };
          o1 = mwb(a, ev + od, fp1, sr, st);
          o2 = mwb(b, ev - od, fp2, -sr, -st);
        } else {
          o1 = fe1 + (a - fe1) * decay -
               convect_aK<SCH>(ar, kr, a, fp1[sr], fp1[2 * sr], lw ? fp1[-sr] : T(0)) -
               convect_aK<SCH>(at, kt, a, fp1[st], fp1[2 * st], lw ? fp1[-st] : T(0));
          o2 = fe2 + (b - fe2) * decay -
               convect_aK<SCH>(ar, kr, b, fp2[-sr], fp2[-2 * sr], lw ? fp2[sr] : T(0)) -
               convect_aK<SCH>(at, kt, b, fp2[-st], fp2[-2 * st], lw ? fp2[st] : T(0));
        }
        store(q1, c, o1);
        store(q2, c, o2);
      }
    }
  }
}

template <class T, int SCH>
static cudaError_t launch_scheme(const CUtensorMap* tmap_in, T* f_out, const StepParams& p, const DvmConst<T>& d,
                                 cudaStream_t stream, int ty_begin, int ty_end) {
  static std::atomic<unsigned long long> configured{0};   // per instantiation and device
  const int smem = step_smem_bytes<T>();
  {
    const cudaError_t e = set_smem_once(step_kernel<T, SCH>, smem, configured);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((p.n_r + kTileR - 1) / kTileR, ty_end - ty_begin);
  step_kernel<T, SCH><<<grid, kThreads64, smem, stream>>>(*tmap_in, f_out, p, d, ty_begin);
  return cudaGetLastError();
}

// Tile rows [ty_begin, ty_end) of the grid (ty_end < 0: to the last tile row);
// an empty range launches nothing.
template <class T>
cudaError_t launch_step(const CUtensorMap* tmap_in, T* f_out, const StepParams& p,
                        const DvmConst<T>& d, cudaStream_t stream, int ty_begin, int ty_end) {
  if (ty_end < 0) ty_end = (p.n_theta + kTileT - 1) / kTileT;
  if (ty_begin < 0 || ty_end <= ty_begin) return cudaSuccess;
  switch (p.scheme) {
    case PCLB_SCHEME_WB: return launch_scheme<T, PCLB_SCHEME_WB>(tmap_in, f_out, p, d, stream, ty_begin, ty_end);
    case PCLB_SCHEME_LW: return launch_scheme<T, PCLB_SCHEME_LW>(tmap_in, f_out, p, d, stream, ty_begin, ty_end);
    case PCLB_SCHEME_UPWIND2:
      return launch_scheme<T, PCLB_SCHEME_UPWIND2>(tmap_in, f_out, p, d, stream, ty_begin, ty_end);
    default: return launch_scheme<T, PCLB_SCHEME_MWB>(tmap_in, f_out, p, d, stream, ty_begin, ty_end);
  }
}

template cudaError_t launch_step<double>(const CUtensorMap*, double*, const StepParams&,
                                         const DvmConst<double>&, cudaStream_t, int, int);

}  // namespace pclb
