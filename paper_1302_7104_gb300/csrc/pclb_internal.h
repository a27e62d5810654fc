// Internal types shared by the host side of the C ABI and the kernels.
// Not part of the public interface (include/pclb.h).
#pragma once

#include <atomic>
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "pclb.h"

namespace pclb {

// The discrete velocity model built here: N_k = 4 shells of kNDirs directions
// plus the rest velocity (Eq. 2), Q = 33 for the octagon.
constexpr int kNDirs = 8;
constexpr int kQ = 1 + 4 * kNDirs;

// Tiling of the fused step kernel.  A tile is kTileR x kTileT interior nodes;
// its shared-memory window holds every velocity plane over
// [r0 - 4, r0 + kTileR + 4) x [t0 - 2, t0 + kTileT + 2): the +-2 stencil halo
// in both directions, with the radial start rounded down to a 16-byte
// boundary so the TMA box starts aligned.
constexpr int kTileR = 32;
constexpr int kTileT = 16;
// FP32 step kernel: tile rows, threads (two radially adjacent nodes each) and
// CTAs per SM
constexpr int kTileT32 = 16;
constexpr int kStepThreads32 = 16 * kTileT32;
constexpr int kCtasPerSm32 = 2;
constexpr int kWinR = kTileR + 8;   // 40 columns
constexpr int kWinT = kTileT + 4;   // 20 rows
constexpr int kLeft = 4;            // column of interior r0 inside the window
constexpr int kStepThreads = 256;   // 8 warps; each thread owns 2 nodes (rows w and w + 8)
constexpr int kPitchAlign = 32;     // row pitch in elements (128 B for float)
constexpr int kGhostRows = 2;       // azimuthal ghost rows stored on each side
// Tile rows of the adjoint kernel (its window holds f and lam for all labels).
constexpr int kAdjRows32 = 16;
constexpr int kAdjRows64 = 8;
// Time a kernel waits for the TMA copies of its own window (mbarrier phase)
// before it reports PCLB_FLAG_TIMEOUT and gives the tile up; the copies of a
// tile given up get the default limit again to land before the CTA exits.
// The step kernels take their first wait's limit from StepParams::wait_ns
// (pclb_set_wait_limit); every other wait uses the default.
constexpr uint64_t kDefaultWaitNs = 2000000000ull;   // 2 s
constexpr uint64_t kMaxWaitNs = 60000000000ull;      // 60 s

// Per-velocity constants, in the arithmetic type T of the kernel, plus the
// double-precision ones the moment / temperature recovery uses.
template <class T>
struct DvmConst {
  T vx[kQ], vy[kQ];           // Cartesian components v_qx, v_qy
  T cx[kQ], cy[kQ];           // unit direction (cos phi_i, sin phi_i); 0 for q = 0
  T speed[5];                 // v_k
  T half_v2[5];               // v_k^2 / 2
  T Fc[5][4];                 // F_k(E) = sum_{n=1..4} Fc[k][n-1] E^n, k = 1..4 (Eq. 11a)
  T Fc_lo[5][4];              // Fc - (double)Fc rounded to T: the low part of a float-float pair
  // Low parts (value - (double)hi, rounded to T) of the velocity constants, so
  // that the FP32 path can use them as float-float pairs; zero for double.
  T vx_lo[kQ], vy_lo[kQ], cx_lo[kQ], cy_lo[kQ];
  T speed_lo[5], half_v2_lo[5];
  // v_3 - v_2 and (v_3^2 - v_2^2)/2 as float-float pairs: the FP32 moments sum
  // shells 2 and 3 direction by direction (their speeds are close and their
  // weights opposite), then correct with these differences.
  T dv23, dv23_lo, dh23, dh23_lo;
  T B0;                       // F_0 = 1 - B0 (F_1 + .. + F_4) (Eq. 11b)
  int8_t shell[kQ];           // k of label q
  int8_t recv_lo[kQ];         // label whose low ghost rows copy rows n_theta-2.. of label q
  int8_t recv_hi[kQ];         // label whose high ghost rows copy rows 0, 1 of label q
};

// Velocity sets with N_i = 16 or 24 (Table I), for the generic kernels; all
// constants in double.
constexpr int kMaxQ = 1 + 4 * 24;
struct DvmG {
  double vx[kMaxQ], vy[kMaxQ];
  double half_v2[5];          // v_k^2 / 2
  double Fc[5][4];            // F_k(E) = sum_{n=1..4} Fc[k][n-1] E^n, k = 1..4 (Eq. 11a)
  double B0;                  // F_0 = 1 - B0 (F_1 + .. + F_4) (Eq. 11b)
  int shell[kMaxQ];
  int recv_lo[kMaxQ], recv_hi[kMaxQ];   // as in DvmConst
  int n_dirs, q;
};

struct StepParams {
  int n_r, n_theta;           // interior nodes
  int pitch;                  // elements per stored row (multiple of kPitchAlign)
  int rows;                   // stored rows per plane: n_theta + 4
  double dt_dr;               // dt / dr
  double dt_dth;              // dt / dtheta
  double decay;               // exp(-dt / tau), Eq. (19), or 1 - dt / tau (forward Euler)
  int bc_kind[2];
  int scheme;                 // pclb_scheme of the convection increments
  const double* cos_t;        // [n_theta] cos(theta_i), host-computed in double
  const double* sin_t;        // [n_theta]
  const double* inv_r;        // [n_r] 1 / r_i
  const double* bc_vals;      // [2 sides][2 layers][4 fields][n_theta] or unused
  const float4* courant;      // [n_theta + 4][4 n_dirs / 2] (stored rows, ghosts included): per
                              // opposite-velocity pair (first label
                              // q of the pair) |C_r|, |C_r|(1 - |C_r|), |v_theta| dt / dtheta,
                              // flags (bit 0: v_r < 0, bit 1: v_theta < 0) as int bits
  const double* courant64;    // the same table in double: [n_theta + 4][pairs][4] (flags as value)
  const float* inv_r_f;       // [n_r] 1 / r_i in float
  const float4* cs_ff;        // [n_theta] cos theta_i, sin theta_i as float-float pairs (hi, lo, hi, lo)
  uint32_t* status;           // device status word (PCLB_FLAG_*)
  uint64_t wait_ns;           // a step's wait for its own window copies before it gives the tile up
};

// Workspace layout (byte offsets from the caller's base pointer).
struct Layout {
  size_t f[2];                // two ping-pong distributions [Q][rows][pitch]
  size_t adj_f;               // a state copy for pclb_adjoint_step
  size_t lam[2];              // ping-pong adjoint variables, same layout as f
  size_t f_bytes;
  size_t cos_t, sin_t, inv_r, bc_vals, courant, courant64, inv_r_f, cs_ff;
  size_t status;              // uint32 status word (+ padding)
  size_t partials;            // double [kDiagBlocks][8] reduction partials
  size_t diag_out;            // double [8]
  size_t stage;               // host-I/O staging: 8 fields [n_theta][n_r]
  size_t adj_scratch;         // adjoint ghost states and wall cotangents
  size_t gen_ghost;           // N_i = 16, 24: radial ghost values [side][layer][n_theta][Q]
  size_t total;
};

// Scratch of one adjoint step (device pointers inside the workspace).
struct AdjScratch {
  unsigned char* ghost;       // [side][layer][n_theta] EqParams of the radial ghost layers
  unsigned char* gwall;       // [side][node][n_theta][4] cotangent the ghosts return
};
// Raises kernel fn's dynamic shared-memory limit to `bytes` once per device
// (the attribute belongs to each device's context); `done` holds one bit per
// device ordinal.
template <class F>
inline cudaError_t set_smem_once(F* fn, int bytes, std::atomic<unsigned long long>& done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = dev < 64 ? (1ull << dev) : 0ull;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_release);
  return e;
}

size_t adjoint_scratch_bytes(int n_theta, int elem);
AdjScratch adjoint_scratch(unsigned char* base, int n_theta, int elem);

constexpr int kDiagBlocks = 304;    // 2 x 152 SMs

// Host helpers shared by the C-ABI translation units (defined in pclb_abi.cu).
pclb_status validate_problem(const pclb_grid* g, const pclb_dvm* d, pclb_precision prec);
template <class T>
void fill_dvm(DvmConst<T>& c, const pclb_dvm& d, const pclb_grid& g);
void set_thread_error(const char* msg);   // text returned by pclb_last_error(NULL)

// Element size of a precision.
inline size_t elem_size(pclb_precision p) { return p == PCLB_FP64 ? 8 : 4; }

}  // namespace pclb

// Host context behind the opaque pclb_ctx handle.
struct pclb_ctx {
  pclb_grid grid;
  pclb_dvm dvm;
  pclb_precision prec;
  double tau, dt;
  int32_t bc_kind[2];   // pclb_bc_kind, possibly with PCLB_BC_NEQ
  int32_t scheme = 0;       // pclb_scheme
  int32_t relaxation = 0;   // pclb_relaxation
  cudaStream_t stream;
  cudaStream_t side = nullptr;        // high-priority stream for the adjoint's wall work
  cudaStream_t capture = nullptr;     // private stream for capturing step graphs
  struct StepGraph {
    int32_t n, cur;                   // steps and starting buffer of the captured sequence
    cudaGraphExec_t exec;
  } graphs[4] = {};
  int32_t n_graphs = 0;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // pclb_run_host with page-locked buffers: the host transfers of each
  // azimuthal slab run on two copy streams and its set-state kernel on a
  // third stream while the steps of other slabs run on `stream` and io_alt
  // (created on first use)
  static constexpr int kIoSlabs = 16;
  cudaStream_t io_in = nullptr, io_set = nullptr, io_out = nullptr, io_alt = nullptr;
  cudaEvent_t io_start = nullptr, io_done = nullptr;
  cudaEvent_t io_loaded[kIoSlabs] = {}, io_isset[kIoSlabs] = {}, io_ready[kIoSlabs] = {};
  unsigned char* ws;
  pclb::Layout lay;
  int cur;                    // which of the two f buffers holds the state
  bool has_state;
  CUtensorMap tmap[2];        // TMA descriptors of the two f buffers
  CUtensorMap tmap_adj[5];    // adjoint-window descriptors: f[0], f[1], adj_f, lam[0], lam[1]
  CUtensorMap tmap_node[5];   // FP32 adjoint node-phase descriptors (tile boxes) of the same buffers
  int cur_lam;                // which lam buffer holds the adjoint variable
  bool has_lam;
  pclb::StepParams sp;
  pclb::DvmConst<float> dvm32;
  pclb::DvmConst<double> dvm64;
  pclb::DvmG dvmg;            // N_i = 16, 24 (the generic kernels)
  char err[512];
};
