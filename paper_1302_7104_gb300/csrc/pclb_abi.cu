// Host side of the C ABI declared in include/pclb.h: argument validation,
// workspace layout, host-computed tables, TMA descriptors, launches, bounded
// waits and error reporting.
#include <initializer_list>
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

#include "dvm_generic.h"
#include "pclb_internal.h"

namespace pclb {
// Step launchers take a range of tile rows, the field kernels a range of
// grid rows (the whole grid by default).
cudaError_t launch_step_f32(const CUtensorMap*, float*, const StepParams&, const DvmConst<float>&,
                            cudaStream_t, int ty_begin = 0, int ty_end = -1);
template <class T>
cudaError_t launch_step(const CUtensorMap*, T*, const StepParams&, const DvmConst<T>&, cudaStream_t,
                        int ty_begin = 0, int ty_end = -1);
template <class T>
cudaError_t launch_set_state(T*, const T*, const T*, const T*, const T*, const StepParams&,
                             const DvmConst<T>&, cudaStream_t, int t_begin = 0, int t_end = -1);
template <class T>
cudaError_t launch_moments(const T*, T*, T*, T*, T*, const StepParams&, const DvmConst<T>&, cudaStream_t,
                           int t_begin = 0, int t_end = -1);
template <class T>
cudaError_t launch_pack(const T*, T*, const StepParams&, cudaStream_t);
template <class T>
cudaError_t launch_unpack(const T*, T*, const StepParams&, const DvmConst<T>&, cudaStream_t);
template <class T>
cudaError_t launch_diagnostics(const T*, double*, double*, const StepParams&, const DvmConst<T>&,
                               double, double, double, cudaStream_t);
template <class T>
cudaError_t launch_noneq(const T*, T*, int, const StepParams&, const DvmConst<T>&, cudaStream_t);
template <class T>
cudaError_t launch_noneq_gen(const T*, T*, int, const StepParams&, const DvmG&, const DvmG32&, cudaStream_t);
template <class T>
cudaError_t launch_adjoint(const CUtensorMap*, const CUtensorMap*, const CUtensorMap*, const CUtensorMap*, const T*,
                           const T*, T*, const AdjScratch&,
                           const StepParams&, const DvmConst<T>&, cudaStream_t, cudaStream_t, cudaEvent_t,
                           cudaEvent_t);
template <class T>
cudaError_t gen_launch_set_state(T*, const T*, const T*, const T*, const T*, const StepParams&, const DvmG&,
                                 cudaStream_t);
template <class T>
cudaError_t gen_launch_moments(const T*, T*, T*, T*, T*, const StepParams&, const DvmG&, cudaStream_t);
template <class T>
cudaError_t gen_launch_pack(const T*, T*, const StepParams&, const DvmG&, cudaStream_t);
template <class T>
cudaError_t gen_launch_unpack(const T*, T*, const StepParams&, const DvmG&, cudaStream_t);
template <class T>
cudaError_t gen_launch_diagnostics(const T*, double*, double*, const StepParams&, const DvmG&, double, double,
                                   double, cudaStream_t);
template <class T>
cudaError_t launch_moments_vjp(const T*, const T*, const T*, const T*, const T*, T*, const StepParams&,
                               const DvmConst<T>&, cudaStream_t);
template <class T>
cudaError_t launch_set_state_vjp(const T*, const T*, const T*, const T*, const T*, T*, T*, T*, T*,
                                 const StepParams&, const DvmConst<T>&, cudaStream_t);
}  // namespace pclb

using namespace pclb;

namespace {

thread_local char g_err[512] = "";
constexpr int kDefaultTimeoutMs = 120000;

struct HostCtx : pclb_ctx {
  std::vector<double> cos_t, sin_t, inv_r, bc_vals;
  std::vector<float> courant, inv_r_f, cs_ff;
  std::vector<double> courant64;
  DvmG32 dvmg32;   // N_i = 16, 24: float tables of the FP32 step and field kernels
};

const DvmG32& dvmg32(const pclb_ctx* c) { return static_cast<const HostCtx*>(c)->dvmg32; }

pclb_status fail(pclb_ctx* ctx, pclb_status st, const char* fmt, ...) {
  char* buf = ctx ? ctx->err : g_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, 512, fmt, ap);
  va_end(ap);
  return st;
}

pclb_status cuda_fail(pclb_ctx* ctx, cudaError_t e, const char* what) {
  return fail(ctx, PCLB_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

namespace pclb {
pclb_status validate_problem(const pclb_grid* g, const pclb_dvm* d, pclb_precision prec) {
  if (!g || !d) return fail(nullptr, PCLB_EINVAL, "grid and dvm must not be NULL");
  if (prec != PCLB_FP32 && prec != PCLB_FP64) return fail(nullptr, PCLB_EINVAL, "unknown precision %d", (int)prec);
  if (g->n_r < 3) return fail(nullptr, PCLB_EINVAL, "n_r = %d; need at least 3 radial nodes", g->n_r);
  if (g->n_theta < 2) return fail(nullptr, PCLB_EINVAL, "n_theta = %d; need at least 2", g->n_theta);
  if (g->n_r > (1 << 20) || g->n_theta > (1 << 20))
    return fail(nullptr, PCLB_EINVAL, "grid %d x %d beyond the supported 2^20 per direction", g->n_r, g->n_theta);
  if (!(g->r_in > 0.0) || !(g->r_out > g->r_in) || !std::isfinite(g->r_out))
    return fail(nullptr, PCLB_EINVAL, "need 0 < r_in < r_out (got %g, %g)", g->r_in, g->r_out);
  if (d->n_dirs != kNDirs && d->n_dirs != 16 && d->n_dirs != 24)
    return fail(nullptr, PCLB_EUNSUPPORTED, "n_dirs = %d; the library implements 8, 16 and 24 directions", d->n_dirs);
  if (g->n_f < 1 || g->n_f > d->n_dirs)
    return fail(nullptr, PCLB_EINVAL, "n_f = %d must be in [1, n_dirs]", g->n_f);
  if (d->speeds[0] != 0.0) return fail(nullptr, PCLB_EINVAL, "speeds[0] must be 0 (rest velocity)");
  for (int k = 1; k <= 4; ++k) {
    if (!(d->speeds[k] > 0.0) || !std::isfinite(d->speeds[k]))
      return fail(nullptr, PCLB_EINVAL, "speeds[%d] must be positive and finite", k);
    for (int j = 1; j < k; ++j)
      if (d->speeds[j] == d->speeds[k]) return fail(nullptr, PCLB_EINVAL, "shell speeds must differ");
  }
  for (int n = 0; n < 5; ++n)
    if (!std::isfinite(d->B[n])) return fail(nullptr, PCLB_EINVAL, "B[%d] is not finite", n);
  return PCLB_OK;
}
}  // namespace pclb

namespace {
using pclb::validate_problem;
pclb_status validate(const pclb_grid* g, const pclb_dvm* d, pclb_precision prec) {
  return validate_problem(g, d, prec);
}

Layout make_layout(const pclb_grid* g, const pclb_dvm* d, pclb_precision prec) {
  Layout L{};
  const size_t es = elem_size(prec);
  const size_t Q = 1 + 4 * (size_t)d->n_dirs, npairs = 2 * (size_t)d->n_dirs;
  const size_t pitch = align_up((size_t)g->n_r, kPitchAlign);
  const size_t rows = (size_t)g->n_theta + 2 * kGhostRows;
  L.f_bytes = align_up(Q * rows * pitch * es, 256);
  size_t off = 0;
  L.f[0] = off; off += L.f_bytes;
  L.f[1] = off; off += L.f_bytes;
  L.adj_f = off; off += L.f_bytes;
  L.lam[0] = off; off += L.f_bytes;
  L.lam[1] = off; off += L.f_bytes;
  L.cos_t = off; off = align_up(off + (size_t)g->n_theta * 8, 256);
  L.sin_t = off; off = align_up(off + (size_t)g->n_theta * 8, 256);
  L.inv_r = off; off = align_up(off + (size_t)g->n_r * 8, 256);
  L.bc_vals = off; off = align_up(off + (size_t)2 * 2 * 4 * g->n_theta * 8, 256);
  L.courant = off; off = align_up(off + (size_t)(g->n_theta + 2 * kGhostRows) * npairs * 16, 256);
  L.courant64 = off; off = align_up(off + (size_t)(g->n_theta + 2 * kGhostRows) * npairs * 32, 256);
  L.inv_r_f = off; off = align_up(off + (size_t)g->n_r * 4, 256);
  L.cs_ff = off; off = align_up(off + (size_t)g->n_theta * 16, 256);
  L.status = off; off = align_up(off + 256, 256);
  L.partials = off; off = align_up(off + (size_t)kDiagBlocks * 8 * 8, 256);
  L.diag_out = off; off = align_up(off + 8 * 8, 256);
  L.stage = off; off = align_up(off + (size_t)8 * g->n_r * g->n_theta * es, 256);
  L.adj_scratch = off; off = align_up(off + adjoint_scratch_bytes(g->n_theta, (int)es), 256);
  L.gen_ghost = off;
  if (d->n_dirs != kNDirs) off = align_up(off + 4 * (size_t)g->n_theta * Q * es, 256);
  L.total = off;
  return L;
}

// Weights of Eq. (11a) as polynomials in E: the numerator is
// sum_n B_n e_{4-n} E^n over the elementary symmetric polynomials e_j of the
// other three shells' squared speeds (e_0 = 1), the denominator
// v_k^2 prod_{l != k} (v_k^2 - v_l^2).
}  // namespace

namespace pclb {
template <class T>
void fill_dvm(DvmConst<T>& c, const pclb_dvm& d, const pclb_grid& g) {
  std::memset(&c, 0, sizeof(c));
  for (int k = 0; k < 5; ++k) {
    const double hv2 = 0.5 * d.speeds[k] * d.speeds[k];
    c.speed[k] = (T)d.speeds[k];
    c.speed_lo[k] = (T)(d.speeds[k] - (double)c.speed[k]);
    c.half_v2[k] = (T)hv2;
    c.half_v2_lo[k] = (T)(hv2 - (double)c.half_v2[k]);
  }
  c.B0 = (T)d.B[0];
  {
    const double dv = d.speeds[3] - d.speeds[2];
    const double dh = 0.5 * (d.speeds[3] * d.speeds[3] - d.speeds[2] * d.speeds[2]);
    c.dv23 = (T)dv;
    c.dv23_lo = (T)(dv - (double)c.dv23);
    c.dh23 = (T)dh;
    c.dh23_lo = (T)(dh - (double)c.dh23);
  }
  for (int k = 1; k <= 4; ++k) {
    const double vk2 = d.speeds[k] * d.speeds[k];
    double o[3];
    int m = 0;
    for (int l = 1; l <= 4; ++l)
      if (l != k) o[m++] = d.speeds[l] * d.speeds[l];
    const double e1 = o[0] + o[1] + o[2];
    const double e2 = o[0] * o[1] + o[1] * o[2] + o[2] * o[0];
    const double e3 = o[0] * o[1] * o[2];
    const double den = vk2 * (vk2 - o[0]) * (vk2 - o[1]) * (vk2 - o[2]);
    const double coef[4] = {d.B[1] * e3 / den, d.B[2] * e2 / den, d.B[3] * e1 / den, d.B[4] / den};
    for (int n = 0; n < 4; ++n) {
      c.Fc[k][n] = (T)coef[n];
      c.Fc_lo[k][n] = (T)(coef[n] - (double)c.Fc[k][n]);
    }
  }
  const int nd = d.n_dirs;
  c.shell[0] = 0;
  c.recv_lo[0] = 0;
  c.recv_hi[0] = 0;
  for (int k = 1; k <= 4; ++k)
    for (int i = 0; i < nd; ++i) {
      const int q = 1 + (k - 1) * nd + i;
      // Unit directions of Eq. (2), taken exactly antisymmetric for opposite
      // directions (i and i + n_dirs/2) as the velocity set is.
      const int ib = i % (nd / 2);
      const double phi = 2.0 * M_PI * ib / nd;
      const double sgn = i < nd / 2 ? 1.0 : -1.0;
      const double cx = sgn * std::cos(phi), cy = sgn * std::sin(phi);
      const double vx = d.speeds[k] * cx, vy = d.speeds[k] * cy;
      c.cx[q] = (T)cx;
      c.cy[q] = (T)cy;
      c.cx_lo[q] = (T)(cx - (double)c.cx[q]);
      c.cy_lo[q] = (T)(cy - (double)c.cy[q]);
      c.vx[q] = (T)vx;
      c.vy[q] = (T)vy;
      c.vx_lo[q] = (T)(vx - (double)c.vx[q]);
      c.vy_lo[q] = (T)(vy - (double)c.vy[q]);
      c.shell[q] = (int8_t)k;
      // Low ghosts of label (k, j) copy rows of label (k, j + n_f); so rows of
      // label (k, i) are received by (k, i - n_f); high ghosts the reverse.
      c.recv_lo[q] = (int8_t)(1 + (k - 1) * nd + ((i - g.n_f) % nd + nd) % nd);
      c.recv_hi[q] = (int8_t)(1 + (k - 1) * nd + (i + g.n_f) % nd);
    }
}
template void fill_dvm<float>(DvmConst<float>&, const pclb_dvm&, const pclb_grid&);

// The same constants in double for N_i = 16, 24 (the generic kernels).
void fill_dvm_generic(DvmG& c, const pclb_dvm& d, const pclb_grid& g) {
  DvmConst<double> base;   // shell-level constants (speeds, weights) as for N_i = 8
  pclb_dvm d8 = d;
  d8.n_dirs = kNDirs;
  pclb_grid g8 = g;
  g8.n_f = kNDirs;
  fill_dvm(base, d8, g8);
  std::memset(&c, 0, sizeof(c));
  for (int k = 0; k < 5; ++k) c.half_v2[k] = base.half_v2[k];
  for (int k = 0; k < 5; ++k)
    for (int n = 0; n < 4; ++n) c.Fc[k][n] = base.Fc[k][n];
  c.B0 = base.B0;
  const int nd = d.n_dirs;
  c.n_dirs = nd;
  c.q = 1 + 4 * nd;
  for (int k = 1; k <= 4; ++k)
    for (int i = 0; i < nd; ++i) {
      const int q = 1 + (k - 1) * nd + i;
      // exactly antisymmetric opposite directions (i and i + n_dirs/2)
      const int ib = i % (nd / 2);
      const double phi = 2.0 * M_PI * ib / nd;
      const double sgn = i < nd / 2 ? 1.0 : -1.0;
      c.vx[q] = d.speeds[k] * sgn * std::cos(phi);
      c.vy[q] = d.speeds[k] * sgn * std::sin(phi);
      c.shell[q] = k;
      c.recv_lo[q] = 1 + (k - 1) * nd + ((i - g.n_f) % nd + nd) % nd;
      c.recv_hi[q] = 1 + (k - 1) * nd + (i + g.n_f) % nd;
    }
}
template void fill_dvm<double>(DvmConst<double>&, const pclb_dvm&, const pclb_grid&);
void set_thread_error(const char* msg) { std::snprintf(g_err, sizeof(g_err), "%s", msg); }
}  // namespace pclb

namespace {

PFN_cuTensorMapEncodeTiled_v12000 get_encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// TMA descriptor of one stored distribution (f or lam layout) at `base`,
// with a box of box_cols columns (kWinR: a stencil window) by box_rows rows
// and one label.
pclb_status encode_map(pclb_ctx* ctx, const void* base, int box_rows, CUtensorMap* out, int box_cols = kWinR) {
  auto enc = get_encode_fn();
  if (!enc) return fail(ctx, PCLB_ECUDA, "cuTensorMapEncodeTiled is not available from the CUDA driver");
  if (reinterpret_cast<uintptr_t>(base) % 16 != 0) return fail(ctx, PCLB_EINVAL, "state buffer not 16-byte aligned");
  const size_t es = elem_size(ctx->prec);
  cuuint64_t dims[3] = {(cuuint64_t)ctx->grid.n_r, (cuuint64_t)ctx->sp.rows, (cuuint64_t)(1 + 4 * ctx->dvm.n_dirs)};
  cuuint64_t strides[2] = {(cuuint64_t)ctx->sp.pitch * es, (cuuint64_t)ctx->sp.pitch * ctx->sp.rows * es};
  cuuint32_t box[3] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(out, ctx->prec == PCLB_FP64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                   3, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(ctx, PCLB_ECUDA, "cuTensorMapEncodeTiled failed (CUresult %d)", (int)r);
  return PCLB_OK;
}

int adj_box_rows(const pclb_ctx* ctx) { return (ctx->prec == PCLB_FP64 ? kAdjRows64 : kAdjRows32) + 4; }

// The node-phase descriptor of the FP32 adjoint: one tile, kTileR x kAdjRows32
// (unused for FP64).
pclb_status encode_node_map(pclb_ctx* ctx, const void* base, CUtensorMap* out) {
  if (ctx->prec != PCLB_FP32) return PCLB_OK;
  return encode_map(ctx, base, kAdjRows32, out, kTileR);
}

pclb_status make_tmap(pclb_ctx* ctx, int which) {
  return encode_map(ctx, ctx->ws + ctx->lay.f[which], ctx->prec == PCLB_FP32 ? kTileT32 + 4 : kWinT,
                    &ctx->tmap[which]);
}

pclb_status bounded_sync(pclb_ctx* ctx, int timeout_ms) {
  cudaEvent_t ev;
  cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaEventCreate");
  e = cudaEventRecord(ev, ctx->stream);
  if (e != cudaSuccess) {
    cudaEventDestroy(ev);
    return cuda_fail(ctx, e, "cudaEventRecord");
  }
  const auto t0 = std::chrono::steady_clock::now();
  pclb_status st = PCLB_OK;
  int sleep_us = 1;
  while (true) {
    e = cudaEventQuery(ev);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) {
      st = cuda_fail(ctx, e, "stream work failed");
      break;
    }
    const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count();
    if (ms > timeout_ms) {
      st = fail(ctx, PCLB_ETIMEOUT, "stream did not finish within %d ms", timeout_ms);
      break;
    }
    std::this_thread::sleep_for(std::chrono::microseconds(sleep_us));
    if (sleep_us < 20) sleep_us *= 2;
  }
  cudaEventDestroy(ev);
  return st;
}

template <class T>
const DvmConst<T>& dvm_of(const pclb_ctx* c);
template <>
const DvmConst<float>& dvm_of<float>(const pclb_ctx* c) { return c->dvm32; }
template <>
const DvmConst<double>& dvm_of<double>(const pclb_ctx* c) { return c->dvm64; }

template <class T>
T* fbuf(pclb_ctx* c, int which) { return reinterpret_cast<T*>(c->ws + c->lay.f[which]); }

pclb_status check_launch(pclb_ctx* ctx, cudaError_t e, const char* what) {
  return e == cudaSuccess ? PCLB_OK : cuda_fail(ctx, e, what);
}

// Caller pointers that kernels dereference element by element must be aligned
// to the element size (a misaligned one would fault on the device): refused
// here with PCLB_EINVAL.
bool misaligned(const pclb_ctx* c, std::initializer_list<const void*> ptrs) {
  const uintptr_t a = c->prec == PCLB_FP32 ? 4 : 8;
  for (const void* p : ptrs)
    if (p && reinterpret_cast<uintptr_t>(p) % a != 0) return true;
  return false;
}
pclb_status misaligned_fail(pclb_ctx* c) {
  return fail(c, PCLB_EINVAL, "pointers must be aligned to the element size (%d bytes)", c->prec == PCLB_FP32 ? 4 : 8);
}

// N_i = 16 or 24: the generic kernels
bool generic(const pclb_ctx* c) { return c->dvm.n_dirs != kNDirs; }

// Captured step graphs depend on the scheme and relaxation (kernel choice and
// parameters): dropped when those change and when the context goes.
void drop_graphs(pclb_ctx* ctx) {
  for (int i = 0; i < ctx->n_graphs; ++i) cudaGraphExecDestroy(ctx->graphs[i].exec);
  ctx->n_graphs = 0;
}

template <class T>
pclb_status do_step(pclb_ctx* ctx, int n) {
  for (int i = 0; i < n; ++i) {
    const int src = ctx->cur, dst = 1 - ctx->cur;
    cudaError_t e;
    if (generic(ctx)) {
      if constexpr (sizeof(T) == 4)
        e = gen_tiled_step_f32(&ctx->tmap[src], fbuf<float>(ctx, src), fbuf<float>(ctx, dst),
                               reinterpret_cast<float*>(ctx->ws + ctx->lay.gen_ghost), ctx->sp, ctx->dvmg,
                               dvmg32(ctx), ctx->stream);
      else
        e = gen_launch_step_f64(fbuf<double>(ctx, src), fbuf<double>(ctx, dst),
                                reinterpret_cast<double*>(ctx->ws + ctx->lay.gen_ghost), ctx->sp, ctx->dvmg,
                                ctx->stream);
    } else if constexpr (sizeof(T) == 4)
      e = launch_step_f32(&ctx->tmap[src], fbuf<float>(ctx, dst), ctx->sp, ctx->dvm32, ctx->stream);
    else
      e = launch_step<T>(&ctx->tmap[src], fbuf<T>(ctx, dst), ctx->sp, dvm_of<T>(ctx), ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "step kernel launch");
    ctx->cur = dst;
  }
  return PCLB_OK;
}

template <class T>
pclb_status do_adjoint(pclb_ctx* ctx, const CUtensorMap* tmap_f, const CUtensorMap* tmap_fn, const void* f) {
  if (!ctx->side) {
    // created on first use: the side stream (highest priority, so that the
    // wall tiles are scheduled as soon as their inputs are ready) and the
    // fork / join events
    int lo = 0, hi = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&ctx->side, cudaStreamNonBlocking, hi);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "adjoint side stream");
  }
  const int src = ctx->cur_lam, dst = 1 - ctx->cur_lam;
  const AdjScratch ws = adjoint_scratch(ctx->ws + ctx->lay.adj_scratch, ctx->grid.n_theta, (int)sizeof(T));
  cudaError_t e = launch_adjoint<T>(tmap_f, &ctx->tmap_adj[3 + src], tmap_fn, &ctx->tmap_node[3 + src],
                                    reinterpret_cast<const T*>(f),
                                    reinterpret_cast<const T*>(ctx->ws + ctx->lay.lam[src]),
                                    reinterpret_cast<T*>(ctx->ws + ctx->lay.lam[dst]), ws, ctx->sp, dvm_of<T>(ctx),
                                    ctx->stream, ctx->side, ctx->ev_fork, ctx->ev_join);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "adjoint kernel launch");
  ctx->cur_lam = dst;
  return PCLB_OK;
}

// ---- pclb_run_host with page-locked host buffers --------------------------
// The grid is cut into S azimuthal slabs of whole tile rows, and five streams
// form a pipeline over them:
//   io_in   copies the input fields of each slab into the staging area, the
//           last slab first (its rows n_theta - 2, n_theta - 1 feed the
//           azimuthal ghost rows that the first slab's step reads);
//   io_set  sets the state of each slab once its fields have landed;
//   stream  (the caller's) and io_alt, alternating by slab: step each slab
//           once its rows and the two rows on either side are set, and
//           compute its moments into the staging area (two streams, so that
//           one slab's step starts while the previous one drains);
//   io_out  copies each slab's moments to the host.
// The transfers run on the copy engines and the set-state kernels beside the
// steps, instead of one after another.  A set-state kernel writes only its
// own slab's rows (and the ghost rows they feed), which no step running at
// the same time reads; the steps of two slabs read set rows and write
// disjoint rows; a moment kernel reads only rows its own step wrote.

void destroy_io(pclb_ctx* ctx) {
  for (cudaStream_t* st : {&ctx->io_in, &ctx->io_set, &ctx->io_out, &ctx->io_alt}) {
    if (*st) cudaStreamDestroy(*st);
    *st = nullptr;
  }
  for (cudaEvent_t* ev : {&ctx->io_start, &ctx->io_done}) {
    if (*ev) cudaEventDestroy(*ev);
    *ev = nullptr;
  }
  for (int s = 0; s < pclb_ctx::kIoSlabs; ++s)
    for (cudaEvent_t* ev : {&ctx->io_loaded[s], &ctx->io_isset[s], &ctx->io_ready[s]}) {
      if (*ev) cudaEventDestroy(*ev);
      *ev = nullptr;
    }
}

pclb_status io_streams(pclb_ctx* ctx) {   // created on first use
  if (ctx->io_in) return PCLB_OK;
  int lo = 0, hi = 0;
  cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->io_in, cudaStreamNonBlocking);
  // the set-state kernels unblock later steps: scheduled first
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&ctx->io_set, cudaStreamNonBlocking, hi);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->io_out, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->io_alt, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->io_start, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->io_done, cudaEventDisableTiming);
  for (int s = 0; s < pclb_ctx::kIoSlabs && e == cudaSuccess; ++s)
    for (cudaEvent_t* ev : {&ctx->io_loaded[s], &ctx->io_isset[s], &ctx->io_ready[s]})
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    destroy_io(ctx);
    return cuda_fail(ctx, e, "host-transfer streams");
  }
  return PCLB_OK;
}

// Number of slabs: about one per 2^17 nodes, at least 2, at most kIoSlabs and
// the number of tile rows.
int io_slab_count(const pclb_ctx* ctx) {
  static_assert(kTileT == kTileT32, "slabs are whole tile rows of either step kernel");
  const long long tiles = (ctx->grid.n_theta + kTileT - 1) / kTileT;
  const long long nodes = (long long)ctx->grid.n_r * ctx->grid.n_theta;
  return (int)std::min(std::min((long long)pclb_ctx::kIoSlabs, tiles), std::max(2ll, nodes >> 17));
}

// First tile rows of the S slabs (bounds[S] = tiles).  With enough tile rows
// the slabs at both ends are smaller (weights 1, 2, 4, ..., 4, 2, 1): the
// first step waits for the first, second and last slab's input, and the call
// ends with the last slabs' moments and copies out.  Every slab has at least
// one tile row.
void io_slab_bounds(int tiles, int S, int* bounds) {
  if (S < 5 || tiles < 4 * S) {
    for (int s = 0; s <= S; ++s) bounds[s] = (int)((long long)s * tiles / S);
    return;
  }
  auto weight = [&](int s) { return (s == 0 || s == S - 1) ? 1 : (s == 1 || s == S - 2) ? 2 : 4; };
  long long total = 0;
  for (int s = 0; s < S; ++s) total += weight(s);
  long long acc = 0;
  for (int s = 0; s < S; ++s) {
    bounds[s] = (int)(acc * tiles / total);
    acc += weight(s);
  }
  bounds[S] = tiles;
}

template <class T>
pclb_status run_host_slabs(pclb_ctx* ctx, const void* const in[4], int n, void* const out[4]) {
  pclb_status st = io_streams(ctx);
  if (st != PCLB_OK) return st;
  const int nt = ctx->grid.n_theta, S = io_slab_count(ctx);
  const int tiles = (nt + kTileT - 1) / kTileT;
  const size_t row_bytes = (size_t)ctx->grid.n_r * sizeof(T), field_bytes = row_bytes * nt;
  unsigned char* stage = ctx->ws + ctx->lay.stage;
  const T* fin[4];
  T* fout[4];
  for (int i = 0; i < 4; ++i) {
    fin[i] = reinterpret_cast<const T*>(stage + i * field_bytes);
    fout[i] = out[i] ? reinterpret_cast<T*>(stage + (4 + i) * field_bytes) : nullptr;
  }
  const bool any_out = out[0] || out[1] || out[2] || out[3];
  cudaStream_t ms = ctx->stream;
  int bounds[pclb_ctx::kIoSlabs + 1];
  io_slab_bounds(tiles, S, bounds);
  auto tile0 = [&](int s) { return bounds[s]; };                         // first tile row of slab s
  auto row0 = [&](int s) { return std::min(tile0(s) * kTileT, nt); };    // first grid row of slab s
  auto slab_of = [&](int t) {                                             // slab of row t (periodic)
    t = ((t % nt) + nt) % nt;
    int s = 0;
    while (t >= row0(s + 1)) ++s;
    return s;
  };
  auto order = [&](int j) { return j == 0 ? S - 1 : j - 1; };   // slabs in the order they are brought in
  auto position = [&](int s) { return s == S - 1 ? 0 : s + 1; };   // inverse of order
  auto cs = [&](int s) { return (s & 1) ? ctx->io_alt : ms; };   // compute stream of slab s
  // the caller's stream waits for everything queued so far on `o`
  auto join = [&](cudaStream_t o) {
    cudaError_t e = cudaEventRecord(ctx->io_done, o);
    return e == cudaSuccess ? cudaStreamWaitEvent(ms, ctx->io_done, 0) : e;
  };
  // on an error: the caller's stream waits for the other four before the
  // error is returned (no copy or kernel of the call outlives it)
  auto bail = [&](pclb_status err) {
    for (cudaStream_t o : {ctx->io_in, ctx->io_set, ctx->io_alt, ctx->io_out}) join(o);
    bounded_sync(ctx, kDefaultTimeoutMs);
    return err;
  };
  auto step = [&](int src, int s) -> cudaError_t {
    if constexpr (sizeof(T) == 4)
      return launch_step_f32(&ctx->tmap[src], fbuf<float>(ctx, 1 - src), ctx->sp, ctx->dvm32, cs(s), tile0(s),
                             tile0(s + 1));
    else
      return launch_step<T>(&ctx->tmap[src], fbuf<T>(ctx, 1 - src), ctx->sp, dvm_of<T>(ctx), cs(s), tile0(s),
                            tile0(s + 1));
  };
  // moments of slab s of buffer b into the staging area (on the slab's
  // compute stream), then their copies to the host on io_out
  auto emit = [&](int b, int s) -> cudaError_t {
    cudaError_t e = launch_moments<T>(fbuf<T>(ctx, b), fout[0], fout[1], fout[2], fout[3], ctx->sp, dvm_of<T>(ctx),
                                      cs(s), row0(s), row0(s + 1));
    if (e == cudaSuccess) e = cudaEventRecord(ctx->io_ready[s], cs(s));
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->io_out, ctx->io_ready[s], 0);
    const size_t off = (size_t)row0(s) * row_bytes, len = (size_t)(row0(s + 1) - row0(s)) * row_bytes;
    for (int i = 0; i < 4 && e == cudaSuccess; ++i)
      if (out[i])
        e = cudaMemcpyAsync(static_cast<unsigned char*>(out[i]) + off, stage + (4 + i) * field_bytes + off, len,
                            cudaMemcpyDeviceToHost, ctx->io_out);
    return e;
  };

  const int src = ctx->cur;
  cudaError_t e = cudaEventRecord(ctx->io_start, ms);   // everything follows earlier work on the stream
  for (cudaStream_t o : {ctx->io_in, ctx->io_set, ctx->io_out, ctx->io_alt})
    if (e == cudaSuccess) e = cudaStreamWaitEvent(o, ctx->io_start, 0);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "host-transfer ordering");
  for (int j = 0; j < S; ++j) {
    const int s = order(j);
    const size_t off = (size_t)row0(s) * row_bytes, len = (size_t)(row0(s + 1) - row0(s)) * row_bytes;
    for (int i = 0; i < 4 && e == cudaSuccess; ++i)
      e = cudaMemcpyAsync(stage + i * field_bytes + off, static_cast<const unsigned char*>(in[i]) + off, len,
                          cudaMemcpyHostToDevice, ctx->io_in);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->io_loaded[s], ctx->io_in);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->io_set, ctx->io_loaded[s], 0);
    if (e == cudaSuccess)
      e = launch_set_state<T>(fbuf<T>(ctx, src), fin[0], fin[1], fin[2], fin[3], ctx->sp, dvm_of<T>(ctx),
                              ctx->io_set, row0(s), row0(s + 1));
    if (e == cudaSuccess) e = cudaEventRecord(ctx->io_isset[s], ctx->io_set);
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "input copy or set_state launch"));
  }

  // the first step slab by slab, each after the set-state kernels of the
  // slabs its stencil reaches (the latest of them in io_set's order); when it
  // is also the last step (or n = 0), each slab's moments follow at once
  for (int c = 0; c < S; ++c) {
    int last = position(c);
    if (n >= 1) {
      const int a = row0(c), b = row0(c + 1);
      for (int t : {a - 2, a - 1, b, b + 1}) last = std::max(last, position(slab_of(t)));
    }
    e = cudaStreamWaitEvent(cs(c), ctx->io_isset[order(last)], 0);
    if (e == cudaSuccess && n >= 1) e = step(src, c);
    if (e == cudaSuccess && n <= 1 && any_out) e = emit(n == 0 ? src : 1 - src, c);
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "step, moments or output copy"));
  }
  ctx->has_state = true;
  if (n >= 1) ctx->cur = 1 - src;
  if (n >= 2) {
    // the steps in between on the whole grid (after every slab's first
    // step), the last one slab by slab again
    if ((e = join(ctx->io_set)) != cudaSuccess || (e = join(ctx->io_alt)) != cudaSuccess)
      return bail(cuda_fail(ctx, e, "host-transfer ordering"));
    if ((st = do_step<T>(ctx, n - 2)) != PCLB_OK) return bail(st);
    e = cudaEventRecord(ctx->io_start, ms);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->io_alt, ctx->io_start, 0);
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "host-transfer ordering"));
    const int s2 = ctx->cur;
    for (int c = 0; c < S; ++c) {
      if ((e = step(s2, c)) != cudaSuccess) return bail(cuda_fail(ctx, e, "step kernel launch"));
      if (any_out && (e = emit(1 - s2, c)) != cudaSuccess) return bail(cuda_fail(ctx, e, "moments or output copy"));
    }
    ctx->cur = 1 - s2;
  }
  // the caller's stream takes up everything: later calls see the new state
  for (cudaStream_t o : {ctx->io_set, ctx->io_alt, ctx->io_out})
    if (e == cudaSuccess) e = join(o);
  if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "host-transfer ordering"));
  return bounded_sync(ctx, kDefaultTimeoutMs);
}

}  // namespace

extern "C" {

int32_t pclb_version(void) { return PCLB_VERSION_MAJOR * 100 + PCLB_VERSION_MINOR; }

const char* pclb_last_error(const pclb_ctx* ctx) { return ctx ? ctx->err : g_err; }

pclb_status pclb_workspace_size(const pclb_grid* grid, const pclb_dvm* dvm, pclb_precision prec,
                                size_t* bytes) {
  if (!bytes) return fail(nullptr, PCLB_EINVAL, "bytes must not be NULL");
  pclb_status st = validate(grid, dvm, prec);
  if (st != PCLB_OK) return st;
  *bytes = make_layout(grid, dvm, prec).total;
  return PCLB_OK;
}

pclb_status pclb_create(const pclb_grid* grid, const pclb_dvm* dvm, double tau, double dt,
                        pclb_precision prec, const pclb_bc* bc, void* workspace,
                        size_t workspace_bytes, void* stream, pclb_ctx** out) {
  if (!out) return fail(nullptr, PCLB_EINVAL, "out must not be NULL");
  *out = nullptr;
  pclb_status st = validate(grid, dvm, prec);
  if (st != PCLB_OK) return st;
  if (!(tau > 0.0) || !std::isfinite(tau)) return fail(nullptr, PCLB_EINVAL, "tau must be positive (got %g)", tau);
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(nullptr, PCLB_EINVAL, "dt must be positive (got %g)", dt);
  if (!bc) return fail(nullptr, PCLB_EINVAL, "bc must not be NULL");
  for (int s = 0; s < 2; ++s) {
    const int base = bc->kind[s] & ~PCLB_BC_NEQ;
    if (base < PCLB_BC_EXTRAP || base > PCLB_BC_DIRICHLET)
      return fail(nullptr, PCLB_EINVAL, "bc kind[%d] = %d is unknown", s, bc->kind[s]);
    if (base != PCLB_BC_EXTRAP && !bc->values[s])
      return fail(nullptr, PCLB_EINVAL, "bc values[%d] must be given for kind %d", s, bc->kind[s]);
  }
  if (!workspace) return fail(nullptr, PCLB_EINVAL, "workspace must not be NULL");
  if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0)
    return fail(nullptr, PCLB_EINVAL, "workspace must be 256-byte aligned");
  const Layout lay = make_layout(grid, dvm, prec);
  if (workspace_bytes < lay.total)
    return fail(nullptr, PCLB_ENOMEM, "workspace has %zu bytes, %zu needed", workspace_bytes, lay.total);

  const int NR = grid->n_r, NT = grid->n_theta;
  const double dr = (grid->r_out - grid->r_in) / (NR - 1);
  const double dth = 2.0 * M_PI * grid->n_f / ((double)dvm->n_dirs * NT);

  // Courant numbers: the largest |C_r| + |C_theta| over labels and nodes
  // (C_theta is largest at the inner wall).
  double cmax = 0.0;
  for (int t = 0; t < NT; ++t) {
    const double th = (t + 1) * dth, c = std::cos(th), s = std::sin(th);
    for (int k = 1; k <= 4; ++k)
      for (int i = 0; i < dvm->n_dirs; ++i) {
        const double phi = 2.0 * M_PI * i / dvm->n_dirs;
        const double vx = dvm->speeds[k] * std::cos(phi), vy = dvm->speeds[k] * std::sin(phi);
        const double cr = std::fabs(vx * c + vy * s) * dt / dr;
        const double ct = std::fabs(-vx * s + vy * c) * dt / (grid->r_in * dth);
        cmax = std::fmax(cmax, cr + ct);
      }
  }
  if (cmax > 1.0)
    return fail(nullptr, PCLB_ECFL, "max |C_r| + |C_theta| = %g exceeds 1 (dt too large)", cmax);

  HostCtx* ctx = new (std::nothrow) HostCtx();
  if (!ctx) return fail(nullptr, PCLB_EINVAL, "out of host memory");
  ctx->grid = *grid;
  ctx->dvm = *dvm;
  ctx->prec = prec;
  ctx->tau = tau;
  ctx->dt = dt;
  ctx->bc_kind[0] = bc->kind[0];
  ctx->bc_kind[1] = bc->kind[1];
  ctx->stream = reinterpret_cast<cudaStream_t>(stream);
  ctx->ws = reinterpret_cast<unsigned char*>(workspace);
  ctx->lay = lay;
  ctx->cur = 0;
  ctx->has_state = false;
  ctx->err[0] = 0;

  ctx->cos_t.resize(NT);
  ctx->sin_t.resize(NT);
  for (int t = 0; t < NT; ++t) {
    const double th = (t + 1) * dth;
    ctx->cos_t[t] = std::cos(th);
    ctx->sin_t[t] = std::sin(th);
  }
  ctx->inv_r.resize(NR);
  for (int r = 0; r < NR; ++r) ctx->inv_r[r] = 1.0 / (grid->r_in + r * dr);
  // Courant table: for every stored row (theta node t = row - 2, including the
  // two ghost rows on each side at theta = (t + 1) dtheta outside the period)
  // and every pair of opposite velocities (first label q = 1 + (k-1) N_i + i,
  // i < N_i / 2).
  const int npairs = 4 * dvm->n_dirs / 2;
  const int nrows = NT + 2 * kGhostRows;
  ctx->courant.resize((size_t)nrows * npairs * 4);
  ctx->courant64.resize((size_t)nrows * npairs * 4);
  for (int t = 0; t < nrows; ++t)
    for (int k = 1; k <= 4; ++k)
      for (int i = 0; i < dvm->n_dirs / 2; ++i) {
        const double phi = 2.0 * M_PI * i / dvm->n_dirs;
        const double vx = dvm->speeds[k] * std::cos(phi), vy = dvm->speeds[k] * std::sin(phi);
        const double th = (t - kGhostRows + 1) * dth;
        const double ct = t >= kGhostRows && t < NT + kGhostRows ? ctx->cos_t[t - kGhostRows] : std::cos(th);
        const double st = t >= kGhostRows && t < NT + kGhostRows ? ctx->sin_t[t - kGhostRows] : std::sin(th);
        const double vr = vx * ct + vy * st;
        const double vt = vy * ct - vx * st;
        const double ar = std::fabs(vr) * dt / dr;
        float* e = ctx->courant.data() + ((size_t)t * npairs + (k - 1) * (dvm->n_dirs / 2) + i) * 4;
        e[0] = (float)ar;
        e[1] = (float)(ar * (1.0 - ar));
        e[2] = (float)(std::fabs(vt) * dt / dth);
        const int flags = (vr < 0.0 ? 1 : 0) | (vt < 0.0 ? 2 : 0);
        std::memcpy(&e[3], &flags, 4);
        double* e64 = ctx->courant64.data() + ((size_t)t * npairs + (k - 1) * (dvm->n_dirs / 2) + i) * 4;
        e64[0] = ar;
        e64[1] = ar * (1.0 - ar);
        e64[2] = std::fabs(vt) * dt / dth;
        e64[3] = (double)flags;
      }
  ctx->inv_r_f.resize(NR);
  for (int r = 0; r < NR; ++r) ctx->inv_r_f[r] = (float)ctx->inv_r[r];
  // cos and sin as float-float pairs for the FP32 field kernels' rotations
  ctx->cs_ff.resize((size_t)NT * 4);
  for (int t = 0; t < NT; ++t) {
    const double cs[2] = {ctx->cos_t[t], ctx->sin_t[t]};
    for (int j = 0; j < 2; ++j) {
      const float hi = (float)cs[j];
      ctx->cs_ff[(size_t)t * 4 + 2 * j] = hi;
      ctx->cs_ff[(size_t)t * 4 + 2 * j + 1] = (float)(cs[j] - (double)hi);
    }
  }
  ctx->bc_vals.assign((size_t)2 * 2 * 4 * NT, 0.0);
  for (int s = 0; s < 2; ++s)
    if ((bc->kind[s] & ~PCLB_BC_NEQ) != PCLB_BC_EXTRAP)
      std::memcpy(ctx->bc_vals.data() + (size_t)s * 2 * 4 * NT, bc->values[s], sizeof(double) * 2 * 4 * NT);

  StepParams& sp = ctx->sp;
  sp.n_r = NR;
  sp.n_theta = NT;
  sp.pitch = (int)align_up((size_t)NR, kPitchAlign);
  sp.rows = NT + 2 * kGhostRows;
  sp.dt_dr = dt / dr;
  sp.dt_dth = dt / dth;
  sp.decay = std::exp(-dt / tau);
  sp.scheme = PCLB_SCHEME_MWB;
  sp.wait_ns = kDefaultWaitNs;
  sp.bc_kind[0] = bc->kind[0];
  sp.bc_kind[1] = bc->kind[1];
  sp.cos_t = reinterpret_cast<const double*>(ctx->ws + lay.cos_t);
  sp.sin_t = reinterpret_cast<const double*>(ctx->ws + lay.sin_t);
  sp.inv_r = reinterpret_cast<const double*>(ctx->ws + lay.inv_r);
  sp.bc_vals = reinterpret_cast<const double*>(ctx->ws + lay.bc_vals);
  sp.courant = reinterpret_cast<const float4*>(ctx->ws + lay.courant);
  sp.courant64 = reinterpret_cast<const double*>(ctx->ws + lay.courant64);
  sp.inv_r_f = reinterpret_cast<const float*>(ctx->ws + lay.inv_r_f);
  sp.cs_ff = reinterpret_cast<const float4*>(ctx->ws + lay.cs_ff);
  sp.status = reinterpret_cast<uint32_t*>(ctx->ws + lay.status);
  if (dvm->n_dirs == kNDirs) {
    fill_dvm(ctx->dvm32, *dvm, *grid);
    fill_dvm(ctx->dvm64, *dvm, *grid);
  } else {
    fill_dvm_generic(ctx->dvmg, *dvm, *grid);
    fill_dvm_generic32(ctx->dvmg32, *dvm, ctx->dvmg);
  }

  struct Up { size_t off; const void* src; size_t n; } ups[] = {
      {lay.cos_t, ctx->cos_t.data(), NT * 8ul}, {lay.sin_t, ctx->sin_t.data(), NT * 8ul},
      {lay.inv_r, ctx->inv_r.data(), NR * 8ul}, {lay.bc_vals, ctx->bc_vals.data(), ctx->bc_vals.size() * 8},
      {lay.courant, ctx->courant.data(), ctx->courant.size() * 4},
      {lay.courant64, ctx->courant64.data(), ctx->courant64.size() * 8}, {lay.inv_r_f, ctx->inv_r_f.data(), NR * 4ul},
      {lay.cs_ff, ctx->cs_ff.data(), NT * 16ul}};
  for (const Up& u : ups) {
    cudaError_t e = cudaMemcpyAsync(ctx->ws + u.off, u.src, u.n, cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) {
      pclb_status s2 = cuda_fail(nullptr, e, "table upload");
      delete ctx;
      return s2;
    }
  }
  cudaError_t e = cudaMemsetAsync(ctx->ws + lay.status, 0, 256, ctx->stream);
  if (e != cudaSuccess) {
    pclb_status s2 = cuda_fail(nullptr, e, "status reset");
    delete ctx;
    return s2;
  }
  ctx->cur_lam = 0;
  ctx->has_lam = false;
  const size_t adj_bufs[5] = {lay.f[0], lay.f[1], lay.adj_f, lay.lam[0], lay.lam[1]};
  for (int w = 0; w < 7; ++w) {
    pclb_status s2 = w < 2 ? make_tmap(ctx, w)
                           : encode_map(ctx, ctx->ws + adj_bufs[w - 2], adj_box_rows(ctx), &ctx->tmap_adj[w - 2]);
    if (s2 == PCLB_OK && w >= 2) s2 = encode_node_map(ctx, ctx->ws + adj_bufs[w - 2], &ctx->tmap_node[w - 2]);
    if (s2 != PCLB_OK) {
      std::snprintf(g_err, sizeof(g_err), "%s", ctx->err);
      delete ctx;
      return s2;
    }
  }
  *out = ctx;
  return PCLB_OK;
}

pclb_status pclb_destroy(pclb_ctx* ctx) {
  if (!ctx) return PCLB_OK;
  pclb_status st = bounded_sync(ctx, kDefaultTimeoutMs);
  if (st != PCLB_OK) std::snprintf(g_err, sizeof(g_err), "%s", ctx->err);
  drop_graphs(ctx);
  if (ctx->capture) cudaStreamDestroy(ctx->capture);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  if (ctx->side) cudaStreamDestroy(ctx->side);
  destroy_io(ctx);
  delete static_cast<HostCtx*>(ctx);
  return st;
}

pclb_status pclb_set_stream(pclb_ctx* ctx, void* stream) {
  if (!ctx) return fail(nullptr, PCLB_EINVAL, "ctx must not be NULL");
  ctx->stream = reinterpret_cast<cudaStream_t>(stream);
  return PCLB_OK;
}

pclb_status pclb_set_state(pclb_ctx* ctx, const void* rho, const void* u_r, const void* u_theta,
                           const void* T) {
  if (!ctx) return fail(nullptr, PCLB_EINVAL, "ctx must not be NULL");
  if (misaligned(ctx, {rho, u_r, u_theta, T})) return misaligned_fail(ctx);
  if (!rho || !u_r || !u_theta || !T) return fail(ctx, PCLB_EINVAL, "field pointers must not be NULL");
  cudaError_t e;
  if (generic(ctx) && ctx->prec == PCLB_FP32)
    e = gen_launch_set_state<float>(fbuf<float>(ctx, ctx->cur), (const float*)rho, (const float*)u_r,
                                    (const float*)u_theta, (const float*)T, ctx->sp, ctx->dvmg, ctx->stream);
  else if (generic(ctx))
    e = gen_launch_set_state<double>(fbuf<double>(ctx, ctx->cur), (const double*)rho, (const double*)u_r,
                                     (const double*)u_theta, (const double*)T, ctx->sp, ctx->dvmg, ctx->stream);
  else if (ctx->prec == PCLB_FP32)
    e = launch_set_state<float>(fbuf<float>(ctx, ctx->cur), (const float*)rho, (const float*)u_r,
                                (const float*)u_theta, (const float*)T, ctx->sp, ctx->dvm32, ctx->stream);
  else
    e = launch_set_state<double>(fbuf<double>(ctx, ctx->cur), (const double*)rho, (const double*)u_r,
                                 (const double*)u_theta, (const double*)T, ctx->sp, ctx->dvm64, ctx->stream);
  pclb_status st = check_launch(ctx, e, "set_state kernel launch");
  if (st == PCLB_OK) ctx->has_state = true;
  return st;
}

pclb_status pclb_set_f(pclb_ctx* ctx, const void* f) {
  if (!ctx) return fail(nullptr, PCLB_EINVAL, "ctx must not be NULL");
  if (misaligned(ctx, {f})) return misaligned_fail(ctx);
  if (!f) return fail(ctx, PCLB_EINVAL, "f must not be NULL");
  cudaError_t e;
  if (generic(ctx))
    e = ctx->prec == PCLB_FP32
            ? gen_launch_unpack<float>((const float*)f, fbuf<float>(ctx, ctx->cur), ctx->sp, ctx->dvmg, ctx->stream)
            : gen_launch_unpack<double>((const double*)f, fbuf<double>(ctx, ctx->cur), ctx->sp, ctx->dvmg, ctx->stream);
  else
    e = ctx->prec == PCLB_FP32
            ? launch_unpack<float>((const float*)f, fbuf<float>(ctx, ctx->cur), ctx->sp, ctx->dvm32, ctx->stream)
            : launch_unpack<double>((const double*)f, fbuf<double>(ctx, ctx->cur), ctx->sp, ctx->dvm64, ctx->stream);
  pclb_status st = check_launch(ctx, e, "set_f kernel launch");
  if (st == PCLB_OK) ctx->has_state = true;
  return st;
}

pclb_status pclb_get_f(pclb_ctx* ctx, void* f) {
  if (!ctx) return fail(nullptr, PCLB_EINVAL, "ctx must not be NULL");
  if (misaligned(ctx, {f})) return misaligned_fail(ctx);
  if (!f) return fail(ctx, PCLB_EINVAL, "f must not be NULL");
  if (!ctx->has_state) return fail(ctx, PCLB_ESTATE, "no state: call pclb_set_state or pclb_set_f first");
  cudaError_t e;
  if (generic(ctx))
    e = ctx->prec == PCLB_FP32
            ? gen_launch_pack<float>(fbuf<float>(ctx, ctx->cur), (float*)f, ctx->sp, ctx->dvmg, ctx->stream)
            : gen_launch_pack<double>(fbuf<double>(ctx, ctx->cur), (double*)f, ctx->sp, ctx->dvmg, ctx->stream);
  else
    e = ctx->prec == PCLB_FP32
            ? launch_pack<float>(fbuf<float>(ctx, ctx->cur), (float*)f, ctx->sp, ctx->stream)
            : launch_pack<double>(fbuf<double>(ctx, ctx->cur), (double*)f, ctx->sp, ctx->stream);
  return check_launch(ctx, e, "get_f kernel launch");
}

pclb_status pclb_step(pclb_ctx* ctx, int32_t n) {
  if (!ctx) return fail(nullptr, PCLB_EINVAL, "ctx must not be NULL");
  if (n < 0) return fail(ctx, PCLB_EINVAL, "n = %d must be >= 0", n);
  if (!ctx->has_state) return fail(ctx, PCLB_ESTATE, "no state: call pclb_set_state or pclb_set_f first");
  return ctx->prec == PCLB_FP32 ? do_step<float>(ctx, n) : do_step<double>(ctx, n);
}

pclb_status pclb_step_states(pclb_ctx* ctx, const void* f_from, void* f_to) {
  if (!ctx) return fail(nullptr, PCLB_EINVAL, "ctx must not be NULL");
  if (!f_from || !f_to) return fail(ctx, PCLB_EINVAL, "f_from and f_to must not be NULL");
  if (f_from == f_to) return fail(ctx, PCLB_EINVAL, "f_from and f_to must be different buffers");
  if ((reinterpret_cast<uintptr_t>(f_from) | reinterpret_cast<uintptr_t>(f_to)) % 16 != 0)
    return fail(ctx, PCLB_EINVAL, "state buffers must be 16-byte aligned");
  cudaError_t e;
  if (generic(ctx) && ctx->prec == PCLB_FP32) {
    CUtensorMap map;
    pclb_status st = encode_map(ctx, f_from, kTileT32 + 4, &map);
    if (st != PCLB_OK) return st;
    e = gen_tiled_step_f32(&map, (const float*)f_from, (float*)f_to,
                           reinterpret_cast<float*>(ctx->ws + ctx->lay.gen_ghost), ctx->sp, ctx->dvmg, dvmg32(ctx),
                           ctx->stream);
  } else if (generic(ctx)) {
    e = gen_launch_step_f64((const double*)f_from, (double*)f_to,
                            reinterpret_cast<double*>(ctx->ws + ctx->lay.gen_ghost), ctx->sp, ctx->dvmg,
                            ctx->stream);
  } else {
    CUtensorMap map;
    pclb_status st = encode_map(ctx, f_from, ctx->prec == PCLB_FP32 ? kTileT32 + 4 : kWinT, &map);
    if (st != PCLB_OK) return st;
    e = ctx->prec == PCLB_FP32 ? launch_step_f32(&map, (float*)f_to, ctx->sp, ctx->dvm32, ctx->stream)
                               : launch_step<double>(&map, (double*)f_to, ctx->sp, ctx->dvm64, ctx->stream);
  }
  return e == cudaSuccess ? PCLB_OK : cuda_fail(ctx, e, "step kernel launch");
}

pclb_status pclb_step_graph(pclb_ctx* ctx, int32_t n) {
  if (!ctx) return fail(nullptr, PCLB_EINVAL, "ctx must not be NULL");
  if (n < 0) return fail(ctx, PCLB_EINVAL, "n = %d must be >= 0", n);
  if (!ctx->has_state) return fail(ctx, PCLB_ESTATE, "no state: call pclb_set_state or pclb_set_f first");
  if (n == 0) return PCLB_OK;
  const int cur = ctx->cur;
  cudaGraphExec_t exec = nullptr;
  for (int i = 0; i < ctx->n_graphs; ++i)
    if (ctx->graphs[i].n == n && ctx->graphs[i].cur == cur) exec = ctx->graphs[i].exec;
  if (!exec) {
    // capture the n launches on a private stream (nothing runs), then keep
    // the instantiated graph for this (n, starting buffer)
    cudaError_t e = cudaSuccess;
    if (!ctx->capture) e = cudaStreamCreateWithFlags(&ctx->capture, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "capture stream");
    cudaStream_t user = ctx->stream;
    ctx->stream = ctx->capture;
    e = cudaStreamBeginCapture(ctx->capture, cudaStreamCaptureModeRelaxed);
    pclb_status st = PCLB_OK;
    if (e == cudaSuccess) st = ctx->prec == PCLB_FP32 ? do_step<float>(ctx, n) : do_step<double>(ctx, n);
    cudaGraph_t graph = nullptr;
    const cudaError_t e_end = e == cudaSuccess ? cudaStreamEndCapture(ctx->capture, &graph) : e;
    ctx->stream = user;
    ctx->cur = cur;
    if (e != cudaSuccess || e_end != cudaSuccess || st != PCLB_OK) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return st != PCLB_OK ? st : cuda_fail(ctx, e != cudaSuccess ? e : e_end, "step graph capture");
    }
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "step graph instantiation");
    if (ctx->n_graphs == 4) {   // drop the oldest
      cudaGraphExecDestroy(ctx->graphs[0].exec);
      for (int i = 1; i < 4; ++i) ctx->graphs[i - 1] = ctx->graphs[i];
      ctx->n_graphs = 3;
    }
    ctx->graphs[ctx->n_graphs++] = {n, cur, exec};
  }
  cudaError_t e = cudaGraphLaunch(exec, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "step graph launch");
  ctx->cur = (cur + n) & 1;
  return PCLB_OK;
}

pclb_status pclb_moments(pclb_ctx* ctx, void* rho, void* u_r, void* u_theta, void* T) {
  if (!ctx) return fail(nullptr, PCLB_EINVAL, "ctx must not be NULL");
  if (misaligned(ctx, {rho, u_r, u_theta, T})) return misaligned_fail(ctx);
  if (!ctx->has_state) return fail(ctx, PCLB_ESTATE, "no state: call pclb_set_state or pclb_set_f first");
  if (!rho && !u_r && !u_theta && !T) return PCLB_OK;
  cudaError_t e;
  if (generic(ctx) && ctx->prec == PCLB_FP32)
    e = gen_launch_moments<float>(fbuf<float>(ctx, ctx->cur), (float*)rho, (float*)u_r, (float*)u_theta,
                                  (float*)T, ctx->sp, ctx->dvmg, ctx->stream);
  else if (generic(ctx))
    e = gen_launch_moments<double>(fbuf<double>(ctx, ctx->cur), (double*)rho, (double*)u_r, (double*)u_theta,
                                   (double*)T, ctx->sp, ctx->dvmg, ctx->stream);
  else if (ctx->prec == PCLB_FP32)
    e = launch_moments<float>(fbuf<float>(ctx, ctx->cur), (float*)rho, (float*)u_r, (float*)u_theta,
                              (float*)T, ctx->sp, ctx->dvm32, ctx->stream);
  else
    e = launch_moments<double>(fbuf<double>(ctx, ctx->cur), (double*)rho, (double*)u_r, (double*)u_theta,
                               (double*)T, ctx->sp, ctx->dvm64, ctx->stream);
  return check_launch(ctx, e, "moments kernel launch");
}

pclb_status pclb_noneq(pclb_ctx* ctx, int32_t groups, void* out) {
  if (!ctx) return fail(nullptr, PCLB_EINVAL, "ctx must not be NULL");
  if (misaligned(ctx, {out})) return misaligned_fail(ctx);
  if (groups < 1 || groups > 15) return fail(ctx, PCLB_EINVAL, "groups = %d must be in 1..15", (int)groups);
  if (!out) return fail(ctx, PCLB_EINVAL, "out must not be NULL");
  if (!ctx->has_state) return fail(ctx, PCLB_ESTATE, "no state: call pclb_set_state or pclb_set_f first");
  cudaError_t e;
  if (generic(ctx))
    e = ctx->prec == PCLB_FP32
            ? launch_noneq_gen<float>(fbuf<float>(ctx, ctx->cur), (float*)out, groups, ctx->sp, ctx->dvmg,
                                      dvmg32(ctx), ctx->stream)
            : launch_noneq_gen<double>(fbuf<double>(ctx, ctx->cur), (double*)out, groups, ctx->sp, ctx->dvmg,
                                       dvmg32(ctx), ctx->stream);
  else if (ctx->prec == PCLB_FP32)
    e = launch_noneq<float>(fbuf<float>(ctx, ctx->cur), (float*)out, groups, ctx->sp, ctx->dvm32, ctx->stream);
  else
    e = launch_noneq<double>(fbuf<double>(ctx, ctx->cur), (double*)out, groups, ctx->sp, ctx->dvm64,
                             ctx->stream);
  return check_launch(ctx, e, "noneq kernel launch");
}

pclb_status pclb_diagnostics(pclb_ctx* ctx, double* out) {
  if (!ctx) return fail(nullptr, PCLB_EINVAL, "ctx must not be NULL");
  if (!out) return fail(ctx, PCLB_EINVAL, "out must not be NULL");
  if (!ctx->has_state) return fail(ctx, PCLB_ESTATE, "no state: call pclb_set_state or pclb_set_f first");
  const double dr = (ctx->grid.r_out - ctx->grid.r_in) / (ctx->grid.n_r - 1);
  const double dth = 2.0 * M_PI * ctx->grid.n_f / ((double)ctx->dvm.n_dirs * ctx->grid.n_theta);
  double* partials = reinterpret_cast<double*>(ctx->ws + ctx->lay.partials);
  double* dout = reinterpret_cast<double*>(ctx->ws + ctx->lay.diag_out);
  cudaError_t e;
  if (generic(ctx))
    e = ctx->prec == PCLB_FP32 ? gen_launch_diagnostics<float>(fbuf<float>(ctx, ctx->cur), partials, dout, ctx->sp,
                                                               ctx->dvmg, dr, dth, ctx->grid.r_in, ctx->stream)
                               : gen_launch_diagnostics<double>(fbuf<double>(ctx, ctx->cur), partials, dout,
                                                                ctx->sp, ctx->dvmg, dr, dth, ctx->grid.r_in,
                                                                ctx->stream);
  else
    e = ctx->prec == PCLB_FP32 ? launch_diagnostics<float>(fbuf<float>(ctx, ctx->cur), partials, dout, ctx->sp,
                                                           ctx->dvm32, dr, dth, ctx->grid.r_in, ctx->stream)
                               : launch_diagnostics<double>(fbuf<double>(ctx, ctx->cur), partials, dout, ctx->sp,
                                                            ctx->dvm64, dr, dth, ctx->grid.r_in, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "diagnostics kernel launch");
  pclb_status st = bounded_sync(ctx, kDefaultTimeoutMs);
  if (st != PCLB_OK) return st;
  e = cudaMemcpy(out, dout, 8 * sizeof(double), cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? PCLB_OK : cuda_fail(ctx, e, "diagnostics copy");
}

pclb_status pclb_status_flags(pclb_ctx* ctx, uint32_t* flags, int32_t clear) {
  if (!ctx) return fail(nullptr, PCLB_EINVAL, "ctx must not be NULL");
  if (!flags) return fail(ctx, PCLB_EINVAL, "flags must not be NULL");
  pclb_status st = bounded_sync(ctx, kDefaultTimeoutMs);
  if (st != PCLB_OK) return st;
  cudaError_t e = cudaMemcpy(flags, ctx->ws + ctx->lay.status, sizeof(uint32_t), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "status copy");
  if (clear) {
    e = cudaMemset(ctx->ws + ctx->lay.status, 0, sizeof(uint32_t));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "status reset");
  }
  if (*flags & PCLB_FLAG_TIMEOUT) return fail(ctx, PCLB_ETIMEOUT, "a kernel timed out waiting for its copies");
  if (*flags) return fail(ctx, PCLB_ENONPHYS, "non-physical state (flags 0x%x)", *flags);
  return PCLB_OK;
}

pclb_status pclb_sync(pclb_ctx* ctx, int32_t timeout_ms) {
  if (!ctx) return fail(nullptr, PCLB_EINVAL, "ctx must not be NULL");
  if (timeout_ms <= 0) return fail(ctx, PCLB_EINVAL, "timeout_ms must be positive");
  return bounded_sync(ctx, timeout_ms);
}

pclb_status pclb_run_host(pclb_ctx* ctx, const void* rho, const void* u_r, const void* u_theta,
                          const void* T, int32_t n, void* out_rho, void* out_u_r, void* out_u_theta,
                          void* out_T) {
  if (!ctx) return fail(nullptr, PCLB_EINVAL, "ctx must not be NULL");
  if (!rho || !u_r || !u_theta || !T) return fail(ctx, PCLB_EINVAL, "input pointers must not be NULL");
  if (n < 0) return fail(ctx, PCLB_EINVAL, "n = %d must be >= 0", n);
  // Page-locked host buffers (the tuned kernels): transfers slab by slab on
  // copy streams, overlapped with the kernels; other host memory goes
  // through staging copies in stream order.
  if (!generic(ctx)) {
    const void* ptrs[8] = {rho, u_r, u_theta, T, out_rho, out_u_r, out_u_theta, out_T};
    bool pinned = true;
    for (int i = 0; i < 8 && pinned; ++i) {
      if (!ptrs[i]) continue;
      cudaPointerAttributes a;
      if (cudaPointerGetAttributes(&a, ptrs[i]) != cudaSuccess) {
        cudaGetLastError();
        pinned = false;
      } else {
        pinned = a.type == cudaMemoryTypeHost;
      }
    }
    if (pinned) {
      const void* in[4] = {rho, u_r, u_theta, T};
      void* out[4] = {out_rho, out_u_r, out_u_theta, out_T};
      return ctx->prec == PCLB_FP32 ? run_host_slabs<float>(ctx, in, n, out) : run_host_slabs<double>(ctx, in, n, out);
    }
  }
  const size_t bytes = (size_t)ctx->grid.n_r * ctx->grid.n_theta * elem_size(ctx->prec);
  unsigned char* stage = ctx->ws + ctx->lay.stage;
  const void* in[4] = {rho, u_r, u_theta, T};
  for (int i = 0; i < 4; ++i) {
    cudaError_t e = cudaMemcpyAsync(stage + i * bytes, in[i], bytes, cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "input copy");
  }
  pclb_status st = pclb_set_state(ctx, stage, stage + bytes, stage + 2 * bytes, stage + 3 * bytes);
  if (st != PCLB_OK) return st;
  if ((st = pclb_step(ctx, n)) != PCLB_OK) return st;
  void* outs[4] = {out_rho, out_u_r, out_u_theta, out_T};
  void* dev[4];
  for (int i = 0; i < 4; ++i) dev[i] = outs[i] ? stage + (4 + i) * bytes : nullptr;
  if ((st = pclb_moments(ctx, dev[0], dev[1], dev[2], dev[3])) != PCLB_OK) return st;
  for (int i = 0; i < 4; ++i) {
    if (!outs[i]) continue;
    cudaError_t e = cudaMemcpyAsync(outs[i], dev[i], bytes, cudaMemcpyDeviceToHost, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "output copy");
  }
  return bounded_sync(ctx, kDefaultTimeoutMs);
}

pclb_status pclb_state_bytes(pclb_ctx* ctx, size_t* bytes) {
  if (!ctx || !bytes) return fail(ctx, PCLB_EINVAL, "ctx and bytes must not be NULL");
  *bytes = ctx->lay.f_bytes;
  return PCLB_OK;
}

pclb_status pclb_save_state(pclb_ctx* ctx, void* state) {
  if (!ctx) return fail(nullptr, PCLB_EINVAL, "ctx must not be NULL");
  if (!state) return fail(ctx, PCLB_EINVAL, "state must not be NULL");
  if (!ctx->has_state) return fail(ctx, PCLB_ESTATE, "no state: call pclb_set_state or pclb_set_f first");
  cudaError_t e = cudaMemcpyAsync(state, ctx->ws + ctx->lay.f[ctx->cur], ctx->lay.f_bytes, cudaMemcpyDeviceToDevice,
                                  ctx->stream);
  return e == cudaSuccess ? PCLB_OK : cuda_fail(ctx, e, "state copy");
}

pclb_status pclb_load_state(pclb_ctx* ctx, const void* state) {
  if (!ctx) return fail(nullptr, PCLB_EINVAL, "ctx must not be NULL");
  if (!state) return fail(ctx, PCLB_EINVAL, "state must not be NULL");
  cudaError_t e = cudaMemcpyAsync(ctx->ws + ctx->lay.f[ctx->cur], state, ctx->lay.f_bytes, cudaMemcpyDeviceToDevice,
                                  ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "state copy");
  ctx->has_state = true;
  return PCLB_OK;
}

pclb_status pclb_lambda_set(pclb_ctx* ctx, const void* lam) {
  if (!ctx) return fail(nullptr, PCLB_EINVAL, "ctx must not be NULL");
  if (misaligned(ctx, {lam})) return misaligned_fail(ctx);
  if (generic(ctx)) return fail(ctx, PCLB_EUNSUPPORTED, "reverse mode implements n_dirs = 8 only");
  if (!lam) return fail(ctx, PCLB_EINVAL, "lam must not be NULL");
  void* dst = ctx->ws + ctx->lay.lam[ctx->cur_lam];
  cudaError_t e = ctx->prec == PCLB_FP32
                      ? launch_unpack<float>((const float*)lam, (float*)dst, ctx->sp, ctx->dvm32, ctx->stream)
                      : launch_unpack<double>((const double*)lam, (double*)dst, ctx->sp, ctx->dvm64, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "lambda unpack launch");
  ctx->has_lam = true;
  return PCLB_OK;
}

pclb_status pclb_lambda_get(pclb_ctx* ctx, void* lam) {
  if (!ctx) return fail(nullptr, PCLB_EINVAL, "ctx must not be NULL");
  if (misaligned(ctx, {lam})) return misaligned_fail(ctx);
  if (generic(ctx)) return fail(ctx, PCLB_EUNSUPPORTED, "reverse mode implements n_dirs = 8 only");
  if (!lam) return fail(ctx, PCLB_EINVAL, "lam must not be NULL");
  if (!ctx->has_lam) return fail(ctx, PCLB_ESTATE, "no adjoint variable: call pclb_lambda_set or pclb_moments_vjp");
  const void* src = ctx->ws + ctx->lay.lam[ctx->cur_lam];
  cudaError_t e = ctx->prec == PCLB_FP32 ? launch_pack<float>((const float*)src, (float*)lam, ctx->sp, ctx->stream)
                                         : launch_pack<double>((const double*)src, (double*)lam, ctx->sp, ctx->stream);
  return e == cudaSuccess ? PCLB_OK : cuda_fail(ctx, e, "lambda pack launch");
}

// The adjoint differentiates the MWB increments and the ghost nodes of every
// wall kind (f = f^eq of the ghost state, plus the wall node's departure for
// non-equilibrium ghosts); the comparison schemes are forward-only.
static pclb_status adjoint_supported(pclb_ctx* ctx) {
  if (generic(ctx)) return fail(ctx, PCLB_EUNSUPPORTED, "reverse mode implements n_dirs = 8 only");
  if (ctx->scheme != PCLB_SCHEME_MWB)
    return fail(ctx, PCLB_EUNSUPPORTED, "the adjoint supports the MWB scheme only (scheme %d)", ctx->scheme);
  return PCLB_OK;
}

pclb_status pclb_set_scheme(pclb_ctx* ctx, int32_t scheme, int32_t relaxation) {
  if (!ctx) return fail(nullptr, PCLB_EINVAL, "ctx must not be NULL");
  if (scheme < PCLB_SCHEME_MWB || scheme > PCLB_SCHEME_UPWIND2)
    return fail(ctx, PCLB_EINVAL, "scheme = %d is unknown", scheme);
  if (relaxation != PCLB_RELAX_EXACT && relaxation != PCLB_RELAX_EULER)
    return fail(ctx, PCLB_EINVAL, "relaxation = %d is unknown", relaxation);
  if (relaxation == PCLB_RELAX_EULER && ctx->dt > 2.0 * ctx->tau)
    return fail(ctx, PCLB_ECFL, "forward-Euler relaxation is unstable for dt / tau = %g > 2", ctx->dt / ctx->tau);
  drop_graphs(ctx);
  ctx->scheme = scheme;
  ctx->relaxation = relaxation;
  ctx->sp.scheme = scheme;
  ctx->sp.decay = relaxation == PCLB_RELAX_EULER ? 1.0 - ctx->dt / ctx->tau : std::exp(-ctx->dt / ctx->tau);
  return PCLB_OK;
}

pclb_status pclb_set_wait_limit(pclb_ctx* ctx, uint64_t limit_ns) {
  if (!ctx) return fail(nullptr, PCLB_EINVAL, "ctx must not be NULL");
  if (limit_ns > kMaxWaitNs) return fail(ctx, PCLB_EINVAL, "limit_ns must be at most %llu", (unsigned long long)kMaxWaitNs);
  drop_graphs(ctx);   // captured launches hold the old parameters
  ctx->sp.wait_ns = limit_ns;
  return PCLB_OK;
}

pclb_status pclb_adjoint_state(pclb_ctx* ctx, const void* f_state) {
  if (!ctx) return fail(nullptr, PCLB_EINVAL, "ctx must not be NULL");
  if (f_state && reinterpret_cast<uintptr_t>(f_state) % 16 != 0)
    return fail(ctx, PCLB_EINVAL, "f_state must be 16-byte aligned");
  if (adjoint_supported(ctx) != PCLB_OK) return PCLB_EUNSUPPORTED;
  if (!ctx->has_lam) return fail(ctx, PCLB_ESTATE, "no adjoint variable: call pclb_lambda_set or pclb_moments_vjp");
  const CUtensorMap *map, *node_map;
  CUtensorMap local, local_node;
  const void* f = f_state;
  if (f_state == nullptr) {
    if (!ctx->has_state) return fail(ctx, PCLB_ESTATE, "no state: call pclb_set_state or pclb_set_f first");
    map = &ctx->tmap_adj[ctx->cur];
    node_map = &ctx->tmap_node[ctx->cur];
    f = ctx->ws + ctx->lay.f[ctx->cur];
  } else {
    pclb_status st = encode_map(ctx, f_state, adj_box_rows(ctx), &local);
    if (st == PCLB_OK) st = encode_node_map(ctx, f_state, &local_node);
    if (st != PCLB_OK) return st;
    map = &local;
    node_map = &local_node;
  }
  return ctx->prec == PCLB_FP32 ? do_adjoint<float>(ctx, map, node_map, f) : do_adjoint<double>(ctx, map, node_map, f);
}

pclb_status pclb_adjoint_step(pclb_ctx* ctx, const void* f_n, const void* lam_np1, void* lam_n) {
  if (!ctx) return fail(nullptr, PCLB_EINVAL, "ctx must not be NULL");
  if (misaligned(ctx, {f_n, lam_np1, lam_n})) return misaligned_fail(ctx);
  if (adjoint_supported(ctx) != PCLB_OK) return PCLB_EUNSUPPORTED;
  if (!f_n || !lam_np1 || !lam_n) return fail(ctx, PCLB_EINVAL, "f_n, lam_np1 and lam_n must not be NULL");
  void* adj = ctx->ws + ctx->lay.adj_f;
  cudaError_t e = ctx->prec == PCLB_FP32
                      ? launch_unpack<float>((const float*)f_n, (float*)adj, ctx->sp, ctx->dvm32, ctx->stream)
                      : launch_unpack<double>((const double*)f_n, (double*)adj, ctx->sp, ctx->dvm64, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "state unpack launch");
  pclb_status st = pclb_lambda_set(ctx, lam_np1);
  if (st != PCLB_OK) return st;
  st = ctx->prec == PCLB_FP32 ? do_adjoint<float>(ctx, &ctx->tmap_adj[2], &ctx->tmap_node[2], adj)
                               : do_adjoint<double>(ctx, &ctx->tmap_adj[2], &ctx->tmap_node[2], adj);
  if (st != PCLB_OK) return st;
  return pclb_lambda_get(ctx, lam_n);
}

pclb_status pclb_moments_vjp(pclb_ctx* ctx, const void* g_rho, const void* g_ur, const void* g_ut, const void* g_T) {
  if (!ctx) return fail(nullptr, PCLB_EINVAL, "ctx must not be NULL");
  if (misaligned(ctx, {g_rho, g_ur, g_ut, g_T})) return misaligned_fail(ctx);
  if (generic(ctx)) return fail(ctx, PCLB_EUNSUPPORTED, "reverse mode implements n_dirs = 8 only");
  if (!ctx->has_state) return fail(ctx, PCLB_ESTATE, "no state: call pclb_set_state or pclb_set_f first");
  void* lam = ctx->ws + ctx->lay.lam[ctx->cur_lam];
  const void* f = ctx->ws + ctx->lay.f[ctx->cur];
  cudaError_t e;
  if (ctx->prec == PCLB_FP32)
    e = launch_moments_vjp<float>((const float*)f, (const float*)g_rho, (const float*)g_ur, (const float*)g_ut,
                                  (const float*)g_T, (float*)lam, ctx->sp, ctx->dvm32, ctx->stream);
  else
    e = launch_moments_vjp<double>((const double*)f, (const double*)g_rho, (const double*)g_ur,
                                   (const double*)g_ut, (const double*)g_T, (double*)lam, ctx->sp, ctx->dvm64,
                                   ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "moments vjp launch");
  ctx->has_lam = true;
  return PCLB_OK;
}

pclb_status pclb_set_state_vjp(pclb_ctx* ctx, const void* rho, const void* u_r, const void* u_theta, const void* T,
                               void* g_rho, void* g_ur, void* g_ut, void* g_T) {
  if (!ctx) return fail(nullptr, PCLB_EINVAL, "ctx must not be NULL");
  if (misaligned(ctx, {rho, u_r, u_theta, T, g_rho, g_ur, g_ut, g_T})) return misaligned_fail(ctx);
  if (generic(ctx)) return fail(ctx, PCLB_EUNSUPPORTED, "reverse mode implements n_dirs = 8 only");
  if (!rho || !u_r || !u_theta || !T) return fail(ctx, PCLB_EINVAL, "field pointers must not be NULL");
  if (!ctx->has_lam) return fail(ctx, PCLB_ESTATE, "no adjoint variable: call pclb_lambda_set first");
  const void* lam = ctx->ws + ctx->lay.lam[ctx->cur_lam];
  cudaError_t e;
  if (ctx->prec == PCLB_FP32)
    e = launch_set_state_vjp<float>((const float*)rho, (const float*)u_r, (const float*)u_theta, (const float*)T,
                                    (const float*)lam, (float*)g_rho, (float*)g_ur, (float*)g_ut, (float*)g_T, ctx->sp,
                                    ctx->dvm32, ctx->stream);
  else
    e = launch_set_state_vjp<double>((const double*)rho, (const double*)u_r, (const double*)u_theta,
                                     (const double*)T, (const double*)lam, (double*)g_rho, (double*)g_ur,
                                     (double*)g_ut, (double*)g_T, ctx->sp, ctx->dvm64, ctx->stream);
  return e == cudaSuccess ? PCLB_OK : cuda_fail(ctx, e, "set_state vjp launch");
}

}  // extern "C"
