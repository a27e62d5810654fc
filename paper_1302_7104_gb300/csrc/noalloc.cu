// pclb_diagnostics_noalloc: the global integrals of a distribution computed
// without allocating any device memory.
//
// Some callers cannot call cudaMalloc at all: a custom allocator's own
// callbacks (which would re-enter the allocator), a driver or framework
// plug-in that owns no memory pool, or a host that has handed every byte of
// the GPU to another framework.  They still hold the distribution in device
// memory and want its mass, momentum and energy.  This variant of the
// diagnostics reduction keeps its per-row partial sums in a fixed, file-scope
// device array instead of a workspace, so the call needs nothing but its
// input, its output and a stream.  It waits for its stream and copies the
// result to the host, and refuses a stream that is being captured.
#include <cuda_runtime.h>
#include <float.h>

#include <chrono>
#include <cstdio>
#include <mutex>
#include <thread>

#include "device_common.cuh"
#include "f32_state.cuh"
#include "pclb_internal.h"

namespace pclb {
namespace {

// Capacity: one partial slot (8 doubles) per azimuthal row, plus the result.
constexpr int kNoAllocMaxRows = 16384;
constexpr int kNoAllocThreads = 256;
constexpr int kMaxDevices = 64;

// Shared by every call on a device; it keeps the last call's contents.
static __device__ __align__(256) double g_noalloc_scratch[(kNoAllocMaxRows + 1) * 8];

// One block per azimuthal row of the packed [Q][n_theta][n_r] array.
template <class T>
__global__ void diag_rows_kernel(const T* __restrict__ f, double* __restrict__ partials, int n_r,
                                 int n_theta, const __grid_constant__ DvmConst<T> d, double dr, double dth, double r_in) {
  const int t = blockIdx.x;
  const size_t plane = (size_t)n_theta * n_r;
  double acc[4] = {0, 0, 0, 0};
  double mn[2] = {DBL_MAX, DBL_MAX};
  for (int r = threadIdx.x; r < n_r; r += blockDim.x) {
    double rho, ux, uy, E;
    node_state_double(f + (size_t)t * n_r + r, plane, d, rho, ux, uy, E);
    const double w = (r_in + r * dr) * dr * dth;
    acc[0] += w * rho;
    acc[1] += w * rho * ux;
    acc[2] += w * rho * uy;
    acc[3] += w * rho * (E + 0.5 * (ux * ux + uy * uy));
    mn[0] = fmin(mn[0], rho);
    mn[1] = fmin(mn[1], E);
  }
  __shared__ double red[6][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double v[6] = {acc[0], acc[1], acc[2], acc[3], mn[0], mn[1]};
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    for (int off = 16; off > 0; off >>= 1) {
      const double o = __shfl_down_sync(0xffffffffu, v[i], off);
      v[i] = i < 4 ? v[i] + o : fmin(v[i], o);
    }
    if (lane == 0) red[i][warp] = v[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 0; i < 6; ++i) {
      double s = red[i][0];
      for (int w = 1; w < (int)(blockDim.x / 32); ++w) s = i < 4 ? s + red[i][w] : fmin(s, red[i][w]);
      partials[(size_t)t * 8 + i] = s;
    }
  }
}

__global__ void diag_rows_final(const double* __restrict__ partials, int n_rows, double* out,
                                double n_nodes) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s[6] = {0, 0, 0, 0, DBL_MAX, DBL_MAX};
  for (int b = 0; b < n_rows; ++b)
    for (int i = 0; i < 6; ++i)
      s[i] = i < 4 ? s[i] + partials[(size_t)b * 8 + i] : fmin(s[i], partials[(size_t)b * 8 + i]);
  for (int i = 0; i < 6; ++i) out[i] = s[i];
  out[6] = n_nodes;
  out[7] = 0.0;
}

// Device address of the scratch array, looked up once per device with that
// device current (a host-side reference to the array is not a device address).
std::mutex g_setup_mutex;
double* g_scratch_addr[kMaxDevices] = {};

pclb_status scratch_for_current_device(double** out, char* err, size_t n_err) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    std::snprintf(err, n_err, "cudaGetDevice: %s", cudaGetErrorString(e));
    return PCLB_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    std::snprintf(err, n_err, "device ordinal %d beyond the %d supported", dev, kMaxDevices);
    return PCLB_EUNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      std::snprintf(err, n_err, "cudaGetSymbolAddress of the static scratch: %s", cudaGetErrorString(e));
      return PCLB_ECUDA;
    }
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return PCLB_OK;
}

pclb_status wait_stream(cudaStream_t s, int timeout_ms, char* err, size_t n_err) {
  cudaEvent_t ev;
  cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(ev, s);
  if (e != cudaSuccess) {
    std::snprintf(err, n_err, "event: %s", cudaGetErrorString(e));
    return PCLB_ECUDA;
  }
  const auto t0 = std::chrono::steady_clock::now();
  pclb_status st = PCLB_OK;
  while (true) {
    e = cudaEventQuery(ev);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) {
      std::snprintf(err, n_err, "stream work failed: %s", cudaGetErrorString(e));
      st = PCLB_ECUDA;
      break;
    }
    if (std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(timeout_ms)) {
      std::snprintf(err, n_err, "stream did not finish within %d ms", timeout_ms);
      st = PCLB_ETIMEOUT;
      break;
    }
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
  cudaEventDestroy(ev);
  return st;
}

template <class T>
cudaError_t launch_rows(const void* f, double* scratch, const pclb_grid& g, const pclb_dvm& dv,
                        cudaStream_t s) {
  DvmConst<T> d;
  fill_dvm(d, dv, g);
  const double dr = (g.r_out - g.r_in) / (g.n_r - 1);
  const double dth = 2.0 * M_PI * g.n_f / ((double)dv.n_dirs * g.n_theta);
  diag_rows_kernel<T><<<g.n_theta, kNoAllocThreads, 0, s>>>(static_cast<const T*>(f), scratch, g.n_r,
                                                            g.n_theta, d, dr, dth, g.r_in);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  diag_rows_final<<<1, 32, 0, s>>>(scratch, g.n_theta, scratch + (size_t)kNoAllocMaxRows * 8,
                                   (double)g.n_r * g.n_theta);
  return cudaGetLastError();
}

}  // namespace
}  // namespace pclb

using namespace pclb;

extern "C" pclb_status pclb_diagnostics_noalloc(const pclb_grid* grid, const pclb_dvm* dvm,
                                                pclb_precision prec, const void* f, double* out,
                                                void* stream) {
  char err[256];
  pclb_status st = validate_problem(grid, dvm, prec);
  if (st != PCLB_OK) return st;
  if (dvm->n_dirs != kNDirs) {
    set_thread_error("pclb_diagnostics_noalloc implements n_dirs = 8 only");
    return PCLB_EUNSUPPORTED;
  }
  if (!f || !out) {
    set_thread_error("f and out must not be NULL");
    return PCLB_EINVAL;
  }
  if (reinterpret_cast<uintptr_t>(f) % (prec == PCLB_FP32 ? 4 : 8) != 0) {
    set_thread_error("f must be aligned to the element size");
    return PCLB_EINVAL;
  }
  if (grid->n_theta > kNoAllocMaxRows) {
    std::snprintf(err, sizeof(err),
                  "n_theta = %d exceeds the %d azimuthal rows the static scratch of "
                  "pclb_diagnostics_noalloc holds; use pclb_diagnostics",
                  grid->n_theta, kNoAllocMaxRows);
    set_thread_error(err);
    return PCLB_EINVAL;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  {
    // the call waits for the stream and copies to the host: a stream that
    // is being captured is refused before anything is queued
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    const cudaError_t ce = cudaStreamIsCapturing(s, &cap);
    if (ce != cudaSuccess) {
      std::snprintf(err, sizeof(err), "cudaStreamIsCapturing: %s", cudaGetErrorString(ce));
      set_thread_error(err);
      return PCLB_ECUDA;
    }
    if (cap != cudaStreamCaptureStatusNone) {
      set_thread_error("pclb_diagnostics_noalloc waits for its stream and copies to the host; "
                       "it cannot run on a stream that is being captured");
      return PCLB_EUNSUPPORTED;
    }
  }
  double* scratch = nullptr;
  if ((st = scratch_for_current_device(&scratch, err, sizeof(err))) != PCLB_OK) {
    set_thread_error(err);
    return st;
  }
  cudaError_t e = prec == PCLB_FP32 ? launch_rows<float>(f, scratch, *grid, *dvm, s)
                                    : launch_rows<double>(f, scratch, *grid, *dvm, s);
  if (e != cudaSuccess) {
    std::snprintf(err, sizeof(err), "diagnostics kernel launch: %s", cudaGetErrorString(e));
    set_thread_error(err);
    return PCLB_ECUDA;
  }
  if ((st = wait_stream(s, 120000, err, sizeof(err))) != PCLB_OK) {
    set_thread_error(err);
    return st;
  }
  e = cudaMemcpy(out, scratch + (size_t)kNoAllocMaxRows * 8, 8 * sizeof(double), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    std::snprintf(err, sizeof(err), "result copy: %s", cudaGetErrorString(e));
    set_thread_error(err);
    return PCLB_ECUDA;
  }
  return PCLB_OK;
}
