// Float tables of the N_i = 16 and 24 velocity sets (Table I) for their FP32
// step (dvm_tiled32.cu), beside the double constants of DvmG; and the entry
// points of the steps of these sets.
#pragma once

#include "pclb.h"
#include "pclb_internal.h"

namespace pclb {

constexpr int kMaxPairsG = kMaxQ / 8;   // N_i / 2 <= 12 opposite-direction pairs per shell

// Float-float constants are pairs (h, l) with h + l the double value.
struct DvmG32 {
  float vx[kMaxQ], vy[kMaxQ];                  // v_q rounded to float
  float cxh[kMaxPairsG], cxl[kMaxPairsG];      // unit vector of direction i < N_i / 2 (Eq. 2)
  float cyh[kMaxPairsG], cyl[kMaxPairsG];
  float sph[5], spl[5], hvh[5], hvl[5];        // v_k and v_k^2 / 2
  float dv23h, dv23l, dh23h, dh23l;            // v_3 - v_2 and (v_3^2 - v_2^2) / 2
  float Fch[5][4], Fcl[5][4];                  // F_k(E) = sum_n Fc[k][n-1] E^n (Eq. 11a)
  float B0h, B0l;                              // F_0 = 1 - B0 sum_k F_k (Eq. 11b)
};

void fill_dvm_generic32(DvmG32& c, const pclb_dvm& d, const DvmG& g);

// One FP64 step of the N_i = 16 or 24 set (dvm_generic.cu): the radial ghost
// layers into ghost [side][layer][n_theta][Q], then one thread per node.
cudaError_t gen_launch_step_f64(const double* f, double* f_out, double* ghost, const StepParams& p, const DvmG& d,
                                cudaStream_t s);

// One FP32 step of the N_i = 16 or 24 set: its radial ghost layers into
// ghost [side][layer][n_theta][Q], then the tiled kernel; tmap describes f
// (box kWinR x (kTileT32 + 4) x 1 over Q planes).
cudaError_t gen_tiled_step_f32(const CUtensorMap* tmap, const float* f, float* f_out, float* ghost,
                               const StepParams& p, const DvmG& d, const DvmG32& c, cudaStream_t s);

}  // namespace pclb
