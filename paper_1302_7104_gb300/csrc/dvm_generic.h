// Float tables of the N_i = 16 and 24 velocity sets (Table I) for the FP32
// generic step, beside the double constants of DvmG.
#pragma once

#include "pclb.h"
#include "pclb_internal.h"

namespace pclb {

constexpr int kMaxPairsG = kMaxQ / 8;   // N_i / 2 <= 12 opposite-direction pairs per shell

struct DvmG32 {
  float vx[kMaxQ], vy[kMaxQ];                  // v_q rounded to float
  float cxh[kMaxPairsG], cxl[kMaxPairsG];      // unit vector of direction i < N_i / 2 (Eq. 2) as
  float cyh[kMaxPairsG], cyl[kMaxPairsG];      //   float-float pairs (hi, lo)
  double speed[5], half_v2[5];                 // v_k and v_k^2 / 2
  double dv23, dh23;                           // v_3 - v_2 and (v_3^2 - v_2^2) / 2
};

void fill_dvm_generic32(DvmG32& c, const pclb_dvm& d);

}  // namespace pclb
