// Single-pass fused step (declared here; the row-window kernel follows).
#pragma once

#include "lbm.h"
#include "lbm_common.cuh"

namespace lbm {

template <typename T>
inline bool fused_supported(const Geo&, const Phys&) {
  return false;
}

template <typename T>
inline lbm_status launch_fused(const Geo&, const Phys&, const T*, T*, const uint16_t*, int, cudaStream_t) {
  return LBM_ERR_STATE;
}

}  // namespace lbm
