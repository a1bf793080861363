// Tiled z-marching fused sweep (placeholder: the simple kernel serves every shape).
#pragma once

#include "pm_common.cuh"

namespace pmgb {

template <typename T>
inline bool tiled_supported(int, int, int, int) { return false; }

template <typename T>
inline long long tiled_num_blocks(int, int, int) { return 0; }

template <typename T>
inline int launch_tiled(const SweepBatch<T> &, int, bool, bool, cudaStream_t) { return 9; }

}  // namespace pmgb
