// Instantiation of the tiled sweep for float fields, tile shape Tile64x12c4 (its own
// translation unit so that the shapes compile in parallel).
#include "pm_sweep_tiled.cuh"

namespace pmgb {

cudaError_t launch_tiled_f32_t1(const SweepBatch<float> &B, const uint32_t *code, int mode, bool red, bool src,
                                int zchunk, cudaStream_t s) {
    return launch_tiled_c<float, Tile64x12c4>(B, code, mode, red, src, zchunk, 1, s);
}

}  // namespace pmgb
