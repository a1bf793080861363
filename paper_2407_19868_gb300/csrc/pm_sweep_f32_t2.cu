// Instantiation of the tiled sweep for float fields, tile shape Tile64x8c4 (its own
// translation unit so that the shapes compile in parallel).
#include "pm_sweep_tiled.cuh"

namespace pmgb {

cudaError_t launch_tiled_f32_t2(const SweepBatch<float> &B, const uint32_t *code, int mode, bool red, bool src,
                                int zchunk, cudaStream_t s) {
    return launch_tiled_c<float, Tile64x8c4>(B, code, mode, red, src, zchunk, 2, s);
}

}  // namespace pmgb
