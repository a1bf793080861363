// Instantiation of the transposed tiled sweep (adjoint solves) for float fields, tile
// shape 64 x 12 cells, four per thread, in its own translation unit.
#include "pm_sweep_tiled.cuh"

namespace pmgb {

cudaError_t launch_tiled_f32_tr(const SweepBatch<float> &B, const uint32_t *code, int mode, bool red, int zchunk,
                                cudaStream_t s) {
    return launch_tiled_tr<float, Tile64x12c4tr>(B, code, mode, red, zchunk, kTileTR, s);
}

}  // namespace pmgb
