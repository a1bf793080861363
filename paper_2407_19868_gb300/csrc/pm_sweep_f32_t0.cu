// Instantiation of the tiled sweep for float fields, tile shape 1 (64 x 12 cells, pairs
// of cells per thread), in its own translation unit so that the shapes compile in
// parallel.
#include "pm_sweep_pair.cuh"

namespace pmgb {

cudaError_t launch_tiled_f32_t0(const SweepBatch<float> &B, const uint32_t *code, int mode, bool red, bool src,
                                int zchunk, cudaStream_t s) {
    return pair::launch_pair<float>(B, code, mode, red, src, zchunk, s);
}

}  // namespace pmgb
