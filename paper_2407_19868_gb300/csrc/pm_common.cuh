// Shared device definitions of the GB300 permeability solver.
//
// Grid and unknowns (Sec. 4, "Grid"): MAC grid, p at cell centres, u_d on the +d face of
// each cell, fields stored as separate arrays [nz][ny][nx] (x fastest).  A face node
// u_d(c) is fluid iff cells c and c+e_d are both pore; the other nodes are
// no-penetration faces and hold exactly 0 in every buffer, so a stencil may read them
// without testing the mask.
//
// Neighbourhood flags (Algorithm 1, "Evaluate neighborhood"), one byte per cell:
//   bit 0  cell c is pore
//   bit 1  node u_x(c) is fluid, bit 2 node u_y(c), bit 3 node u_z(c)
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pmgb {

constexpr int kFlagCell = 1;
__host__ __device__ constexpr int node_bit(int d) { return 2 << d; }

// Stencil code word of a cell (computed once per geometry by code_kernel):
//   bit 0        cell is pore
//   bits 1..3    node u_x, u_y, u_z fluid
//   bits 4..21   3-bit wall code of node u_d across axis i at bit code_shift(d, i):
//                kind (bits 0-1) and side (bit 2) of the Appendix B case
//                  kind 0  case 6, both neighbours fluid      u(-1) + u(+1) - 2 u0
//                  kind 1  case 1, walls at -1/2 and +1/2     -8 u0
//                  kind 2  cases 4/5, one wall, node at +-2   2 u(+-1) - 5 u0 - u(+-2) / 5
//                  kind 3  cases 2/3, one wall, no node at +-2 (8 u(+-1) - 16 u0) / 3
//                  side 1  the fluid side is + (cases 2, 4); 0 otherwise
//                The two codes of node u_d are adjacent: a 6-bit field at bit
//                node_shift(d), the lower perpendicular axis in its low 3 bits.
__host__ __device__ constexpr int node_shift(int d) { return 4 + 6 * d; }
__host__ __device__ constexpr int code_shift(int d, int i) {
    return node_shift(d) + (i == (d == 0 ? 1 : 0) ? 0 : 3);
}

// Transposed stencil code of a cell (adjoint solves; tcode_kernel), two words per cell.
// The transpose of the wall stencil gathers, for node a along axis i, the coefficients
// that its neighbours b = a + m e_i (|m| <= 2) apply to a.  Per node u_d and
// perpendicular axis i an 8-bit slot (slot index tslot(d, i), word slot / 4, bit
// 8 (slot % 4)):
//   bits 0-1  wall kind of a itself (its diagonal coefficient)
//   bits 2-3  wall kind of the node at -1 (its coefficient on a, which is its
//             coefficient on both of its +-1 neighbours)
//   bits 4-5  wall kind of the node at +1
//   bit 6     the node at -2 is a case 4/5 node whose far node is +2 (coefficient -1/5)
//   bit 7     the node at +2 is a case 4/5 node whose far node is -2 (coefficient -1/5)
__host__ __device__ constexpr int tslot(int d, int i) { return 2 * d + (i == (d == 0 ? 1 : 0) ? 0 : 1); }

// Sweep variants.  The fused sweep works on the staggered state (u^n, p^{n-1}): it first
// forms p^n = p^{n-1} - dt c^2 (D u^n - r_p) on the cells it needs, then
// u^{n+1} = u^n + dt R_u(u^n, p^n).  This is exactly the paper's order (velocity update,
// then pressure update with the new velocity) regrouped so that one pass reads each
// field once: the pressure of iteration n is finished in the pass that also does the
// velocity of iteration n+1.
enum SweepMode : int {
    kModeU = 1,   // u^{1} from (u^0, p^0); p copied (first iteration)
    kModePU = 2,  // p^n from (u^n, p^{n-1}), then u^{n+1}
    kModeP = 3    // p^n only (last half-step, brings p level with u)
};

template <typename T>
struct SweepProblem {
    const T *uin;    // 3N
    const T *pin;    // N
    T *uout;         // 3N
    T *pout;         // N
    const T *src;    // 4N source (r_u x3, r_p) or nullptr
    T f[3];          // body force per face direction (the drive)
    T pres[2];       // fixed-pressure axis: inlet and outlet reservoir pressures
    double *partials;  // [nblocks][4] block sums (q_x, q_y, q_z, |div|^2) or nullptr
    // geometry of this problem (multi-geometry batches; otherwise equal to the batch's)
    const uint32_t *code;
    int nx, ny, nz, zchunk;
    int tiles_x, tiles_y;
    long long unit_begin;  // first CTA of this problem in a multi-geometry launch
};

// Problems per sweep launch: up to kMaxSame drives on one geometry, or up to kMaxBatch
// (geometry, drive) problems in a multi-geometry batch.
constexpr int kMaxSame = 4;
constexpr int kMaxBatch = 64;

template <typename T>
struct SweepBatch {
    int nx, ny, nz;
    int per[3];            // 1 = periodic axis, 0 = wall (outside counts as solid)
    long long N;
    const uint8_t *flags;  // N
    const uint32_t *code;  // N stencil codes (wall cases), used by the transposed sweep
    const uint32_t *tcode; // [N][2] transposed stencil codes (tiled transposed sweep)
    const T *alpha;        // N per-cell drag or nullptr
    T inv_re, dt, dtc2;
    int nprob;
    int multi;             // 1: problems have their own geometry (tiled kernel, one unit per CTA)
    const int *active;     // device, per problem, 0 = skip (converged); nullptr = all active
    int pres_axis;         // fixed-pressure axis + 1 (reservoir layers 0 and n - 1); 0 = none
    int zsplit;            // chunked tiled schedules: sub-chunks of each column's last plane
                           // chunk (split_last in pm_sweep_tiled.cuh); 1 = none
    SweepProblem<T> prob[kMaxBatch];
};

// Neighbour coordinate v (= x + m, |m| <= 2) on an axis of n cells: periodic wrap, or -1
// outside a wall axis.
__device__ __forceinline__ int nb_coord(int v, int n, int periodic) {
    if (v < 0) {
        if (!periodic) return -1;
        do { v += n; } while (v < 0);
    } else if (v >= n) {
        if (!periodic) return -1;
        do { v -= n; } while (v >= n);
    }
    return v;
}

}  // namespace pmgb
