// Tiled z-marching fused sweep.
//
// A CTA owns a TX x TY column tile of the (x, y) plane and marches along z over a chunk
// of planes.  Each plane of the five input arrays (u_x, u_y, u_z, p, stencil code) is
// copied with its 2-voxel halo into a 6-stage shared-memory ring by cp.async, three
// planes ahead of use, so each field value comes from DRAM once per sweep and the
// neighbour reuse is served by shared memory (x, y) and per-thread register queues (z).
//
// Per step t the CTA
//   reads plane t of its own column into the z queues,
//   forms p^n on plane t-1 (own cells and the +x / +y halo cells),
//   updates u on plane t-2 with p^n of planes t-2 and t-1 and writes u^{n+1}, p^n.
// The neighbourhood (Algorithm 1, "Evaluate neighborhood") is precomputed once per
// geometry as one 32-bit code per cell (code_kernel), so the sweep reads no mask
// neighbours at all.
#pragma once

#include "pm_common.cuh"

namespace pmgb {

// ------------------------------------------------------------------ stencil codes
// bit 0          cell is pore
// bits 1..3      node u_x, u_y, u_z fluid
// 3-bit fields   wall case of node u_d along perpendicular axis i (Appendix B), stored as
//                kind (bits 0-1) and side (bit 2):
//                  kind 0  case 6, both neighbours fluid      u(-1) + u(+1) - 2 u0
//                  kind 1  case 1, walls at -1/2 and +1/2     -8 u0
//                  kind 2  cases 4/5, one wall, node at +-2   2 u(+-1) - 5 u0 - u(+-2) / 5
//                  kind 3  cases 2/3, one wall, no node at +-2 (8 u(+-1) - 16 u0) / 3
//                  side 1  the fluid side is + (cases 2, 4); 0 otherwise
__host__ __device__ constexpr int code_shift(int d, int i) {
    return d == 0 ? (i == 1 ? 4 : 7) : d == 1 ? (i == 0 ? 10 : 13) : (i == 0 ? 16 : 19);
}

__device__ __forceinline__ bool cell_pore(const uint8_t *mask, int x, int y, int z, int nx, int ny, int nz,
                                          const int per[3]) {
    x = nb_coord(x, nx, per[0]);
    y = nb_coord(y, ny, per[1]);
    z = nb_coord(z, nz, per[2]);
    if (x < 0 || y < 0 || z < 0) return false;
    return mask[(long long)x + (long long)nx * ((long long)y + (long long)ny * z)] == 0;
}

__device__ __forceinline__ bool node_fluid_at(const uint8_t *mask, int d, int x, int y, int z, int nx, int ny,
                                              int nz, const int per[3]) {
    // coordinates may be up to 3 cells outside; wrap / wall handled per axis
    if (!cell_pore(mask, x, y, z, nx, ny, nz, per)) return false;
    return cell_pore(mask, x + (d == 0), y + (d == 1), z + (d == 2), nx, ny, nz, per);
}

__global__ void code_kernel(const uint8_t *__restrict__ mask, int nx, int ny, int nz, int px, int py, int pz,
                            uint32_t *__restrict__ code) {
    const int per[3] = {px, py, pz};
    const long long N = (long long)nx * ny * nz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(c % nx);
        const long long r = c / nx;
        const int y = (int)(r % ny), z = (int)(r / ny);
        uint32_t w = 0;
        if (mask[c] == 0) {
            w |= 1u;
            for (int d = 0; d < 3; ++d) {
                if (!node_fluid_at(mask, d, x, y, z, nx, ny, nz, per)) continue;
                w |= (uint32_t)node_bit(d);
                for (int i = 0; i < 3; ++i) {
                    if (i == d) continue;
                    bool F[5];
                    for (int m = -2; m <= 2; ++m) {
                        if (m == 0) continue;
                        F[m + 2] = node_fluid_at(mask, d, x + (i == 0) * m, y + (i == 1) * m, z + (i == 2) * m,
                                                 nx, ny, nz, per);
                    }
                    // Fig. neighborhoodCases / Appendix B
                    uint32_t k;
                    if (!F[1] && !F[3]) k = 1u;                        // case 1
                    else if (!F[1]) k = (F[4] ? 2u : 3u) | 4u;         // case 4 / 2
                    else if (!F[3]) k = F[0] ? 2u : 3u;                // case 5 / 3
                    else k = 0u;                                       // case 6
                    w |= k << code_shift(d, i);
                }
            }
        }
        code[c] = w;
    }
}

// ------------------------------------------------------------------ cp.async helpers
// 16-byte asynchronous global -> shared copies (L2 only: the tile is staged in shared
// memory, nothing is reused from L1).
__device__ __forceinline__ void cp_async16(void *s, const void *g) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(s);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ------------------------------------------------------------------ kernel
// Tile TX x TY cells, thread (tx, ty) owns cell (x0 + tx, y0 + ty).  Shared-memory boxes
// are BX = TX + 8 wide (x0 - 4 .. x0 + TX + 3, whole 16-byte chunks) and BY = TY + 4 high
// (y0 - 2 .. y0 + TY + 1); the stencil needs +-2 in x and y.
constexpr int kTX = 32, kTY = 8, kBX = kTX + 8, kBY = kTY + 4, kPL = kBX * kBY, kStages = 6;
constexpr int kNT = kTX * kTY;

template <typename T>
struct TiledSmem {
    T ux[kStages][kPL];
    T uy[kStages][kPL];
    T uz[kStages][kPL];
    T pin[kStages][kPL];
    uint32_t cd[kStages][kPL];
    T pn[2][kPL];
};

// Appendix B second derivative across the flow from the 3-bit wall code (kind, side).
// Non-fluid nodes hold 0, so u(-1) + u(+1) is the one-sided neighbour when a wall is
// on the other side.
template <typename T>
__device__ __forceinline__ T perp_code(uint32_t k3, T um2, T um1, T u0, T up1, T up2) {
    const uint32_t kind = k3 & 3u;
    const T v1 = um1 + up1;
    const T v2 = (k3 & 4u) ? up2 : um2;
    const T A = kind == 0u ? T(1) : (kind == 2u ? T(2) : T(8) / T(3));
    const T Bc = kind == 0u ? T(-2) : (kind == 1u ? T(-8) : (kind == 2u ? T(-5) : T(-16) / T(3)));
    const T C = kind == 2u ? T(-1) / T(5) : T(0);
    return A * v1 + Bc * u0 + C * v2;
}

template <typename T, int MODE, bool REDUCE, bool SRC>
__global__ void __launch_bounds__(kNT, 3)
    sweep_tiled_kernel(const SweepBatch<T> B, const uint32_t *__restrict__ code, int zchunk, int tiles_x,
                       int tiles_y) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TiledSmem<T> &S = *reinterpret_cast<TiledSmem<T> *>(smem_raw);
    const int nx = B.nx, ny = B.ny, nz = B.nz;
    const long long N = B.N, plane = (long long)nx * ny;
    const int tid = threadIdx.x;
    const int tx = tid % kTX, ty = tid / kTX;
    const int pi = blockIdx.x % B.nprob;
    const int tile = blockIdx.x / B.nprob;
    const int x0 = (tile % tiles_x) * kTX, y0 = (tile / tiles_x) * kTY;
    const int m0 = blockIdx.y * zchunk;
    const int m1 = min(m0 + zchunk, nz);
    const SweepProblem<T> &P = B.prob[pi];
    const T *__restrict__ gux = P.uin;
    const T *__restrict__ guy = P.uin + N;
    const T *__restrict__ guz = P.uin + 2 * N;
    const T *__restrict__ gp = P.pin;

    // Copy plan.  Field boxes are kBY rows of FCH 16-byte chunks, the code box kBY rows
    // of CCH chunks; chunk starts are multiples of 4 cells (nx % 4 == 0), so a chunk
    // wraps around a periodic boundary as a whole.  fo / co: in-plane element offset of
    // this thread's field / code chunk (-1: none or outside a wall), fs / cs: its place
    // in the box.
    constexpr int FE = 16 / (int)sizeof(T), FCH = kBX / FE, CCH = kBX / 4;
    int fo[2] = {-1, -1}, fs[2] = {0, 0};
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int c = tid + r * kNT;
        if (c < FCH * kBY) {
            const int hy = c / FCH, hx = (c % FCH) * FE;
            fs[r] = hy * kBX + hx;
            const int gx = nb_coord(x0 - 4 + hx, nx, B.per[0]), gy = nb_coord(y0 - 2 + hy, ny, B.per[1]);
            if (gx >= 0 && gy >= 0) fo[r] = gx + nx * gy;
        }
    }
    int co = -1, cs = 0;
    if (tid < CCH * kBY) {
        const int hy = tid / CCH, hx = (tid % CCH) * 4;
        cs = hy * kBX + hx;
        const int gx = nb_coord(x0 - 4 + hx, nx, B.per[0]), gy = nb_coord(y0 - 2 + hy, ny, B.per[1]);
        if (gx >= 0 && gy >= 0) co = gx + nx * gy;
    }
    auto issue_plane = [&](int k) {
        const int slot = ((k % kStages) + kStages) % kStages;
        const int gz = nb_coord(k, nz, B.per[2]);
        const long long po = (long long)gz * plane;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            if (tid + r * kNT >= FCH * kBY) continue;
            const int e = fs[r];
            if (gz >= 0 && fo[r] >= 0) {
                const long long o = po + fo[r];
                cp_async16(&S.ux[slot][e], gux + o);
                cp_async16(&S.uy[slot][e], guy + o);
                cp_async16(&S.uz[slot][e], guz + o);
                cp_async16(&S.pin[slot][e], gp + o);
            } else {
#pragma unroll
                for (int j = 0; j < FE; ++j) {
                    S.ux[slot][e + j] = T(0);
                    S.uy[slot][e + j] = T(0);
                    S.uz[slot][e + j] = T(0);
                    S.pin[slot][e + j] = T(0);
                }
            }
        }
        if (tid < CCH * kBY) {
            if (gz >= 0 && co >= 0) cp_async16(&S.cd[slot][cs], code + po + co);
            else
                for (int j = 0; j < 4; ++j) S.cd[slot][cs + j] = 0u;
        }
        cp_async_commit();
    };

    const int own = (ty + 2) * kBX + (tx + 4);
    const int gx_own = x0 + tx, gy_own = y0 + ty;
    const bool real = gx_own < nx && gy_own < ny;
    const long long gin_own = (long long)gx_own + (long long)nx * gy_own;
    // tile positions past the domain edge stand for their periodic image (or for solid
    // outside a wall): their pressure is formed at the wrapped index, nothing is written
    long long gin_wrap = -1;
    {
        const int wx = nb_coord(gx_own, nx, B.per[0]), wy = nb_coord(gy_own, ny, B.per[1]);
        if (wx >= 0 && wy >= 0) gin_wrap = (long long)wx + (long long)nx * wy;
    }
    // halo p^n cells: column x0+TX (rows of the tile) and row y0+TY (columns of the tile)
    const bool halo = tid < kTX + kTY;
    const int hsx = tid < kTY ? kTX + 4 : (tid - kTY) + 4;
    const int hsy = tid < kTY ? tid + 2 : kTY + 2;
    long long hg = -1;
    if (halo && SRC) {
        const int gx = nb_coord(x0 + hsx - 4, nx, B.per[0]), gy = nb_coord(y0 + hsy - 2, ny, B.per[1]);
        if (gx >= 0 && gy >= 0) hg = (long long)gx + (long long)nx * gy;
    }

    T qx[5] = {T(0), T(0), T(0), T(0), T(0)};
    T qy[5] = {T(0), T(0), T(0), T(0), T(0)};
    T qz[3] = {T(0), T(0), T(0)};
    T pn_prev = T(0), pn_cur = T(0);
    double acc[4] = {0.0, 0.0, 0.0, 0.0};

    const int t0 = m0 - 2;
    issue_plane(t0);
    issue_plane(t0 + 1);
    issue_plane(t0 + 2);

    // p^n at box position e on plane k (ring slots sk, skm = plane k-1), in-plane index g
    auto pressure = [&](int e, int sk, int skm, int k, long long g, T &div_out) -> T {
        const uint32_t c = S.cd[sk][e];
        div_out = T(0);
        if (!(c & 1u)) return T(0);
        const T p0 = S.pin[sk][e];
        if (MODE == kModeU) return p0;
        const T dv = (S.ux[sk][e] - S.ux[sk][e - 1]) + (S.uy[sk][e] - S.uy[sk][e - kBX]) +
                     (S.uz[sk][e] - S.uz[skm][e]);
        div_out = dv;
        T rp = T(0);
        if (SRC && g >= 0) {
            const int gz = nb_coord(k, nz, B.per[2]);
            if (gz >= 0) rp = P.src[3 * N + (long long)gz * plane + g];
        }
        return p0 - B.dtc2 * (dv - rp);
    };

    int st2 = ((t0 - 2) % kStages + kStages) % kStages;  // ring slots of planes t-2, t-1, t
    int st1 = (st2 + 1) % kStages, st = (st2 + 2) % kStages;
    for (int t = t0; t <= m1 + 1; ++t) {
        cp_async_wait<2>();
        __syncthreads();
        issue_plane(t + 3);
        // z queues of the own column
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            qx[i] = qx[i + 1];
            qy[i] = qy[i + 1];
        }
        qx[4] = S.ux[st][own];
        qy[4] = S.uy[st][own];
        qz[0] = qz[1];
        qz[1] = qz[2];
        qz[2] = S.uz[st1][own];
        // p^n on plane t-1: own cell and halo cells
        pn_prev = pn_cur;
        {
            T dv;
            pn_cur = pressure(own, st1, st2, t - 1, gin_wrap, dv);
            S.pn[(t - 1) & 1][own] = pn_cur;
            if (REDUCE && real && t - 1 >= m0 && t - 1 < m1 && MODE != kModeU) acc[3] += (double)dv * (double)dv;
            if (halo) {
                T dh;
                const int e = hsy * kBX + hsx;
                S.pn[(t - 1) & 1][e] = pressure(e, st1, st2, t - 1, hg, dh);
            }
        }
        const int m = t - 2;
        const int sm = st2;
        st2 = st1;
        st1 = st;
        st = st == kStages - 1 ? 0 : st + 1;
        if (m < m0 || !real) continue;
        // ---------------------------------------------------------- update on plane m
        const long long gidx = (long long)m * plane + gin_own;
        T un[3];
        if (MODE == kModeP) {
            un[0] = qx[2];
            un[1] = qy[2];
            un[2] = qz[1];
        } else {
            const uint32_t c = S.cd[sm][own];
            const T *PN = S.pn[m & 1];
            const T *ux = S.ux[sm], *uy = S.uy[sm], *uz = S.uz[sm];
            // u_x: along x (box), across y (box) and z (queue)
            {
                const T u0 = qx[2];
                T lap = ux[own + 1] - T(2) * u0 + ux[own - 1];
                lap += perp_code((c >> code_shift(0, 1)) & 7u, ux[own - 2 * kBX], ux[own - kBX], u0, ux[own + kBX],
                                 ux[own + 2 * kBX]);
                lap += perp_code((c >> code_shift(0, 2)) & 7u, qx[0], qx[1], u0, qx[3], qx[4]);
                un[0] = u0;
                if (c & node_bit(0)) {
                    if (B.alpha) {
                        const long long g2 = (long long)m * plane +
                                             (long long)nb_coord(gx_own + 1, nx, B.per[0]) + (long long)nx * gy_own;
                        lap -= T(0.5) * (B.alpha[gidx] + B.alpha[g2]) * u0;
                    }
                    T R = B.inv_re * lap - (PN[own + 1] - pn_prev) + P.f[0];
                    if (SRC) R += P.src[gidx];
                    un[0] = u0 + B.dt * R;
                }
            }
            // u_y: along y (box), across x (box) and z (queue)
            {
                const T u0 = qy[2];
                T lap = uy[own + kBX] - T(2) * u0 + uy[own - kBX];
                lap += perp_code((c >> code_shift(1, 0)) & 7u, uy[own - 2], uy[own - 1], u0, uy[own + 1], uy[own + 2]);
                lap += perp_code((c >> code_shift(1, 2)) & 7u, qy[0], qy[1], u0, qy[3], qy[4]);
                un[1] = u0;
                if (c & node_bit(1)) {
                    if (B.alpha) {
                        const long long g2 = (long long)m * plane + (long long)gx_own +
                                             (long long)nx * nb_coord(gy_own + 1, ny, B.per[1]);
                        lap -= T(0.5) * (B.alpha[gidx] + B.alpha[g2]) * u0;
                    }
                    T R = B.inv_re * lap - (PN[own + kBX] - pn_prev) + P.f[1];
                    if (SRC) R += P.src[N + gidx];
                    un[1] = u0 + B.dt * R;
                }
            }
            // u_z: along z (queue), across x and y (box)
            {
                const T u0 = qz[1];
                T lap = qz[2] - T(2) * u0 + qz[0];
                lap += perp_code((c >> code_shift(2, 0)) & 7u, uz[own - 2], uz[own - 1], u0, uz[own + 1], uz[own + 2]);
                lap += perp_code((c >> code_shift(2, 1)) & 7u, uz[own - 2 * kBX], uz[own - kBX], u0, uz[own + kBX],
                                 uz[own + 2 * kBX]);
                un[2] = u0;
                if (c & node_bit(2)) {
                    if (B.alpha) {
                        const long long g2 = (long long)nb_coord(m + 1, nz, B.per[2]) * plane + gin_own;
                        lap -= T(0.5) * (B.alpha[gidx] + B.alpha[g2]) * u0;
                    }
                    T R = B.inv_re * lap - (pn_cur - pn_prev) + P.f[2];
                    if (SRC) R += P.src[2 * N + gidx];
                    un[2] = u0 + B.dt * R;
                }
            }
        }
        P.uout[gidx] = un[0];
        P.uout[N + gidx] = un[1];
        P.uout[2 * N + gidx] = un[2];
        P.pout[gidx] = pn_prev;
        if (REDUCE) {
            acc[0] += (double)un[0];
            acc[1] += (double)un[1];
            acc[2] += (double)un[2];
        }
    }
    cp_async_wait<0>();
    if (REDUCE) {
        for (int k = 0; k < 4; ++k)
            for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], o);
        __shared__ double red[kNT / 32][4];
        const int warp = tid >> 5, lane = tid & 31;
        if (lane == 0)
            for (int k = 0; k < 4; ++k) red[warp][k] = acc[k];
        __syncthreads();
        if (tid < 4) {
            double s = 0.0;
            for (int w = 0; w < kNT / 32; ++w) s += red[w][tid];
            const long long blk = (long long)tile * gridDim.y + blockIdx.y;
            P.partials[blk * 4 + tid] = s;
        }
    }
}

// ------------------------------------------------------------------ host helpers
struct TiledShape {
    int tiles_x, tiles_y, zchunk, nzc;
};

inline TiledShape tiled_shape(int nx, int ny, int nz) {
    TiledShape s;
    s.tiles_x = (nx + kTX - 1) / kTX;
    s.tiles_y = (ny + kTY - 1) / kTY;
    // z chunks: long enough to amortise the 4-plane start-up, enough CTAs to fill the GPU
    int zc = 64;
    while (zc > 8 && (long long)s.tiles_x * s.tiles_y * ((nz + zc - 1) / zc) < 152 * 6) zc /= 2;
    s.zchunk = zc < nz ? zc : nz;
    s.nzc = (nz + s.zchunk - 1) / s.zchunk;
    return s;
}

// The tiled kernel copies whole 16-byte chunks of 4 cells: x extents must be multiples
// of 4 (the simple kernel serves the other shapes); in-plane offsets are 32-bit.
template <typename T>
inline bool tiled_supported(int nx, int ny, int nz, int nprob) {
    return nx >= 4 && nx % 4 == 0 && ny >= 1 && nz >= 1 && nprob >= 1 && nprob <= kMaxBatch &&
           (long long)nx * ny < (1ll << 31);
}

template <typename T>
inline long long tiled_num_blocks(int nx, int ny, int nz) {
    TiledShape s = tiled_shape(nx, ny, nz);
    return (long long)s.tiles_x * s.tiles_y * s.nzc;
}

template <typename T, int MODE, bool RED, bool SRC>
inline cudaError_t launch_tiled_t(const SweepBatch<T> &B, const uint32_t *code, cudaStream_t s) {
    const TiledShape sh = tiled_shape(B.nx, B.ny, B.nz);
    const size_t smem = sizeof(TiledSmem<T>);
    auto kern = sweep_tiled_kernel<T, MODE, RED, SRC>;
    static bool attr_set = false;  // per instantiation
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    dim3 grid((unsigned)(sh.tiles_x * sh.tiles_y * B.nprob), (unsigned)sh.nzc, 1);
    kern<<<grid, kNT, smem, s>>>(B, code, sh.zchunk, sh.tiles_x, sh.tiles_y);
    return cudaGetLastError();
}

template <typename T>
inline int launch_tiled(const SweepBatch<T> &B, const uint32_t *code, int mode, bool red, bool src, cudaStream_t s) {
    cudaError_t e;
#define PM_TL(M)                                                                            \
    if (red) e = src ? launch_tiled_t<T, M, true, true>(B, code, s) : launch_tiled_t<T, M, true, false>(B, code, s); \
    else e = src ? launch_tiled_t<T, M, false, true>(B, code, s) : launch_tiled_t<T, M, false, false>(B, code, s);
    if (mode == kModeU) {
        PM_TL(kModeU)
    } else if (mode == kModePU) {
        PM_TL(kModePU)
    } else {
        PM_TL(kModeP)
    }
#undef PM_TL
    return e == cudaSuccess ? 0 : (e == cudaErrorMemoryAllocation ? 6 : 7);
}

}  // namespace pmgb
