// Device kernels of the GB300 permeability solver: neighbourhood evaluation, the fused
// pseudo-time sweep, FP64 reductions and small field utilities.
#pragma once

#include "pm_common.cuh"

namespace pmgb {

// ------------------------------------------------------------------ neighbourhood
// Algorithm 1 "Evaluate neighborhood": per cell the pore flag and the fluid flags of its
// three +d face nodes (Sec. 4: a face between two pore cells carries flow; every face
// touching solid is a no-slip / no-penetration face).  pax >= 0: fixed-pressure axis,
// whose first and last layers are reservoirs without flow across the axis.
__global__ void classify_kernel(const uint8_t *__restrict__ mask, int nx, int ny, int nz, int px,
                                int py, int pz, int pax, uint8_t *__restrict__ flags) {
    long long N = (long long)nx * ny * nz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        int x = (int)(c % nx);
        long long r = c / nx;
        int y = (int)(r % ny);
        int z = (int)(r / ny);
        uint8_t f = 0;
        if (!mask[c]) {
            f |= kFlagCell;
            int xp = nb_coord(x + 1, nx, px), yp = nb_coord(y + 1, ny, py), zp = nb_coord(z + 1, nz, pz);
            if (xp >= 0 && !mask[xp + (long long)nx * (y + (long long)ny * z)]) f |= node_bit(0);
            if (yp >= 0 && !mask[x + (long long)nx * (yp + (long long)ny * z)]) f |= node_bit(1);
            if (zp >= 0 && !mask[x + (long long)nx * (y + (long long)ny * zp)]) f |= node_bit(2);
            if (pax >= 0) {
                const int v = pax == 0 ? x : (pax == 1 ? y : z), n = pax == 0 ? nx : (pax == 1 ? ny : nz);
                if (v == 0 || v == n - 1) f &= (uint8_t)(kFlagCell | node_bit(pax));
            }
        }
        flags[c] = f;
    }
}

// Pre-processing (Sec. 5, mirroring for symmetric periodicity): out, 2n long along every
// axis with m_a = 1, holds the mask followed by its reflection, so the doubled domain is
// periodic.
__global__ void mirror_kernel(const uint8_t *__restrict__ in, int nx, int ny, int nz, int mx, int my, int mz,
                              uint8_t *__restrict__ out) {
    const int ox = nx << mx, oy = ny << my, oz = nz << mz;
    const long long M = (long long)ox * oy * oz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < M;
         c += (long long)gridDim.x * blockDim.x) {
        int x = (int)(c % ox);
        const long long r = c / ox;
        int y = (int)(r % oy), z = (int)(r / oy);
        if (x >= nx) x = 2 * nx - 1 - x;
        if (y >= ny) y = 2 * ny - 1 - y;
        if (z >= nz) z = 2 * nz - 1 - z;
        out[c] = in[(long long)x + (long long)nx * ((long long)y + (long long)ny * z)];
    }
}

// Width extension of a mask for the tiled kernel (x extent a multiple of 4): the first
// rep * nx columns of out repeat the mask periodically (a periodic x axis, where the
// repeated domain has the same fixed point), the remaining columns up to nxo are solid
// (a wall x axis, where outside the box counts as solid anyway).
__global__ void extend_x_kernel(const uint8_t *__restrict__ in, int nx, int ny, int nz, int nxo, int rep,
                                uint8_t *__restrict__ out) {
    const long long M = (long long)nxo * ny * nz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < M;
         c += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(c % nxo);
        const long long r = c / nxo;
        out[c] = x < rep * nx ? in[(long long)(x % nx) + (long long)nx * r] : (uint8_t)1;
    }
}

// Mask with its y and z axes exchanged: out[y][z][x] = in[z][y][x] (thin domains are
// solved with the long axis as the one the tiled kernel marches along).
__global__ void swap_yz_kernel(const uint8_t *__restrict__ in, int nx, int ny, int nz, uint8_t *__restrict__ out) {
    const long long M = (long long)nx * ny * nz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < M;
         c += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(c % nx);
        const long long r = c / nx;
        const int z = (int)(r % nz), y = (int)(r / nz);  // out index: (y, z, x)
        out[c] = in[(long long)x + (long long)nx * ((long long)y + (long long)ny * z)];
    }
}

// Zero the values on non-fluid faces and solid cells (the invariant every sweep relies
// on), used on caller-provided starting fields.
template <typename T>
__global__ void sanitize_kernel(const uint8_t *__restrict__ flags, long long N, T *u, T *p) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        uint8_t f = flags[c];
        for (int d = 0; d < 3; ++d)
            if (!(f & node_bit(d))) u[d * N + c] = T(0);
        if (!(f & kFlagCell)) p[c] = T(0);
    }
}

// ------------------------------------------------------------------ stencil codes
// Layout: code_shift in pm_common.cuh.

__device__ __forceinline__ bool cell_pore(const uint8_t *mask, int x, int y, int z, int nx, int ny, int nz,
                                          const int per[3]) {
    x = nb_coord(x, nx, per[0]);
    y = nb_coord(y, ny, per[1]);
    z = nb_coord(z, nz, per[2]);
    if (x < 0 || y < 0 || z < 0) return false;
    return mask[(long long)x + (long long)nx * ((long long)y + (long long)ny * z)] == 0;
}

// pax >= 0: fixed-pressure axis; its first and last cell layers are reservoirs whose only
// fluid nodes are those along the axis (no cross flow inside a reservoir), as in
// classify_kernel.  The axis is not periodic, so a coordinate along it is never wrapped.
__device__ __forceinline__ bool node_fluid_at(const uint8_t *mask, int d, int x, int y, int z, int nx, int ny,
                                              int nz, const int per[3], int pax = -1) {
    // coordinates may be up to 3 cells outside; wrap / wall handled per axis
    if (!cell_pore(mask, x, y, z, nx, ny, nz, per)) return false;
    if (pax >= 0 && d != pax) {
        const int v = pax == 0 ? x : (pax == 1 ? y : z), n = pax == 0 ? nx : (pax == 1 ? ny : nz);
        if (v == 0 || v == n - 1) return false;
    }
    return cell_pore(mask, x + (d == 0), y + (d == 1), z + (d == 2), nx, ny, nz, per);
}

__global__ void code_kernel(const uint8_t *__restrict__ mask, int nx, int ny, int nz, int px, int py, int pz,
                            int pax, uint32_t *__restrict__ code) {
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
                if (!node_fluid_at(mask, d, x, y, z, nx, ny, nz, per, pax)) continue;
                w |= (uint32_t)node_bit(d);
                for (int i = 0; i < 3; ++i) {
                    if (i == d) continue;
                    bool F[5];
                    for (int m = -2; m <= 2; ++m) {
                        if (m == 0) continue;
                        F[m + 2] = node_fluid_at(mask, d, x + (i == 0) * m, y + (i == 1) * m, z + (i == 2) * m,
                                                 nx, ny, nz, per, pax);
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

// Transposed stencil codes (layout: tslot in pm_common.cuh) from the stencil codes.
__global__ void tcode_kernel(const uint32_t *__restrict__ code, int nx, int ny, int nz, int px, int py, int pz,
                             uint32_t *__restrict__ tcode) {
    const int per[3] = {px, py, pz};
    const int n[3] = {nx, ny, nz};
    const long long N = (long long)nx * ny * nz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        const int co[3] = {(int)(c % nx), (int)((c / nx) % ny), (int)(c / ((long long)nx * ny))};
        const uint32_t w = code[c];
        uint32_t t[2] = {0u, 0u};
        for (int d = 0; d < 3; ++d) {
            if (!(w & (uint32_t)node_bit(d))) continue;
            for (int i = 0; i < 3; ++i) {
                if (i == d) continue;
                const int sh = code_shift(d, i);
                uint32_t slot = (w >> sh) & 3u;
                for (int m = -2; m <= 2; ++m) {
                    if (m == 0) continue;
                    int q[3] = {co[0], co[1], co[2]};
                    q[i] = nb_coord(q[i] + m, n[i], per[i]);
                    if (q[i] < 0) continue;  // outside a wall: no node
                    const uint32_t wb = code[(long long)q[0] + (long long)nx * ((long long)q[1] + (long long)ny * q[2])];
                    if (!(wb & (uint32_t)node_bit(d))) continue;
                    const uint32_t k3 = (wb >> sh) & 7u, kind = k3 & 3u;
                    if (m == -1) slot |= kind << 2;
                    if (m == 1) slot |= kind << 4;
                    if (m == -2 && kind == 2u && (k3 & 4u)) slot |= 64u;
                    if (m == 2 && kind == 2u && !(k3 & 4u)) slot |= 128u;
                }
                const int s = tslot(d, i);
                t[s / 4] |= slot << (8 * (s % 4));
            }
        }
        tcode[2 * c] = t[0];
        tcode[2 * c + 1] = t[1];
    }
}

// ------------------------------------------------------------------ wall stencil
// Sec. 4 / Appendix B: second derivative of a face velocity along an axis perpendicular
// to its direction, from the node itself (u0) and the nodes at -2, -1, +1, +2 with their
// fluid flags.  A missing neighbour at +-1 is a no-slip wall half a spacing away.
//   case 1  walls on both sides         -8 u0
//   case 2  wall at -1/2, no node at +2  (8 u(+1) - 16 u0) / 3
//   case 3  mirror of case 2             (8 u(-1) - 16 u0) / 3
//   case 4  wall at -1/2, node at +2     2 u(+1) - 5 u0 - u(+2) / 5
//   case 5  mirror of case 4             2 u(-1) - 5 u0 - u(-2) / 5
//   case 6  both neighbours fluid        u(-1) - 2 u0 + u(+1)
// Non-fluid node values are exactly 0, so the selects only choose coefficients.
template <typename T>
__device__ __forceinline__ T perp_d2(T u0, T um2, T um1, T up1, T up2, bool Fm2, bool Fm1, bool Fp1,
                                     bool Fp2) {
    const T c83 = T(8) / T(3), c163 = T(16) / T(3), c15 = T(1) / T(5);
    if (Fm1 && Fp1) return um1 - T(2) * u0 + up1;
    if (!Fm1 && !Fp1) return T(-8) * u0;
    if (Fp1) return Fp2 ? (T(2) * up1 - T(5) * u0 - c15 * up2) : (c83 * up1 - c163 * u0);
    return Fm2 ? (T(2) * um1 - T(5) * u0 - c15 * um2) : (c83 * um1 - c163 * u0);
}

// Coefficients of the 3-bit wall code (kind, side) of a stencil code word:
// the second derivative across the flow of node b is
//   A (u(b-1) + u(b+1)) + B u(b) + Cm u(b-2) + Cp u(b+2).
template <typename T>
__device__ __forceinline__ void wall_coef(uint32_t k3, T &A, T &Bc, T &Cm, T &Cp) {
    const uint32_t kind = k3 & 3u;
    A = kind == 0u ? T(1) : (kind == 2u ? T(2) : (kind == 3u ? T(8) / T(3) : T(0)));
    Bc = kind == 0u ? T(-2) : (kind == 1u ? T(-8) : (kind == 2u ? T(-5) : T(-16) / T(3)));
    const T c = kind == 2u ? T(-1) / T(5) : T(0);
    Cm = (k3 & 4u) ? T(0) : c;
    Cp = (k3 & 4u) ? c : T(0);
}

// ------------------------------------------------------------------ simple fused sweep
// Reference implementation: one thread per cell, every operand loaded from global memory
// (L1/L2 serve the neighbour reuse).  It defines the arithmetic the tiled kernel must
// reproduce and serves small domains.
// TR: use the transpose of the viscous operator (adjoint solves).  Node a's transposed
// term along axis i gathers, from each node b within two cells, b's own coefficient for
// the offset that reaches a (read from b's stencil code).
template <typename T, int MODE, bool REDUCE, bool SRC, bool TR = false>
__global__ void __launch_bounds__(256) sweep_simple_kernel(const SweepBatch<T> B) {
    const int nx = B.nx, ny = B.ny, nz = B.nz;
    const long long N = B.N;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z % nz;
    const int pi = blockIdx.z / nz;
    const SweepProblem<T> &P = B.prob[pi];
    const bool active = (x < nx) && (y < ny);
    const uint8_t *__restrict__ fl = B.flags;

    auto lin = [&](int xx, int yy, int zz) -> long long {
        return (long long)xx + (long long)nx * ((long long)yy + (long long)ny * zz);
    };
    // coordinates of neighbours, -1 outside a wall axis
    auto cx = [&](int m) { return nb_coord(x + m, nx, B.per[0]); };
    auto cy = [&](int m) { return nb_coord(y + m, ny, B.per[1]); };
    auto cz = [&](int m) { return nb_coord(z + m, nz, B.per[2]); };
    auto U = [&](int d, int xx, int yy, int zz) -> T {
        if (xx < 0 || yy < 0 || zz < 0) return T(0);
        return P.uin[d * N + lin(xx, yy, zz)];
    };
    auto F = [&](int d, int xx, int yy, int zz) -> bool {
        if (xx < 0 || yy < 0 || zz < 0) return false;
        return (fl[lin(xx, yy, zz)] & node_bit(d)) != 0;
    };
    // fixed-pressure axis: 0 = inlet reservoir layer, 1 = outlet reservoir layer, -1 otherwise
    const int pax = B.pres_axis - 1;
    const int npax = pax == 0 ? nx : (pax == 1 ? ny : nz);
    auto reservoir = [&](int xx, int yy, int zz) -> int {
        if (pax < 0) return -1;
        const int v = pax == 0 ? xx : (pax == 1 ? yy : zz);
        return v == 0 ? 0 : (v == npax - 1 ? 1 : -1);
    };
    // p^n at a cell (MODE kModeU: p^n is the input); reservoirs hold their fixed pressure
    T div_own = T(0);
    auto pn = [&](int xx, int yy, int zz, bool own) -> T {
        long long c = lin(xx, yy, zz);
        if (!(fl[c] & kFlagCell)) return T(0);
        const int res = reservoir(xx, yy, zz);
        if (res >= 0) return P.pres[res];
        T p0 = P.pin[c];
        if (MODE == kModeU) return p0;
        int xm = nb_coord(xx - 1, nx, B.per[0]), ym = nb_coord(yy - 1, ny, B.per[1]),
            zm = nb_coord(zz - 1, nz, B.per[2]);
        T dv = (P.uin[c] - U(0, xm, yy, zz)) + (P.uin[N + c] - U(1, xx, ym, zz)) +
               (P.uin[2 * N + c] - U(2, xx, yy, zm));
        if (own) div_own = dv;
        T rp = SRC ? P.src[3 * N + c] : T(0);
        return p0 - B.dtc2 * (dv - rp);
    };

    T unew[3] = {T(0), T(0), T(0)};
    if (active) {
        const long long c = lin(x, y, z);
        const uint8_t f0 = fl[c];
        const T p_c = pn(x, y, z, true);
        P.pout[c] = p_c;
        if (MODE == kModeP)
            for (int d = 0; d < 3; ++d) P.uout[d * N + c] = P.uin[d * N + c];
        if (MODE != kModeP) {
            const int xm1 = cx(-1), xp1 = cx(1), xm2 = cx(-2), xp2 = cx(2);
            const int ym1 = cy(-1), yp1 = cy(1), ym2 = cy(-2), yp2 = cy(2);
            const int zm1 = cz(-1), zp1 = cz(1), zm2 = cz(-2), zp2 = cz(2);
            for (int d = 0; d < 3; ++d) {
                T un = T(0);
                if (f0 & node_bit(d)) {
                    const T u0 = P.uin[d * N + c];
                    T lap;
                    // along the flow direction: 3-point, non-fluid neighbours are 0; the
                    // inlet / outlet face of a fixed-pressure axis has a zero-gradient
                    // neighbour outside
                    T up = d == 0 ? U(0, xp1, y, z) : (d == 1 ? U(1, x, yp1, z) : U(2, x, y, zp1));
                    T um = d == 0 ? U(0, xm1, y, z) : (d == 1 ? U(1, x, ym1, z) : U(2, x, y, zm1));
                    if (d == pax) {
                        const int v = d == 0 ? x : (d == 1 ? y : z);
                        if (v == 0) um = u0;
                        if (v == npax - 2) up = u0;
                    }
                    lap = up - T(2) * u0 + um;
                    if (!TR) {
                        if (d != 0)
                            lap += perp_d2(u0, U(d, xm2, y, z), U(d, xm1, y, z), U(d, xp1, y, z), U(d, xp2, y, z),
                                           F(d, xm2, y, z), F(d, xm1, y, z), F(d, xp1, y, z), F(d, xp2, y, z));
                        if (d != 1)
                            lap += perp_d2(u0, U(d, x, ym2, z), U(d, x, ym1, z), U(d, x, yp1, z), U(d, x, yp2, z),
                                           F(d, x, ym2, z), F(d, x, ym1, z), F(d, x, yp1, z), F(d, x, yp2, z));
                        if (d != 2)
                            lap += perp_d2(u0, U(d, x, y, zm2), U(d, x, y, zm1), U(d, x, y, zp1), U(d, x, y, zp2),
                                           F(d, x, y, zm2), F(d, x, y, zm1), F(d, x, y, zp1), F(d, x, y, zp2));
                    } else {
                        // transpose: sum over b = a + m e_i of b's coefficient for offset -m
                        auto trans = [&](int i, const int cm2[3], const int cm1[3], const int cp1[3],
                                         const int cp2[3]) -> T {
                            const int sh = code_shift(d, i);
                            auto k3 = [&](const int q[3]) -> uint32_t {
                                return (B.code[lin(q[0], q[1], q[2])] >> sh) & 7u;
                            };
                            T A, Bc, Cm, Cp, acc;
                            wall_coef<T>((B.code[c] >> sh) & 7u, A, Bc, Cm, Cp);
                            acc = Bc * u0;
                            if (cm1[0] >= 0 && cm1[1] >= 0 && cm1[2] >= 0) {
                                wall_coef<T>(k3(cm1), A, Bc, Cm, Cp);
                                acc += A * U(d, cm1[0], cm1[1], cm1[2]);
                            }
                            if (cp1[0] >= 0 && cp1[1] >= 0 && cp1[2] >= 0) {
                                wall_coef<T>(k3(cp1), A, Bc, Cm, Cp);
                                acc += A * U(d, cp1[0], cp1[1], cp1[2]);
                            }
                            if (cm2[0] >= 0 && cm2[1] >= 0 && cm2[2] >= 0) {
                                wall_coef<T>(k3(cm2), A, Bc, Cm, Cp);
                                acc += Cp * U(d, cm2[0], cm2[1], cm2[2]);
                            }
                            if (cp2[0] >= 0 && cp2[1] >= 0 && cp2[2] >= 0) {
                                wall_coef<T>(k3(cp2), A, Bc, Cm, Cp);
                                acc += Cm * U(d, cp2[0], cp2[1], cp2[2]);
                            }
                            return acc;
                        };
                        if (d != 0) {
                            const int a[3] = {xm2, y, z}, b1[3] = {xm1, y, z}, b2[3] = {xp1, y, z}, b3[3] = {xp2, y, z};
                            lap += trans(0, a, b1, b2, b3);
                        }
                        if (d != 1) {
                            const int a[3] = {x, ym2, z}, b1[3] = {x, ym1, z}, b2[3] = {x, yp1, z}, b3[3] = {x, yp2, z};
                            lap += trans(1, a, b1, b2, b3);
                        }
                        if (d != 2) {
                            const int a[3] = {x, y, zm2}, b1[3] = {x, y, zm1}, b2[3] = {x, y, zp1}, b3[3] = {x, y, zp2};
                            lap += trans(2, a, b1, b2, b3);
                        }
                    }
                    // the +d cell exists and is pore because the node is fluid
                    int ex = d == 0 ? xp1 : x, ey = d == 1 ? yp1 : y, ez = d == 2 ? zp1 : z;
                    if (B.alpha) lap -= T(0.5) * (B.alpha[c] + B.alpha[lin(ex, ey, ez)]) * u0;
                    const T grad = pn(ex, ey, ez, false) - p_c;
                    T R = B.inv_re * lap - grad + P.f[d];
                    if (SRC) R += P.src[d * N + c];
                    un = u0 + B.dt * R;
                }
                unew[d] = un;
                P.uout[d * N + c] = un;
            }
        }
    }
    if (REDUCE) {
        // FP64 block reduction: warp shuffles, then one partial per warp in shared memory
        double v[4];
        if (MODE == kModeP) {
            if (active) {
                long long c = lin(x, y, z);
                v[0] = (double)P.uin[c]; v[1] = (double)P.uin[N + c]; v[2] = (double)P.uin[2 * N + c];
            } else v[0] = v[1] = v[2] = 0.0;
        } else {
            v[0] = (double)unew[0]; v[1] = (double)unew[1]; v[2] = (double)unew[2];
        }
        v[3] = active ? (double)div_own * (double)div_own : 0.0;
        for (int k = 0; k < 4; ++k)
            for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
        __shared__ double sred[8][4];
        const int tid = threadIdx.y * blockDim.x + threadIdx.x;
        const int warp = tid >> 5, lane = tid & 31;
        if (lane == 0)
            for (int k = 0; k < 4; ++k) sred[warp][k] = v[k];
        __syncthreads();
        if (tid < 4) {
            double s = 0.0;
            const int nw = (blockDim.x * blockDim.y) >> 5;
            for (int w = 0; w < nw; ++w) s += sred[w][tid];
            const long long blk = (long long)blockIdx.x + (long long)gridDim.x *
                                  ((long long)blockIdx.y + (long long)gridDim.y * (long long)z);
            P.partials[blk * 4 + tid] = s;
        }
    }
}

// ------------------------------------------------------------------ defect correction
// Steady residual of the discrete Stokes system in FP64 (Sec. 3, 4), for the defect
// correction of FP32 sweeps:
//   r_u(d, c) = (1/Re) [A_d u + sum_{i != d} S_i u](c) - (p(c+e_d) - p(c)) + f_d  (fluid nodes)
//   r_p(c)    = -(D u)(c)                                                      (pore cells)
// stored as FP32: the correction only needs r to a few digits relative to itself.
__global__ void residual64_kernel(const uint8_t *__restrict__ fl, int nx, int ny, int nz, int px, int py,
                                  int pz, const double *__restrict__ u, const double *__restrict__ p,
                                  double inv_re, double f0, double f1, double f2, float *__restrict__ r) {
    const long long N = (long long)nx * ny * nz;
    const double f[3] = {f0, f1, f2};
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(c % nx);
        const long long rr = c / nx;
        const int y = (int)(rr % ny), z = (int)(rr / ny);
        auto lin = [&](int xx, int yy, int zz) -> long long {
            return (long long)xx + (long long)nx * ((long long)yy + (long long)ny * zz);
        };
        auto U = [&](int d, int xx, int yy, int zz) -> double {
            return (xx < 0 || yy < 0 || zz < 0) ? 0.0 : u[d * N + lin(xx, yy, zz)];
        };
        auto F = [&](int d, int xx, int yy, int zz) -> bool {
            return !(xx < 0 || yy < 0 || zz < 0) && (fl[lin(xx, yy, zz)] & node_bit(d));
        };
        const int xm1 = nb_coord(x - 1, nx, px), xp1 = nb_coord(x + 1, nx, px);
        const int xm2 = nb_coord(x - 2, nx, px), xp2 = nb_coord(x + 2, nx, px);
        const int ym1 = nb_coord(y - 1, ny, py), yp1 = nb_coord(y + 1, ny, py);
        const int ym2 = nb_coord(y - 2, ny, py), yp2 = nb_coord(y + 2, ny, py);
        const int zm1 = nb_coord(z - 1, nz, pz), zp1 = nb_coord(z + 1, nz, pz);
        const int zm2 = nb_coord(z - 2, nz, pz), zp2 = nb_coord(z + 2, nz, pz);
        const uint8_t f0c = fl[c];
        for (int d = 0; d < 3; ++d) {
            double R = 0.0;
            if (f0c & node_bit(d)) {
                const double u0 = u[d * N + c];
                double lap;
                if (d == 0) lap = U(0, xp1, y, z) - 2.0 * u0 + U(0, xm1, y, z);
                else if (d == 1) lap = U(1, x, yp1, z) - 2.0 * u0 + U(1, x, ym1, z);
                else lap = U(2, x, y, zp1) - 2.0 * u0 + U(2, x, y, zm1);
                if (d != 0)
                    lap += perp_d2(u0, U(d, xm2, y, z), U(d, xm1, y, z), U(d, xp1, y, z), U(d, xp2, y, z),
                                   F(d, xm2, y, z), F(d, xm1, y, z), F(d, xp1, y, z), F(d, xp2, y, z));
                if (d != 1)
                    lap += perp_d2(u0, U(d, x, ym2, z), U(d, x, ym1, z), U(d, x, yp1, z), U(d, x, yp2, z),
                                   F(d, x, ym2, z), F(d, x, ym1, z), F(d, x, yp1, z), F(d, x, yp2, z));
                if (d != 2)
                    lap += perp_d2(u0, U(d, x, y, zm2), U(d, x, y, zm1), U(d, x, y, zp1), U(d, x, y, zp2),
                                   F(d, x, y, zm2), F(d, x, y, zm1), F(d, x, y, zp1), F(d, x, y, zp2));
                const long long ce = lin(d == 0 ? xp1 : x, d == 1 ? yp1 : y, d == 2 ? zp1 : z);
                R = inv_re * lap - (p[ce] - p[c]) + f[d];
            }
            r[d * N + c] = (float)R;
        }
        double rp = 0.0;
        if (f0c & kFlagCell)
            rp = -((u[c] - U(0, xm1, y, z)) + (u[N + c] - U(1, x, ym1, z)) + (u[2 * N + c] - U(2, x, y, zm1)));
        r[3 * N + c] = (float)rp;
    }
}

// x64 += d32 over the 4N values of one state, and FP64 block sums of the new u
// (partials[blk][0..2]; [3] = 0) for the mean velocity.
__global__ void accumulate_kernel(double *__restrict__ u64, double *__restrict__ p64, const float *__restrict__ du,
                                  const float *__restrict__ dp, long long N, double *__restrict__ partials) {
    double a[3] = {0.0, 0.0, 0.0};
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        for (int d = 0; d < 3; ++d) {
            const double v = u64[d * N + c] + (double)du[d * N + c];
            u64[d * N + c] = v;
            a[d] += v;
        }
        p64[c] += (double)dp[c];
    }
    for (int k = 0; k < 3; ++k)
        for (int o = 16; o > 0; o >>= 1) a[k] += __shfl_down_sync(0xffffffffu, a[k], o);
    __shared__ double red[8][3];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        for (int k = 0; k < 3; ++k) red[warp][k] = a[k];
    __syncthreads();
    if (threadIdx.x < 4) {
        double s = 0.0;
        if (threadIdx.x < 3)
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w][threadIdx.x];
        partials[blockIdx.x * 4 + threadIdx.x] = s;
    }
}

// ------------------------------------------------------------------ sensitivity
// dJ/d alpha_c = scale * sum_{i,j} w_ij sum over the six faces F of cell c of v^(i)_F u^(j)_F
// with u^(j) the forward and v^(i) the transposed (adjoint) solutions; scale carries
// -1 / (2 Re^2 N) and the length units of k.
template <typename T>
struct SensArgs {
    const T *fwd[3];  // u fields (3N) of the forward solves, nullptr if unused
    const T *adj[3];  // u fields (3N) of the adjoint solves
    double w[3][3];
};

template <typename T>
__global__ void sensitivity_kernel(const SensArgs<T> A, int nx, int ny, int nz, int px, int py, int pz,
                                   double scale, float *__restrict__ out) {
    const long long N = (long long)nx * ny * nz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(c % nx);
        const long long r = c / nx;
        const int y = (int)(r % ny), z = (int)(r / ny);
        const int xm = nb_coord(x - 1, nx, px), ym = nb_coord(y - 1, ny, py), zm = nb_coord(z - 1, nz, pz);
        const long long lower[3] = {
            xm >= 0 ? (long long)xm + (long long)nx * ((long long)y + (long long)ny * z) : -1,
            ym >= 0 ? (long long)x + (long long)nx * ((long long)ym + (long long)ny * z) : -1,
            zm >= 0 ? (long long)x + (long long)nx * ((long long)y + (long long)ny * zm) : -1};
        double s = 0.0;
        for (int i = 0; i < 3; ++i) {
            if (!A.adj[i]) continue;
            for (int j = 0; j < 3; ++j) {
                if (!A.fwd[j] || A.w[i][j] == 0.0) continue;
                double t = 0.0;
                for (int d = 0; d < 3; ++d) {
                    t += (double)A.adj[i][d * N + c] * (double)A.fwd[j][d * N + c];
                    if (lower[d] >= 0) t += (double)A.adj[i][d * N + lower[d]] * (double)A.fwd[j][d * N + lower[d]];
                }
                s += A.w[i][j] * t;
            }
        }
        out[c] = (float)(scale * s);
    }
}

// FP64 block sums of the three velocity components of one state (partials[blk][0..2],
// [3] = 0), for the mean velocity of fields handed over by the caller.
template <typename T>
__global__ void sum_u_kernel(const T *__restrict__ u, long long N, double *__restrict__ partials) {
    double a[3] = {0.0, 0.0, 0.0};
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x)
        for (int d = 0; d < 3; ++d) a[d] += (double)u[d * N + c];
    for (int k = 0; k < 3; ++k)
        for (int o = 16; o > 0; o >>= 1) a[k] += __shfl_down_sync(0xffffffffu, a[k], o);
    __shared__ double red[8][3];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        for (int k = 0; k < 3; ++k) red[warp][k] = a[k];
    __syncthreads();
    if (threadIdx.x < 4) {
        double s = 0.0;
        if (threadIdx.x < 3)
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w][threadIdx.x];
        partials[blockIdx.x * 4 + threadIdx.x] = s;
    }
}

// Sums the block partials of each problem in a fixed order (deterministic) and scales
// by 1/N: out[prob][0..2] = q_d, out[prob][3] = |D u|^2.
__global__ void reduce_partials_kernel(const double *partials, long long nblk, long long N,
                                       double *out) {
    const double *P = partials + (size_t)blockIdx.x * nblk * 4;
    __shared__ double s[256][4];
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long b = threadIdx.x; b < nblk; b += blockDim.x)
        for (int k = 0; k < 4; ++k) a[k] += P[b * 4 + k];
    for (int k = 0; k < 4; ++k) s[threadIdx.x][k] = a[k];
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st)
            for (int k = 0; k < 4; ++k) s[threadIdx.x][k] += s[threadIdx.x + st][k];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int k = 0; k < 3; ++k) out[blockIdx.x * 4 + k] = s[0][k] / (double)N;
        out[blockIdx.x * 4 + 3] = s[0][3];
    }
}

// Per-problem window sums of a multi-geometry launch: problem k owns partials
// [begin, begin + count) and has N cells; out[k][0..2] = q_d, out[k][3] = |D u|^2.
struct ReduceRange {
    long long begin, count;
    double N;
};

__global__ void reduce_ranges_kernel(const double *partials, const ReduceRange *rr, double *out) {
    const ReduceRange R = rr[blockIdx.x];
    __shared__ double s[256][4];
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long b = threadIdx.x; b < R.count; b += blockDim.x)
        for (int k = 0; k < 4; ++k) a[k] += partials[(R.begin + b) * 4 + k];
    for (int k = 0; k < 4; ++k) s[threadIdx.x][k] = a[k];
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st)
            for (int k = 0; k < 4; ++k) s[threadIdx.x][k] += s[threadIdx.x + st][k];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int k = 0; k < 3; ++k) out[blockIdx.x * 4 + k] = s[0][k] / R.N;
        out[blockIdx.x * 4 + 3] = s[0][3];
    }
}

// x = 0, n elements (also for buffers in host memory, where a memset may not apply).
template <typename T>
__global__ void fill_zero_kernel(T *__restrict__ x, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        x[i] = T(0);
}

// out = f (cur - prev), n elements (out may alias cur: each element is read before it is
// written).  Geometric-tail estimate of the remaining error of an iteration from its
// change over the last window.
template <typename T>
__global__ void extrapolate_kernel(T *out, const T *cur, const T *__restrict__ prev, T f, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = f * (cur[i] - prev[i]);
}

// y = a * x (type conversion allowed), n elements.
template <typename TO, typename TI>
__global__ void scale_copy_kernel(TO *__restrict__ y, const TI *__restrict__ x, double a, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        y[i] = (TO)(a * (double)x[i]);
}

}  // namespace pmgb
