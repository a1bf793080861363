// Tiled z-marching fused sweep.
//
// A CTA owns a TX x TY column tile of the (x, y) plane and marches along z over a chunk
// of planes.  Each plane of the five input arrays (u_x, u_y, u_z, p, stencil code) is
// copied with its 2-voxel halo into a 5-stage shared-memory ring by cp.async, two planes
// ahead of use, so each field value comes from DRAM once per sweep and the neighbour
// reuse is served by shared memory (x, y) and per-thread register queues (z).
//
// Per step t the CTA
//   reads plane t of its own column into the z queues,
//   forms p^n on plane t-1 (own cells and the +x / +y halo cells),
//   updates u on plane t-2 with p^n of planes t-2 and t-1 and writes u^{n+1}, p^n.
// The neighbourhood (Algorithm 1, "Evaluate neighborhood") is precomputed once per
// geometry as one 32-bit code per cell (code_kernel), so the sweep reads no mask
// neighbours at all.
#pragma once

#include <atomic>
#include <type_traits>

#include "pm_common.cuh"

namespace pmgb {

// ------------------------------------------------------------------ cp.async helpers
// 16-byte asynchronous global -> shared copies (L2 only: the tile is staged in shared
// memory, nothing is reused from L1).
// zero-filling form: src_bytes = 0 reads nothing and writes 16 zero bytes
__device__ __forceinline__ void cp_async16z(void *s, const void *g, unsigned src_bytes) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(s);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(g), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ------------------------------------------------------------------ tile shapes
// A CTA covers TX x TY cells of the (x, y) plane; each thread owns CPT x-adjacent cells
// of one tile row (LPR = TX / CPT threads per row); the ring holds STAGES planes, AHEAD =
// STAGES - 3 of them in flight; MINB CTAs per SM for FP32 (one for FP64).  Shared-memory
// boxes are BX = TX + 8 wide (x0 - 4 .. x0 + TX + 3, whole 16-byte chunks) and BY = TY + 4
// high (y0 - 2 .. y0 + TY + 1): the stencil reaches +-2 in x and y.  p^n, the input
// pressure and the stencil codes are needed on box rows 2 .. TY + 2 only (tile rows and
// the +y halo row), u_y on rows 1 .. TY + 2, u_x and u_z on all rows.
template <int TX_, int TY_, int CPT_, int STAGES_, int MINB_>
struct TileCfg {
    static constexpr int TX = TX_, TY = TY_, CPT = CPT_, STAGES = STAGES_, MINB = MINB_;
    static constexpr int LPR = TX / CPT, NT = LPR * TY, NW = NT / 32;
    static constexpr int BX = TX + 8, BY = TY + 4, PL = BX * BY;
    static constexpr int AHEAD = STAGES - 3;
    static constexpr int PNL = (TY + 1) * BX, PNo = 2 * BX;
    static constexpr int UYL = (TY + 2) * BX, UYo = BX;
    static_assert(TX % CPT == 0 && 32 % LPR == 0 && NT % 32 == 0 && NW >= 2 && TY <= 32, "tile shape");
    static_assert(CPT == 2 || CPT == 4, "cells per thread");
    static_assert(AHEAD >= 1, "ring depth");
};
// The shapes the autotuner chooses from (pm_options.tile = index + 1).
using Tile64x12c2 = TileCfg<64, 12, 2, 5, 2>;  // 384 threads, 2 CTAs / SM
using Tile64x12c4 = TileCfg<64, 12, 4, 5, 2>;  // 192 threads, 2 CTAs / SM
using Tile64x8c4 = TileCfg<64, 8, 4, 4, 3>;    // 128 threads, 3 CTAs / SM
constexpr int kNumTiles = 3;
// the transposed sweep (more registers: one CTA per SM), shape index kTileTR
using Tile64x12c4tr = TileCfg<64, 12, 4, 5, 1>;
constexpr int kTileTR = 3;
// Chunked schedules (zchunk > 0): chunk-major units of one (column, chunk of zchunk planes)
// per CTA.  The last chunk of every column (planes (K-1) zchunk .. nz-1, K chunks) may be
// cut into `split` equal sub-chunks: the units that start last are then short and fill
// the last wave of CTAs instead of leaving slots idle.  split_last() is the number of
// non-empty sub-chunks for a requested split; chunk_unit() maps unit u to its column and
// plane range [m0, m1).  The arithmetic per cell does not depend on the split.
constexpr int kSplits[3] = {1, 2, 4};  // splits the autotuner tries
__host__ __device__ inline int split_last(int nz, int zchunk, int split) {
    const int K = (nz + zchunk - 1) / zchunk, len = nz - (K - 1) * zchunk;
    int S = split < 1 ? 1 : (split > len ? len : split);
    while (S > 1 && (S - 1) * ((len + S - 1) / S) >= len) --S;
    return S;
}
__host__ __device__ inline void chunk_unit(long long u, long long C, int nz, int zchunk, int S, long long &col,
                                           int &m0, int &m1) {
    const int K = (nz + zchunk - 1) / zchunk;
    const long long full = (long long)(K - 1) * C;
    if (u < full) {
        col = u % C;
        m0 = (int)(u / C) * zchunk;
        m1 = m0 + zchunk;
    } else {
        const long long j = u - full;
        const int last0 = (K - 1) * zchunk, L = (nz - last0 + S - 1) / S;
        col = j % C;
        m0 = last0 + (int)(j / C) * L;
        m1 = m0 + L < nz ? m0 + L : nz;
    }
}

// FP64 fields use the first shape only.
template <typename T>
inline int tile_count() {
    return sizeof(T) == 4 ? kNumTiles : 1;
}
struct TileDims {
    int tx, ty;
};
__host__ __device__ constexpr TileDims tile_dims(int t) {
    return t == 2 ? TileDims{64, 8} : TileDims{64, 12};
}
constexpr int kMaxTileTX = 64;

// One ring stage: the five arrays of one plane, contiguous, so that every access is a
// per-step stage pointer plus a compile-time offset.  Arrays that need fewer box rows
// start at a later row: u_y at row 1 (index = box index - UYo), p and the codes at row 2
// (index = box index - PNo).
template <typename T, class C>
struct TiledStage {
    T ux[C::PL];
    T uz[C::PL];
    T uy[C::UYL];
    T pin[C::PNL];
    uint32_t cd[C::PNL];
};

// Wall coefficients per wall kind.  Non-fluid nodes hold 0, so with S = u(-1) + u(+1)
// every Appendix B case is
//   A (S - 2 u0) + K (u0 + u(far) / 5),   far = +2 if side else -2,
//   case 6 (kind 0): A = 1;  case 1 (kind 1, S = 0): A = 4;  cases 2/3 (kind 3): A = 8/3;
//   cases 4/5 (kind 2): A = 2, K = -1  (2 S - 5 u0 - u(far) / 5);  K = 0 otherwise.
// One entry (A, K) is one 8-byte shared-memory load; the table is one bank row, so a
// warp's lookups never conflict.
template <typename T>
struct alignas(2 * sizeof(T)) WallCoef {
    T A, K;
};

template <typename T, class C>
struct TiledSmem {
    TiledStage<T, C> st[C::STAGES];
    T pn[2][C::PNL];  // index: box index - 2 BX
    WallCoef<T> coef[4];
    T tA[4], tB[4];   // transposed sweep: off-diagonal (A) and diagonal (B) coefficient per wall kind
};

// A group of N x-adjacent values, aligned for one vector access of up to 16 bytes.
template <typename T, int N>
struct alignas(N * sizeof(T) < 16 ? N * sizeof(T) : 16) VecT {
    T v[N];
};
// Loads / stores of N x-adjacent values (shared or global), in 16-byte pieces at most.
template <int N, typename T>
__device__ __forceinline__ void ldv(T (&o)[N], const T *p) {
    constexpr int E = (N * sizeof(T) <= 16) ? N : 16 / (int)sizeof(T);
#pragma unroll
    for (int i = 0; i < N; i += E) {
        const VecT<T, E> w = *reinterpret_cast<const VecT<T, E> *>(p + i);
#pragma unroll
        for (int j = 0; j < E; ++j) o[i + j] = w.v[j];
    }
}
template <int N, typename T>
__device__ __forceinline__ void stv(T *p, const T (&a)[N]) {
    constexpr int E = (N * sizeof(T) <= 16) ? N : 16 / (int)sizeof(T);
#pragma unroll
    for (int i = 0; i < N; i += E) {
        VecT<T, E> w;
#pragma unroll
        for (int j = 0; j < E; ++j) w.v[j] = a[i + j];
        *reinterpret_cast<VecT<T, E> *>(p + i) = w;
    }
}
template <typename T>
struct alignas(2 * sizeof(T)) Pair {
    T a, b;
};
template <typename T>
__device__ __forceinline__ Pair<T> ld2(const T *p) {
    return *reinterpret_cast<const Pair<T> *>(p);
}

// Byte offset of the coefficient-table entry of the wall kind at bit sh of word c (one
// shift and one mask: entries are 2 T, a power of two).
template <typename T>
__device__ __forceinline__ uint32_t coef_offset(uint32_t c, int sh) {
    constexpr int lg = sizeof(T) == 4 ? 3 : 4;
    static_assert(sizeof(WallCoef<T>) == (1u << lg), "entry size");
    return (c >> (sh - lg)) & (3u << lg);
}

// ------------------------------------------------------------------ kernel
// Thread (cx, ty) owns the cells x0 + CPT cx .. x0 + CPT cx + CPT - 1 of tile row y0 + ty.
// Per step t the CTA
//   reads plane t of its own cells into the z queues,
//   forms p^n on plane t-1 (own cells and the +x / +y halo cells),
//   updates u on plane t-2 with p^n of planes t-2 and t-1 and writes u^{n+1}, p^n.
// Every shape does the same arithmetic per cell in the same order (bit-identical fields).
// TR: the transposed viscous operator (adjoint solves), from the transposed stencil codes.
template <typename T, class C, int MODE, bool REDUCE, bool SRC, bool ALPHA, bool TR = false>
__global__ void __launch_bounds__(C::NT, sizeof(T) == 4 ? C::MINB : 1)
    sweep_tiled_kernel(const SweepBatch<T> B, const uint32_t *__restrict__ code, int tiles_x, int tiles_y,
                       long long per_cta, int zchunk) {
    constexpr int TX = C::TX, TY = C::TY, CPT = C::CPT, BX = C::BX, BY = C::BY, NT = C::NT;
    constexpr int STAGES = C::STAGES, AHEAD = C::AHEAD, PNo = C::PNo, UYo = C::UYo, PL = C::PL;
    // single geometry: B.nx.. and the arguments; multi-geometry: per problem (below)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TiledSmem<T, C> &S = *reinterpret_cast<TiledSmem<T, C> *>(smem_raw);
    int nx = B.nx, ny = B.ny, nz = B.nz;
    long long N = B.N, plane = (long long)nx * ny;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int cx = tid % C::LPR, ty = tid / C::LPR;
    const unsigned char *coef_bytes = reinterpret_cast<const unsigned char *>(S.coef);
    __shared__ double red_sum[kMaxSame][4];  // per drive: FP64 sums of this CTA
    __shared__ double red[C::NW][4];
    if (REDUCE && tid < kMaxSame * 4) red_sum[tid / 4][tid % 4] = 0.0;
    // multi-geometry launch: this CTA's problem (prefix table of CTA counts)
    int mp = 0;
    if (B.multi) {
        while (mp + 1 < B.nprob && (long long)blockIdx.x >= B.prob[mp + 1].unit_begin) ++mp;
        if (B.active && !B.active[mp]) return;
        nx = B.prob[mp].nx;
        ny = B.prob[mp].ny;
        nz = B.prob[mp].nz;
        plane = (long long)nx * ny;
        N = plane * nz;
        code = B.prob[mp].code;
        tiles_x = B.prob[mp].tiles_x;
        tiles_y = B.prob[mp].tiles_y;
    }

    if (tid < 4) {
        // Appendix B: kind 0 case 6, kind 1 case 1, kind 2 cases 4/5, kind 3 cases 2/3
        const int kind = tid;
        WallCoef<T> w;
        w.A = kind == 0 ? T(1) : (kind == 1 ? T(4) : (kind == 2 ? T(2) : T(8) / T(3)));
        w.K = kind == 2 ? T(-1) : T(0);
        S.coef[tid] = w;
        // Appendix B stencils as (A on the nodes at +-1, B on the node itself) per kind
        S.tA[tid] = kind == 0 ? T(1) : (kind == 2 ? T(2) : (kind == 3 ? T(8) / T(3) : T(0)));
        S.tB[tid] = kind == 0 ? T(-2) : (kind == 1 ? T(-8) : (kind == 2 ? T(-5) : T(-16) / T(3)));
    }

    // Persistent CTAs over columns (a column = one drive on one x-y tile, all planes).
    // Phase 1: rounds in which CTA b marches whole column r G + b, so that all CTAs are at
    // the same plane and the tile halos they share are served by L2.  Phase 2: the
    // remaining columns, column by column, split into equal contiguous plane ranges
    // (short pieces, neighbouring columns again at similar planes).  Every CTA gets the
    // same number of plane steps, with at most one restart of its plane pipeline.
    // zchunk > 0 instead: one (column, plane chunk) unit per CTA, chunk-major order.
    const long long G = gridDim.x, Cn = (long long)B.nprob * tiles_x * tiles_y;
    const long long rounds = zchunk > 0 ? 0 : Cn / G, rem_total = zchunk > 0 ? 0 : (Cn - rounds * G) * nz;
    long long pos = (long long)blockIdx.x * per_cta;
    const long long pos_end = min(rem_total, pos + per_cta);
    for (long long it = 0;; ++it) {
    long long col;
    int m0, m1;
    if (B.multi) {
        // one (column, plane chunk) unit of problem mp, chunk-major
        if (it > 0) break;
        const long long lu = (long long)blockIdx.x - B.prob[mp].unit_begin;
        const long long Cm = (long long)tiles_x * tiles_y;
        const int zc = B.prob[mp].zchunk;
        col = (long long)mp + B.nprob * (lu % Cm);  // decoded below as (drive mp, tile lu % Cm)
        m0 = (int)(lu / Cm) * zc;
        m1 = min(nz, m0 + zc);
    } else if (zchunk > 0) {
        if (it > 0) break;
        chunk_unit(blockIdx.x, Cn, nz, zchunk, split_last(nz, zchunk, B.zsplit), col, m0, m1);
    } else if (it < rounds) {
        col = it * G + blockIdx.x;
        m0 = 0;
        m1 = nz;
    } else {
        if (pos >= pos_end) break;
        col = rounds * G + pos / nz;
        m0 = (int)(pos % nz);
        m1 = (int)min((long long)nz, m0 + (pos_end - pos));
        pos += m1 - m0;
    }
    const int pi = (int)(col % B.nprob);
    const int tile = (int)(col / B.nprob);
    const int rs = B.multi ? 0 : pi;  // slot of red_sum
    const int x0 = (tile % tiles_x) * TX, y0 = (tile / tiles_x) * TY;
    const SweepProblem<T> &P = B.prob[pi];
    const T *__restrict__ gux = P.uin;
    const T *__restrict__ guy = P.uin + N;
    const T *__restrict__ guz = P.uin + 2 * N;
    const T *__restrict__ gp = P.pin;

    // Copy plan.  Field boxes are BY rows of FCH 16-byte chunks, the code box TY + 1 rows
    // of CCH chunks; chunk starts are multiples of 4 cells (nx % 4 == 0), so a chunk
    // wraps around a periodic boundary as a whole.  fo / co: in-plane element offset of
    // this thread's field / code chunk (-1: none or outside a wall), fs / cs: its place
    // in the box.
    constexpr int FE = 16 / (int)sizeof(T), FCH = BX / FE, CCH = BX / 4;
    constexpr int FR = (FCH * BY + NT - 1) / NT;
    constexpr int CR = (CCH * (TY + 1) + NT - 1) / NT;
    int fo[FR], fs[FR];
    bool fhas[FR], fuy[FR], fp[FR];  // chunk exists / row also holds u_y / also p
#pragma unroll
    for (int r = 0; r < FR; ++r) {
        const int c = tid + r * NT;
        fo[r] = -1;
        fs[r] = 0;
        fhas[r] = c < FCH * BY;
        fuy[r] = fp[r] = false;
        if (fhas[r]) {
            const int hy = c / FCH, hx = (c % FCH) * FE;
            fs[r] = hy * BX + hx;
            fuy[r] = hy >= 1 && hy <= TY + 2;
            fp[r] = hy >= 2 && hy <= TY + 2;
            const int gx = nb_coord(x0 - 4 + hx, nx, B.per[0]), gy = nb_coord(y0 - 2 + hy, ny, B.per[1]);
            if (gx >= 0 && gy >= 0) fo[r] = gx + nx * gy;
        }
    }
    // code chunks: box rows 2 .. TY + 2; cs is the index in the stage's code array
    int co[CR], cs[CR];
    bool chas[CR];
#pragma unroll
    for (int r = 0; r < CR; ++r) {
        const int c = tid + r * NT;
        co[r] = -1;
        cs[r] = 0;
        chas[r] = c < CCH * (TY + 1);
        if (chas[r]) {
            const int hy = 2 + c / CCH, hx = (c % CCH) * 4;
            cs[r] = hy * BX + hx - PNo;
            const int gx = nb_coord(x0 - 4 + hx, nx, B.per[0]), gy = nb_coord(y0 - 2 + hy, ny, B.per[1]);
            if (gx >= 0 && gy >= 0) co[r] = gx + nx * gy;
        }
    }
    auto issue_plane = [&](int k, int slot) {
        TiledStage<T, C> &Gs = S.st[slot];
        const int gz = nb_coord(k, nz, B.per[2]);
        const long long po = (long long)gz * plane;
#pragma unroll
        for (int r = 0; r < FR; ++r) {
            if (!fhas[r]) continue;
            const int e = fs[r];
            // outside a wall: the zero-filling copy reads nothing (a valid address is given)
            const bool in = gz >= 0 && fo[r] >= 0;
            const long long o = in ? po + fo[r] : 0;
            const unsigned nb = in ? 16u : 0u;
            cp_async16z(&Gs.ux[e], gux + o, nb);
            cp_async16z(&Gs.uz[e], guz + o, nb);
            if (fuy[r]) cp_async16z(&Gs.uy[e - UYo], guy + o, nb);
            if (fp[r]) cp_async16z(&Gs.pin[e - PNo], gp + o, nb);
        }
#pragma unroll
        for (int r = 0; r < CR; ++r) {
            if (!chas[r]) continue;
            const bool in = gz >= 0 && co[r] >= 0;
            cp_async16z(&Gs.cd[cs[r]], code + (in ? po + co[r] : 0), in ? 16u : 0u);
        }
        cp_async_commit();
    };

    const int own = (ty + 2) * BX + 4 + CPT * cx;  // box index of the first own cell
    const int gx_own = x0 + CPT * cx, gy_own = y0 + ty;
    const bool real0 = gx_own < nx && gy_own < ny;       // nx % 4 == 0: all own cells or none
    const long long gin_own = (long long)gx_own + (long long)nx * gy_own;
    // tile positions past the domain edge stand for their periodic image (or for solid
    // outside a wall): their pressure is formed at the wrapped index, nothing is written
    long long gin_wrap = -1;
    {
        const int wx = nb_coord(gx_own, nx, B.per[0]), wy = nb_coord(gy_own, ny, B.per[1]);
        if (wx >= 0 && wy >= 0) gin_wrap = (long long)wx + (long long)nx * wy;
    }
    // halo p^n: the threads of the last tile row take the row y0 + TY (CPT cells each), the
    // last TY lanes of the warp before the last one the column x0 + TX (single cells)
    const bool hrow = ty == TY - 1, hcol = warp == C::NW - 2 && lane >= 32 - TY;
    const int hown = hrow ? (TY + 2) * BX + 4 + CPT * cx : (lane - (32 - TY) + 2) * BX + TX + 4;
    long long hg = -1;
    if ((hrow || hcol) && SRC) {
        const int gx = nb_coord(x0 + (hown % BX) - 4, nx, B.per[0]), gy = nb_coord(y0 + hown / BX - 2, ny, B.per[1]);
        if (gx >= 0 && gy >= 0) hg = (long long)gx + (long long)nx * gy;
    }
    // offsets to the +x / +y cell for the drag term; at a wall the face is not fluid and the
    // value is discarded, so the cell itself stands in (keeps the read in bounds)
    const int wxp = nb_coord(gx_own + CPT, nx, B.per[0]), wyp = nb_coord(gy_own + 1, ny, B.per[1]);
    const long long exl_off = wxp >= 0 ? (long long)wxp - (gx_own + CPT) : -1;  // last cell's +x
    const long long ey_off = wyp >= 0 ? ((long long)wyp - gy_own) * nx : 0;

    T qx[5][CPT], qy[5][CPT], qz[5][CPT];
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = 0; j < CPT; ++j) qx[i][j] = qy[i][j] = qz[i][j] = T(0);
    T pn_m[CPT];  // own p^n on the plane being updated (m)
#pragma unroll
    for (int j = 0; j < CPT; ++j) pn_m[j] = T(0);
    double acc[4] = {0.0, 0.0, 0.0, 0.0};

    const int t0 = m0 - 2;
    int s2 = ((t0 - 2) % STAGES + STAGES) % STAGES;  // ring stages of planes t-2, t-1, t
    int s1 = (s2 + 1) % STAGES, s0 = (s2 + 2) % STAGES;
    {
        int sl = s0;
        for (int k = 0; k < AHEAD; ++k) {
            issue_plane(t0 + k, sl);
            sl = sl == STAGES - 1 ? 0 : sl + 1;
        }
    }

    // p^n of one cell at box position e of plane k (stage K), the plane below in KM
    auto press1 = [&](const TiledStage<T, C> &K, const TiledStage<T, C> &KM, int e, int k, long long g) -> T {
        const T dv = (K.ux[e] - K.ux[e - 1]) + (K.uy[e - UYo] - K.uy[e - BX - UYo]) + (K.uz[e] - KM.uz[e]);
        T rp = T(0);
        if (SRC && g >= 0) {
            const int gz = nb_coord(k, nz, B.per[2]);
            if (gz >= 0) rp = P.src[3 * N + (long long)gz * plane + g];
        }
        const T p0 = K.pin[e - PNo];
        const T pn = MODE == kModeU ? p0 : p0 - B.dtc2 * (dv - rp);
        return (K.cd[e - PNo] & 1u) ? pn : T(0);
    };
    // second derivative across the flow (Appendix B) from the 3-bit wall code, added to lap
    auto perp = [&](T &lap, uint32_t cc, int sh, T um2, T um1, T u0, T up1, T up2) {
        const WallCoef<T> w = *reinterpret_cast<const WallCoef<T> *>(coef_bytes + coef_offset<T>(cc, sh));
        const uint32_t n = cc >> sh;
        lap = fma(w.A, fma(T(-2), u0, um1 + up1), lap);
        const T far = (n & 4u) ? up2 : um2;
        lap = fma(w.K, fma(T(1) / T(5), far, u0), lap);
    };
    // its transpose from the 8-bit slot of the transposed code: the node's own diagonal
    // coefficient and the coefficients its neighbours apply to it
    auto perp_t = [&](T &lap, uint32_t tw, int sh, T um2, T um1, T u0, T up1, T up2) {
        const uint32_t f = tw >> sh;
        const T cm2 = (f & 64u) ? T(-1) / T(5) : T(0), cp2 = (f & 128u) ? T(-1) / T(5) : T(0);
        T acc = S.tB[f & 3u] * u0;
        acc = fma(S.tA[(f >> 2) & 3u], um1, acc);
        acc = fma(S.tA[(f >> 4) & 3u], up1, acc);
        acc = fma(cm2, um2, acc);
        acc = fma(cp2, up2, acc);
        lap += acc;
    };
    // transposed codes of the own cells, loaded one step ahead of the update that uses them
    uint32_t tcn[2 * CPT];
    auto load_tc = [&](int k) {
#pragma unroll
        for (int j = 0; j < 2 * CPT; ++j) tcn[j] = 0u;
        if (TR && k >= m0 && k < m1 && real0) ldv(tcn, B.tcode + 2 * ((long long)k * plane + gin_own));
    };
    load_tc(t0 - 2);

    T *outx = P.uout + (long long)m0 * plane + gin_own;
    T *outp = P.pout + (long long)m0 * plane + gin_own;
    const int tend = m1 + 1;
    // one plane step; kRot = step index mod 5.  The z queues are circular with compile-time
    // slots, so advancing them moves no registers: after this step's load, queue entry k
    // (u_x, u_y: planes m-2 .. m+2 of the updated plane m = t-2; u_z: planes m-1 .. m+1 as
    // entries 0 .. 2) lives in slot (kRot + 1 + k) % 5.  The loop below unrolls five steps.
    auto step = [&](auto Rc, int t) {
        constexpr int kRot = decltype(Rc)::value;
        constexpr int Q0 = (kRot + 1) % 5, Q1 = (kRot + 2) % 5, Q2 = (kRot + 3) % 5, Q3 = (kRot + 4) % 5,
                      Q4 = kRot % 5;
        cp_async_wait<AHEAD - 1>();
        __syncthreads();
        {
            int sl = s0 + AHEAD;
            if (sl >= STAGES) sl -= STAGES;
            issue_plane(t + AHEAD, sl);
        }
        uint32_t tc[2 * CPT];
        if (TR) {
#pragma unroll
            for (int j = 0; j < 2 * CPT; ++j) tc[j] = tcn[j];
            load_tc(t - 1);
        }
        const TiledStage<T, C> &G0 = S.st[s0], &G1 = S.st[s1], &G2 = S.st[s2];
        // z queues of the own cells
        ldv(qx[Q4], &G0.ux[own]);
        ldv(qy[Q4], &G0.uy[own - UYo]);
        ldv(qz[(kRot + 3) % 5], &G1.uz[own]);
        // own p^n on plane t-1 (kept in registers until after the update of plane t-2)
        T pn_new[CPT];
        {
            uint32_t cd[CPT];
            T pin[CPT], uyd[CPT];
            ldv(cd, &G1.cd[own - PNo]);
            ldv(pin, &G1.pin[own - PNo]);
            ldv(uyd, &G1.uy[own - BX - UYo]);
            const T uxl = G1.ux[own - 1];
            T rp[CPT];
#pragma unroll
            for (int j = 0; j < CPT; ++j) rp[j] = T(0);
            if (SRC && gin_wrap >= 0) {
                const int gz = nb_coord(t - 1, nz, B.per[2]);
                if (gz >= 0) ldv(rp, P.src + 3 * N + (long long)gz * plane + gin_wrap);
            }
#pragma unroll
            for (int j = 0; j < CPT; ++j) {
                const T left = j == 0 ? uxl : qx[Q3][j - 1];
                T dv = (qx[Q3][j] - left) + (qy[Q3][j] - uyd[j]) + (qz[(kRot + 1 + 2) % 5][j] - qz[(kRot + 1 + 1) % 5][j]);
                const bool pore = cd[j] & 1u;
                pn_new[j] = pore ? (MODE == kModeU ? pin[j] : pin[j] - B.dtc2 * (dv - rp[j])) : T(0);
                if (REDUCE && real0 && t - 1 >= m0 && t - 1 < m1 && MODE != kModeU) {
                    dv = pore ? dv : T(0);
                    acc[3] += (double)dv * (double)dv;
                }
            }
        }
        const int m = t - 2;
        if (m >= m0 && real0) {
            // ------------------------------------------------------ update on plane m
            T ux_n[CPT], uy_n[CPT], uz_n[CPT];
            if (MODE == kModeP) {
#pragma unroll
                for (int j = 0; j < CPT; ++j) {
                    ux_n[j] = qx[Q2][j];
                    uy_n[j] = qy[Q2][j];
                    uz_n[j] = qz[(kRot + 1 + 1) % 5][j];
                }
            } else {
                uint32_t c[CPT];
                ldv(c, &G2.cd[own - PNo]);
                const T *PN = S.pn[m & 1];  // index: box index - 2 BX
                const T *ux = G2.ux, *uy = G2.uy, *uz = G2.uz;
                const long long gidx = (long long)m * plane + gin_own;
                // u_x: along x (box), across y (box) and z (queue)
                {
                    const T *u0 = qx[Q2];
                    const Pair<T> L = ld2(&ux[own - 2]), R = ld2(&ux[own + CPT]);
                    T ym2[CPT], ym1[CPT], yp1[CPT], yp2[CPT], ext[CPT + 4], sx[CPT];
                    ldv(ym2, &ux[own - 2 * BX]);
                    ldv(ym1, &ux[own - BX]);
                    ldv(yp1, &ux[own + BX]);
                    ldv(yp2, &ux[own + 2 * BX]);
                    ext[0] = L.a;
                    ext[1] = L.b;
#pragma unroll
                    for (int j = 0; j < CPT; ++j) ext[j + 2] = u0[j];
                    ext[CPT + 2] = R.a;
                    ext[CPT + 3] = R.b;
                    if (SRC) ldv(sx, P.src + gidx);
                    const T pr = PN[own - 2 * BX + CPT];
#pragma unroll
                    for (int j = 0; j < CPT; ++j) {
                        T lap = fma(T(-2), u0[j], ext[j + 3] + ext[j + 1]);
                        if constexpr (TR) perp_t(lap, tc[2 * j + tslot(0, 1) / 4], 8 * (tslot(0, 1) % 4), ym2[j], ym1[j], u0[j], yp1[j], yp2[j]);
                        else perp(lap, c[j], code_shift(0, 1), ym2[j], ym1[j], u0[j], yp1[j], yp2[j]);
                        if constexpr (TR) perp_t(lap, tc[2 * j + tslot(0, 2) / 4], 8 * (tslot(0, 2) % 4), qx[Q0][j], qx[Q1][j], u0[j], qx[Q3][j], qx[Q4][j]);
                        else perp(lap, c[j], code_shift(0, 2), qx[Q0][j], qx[Q1][j], u0[j], qx[Q3][j], qx[Q4][j]);
                        if (ALPHA) {
                            const long long xr = gidx + j + 1 + (j == CPT - 1 ? exl_off : 0);
                            lap -= T(0.5) * (B.alpha[gidx + j] + B.alpha[xr]) * u0[j];
                        }
                        const T right = j == CPT - 1 ? pr : pn_m[j + 1];
                        T R0 = fma(B.inv_re, lap, P.f[0] - (right - pn_m[j]));
                        if (SRC) R0 += sx[j];
                        ux_n[j] = (c[j] & node_bit(0)) ? fma(B.dt, R0, u0[j]) : u0[j];
                    }
                }
                // u_y: along y (box), across x (box) and z (queue)
                {
                    const T *u0 = qy[Q2];
                    const int oy = own - UYo;
                    const Pair<T> L = ld2(&uy[oy - 2]), R = ld2(&uy[oy + CPT]);
                    T ym1[CPT], yp1[CPT], pny[CPT], ext[CPT + 4], sy[CPT];
                    ldv(ym1, &uy[oy - BX]);
                    ldv(yp1, &uy[oy + BX]);
                    ldv(pny, &PN[own - BX]);
                    ext[0] = L.a;
                    ext[1] = L.b;
#pragma unroll
                    for (int j = 0; j < CPT; ++j) ext[j + 2] = u0[j];
                    ext[CPT + 2] = R.a;
                    ext[CPT + 3] = R.b;
                    if (SRC) ldv(sy, P.src + N + gidx);
#pragma unroll
                    for (int j = 0; j < CPT; ++j) {
                        T lap = fma(T(-2), u0[j], yp1[j] + ym1[j]);
                        if constexpr (TR) perp_t(lap, tc[2 * j + tslot(1, 0) / 4], 8 * (tslot(1, 0) % 4), ext[j], ext[j + 1], ext[j + 2], ext[j + 3], ext[j + 4]);
                        else perp(lap, c[j], code_shift(1, 0), ext[j], ext[j + 1], ext[j + 2], ext[j + 3], ext[j + 4]);
                        if constexpr (TR) perp_t(lap, tc[2 * j + tslot(1, 2) / 4], 8 * (tslot(1, 2) % 4), qy[Q0][j], qy[Q1][j], u0[j], qy[Q3][j], qy[Q4][j]);
                        else perp(lap, c[j], code_shift(1, 2), qy[Q0][j], qy[Q1][j], u0[j], qy[Q3][j], qy[Q4][j]);
                        if (ALPHA) lap -= T(0.5) * (B.alpha[gidx + j] + B.alpha[gidx + j + ey_off]) * u0[j];
                        T R0 = fma(B.inv_re, lap, P.f[1] - (pny[j] - pn_m[j]));
                        if (SRC) R0 += sy[j];
                        uy_n[j] = (c[j] & node_bit(1)) ? fma(B.dt, R0, u0[j]) : u0[j];
                    }
                }
                // u_z: along z (queue), across x and y (box)
                {
                    const T *u0 = qz[(kRot + 1 + 1) % 5];
                    const Pair<T> L = ld2(&uz[own - 2]), R = ld2(&uz[own + CPT]);
                    T ym2[CPT], ym1[CPT], yp1[CPT], yp2[CPT], ext[CPT + 4], sz[CPT];
                    ldv(ym2, &uz[own - 2 * BX]);
                    ldv(ym1, &uz[own - BX]);
                    ldv(yp1, &uz[own + BX]);
                    ldv(yp2, &uz[own + 2 * BX]);
                    ext[0] = L.a;
                    ext[1] = L.b;
#pragma unroll
                    for (int j = 0; j < CPT; ++j) ext[j + 2] = u0[j];
                    ext[CPT + 2] = R.a;
                    ext[CPT + 3] = R.b;
                    if (SRC) ldv(sz, P.src + 2 * N + gidx);
                    long long g2 = 0;
                    if (ALPHA) {
                        const int zp = nb_coord(m + 1, nz, B.per[2]);
                        g2 = (long long)(zp >= 0 ? zp : m) * plane + gin_own;
                    }
#pragma unroll
                    for (int j = 0; j < CPT; ++j) {
                        T lap = fma(T(-2), u0[j], qz[(kRot + 1 + 2) % 5][j] + qz[(kRot + 1 + 0) % 5][j]);
                        if constexpr (TR) perp_t(lap, tc[2 * j + tslot(2, 0) / 4], 8 * (tslot(2, 0) % 4), ext[j], ext[j + 1], ext[j + 2], ext[j + 3], ext[j + 4]);
                        else perp(lap, c[j], code_shift(2, 0), ext[j], ext[j + 1], ext[j + 2], ext[j + 3], ext[j + 4]);
                        if constexpr (TR) perp_t(lap, tc[2 * j + tslot(2, 1) / 4], 8 * (tslot(2, 1) % 4), ym2[j], ym1[j], u0[j], yp1[j], yp2[j]);
                        else perp(lap, c[j], code_shift(2, 1), ym2[j], ym1[j], u0[j], yp1[j], yp2[j]);
                        if (ALPHA) lap -= T(0.5) * (B.alpha[gidx + j] + B.alpha[g2 + j]) * u0[j];
                        T R0 = fma(B.inv_re, lap, P.f[2] - (pn_new[j] - pn_m[j]));
                        if (SRC) R0 += sz[j];
                        uz_n[j] = (c[j] & node_bit(2)) ? fma(B.dt, R0, u0[j]) : u0[j];
                    }
                }
            }
            stv(outx, ux_n);
            stv(outx + N, uy_n);
            stv(outx + 2 * N, uz_n);
            stv(outp, pn_m);
            outx += plane;
            outp += plane;
            if (REDUCE) {
#pragma unroll
                for (int j = 0; j < CPT; ++j) {
                    acc[0] += (double)ux_n[j];
                    acc[1] += (double)uy_n[j];
                    acc[2] += (double)uz_n[j];
                }
            }
        }
        // publish p^n of plane t-1 (own cells and halo cells) for the next step's update
        stv(&S.pn[(t - 1) & 1][own - 2 * BX], pn_new);
        if (hrow) {
            // the +y halo row, CPT cells per thread (same arithmetic as press1)
            uint32_t hc[CPT];
            T hp[CPT], hux[CPT], huy[CPT], huyd[CPT], huz[CPT], huzd[CPT], hr[CPT], hn[CPT];
            ldv(hc, &G1.cd[hown - PNo]);
            ldv(hp, &G1.pin[hown - PNo]);
            ldv(hux, &G1.ux[hown]);
            const T huxl = G1.ux[hown - 1];
            ldv(huy, &G1.uy[hown - UYo]);
            ldv(huyd, &G1.uy[hown - BX - UYo]);
            ldv(huz, &G1.uz[hown]);
            ldv(huzd, &G2.uz[hown]);
#pragma unroll
            for (int j = 0; j < CPT; ++j) hr[j] = T(0);
            if (SRC && hg >= 0) {
                const int gz = nb_coord(t - 1, nz, B.per[2]);
                if (gz >= 0) ldv(hr, P.src + 3 * N + (long long)gz * plane + hg);
            }
#pragma unroll
            for (int j = 0; j < CPT; ++j) {
                const T left = j == 0 ? huxl : hux[j - 1];
                const T dv = (hux[j] - left) + (huy[j] - huyd[j]) + (huz[j] - huzd[j]);
                hn[j] = (hc[j] & 1u) ? (MODE == kModeU ? hp[j] : hp[j] - B.dtc2 * (dv - hr[j])) : T(0);
            }
            stv(&S.pn[(t - 1) & 1][hown - 2 * BX], hn);
        } else if (hcol) {
            S.pn[(t - 1) & 1][hown - 2 * BX] = press1(G1, G2, hown, t - 1, hg);
        }
#pragma unroll
        for (int j = 0; j < CPT; ++j) pn_m[j] = pn_new[j];
        s2 = s1;
        s1 = s0;
        s0 = s0 == STAGES - 1 ? 0 : s0 + 1;
        };
    for (int t = t0; t <= tend; t += 5) {
        step(std::integral_constant<int, 0>{}, t);
        if (t + 1 > tend) break;
        step(std::integral_constant<int, 1>{}, t + 1);
        if (t + 2 > tend) break;
        step(std::integral_constant<int, 2>{}, t + 2);
        if (t + 3 > tend) break;
        step(std::integral_constant<int, 3>{}, t + 3);
        if (t + 4 > tend) break;
        step(std::integral_constant<int, 4>{}, t + 4);
    }
    // drain this column's copies before the ring is reused
    cp_async_wait<0>();
    if (REDUCE) {
        for (int q = 0; q < 4; ++q)
            for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_down_sync(0xffffffffu, acc[q], o);
        if (lane == 0)
            for (int q = 0; q < 4; ++q) red[warp][q] = acc[q];
        __syncthreads();
        if (tid < 4) {
            double sum = 0.0;
            for (int w = 0; w < C::NW; ++w) sum += red[w][tid];
            red_sum[rs][tid] += sum;
        }
    }
    __syncthreads();
    }  // persistent loop
    (void)PL;
    if (REDUCE) {
        if (B.multi) {
            if (tid < 4) B.prob[mp].partials[((long long)blockIdx.x - B.prob[mp].unit_begin) * 4 + tid] = red_sum[0][tid];
        } else if (tid < B.nprob * 4) {
            B.prob[tid / 4].partials[blockIdx.x * 4 + (tid % 4)] = red_sum[tid / 4][tid % 4];
        }
    }
}

// ------------------------------------------------------------------ host helpers
struct TiledShape {
    int tiles_x, tiles_y, grid, zchunk;
    long long per_cta;
};

// Current device, or 0 if it cannot be read.
inline int current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        dev = 0;
    }
    return dev;
}

// Number of SMs of the current device (the persistent grid is a multiple of it), read
// once per device.
inline int tiled_grid_size() {
    constexpr int kDevs = 64;
    static std::atomic<int> sms_of[kDevs];
    const int dev = current_device();
    if (dev < 0 || dev >= kDevs) return 152;
    int sms = sms_of[dev].load(std::memory_order_relaxed);
    if (sms <= 0) {
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
            (void)cudaGetLastError();
            sms = 152;
        }
        sms_of[dev].store(sms, std::memory_order_relaxed);
    }
    return sms;
}

// CTAs per SM of a tile shape (FP64: one).
template <typename T>
inline int tile_min_blocks(int tile) {
    if (sizeof(T) != 4) return 1;
    return tile == 0 ? Tile64x12c2::MINB
                     : (tile == 1 ? Tile64x12c4::MINB : (tile == 2 ? Tile64x8c4::MINB : Tile64x12c4tr::MINB));
}

// Launch geometry.  zchunk = 0: persistent CTAs (MINB per SM, whole-column rounds then
// equal plane ranges); zchunk > 0: one CTA per (column, chunk of zchunk planes), the last
// chunk of each column cut into split_last(nz, zchunk, zsplit) sub-chunks.
template <typename T>
inline TiledShape tiled_shape(int nx, int ny, int nz, int nprob = 1, int zchunk = 0, int tile = 0, int zsplit = 1) {
    TiledShape s;
    const TileDims td = tile_dims(tile);
    s.tiles_x = (nx + td.tx - 1) / td.tx;
    s.tiles_y = (ny + td.ty - 1) / td.ty;
    const long long C = (long long)nprob * s.tiles_x * s.tiles_y;
    s.zchunk = zchunk > 0 ? (zchunk < nz ? zchunk : nz) : 0;
    if (s.zchunk > 0) {
        s.grid = (int)(C * ((nz + s.zchunk - 1) / s.zchunk - 1 + split_last(nz, s.zchunk, zsplit)));
        s.per_cta = 0;
    } else {
        s.grid = tiled_grid_size() * tile_min_blocks<T>(tile);
        // plane steps per CTA in the second phase (columns left after whole rounds)
        const long long rem = (C - (C / s.grid) * s.grid) * nz;
        s.per_cta = (rem + s.grid - 1) / s.grid;
    }
    return s;
}

// Schedules the autotuner tries for a tile shape: persistent, and plane chunks giving
// about 3..8 CTAs of work per resident CTA slot.
inline int tiled_candidates(int nx, int ny, int nz, int nprob, int out[8], int tile = 0) {
    int n = 0;
    out[n++] = 0;
    const TileDims td = tile_dims(tile);
    const long long C = (long long)nprob * ((nx + td.tx - 1) / td.tx) * ((ny + td.ty - 1) / td.ty);
    const long long slots = (long long)tiled_grid_size() * tile_min_blocks<float>(tile);
    for (int w = 3; w <= 8 && n < 8; ++w) {
        long long chunks = (w * slots + C - 1) / C;
        if (chunks < 1) chunks = 1;
        int zc = (int)((nz + chunks - 1) / chunks);
        if (zc < 12) zc = 12;
        if (zc > nz) zc = nz;
        bool dup = false;
        for (int i = 0; i < n; ++i) dup |= out[i] == zc;
        if (!dup) out[n++] = zc;
    }
    return n;
}

// The tiled kernel copies whole 16-byte chunks of 4 cells: x extents must be multiples
// of 4 (the simple kernel serves the other shapes); in-plane offsets are 32-bit.
template <typename T>
inline bool tiled_supported(int nx, int ny, int nz, int nprob) {
    return nx >= 4 && nx % 4 == 0 && ny >= 1 && nz >= 1 && nprob >= 1 && nprob <= kMaxBatch &&
           (long long)nx * ny < (1ll << 31);
}

// Number of reduction partials per drive written by one launch (one per CTA).
template <typename T>
inline long long tiled_num_blocks(int nx, int ny, int nz, int nprob, int zchunk = 0, int tile = 0, int zsplit = 1) {
    return tiled_shape<T>(nx, ny, nz, nprob, zchunk, tile, zsplit).grid;
}

// Largest grid over the autotuner's candidates of every tile shape (sizes the
// reduction buffers).
template <typename T>
inline long long tiled_max_blocks(int nx, int ny, int nz, int nprob) {
    long long g = 0;
    for (int t = 0; t < tile_count<T>(); ++t) {
        int cand[8];
        const int n = tiled_candidates(nx, ny, nz, nprob, cand, t);
        for (int i = 0; i < n; ++i)
            for (int sp : kSplits) {
                const long long b = tiled_num_blocks<T>(nx, ny, nz, nprob, cand[i], t, sp);
                g = b > g ? b : g;
            }
    }
    return g;
}

template <typename T, class C, int MODE, bool RED, bool SRC, bool ALPHA, bool TR = false>
inline cudaError_t launch_tiled_t(const SweepBatch<T> &B, const uint32_t *code, int zchunk, int tile,
                                  cudaStream_t s) {
    TiledShape sh = B.multi ? TiledShape{} : tiled_shape<T>(B.nx, B.ny, B.nz, B.nprob, zchunk, tile, B.zsplit);
    if (B.multi) {
        const SweepProblem<T> &L = B.prob[B.nprob - 1];
        sh.grid = (int)(L.unit_begin + (long long)L.tiles_x * L.tiles_y * ((L.nz + L.zchunk - 1) / L.zchunk));
    }
    const size_t smem = sizeof(TiledSmem<T, C>);
    auto kern = sweep_tiled_kernel<T, C, MODE, RED, SRC, ALPHA, TR>;
    // the shared-memory attributes are per device: one bit per device and instantiation
    static std::atomic<unsigned long long> attr_set{0};
    const int dev = current_device();
    const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
    if (!bit || !(attr_set.load(std::memory_order_acquire) & bit)) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess) return e;
        attr_set.fetch_or(bit, std::memory_order_acq_rel);
    }
    kern<<<sh.grid, C::NT, smem, s>>>(B, code, sh.tiles_x, sh.tiles_y, sh.per_cta, sh.zchunk);
    return cudaGetLastError();
}

template <typename T, class C, int MODE>
inline cudaError_t launch_tiled_m(const SweepBatch<T> &B, const uint32_t *code, bool red, bool src, int zc, int tile,
                                  cudaStream_t s) {
    const bool alpha = B.alpha != nullptr;
    if (red) {
        if (src) return alpha ? launch_tiled_t<T, C, MODE, true, true, true>(B, code, zc, tile, s)
                              : launch_tiled_t<T, C, MODE, true, true, false>(B, code, zc, tile, s);
        return alpha ? launch_tiled_t<T, C, MODE, true, false, true>(B, code, zc, tile, s)
                     : launch_tiled_t<T, C, MODE, true, false, false>(B, code, zc, tile, s);
    }
    if (src) return alpha ? launch_tiled_t<T, C, MODE, false, true, true>(B, code, zc, tile, s)
                          : launch_tiled_t<T, C, MODE, false, true, false>(B, code, zc, tile, s);
    return alpha ? launch_tiled_t<T, C, MODE, false, false, true>(B, code, zc, tile, s)
                 : launch_tiled_t<T, C, MODE, false, false, false>(B, code, zc, tile, s);
}

template <typename T, class C>
inline cudaError_t launch_tiled_c(const SweepBatch<T> &B, const uint32_t *code, int mode, bool red, bool src,
                                  int zchunk, int tile, cudaStream_t s) {
    if (mode == kModeU) return launch_tiled_m<T, C, kModeU>(B, code, red, src, zchunk, tile, s);
    if (mode == kModePU) return launch_tiled_m<T, C, kModePU>(B, code, red, src, zchunk, tile, s);
    return launch_tiled_m<T, C, kModeP>(B, code, red, src, zchunk, tile, s);
}

// Transposed sweep (adjoint solves; drag and reductions as needed, no source term).
template <typename T, class C>
inline cudaError_t launch_tiled_tr(const SweepBatch<T> &B, const uint32_t *code, int mode, bool red, int zc,
                                   int tile, cudaStream_t s) {
    const bool alpha = B.alpha != nullptr;
#define PM_TR_LAUNCH(M)                                                                                   \
    return red ? (alpha ? launch_tiled_t<T, C, M, true, false, true, true>(B, code, zc, tile, s)          \
                        : launch_tiled_t<T, C, M, true, false, false, true>(B, code, zc, tile, s))        \
               : (alpha ? launch_tiled_t<T, C, M, false, false, true, true>(B, code, zc, tile, s)         \
                        : launch_tiled_t<T, C, M, false, false, false, true>(B, code, zc, tile, s));
    if (mode == kModeU) { PM_TR_LAUNCH(kModeU) }
    if (mode == kModePU) { PM_TR_LAUNCH(kModePU) }
    PM_TR_LAUNCH(kModeP)
#undef PM_TR_LAUNCH
}

// Per-shape launchers, each compiled in its own translation unit (pm_sweep_*.cu).
cudaError_t launch_tiled_f32_t0(const SweepBatch<float> &B, const uint32_t *code, int mode, bool red, bool src,
                                int zchunk, cudaStream_t s);
cudaError_t launch_tiled_f32_t1(const SweepBatch<float> &B, const uint32_t *code, int mode, bool red, bool src,
                                int zchunk, cudaStream_t s);
cudaError_t launch_tiled_f32_t2(const SweepBatch<float> &B, const uint32_t *code, int mode, bool red, bool src,
                                int zchunk, cudaStream_t s);
cudaError_t launch_tiled_f64_t0(const SweepBatch<double> &B, const uint32_t *code, int mode, bool red, bool src,
                                int zchunk, cudaStream_t s);
cudaError_t launch_tiled_f32_tr(const SweepBatch<float> &B, const uint32_t *code, int mode, bool red, int zchunk,
                                cudaStream_t s);

// Transposed sweep of FP32 fields (tile shape kTileTR: 64 x 12 cells, four per thread, one
// CTA per SM).  Returns a pm_status.
inline int launch_tiled_transposed(const SweepBatch<float> &B, const uint32_t *code, int mode, bool red, int zchunk,
                                   cudaStream_t s) {
    const cudaError_t e = launch_tiled_f32_tr(B, code, mode, red, zchunk, s);
    return e == cudaSuccess ? 0 : (e == cudaErrorMemoryAllocation ? 6 : 7);
}

// One sweep launch with tile shape `tile` (0: 64 x 12, two cells per thread; 1: 64 x 12,
// four cells per thread; 2: 64 x 8, four cells per thread); FP64 fields use shape 0 (the
// FP64 kernel is bound by the FP64 rate).  Returns a pm_status.
inline int launch_tiled(const SweepBatch<float> &B, const uint32_t *code, int mode, bool red, bool src, int zchunk,
                        cudaStream_t s, int tile = 0) {
    const cudaError_t e = tile == 1   ? launch_tiled_f32_t1(B, code, mode, red, src, zchunk, s)
                          : tile == 2 ? launch_tiled_f32_t2(B, code, mode, red, src, zchunk, s)
                                      : launch_tiled_f32_t0(B, code, mode, red, src, zchunk, s);
    return e == cudaSuccess ? 0 : (e == cudaErrorMemoryAllocation ? 6 : 7);
}
inline int launch_tiled(const SweepBatch<double> &B, const uint32_t *code, int mode, bool red, bool src, int zchunk,
                        cudaStream_t s, int = 0) {
    const cudaError_t e = launch_tiled_f64_t0(B, code, mode, red, src, zchunk, s);
    return e == cudaSuccess ? 0 : (e == cudaErrorMemoryAllocation ? 6 : 7);
}

}  // namespace pmgb
