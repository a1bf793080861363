// Tiled z-marching fused sweep, tile shape 1 (64 x 12 cells, a pair of x-adjacent cells
// per thread, 384 threads, 5-stage ring two planes ahead, 2 CTAs per SM).  The arithmetic
// per cell is the one of the general kernel in pm_sweep_tiled.cuh (bit-identical fields);
// this version is written out for pairs so that it fits 80 registers without spills.
//
// A CTA owns a TX x TY column tile of the (x, y) plane and marches along z over a chunk
// of planes.  Each plane of the five input arrays (u_x, u_y, u_z, p, stencil code) is
// copied with its 2-voxel halo into the shared-memory ring by 16-byte cp.async, so each
// field value comes from DRAM once per sweep and the neighbour reuse is served by shared
// memory (x, y) and per-thread register queues (z).
#pragma once

#include "pm_sweep_tiled.cuh"

namespace pmgb {
namespace pair {

// ------------------------------------------------------------------ cp.async helpers (pair kernel)
// 16-byte asynchronous global -> shared copies (L2 only: the tile is staged in shared
// memory, nothing is reused from L1).
__device__ __forceinline__ void cp_async16(void *s, const void *g) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(s);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(g) : "memory");
}
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

// ------------------------------------------------------------------ kernel
// Tile TX x TY cells, thread (lane, ty) owns the pair of cells (x0 + 2 lane, y0 + ty) and
// (x0 + 2 lane + 1, y0 + ty).  Shared-memory boxes are BX = TX + 8 wide (x0 - 4 ..
// x0 + TX + 3, whole 16-byte chunks) and BY = TY + 4 high (y0 - 2 .. y0 + TY + 1); the
// stencil needs +-2 in x and y.
constexpr int kTX = 64, kTY = 12, kBX = kTX + 8, kBY = kTY + 4, kPL = kBX * kBY;
// Ring of kStages planes: planes t-2, t-1, t are read in step t while the copies of the
// next kAhead planes are in flight.
constexpr int kStages = 5, kAhead = kStages - 3;
// p^n, the input pressure and the stencil codes are needed on box rows 2 .. kTY + 2 (tile
// rows and the +y halo row) only, u_y on rows 1 .. kTY + 2; u_x and u_z on all rows
constexpr int kPNL = (kTY + 1) * kBX, kPNo = 2 * kBX;
constexpr int kUYL = (kTY + 2) * kBX, kUYo = kBX;
// CTAs per SM the FP32 kernel is built for (registers and shared memory)
constexpr int kMinBlocks = 2;
constexpr int kNT = (kTX / 2) * kTY;

// One ring stage: the five arrays of one plane, contiguous, so that every access is a
// per-step stage pointer plus a compile-time offset.  Arrays that need fewer box rows
// start at a later row: u_y at row 1 (index = box index - kUYo), p and the codes at
// row 2 (index = box index - kPNo).
template <typename T>
struct TiledStage {
    T ux[kPL];
    T uz[kPL];
    T uy[kUYL];
    T pin[kPNL];
    uint32_t cd[kPNL];
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

template <typename T>
struct TiledSmem {
    TiledStage<T> st[kStages];
    T pn[2][kPNL];  // index: box index - 2 kBX
    WallCoef<T> coef[4];
};

// A pair of x-adjacent values (aligned for one 2-wide shared-memory access).
template <typename T>
struct alignas(2 * sizeof(T)) Pair {
    T a, b;
};
template <typename T>
__device__ __forceinline__ Pair<T> ld2(const T *p) {
    return *reinterpret_cast<const Pair<T> *>(p);
}
template <typename T>
__device__ __forceinline__ Pair<uint32_t> ld2u(const uint32_t *p) {
    return *reinterpret_cast<const Pair<uint32_t> *>(p);
}

// Byte offset of the coefficient-table entry of the wall kind at bit sh of word c (one
// shift and one mask: entries are 2 T, a power of two).
template <typename T>
__device__ __forceinline__ uint32_t coef_offset(uint32_t c, int sh) {
    constexpr int lg = sizeof(T) == 4 ? 3 : 4;
    static_assert(sizeof(WallCoef<T>) == (1u << lg), "entry size");
    return (c >> (sh - lg)) & (3u << lg);
}

// PRES: fixed-pressure axis B.pres_axis - 1 (single geometry, no source, no drag).  Its
// first and last cell layers are reservoirs whose pore cells hold the fixed pressures
// P.pres[0] / P.pres[1] (their cross-flow nodes are non-fluid in the stencil codes), and
// the axial second difference of the nodes on the inlet face (coordinate 0) and on the
// outlet face (coordinate n - 2) takes the node itself as its outer neighbour (zero
// gradient), as in the simple kernel.
template <typename T, int MODE, bool REDUCE, bool SRC, bool ALPHA, bool PRES = false>
__global__ void __launch_bounds__(kNT, sizeof(T) == 4 ? kMinBlocks : 1)
    sweep_tiled_kernel(const SweepBatch<T> B, const uint32_t *__restrict__ code, int tiles_x, int tiles_y,
                       long long per_cta, int zchunk) {
    // single geometry: B.nx.. and the arguments; multi-geometry: per problem (below)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TiledSmem<T> &S = *reinterpret_cast<TiledSmem<T> *>(smem_raw);
    int nx = B.nx, ny = B.ny, nz = B.nz;
    long long N = B.N, plane = (long long)nx * ny;
    const int tid = threadIdx.x;
    const int lane = tid & 31, ty = tid >> 5;
    const unsigned char *coef_bytes = reinterpret_cast<const unsigned char *>(S.coef);
    __shared__ double red_sum[kMaxSame][4];  // per drive: FP64 sums of this CTA
    __shared__ double red[kNT / 32][4];
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
    }

    // fixed-pressure axis and its length (PRES only)
    const int pax = PRES ? B.pres_axis - 1 : -1;
    const int npax = pax == 0 ? nx : (pax == 1 ? ny : nz);

    // Persistent CTAs over columns (a column = one drive on one x-y tile, all planes).
    // Phase 1: rounds in which CTA b marches whole column r G + b, so that all CTAs are at
    // the same plane and the tile halos they share are served by L2.  Phase 2: the
    // remaining columns, column by column, split into equal contiguous plane ranges
    // (short pieces, neighbouring columns again at similar planes).  Every CTA gets the
    // same number of plane steps, with at most one restart of its plane pipeline.
    // zchunk > 0 instead: one (column, plane chunk) unit per CTA, chunk-major order.
    const long long G = gridDim.x, C = (long long)B.nprob * tiles_x * tiles_y;
    const long long rounds = zchunk > 0 ? 0 : C / G, rem_total = zchunk > 0 ? 0 : (C - rounds * G) * nz;
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
        chunk_unit(blockIdx.x, C, nz, zchunk, split_last(nz, zchunk, B.zsplit), col, m0, m1);
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
    const int x0 = (tile % tiles_x) * kTX, y0 = (tile / tiles_x) * kTY;
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
    constexpr int FR = (FCH * kBY + kNT - 1) / kNT;
    int fo[FR], fs[FR];
    bool fhas[FR], fuy[FR], fp[FR];  // chunk exists / row also holds u_y / also p
#pragma unroll
    for (int r = 0; r < FR; ++r) {
        const int c = tid + r * kNT;
        fo[r] = -1;
        fs[r] = 0;
        fhas[r] = c < FCH * kBY;
        fuy[r] = fp[r] = false;
        if (fhas[r]) {
            const int hy = c / FCH, hx = (c % FCH) * FE;
            fs[r] = hy * kBX + hx;
            fuy[r] = hy >= 1 && hy <= kTY + 2;
            fp[r] = hy >= 2 && hy <= kTY + 2;
            const int gx = nb_coord(x0 - 4 + hx, nx, B.per[0]), gy = nb_coord(y0 - 2 + hy, ny, B.per[1]);
            if (gx >= 0 && gy >= 0) fo[r] = gx + nx * gy;
        }
    }
    // code chunks: box rows 2 .. kTY + 2; cs is the index in the stage's code array
    int co = -1, cs = 0;
    const bool chas = tid < CCH * (kTY + 1);
    if (chas) {
        const int hy = 2 + tid / CCH, hx = (tid % CCH) * 4;
        cs = hy * kBX + hx - kPNo;
        const int gx = nb_coord(x0 - 4 + hx, nx, B.per[0]), gy = nb_coord(y0 - 2 + hy, ny, B.per[1]);
        if (gx >= 0 && gy >= 0) co = gx + nx * gy;
    }
    auto issue_plane = [&](int k, int slot) {
        TiledStage<T> &G = S.st[slot];
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
            cp_async16z(&G.ux[e], gux + o, nb);
            cp_async16z(&G.uz[e], guz + o, nb);
            if (fuy[r]) cp_async16z(&G.uy[e - kUYo], guy + o, nb);
            if (fp[r]) cp_async16z(&G.pin[e - kPNo], gp + o, nb);
        }
        if (chas) {
            const bool in = gz >= 0 && co >= 0;
            cp_async16z(&G.cd[cs], code + (in ? po + co : 0), in ? 16u : 0u);
        }
        cp_async_commit();
    };

    const int own = (ty + 2) * kBX + 4 + 2 * lane;  // box index of the first cell of the pair
    const int gx_own = x0 + 2 * lane, gy_own = y0 + ty;
    const bool real0 = gx_own < nx && gy_own < ny;       // nx % 4 == 0: both cells or neither
    const long long gin_own = (long long)gx_own + (long long)nx * gy_own;
    // tile positions past the domain edge stand for their periodic image (or for solid
    // outside a wall): their pressure is formed at the wrapped index, nothing is written
    long long gin_wrap = -1;
    {
        const int wx = nb_coord(gx_own, nx, B.per[0]), wy = nb_coord(gy_own, ny, B.per[1]);
        if (wx >= 0 && wy >= 0) gin_wrap = (long long)wx + (long long)nx * wy;
    }
    // halo p^n: the last warp takes the row y0 + TY (pairs), the last TY lanes of the
    // warp before it the column x0 + TX (single cells); for FP32 these lanes issue no
    // copies (288 chunks per array), which balances the work before the barrier
    const bool hrow = ty == kTY - 1, hcol = ty == kTY - 2 && lane >= 32 - kTY;
    const int hown = hrow ? (kTY + 2) * kBX + 4 + 2 * lane : (lane - (32 - kTY) + 2) * kBX + kTX + 4;
    long long hg = -1;
    if ((hrow || hcol) && SRC) {
        const int gx = nb_coord(x0 + (hown % kBX) - 4, nx, B.per[0]), gy = nb_coord(y0 + hown / kBX - 2, ny, B.per[1]);
        if (gx >= 0 && gy >= 0) hg = (long long)gx + (long long)nx * gy;
    }
    // offsets to the +x / +y cell for the drag term; at a wall the face is not fluid and the
    // value is discarded, so the cell itself stands in (keeps the read in bounds)
    const int wxp = nb_coord(gx_own + 2, nx, B.per[0]), wyp = nb_coord(gy_own + 1, ny, B.per[1]);
    const long long ex1_off = wxp >= 0 ? (long long)wxp - (gx_own + 1) : 0;  // second cell's +x
    const long long ey_off = wyp >= 0 ? ((long long)wyp - gy_own) * nx : 0;

    // PRES: reservoir of the cell at box index e on plane k (0 inlet, 1 outlet, -1 none);
    // coordinates outside the box along the (non-periodic) axis are no reservoir
    auto reservoir = [&](int e, int k) -> int {
        const int v = pax == 0 ? x0 + e % kBX - 4 : (pax == 1 ? y0 + e / kBX - 2 : k);
        return v == 0 ? 0 : (v == npax - 1 ? 1 : -1);
    };
    // p^n of a reservoir cell: its fixed pressure if pore (code bit 0), else 0
    auto res_p = [&](int r, uint32_t c) -> T { return (c & 1u) ? P.pres[r] : T(0); };

    Pair<T> qx[5], qy[5], qz[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) qx[i] = qy[i] = Pair<T>{T(0), T(0)};
#pragma unroll
    for (int i = 0; i < 5; ++i) qz[i] = Pair<T>{T(0), T(0)};
    Pair<T> pn_m{T(0), T(0)};  // own p^n on the plane being updated (m)
    double acc[4] = {0.0, 0.0, 0.0, 0.0};

    const int t0 = m0 - 2;
    int s2 = ((t0 - 2) % kStages + kStages) % kStages;  // ring stages of planes t-2, t-1, t
    int s1 = (s2 + 1) % kStages, s0 = (s2 + 2) % kStages;
    {
        int sl = s0;
        for (int k = 0; k < kAhead; ++k) {
            issue_plane(t0 + k, sl);
            sl = sl == kStages - 1 ? 0 : sl + 1;
        }
    }

    // p^n of one cell at box position e of plane k (stage K), the plane below in KM
    auto press1 = [&](const TiledStage<T> &K, const TiledStage<T> &KM, int e, int k, long long g) -> T {
        const T dv = (K.ux[e] - K.ux[e - 1]) + (K.uy[e - kUYo] - K.uy[e - kBX - kUYo]) + (K.uz[e] - KM.uz[e]);
        T rp = T(0);
        if (SRC && g >= 0) {
            const int gz = nb_coord(k, nz, B.per[2]);
            if (gz >= 0) rp = P.src[3 * N + (long long)gz * plane + g];
        }
        const T p0 = K.pin[e - kPNo];
        if (PRES) {
            const int r = reservoir(e, k);
            if (r >= 0) return res_p(r, K.cd[e - kPNo]);
        }
        const T pn = MODE == kModeU ? p0 : p0 - B.dtc2 * (dv - rp);
        return pn;  // a solid cell keeps p = 0: its six faces hold 0, so dv = 0 and rp = 0
    };
    // second derivative across the flow (Appendix B) from the 3-bit wall code, added to lap
    auto perp = [&](T &lap, uint32_t cc, int sh, T um2, T um1, T u0, T up1, T up2) {
        const WallCoef<T> w = *reinterpret_cast<const WallCoef<T> *>(coef_bytes + coef_offset<T>(cc, sh));
        const uint32_t n = cc >> sh;
        lap = fma(w.A, fma(T(-2), u0, um1 + up1), lap);
        const T far = (n & 4u) ? up2 : um2;
        lap = fma(w.K, fma(T(1) / T(5), far, u0), lap);
    };

    T *outx = P.uout + (long long)m0 * plane + gin_own;
    T *outp = P.pout + (long long)m0 * plane + gin_own;
    const int tend = m1 + 1;
    // one plane step; kRot = step index mod 5.  The z queues are circular with compile-time
    // slots, so advancing them moves no registers: after this step's load, queue entry k
    // (u_x, u_y: planes m-2 .. m+2 of the updated plane m = t-2; u_z: planes m-1 .. m+1 as
    // entries 0 .. 2) lives in slot (kRot + 1 + k) % 5.  The loop below unrolls five steps.
    auto step = [&](auto Rc, int t) {
        constexpr int kRot = decltype(Rc)::value;
        cp_async_wait<kAhead - 1>();
        __syncthreads();
        {
            int sl = s0 + kAhead;
            if (sl >= kStages) sl -= kStages;
            issue_plane(t + kAhead, sl);
        }
        if (SRC && real0 && t >= m0 && t < m1) {
            // the source of plane t is read two steps (velocity) and one step (pressure)
            // from now: bring its lines into L2 without holding registers
            const long long g = (long long)t * plane + gin_own;
            asm volatile("prefetch.global.L2 [%0];\n" ::"l"(P.src + g));
            asm volatile("prefetch.global.L2 [%0];\n" ::"l"(P.src + N + g));
            asm volatile("prefetch.global.L2 [%0];\n" ::"l"(P.src + 2 * N + g));
            asm volatile("prefetch.global.L2 [%0];\n" ::"l"(P.src + 3 * N + g));
        }
        const TiledStage<T> &G0 = S.st[s0], &G1 = S.st[s1], &G2 = S.st[s2];
        // z queues of the own column pair
        qx[kRot % 5] = ld2(&G0.ux[own]);
        qy[kRot % 5] = ld2(&G0.uy[own - kUYo]);
        qz[(kRot + 3) % 5] = ld2(&G1.uz[own]);
        // own p^n on plane t-1 (kept in registers until after the update of plane t-2)
        Pair<T> pn_new;
        {
            const Pair<T> pin = ld2(&G1.pin[own - kPNo]);
            const Pair<T> uyd = ld2(&G1.uy[own - kBX - kUYo]);
            const T uxl = G1.ux[own - 1];
            T dv0 = (qx[(kRot + 1 + 3) % 5].a - uxl) + (qy[(kRot + 1 + 3) % 5].a - uyd.a) + (qz[(kRot + 1 + 2) % 5].a - qz[(kRot + 1 + 1) % 5].a);
            T dv1 = (qx[(kRot + 1 + 3) % 5].b - qx[(kRot + 1 + 3) % 5].a) + (qy[(kRot + 1 + 3) % 5].b - uyd.b) + (qz[(kRot + 1 + 2) % 5].b - qz[(kRot + 1 + 1) % 5].b);
            T rp0 = T(0), rp1 = T(0);
            if (SRC && gin_wrap >= 0) {
                const int gz = nb_coord(t - 1, nz, B.per[2]);
                if (gz >= 0) {
                    const Pair<T> r = ld2(P.src + 3 * N + (long long)gz * plane + gin_wrap);
                    rp0 = r.a;
                    rp1 = r.b;
                }
            }
            // no pore test: a solid cell has six non-fluid faces (exactly 0), so dv = 0, the
            // source is 0 there and p stays 0
            pn_new.a = MODE == kModeU ? pin.a : pin.a - B.dtc2 * (dv0 - rp0);
            pn_new.b = MODE == kModeU ? pin.b : pin.b - B.dtc2 * (dv1 - rp1);
            if (PRES) {
                const int ra = reservoir(own, t - 1), rb = reservoir(own + 1, t - 1);
                if (ra >= 0 || rb >= 0) {
                    const Pair<uint32_t> cc = ld2u<T>(&G1.cd[own - kPNo]);
                    if (ra >= 0) {
                        pn_new.a = res_p(ra, cc.a);
                        dv0 = T(0);  // a reservoir has no continuity residual
                    }
                    if (rb >= 0) {
                        pn_new.b = res_p(rb, cc.b);
                        dv1 = T(0);
                    }
                }
            }
            if (REDUCE && real0 && t - 1 >= m0 && t - 1 < m1 && MODE != kModeU) {
                acc[3] += (double)dv0 * (double)dv0 + (double)dv1 * (double)dv1;
            }
        }
        const int m = t - 2;
        if (m >= m0 && real0) {
            // ------------------------------------------------------ update on plane m
            Pair<T> ux_n, uy_n, uz_n;
            if (MODE == kModeP) {
                ux_n = qx[(kRot + 1 + 2) % 5];
                uy_n = qy[(kRot + 1 + 2) % 5];
                uz_n = qz[(kRot + 1 + 1) % 5];
            } else {
                const Pair<uint32_t> c = ld2u<T>(&G2.cd[own - kPNo]);
                const T *PN = S.pn[m & 1];  // index: box index - 2 kBX
                const T *ux = G2.ux, *uy = G2.uy, *uz = G2.uz;
                const long long gidx = (long long)m * plane + gin_own;
                // u_x: along x (box), across y (box) and z (queue)
                {
                    const Pair<T> u0 = qx[(kRot + 1 + 2) % 5];
                    const Pair<T> L = ld2(&ux[own - 2]), R = ld2(&ux[own + 2]);
                    const Pair<T> ym2 = ld2(&ux[own - 2 * kBX]), ym1 = ld2(&ux[own - kBX]);
                    const Pair<T> yp1 = ld2(&ux[own + kBX]), yp2 = ld2(&ux[own + 2 * kBX]);
                    // -x / +x neighbours of the two cells (the pair's own values inside)
                    T xm0 = L.b, xp0 = u0.b, xm1 = u0.a, xp1 = R.a;
                    if (PRES && pax == 0) {
                        // inlet / outlet faces of a fixed-pressure x axis: zero gradient
                        if (gx_own == 0) xm0 = u0.a;
                        if (gx_own == nx - 2) xp0 = u0.a;
                        if (gx_own + 1 == nx - 2) xp1 = u0.b;
                    }
                    T lap0 = fma(T(-2), u0.a, xp0 + xm0);
                    T lap1 = fma(T(-2), u0.b, xp1 + xm1);
                    perp(lap0, c.a, code_shift(0, 1), ym2.a, ym1.a, u0.a, yp1.a, yp2.a);
                    perp(lap1, c.b, code_shift(0, 1), ym2.b, ym1.b, u0.b, yp1.b, yp2.b);
                    perp(lap0, c.a, code_shift(0, 2), qx[(kRot + 1 + 0) % 5].a, qx[(kRot + 1 + 1) % 5].a, u0.a, qx[(kRot + 1 + 3) % 5].a, qx[(kRot + 1 + 4) % 5].a);
                    perp(lap1, c.b, code_shift(0, 2), qx[(kRot + 1 + 0) % 5].b, qx[(kRot + 1 + 1) % 5].b, u0.b, qx[(kRot + 1 + 3) % 5].b, qx[(kRot + 1 + 4) % 5].b);
                    if (ALPHA) {
                        lap0 -= T(0.5) * (B.alpha[gidx] + B.alpha[gidx + 1]) * u0.a;
                        lap1 -= T(0.5) * (B.alpha[gidx + 1] + B.alpha[gidx + 1 + ex1_off]) * u0.b;
                    }
                    const T pr = PN[own - 2 * kBX + 2];
                    T R0 = fma(B.inv_re, lap0, P.f[0] - (pn_m.b - pn_m.a));
                    T R1 = fma(B.inv_re, lap1, P.f[0] - (pr - pn_m.b));
                    if (SRC) {
                        const Pair<T> sx = ld2(P.src + gidx);
                        R0 += sx.a;
                        R1 += sx.b;
                    }
                    ux_n.a = (c.a & node_bit(0)) ? fma(B.dt, R0, u0.a) : u0.a;
                    ux_n.b = (c.b & node_bit(0)) ? fma(B.dt, R1, u0.b) : u0.b;
                }
                // u_y: along y (box), across x (box) and z (queue)
                {
                    const Pair<T> u0 = qy[(kRot + 1 + 2) % 5];
                    const int oy = own - kUYo;
                    const Pair<T> L = ld2(&uy[oy - 2]), R = ld2(&uy[oy + 2]);
                    Pair<T> ym1 = ld2(&uy[oy - kBX]), yp1 = ld2(&uy[oy + kBX]);
                    if (PRES && pax == 1) {
                        if (gy_own == 0) ym1 = u0;
                        if (gy_own == ny - 2) yp1 = u0;
                    }
                    T lap0 = fma(T(-2), u0.a, yp1.a + ym1.a);
                    T lap1 = fma(T(-2), u0.b, yp1.b + ym1.b);
                    perp(lap0, c.a, code_shift(1, 0), L.a, L.b, u0.a, u0.b, R.a);
                    perp(lap1, c.b, code_shift(1, 0), L.b, u0.a, u0.b, R.a, R.b);
                    perp(lap0, c.a, code_shift(1, 2), qy[(kRot + 1 + 0) % 5].a, qy[(kRot + 1 + 1) % 5].a, u0.a, qy[(kRot + 1 + 3) % 5].a, qy[(kRot + 1 + 4) % 5].a);
                    perp(lap1, c.b, code_shift(1, 2), qy[(kRot + 1 + 0) % 5].b, qy[(kRot + 1 + 1) % 5].b, u0.b, qy[(kRot + 1 + 3) % 5].b, qy[(kRot + 1 + 4) % 5].b);
                    if (ALPHA) {
                        lap0 -= T(0.5) * (B.alpha[gidx] + B.alpha[gidx + ey_off]) * u0.a;
                        lap1 -= T(0.5) * (B.alpha[gidx + 1] + B.alpha[gidx + 1 + ey_off]) * u0.b;
                    }
                    const Pair<T> pny = ld2(&PN[own - kBX]);
                    T R0 = fma(B.inv_re, lap0, P.f[1] - (pny.a - pn_m.a));
                    T R1 = fma(B.inv_re, lap1, P.f[1] - (pny.b - pn_m.b));
                    if (SRC) {
                        const Pair<T> sy = ld2(P.src + N + gidx);
                        R0 += sy.a;
                        R1 += sy.b;
                    }
                    uy_n.a = (c.a & node_bit(1)) ? fma(B.dt, R0, u0.a) : u0.a;
                    uy_n.b = (c.b & node_bit(1)) ? fma(B.dt, R1, u0.b) : u0.b;
                }
                // u_z: along z (queue), across x and y (box)
                {
                    const Pair<T> u0 = qz[(kRot + 1 + 1) % 5];
                    const Pair<T> L = ld2(&uz[own - 2]), R = ld2(&uz[own + 2]);
                    const Pair<T> ym2 = ld2(&uz[own - 2 * kBX]), ym1 = ld2(&uz[own - kBX]);
                    const Pair<T> yp1 = ld2(&uz[own + kBX]), yp2 = ld2(&uz[own + 2 * kBX]);
                    Pair<T> zp1 = qz[(kRot + 1 + 2) % 5], zm1 = qz[(kRot + 1 + 0) % 5];
                    if (PRES && pax == 2) {
                        if (m == 0) zm1 = u0;
                        if (m == nz - 2) zp1 = u0;
                    }
                    T lap0 = fma(T(-2), u0.a, zp1.a + zm1.a);
                    T lap1 = fma(T(-2), u0.b, zp1.b + zm1.b);
                    perp(lap0, c.a, code_shift(2, 0), L.a, L.b, u0.a, u0.b, R.a);
                    perp(lap1, c.b, code_shift(2, 0), L.b, u0.a, u0.b, R.a, R.b);
                    perp(lap0, c.a, code_shift(2, 1), ym2.a, ym1.a, u0.a, yp1.a, yp2.a);
                    perp(lap1, c.b, code_shift(2, 1), ym2.b, ym1.b, u0.b, yp1.b, yp2.b);
                    if (ALPHA) {
                        const int zp = nb_coord(m + 1, nz, B.per[2]);
                        const long long g2 = (long long)(zp >= 0 ? zp : m) * plane + gin_own;
                        lap0 -= T(0.5) * (B.alpha[gidx] + B.alpha[g2]) * u0.a;
                        lap1 -= T(0.5) * (B.alpha[gidx + 1] + B.alpha[g2 + 1]) * u0.b;
                    }
                    T R0 = fma(B.inv_re, lap0, P.f[2] - (pn_new.a - pn_m.a));
                    T R1 = fma(B.inv_re, lap1, P.f[2] - (pn_new.b - pn_m.b));
                    if (SRC) {
                        const Pair<T> sz = ld2(P.src + 2 * N + gidx);
                        R0 += sz.a;
                        R1 += sz.b;
                    }
                    uz_n.a = (c.a & node_bit(2)) ? fma(B.dt, R0, u0.a) : u0.a;
                    uz_n.b = (c.b & node_bit(2)) ? fma(B.dt, R1, u0.b) : u0.b;
                }
            }
            *reinterpret_cast<Pair<T> *>(outx) = ux_n;
            *reinterpret_cast<Pair<T> *>(outx + N) = uy_n;
            *reinterpret_cast<Pair<T> *>(outx + 2 * N) = uz_n;
            *reinterpret_cast<Pair<T> *>(outp) = pn_m;
            outx += plane;
            outp += plane;
            if (REDUCE) {
                acc[0] += (double)ux_n.a + (double)ux_n.b;
                acc[1] += (double)uy_n.a + (double)uy_n.b;
                acc[2] += (double)uz_n.a + (double)uz_n.b;
            }
        }
        // publish p^n of plane t-1 (own pair and halo cells) for the next step's update
        *reinterpret_cast<Pair<T> *>(&S.pn[(t - 1) & 1][own - 2 * kBX]) = pn_new;
        if (hrow) {
            // the +y halo row as pairs (same arithmetic as press1, 2-wide loads)
            const Pair<T> hp = ld2(&G1.pin[hown - kPNo]);
            const Pair<T> hux = ld2(&G1.ux[hown]);
            const T huxl = G1.ux[hown - 1];
            const Pair<T> huy = ld2(&G1.uy[hown - kUYo]), huyd = ld2(&G1.uy[hown - kBX - kUYo]);
            const Pair<T> huz = ld2(&G1.uz[hown]), huzd = ld2(&G2.uz[hown]);
            const T dv0 = (hux.a - huxl) + (huy.a - huyd.a) + (huz.a - huzd.a);
            const T dv1 = (hux.b - hux.a) + (huy.b - huyd.b) + (huz.b - huzd.b);
            T rp0 = T(0), rp1 = T(0);
            if (SRC && hg >= 0) {
                const int gz = nb_coord(t - 1, nz, B.per[2]);
                if (gz >= 0) {
                    rp0 = P.src[3 * N + (long long)gz * plane + hg];
                    rp1 = P.src[3 * N + (long long)gz * plane + hg + 1];
                }
            }
            Pair<T> hn;
            hn.a = MODE == kModeU ? hp.a : hp.a - B.dtc2 * (dv0 - rp0);
            hn.b = MODE == kModeU ? hp.b : hp.b - B.dtc2 * (dv1 - rp1);
            if (PRES) {
                const int ra = reservoir(hown, t - 1), rb = reservoir(hown + 1, t - 1);
                if (ra >= 0 || rb >= 0) {
                    const Pair<uint32_t> cc = ld2u<T>(&G1.cd[hown - kPNo]);
                    if (ra >= 0) hn.a = res_p(ra, cc.a);
                    if (rb >= 0) hn.b = res_p(rb, cc.b);
                }
            }
            *reinterpret_cast<Pair<T> *>(&S.pn[(t - 1) & 1][hown - 2 * kBX]) = hn;
        } else if (hcol) {
            S.pn[(t - 1) & 1][hown - 2 * kBX] = press1(G1, G2, hown, t - 1, hg);
        }
        pn_m = pn_new;
        s2 = s1;
        s1 = s0;
        s0 = s0 == kStages - 1 ? 0 : s0 + 1;
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
            for (int q = 0; q < 4; ++q) red[ty][q] = acc[q];
        __syncthreads();
        if (tid < 4) {
            double sum = 0.0;
            for (int w = 0; w < kNT / 32; ++w) sum += red[w][tid];
            red_sum[rs][tid] += sum;
        }
    }
    __syncthreads();
    }  // persistent loop
    if (REDUCE) {
        if (B.multi) {
            if (tid < 4) B.prob[mp].partials[((long long)blockIdx.x - B.prob[mp].unit_begin) * 4 + tid] = red_sum[0][tid];
        } else if (tid < B.nprob * 4) {
            B.prob[tid / 4].partials[blockIdx.x * 4 + (tid % 4)] = red_sum[tid / 4][tid % 4];
        }
    }
}

// ------------------------------------------------------------------ launch
template <typename T, int MODE, bool RED, bool SRC, bool ALPHA, bool PRES = false>
inline cudaError_t launch_pair_t(const SweepBatch<T> &B, const uint32_t *code, int zchunk, cudaStream_t s) {
    TiledShape sh = B.multi ? TiledShape{} : tiled_shape<T>(B.nx, B.ny, B.nz, B.nprob, zchunk, 0, B.zsplit);
    if (B.multi) {
        const SweepProblem<T> &L = B.prob[B.nprob - 1];
        sh.grid = (int)(L.unit_begin + (long long)L.tiles_x * L.tiles_y * ((L.nz + L.zchunk - 1) / L.zchunk));
    }
    const size_t smem = sizeof(TiledSmem<T>);
    auto kern = sweep_tiled_kernel<T, MODE, RED, SRC, ALPHA, PRES>;
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
    kern<<<sh.grid, kNT, smem, s>>>(B, code, sh.tiles_x, sh.tiles_y, sh.per_cta, sh.zchunk);
    return cudaGetLastError();
}

template <typename T, int MODE>
inline cudaError_t launch_pair_m(const SweepBatch<T> &B, const uint32_t *code, bool red, bool src, int zc,
                                 cudaStream_t s) {
    const bool alpha = B.alpha != nullptr;
    if (B.pres_axis) {
        // fixed-pressure axis: single geometry, no source, no drag
        if (src || alpha || B.multi) return cudaErrorNotSupported;
        return red ? launch_pair_t<T, MODE, true, false, false, true>(B, code, zc, s)
                   : launch_pair_t<T, MODE, false, false, false, true>(B, code, zc, s);
    }
    if (red) {
        if (src) return alpha ? launch_pair_t<T, MODE, true, true, true>(B, code, zc, s)
                              : launch_pair_t<T, MODE, true, true, false>(B, code, zc, s);
        return alpha ? launch_pair_t<T, MODE, true, false, true>(B, code, zc, s)
                     : launch_pair_t<T, MODE, true, false, false>(B, code, zc, s);
    }
    if (src) return alpha ? launch_pair_t<T, MODE, false, true, true>(B, code, zc, s)
                          : launch_pair_t<T, MODE, false, true, false>(B, code, zc, s);
    return alpha ? launch_pair_t<T, MODE, false, false, true>(B, code, zc, s)
                 : launch_pair_t<T, MODE, false, false, false>(B, code, zc, s);
}

template <typename T>
inline cudaError_t launch_pair(const SweepBatch<T> &B, const uint32_t *code, int mode, bool red, bool src,
                               int zchunk, cudaStream_t s) {
    if (mode == kModeU) return launch_pair_m<T, kModeU>(B, code, red, src, zchunk, s);
    if (mode == kModePU) return launch_pair_m<T, kModePU>(B, code, red, src, zchunk, s);
    return launch_pair_m<T, kModeP>(B, code, red, src, zchunk, s);
}

}  // namespace pair
}  // namespace pmgb
