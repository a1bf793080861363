// Percolation check on the device (Sec. 5.1 assumes a percolating pore space; a drive
// along an axis without a fluid path around the periodic domain has no steady flow).
//
// 1. Components of the pore cells over face neighbours inside the box (no periodic
//    wrap): union-find on a label array whose links always point to a smaller cell
//    index, roots joined by atomicMin, then every label replaced by its root.
// 2. Pairs of pore cells across the periodic face of axis a (last layer -> first
//    layer): both cells in one component closes a loop that winds once around a, so
//    flow along a is possible.  Pairs that join two different components go into a small
//    hash set (component A, component B, axis) for the host, which finishes the search
//    on the graph of components with winding numbers (a few nodes and edges).
// 3. The number of pore cells (zero -> no fluid).
#pragma once

#include <cstdint>

namespace pmgb {

constexpr uint32_t kNoLabel = 0xffffffffu;
constexpr int kWrapSlots = 1 << 14;  // hash slots per axis for component pairs
constexpr unsigned long long kWrapEmpty = ~0ull;

// Root of x; parent links only ever decrease, so the walk ends.  L2 loads: other threads
// relink roots while the union kernel runs.
__device__ __forceinline__ uint32_t cc_find(const uint32_t *lab, uint32_t x) {
    uint32_t p = __ldcg(lab + x);
    while (p != x) {
        x = p;
        p = __ldcg(lab + x);
    }
    return x;
}

__global__ void cc_init_kernel(const uint8_t *__restrict__ mask, long long N, uint32_t *__restrict__ lab,
                               unsigned long long *__restrict__ n_pore) {
    unsigned long long cnt = 0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        const bool pore = mask[c] == 0;
        lab[c] = pore ? (uint32_t)c : kNoLabel;
        cnt += pore;
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(n_pore, cnt);
}

__global__ void count_pore_kernel(const uint8_t *__restrict__ mask, long long N, unsigned long long *n_pore) {
    unsigned long long cnt = 0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x)
        cnt += mask[c] == 0;
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(n_pore, cnt);
}

// Joins the components of pore cells a and b.  Each retry moves b to a strictly smaller
// index, so the loop ends; the bound only guards against a corrupted label array.
__device__ __forceinline__ void cc_unite(uint32_t *lab, uint32_t a, uint32_t b, int *err) {
    for (long long guard = 0; guard < (1ll << 32); ++guard) {
        a = cc_find(lab, a);
        b = cc_find(lab, b);
        if (a == b) return;
        if (a > b) {
            const uint32_t t = a;
            a = b;
            b = t;
        }
        const uint32_t old = atomicMin(lab + b, a);
        if (old == b) return;
        b = old;
    }
    *err = 1;
}

__global__ void cc_union_kernel(int nx, int ny, int nz, uint32_t *lab, int *err) {
    const long long plane = (long long)nx * ny, N = plane * nz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        if (__ldcg(lab + c) == kNoLabel) continue;
        const int x = (int)(c % nx);
        const long long r = c / nx;
        const int y = (int)(r % ny), z = (int)(r / ny);
        if (x + 1 < nx && __ldcg(lab + c + 1) != kNoLabel) cc_unite(lab, (uint32_t)c, (uint32_t)(c + 1), err);
        if (y + 1 < ny && __ldcg(lab + c + nx) != kNoLabel) cc_unite(lab, (uint32_t)c, (uint32_t)(c + nx), err);
        if (z + 1 < nz && __ldcg(lab + c + plane) != kNoLabel)
            cc_unite(lab, (uint32_t)c, (uint32_t)(c + plane), err);
    }
}

__global__ void cc_compress_kernel(long long N, uint32_t *lab) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        const uint32_t v = lab[c];
        if (v != kNoLabel && v != (uint32_t)c) lab[c] = cc_find(lab, v);
    }
}

// Pore pairs across the periodic faces.  wraps[a] = 1 when a pair joins a component to
// itself; other pairs (root A at the last layer, root B at the first) are inserted into
// the hash set table[a] (key A << 32 | B); a full table sets overflow.
__global__ void cc_wrap_kernel(int nx, int ny, int nz, int px, int py, int pz, const uint32_t *__restrict__ lab,
                               int *wraps, unsigned long long *table, int *overflow) {
    const long long plane = (long long)nx * ny;
    const long long fx = (long long)ny * nz, fy = (long long)nx * nz, fz = plane;
    const long long total = fx + fy + fz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        int a;
        long long hi, lo;  // cell on the last layer, its neighbour across the face
        if (i < fx) {
            a = 0;
            if (!px) continue;
            const long long row = i;  // (y, z)
            hi = row * nx + (nx - 1);
            lo = row * nx;
        } else if (i < fx + fy) {
            a = 1;
            if (!py) continue;
            const long long j = i - fx;
            const long long x = j % nx, z = j / nx;
            hi = x + nx * ((long long)(ny - 1) + (long long)ny * z);
            lo = x + plane * z;
        } else {
            a = 2;
            if (!pz) continue;
            const long long j = i - fx - fy;
            hi = j + plane * (nz - 1);
            lo = j;
        }
        const uint32_t A = lab[hi], B = lab[lo];
        if (A == kNoLabel || B == kNoLabel) continue;
        if (A == B) {
            wraps[a] = 1;
            continue;
        }
        const unsigned long long key = ((unsigned long long)A << 32) | B;
        unsigned long long *T = table + (size_t)a * kWrapSlots;
        uint32_t h = (A * 0x9E3779B1u) ^ (B * 0x85EBCA77u);
        h ^= h >> 15;
        bool placed = false;
        for (int probe = 0; probe < kWrapSlots; ++probe) {
            const uint32_t s = (h + (uint32_t)probe) & (kWrapSlots - 1);
            const unsigned long long cur = __ldcg(T + s);
            if (cur == key) {
                placed = true;
                break;
            }
            if (cur == kWrapEmpty) {
                const unsigned long long prev = atomicCAS(T + s, kWrapEmpty, key);
                if (prev == kWrapEmpty || prev == key) {
                    placed = true;
                    break;
                }
            }
        }
        if (!placed) *overflow = 1;
    }
}

}  // namespace pmgb
