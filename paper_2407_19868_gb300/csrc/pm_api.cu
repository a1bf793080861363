// Host driver and C ABI of the GB300 permeability solver (see include/poremaps_gb.h).
//
// Call flow of a solve (Algorithm 1 of the paper, one GPU, no halo exchange):
//   mask -> device -> neighbourhood flags (classify_kernel)
//   -> percolation check (device union-find over the pore cells plus a winding search on
//      the small graph of components, Sec. 5.1 assumes percolation)
//   -> first sweep (velocity of iteration 1)
//   -> windows of M fused sweeps, the last one with FP64 block sums, captured once as a
//      CUDA graph and replayed; after each window 4 doubles per drive come back to the
//      host for the convergence criterion (the only host<->device traffic in the loop)
//   -> last half sweep (pressure of the last iteration)
//   -> optional FP64 defect correction -> Darcy (Appendix C) -> symmetrise.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <array>
#include <mutex>
#include <unordered_map>
#include <utility>
#include <vector>

#include "../../include/poremaps_gb.h"
#include "pm_kernels.cuh"
#include "pm_percolation.cuh"
#include "pm_sweep_tiled.cuh"

using namespace pmgb;

namespace {

constexpr int kVersion = 200;  // 0.2.0

struct Status {
    int code = PM_OK;
};

int map_cuda(cudaError_t e) {
    if (e == cudaSuccess) return PM_OK;
    if (e == cudaErrorMemoryAllocation) return PM_ERR_OOM;
    return PM_ERR_CUDA;
}

#define PM_CK(call)                                      \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) {                         \
            (void)cudaGetLastError();                    \
            return map_cuda(e_);                         \
        }                                                \
    } while (0)

// Stream-ordered memory pool of the library, one per device, created on first use.  Its
// release threshold is unlimited, so scratch freed at the end of a call stays reserved
// for the next call of the same or a smaller size instead of going back to the driver
// (pm_release_memory returns it).
constexpr int kMaxDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pools[kMaxDevices] = {};

int library_pool(cudaMemPool_t *out) {
    int dev = 0;
    PM_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return PM_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_pools[dev]) {
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        PM_CK(cudaMemPoolCreate(&pool, &props));
        uint64_t keep = ~0ull;
        cudaError_t e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            cudaMemPoolDestroy(pool);
            return map_cuda(e);
        }
        g_pools[dev] = pool;
    }
    *out = g_pools[dev];
    return PM_OK;
}

// Stream-ordered scratch from the library pool, freed (back into the pool) when the
// owner goes out of scope; pinned host buffers (fields placed in host memory) are freed
// after the stream has finished with them.
struct Scratch {
    cudaStream_t s = nullptr;
    std::vector<void *> ptrs, host;
    explicit Scratch(cudaStream_t st) : s(st) {}
    ~Scratch() {
        for (void *p : ptrs) cudaFreeAsync(p, s);
        if (!host.empty()) {
            cudaStreamSynchronize(s);
            for (void *p : host) cudaFreeHost(p);
        }
    }
    // zero-filled buffer in pinned host memory that kernels read and write directly
    // (over NVLink-C2C on a Grace CPU, PCIe elsewhere)
    template <typename T>
    int alloc_host(T **p, size_t count) {
        *p = nullptr;
        void *v = nullptr;
        cudaError_t e = cudaHostAlloc(&v, count * sizeof(T) + 16, cudaHostAllocPortable | cudaHostAllocMapped);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return PM_ERR_OOM;
        }
        std::memset(v, 0, count * sizeof(T) + 16);
        host.push_back(v);
        void *d = nullptr;
        e = cudaHostGetDevicePointer(&d, v, 0);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return map_cuda(e);
        }
        *p = static_cast<T *>(d);
        return PM_OK;
    }
    template <typename T>
    int alloc(T **p, size_t count) {
        *p = nullptr;
        cudaMemPool_t pool = nullptr;
        int st = library_pool(&pool);
        if (st) return st;
        void *v = nullptr;
        cudaError_t e = cudaMallocFromPoolAsync(&v, count * sizeof(T) + 16, pool, s);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return map_cuda(e);
        }
        ptrs.push_back(v);
        *p = static_cast<T *>(v);
        return PM_OK;
    }
};

// Small pinned host blocks for the per-window reduction results, kept for reuse (a
// cudaMallocHost per solve would cost more than the solve of a small domain).
constexpr size_t kPinnedBlock = 4096;
std::mutex g_pinned_mu;
std::vector<void *> g_pinned_free;

void *pinned_get() {
    {
        std::lock_guard<std::mutex> lock(g_pinned_mu);
        if (!g_pinned_free.empty()) {
            void *p = g_pinned_free.back();
            g_pinned_free.pop_back();
            return p;
        }
    }
    void *p = nullptr;
    if (cudaMallocHost(&p, kPinnedBlock) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return p;
}
void pinned_put(void *p) {
    if (!p) return;
    std::lock_guard<std::mutex> lock(g_pinned_mu);
    g_pinned_free.push_back(p);
}

// Internal stream ordered after the caller's stream; at destruction the caller's stream
// is ordered after all internal work.
struct StreamScope {
    cudaStream_t user = nullptr, s = nullptr;
    cudaEvent_t ev = nullptr;
    int status = PM_OK;
    explicit StreamScope(void *user_stream) : user(static_cast<cudaStream_t>(user_stream)) {
        cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(ev, user);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev, 0);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            status = map_cuda(e);
        }
    }
    ~StreamScope() {
        if (s) {
            if (ev) {
                cudaEventRecord(ev, s);
                cudaStreamWaitEvent(user, ev, 0);
            }
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
        if (ev) cudaEventDestroy(ev);
    }
};

// Kernel launches issued by this host thread (a graph replay counts its kernels), read
// by the entry points for pm_stats.kernel_launches.
thread_local long long t_launches = 0;
inline void note_launch(long long n = 1) { t_launches += n; }

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// Grid of a 256-thread grid-stride kernel over n items: enough blocks for every item, at
// most 32 per SM.
int launch_grid(long long n) {
    const long long b = (n + 255) / 256, cap = 32ll * tiled_grid_size();
    return (int)(b < cap ? (b < 1 ? 1 : b) : cap);
}

// ------------------------------------------------------------------ geometry
struct Geometry {
    int nx = 0, ny = 0, nz = 0;
    int per[3] = {1, 1, 1};
    int pax = -1;               // fixed-pressure axis, -1 if none
    long long N = 0;
    const uint8_t *mask = nullptr;  // device copy of the mask (or the caller's device mask)
    uint8_t *flags = nullptr;   // device, one byte per cell (simple kernel)
    uint32_t *code = nullptr;   // device, one stencil code word per cell (tiled kernel)
    uint32_t *tcode = nullptr;  // device, two transposed code words per cell (adjoint, on demand)
};

// Transposed stencil codes of a geometry (the tiled transposed sweep of adjoint solves).
int build_tcode(Geometry &g, cudaStream_t s, Scratch &scr) {
    int st = scr.alloc(&g.tcode, (size_t)(2 * g.N));
    if (st) return st;
    tcode_kernel<<<launch_grid(g.N), 256, 0, s>>>(g.code, g.nx, g.ny, g.nz, g.per[0], g.per[1], g.per[2], g.tcode);
    note_launch();
    PM_CK(cudaGetLastError());
    return PM_OK;
}

// Fixed-pressure axis of a domain, -1 if none.
int pressure_axis(const pm_domain *dom) {
    for (int a = 0; a < 3; ++a)
        if (dom->bc[a] == PM_BC_PRESSURE) return a;
    return -1;
}

int validate_domain(const pm_domain *dom) {
    if (!dom || !dom->mask) return PM_ERR_INVALID_ARG;
    if (dom->nx < 1 || dom->ny < 1 || dom->nz < 1) return PM_ERR_INVALID_ARG;
    int npres = 0;
    for (int a = 0; a < 3; ++a) {
        if (dom->bc[a] != PM_BC_PERIODIC && dom->bc[a] != PM_BC_WALL && dom->bc[a] != PM_BC_PRESSURE)
            return PM_ERR_INVALID_ARG;
        if (dom->bc[a] == PM_BC_PRESSURE) {
            const int n = a == 0 ? dom->nx : (a == 1 ? dom->ny : dom->nz);
            if (++npres > 1 || n < 3) return PM_ERR_INVALID_ARG;  // one axis, two reservoirs + 1 layer
        }
    }
    if (!(dom->voxel_size > 0) || !(dom->viscosity > 0)) return PM_ERR_INVALID_ARG;
    return PM_OK;
}

int validate_options(const pm_options *o) {
    if (!o) return PM_ERR_INVALID_ARG;
    if (!(o->tol > 0) || o->check_every < 1 || o->max_iter < 1) return PM_ERR_INVALID_ARG;
    if (o->precision < PM_FP32_RED64 || o->precision > PM_FP64) return PM_ERR_INVALID_ARG;
    if (!(o->dt_safety > 0) || !(o->Re > 0) || !(o->c2 > 0)) return PM_ERR_INVALID_ARG;
    if (o->schedule < -1 || o->schedule_split < 0 || o->schedule_split > 64) return PM_ERR_INVALID_ARG;
    if (o->tile < 0 || o->tile > kNumTiles) return PM_ERR_INVALID_ARG;
    if (o->field_memory < 0 || o->field_memory > 2 || o->sequence < 0 || o->sequence > 1) return PM_ERR_INVALID_ARG;
    if (o->dc_extrapolate < 0 || o->dc_extrapolate > 1) return PM_ERR_INVALID_ARG;
    return PM_OK;
}

// Host copy of the mask (needed by the percolation search).
int host_mask(const pm_domain *dom, std::vector<uint8_t> &out) {
    size_t N = (size_t)dom->nx * dom->ny * dom->nz;
    out.resize(N);
    if (dom->mask_on_device) {
        PM_CK(cudaMemcpy(out.data(), dom->mask, N, cudaMemcpyDeviceToHost));
    } else {
        std::memcpy(out.data(), dom->mask, N);
    }
    return PM_OK;
}

int build_geometry(const pm_domain *dom, cudaStream_t s, Scratch &scr, Geometry &g) {
    g.nx = dom->nx;
    g.ny = dom->ny;
    g.nz = dom->nz;
    for (int a = 0; a < 3; ++a) g.per[a] = dom->bc[a] == PM_BC_PERIODIC;
    g.pax = pressure_axis(dom);
    g.N = (long long)g.nx * g.ny * g.nz;
    int st = scr.alloc(&g.flags, (size_t)g.N);
    if (st) return st;
    const uint8_t *dmask = dom->mask;
    if (!dom->mask_on_device) {
        uint8_t *m = nullptr;
        if ((st = scr.alloc(&m, (size_t)g.N))) return st;
        PM_CK(cudaMemcpyAsync(m, dom->mask, (size_t)g.N, cudaMemcpyHostToDevice, s));
        dmask = m;
    }
    g.mask = dmask;
    classify_kernel<<<launch_grid(g.N), 256, 0, s>>>(dmask, g.nx, g.ny, g.nz, g.per[0], g.per[1], g.per[2],
                                                     g.pax, g.flags);
    note_launch(1);
    PM_CK(cudaGetLastError());
    if ((st = scr.alloc(&g.code, (size_t)g.N))) return st;
    code_kernel<<<launch_grid(g.N), 256, 0, s>>>(dmask, g.nx, g.ny, g.nz, g.per[0], g.per[1], g.per[2], g.pax,
                                                 g.code);
    note_launch(1);
    PM_CK(cudaGetLastError());
    return PM_OK;
}

// Does a face-connected path of pore cells wrap the periodic domain along each axis?
// Breadth-first search that carries, per visited cell, how often the path to it crossed
// each periodic boundary; meeting a visited cell with another crossing count along
// axis a closes a loop that wraps around a.
// Fixed-pressure axis a: is there a path of pore cells from the inlet reservoir layer to
// the outlet one?  Reservoir cells carry no flow across the axis, so a path leaves a
// reservoir only along a.
int percolation_pressure(const std::vector<uint8_t> &mask, int nx, int ny, int nz, const int per[3], int a) {
    const long long N = (long long)nx * ny * nz;
    const int n[3] = {nx, ny, nz};
    std::vector<uint8_t> seen((size_t)N, 0);
    std::vector<long long> queue;
    auto coord = [&](long long c, int ax) {
        return ax == 0 ? (int)(c % nx) : (ax == 1 ? (int)((c / nx) % ny) : (int)(c / ((long long)nx * ny)));
    };
    for (long long c = 0; c < N; ++c)
        if (!mask[c] && coord(c, a) == 0) {
            seen[c] = 1;
            queue.push_back(c);
        }
    for (size_t h = 0; h < queue.size(); ++h) {
        const long long c = queue[h];
        const int co[3] = {coord(c, 0), coord(c, 1), coord(c, 2)};
        if (co[a] == n[a] - 1) return 1;
        for (int ax = 0; ax < 3; ++ax) {
            if (co[a] == 0 && ax != a) continue;
            for (int m = -1; m <= 1; m += 2) {
                int cc[3] = {co[0], co[1], co[2]};
                cc[ax] += m;
                if (cc[ax] < 0 || cc[ax] >= n[ax]) {
                    if (!per[ax]) continue;
                    cc[ax] = (cc[ax] + n[ax]) % n[ax];
                }
                const long long b = cc[0] + (long long)nx * (cc[1] + (long long)ny * cc[2]);
                if (mask[b] || seen[b]) continue;
                seen[b] = 1;
                queue.push_back(b);
            }
        }
    }
    return 0;
}

void percolation_host(const std::vector<uint8_t> &mask, int nx, int ny, int nz, const int per[3],
                      int out[3]) {
    const long long N = (long long)nx * ny * nz;
    out[0] = out[1] = out[2] = 0;
    std::vector<uint8_t> seen((size_t)N, 0);
    std::vector<int16_t> wind((size_t)N * 3);
    std::vector<long long> queue;
    queue.reserve(1 << 16);
    const int n[3] = {nx, ny, nz};
    for (long long s0 = 0; s0 < N; ++s0) {
        if (mask[s0] || seen[s0]) continue;
        queue.clear();
        queue.push_back(s0);
        seen[s0] = 1;
        wind[s0 * 3] = wind[s0 * 3 + 1] = wind[s0 * 3 + 2] = 0;
        for (size_t h = 0; h < queue.size(); ++h) {
            long long c = queue[h];
            int co[3] = {(int)(c % nx), (int)((c / nx) % ny), (int)(c / ((long long)nx * ny))};
            for (int a = 0; a < 3; ++a)
                for (int m = -1; m <= 1; m += 2) {
                    int cc[3] = {co[0], co[1], co[2]};
                    int w = 0;
                    cc[a] += m;
                    if (cc[a] < 0 || cc[a] >= n[a]) {
                        if (!per[a]) continue;
                        w = cc[a] < 0 ? -1 : 1;
                        cc[a] = (cc[a] + n[a]) % n[a];
                    }
                    long long b = cc[0] + (long long)nx * (cc[1] + (long long)ny * cc[2]);
                    if (mask[b]) continue;
                    int16_t wn[3] = {wind[c * 3], wind[c * 3 + 1], wind[c * 3 + 2]};
                    wn[a] = (int16_t)(wn[a] + w);
                    if (!seen[b]) {
                        seen[b] = 1;
                        for (int k = 0; k < 3; ++k) wind[b * 3 + k] = wn[k];
                        queue.push_back(b);
                    } else {
                        for (int k = 0; k < 3; ++k)
                            if (wind[b * 3 + k] != wn[k]) out[k] = 1;
                    }
                }
        }
    }
}

// Pore count and percolation of a device mask (pm_percolation.cuh): union-find of the
// pore cells inside the box on the device, then a search with winding numbers on the
// graph whose nodes are those components and whose edges are the pore pairs across the
// periodic faces.  A loop in that graph with a nonzero winding along axis a is a fluid
// path around the domain along a (the same criterion as percolation_host).  out[a] is
// set for periodic axes only; check = false counts the pore cells only.
int percolation_device(const Geometry &g, bool check, cudaStream_t s, Scratch &scr, long long *n_pore,
                       int out[3]) {
    const long long N = g.N;
    out[0] = out[1] = out[2] = 0;
    struct Info {
        unsigned long long n_pore;
        int wraps[3];
        int overflow;
        int err;
        int pad;
    };
    if (N >= (long long)kNoLabel) {
        // beyond 32-bit labels: host search on a copy of the mask
        std::vector<uint8_t> hm((size_t)N);
        PM_CK(cudaMemcpyAsync(hm.data(), g.mask, (size_t)N, cudaMemcpyDeviceToHost, s));
        PM_CK(cudaStreamSynchronize(s));
        long long c = 0;
        for (uint8_t v : hm) c += v == 0;
        *n_pore = c;
        if (check && c > 0) percolation_host(hm, g.nx, g.ny, g.nz, g.per, out);
        return PM_OK;
    }
    uint32_t *lab = nullptr;
    Info *info = nullptr;
    unsigned long long *table = nullptr;
    int st;
    if ((st = scr.alloc(&info, 1))) return st;
    PM_CK(cudaMemsetAsync(info, 0, sizeof(Info), s));
    if (check) {
        if ((st = scr.alloc(&lab, (size_t)N)) || (st = scr.alloc(&table, (size_t)3 * kWrapSlots))) return st;
        PM_CK(cudaMemsetAsync(table, 0xff, sizeof(unsigned long long) * 3 * kWrapSlots, s));
        cc_init_kernel<<<launch_grid(N), 256, 0, s>>>(g.mask, N, lab, &info->n_pore);
        cc_union_kernel<<<launch_grid(N), 256, 0, s>>>(g.nx, g.ny, g.nz, lab, &info->err);
        cc_compress_kernel<<<launch_grid(N), 256, 0, s>>>(N, lab);
        const long long faces = (long long)g.ny * g.nz + (long long)g.nx * g.nz + (long long)g.nx * g.ny;
        cc_wrap_kernel<<<launch_grid(faces), 256, 0, s>>>(g.nx, g.ny, g.nz, g.per[0], g.per[1], g.per[2], lab,
                                                         info->wraps, table, &info->overflow);
        note_launch(4);
    } else {
        count_pore_kernel<<<launch_grid(N), 256, 0, s>>>(g.mask, N, &info->n_pore);
        note_launch();
    }
    PM_CK(cudaGetLastError());
    Info h;
    PM_CK(cudaMemcpyAsync(&h, info, sizeof(Info), cudaMemcpyDeviceToHost, s));
    PM_CK(cudaStreamSynchronize(s));
    *n_pore = (long long)h.n_pore;
    if (!check || h.n_pore == 0) return PM_OK;
    if (h.err) return PM_ERR_CUDA;
    if (h.overflow) {
        // more distinct component pairs than the hash set holds: host search
        std::vector<uint8_t> hm((size_t)N);
        PM_CK(cudaMemcpyAsync(hm.data(), g.mask, (size_t)N, cudaMemcpyDeviceToHost, s));
        PM_CK(cudaStreamSynchronize(s));
        percolation_host(hm, g.nx, g.ny, g.nz, g.per, out);
        return PM_OK;
    }
    for (int a = 0; a < 3; ++a) out[a] = h.wraps[a] != 0;
    std::vector<unsigned long long> ht((size_t)3 * kWrapSlots);
    PM_CK(cudaMemcpyAsync(ht.data(), table, sizeof(unsigned long long) * ht.size(), cudaMemcpyDeviceToHost, s));
    PM_CK(cudaStreamSynchronize(s));
    // graph of components: edge A -> B crosses the periodic face of axis a in the + sense
    std::unordered_map<uint32_t, int> id;
    struct Edge {
        int to, axis, sign;
    };
    std::vector<std::vector<Edge>> adj;
    auto node = [&](uint32_t lbl) {
        auto it = id.find(lbl);
        if (it != id.end()) return it->second;
        const int k = (int)adj.size();
        id.emplace(lbl, k);
        adj.emplace_back();
        return k;
    };
    for (int a = 0; a < 3; ++a)
        for (int i = 0; i < kWrapSlots; ++i) {
            const unsigned long long key = ht[(size_t)a * kWrapSlots + i];
            if (key == kWrapEmpty) continue;
            const int A = node((uint32_t)(key >> 32)), B = node((uint32_t)(key & 0xffffffffu));
            adj[(size_t)A].push_back({B, a, +1});
            adj[(size_t)B].push_back({A, a, -1});
        }
    const size_t n = adj.size();
    std::vector<std::array<long long, 3>> wind(n);
    std::vector<uint8_t> seen(n, 0);
    std::vector<int> queue;
    for (size_t s0 = 0; s0 < n; ++s0) {
        if (seen[s0]) continue;
        seen[s0] = 1;
        wind[s0] = {0, 0, 0};
        queue.assign(1, (int)s0);
        for (size_t h2 = 0; h2 < queue.size(); ++h2) {
            const int c = queue[h2];
            for (const Edge &e : adj[(size_t)c]) {
                std::array<long long, 3> w = wind[(size_t)c];
                w[e.axis] += e.sign;
                if (!seen[(size_t)e.to]) {
                    seen[(size_t)e.to] = 1;
                    wind[(size_t)e.to] = w;
                    queue.push_back(e.to);
                } else {
                    for (int k = 0; k < 3; ++k)
                        if (wind[(size_t)e.to][k] != w[k]) out[k] = 1;
                }
            }
        }
    }
    return PM_OK;
}

double time_step(const pm_options *o) {
    // 12 c2 dt^2 + (40 / Re) dt - 4 = 0: acoustic bound of the velocity-then-pressure
    // update (cell Laplacian eigenvalues <= 12) plus the viscous Gershgorin bound
    // (<= 20 / Re) of the explicit velocity update
    const double a = 12.0 * o->c2, b = 40.0 / o->Re, c = -4.0;
    return o->dt_safety * (-b + std::sqrt(b * b - 4.0 * a * c)) / (2.0 * a);
}

// ------------------------------------------------------------------ solver state
template <typename T>
struct Fields {
    T *u[2] = {nullptr, nullptr};
    T *p[2] = {nullptr, nullptr};
    int cur = 0;  // buffer holding the latest state
};

template <typename T>
struct Solver {
    const Geometry &g;
    const pm_options &o;
    cudaStream_t s;
    Scratch &scr;
    int nprob = 0;
    Fields<T> F[kMaxBatch];
    int dir[kMaxBatch] = {0, 0, 0, 0};
    double force[kMaxBatch] = {0, 0, 0, 0};
    const T *src[kMaxBatch] = {nullptr, nullptr, nullptr, nullptr};
    double *partials = nullptr;  // [nprob][nblk][4] (multi: [total_units][4])
    long long unit_begin_h[kMaxBatch] = {};
    double *dq = nullptr;        // [nprob][4]
    double *hq = nullptr;        // pinned [nprob][4]
    long long nblk = 0;
    T dt = 0, dtc2 = 0, inv_re = 0;
    const T *alpha = nullptr;
    bool transposed = false;  // adjoint solves: transpose of the viscous operator
    int zchunk = 0;           // tiled-kernel schedule (0 = persistent), from the options or tune()
    int zsplit = 1;           // chunked schedules: sub-chunks of each column's last chunk (tune())
    int tile = 0;             // tiled-kernel tile shape (index), from the options or tune()
    // multi-geometry batch: problem k lives on geometry *geo[k]
    bool multi = false;
    const Geometry *geo[kMaxBatch] = {};
    ReduceRange *ranges = nullptr;  // device, per problem
    int *active = nullptr;          // device, per problem
    int active_h[kMaxBatch] = {};
    long long total_units = 0;
    double t_setup = 0.0;  // host seconds from the entry point to the first sweep
    bool capturing = false;  // launches go into a graph (counted when it is replayed)
    bool tuned = false;      // tile shape and split chosen (tune() ran once)
    const Geometry &G(int k) const { return multi ? *geo[k] : g; }

    Solver(const Geometry &gg, const pm_options &oo, cudaStream_t ss, Scratch &sc)
        : g(gg), o(oo), s(ss), scr(sc) {}
    ~Solver() {
        pinned_put(hq);
    }

    dim3 block() const { return dim3(32, 8, 1); }
    dim3 grid() const { return dim3((g.nx + 31) / 32, (g.ny + 7) / 8, (unsigned)(g.nz * nprob)); }

    int init(int np) {
        nprob = np;
        const double dts = time_step(&o);
        dt = (T)dts;
        dtc2 = (T)(dts * o.c2);
        inv_re = (T)(1.0 / o.Re);
        dim3 gr = grid();
        nblk = (long long)gr.x * gr.y * g.nz;
        zchunk = o.schedule > 0 ? o.schedule : 0;
        zsplit = zchunk > 0 && o.schedule_split > 1 ? o.schedule_split : 1;
        tile = o.tile > 0 && o.tile <= tile_count<T>() ? o.tile - 1 : 0;
        long long nblk_t = tiled_max_blocks<T>(g.nx, g.ny, g.nz, np);
        if (zchunk > 0)
            for (int t = 0; t < tile_count<T>(); ++t) {
                const long long b = tiled_num_blocks<T>(g.nx, g.ny, g.nz, np, zchunk, t, zsplit);
                nblk_t = b > nblk_t ? b : nblk_t;
            }
        if (transposed) {
            tile = kTileTR;
            int cand[8];
            const int n = tiled_candidates(g.nx, g.ny, g.nz, np, cand, kTileTR);
            for (int i = 0; i < n; ++i)
                for (int sp : kSplits)
                    nblk_t = std::max(nblk_t, tiled_num_blocks<T>(g.nx, g.ny, g.nz, np, cand[i], kTileTR, sp));
            if (zchunk > 0)
                nblk_t = std::max(nblk_t, tiled_num_blocks<T>(g.nx, g.ny, g.nz, np, zchunk, kTileTR, zsplit));
        }
        const long long nblk_max = nblk > nblk_t ? nblk : nblk_t;
        int st;
        for (int k = 0; k < nprob; ++k) {
            const long long Nk = G(k).N;
            for (int b = 0; b < 2; ++b) {
                // field placement: device memory, or pinned host memory for buffer 1
                // (field_memory 1) or both buffers (2) -- domains beyond device memory
                if (o.field_memory > b) {
                    if ((st = scr.alloc_host(&F[k].u[b], (size_t)(3 * Nk)))) return st;
                    if ((st = scr.alloc_host(&F[k].p[b], (size_t)Nk))) return st;
                    continue;
                }
                if ((st = scr.alloc(&F[k].u[b], (size_t)(3 * Nk)))) return st;
                if ((st = scr.alloc(&F[k].p[b], (size_t)Nk))) return st;
                PM_CK(cudaMemsetAsync(F[k].u[b], 0, sizeof(T) * 3 * Nk, s));
                PM_CK(cudaMemsetAsync(F[k].p[b], 0, sizeof(T) * Nk, s));
            }
            F[k].cur = 0;
        }
        if (multi) {
            // partials for the largest unit count over the tile shapes
            long long most = 0;
            for (int t = 0; t < tile_count<T>(); ++t) most = std::max(most, multi_units(t, nullptr));
            if ((st = scr.alloc(&partials, (size_t)(most * 4)))) return st;
            if ((st = scr.alloc(&ranges, (size_t)nprob)) || (st = scr.alloc(&active, (size_t)nprob))) return st;
            if ((st = set_multi_tile(tile))) return st;
            for (int k = 0; k < nprob; ++k) active_h[k] = 1;
            PM_CK(cudaMemcpyAsync(active, active_h, sizeof(int) * nprob, cudaMemcpyHostToDevice, s));
            PM_CK(cudaStreamSynchronize(s));
        } else if ((st = scr.alloc(&partials, (size_t)(nprob * nblk_max * 4)))) {
            return st;
        }
        if ((st = scr.alloc(&dq, (size_t)(nprob * 4)))) return st;
        static_assert(sizeof(double) * kMaxBatch * 4 <= kPinnedBlock, "pinned block size");
        hq = static_cast<double *>(pinned_get());
        if (!hq) return PM_ERR_OOM;
        return PM_OK;
    }

    // Multi-geometry launch with tile shape t: one CTA per (column, chunk of at most 64
    // planes) of every problem.  Returns the number of CTAs; fills rh (per-problem ranges
    // of the reduction partials) when given.
    long long multi_units(int t, ReduceRange *rh) {
        const TileDims td = tile_dims(t);
        long long u = 0;
        for (int k = 0; k < nprob; ++k) {
            const Geometry &q = G(k);
            const long long tiles = (long long)((q.nx + td.tx - 1) / td.tx) * ((q.ny + td.ty - 1) / td.ty);
            const int zc = q.nz < 64 ? q.nz : 64;
            const long long cnt = tiles * ((q.nz + zc - 1) / zc);
            if (rh) {
                unit_begin_h[k] = u;
                rh[k] = {u, cnt, (double)q.N};
            }
            u += cnt;
        }
        return u;
    }
    // Switches a multi-geometry solver to tile shape t (unit table and reduction ranges).
    int set_multi_tile(int t) {
        ReduceRange rh[kMaxBatch];
        tile = t;
        total_units = multi_units(t, rh);
        PM_CK(cudaMemcpyAsync(ranges, rh, sizeof(ReduceRange) * nprob, cudaMemcpyHostToDevice, s));
        PM_CK(cudaStreamSynchronize(s));
        return PM_OK;
    }

    // Copy a caller state (same type, iteration units) into the current buffers.
    int load_state(int k, const T *u, const T *p) {
        if (u) PM_CK(cudaMemcpyAsync(F[k].u[F[k].cur], u, sizeof(T) * 3 * G(k).N, cudaMemcpyDefault, s));
        if (p) PM_CK(cudaMemcpyAsync(F[k].p[F[k].cur], p, sizeof(T) * G(k).N, cudaMemcpyDefault, s));
        sanitize_kernel<T><<<launch_grid(G(k).N), 256, 0, s>>>(G(k).flags, G(k).N, F[k].u[F[k].cur], F[k].p[F[k].cur]);
        note_launch();
        PM_CK(cudaGetLastError());
        return PM_OK;
    }

    SweepBatch<T> batch(bool reduce) {
        SweepBatch<T> B{};
        B.nx = g.nx;
        B.ny = g.ny;
        B.nz = g.nz;
        for (int a = 0; a < 3; ++a) B.per[a] = g.per[a];
        B.N = g.N;
        B.flags = g.flags;
        B.code = g.code;
        B.tcode = g.tcode;
        B.alpha = alpha;
        B.inv_re = inv_re;
        B.dt = dt;
        B.dtc2 = dtc2;
        B.nprob = nprob;
        for (int k = 0; k < nprob; ++k) {
            SweepProblem<T> &P = B.prob[k];
            P.uin = F[k].u[F[k].cur];
            P.pin = F[k].p[F[k].cur];
            P.uout = F[k].u[1 - F[k].cur];
            P.pout = F[k].p[1 - F[k].cur];
            P.src = src[k];
            for (int d = 0; d < 3; ++d) P.f[d] = (T)(d == dir[k] && g.pax < 0 ? force[k] : 0.0);
            if (g.pax >= 0) {
                // fixed-pressure drive: p_in - p_out = force x (n - 1), centred on 0
                const int n = g.pax == 0 ? g.nx : (g.pax == 1 ? g.ny : g.nz);
                P.pres[0] = (T)(0.5 * force[k] * (n - 1));
                P.pres[1] = (T)(-0.5 * force[k] * (n - 1));
            }
            const Geometry &q = G(k);
            P.code = q.code;
            P.nx = q.nx;
            P.ny = q.ny;
            P.nz = q.nz;
            const TileDims td = tile_dims(tile);
            P.zchunk = q.nz < 64 ? q.nz : 64;
            P.tiles_x = (q.nx + td.tx - 1) / td.tx;
            P.tiles_y = (q.ny + td.ty - 1) / td.ty;
            P.unit_begin = unit_begin_h[k];
            if (multi)
                P.partials = reduce ? partials + (size_t)unit_begin_h[k] * 4 : nullptr;
            else
                P.partials = reduce ? partials + (size_t)k * reduce_blocks() * 4 : nullptr;
        }
        B.multi = multi ? 1 : 0;
        B.active = multi ? active : nullptr;
        B.pres_axis = g.pax + 1;
        B.zsplit = multi ? 1 : zsplit;
        return B;
    }

    template <int MODE, bool RED>
    void launch_simple(const SweepBatch<T> &B, bool has_src) {
        if (transposed)
            sweep_simple_kernel<T, MODE, RED, false, true><<<grid(), block(), 0, s>>>(B);
        else if (has_src)
            sweep_simple_kernel<T, MODE, RED, true><<<grid(), block(), 0, s>>>(B);
        else
            sweep_simple_kernel<T, MODE, RED, false><<<grid(), block(), 0, s>>>(B);
    }

    bool use_tiled() const {
        if (multi) return true;  // batches are built only from tiled-kernel shapes
        if (transposed && (sizeof(T) != 4 || !g.tcode)) return false;  // FP64 adjoint: simple kernel
        // a fixed-pressure axis runs on tile shape 1 only (the pair kernel's reservoir variant)
        return o.kernel == 0 && (g.pax < 0 || tile == 0) && tiled_supported<T>(g.nx, g.ny, g.nz, nprob);
    }

    // One sweep of the given mode; flips the ping-pong buffers.
    int sweep(int mode, bool reduce) {
        SweepBatch<T> B = batch(reduce);
        bool has_src = false;
        for (int k = 0; k < nprob; ++k) has_src |= src[k] != nullptr;
        if (use_tiled()) {
            int st;
            if constexpr (sizeof(T) == 4) {
                st = transposed ? launch_tiled_transposed(B, g.code, mode, reduce, zchunk, s)
                                : launch_tiled(B, g.code, mode, reduce, has_src, zchunk, s, tile);
            } else {
                st = launch_tiled(B, g.code, mode, reduce, has_src, zchunk, s, tile);
            }
            if (st) return st;
        } else if (mode == kModeU) {
            reduce ? launch_simple<kModeU, true>(B, has_src) : launch_simple<kModeU, false>(B, has_src);
        } else if (mode == kModePU) {
            reduce ? launch_simple<kModePU, true>(B, has_src) : launch_simple<kModePU, false>(B, has_src);
        } else {
            reduce ? launch_simple<kModeP, true>(B, has_src) : launch_simple<kModeP, false>(B, has_src);
        }
        PM_CK(cudaGetLastError());
        if (!capturing) note_launch();
        for (int k = 0; k < nprob; ++k) F[k].cur ^= 1;
        return PM_OK;
    }

    long long reduce_blocks() const {
        return use_tiled() ? tiled_num_blocks<T>(g.nx, g.ny, g.nz, nprob, zchunk, tile, zsplit) : nblk;
    }

    int reduce_to_host_async() {
        if (multi)
            reduce_ranges_kernel<<<nprob, 256, 0, s>>>(partials, ranges, dq);
        else
            reduce_partials_kernel<<<nprob, 256, 0, s>>>(partials, reduce_blocks(), g.N, dq);
        PM_CK(cudaGetLastError());
        if (!capturing) note_launch();
        PM_CK(cudaMemcpyAsync(hq, dq, sizeof(double) * nprob * 4, cudaMemcpyDeviceToHost, s));
        return PM_OK;
    }

    // Autotuner of the tiled kernel: times `reps` pairs of sweeps (after one untimed pair)
    // for every tile shape x work split (persistent, or plane chunks) that the options do
    // not pin, with CUDA events, and keeps the fastest.  Multi-geometry batches tune the
    // tile shape only (their split is one CTA per column chunk).  The result is cached per
    // (device, precision, shapes of the problems).  The timed sweeps are ordinary
    // iterations of the solve (pairs, so the ping-pong parity is unchanged); returns
    // their number.
    int tune(int reps = 2) {
        if (!use_tiled()) return 0;
        struct Entry {
            int dev, size;
            std::vector<long long> key;
            int tile, zchunk, zsplit;
        };
        static std::mutex mu;
        static std::vector<Entry> cache;
        const int dev = current_device();
        bool has_src = false;
        for (int k = 0; k < nprob; ++k) has_src |= src[k] != nullptr;
        std::vector<long long> key{multi ? 1 : 0, nprob,      o.tile, o.schedule, o.schedule_split,
                                   transposed ? 1 : 0, has_src ? 1 : 0};
        for (int k = 0; k < (multi ? nprob : 1); ++k) {
            key.push_back(G(k).nx);
            key.push_back(G(k).ny);
            key.push_back(G(k).nz);
        }
        {
            std::lock_guard<std::mutex> lock(mu);
            for (const Entry &e : cache)
                if (e.dev == dev && e.size == (int)sizeof(T) && e.key == key) {
                    if (multi && e.tile != tile && set_multi_tile(e.tile)) return 0;
                    tile = e.tile;
                    zchunk = e.zchunk;
                    zsplit = e.zsplit;
                    return 0;
                }
        }
        struct Cand {
            int tile, zchunk, zsplit;
        };
        std::vector<Cand> cand;
        for (int t = 0; t < (transposed ? kTileTR + 1 : tile_count<T>()); ++t) {
            if (transposed ? t != kTileTR : (o.tile > 0 && o.tile <= tile_count<T>() && t != o.tile - 1)) continue;
            if (g.pax >= 0 && t != 0) continue;
            if (multi || o.schedule != 0) {
                cand.push_back({t, multi ? 0 : zchunk, multi ? 1 : zsplit});
                continue;
            }
            int zc[8];
            const int n = tiled_candidates(g.nx, g.ny, g.nz, nprob, zc, t);
            for (int i = 0; i < n; ++i) {
                cand.push_back({t, zc[i], 1});
                if (zc[i] == 0) continue;  // persistent CTAs: no chunks
                int prev = 1;
                for (int sp : kSplits) {
                    const int eff = split_last(g.nz, zc[i] < g.nz ? zc[i] : g.nz, sp);
                    if (eff > prev) cand.push_back({t, zc[i], eff});
                    prev = eff > prev ? eff : prev;
                }
            }
        }
        cudaEvent_t a, b;
        if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
            (void)cudaGetLastError();
            return 0;
        }
        float best = 1e30f;
        Cand pick = cand.empty() ? Cand{tile, zchunk, zsplit} : cand[0];
        int done = 0;
        for (const auto &c : cand) {
            if (multi) {
                if (set_multi_tile(c.tile)) break;
            } else {
                tile = c.tile;
            }
            zchunk = c.zchunk;
            zsplit = c.zsplit;
            bool ok = sweep(kModePU, false) == PM_OK && sweep(kModePU, false) == PM_OK;
            cudaEventRecord(a, s);
            for (int r = 0; r < 2 * reps && ok; ++r) ok = sweep(kModePU, false) == PM_OK;
            cudaEventRecord(b, s);
            done += 2 * reps + 2;
            float ms = 0.f;
            if (ok && cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&ms, a, b) == cudaSuccess &&
                ms < best) {
                best = ms;
                pick = c;
            }
        }
        (void)cudaGetLastError();
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        if (multi) {
            if (set_multi_tile(pick.tile)) return done;
        } else {
            tile = pick.tile;
        }
        zchunk = pick.zchunk;
        zsplit = pick.zsplit;
        std::lock_guard<std::mutex> lock(mu);
        cache.push_back(Entry{dev, (int)sizeof(T), key, tile, zchunk, zsplit});
        return done;
    }

    // Reduction of the current state (a pressure-only pass would change p; instead run
    // the sums on a copy-free pass: P-mode reads u and writes p of the other buffer).
    int window(int M) {
        int st;
        for (int i = 0; i < M; ++i)
            if ((st = sweep(kModePU, i == M - 1))) return st;
        return reduce_to_host_async();
    }
};

struct Monitor {
    double q_prev[3] = {0, 0, 0};
    double d_prev = -1.0, d_best = INFINITY;
    double delta = INFINITY, err = INFINITY;
    int stalled = 0;  // consecutive windows without a new smallest change (any decrease counts:
                      // a slow but steady convergence keeps setting new minima, while at
                      // the FP32 floor the change only fluctuates)
    bool converged = false;
    // Window criterion (reading of Sec. 7.1, eps = delta|q| / |q|): relative change of
    // the mean velocity over one window, and its geometric-tail extrapolation.  ref > 0
    // replaces |q_dir| as the denominator (defect correction: the correction's mean is
    // measured against the full solution's).
    void update(const double q[3], int dir, double tol, double ref_in = 0.0) {
        const double ref = ref_in > 0 ? ref_in : std::fabs(q[dir]);
        double ch = 0.0;
        for (int d = 0; d < 3; ++d) ch = std::fmax(ch, std::fabs(q[d] - q_prev[d]));
        delta = ref > 0 ? ch / ref : INFINITY;
        if (ch == 0.0)
            err = 0.0;
        else if (d_prev > 0 && delta < d_prev) {
            double r = delta / d_prev;
            err = delta * r / (1.0 - r);
        } else
            err = INFINITY;
        d_prev = delta;
        if (delta < d_best) {
            d_best = delta;
            stalled = 0;
        } else
            ++stalled;
        for (int d = 0; d < 3; ++d) q_prev[d] = q[d];
        converged = delta < tol && err < tol;
    }
};

// Criterion of one run: tolerance, optional fixed reference scale per drive, and whether
// a stall (no new smallest change for 6 windows) ends the run (FP32 floor).
struct RunCriterion {
    double tol = 0.0;
    double ref[kMaxBatch] = {0, 0, 0, 0};
    bool stop_on_stall = false;
    long long max_iter = 0;
    bool retune = false;  // run the autotuner again (the sweep variant changed)
    // if set: before every window, the state of each problem is copied here (the state
    // one window before the end is then available for an extrapolation)
    void *prev_u[kMaxBatch] = {};
    void *prev_p[kMaxBatch] = {};
};

// Runs the batch to convergence from the loaded state.  Returns a pm_status.
template <typename T>
int run_to_convergence(Solver<T> &S, pm_stats *st, double t0, const RunCriterion *crit = nullptr) {
    const pm_options &o = S.o;
    RunCriterion defc;
    defc.tol = o.tol;
    defc.max_iter = o.max_iter;
    const RunCriterion &C = crit ? *crit : defc;
    int M = o.check_every + (o.check_every & 1);
    Monitor mon[kMaxBatch];
    long long conv_iter[kMaxBatch];
    for (int k = 0; k < kMaxBatch; ++k) conv_iter[k] = -1;
    int status = PM_OK;
    long long iters = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    double win_ms = 0.0;
    long long win_sweeps = 0;
    PM_CK(cudaEventCreate(&e0));
    PM_CK(cudaEventCreate(&e1));
    int rc = S.sweep(kModeU, false);
    if (rc) status = rc;
    iters = 1;
    if (!rc && o.autotune && (o.schedule == 0 || o.tile == 0) && (!crit || crit->retune || !S.tuned))
        iters += S.tune();
    S.tuned = true;
    bool done = status != PM_OK;
    bool use_graph = o.use_graph != 0;
    if (!done && use_graph) {
        // capture one window; M is even so the ping-pong roles repeat
        const int cur0 = S.F[0].cur;
        cudaError_t e = cudaStreamBeginCapture(S.s, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            S.capturing = true;
            rc = S.window(M);
            S.capturing = false;
            e = cudaStreamEndCapture(S.s, &graph);
            if (rc == PM_OK && e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
            if (e != cudaSuccess || rc != PM_OK) {
                (void)cudaGetLastError();
                use_graph = false;
                if (exec) cudaGraphExecDestroy(exec);
                exec = nullptr;
            }
        } else {
            (void)cudaGetLastError();
            use_graph = false;
        }
        for (int k = 0; k < S.nprob; ++k) S.F[k].cur = cur0;
    }
    while (!done) {
        if (C.prev_u[0]) {
            bool ok = true;
            for (int k = 0; k < S.nprob && ok; ++k) {
                const long long Nk = S.G(k).N;
                ok = cudaMemcpyAsync(C.prev_u[k], S.F[k].u[S.F[k].cur], sizeof(T) * 3 * Nk, cudaMemcpyDefault,
                                     S.s) == cudaSuccess &&
                     cudaMemcpyAsync(C.prev_p[k], S.F[k].p[S.F[k].cur], sizeof(T) * Nk, cudaMemcpyDefault, S.s) ==
                         cudaSuccess;
            }
            if (!ok) {
                status = map_cuda(cudaGetLastError());
                break;
            }
        }
        cudaEventRecord(e0, S.s);
        if (use_graph) {
            cudaError_t e = cudaGraphLaunch(exec, S.s);
            if (e != cudaSuccess) {
                status = map_cuda(e);
                break;
            }
            note_launch(M + 1);
        } else if ((rc = S.window(M))) {
            status = rc;
            break;
        }
        cudaEventRecord(e1, S.s);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            status = map_cuda(e);
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        win_ms += ms;
        win_sweeps += M;
        iters += M;
        bool all = true, bad = false;
        for (int k = 0; k < S.nprob; ++k) {
            const double *q = S.hq + 4 * k;
            if (!std::isfinite(q[0]) || !std::isfinite(q[1]) || !std::isfinite(q[2]) || !std::isfinite(q[3]))
                bad = true;
            mon[k].update(q, S.dir[k], C.tol, C.ref[k]);
            if (mon[k].converged && conv_iter[k] < 0) conv_iter[k] = iters;
            all = all && (mon[k].converged || (C.stop_on_stall && mon[k].stalled >= 6));
            if (st) {
                st[k].div_res = std::sqrt(q[3]);
                for (int d = 0; d < 3; ++d) st[k].q[d] = q[d];
            }
        }
        if (bad) {
            status = PM_ERR_DIVERGED;
            break;
        }
        if (all) break;
        if (S.multi) {
            // converged problems stop sweeping (even windows keep their buffer parity)
            bool changed = false;
            for (int k = 0; k < S.nprob; ++k) {
                const int a = mon[k].converged ? 0 : 1;
                changed |= a != S.active_h[k];
                S.active_h[k] = a;
            }
            if (changed) {
                cudaError_t e2 = cudaMemcpyAsync(S.active, S.active_h, sizeof(int) * S.nprob, cudaMemcpyHostToDevice, S.s);
                if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(S.s);
                if (e2 != cudaSuccess) {
                    status = map_cuda(e2);
                    break;
                }
            }
        }
        if (iters >= C.max_iter) {
            status = PM_ERR_NOT_CONVERGED;
            break;
        }
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    // last half step: pressure of the last iteration, plus the sums of the final state
    if (S.multi && (status == PM_OK || status == PM_ERR_NOT_CONVERGED)) {
        for (int k = 0; k < S.nprob; ++k) S.active_h[k] = 1;
        cudaError_t e2 = cudaMemcpyAsync(S.active, S.active_h, sizeof(int) * S.nprob, cudaMemcpyHostToDevice, S.s);
        if (e2 != cudaSuccess) status = map_cuda(e2);
    }
    if (status == PM_OK || status == PM_ERR_NOT_CONVERGED) {
        if ((rc = S.sweep(kModeP, true)) || (rc = S.reduce_to_host_async())) status = rc;
        else {
            cudaError_t e = cudaStreamSynchronize(S.s);
            if (e != cudaSuccess) status = map_cuda(e);
        }
        if (st && status != PM_ERR_CUDA)
            for (int k = 0; k < S.nprob; ++k)
                for (int d = 0; d < 3; ++d) st[k].q[d] = S.hq[4 * k + d];
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st)
        for (int k = 0; k < S.nprob; ++k) {
            st[k].iters = (S.multi && conv_iter[k] >= 0) ? conv_iter[k] + 1 : iters;
            st[k].delta = mon[k].delta;
            st[k].err_est = mon[k].err;
            bool src = false;
            for (int q = 0; q < S.nprob; ++q) src |= S.src[q] != nullptr;
            (src ? st[k].sweep_ms_src : st[k].sweep_ms) = win_sweeps ? win_ms / (double)win_sweeps : 0.0;
            (src ? st[k].sweeps_timed_src : st[k].sweeps_timed) = win_sweeps;
            st[k].seconds = now_s() - t0;
            // a member of a multi-geometry batch that met its criterion is converged even when
            // others ran into the iteration limit
            st[k].status = (S.multi && conv_iter[k] >= 0 && status == PM_ERR_NOT_CONVERGED) ? PM_OK : status;
            st[k].schedule = S.use_tiled() && !S.multi ? (S.zchunk > 0 ? S.zchunk : -1) : 0;
            st[k].setup_seconds = S.t_setup;
            st[k].tile = S.use_tiled() ? S.tile + 1 : 0;
            st[k].schedule_split = S.use_tiled() && !S.multi && S.zchunk > 0 ? S.zsplit : 0;
        }
    return status;
}

// Defect correction (precision pattern, not in the paper): FP32 sweeps to their floor,
// then rounds of  r = b - K x64 (FP64 residual)  ->  K d = r by FP32 sweeps from d = 0
// ->  x64 += d  until a round moves the mean velocity by less than tol.  The FP32 sweeps
// only ever carry a correction, so their rounding is relative to the correction.
// On return u64 / p64 hold the FP64 state of every drive and st[k].q its mean velocity.
int defect_correction(Solver<float> &S, const Geometry &g, pm_stats *st, double t0, double **u64, double **p64) {
    const pm_options &o = S.o;
    const long long N = g.N;
    RunCriterion c1;
    c1.tol = o.dc_switch_tol > o.tol ? o.dc_switch_tol : o.tol;
    c1.max_iter = o.max_iter;
    c1.stop_on_stall = true;
    float *prev_u[kMaxBatch] = {}, *prev_p[kMaxBatch] = {};
    if (o.dc_extrapolate) {
        int rc0;
        for (int k = 0; k < S.nprob; ++k) {
            if ((rc0 = S.scr.alloc(&prev_u[k], 3 * (size_t)N)) || (rc0 = S.scr.alloc(&prev_p[k], (size_t)N)))
                return rc0;
            c1.prev_u[k] = prev_u[k];
            c1.prev_p[k] = prev_p[k];
        }
    }
    int status = run_to_convergence<float>(S, st, t0, &c1);
    // geometric-tail factor r / (1 - r) of each drive's FP32 phase (0: start from zero)
    double tail[kMaxBatch] = {};
    if (o.dc_extrapolate)
        for (int k = 0; k < S.nprob; ++k) {
            const double f = st[k].delta > 0 ? st[k].err_est / st[k].delta : 0.0;
            tail[k] = std::isfinite(f) && f > 0 && f <= 49.0 ? f : 0.0;
        }
    if (status != PM_OK && status != PM_ERR_NOT_CONVERGED) return status;
    long long iters = st[0].iters, timed = 0;
    double ms = 0.0;
    float *r32[kMaxBatch] = {nullptr, nullptr, nullptr, nullptr};
    double q64[kMaxBatch][3];
    int rc;
    const int nb = tiled_grid_size() * 4;
    double *part = nullptr;
    if ((rc = S.scr.alloc(&part, (size_t)S.nprob * nb * 4))) return rc;
    for (int k = 0; k < S.nprob; ++k) {
        if ((rc = S.scr.alloc(&u64[k], 3 * (size_t)N)) || (rc = S.scr.alloc(&p64[k], (size_t)N)) ||
            (rc = S.scr.alloc(&r32[k], 4 * (size_t)N)))
            return rc;
        scale_copy_kernel<double, float><<<launch_grid(3 * N), 256, 0, S.s>>>(u64[k], S.F[k].u[S.F[k].cur], 1.0, 3 * N);
        scale_copy_kernel<double, float><<<launch_grid(N), 256, 0, S.s>>>(p64[k], S.F[k].p[S.F[k].cur], 1.0, N);
        note_launch(2);
        for (int d = 0; d < 3; ++d) q64[k][d] = st[k].q[d];
    }
    PM_CK(cudaGetLastError());
    int rounds = 0;
    pm_stats rs[kMaxBatch];
    // the residual carries the drive; the correction solves K d = r have no body force
    double force[kMaxBatch];
    for (int k = 0; k < S.nprob; ++k) force[k] = S.force[k];
    for (rounds = 1; rounds <= o.dc_max_rounds; ++rounds) {
        RunCriterion c2;
        c2.tol = o.tol;
        c2.max_iter = o.max_iter;
        c2.stop_on_stall = true;
        for (int k = 0; k < S.nprob; ++k) {
            double f[3] = {0, 0, 0};
            f[S.dir[k]] = force[k];
            S.force[k] = 0.0;
            residual64_kernel<<<launch_grid(N), 256, 0, S.s>>>(g.flags, g.nx, g.ny, g.nz, g.per[0], g.per[1], g.per[2],
                                                               u64[k], p64[k], 1.0 / o.Re, f[0], f[1], f[2], r32[k]);
            note_launch();
            // first round with extrapolation: buffer 0 starts from the estimated remaining
            // error of the FP32 phase (the FP64 master already holds that phase's state)
            const bool ext = rounds == 1 && tail[k] > 0;
            if (ext) {
                const int c = S.F[k].cur;
                extrapolate_kernel<float><<<launch_grid(3 * N), 256, 0, S.s>>>(S.F[k].u[0], S.F[k].u[c], prev_u[k],
                                                                              (float)tail[k], 3 * N);
                extrapolate_kernel<float><<<launch_grid(N), 256, 0, S.s>>>(S.F[k].p[0], S.F[k].p[c], prev_p[k],
                                                                          (float)tail[k], N);
                note_launch(2);
            }
            for (int b = ext ? 1 : 0; b < 2; ++b) {
                // a kernel, not a memset: the buffers may be in host memory (field_memory)
                fill_zero_kernel<float><<<launch_grid(3 * N), 256, 0, S.s>>>(S.F[k].u[b], 3 * N);
                fill_zero_kernel<float><<<launch_grid(N), 256, 0, S.s>>>(S.F[k].p[b], N);
                note_launch(2);
            }
            S.F[k].cur = 0;
            S.src[k] = r32[k];
            c2.ref[k] = std::fabs(q64[k][S.dir[k]]);
        }
        PM_CK(cudaGetLastError());
        std::memset(rs, 0, sizeof(rs));
        // the correction sweeps also read the source: their best tile shape and split are
        // tuned on their own (in the first round, as iterations of that round)
        c2.retune = rounds == 1;
        status = run_to_convergence<float>(S, rs, t0, &c2);
        if (status != PM_OK && status != PM_ERR_NOT_CONVERGED) break;
        iters += rs[0].iters;
        timed += rs[0].sweeps_timed_src;
        ms += rs[0].sweep_ms_src * (double)rs[0].sweeps_timed_src;
        double moved = 0.0;
        for (int k = 0; k < S.nprob; ++k) {
            accumulate_kernel<<<nb, 256, 0, S.s>>>(u64[k], p64[k], S.F[k].u[S.F[k].cur], S.F[k].p[S.F[k].cur], N,
                                                  part + (size_t)k * nb * 4);
        }
        reduce_partials_kernel<<<S.nprob, 256, 0, S.s>>>(part, nb, N, S.dq);
        note_launch(S.nprob + 1);
        PM_CK(cudaGetLastError());
        PM_CK(cudaMemcpyAsync(S.hq, S.dq, sizeof(double) * S.nprob * 4, cudaMemcpyDeviceToHost, S.s));
        PM_CK(cudaStreamSynchronize(S.s));
        for (int k = 0; k < S.nprob; ++k) {
            const double ref = std::fabs(S.hq[4 * k + S.dir[k]]);
            for (int d = 0; d < 3; ++d) {
                const double qn = S.hq[4 * k + d];
                if (!std::isfinite(qn)) status = PM_ERR_DIVERGED;
                moved = std::fmax(moved, ref > 0 ? std::fabs(qn - q64[k][d]) / ref : INFINITY);
                q64[k][d] = qn;
            }
            st[k].delta = rs[k].delta;
            st[k].err_est = rs[k].err_est;
            st[k].div_res = rs[k].div_res;
        }
        if (status == PM_ERR_DIVERGED) break;
        if (moved < o.tol) {
            status = PM_OK;
            break;
        }
        status = PM_ERR_NOT_CONVERGED;
    }
    for (int k = 0; k < S.nprob; ++k) {
        S.src[k] = nullptr;
        S.force[k] = force[k];
        for (int d = 0; d < 3; ++d) st[k].q[d] = q64[k][d];
        st[k].iters = iters;
        st[k].sweeps_timed_src = timed;
        st[k].sweep_ms_src = timed ? ms / (double)timed : 0.0;
        st[k].dc_rounds = rounds > o.dc_max_rounds ? o.dc_max_rounds : rounds;
        st[k].seconds = now_s() - t0;
        st[k].status = status;
    }
    return status;
}

template <typename T>
int iterate_impl(const pm_domain *dom, int dir, double drive, const pm_options *o, int64_t n, T *u, T *p,
                 cudaStream_t s, Scratch &scr) {
    Geometry g;
    int st = build_geometry(dom, s, scr, g);
    if (st) return st;
    Solver<T> S(g, *o, s, scr);
    if ((st = S.init(1))) return st;
    S.dir[0] = dir;
    S.force[0] = drive;
    if ((st = S.load_state(0, u, p))) return st;
    if (n > 0) {
        if ((st = S.sweep(kModeU, false))) return st;
        for (int64_t i = 1; i < n; ++i)
            if ((st = S.sweep(kModePU, false))) return st;
        if ((st = S.sweep(kModeP, false))) return st;
    }
    PM_CK(cudaMemcpyAsync(u, S.F[0].u[S.F[0].cur], sizeof(T) * 3 * g.N, cudaMemcpyDefault, s));
    PM_CK(cudaMemcpyAsync(p, S.F[0].p[S.F[0].cur], sizeof(T) * g.N, cudaMemcpyDefault, s));
    return PM_OK;
}

// Solve a batch of drive directions on one geometry.  Fields stay on the device in
// S.F; the caller extracts what it needs.
template <typename T>
int solve_batch(const Geometry &g, const pm_options *o, cudaStream_t s, Scratch &scr, int np, const int *dirs,
                Solver<T> &S, pm_stats *st, double t0) {
    int rc = S.init(np);
    if (rc) return rc;
    for (int k = 0; k < np; ++k) {
        S.dir[k] = dirs[k];
        S.force[k] = 1.0;  // Sec. 4: grad p = 1 per voxel in iteration units
    }
    return run_to_convergence<T>(S, st, t0);
}

inline int dc_dispatch(Solver<float> &S, const Geometry &g, pm_stats *st, double t0, double **u64, double **p64) {
    return defect_correction(S, g, st, t0, u64, p64);
}
inline int dc_dispatch(Solver<double> &, const Geometry &, pm_stats *, double, double **, double **) {
    return PM_ERR_UNSUPPORTED;
}

template <typename T>
int tensor_like(const pm_domain *dom, const pm_options *o, int ndirs, const int *dirs_in, double drive,
                       float *u_out, float *p_out, const float *u0, const float *p0, double kcols[3][3],
                       pm_stats *st, void *cuda_stream) {
    const double t0 = now_s();
    const long long l0 = t_launches;
    const int pax = pressure_axis(dom);
    if (pax >= 0 && o->precision == PM_FP32_DC64) return PM_ERR_UNSUPPORTED;
    for (int k = 0; k < ndirs; ++k)
        for (int i = 0; i < 3; ++i) kcols[k][i] = 0.0;
    StreamScope ss(cuda_stream);
    if (ss.status) return ss.status;
    int status = PM_OK, rc;
    pm_stats bst[kMaxBatch];
    std::memset(bst, 0, sizeof(bst));
    int dirs[3], np = 0, slot[3] = {-1, -1, -1};
    bool blocked = false;
    {
        Scratch scr(ss.s);
        Geometry g;
        if ((rc = build_geometry(dom, ss.s, scr, g))) return rc;
        // pore count and percolation on the device (Sec. 5.1)
        int perc[3] = {1, 1, 1}, wraps[3];
        long long n_pore = 0;
        if ((rc = percolation_device(g, o->check_percolation != 0, ss.s, scr, &n_pore, wraps))) return rc;
        if (n_pore == 0) return PM_ERR_NO_FLUID;
        if (o->check_percolation) {
            for (int a = 0; a < 3; ++a) perc[a] = wraps[a];
            if (pax >= 0) {
                std::vector<uint8_t> hm;
                if ((rc = host_mask(dom, hm))) return rc;
                perc[pax] = percolation_pressure(hm, dom->nx, dom->ny, dom->nz, g.per, pax);
            }
        }
        for (int k = 0; k < ndirs; ++k) {
            if (st) {
                std::memset(&st[k], 0, sizeof(pm_stats));
                st[k].percolates = perc[dirs_in[k]];
                st[k].n_fluid = n_pore;
            }
            if (perc[dirs_in[k]]) {
                slot[k] = np;
                dirs[np++] = dirs_in[k];
            } else
                blocked = true;
        }
        if (np > 0) {
            Solver<T> S(g, *o, ss.s, scr);
            rc = S.init(np);
            if (rc) return rc;
            S.t_setup = now_s() - t0;
            const double uscale = drive * dom->voxel_size * dom->voxel_size / (dom->viscosity * o->Re);
            const double pscale = drive * dom->voxel_size;
            for (int k = 0; k < np; ++k) {
                S.dir[k] = dirs[k];
                S.force[k] = 1.0;
            }
            if (u0 || p0) {
                // warm start (single drive only): Darcy-scaled float -> iteration units
                T *ut = S.F[0].u[0], *pt = S.F[0].p[0];
                if (u0) scale_copy_kernel<T, float><<<launch_grid(3 * g.N), 256, 0, ss.s>>>(ut, u0, 1.0 / uscale, 3 * g.N);
                if (p0) scale_copy_kernel<T, float><<<launch_grid(g.N), 256, 0, ss.s>>>(pt, p0, 1.0 / pscale, g.N);
                sanitize_kernel<T><<<launch_grid(g.N), 256, 0, ss.s>>>(g.flags, g.N, ut, pt);
                if (cudaGetLastError() != cudaSuccess) return PM_ERR_CUDA;
            }
            double *u64[kMaxBatch] = {nullptr, nullptr, nullptr, nullptr};
            double *p64[kMaxBatch] = {nullptr, nullptr, nullptr, nullptr};
            if (o->precision == PM_FP32_DC64)
                status = dc_dispatch(S, g, bst, t0, u64, p64);
            else
                status = run_to_convergence<T>(S, bst, t0);
            if (status == PM_OK || status == PM_ERR_NOT_CONVERGED) {
                if (u_out) {
                    if (u64[0])
                        scale_copy_kernel<float, double><<<launch_grid(3 * g.N), 256, 0, ss.s>>>(u_out, u64[0], uscale,
                                                                                                3 * g.N);
                    else
                        scale_copy_kernel<float, T><<<launch_grid(3 * g.N), 256, 0, ss.s>>>(
                            u_out, S.F[0].u[S.F[0].cur], uscale, 3 * g.N);
                }
                if (p_out) {
                    if (p64[0])
                        scale_copy_kernel<float, double><<<launch_grid(g.N), 256, 0, ss.s>>>(p_out, p64[0], pscale, g.N);
                    else
                        scale_copy_kernel<float, T><<<launch_grid(g.N), 256, 0, ss.s>>>(p_out, S.F[0].p[S.F[0].cur],
                                                                                       pscale, g.N);
                }
                if (cudaGetLastError() != cudaSuccess) status = PM_ERR_CUDA;
            }
        }
    }
    cudaError_t e = cudaStreamSynchronize(ss.s);
    if (e != cudaSuccess && status == PM_OK) status = map_cuda(e);
    for (int k = 0; k < ndirs; ++k) {
        if (slot[k] < 0) continue;
        const pm_stats &b = bst[slot[k]];
        // Appendix C: k_ij = mu q_i^(j) / h_j; iteration units mu = 1/Re, h = 1 -> q / Re.
        // Fixed-pressure axis a (n cells): the flow crosses the n - 1 face planes between
        // the layers, the cross components live in the n - 2 interior layers.
        for (int i = 0; i < 3; ++i) {
            double sup = 1.0;
            if (pax >= 0) {
                const double n = pax == 0 ? dom->nx : (pax == 1 ? dom->ny : dom->nz);
                sup = i == pax ? n / (n - 1.0) : n / (n - 2.0);
            }
            kcols[k][i] = sup * b.q[i] / o->Re * dom->voxel_size * dom->voxel_size;
        }
        if (st) {
            const int perc_k = st[k].percolates;
            const long long nf = st[k].n_fluid;
            st[k] = b;
            st[k].percolates = perc_k;
            st[k].n_fluid = nf;
        }
        if (st) st[k].kernel_launches = t_launches - l0;
    }
    if (status == PM_OK && blocked) status = PM_ERR_NOT_PERCOLATING;
    return status;
}

// ------------------------------------------------------------------ allocation-free iterate
// Fixed scratch of pm_iterate_noalloc: a copy of the mask, the neighbourhood flags and
// stencil codes, and the second buffer of the ping-pong pair (FP64 worst case).  It is
// a file-scope device array, so it exists on every GPU that loads the library until the
// process exits, and all calls share it.
constexpr long long kNoAllocMaxCells = 1ll << 17;
constexpr size_t kNoAllocBytes = (size_t)kNoAllocMaxCells * (1 + 1 + 4 + 4 * sizeof(double)) + 8 * 256;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of the scratch on the current device.  Host code only sees a host-side
// stand-in under the array's name, so the address is looked up once per device (with
// that device current) and cached.
int noalloc_scratch(unsigned char **out) {
    static std::mutex mu;
    static unsigned char *addr[256] = {};
    int dev = 0;
    PM_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) return PM_ERR_CUDA;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return map_cuda(e);
        }
        addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = addr[dev];
    return PM_OK;
}

template <typename T>
int iterate_noalloc_impl(const pm_domain *dom, int dir, double drive, const pm_options *o, int64_t n, T *u, T *p,
                         cudaStream_t s, unsigned char *scr) {
    const long long N = (long long)dom->nx * dom->ny * dom->nz;
    auto carve = [&](size_t bytes) {
        unsigned char *q = scr;
        scr += (bytes + 255) / 256 * 256;
        return q;
    };
    uint8_t *mask = carve((size_t)N);
    uint8_t *flags = carve((size_t)N);
    uint32_t *code = reinterpret_cast<uint32_t *>(carve(4 * (size_t)N));
    T *u2 = reinterpret_cast<T *>(carve(3 * sizeof(T) * (size_t)N));
    T *p2 = reinterpret_cast<T *>(carve(sizeof(T) * (size_t)N));
    const int per[3] = {dom->bc[0] == PM_BC_PERIODIC, dom->bc[1] == PM_BC_PERIODIC, dom->bc[2] == PM_BC_PERIODIC};
    PM_CK(cudaMemcpyAsync(mask, dom->mask, (size_t)N, dom->mask_on_device ? cudaMemcpyDeviceToDevice
                                                                          : cudaMemcpyHostToDevice, s));
    classify_kernel<<<launch_grid(N), 256, 0, s>>>(mask, dom->nx, dom->ny, dom->nz, per[0], per[1], per[2], -1,
                                                   flags);
    code_kernel<<<launch_grid(N), 256, 0, s>>>(mask, dom->nx, dom->ny, dom->nz, per[0], per[1], per[2], -1, code);
    sanitize_kernel<T><<<launch_grid(N), 256, 0, s>>>(flags, N, u, p);
    PM_CK(cudaGetLastError());
    if (n == 0) return PM_OK;
    const double dts = time_step(o);
    SweepBatch<T> B{};
    B.nx = dom->nx;
    B.ny = dom->ny;
    B.nz = dom->nz;
    for (int a = 0; a < 3; ++a) B.per[a] = per[a];
    B.N = N;
    B.flags = flags;
    B.alpha = nullptr;
    B.inv_re = (T)(1.0 / o->Re);
    B.dt = (T)dts;
    B.dtc2 = (T)(dts * o->c2);
    B.nprob = 1;
    B.zsplit = o->schedule > 0 && o->schedule_split > 1 ? o->schedule_split : 1;
    for (int d = 0; d < 3; ++d) B.prob[0].f[d] = (T)(d == dir ? drive : 0.0);
    // ping-pong between the caller's fields (buffer 0) and the scratch (buffer 1)
    T *ub[2] = {u, u2}, *pb[2] = {p, p2};
    int cur = 0;
    auto step = [&](int mode) -> int {
        B.prob[0].uin = ub[cur];
        B.prob[0].pin = pb[cur];
        B.prob[0].uout = ub[1 - cur];
        B.prob[0].pout = pb[1 - cur];
        B.prob[0].src = nullptr;
        B.prob[0].partials = nullptr;
        int st;
        if (o->kernel == 0 && tiled_supported<T>(B.nx, B.ny, B.nz, 1)) {
            if ((st = launch_tiled(B, code, mode, false, false, o->schedule > 0 ? o->schedule : 0, s,
                                      o->tile > 0 && o->tile <= tile_count<T>() ? o->tile - 1 : 0)))
                return st;
        } else {
            dim3 blk(32, 8, 1), grd((B.nx + 31) / 32, (B.ny + 7) / 8, (unsigned)B.nz);
            if (mode == kModeU) sweep_simple_kernel<T, kModeU, false, false><<<grd, blk, 0, s>>>(B);
            else if (mode == kModePU) sweep_simple_kernel<T, kModePU, false, false><<<grd, blk, 0, s>>>(B);
            else sweep_simple_kernel<T, kModeP, false, false><<<grd, blk, 0, s>>>(B);
        }
        PM_CK(cudaGetLastError());
        cur ^= 1;
        return PM_OK;
    };
    int st;
    if ((st = step(kModeU))) return st;
    for (int64_t i = 1; i < n; ++i)
        if ((st = step(kModePU))) return st;
    if ((st = step(kModeP))) return st;
    if (cur == 1) {
        PM_CK(cudaMemcpyAsync(u, u2, 3 * sizeof(T) * (size_t)N, cudaMemcpyDeviceToDevice, s));
        PM_CK(cudaMemcpyAsync(p, p2, sizeof(T) * (size_t)N, cudaMemcpyDeviceToDevice, s));
    }
    return PM_OK;
}

// Adjoint sensitivity (differentiation pattern, not in the paper).  J = sum w_ij k_ij with
// a per-cell drag alpha; forward solves for the drives j with a nonzero column of w,
// transposed solves for the rows i, then the face products (sensitivity_kernel).
template <typename T>
int sensitivity_impl(const pm_domain *dom, const float *alpha, const double w[9], const pm_options *o,
                     float *dJ, double *J, double *k_raw, void *const u_fwd[3], int fwd_given, cudaStream_t s,
                     Scratch &scr, double t0) {
    Geometry g;
    int rc = build_geometry(dom, s, scr, g);
    if (rc) return rc;
    {
        long long n_pore = 0;
        int wraps[3];
        if ((rc = percolation_device(g, false, s, scr, &n_pore, wraps))) return rc;
        if (n_pore == 0) return PM_ERR_NO_FLUID;
    }
    const T *alpha_t = nullptr;
    if (alpha) {
        if (sizeof(T) == sizeof(float)) {
            alpha_t = reinterpret_cast<const T *>(alpha);
        } else {
            T *a = nullptr;
            if ((rc = scr.alloc(&a, (size_t)g.N))) return rc;
            scale_copy_kernel<T, float><<<launch_grid(g.N), 256, 0, s>>>(a, alpha, 1.0, g.N);
            note_launch();
            PM_CK(cudaGetLastError());
            alpha_t = a;
        }
    }
    // forward drives: every column j of w with a nonzero entry (all three when dJ is NULL);
    // those whose fields the caller hands over are not solved again
    int fdirs[3], nf = 0, gdirs[3], ng = 0, adirs[3], na = 0;
    for (int j = 0; j < 3; ++j) {
        // no w: all three drives, forward only; no dJ: the drives of w's columns, forward only
        bool col = !w, row = false;
        for (int i = 0; i < 3 && w; ++i) {
            col |= w[3 * i + j] != 0.0;
            row |= dJ && w[3 * j + i] != 0.0;
        }
        if (col) {
            if (fwd_given && u_fwd && u_fwd[j]) gdirs[ng++] = j;
            else fdirs[nf++] = j;
        }
        if (row) adirs[na++] = j;
    }
    if (nf + ng == 0) return PM_ERR_INVALID_ARG;
    if (na > 0 && sizeof(T) == 4 && o->kernel == 0 && (rc = build_tcode(g, s, scr))) return rc;
    Solver<T> F(g, *o, s, scr), A(g, *o, s, scr);
    A.transposed = true;
    if ((nf > 0 && (rc = F.init(nf))) || (na > 0 && (rc = A.init(na)))) return rc;
    F.alpha = alpha_t;
    A.alpha = alpha_t;
    for (int k = 0; k < nf; ++k) {
        F.dir[k] = fdirs[k];
        F.force[k] = 1.0;
    }
    for (int k = 0; k < na; ++k) {
        A.dir[k] = adirs[k];
        A.force[k] = 1.0;
    }
    pm_stats sf[kMaxBatch], sa[kMaxBatch];
    std::memset(sf, 0, sizeof(sf));
    std::memset(sa, 0, sizeof(sa));
    int st = PM_OK;
    if (nf > 0) {
        st = run_to_convergence<T>(F, sf, t0);
        if (st != PM_OK && st != PM_ERR_NOT_CONVERGED) return st;
    }
    if (na > 0) {
        int st2 = run_to_convergence<T>(A, sa, t0);
        if (st2 != PM_OK && st2 != PM_ERR_NOT_CONVERGED) return st2;
        if (st == PM_OK) st = st2;
    }
    SensArgs<T> args{};
    double kr[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    const double dx2 = dom->voxel_size * dom->voxel_size;
    for (int k = 0; k < nf; ++k) {
        const int j = fdirs[k];
        args.fwd[j] = F.F[k].u[F.F[k].cur];
        for (int i = 0; i < 3; ++i) kr[3 * i + j] = sf[k].q[i] / o->Re * dx2;
        if (u_fwd && u_fwd[j] && !fwd_given)
            PM_CK(cudaMemcpyAsync(u_fwd[j], args.fwd[j], sizeof(T) * 3 * g.N, cudaMemcpyDefault, s));
    }
    if (ng > 0) {
        // mean velocities of the handed-over fields (Appendix C columns)
        const int nb = tiled_grid_size() * 4;
        double *part = nullptr, *dq = nullptr;
        if ((rc = scr.alloc(&part, (size_t)ng * nb * 4)) || (rc = scr.alloc(&dq, (size_t)ng * 4))) return rc;
        for (int k = 0; k < ng; ++k) {
            args.fwd[gdirs[k]] = static_cast<const T *>(u_fwd[gdirs[k]]);
            sum_u_kernel<T><<<nb, 256, 0, s>>>(args.fwd[gdirs[k]], g.N, part + (size_t)k * nb * 4);
        }
        reduce_partials_kernel<<<ng, 256, 0, s>>>(part, nb, g.N, dq);
        note_launch(ng + 1);
        PM_CK(cudaGetLastError());
        double hq[3 * 4];
        PM_CK(cudaMemcpyAsync(hq, dq, sizeof(double) * 4 * ng, cudaMemcpyDeviceToHost, s));
        PM_CK(cudaStreamSynchronize(s));
        for (int k = 0; k < ng; ++k)
            for (int i = 0; i < 3; ++i) kr[3 * i + gdirs[k]] = hq[4 * k + i] / o->Re * dx2;
    }
    for (int k = 0; k < na; ++k) args.adj[adirs[k]] = A.F[k].u[A.F[k].cur];
    double Jv = 0.0;
    for (int i = 0; i < 3 && w; ++i)
        for (int j = 0; j < 3; ++j) {
            args.w[i][j] = w[3 * i + j];
            Jv += w[3 * i + j] * kr[3 * i + j];
        }
    // dk_ij/d alpha_c = -(1 / (2 Re^2 N)) sum_F v^(i)_F u^(j)_F  (unit drive), times dx^2
    const double scale = -dx2 / (2.0 * o->Re * o->Re * (double)g.N);
    if (dJ) {
        sensitivity_kernel<T><<<launch_grid(g.N), 256, 0, s>>>(args, g.nx, g.ny, g.nz, g.per[0], g.per[1],
                                                              g.per[2], scale, dJ);
        note_launch();
        PM_CK(cudaGetLastError());
    }
    PM_CK(cudaStreamSynchronize(s));
    if (J) *J = Jv;
    if (k_raw)
        for (int i = 0; i < 9; ++i) k_raw[i] = kr[i];
    return st;
}

// Domain of an x extent that the tiled kernel takes (a multiple of 4): a periodic x axis
// is repeated 2 or 4 times (the periodic extension is the same discrete problem: the
// fixed point repeats and the mean velocities are unchanged); a wall x axis is padded with
// solid columns (the mean over the padded box is N'/N times the mean over the domain).
// The extended mask lives in scratch; *qscale converts mean velocities back, *rep counts
// the copies.
int extend_x(const pm_domain *dom, cudaStream_t s, Scratch &scr, pm_domain *out, double *qscale, int *rep) {
    *out = *dom;
    *qscale = 1.0;
    *rep = 1;
    if (dom->nx % 4 == 0) return PM_OK;
    const bool periodic = dom->bc[0] == PM_BC_PERIODIC;
    const int r = periodic ? (dom->nx % 2 == 0 ? 2 : 4) : 1;
    const int nxo = periodic ? r * dom->nx : (dom->nx + 3) / 4 * 4;
    const long long N = (long long)dom->nx * dom->ny * dom->nz, M = (long long)nxo * dom->ny * dom->nz;
    const uint8_t *src = dom->mask;
    int st;
    if (!dom->mask_on_device) {
        uint8_t *m = nullptr;
        if ((st = scr.alloc(&m, (size_t)N))) return st;
        PM_CK(cudaMemcpyAsync(m, dom->mask, (size_t)N, cudaMemcpyHostToDevice, s));
        src = m;
    }
    uint8_t *ext = nullptr;
    if ((st = scr.alloc(&ext, (size_t)M))) return st;
    extend_x_kernel<<<launch_grid(M), 256, 0, s>>>(src, dom->nx, dom->ny, dom->nz, nxo, r, ext);
    note_launch();
    PM_CK(cudaGetLastError());
    out->nx = nxo;
    out->mask = ext;
    out->mask_on_device = 1;
    *qscale = periodic ? 1.0 : (double)M / (double)N;
    *rep = r;
    return PM_OK;
}

// A thin domain (a few cells along z, many along y) is solved with its y and z axes
// exchanged, so that the tiled kernel marches along the long axis instead of restarting its
// plane pipeline every few planes.  The discrete operator treats every axis alike (the
// same stencils along x, y and z), so the exchanged problem is the same problem with k's
// rows and columns 1 and 2 exchanged.  Returns whether the axes were exchanged; *out then
// describes the exchanged mask (in scratch).
int swap_thin_yz(const pm_domain *dom, cudaStream_t s, Scratch &scr, pm_domain *out, bool *swapped) {
    *out = *dom;
    *swapped = false;
    if (!(dom->nz <= 16 && dom->ny >= 8 * dom->nz)) return PM_OK;
    const long long N = (long long)dom->nx * dom->ny * dom->nz;
    const uint8_t *src = dom->mask;
    int st;
    if (!dom->mask_on_device) {
        uint8_t *m = nullptr;
        if ((st = scr.alloc(&m, (size_t)N))) return st;
        PM_CK(cudaMemcpyAsync(m, dom->mask, (size_t)N, cudaMemcpyHostToDevice, s));
        src = m;
    }
    uint8_t *t = nullptr;
    if ((st = scr.alloc(&t, (size_t)N))) return st;
    swap_yz_kernel<<<launch_grid(N), 256, 0, s>>>(src, dom->nx, dom->ny, dom->nz, t);
    note_launch();
    PM_CK(cudaGetLastError());
    out->ny = dom->nz;
    out->nz = dom->ny;
    out->bc[1] = dom->bc[2];
    out->bc[2] = dom->bc[1];
    out->mask = t;
    out->mask_on_device = 1;
    *swapped = true;
    return PM_OK;
}

// Many geometries in one solve.  Batch mode: every (domain, drive) problem is a member of
// each sweep launch (one CTA per column chunk of each), windows are one captured graph,
// converged problems are switched off through device flags.  Sequence mode
// (opt->sequence): the domains are solved in order, the drives of one domain batched in
// each launch, and each domain starts from the converged fields of the one before it when
// the two have the same size (a precipitation sequence, Sec. 7.3, changes little from one
// image to the next); the fields are set to 0 where the new geometry has no fluid.
template <typename T>
int batch_impl(int nd, const pm_domain *doms, const int32_t *drives, const pm_options *o, double *k_out,
               double *k_raw, pm_stats *st, cudaStream_t s, Scratch &scr, double t0) {
    const long long l0 = t_launches;
    std::vector<Geometry> geos((size_t)nd);
    std::vector<double> qscale((size_t)nd, 1.0);
    std::vector<char> swapped((size_t)nd, 0);
    // axis a of the solved problem is axis ax(d, a) of domain d
    auto ax = [&](int d, int a) { return swapped[(size_t)d] && a > 0 ? 3 - a : a; };
    struct Prob {
        int d, j;
    };
    std::vector<Prob> probs;
    int status = PM_OK;
    for (int d = 0; d < nd; ++d) {
        for (int i = 0; i < 9; ++i) {
            k_out[9 * d + i] = 0.0;
            if (k_raw) k_raw[9 * d + i] = 0.0;
        }
        pm_domain sd, ed;
        bool sw = false;
        int rep = 1;
        int rc = swap_thin_yz(&doms[d], s, scr, &sd, &sw);
        if (rc) return rc;
        swapped[(size_t)d] = sw;
        if ((rc = extend_x(&sd, s, scr, &ed, &qscale[(size_t)d], &rep))) return rc;
        if ((rc = build_geometry(&ed, s, scr, geos[(size_t)d]))) return rc;
        int perc[3] = {1, 1, 1}, wraps[3];
        long long n_pore = 0;
        if ((rc = percolation_device(geos[(size_t)d], o->check_percolation != 0, s, scr, &n_pore, wraps))) return rc;
        if (n_pore == 0) return PM_ERR_NO_FLUID;
        if (o->check_percolation)
            for (int a = 0; a < 3; ++a) perc[a] = wraps[a];
        const int want = drives && drives[d] ? drives[d] : 7;
        for (int j = 0; j < 3; ++j) {
            // j: axis of the solved problem; the domain's axis is ax(d, j)
            const int jd = ax(d, j);
            if (st) {
                std::memset(&st[3 * d + jd], 0, sizeof(pm_stats));
                st[3 * d + jd].percolates = perc[j];
                st[3 * d + jd].n_fluid = n_pore / rep;
            }
            if (!(want & (1 << jd))) continue;
            if (!perc[j]) {
                status = PM_ERR_NOT_PERCOLATING;
                continue;
            }
            probs.push_back({d, j});
        }
    }
    // k column j of domain d from the converged mean velocities of problem k (j and the
    // components of q are axes of the solved problem; ax maps them to the domain's)
    auto record = [&](int d, int j, const pm_stats &b) {
        const double dx2 = doms[d].voxel_size * doms[d].voxel_size;
        const int jd = ax(d, j);
        for (int i = 0; i < 3; ++i) {
            const int id = ax(d, i);
            const double kij = qscale[(size_t)d] * b.q[i] / o->Re * dx2;  // Appendix C, column j
            if (k_raw) k_raw[9 * d + 3 * id + jd] = kij;
            k_out[9 * d + 3 * id + jd] += 0.5 * kij;
            k_out[9 * d + 3 * jd + id] += 0.5 * kij;
        }
        if (st) {
            const int perc = st[3 * d + jd].percolates;
            const long long nf = st[3 * d + jd].n_fluid;
            st[3 * d + jd] = b;
            for (int i = 0; i < 3; ++i) st[3 * d + jd].q[ax(d, i)] = qscale[(size_t)d] * b.q[i];
            st[3 * d + jd].percolates = perc;
            st[3 * d + jd].n_fluid = nf;
        }
    };
    if (o->sequence) {
        // warm-start fields per drive (iteration units), from the previous domain
        T *wu[3] = {nullptr, nullptr, nullptr}, *wp[3] = {nullptr, nullptr, nullptr};
        bool warm[3] = {false, false, false};
        long long wN = -1;
        int wshape[3] = {0, 0, 0};
        size_t pi = 0;
        for (int d = 0; d < nd; ++d) {
            const Geometry &g = geos[(size_t)d];
            int dirs[3], np = 0;
            while (pi < probs.size() && probs[pi].d == d) dirs[np++] = probs[pi++].j;
            const bool same = g.nx == wshape[0] && g.ny == wshape[1] && g.nz == wshape[2];
            if (!same) warm[0] = warm[1] = warm[2] = false;
            if (np == 0) continue;
            if (wN < 0) {
                wN = g.N;
                for (int j = 0; j < 3; ++j) {
                    int rc;
                    if ((rc = scr.alloc(&wu[j], (size_t)(3 * g.N))) || (rc = scr.alloc(&wp[j], (size_t)g.N))) return rc;
                }
            }
            Solver<T> S(g, *o, s, scr);
            int rc = S.init(np);
            if (rc) return rc;
            for (int k = 0; k < np; ++k) {
                S.dir[k] = dirs[k];
                S.force[k] = 1.0;
                if (same && warm[dirs[k]] && (rc = S.load_state(k, wu[dirs[k]], wp[dirs[k]]))) return rc;
            }
            S.t_setup = now_s() - t0;
            pm_stats bst[kMaxBatch];
            std::memset(bst, 0, sizeof(bst));
            rc = run_to_convergence<T>(S, bst, t0);
            if (rc != PM_OK && rc != PM_ERR_NOT_CONVERGED) return rc;
            if (rc == PM_ERR_NOT_CONVERGED && status == PM_OK) status = rc;
            for (int k = 0; k < np; ++k) record(d, dirs[k], bst[k]);
            // keep this domain's fields for the next one (same size only)
            if (g.N <= wN) {
                for (int k = 0; k < np; ++k) {
                    const int j = dirs[k];
                    PM_CK(cudaMemcpyAsync(wu[j], S.F[k].u[S.F[k].cur], sizeof(T) * 3 * g.N, cudaMemcpyDefault, s));
                    PM_CK(cudaMemcpyAsync(wp[j], S.F[k].p[S.F[k].cur], sizeof(T) * g.N, cudaMemcpyDefault, s));
                    warm[j] = true;
                }
                for (int j = 0; j < 3; ++j) {
                    bool solved = false;
                    for (int k = 0; k < np; ++k) solved |= dirs[k] == j;
                    if (!solved) warm[j] = false;
                }
                wshape[0] = g.nx;
                wshape[1] = g.ny;
                wshape[2] = g.nz;
            } else {
                warm[0] = warm[1] = warm[2] = false;
                wshape[0] = wshape[1] = wshape[2] = 0;
            }
        }
    } else {
        for (size_t g0 = 0; g0 < probs.size(); g0 += kMaxBatch) {
            const int np = (int)std::min<size_t>(kMaxBatch, probs.size() - g0);
            Solver<T> S(geos[(size_t)probs[g0].d], *o, s, scr);
            S.multi = true;
            for (int k = 0; k < np; ++k) {
                S.geo[k] = &geos[(size_t)probs[g0 + k].d];
                S.dir[k] = probs[g0 + k].j;
                S.force[k] = 1.0;
            }
            int rc = S.init(np);
            if (rc) return rc;
            S.t_setup = now_s() - t0;
            pm_stats bst[kMaxBatch];
            std::memset(bst, 0, sizeof(bst));
            rc = run_to_convergence<T>(S, bst, t0);
            if (rc != PM_OK && rc != PM_ERR_NOT_CONVERGED) return rc;
            if (rc == PM_ERR_NOT_CONVERGED && status == PM_OK) status = rc;
            for (int k = 0; k < np; ++k) record(probs[g0 + k].d, probs[g0 + k].j, bst[k]);
        }
    }
    if (st)
        for (int i = 0; i < 3 * nd; ++i) st[i].kernel_launches = t_launches - l0;
    return status;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

void pm_default_options(pm_options *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->tol = 1e-6;
    o->check_every = 200;
    o->max_iter = 2000000;
    o->precision = PM_FP32_RED64;
    o->dt_safety = 0.9;
    o->Re = 0.01;
    o->c2 = 1.5e6;
    o->use_graph = 1;
    o->check_percolation = 1;
    o->dc_switch_tol = 1e-6;
    o->dc_max_rounds = 8;
    o->kernel = 0;
    o->autotune = 1;
}

const char *pm_strerror(int s) {
    switch (s) {
    case PM_OK: return "ok";
    case PM_ERR_INVALID_ARG: return "invalid argument";
    case PM_ERR_NO_FLUID: return "the mask has no pore voxel";
    case PM_ERR_NOT_PERCOLATING: return "no fluid path wraps the domain along a drive axis";
    case PM_ERR_NOT_CONVERGED: return "iteration limit reached before the tolerance";
    case PM_ERR_DIVERGED: return "non-finite values in the iteration";
    case PM_ERR_OOM: return "device memory allocation failed";
    case PM_ERR_CUDA: return "CUDA runtime error";
    case PM_ERR_TIMEOUT: return "bounded device wait ran out";
    case PM_ERR_UNSUPPORTED: return "option combination not supported";
    case PM_ERR_TOO_LARGE: return "domain larger than the fixed scratch of pm_iterate_noalloc (131072 cells)";
    default: return "unknown status";
    }
}

int pm_version(void) { return kVersion; }

int pm_release_memory(void) {
    int dev = 0;
    PM_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return PM_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (g_pools[dev]) PM_CK(cudaMemPoolTrimTo(g_pools[dev], 0));
    return PM_OK;
}

// Sec. 2: eigenvalues / eigenvectors of the symmetric part of k by cyclic Jacobi
// rotations (each rotation zeroes one off-diagonal pair; sweeps until the off-diagonal
// mass is below machine precision relative to the diagonal).
int pm_principal_axes(const double k[9], double lambda[3], double axes[9]) {
    if (!k || !lambda) return PM_ERR_INVALID_ARG;
    double a[3][3], v[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            if (!std::isfinite(k[3 * i + j])) return PM_ERR_INVALID_ARG;
            a[i][j] = 0.5 * (k[3 * i + j] + k[3 * j + i]);
        }
    for (int sweep = 0; sweep < 64; ++sweep) {
        double off = 0.0, diag = 0.0;
        for (int i = 0; i < 3; ++i) {
            diag += a[i][i] * a[i][i];
            for (int j = i + 1; j < 3; ++j) off += a[i][j] * a[i][j];
        }
        if (off <= 1e-34 * diag || off == 0.0) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                if (a[p][q] == 0.0) continue;
                // rotation angle that zeroes a[p][q]: tan(2 theta) = 2 a_pq / (a_qq - a_pp)
                const double theta = 0.5 * (a[q][q] - a[p][p]) / a[p][q];
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int r = 0; r < 3; ++r) {  // columns p, q of a
                    const double arp = a[r][p], arq = a[r][q];
                    a[r][p] = c * arp - s * arq;
                    a[r][q] = s * arp + c * arq;
                }
                for (int r = 0; r < 3; ++r) {  // rows p, q
                    const double apr = a[p][r], aqr = a[q][r];
                    a[p][r] = c * apr - s * aqr;
                    a[q][r] = s * apr + c * aqr;
                }
                for (int r = 0; r < 3; ++r) {
                    const double vrp = v[r][p], vrq = v[r][q];
                    v[r][p] = c * vrp - s * vrq;
                    v[r][q] = s * vrp + c * vrq;
                }
            }
    }
    int ord[3] = {0, 1, 2};
    for (int i = 0; i < 3; ++i)
        for (int j = i + 1; j < 3; ++j)
            if (a[ord[j]][ord[j]] < a[ord[i]][ord[i]]) std::swap(ord[i], ord[j]);
    for (int j = 0; j < 3; ++j) {
        const int c = ord[j];
        lambda[j] = a[c][c];
        if (!axes) continue;
        int big = 0;
        for (int i = 1; i < 3; ++i)
            if (std::fabs(v[i][c]) > std::fabs(v[big][c])) big = i;
        const double sg = v[big][c] < 0 ? -1.0 : 1.0;
        for (int i = 0; i < 3; ++i) axes[3 * i + j] = sg * v[i][c];
    }
    return PM_OK;
}

int pm_mirror_mask(const uint8_t *mask, int32_t nx, int32_t ny, int32_t nz, int32_t axes, int32_t on_device,
                   uint8_t *out, void *cuda_stream) {
    if (!mask || !out || nx < 1 || ny < 1 || nz < 1 || axes < 0 || axes > 7) return PM_ERR_INVALID_ARG;
    const int mx = axes & 1, my = (axes >> 1) & 1, mz = (axes >> 2) & 1;
    const long long ox = (long long)nx << mx, oy = (long long)ny << my, oz = (long long)nz << mz;
    if (on_device) {
        cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
        mirror_kernel<<<launch_grid(ox * oy * oz), 256, 0, s>>>(mask, nx, ny, nz, mx, my, mz, out);
        PM_CK(cudaGetLastError());
        PM_CK(cudaStreamSynchronize(s));
        return PM_OK;
    }
    for (long long z = 0; z < oz; ++z)
        for (long long y = 0; y < oy; ++y)
            for (long long x = 0; x < ox; ++x) {
                const long long sx = x < nx ? x : 2 * nx - 1 - x, sy = y < ny ? y : 2 * ny - 1 - y,
                                sz = z < nz ? z : 2 * nz - 1 - z;
                out[x + ox * (y + oy * z)] = mask[sx + nx * (sy + ny * sz)];
            }
    return PM_OK;
}

// Components of face-connected pore cells by breadth-first search; a component is kept
// when it wraps a periodic axis (two paths to one cell that cross that boundary a
// different number of times) or holds cells in both end layers of a fixed-pressure axis.
int pm_remove_isolated_pores(const uint8_t *mask, int32_t nx, int32_t ny, int32_t nz, const int32_t bc[3],
                             uint8_t *out, int64_t *removed) {
    if (!mask || !out || !bc || nx < 1 || ny < 1 || nz < 1) return PM_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a)
        if (bc[a] != PM_BC_PERIODIC && bc[a] != PM_BC_WALL && bc[a] != PM_BC_PRESSURE) return PM_ERR_INVALID_ARG;
    const long long N = (long long)nx * ny * nz;
    const int n[3] = {nx, ny, nz};
    std::vector<uint8_t> m(mask, mask + N), seen((size_t)N, 0);
    std::vector<int16_t> wind((size_t)N * 3);
    std::vector<long long> comp;
    long long gone = 0;
    for (long long s0 = 0; s0 < N; ++s0) {
        if (m[s0] || seen[s0]) continue;
        comp.clear();
        comp.push_back(s0);
        seen[s0] = 1;
        wind[s0 * 3] = wind[s0 * 3 + 1] = wind[s0 * 3 + 2] = 0;
        bool flows = false, lo[3] = {false, false, false}, hi[3] = {false, false, false};
        for (size_t h = 0; h < comp.size(); ++h) {
            const long long c = comp[h];
            const int co[3] = {(int)(c % nx), (int)((c / nx) % ny), (int)(c / ((long long)nx * ny))};
            for (int a = 0; a < 3; ++a) {
                lo[a] = lo[a] || co[a] == 0;
                hi[a] = hi[a] || co[a] == n[a] - 1;
                for (int dm = -1; dm <= 1; dm += 2) {
                    int cc[3] = {co[0], co[1], co[2]};
                    int w = 0;
                    cc[a] += dm;
                    if (cc[a] < 0 || cc[a] >= n[a]) {
                        if (bc[a] != PM_BC_PERIODIC) continue;
                        w = cc[a] < 0 ? -1 : 1;
                        cc[a] = (cc[a] + n[a]) % n[a];
                    }
                    const long long b = cc[0] + (long long)nx * (cc[1] + (long long)ny * cc[2]);
                    if (m[b]) continue;
                    int16_t wn[3] = {wind[c * 3], wind[c * 3 + 1], wind[c * 3 + 2]};
                    wn[a] = (int16_t)(wn[a] + w);
                    if (!seen[b]) {
                        seen[b] = 1;
                        for (int k = 0; k < 3; ++k) wind[b * 3 + k] = wn[k];
                        comp.push_back(b);
                    } else {
                        for (int k = 0; k < 3; ++k)
                            if (wind[b * 3 + k] != wn[k]) flows = true;
                    }
                }
            }
        }
        for (int a = 0; a < 3; ++a)
            if (bc[a] == PM_BC_PRESSURE && lo[a] && hi[a] && n[a] >= 2) flows = true;
        if (!flows) {
            for (long long c : comp) m[c] = 1;
            gone += (long long)comp.size();
        }
    }
    std::memcpy(out, m.data(), (size_t)N);
    if (removed) *removed = gone;
    return PM_OK;
}

int pm_anisotropy_class(const double lambda[3], double rel_tol) {
    if (!lambda || !(rel_tol >= 0)) return -1;
    double m = 0.0;
    for (int i = 0; i < 3; ++i) {
        if (!std::isfinite(lambda[i])) return -1;
        m = std::fmax(m, std::fabs(lambda[i]));
    }
    auto eq = [&](double x, double y) { return std::fabs(x - y) <= rel_tol * m; };
    const int n = eq(lambda[0], lambda[1]) + eq(lambda[0], lambda[2]) + eq(lambda[1], lambda[2]);
    return n >= 2 ? 0 : (n == 1 ? 1 : 2);
}

double pm_time_step(const pm_options *o) { return o ? time_step(o) : 0.0; }

int pm_iterate(const pm_domain *dom, int dir, double drive, const pm_options *o, int64_t n, void *u, void *p,
               void *cuda_stream) {
    int st = validate_domain(dom);
    if (st) return st;
    if ((st = validate_options(o))) return st;
    if (dir < 0 || dir > 2 || !u || !p || n < 0) return PM_ERR_INVALID_ARG;
    if (o->precision == PM_FP32_DC64) return PM_ERR_INVALID_ARG;
    if (pressure_axis(dom) >= 0 && dir != pressure_axis(dom)) return PM_ERR_INVALID_ARG;
    StreamScope ss(cuda_stream);
    if (ss.status) return ss.status;
    {
        Scratch scr(ss.s);
        if (o->precision == PM_FP64)
            st = iterate_impl<double>(dom, dir, drive, o, n, (double *)u, (double *)p, ss.s, scr);
        else
            st = iterate_impl<float>(dom, dir, drive, o, n, (float *)u, (float *)p, ss.s, scr);
    }
    cudaError_t e = cudaStreamSynchronize(ss.s);
    if (!st && e != cudaSuccess) st = map_cuda(e);
    return st;
}

int pm_iterate_noalloc(const pm_domain *dom, int dir, double drive, const pm_options *o, int64_t n, void *u,
                       void *p, void *cuda_stream) {
    int st = validate_domain(dom);
    if (st) return st;
    if ((st = validate_options(o))) return st;
    if (dir < 0 || dir > 2 || !u || !p || n < 0) return PM_ERR_INVALID_ARG;
    if (o->precision == PM_FP32_DC64) return PM_ERR_INVALID_ARG;
    if (pressure_axis(dom) >= 0) return PM_ERR_UNSUPPORTED;
    if ((long long)dom->nx * dom->ny * dom->nz > kNoAllocMaxCells) return PM_ERR_TOO_LARGE;
    // the caller's fields are one buffer of the ping-pong pair, read by 16-byte bulk copies
    if (reinterpret_cast<uintptr_t>(u) % 16 || reinterpret_cast<uintptr_t>(p) % 16) return PM_ERR_INVALID_ARG;
    unsigned char *scr = nullptr;
    if ((st = noalloc_scratch(&scr))) return st;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (o->precision == PM_FP64)
        st = iterate_noalloc_impl<double>(dom, dir, drive, o, n, (double *)u, (double *)p, s, scr);
    else
        st = iterate_noalloc_impl<float>(dom, dir, drive, o, n, (float *)u, (float *)p, s, scr);
    if (st) return st;
    // the host mask (if any) is read by an asynchronous copy: finish before returning
    cudaError_t e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? PM_OK : map_cuda(e);
}

int pm_solve_direction(const pm_domain *dom, int dir, double drive, const pm_options *o, float *u, float *p,
                       const float *u0, const float *p0, double *k_col, pm_stats *st, void *cuda_stream) {
    int rc = validate_domain(dom);
    if (rc) return rc;
    if ((rc = validate_options(o))) return rc;
    if (dir < 0 || dir > 2 || !(drive > 0)) return PM_ERR_INVALID_ARG;
    if (pressure_axis(dom) >= 0 && dir != pressure_axis(dom)) return PM_ERR_INVALID_ARG;
    double kc[3][3];
    pm_stats local;
    int dirs[1] = {dir};
    if (o->precision == PM_FP64)
        rc = tensor_like<double>(dom, o, 1, dirs, drive, u, p, u0, p0, kc, st ? st : &local, cuda_stream);
    else
        rc = tensor_like<float>(dom, o, 1, dirs, drive, u, p, u0, p0, kc, st ? st : &local, cuda_stream);
    if (k_col)
        for (int i = 0; i < 3; ++i) k_col[i] = kc[0][i];
    return rc;
}

int pm_sensitivity(const pm_domain *dom, const float *alpha, const double w[9], const pm_options *o,
                   float *dJ_dalpha, double *J, double k_raw[9], void *const u_fwd[3], int32_t fwd_given,
                   void *cuda_stream) {
    int rc = validate_domain(dom);
    if (rc) return rc;
    if ((rc = validate_options(o))) return rc;
    if (dJ_dalpha && !w) return PM_ERR_INVALID_ARG;
    if (o->precision == PM_FP32_DC64 || pressure_axis(dom) >= 0) return PM_ERR_UNSUPPORTED;
    const double t0 = now_s();
    StreamScope ss(cuda_stream);
    if (ss.status) return ss.status;
    {
        Scratch scr(ss.s);
        if (o->precision == PM_FP64)
            rc = sensitivity_impl<double>(dom, alpha, w, o, dJ_dalpha, J, k_raw, u_fwd, fwd_given, ss.s, scr, t0);
        else
            rc = sensitivity_impl<float>(dom, alpha, w, o, dJ_dalpha, J, k_raw, u_fwd, fwd_given, ss.s, scr, t0);
    }
    cudaError_t e = cudaStreamSynchronize(ss.s);
    if (rc == PM_OK && e != cudaSuccess) rc = map_cuda(e);
    return rc;
}

int pm_batch_ktensor(int n_domains, const pm_domain *doms, const int32_t *drives, const pm_options *o,
                     double *k_out, double *k_raw, pm_stats *st, void *cuda_stream) {
    if (n_domains < 1 || !doms || !k_out) return PM_ERR_INVALID_ARG;
    int rc = validate_options(o);
    if (rc) return rc;
    if (o->precision == PM_FP32_DC64) return PM_ERR_UNSUPPORTED;
    for (int d = 0; d < n_domains; ++d) {
        if ((rc = validate_domain(&doms[d]))) return rc;
        if (pressure_axis(&doms[d]) >= 0) return PM_ERR_UNSUPPORTED;
        for (int a = 0; a < 3; ++a)
            if (doms[d].bc[a] != doms[0].bc[a]) return PM_ERR_UNSUPPORTED;
        if (drives && (drives[d] < 0 || drives[d] > 7)) return PM_ERR_INVALID_ARG;
    }
    const double t0 = now_s();
    StreamScope ss(cuda_stream);
    if (ss.status) return ss.status;
    {
        Scratch scr(ss.s);
        if (o->precision == PM_FP64)
            rc = batch_impl<double>(n_domains, doms, drives, o, k_out, k_raw, st, ss.s, scr, t0);
        else
            rc = batch_impl<float>(n_domains, doms, drives, o, k_out, k_raw, st, ss.s, scr, t0);
    }
    cudaError_t e = cudaStreamSynchronize(ss.s);
    if ((rc == PM_OK || rc == PM_ERR_NOT_PERCOLATING) && e != cudaSuccess) rc = map_cuda(e);
    return rc;
}

int pm_permeability_tensor(const pm_domain *dom, double drive, const pm_options *o, double k_out[9],
                           double k_raw[9], pm_stats st[3], void *cuda_stream) {
    int rc = validate_domain(dom);
    if (rc) return rc;
    if ((rc = validate_options(o))) return rc;
    if (!k_out || !(drive > 0)) return PM_ERR_INVALID_ARG;
    if (pressure_axis(dom) >= 0) return PM_ERR_UNSUPPORTED;  // one drive only: pm_solve_direction
    double kc[3][3];
    int dirs[3] = {0, 1, 2};
    if (o->precision == PM_FP64)
        rc = tensor_like<double>(dom, o, 3, dirs, drive, nullptr, nullptr, nullptr, nullptr, kc, st, cuda_stream);
    else
        rc = tensor_like<float>(dom, o, 3, dirs, drive, nullptr, nullptr, nullptr, nullptr, kc, st, cuda_stream);
    // kc[j][i] = k_ij (column j from drive j); Sec. 6.4 / Appendix C: average off-diagonals
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            if (k_raw) k_raw[3 * i + j] = kc[j][i];
            k_out[3 * i + j] = 0.5 * (kc[j][i] + kc[i][j]);
        }
    return rc;
}

}  // extern "C"
