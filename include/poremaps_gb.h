/*
 * poremaps_gb.h - C ABI of the GB300 permeability solver (libpm_gb300.so).
 *
 * The library computes the intrinsic permeability tensor k of a binary voxel image by
 * the method of Krach, Ruf and Steeb, "POREMAPS: A finite difference based Porous Media
 * Anisotropic Permeability Solver for Stokes flow" (arXiv 2407.19868):
 *   - pseudo-unsteady (artificial compressibility) Stokes equations, Sec. 3 and
 *     Appendix A, stepped in pseudo time on a staggered MAC grid, Sec. 4 "Grid";
 *   - no-slip / no-penetration at the voxel faces between pore and solid through the
 *     Taylor-series wall cases of Sec. 4 and Appendix B; periodic outer boundaries
 *     (or no-slip walls), Sec. 4 "Boundary ...";
 *   - per iteration the velocity update, then the pressure update with the new
 *     velocities, then the evaluation of permeability and convergence (Algorithm 1);
 *   - k from Darcy's law with one drive per axis, Eq. (darcy), Eq. (cases_pressure)
 *     and Appendix C, off-diagonals averaged (Sec. 6.4, Appendix C).
 *
 * Conventions used by every entry point
 *   - Masks are uint8 arrays in C order [nz][ny][nx] (x fastest); nonzero = solid.
 *   - Fields are structure-of-arrays: u = [u_x | u_y | u_z], each nx*ny*nz long, u_d(c)
 *     lives on the +d face of cell c; p lives at cell centres.  Non-fluid faces hold 0.
 *   - Fields passed to or returned by pm_iterate are in the paper's iteration units
 *     (Sec. 4: length 1 voxel, velocity 1 voxel/s, Re and c*^2 from pm_options); the
 *     drive is a body force f on the fluid faces normal to the drive axis, which is the
 *     same discrete problem as the paper's pressure gradient with a periodic jump.
 *   - pm_solve_direction returns Darcy-scaled fields: u in the units of
 *     drive * voxel_size^2 / viscosity (m/s for SI inputs), p in drive * voxel_size.
 *   - k is returned in voxel_size^2 units (m^2 for voxel_size in metres).
 *   - cuda_stream is a cudaStream_t (NULL = legacy default stream).  The library runs
 *     on its own internal stream ordered after cuda_stream and orders cuda_stream after
 *     its work; device outputs are complete on cuda_stream when the call returns.
 *   - Ownership: the caller owns every pointer it passes and keeps device pointers valid
 *     for the call; the library never frees caller memory.  Scratch (ping-pong fields,
 *     neighbourhood codes, FP64 master copies, reduction buffers) comes from the
 *     library's own stream-ordered memory pool (one per device) inside each call and
 *     goes back to that pool before the call returns; the pool keeps it reserved for the
 *     next call (no allocation cost when the same or a smaller domain comes again) until
 *     pm_release_memory hands it back to the driver.
 *   - Errors: every function returns a pm_status; nothing throws or aborts.  On an error
 *     return, outputs may be partially written.
 */
#ifndef POREMAPS_GB_H
#define POREMAPS_GB_H

#include <stdint.h>

#if defined(__GNUC__)
#define PM_API __attribute__((visibility("default")))
#else
#define PM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum pm_status {
    PM_OK = 0,
    PM_ERR_INVALID_ARG = 1,     /* NULL pointer, bad enum, dims < 1, bad option */
    PM_ERR_NO_FLUID = 2,        /* the mask has no pore voxel */
    PM_ERR_NOT_PERCOLATING = 3, /* no fluid path wraps the domain along a drive axis;
                                   that k column is 0, the others are still computed */
    PM_ERR_NOT_CONVERGED = 4,   /* max_iter reached; outputs valid, stats say how far */
    PM_ERR_DIVERGED = 5,        /* NaN or Inf in the reductions */
    PM_ERR_OOM = 6,             /* device allocation failed */
    PM_ERR_CUDA = 7,            /* any other CUDA runtime error */
    PM_ERR_TIMEOUT = 8,         /* a bounded device wait ran out (reserved: no kernel of
                                   this version waits on another thread or device) */
    PM_ERR_UNSUPPORTED = 9,     /* option combination not implemented */
    PM_ERR_TOO_LARGE = 10       /* domain exceeds pm_iterate_noalloc's fixed scratch */
} pm_status;

/* Outer boundary per axis.
 *   PM_BC_PERIODIC  the domain repeats (Sec. 4; the drive is a pressure jump across it)
 *   PM_BC_WALL      no-slip wall: the cells outside the box count as solid
 *   PM_BC_PRESSURE  fixed-pressure inlet/outlet (Sec. 4 names a fixed pressure in the main
 *                   flow direction; this is the library's reading of it): the first and
 *                   the last cell layer along the axis are reservoirs with fixed pressures
 *                   p_in and p_out and no flow inside them (their velocities across the
 *                   axis are 0); outside the box counts as solid; the inlet and outlet
 *                   faces use a zero-gradient axial neighbour.  At most one axis, with at
 *                   least 3 cells; the drive must be along it (p_in - p_out = drive x
 *                   (n_axis - 1) dx).  Supported by pm_iterate and pm_solve_direction
 *                   (PM_FP32_RED64 and PM_FP64); the other entry points return
 *                   PM_ERR_UNSUPPORTED. */
enum { PM_BC_PERIODIC = 0, PM_BC_WALL = 1, PM_BC_PRESSURE = 2 };

/* Arithmetic of the pseudo-time sweeps. */
enum {
    PM_FP32_RED64 = 0, /* FP32 fields, FP64 reductions (mean velocity, residual) */
    PM_FP32_DC64 = 1,  /* as above, then FP64 defect correction: r = b - K x in FP64,
                          K d = r by FP32 sweeps, x += d, until the tolerance holds */
    PM_FP64 = 2        /* FP64 fields throughout */
};

typedef struct pm_domain {
    int32_t nx, ny, nz;       /* voxels per axis, each >= 1 */
    const uint8_t *mask;      /* [nz][ny][nx], nonzero = solid; host or device */
    int32_t mask_on_device;   /* 1: mask is a device pointer */
    double voxel_size;        /* dx; k is returned in dx^2 units (m^2 if dx in m) */
    double viscosity;         /* mu; scales the returned velocities only */
    int32_t bc[3];            /* per axis x, y, z: PM_BC_PERIODIC, PM_BC_WALL or PM_BC_PRESSURE */
} pm_domain;

typedef struct pm_options {
    double tol;               /* stop when the mean velocity changed by less than tol
                                 (relative to the driven component) over one window,
                                 both measured and extrapolated (geometric tail) */
    int32_t check_every;      /* window length M in sweeps (rounded up to even) */
    int64_t max_iter;         /* sweep limit per drive */
    int32_t precision;        /* PM_FP32_RED64, PM_FP32_DC64 or PM_FP64 */
    double dt_safety;         /* pseudo-time step = dt_safety x stability root (0.9) */
    double Re;                /* Reynolds number (Sec. 4: 0.01) */
    double c2;                /* squared artificial speed of sound (Sec. 4: 1.5e6).  The
                                 converged k does not depend on it, the number of
                                 iterations does: long thin cells converge faster with a
                                 larger value, compact packs with a smaller one */
    int32_t use_graph;        /* 1: replay each window as a captured CUDA graph */
    int32_t check_percolation;/* 1: percolation search before solving (device union-find
                                 of the pore cells, winding search on the host over the
                                 components that meet at the periodic faces) */
    double dc_switch_tol;     /* PM_FP32_DC64: leave plain FP32 sweeps at this change */
    int32_t dc_max_rounds;    /* PM_FP32_DC64: maximum correction rounds */
    int32_t kernel;           /* 0 = default sweep kernel, 1 = simple reference kernel */
    int32_t autotune;         /* 1: time the tiled kernel's tile shapes and work splits on
                                 the first sweeps of the first solve of a shape and keep the
                                 fastest (those sweeps are iterations of the solve and are
                                 counted); cached per device, precision and sweep variant */
    int32_t schedule;         /* tiled kernel's work split: 0 = automatic (the autotuner's
                                 choice when autotune is set, else persistent CTAs),
                                 -1 = persistent CTAs, n > 0 = one CTA per tile column
                                 and chunk of n planes (a pinned n keeps every chunk whole;
                                 the autotuner may also cut each column's last chunk into
                                 shorter pieces, reported in pm_stats.schedule_split) */
    int32_t tile;             /* tiled kernel's tile shape: 0 = automatic (the autotuner's
                                 choice when autotune is set, else 1); 1 = 64 x 12 cells,
                                 two per thread; 2 = 64 x 12, four per thread; 3 = 64 x 8,
                                 four per thread (FP32 fields; FP64 fields always use 1).
                                 Every shape gives the same fields, bit for bit.  (The
                                 transposed sweep of adjoint solves has its own shape,
                                 reported as 4.) */
    int32_t sequence;         /* pm_batch_ktensor: 0 = every (domain, drive) problem in each
                                 sweep launch; 1 = the domains in order, each starting from
                                 the converged fields of the previous one (same size) */
    int32_t field_memory;     /* where the ping-pong field buffers live: 0 = device memory;
                                 1 = the second buffer of each drive in pinned host memory,
                                 2 = both buffers there.  The kernels read and write host
                                 memory directly (over NVLink-C2C on a Grace CPU), so a
                                 domain whose fields do not fit device memory can be solved;
                                 device memory then holds the stencil codes and flags (5 B
                                 per cell) plus, with 1, one FP32 buffer (16 B per cell and
                                 drive).  Same fields, bit for bit; slower by the ratio of
                                 the link's bandwidth to the device memory's. */
    int32_t schedule_split;   /* with a pinned schedule n > 0: cut the last chunk of planes
                                 of every tile column into this many shorter pieces (0 or 1
                                 = none; at most 64).  Same fields, bit for bit. */
    int32_t dc_extrapolate;   /* PM_FP32_DC64: 1 = start the first correction solve from the
                                 geometric-tail estimate of the FP32 phase's remaining error
                                 (its change over the last window times r / (1 - r), r the
                                 window-to-window ratio of the mean-velocity change; 0 < r
                                 <= 0.98), 0 = from zero.  The rounds stop by the same test
                                 either way. */
    int32_t reserved[1];
} pm_options;

typedef struct pm_stats {
    int64_t iters;            /* pseudo-time iterations taken */
    double q[3];              /* mean velocity q_d (iteration units) at the end */
    double delta;             /* last window's relative change */
    double err_est;           /* extrapolated remaining change */
    double div_res;           /* L2 norm of the discrete divergence (iteration units) */
    double seconds;           /* wall time of the call */
    double sweep_ms;          /* CUDA-event time per sweep launch (mean over windows) */
    int64_t sweeps_timed;     /* sweeps inside the timed windows */
    int32_t dc_rounds;        /* defect-correction rounds done */
    int32_t status;           /* pm_status of this drive */
    int32_t percolates;       /* 1 if a fluid path wraps the domain along the drive */
    int32_t schedule;         /* tiled kernel's work split used (-1 persistent, n > 0 chunks
                                 of n planes; 0 = simple kernel or multi-geometry batch) */
    double setup_seconds;     /* wall time from the call's entry to its first sweep (mask
                                 ingest, neighbourhood, percolation, allocation) */
    int64_t n_fluid;          /* pore voxels of the domain */
    double sweep_ms_src;      /* as sweep_ms for the sweeps that carry a source term (the
                                 correction solves of PM_FP32_DC64); sweep_ms then covers
                                 the plain FP32 phase only */
    int64_t sweeps_timed_src; /* sweeps inside those timed windows */
    int64_t kernel_launches;  /* kernels launched by the call (a replayed window graph counts
                                 the kernels it holds) */
    int32_t tile;             /* tiled kernel's tile shape used (pm_options.tile numbering;
                                 0 = simple kernel) */
    int32_t schedule_split;   /* with schedule n > 0: the last chunk of planes of every tile
                                 column was cut into this many shorter pieces, so that the
                                 work units that start last fill the GPU's last wave of
                                 blocks (1 = not cut; 0 = no chunked schedule) */
} pm_stats;

/* Fills *opt with the defaults: tol 1e-6, check_every 200, max_iter 2e6,
 * PM_FP32_RED64, dt_safety 0.9, Re 0.01, c2 1.5e6, graphs on, percolation check on,
 * dc_switch_tol 1e-6, dc_max_rounds 8, autotune on, tile and schedule automatic, batch
 * mode. */
PM_API void pm_default_options(pm_options *opt);

/* Returns the scratch memory that the library's pool keeps between calls on the current
 * device to the driver (memory of calls still running stays).  Errors: PM_ERR_CUDA. */
PM_API int pm_release_memory(void);

/* Human-readable text of a pm_status (static storage). */
PM_API const char *pm_strerror(int status);

/* Library version, major * 10000 + minor * 100 + patch. */
PM_API int pm_version(void);

/* Pseudo-time step used for given options (the paper does not state one): dt_safety x
 * the positive root of 12 c2 dt^2 + 40 dt / Re - 4 = 0. */
PM_API double pm_time_step(const pm_options *opt);

/* Advance n pseudo-time iterations of Algorithm 1 in place, paper order (velocity update
 * from the old state, then pressure update with the new velocities), drive = body force
 * f on the fluid faces normal to axis dir (iteration units, Sec. 4).
 *   u: device, 3*N values, p: device, N values; float for PM_FP32_*, double for PM_FP64.
 *   Values on non-fluid faces / solid cells are set to 0 on entry.
 *   With a PM_BC_PRESSURE axis, dir must be that axis; drive sets p_in - p_out =
 *   drive x (n_axis - 1) (no body force) and the reservoir cells of p hold p_in / p_out.
 *   Errors: PM_ERR_INVALID_ARG, PM_ERR_OOM, PM_ERR_CUDA. */
PM_API int pm_iterate(const pm_domain *dom, int dir, double drive, const pm_options *opt, int64_t n,
               void *u, void *p, void *cuda_stream);

/* pm_iterate without any device memory allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc -- for example code running
 * under another allocator that has already reserved the GPU's memory (a framework's
 * caching allocator), or a latency-critical loop in which cudaMalloc / cudaFree would
 * synchronise the device.
 *   Same arguments, units and results as pm_iterate (the same kernels with the same work
 *   split: opt->kernel and opt->schedule are honoured, opt->autotune is ignored -- a
 *   schedule of 0 means persistent CTAs); u and p are updated in place.
 *   u and p must start on 16-byte boundaries (they are one buffer of the ping-pong pair).
 *   Errors as pm_iterate, and: PM_ERR_TOO_LARGE above nx * ny * nz = 131072 cells (e.g.
 *   64 x 64 x 32); PM_ERR_UNSUPPORTED for a PM_BC_PRESSURE axis (pm_iterate takes it);
 *   PM_ERR_INVALID_ARG for u or p off a 16-byte boundary.
 *   Scratch: a fixed 5 MB device array inside the library (a copy of the mask, the
 *   neighbourhood codes and the second field buffer).  Every GPU that loads the library
 *   holds it until the process exits.  The first call on a device looks up its device
 *   address (cudaGetSymbolAddress) with that device current; make that first call before
 *   any stream capture.
 *   All calls share the one array: calls whose work overlaps on the GPU (other streams,
 *   other host threads) race and corrupt each other; serialise them.  Each call
 *   rewrites every scratch value it reads, so nothing carries over between calls.
 *   The call runs on cuda_stream itself and returns after it has finished. */
PM_API int pm_iterate_noalloc(const pm_domain *dom, int dir, double drive, const pm_options *opt, int64_t n,
                              void *u, void *p, void *cuda_stream);

/* One drive direction to convergence (Algorithm 1, Sec. 4 "Permeability computation").
 *   dir: 0, 1, 2 = drive along e_1, e_2, e_3 (case a, b, c of Eq. cases_pressure).
 *   drive: |h| (pressure gradient magnitude, e.g. Pa/m); scales the returned fields.
 *   u (device, 3N floats) / p (device, N floats): Darcy-scaled fields out, or NULL.
 *   u0 / p0 (device, same layout and units as u / p): warm start, or NULL for zero.
 *   k_col (host, 3 doubles, may be NULL): column dir of k (Appendix C), dx^2 units.
 *   st (host, may be NULL): statistics.
 *   With a PM_BC_PRESSURE axis (dir must be that axis): the superficial velocities are the
 *   mean flux per face plane between the layers (q_dir n / (n - 1)) and the mean of the
 *   cross components over the n - 2 interior layers (q_i n / (n - 2)); p includes the
 *   fixed reservoir pressures.  PM_FP32_DC64 is not supported there (PM_ERR_UNSUPPORTED).
 *   Errors: PM_ERR_INVALID_ARG, PM_ERR_NO_FLUID, PM_ERR_NOT_PERCOLATING (k_col = 0),
 *   PM_ERR_NOT_CONVERGED, PM_ERR_DIVERGED, PM_ERR_UNSUPPORTED, PM_ERR_OOM, PM_ERR_CUDA. */
PM_API int pm_solve_direction(const pm_domain *dom, int dir, double drive, const pm_options *opt,
                       float *u, float *p, const float *u0, const float *p0, double *k_col,
                       pm_stats *st, void *cuda_stream);

/* Full tensor: the three drives of Eq. (cases_pressure) solved together, batched in each
 * sweep launch over the shared mask; k from the nine Darcy equations of Appendix C.
 *   k_out (host, 9 doubles, row-major): symmetrised k_ij = (k_ij + k_ji) / 2.
 *   k_raw (host, 9 doubles or NULL): column j from drive j before averaging.
 *   st (host, 3 entries or NULL): per drive statistics.
 *   A non-percolating axis gives a zero row and column and PM_ERR_NOT_PERCOLATING.
 *   Other errors as pm_solve_direction. */
PM_API int pm_permeability_tensor(const pm_domain *dom, double drive, const pm_options *opt,
                           double k_out[9], double k_raw[9], pm_stats st[3], void *cuda_stream);

/* Permeability tensors of many geometries in one solve (e.g. the images of a clogging
 * sequence, Sec. 7.3, and cropped sub-domains of uneven sizes): every (domain, drive)
 * problem of Eq. (cases_pressure) is a member of each sweep launch, the windows run as one
 * captured CUDA graph, and each problem stops sweeping when its criterion holds.  Problems
 * are processed in groups of up to 64.  With opt->sequence = 1 the domains are solved one
 * after another instead (their drives batched), each starting from the converged fields of
 * the previous domain when the two have the same size.
 *   doms: host array of n_domains domains sharing the boundary conditions (else
 *   PM_ERR_UNSUPPORTED).  An x extent that is not a multiple of 4 is handled inside: a
 *   periodic x axis is repeated 2 or 4 times (the same discrete problem), a wall x axis
 *   padded with solid columns; a thin domain (nz <= 16 and ny >= 8 nz) is solved with its
 *   y and z axes exchanged (the kernel then marches along the long axis; the stencils are
 *   the same along every axis).  k and the statistics refer to the domain as given.
 *   drives: host, n_domains bit masks (bit j = drive along e_(j+1)), or NULL / 0 for all.
 *   k_out: host, 9 doubles per domain (row-major, symmetrised); k_raw: same, unsymmetrised,
 *   or NULL.  st: host, 3 pm_stats per domain (per drive), or NULL.
 *   Non-percolating or unrequested drives leave zero columns (PM_ERR_NOT_PERCOLATING is
 *   returned if any requested drive does not percolate; the rest is computed).
 *   Precision PM_FP32_RED64 or PM_FP64. */
PM_API int pm_batch_ktensor(int n_domains, const pm_domain *doms, const int32_t *drives, const pm_options *opt,
                            double *k_out, double *k_raw, pm_stats *st, void *cuda_stream);

/* Adjoint sensitivity of J = sum_ij w_ij k_ij to a per-cell drag field alpha (not in the
 * paper: the steady momentum equation of Sec. 3 / 4 gains -(1/Re) alpha_f u with the face
 * value alpha_f = (alpha(c) + alpha(c+e_d)) / 2, alpha in units of mu / dx^2; alpha = 0 is
 * the paper's problem).  Forward solves for every drive j with a nonzero column of w,
 * solves of the transposed system (viscous operator transposed) for every row i, then
 *   dJ/d alpha_c = -(dx^2 / (2 Re^2 N)) sum_ij w_ij sum_{faces F of c} v^(i)_F u^(j)_F
 * (u^(j), v^(i) in iteration units for a unit drive).  FP32 fields run the transposed
 * solves on the tiled kernel (four cells per thread); FP64 fields on the simple kernel.
 *   alpha: device, N floats, or NULL for 0.      w: host, 9 doubles, row-major.
 *   dJ_dalpha: device, N floats, caller-owned, written for every cell (dx^2 units of k);
 *   NULL: forward only -- the drives of the nonzero columns of w (all three when w is
 *   NULL) are solved with alpha, and J and k_raw are returned.
 *   J (host, may be NULL): the objective.  k_raw (host, 9 or NULL): the forward columns.
 *   u_fwd (host array of 3 device pointers, or NULL; NULL entries allowed): the forward
 *   velocity fields u^(j) = [u_x | u_y | u_z] of drive j, 3N values in iteration units for
 *   a unit drive (float for PM_FP32_RED64, double for PM_FP64).  fwd_given = 0: each
 *   non-NULL entry of a solved drive receives its converged field.  fwd_given = 1: the
 *   non-NULL entries hold converged fields from an earlier call on the same mask, alpha and
 *   options (for example the forward pass of an autograd function), those drives are not
 *   solved again and their k columns come from the given fields.
 *   Precision PM_FP32_RED64 or PM_FP64 (PM_FP32_DC64: PM_ERR_UNSUPPORTED).
 *   Errors: PM_ERR_INVALID_ARG (w all zero, or dJ_dalpha without w), PM_ERR_NO_FLUID, PM_ERR_NOT_CONVERGED,
 *   PM_ERR_DIVERGED, PM_ERR_OOM, PM_ERR_CUDA. */
PM_API int pm_sensitivity(const pm_domain *dom, const float *alpha, const double w[9], const pm_options *opt,
                          float *dJ_dalpha, double *J, double k_raw[9], void *const u_fwd[3], int32_t fwd_given,
                          void *cuda_stream);

/* Pre-processing (Sec. 5 "Processing input data": mirroring for symmetric periodicity).
 * Writes the mask followed by its mirror image along every axis whose bit is set in axes
 * (bit 0 = x, 1 = y, 2 = z), so that the doubled domain is periodic and symmetric under
 * the reflection (its k has no coupling between a mirrored axis and the others).
 *   mask: nx*ny*nz bytes [nz][ny][nx]; out: (nx << mx)(ny << my)(nz << mz) bytes, caller-
 *   owned, same layout; both host memory (on_device = 0, a plain loop on the host) or both
 *   device memory (on_device = 1, one kernel on cuda_stream, returns after it finished).
 *   Errors: PM_ERR_INVALID_ARG (NULL, sizes < 1, axes outside 0..7), PM_ERR_CUDA. */
PM_API int pm_mirror_mask(const uint8_t *mask, int32_t nx, int32_t ny, int32_t nz, int32_t axes,
                          int32_t on_device, uint8_t *out, void *cuda_stream);

/* Pre-processing (Sec. 5: elimination of disconnected pore spaces; host only).  Copies the
 * mask to out and turns solid every face-connected component of pore cells that carries
 * no flow through the domain: one that wraps around no periodic axis and does not join
 * the first and the last layer of a PM_BC_PRESSURE axis (wall axes connect nothing).  Such
 * pores hold u = 0 at the fixed point, so k is unchanged; the iteration loses unknowns.
 *   mask, out: host, nx*ny*nz bytes [nz][ny][nx] (may be the same buffer).
 *   bc: per axis PM_BC_*.  removed (may be NULL): number of pore cells turned solid.
 *   Errors: PM_ERR_INVALID_ARG. */
PM_API int pm_remove_isolated_pores(const uint8_t *mask, int32_t nx, int32_t ny, int32_t nz, const int32_t bc[3],
                                    uint8_t *out, int64_t *removed);

/* Spectral form of a permeability tensor (Sec. 2, Eq. 3dK_eigen): principal permeabilities
 * lambda (ascending) and principal axes, from the symmetric part of k (host only, no GPU).
 *   k: host, 9 doubles, row-major.  lambda: host, 3 doubles out.
 *   axes: host, 9 doubles out, or NULL; column j (axes[3*i + j], i = 0..2) is the unit
 *   principal axis of lambda[j], signed so that its largest-magnitude component is positive
 *   (the rotation tensor R of Sec. 2 up to the order and signs of its columns).
 *   Cyclic Jacobi rotations to machine precision.
 *   Errors: PM_ERR_INVALID_ARG (NULL or non-finite input). */
PM_API int pm_principal_axes(const double k[9], double lambda[3], double axes[9]);

/* Material class of Sec. 2 from the principal permeabilities: 0 isotropy (all three equal),
 * 1 transverse anisotropy (exactly two equal), 2 orthotropy (all different); two values
 * count as equal when they differ by at most rel_tol x the largest |lambda|.
 * Returns the class, or -1 for NULL / non-finite input or rel_tol < 0. */
PM_API int pm_anisotropy_class(const double lambda[3], double rel_tol);

#ifdef __cplusplus
}
#endif
#endif /* POREMAPS_GB_H */
