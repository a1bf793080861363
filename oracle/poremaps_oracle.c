/*
 * Plain FP64 CPU oracle of the POREMAPS pseudo-unsteady Stokes permeability method
 * (Krach, Ruf, Steeb, "POREMAPS: A finite difference based Porous Media Anisotropic
 * Permeability Solver for Stokes flow", arXiv 2407.19868).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct reference that
 * the CUDA library is checked against.  Only the test suite, the package smoke check
 * and the benchmark's CPU-baseline / reference legs may build or call it.  It shares
 * no code, header, table or helper with the CUDA library.
 *
 * What it computes, in the paper's order (Algorithm 1):
 *   - "Evaluate neighborhood": for every face-velocity node and each direction
 *     perpendicular to it, the wall case 1..6 of Appendix B (Fig. neighborhoodCases).
 *   - loop: "Compute velocity field" (explicit pseudo-time step of the momentum
 *     equation, Sec. 3 and Sec. 4), then "Compute pressure field" from the NEW
 *     velocities (artificial compressibility, Sec. 3), then "Evaluate permeability
 *     and convergence criterion" (Darcy, Eq. darcy, Appendix C).
 *
 * Discretisation (Sec. 4, "Grid" and "Boundary ..."): MAC grid, pressure p at cell
 * centres, velocity component u_d on the +d face of each cell.  Cell c is solid iff
 * its mask byte is nonzero.  A velocity node u_d(c) is fluid iff both cells it
 * separates (c and c+e_d) are fluid; every other node is a no-penetration face and
 * holds exactly 0.  Outer boundaries per axis: periodic, or a no-slip wall (cells
 * outside the box count as solid).
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   - the driving pressure gradient h along e_j is applied as a uniform body force f
 *     on the fluid j-faces with a periodic pressure fluctuation; this equals the
 *     paper's pressure ramp with a periodic jump exactly on the discrete grid;
 *   - the second derivative ALONG the flow direction is the 3-point stencil, a
 *     non-fluid neighbour contributing 0 (it is a no-penetration face at distance 1);
 *   - a non-fluid node at +-1 perpendicular to the flow is read as a no-slip wall
 *     half a spacing away (Appendix B, first equation of each system);
 *   - cases 7/8 (4b/5b) are only needed at MPI halo layers; on one periodic domain the
 *     +-2 neighbour always exists, so classification uses cases 1..6 only; the
 *     coefficients of 7/8 are still provided for the tests.
 *   - optional per-cell drag alpha (not in the paper; alpha = 0 is the paper): the
 *     momentum residual gains -(1/Re) * alpha_f * u with alpha_f = (alpha(c) +
 *     alpha(c+e_d)) / 2 on the face.
 *   - fixed-pressure inlet/outlet (Sec. 4 names a fixed pressure in the main flow
 *     direction only in words; one axis a at most): the first and the last cell layer
 *     along a are pressure reservoirs.  Their pressures are fixed (p_in, p_out), they
 *     hold no velocity across a (their u_b, b != a, are non-fluid), and outside the box
 *     along a counts as solid.  The n_a - 1 face planes u_a(0) .. u_a(n_a - 2) between
 *     the layers carry the flow; at the inlet face u_a(0) and the outlet face
 *     u_a(n_a - 2) the missing axial neighbour takes the face's own value (zero
 *     gradient).  No body force: the drive h gives p_in - p_out = h (n_a - 1).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PERIODIC 0
#define OR_WALL 1
#define OR_PRESSURE 2
#define OR_MAXOFF 4 /* neighbour offsets -4..4 are tabulated per axis */

typedef struct {
    int64_t n[3];          /* nx, ny, nz; x fastest */
    int64_t N;
    int32_t bc[3];
    int pax;               /* fixed-pressure axis, -1 if none */
    uint8_t *solid;        /* copy of the input mask */
    uint8_t *cell_fluid;   /* [N] */
    uint8_t *node_fluid;   /* [3][N] */
    uint8_t *perp_case;    /* [3][3][N]: case of node u_d(c) along axis i (i != d); 0 = not fluid */
    int64_t *wrap[3];      /* wrap[a][(m + OR_MAXOFF) * n[a] + x]: coordinate x + m on axis a, -1 outside */
} or_ctx;

typedef struct {
    double Re;             /* Reynolds number; the viscous term carries 1/Re (Sec. 3) */
    double c2;             /* squared artificial speed of sound c*^2 (Sec. 3) */
    double dt;             /* pseudo-time step */
    double f[3];           /* body force on the d-faces (the drive) */
    const double *alpha;   /* per-cell drag, may be NULL */
    int32_t transposed;    /* 1: use the transpose of the viscous operator (adjoint) */
    double p_res[2];       /* fixed-pressure axis: reservoir pressures p_in, p_out */
} or_params;

/* ---------------------------------------------------------------- geometry */

static inline int64_t or_index(const or_ctx *g, int64_t x, int64_t y, int64_t z) {
    return x + g->n[0] * (y + g->n[1] * z);
}

/* Linear index of the cell at offset m along axis a from cell (x,y,z); -1 if it lies
 * outside a wall axis. */
static inline int64_t or_nb(const or_ctx *g, int64_t x, int64_t y, int64_t z, int a, int m) {
    const int64_t nx = g->n[0], ny = g->n[1], nz = g->n[2];
    int64_t v;
    switch (a) {
    case 0:
        v = g->wrap[0][(int64_t)(m + OR_MAXOFF) * nx + x];
        return v < 0 ? -1 : v + nx * (y + ny * z);
    case 1:
        v = g->wrap[1][(int64_t)(m + OR_MAXOFF) * ny + y];
        return v < 0 ? -1 : x + nx * (v + ny * z);
    default:
        v = g->wrap[2][(int64_t)(m + OR_MAXOFF) * nz + z];
        return v < 0 ? -1 : x + nx * (y + ny * v);
    }
}

static inline void or_coords(const or_ctx *g, int64_t c, int64_t *x, int64_t *y, int64_t *z) {
    *x = c % g->n[0];
    int64_t r = c / g->n[0];
    *y = r % g->n[1];
    *z = r / g->n[1];
}

/* Layer of cell (x,y,z) along the fixed-pressure axis: 0 = inlet reservoir, 1 = outlet
 * reservoir, -1 = interior (or no such axis). */
static inline int or_reservoir(const or_ctx *g, int64_t x, int64_t y, int64_t z) {
    if (g->pax < 0) return -1;
    const int64_t v = g->pax == 0 ? x : (g->pax == 1 ? y : z);
    return v == 0 ? 0 : (v == g->n[g->pax] - 1 ? 1 : -1);
}

/* Pressure of cell c: the fixed reservoir value in a reservoir layer, else p[c]. */
static inline double or_p(const or_ctx *g, const or_params *P, const double *p, int64_t c) {
    int64_t x, y, z;
    or_coords(g, c, &x, &y, &z);
    const int r = or_reservoir(g, x, y, z);
    return r < 0 ? p[c] : P->p_res[r];
}

/* Appendix B / Fig. neighborhoodCases: case of a fluid node from the fluid flags of
 * the nodes at offsets -2, -1, +1, +2 along a perpendicular axis. */
int or_classify(int Fm2, int Fm1, int Fp1, int Fp2) {
    if (!Fm1 && !Fp1) return 1;           /* walls at -1/2 and +1/2 */
    if (!Fm1 && Fp1) return Fp2 ? 4 : 2;  /* wall at -1/2 */
    if (Fm1 && !Fp1) return Fm2 ? 5 : 3;  /* wall at +1/2 */
    return 6;                             /* interior */
}

/* Appendix B: coefficients of the perpendicular second derivative of case k for the
 * node values at offsets -2..+2 (columns 0..4).  Row 0 = not a fluid node. */
static const double OR_COEF[9][5] = {
    {0.0, 0.0, 0.0, 0.0, 0.0},
    {0.0, 0.0, -8.0, 0.0, 0.0},                       /* 1: walls at -1/2 and +1/2 */
    {0.0, 0.0, -16.0 / 3.0, 8.0 / 3.0, 0.0},          /* 2: wall at -1/2, no node at +2 */
    {0.0, 8.0 / 3.0, -16.0 / 3.0, 0.0, 0.0},          /* 3: wall at +1/2, no node at -2 */
    {0.0, 0.0, -5.0, 2.0, -1.0 / 5.0},                /* 4: wall at -1/2 */
    {-1.0 / 5.0, 2.0, -5.0, 0.0, 0.0},                /* 5: wall at +1/2 */
    {0.0, 1.0, -2.0, 1.0, 0.0},                       /* 6: interior */
    {0.0, 0.0, -4.0, 4.0 / 3.0, 0.0},                 /* 7 (4b) */
    {0.0, 4.0 / 3.0, -4.0, 0.0, 0.0},                 /* 8 (5b) */
};

void or_case_coeffs(int k, double c[5]) {
    for (int i = 0; i < 5; ++i) c[i] = (k >= 0 && k <= 8) ? OR_COEF[k][i] : 0.0;
}

void or_ctx_destroy(or_ctx *g) {
    if (!g) return;
    free(g->solid);
    free(g->cell_fluid);
    free(g->node_fluid);
    free(g->perp_case);
    for (int a = 0; a < 3; ++a) free(g->wrap[a]);
    free(g);
}

/* Builds the context and runs "Evaluate neighborhood" (Algorithm 1). */
or_ctx *or_ctx_create(int64_t nx, int64_t ny, int64_t nz, const int32_t bc[3], const uint8_t *mask) {
    or_ctx *g = (or_ctx *)calloc(1, sizeof(or_ctx));
    if (!g) return NULL;
    g->n[0] = nx; g->n[1] = ny; g->n[2] = nz;
    g->N = nx * ny * nz;
    g->pax = -1;
    for (int a = 0; a < 3; ++a) {
        g->bc[a] = bc[a];
        if (bc[a] == OR_PRESSURE && g->pax < 0) g->pax = a;
    }
    int64_t N = g->N;
    g->solid = (uint8_t *)malloc((size_t)N);
    g->cell_fluid = (uint8_t *)malloc((size_t)N);
    g->node_fluid = (uint8_t *)calloc((size_t)(3 * N), 1);
    g->perp_case = (uint8_t *)calloc((size_t)(9 * N), 1);
    int ok = g->solid && g->cell_fluid && g->node_fluid && g->perp_case;
    for (int a = 0; a < 3 && ok; ++a) {
        int64_t n = g->n[a];
        g->wrap[a] = (int64_t *)malloc(sizeof(int64_t) * (size_t)((2 * OR_MAXOFF + 1) * n));
        if (!g->wrap[a]) { ok = 0; break; }
        for (int m = -OR_MAXOFF; m <= OR_MAXOFF; ++m)
            for (int64_t x = 0; x < n; ++x) {
                int64_t v = x + m;
                if (bc[a] == OR_PERIODIC) v = ((v % n) + n) % n;
                else if (v < 0 || v >= n) v = -1;
                g->wrap[a][(int64_t)(m + OR_MAXOFF) * n + x] = v;
            }
    }
    if (!ok) { or_ctx_destroy(g); return NULL; }
    memcpy(g->solid, mask, (size_t)N);
    for (int64_t c = 0; c < N; ++c) g->cell_fluid[c] = mask[c] ? 0 : 1;

    #pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < N; ++c) {
        int64_t x, y, z;
        or_coords(g, c, &x, &y, &z);
        const int res = or_reservoir(g, x, y, z);
        for (int d = 0; d < 3; ++d) {
            int64_t cp = or_nb(g, x, y, z, d, +1);
            g->node_fluid[d * N + c] = (g->cell_fluid[c] && cp >= 0 && g->cell_fluid[cp]) ? 1 : 0;
            if (res >= 0 && d != g->pax) g->node_fluid[d * N + c] = 0;  /* reservoirs carry no cross flow */
        }
    }
    #pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < N; ++c) {
        int64_t x, y, z;
        or_coords(g, c, &x, &y, &z);
        for (int d = 0; d < 3; ++d) {
            if (!g->node_fluid[d * N + c]) continue;
            for (int i = 0; i < 3; ++i) {
                if (i == d) continue;
                int F[5];
                for (int m = -2; m <= 2; ++m) {
                    if (m == 0) continue;
                    int64_t b = or_nb(g, x, y, z, i, m);
                    F[m + 2] = (b >= 0) ? g->node_fluid[d * N + b] : 0;
                }
                g->perp_case[(d * 3 + i) * N + c] = (uint8_t)or_classify(F[0], F[1], F[3], F[4]);
            }
        }
    }
    return g;
}

int64_t or_ctx_size(const or_ctx *g) { return g->N; }

void or_ctx_tables(const or_ctx *g, uint8_t *node_fluid, uint8_t *perp_case) {
    if (node_fluid) memcpy(node_fluid, g->node_fluid, (size_t)(3 * g->N));
    if (perp_case) memcpy(perp_case, g->perp_case, (size_t)(9 * g->N));
}

/* ---------------------------------------------------------------- operators */

/* Value of velocity component d at cell index b (-1 = outside); non-fluid nodes are 0. */
static inline double or_u(const or_ctx *g, const double *U, int d, int64_t b) {
    return (b >= 0 && g->node_fluid[d * g->N + b]) ? U[d * g->N + b] : 0.0;
}

/* Steady momentum residual (Sec. 3, Sec. 4) at every node:
 *   R_d(c) = (1/Re) [ A_d u + sum_{i != d} S_i u - alpha_f u ](c) - (p(c+e_d) - p(c)) + f_d
 * on fluid nodes and 0 on the others.  U = [ux | uy | uz], each N long. */
void or_momentum_residual(const or_ctx *g, const or_params *P, const double *U, const double *p, double *R) {
    const int64_t N = g->N, nx = g->n[0], ny = g->n[1], nz = g->n[2];
    const double inv_re = 1.0 / P->Re;
    const uint8_t *node_fluid = g->node_fluid, *perp_case = g->perp_case;
    for (int d = 0; d < 3; ++d) {
        const double *Ud = U + d * N;
        double *Rd = R + d * N;
        const uint8_t *nf = node_fluid + d * N;
        #pragma omp parallel for collapse(2) schedule(static)
        for (int64_t z = 0; z < nz; ++z)
            for (int64_t y = 0; y < ny; ++y)
                for (int64_t x = 0; x < nx; ++x) {
                    const int64_t c = or_index(g, x, y, z);
                    if (!nf[c]) { Rd[c] = 0.0; continue; }
                    const double u0 = Ud[c];
                    const int64_t cp = or_nb(g, x, y, z, d, +1);
                    const int64_t cm = or_nb(g, x, y, z, d, -1);
                    /* along the flow direction: 3-point second difference; a non-fluid
                     * neighbour (or one outside a wall) contributes 0 */
                    double up = (cp >= 0 && nf[cp]) ? Ud[cp] : 0.0, um = (cm >= 0 && nf[cm]) ? Ud[cm] : 0.0;
                    if (d == g->pax) {
                        /* inlet / outlet face: zero-gradient axial neighbour */
                        const int64_t v = d == 0 ? x : (d == 1 ? y : z);
                        if (v == 0) um = u0;
                        if (v == g->n[d] - 2) up = u0;
                    }
                    double lap = up - 2.0 * u0 + um;
                    for (int i = 0; i < 3; ++i) {
                        if (i == d) continue;
                        if (!P->transposed) {
                            const double *co = OR_COEF[perp_case[(d * 3 + i) * N + c]];
                            /* a nonzero coefficient only ever points at a fluid node */
                            for (int m = -2; m <= 2; ++m)
                                if (co[m + 2] != 0.0) lap += co[m + 2] * Ud[or_nb(g, x, y, z, i, m)];
                        } else {
                            /* transpose: node b = c - m e_i applies its coefficient for offset m to c */
                            for (int m = -2; m <= 2; ++m) {
                                const int64_t b = or_nb(g, x, y, z, i, -m);
                                if (b < 0 || !nf[b]) continue;
                                lap += OR_COEF[perp_case[(d * 3 + i) * N + b]][m + 2] * Ud[b];
                            }
                        }
                    }
                    if (P->alpha) lap -= 0.5 * (P->alpha[c] + P->alpha[cp]) * u0;
                    Rd[c] = inv_re * lap - (or_p(g, P, p, cp) - or_p(g, P, p, c)) + P->f[d];
                }
    }
}

/* Discrete divergence on fluid cells: D u(c) = sum_d u_d(c) - u_d(c - e_d); 0 on solid cells. */
void or_divergence(const or_ctx *g, const double *U, double *div) {
    const int64_t nx = g->n[0], ny = g->n[1], nz = g->n[2];
    #pragma omp parallel for collapse(2) schedule(static)
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) {
                const int64_t c = or_index(g, x, y, z);
                if (!g->cell_fluid[c] || or_reservoir(g, x, y, z) >= 0) { div[c] = 0.0; continue; }
                double s = 0.0;
                for (int d = 0; d < 3; ++d) s += or_u(g, U, d, c) - or_u(g, U, d, or_nb(g, x, y, z, d, -1));
                div[c] = s;
            }
}

/* Algorithm 1, loop body, n times: velocity update from the old state, then the
 * pressure update from the NEW velocities (p <- p - dt c^2 div u). */
void or_iterate(const or_ctx *g, const or_params *P, double *U, double *p, int64_t n_iter) {
    const int64_t N = g->N;
    double *R = (double *)malloc(sizeof(double) * (size_t)(3 * N));
    double *div = (double *)malloc(sizeof(double) * (size_t)N);
    for (int64_t it = 0; it < n_iter; ++it) {
        or_momentum_residual(g, P, U, p, R);
        #pragma omp parallel for schedule(static)
        for (int64_t k = 0; k < 3 * N; ++k) U[k] += P->dt * R[k];
        or_divergence(g, U, div);
        #pragma omp parallel for schedule(static)
        for (int64_t c = 0; c < N; ++c) {
            if (!g->cell_fluid[c]) continue;
            /* reservoir cells keep their fixed pressure; div is 0 there */
            p[c] = or_p(g, P, p, c) - P->dt * P->c2 * div[c];
        }
    }
    free(R);
    free(div);
}

/* Superficial (Darcy) velocity q_d = (1/N) sum over all cells of u_d, summed per
 * z-plane and then over planes in a fixed order (deterministic). */
void or_mean_velocity(const or_ctx *g, const double *U, double q[3]) {
    const int64_t N = g->N, nz = g->n[2], plane = g->n[0] * g->n[1];
    double *part = (double *)calloc((size_t)(3 * nz), sizeof(double));
    #pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < nz; ++z)
        for (int d = 0; d < 3; ++d) {
            double s = 0.0;
            for (int64_t k = 0; k < plane; ++k) s += U[d * N + z * plane + k];
            part[d * nz + z] = s;
        }
    for (int d = 0; d < 3; ++d) {
        double s = 0.0;
        for (int64_t z = 0; z < nz; ++z) s += part[d * nz + z];
        q[d] = s / (double)N;
    }
    free(part);
}

/* Iterate until the relative change of the mean velocity over a window of
 * `check_every` iterations, extrapolated as a geometric tail, is below tol
 * (reading of the criterion eps = delta|q| / |q| of Sec. 7.1).
 * info[0] = last window change delta, info[1] = estimated remaining change,
 * info[2] = L2 norm of the divergence.  Returns the iteration count, or -n if
 * max_iter was reached first. */
int64_t or_solve(const or_ctx *g, const or_params *P, int dir, double tol, int64_t check_every,
                 int64_t max_iter, double *U, double *p, double q[3], double info[3]) {
    double qp[3], qn[3];
    or_mean_velocity(g, U, qp);
    double d_prev = -1.0, delta = INFINITY, err = INFINITY;
    int64_t it = 0;
    int conv = 0;
    while (it < max_iter) {
        or_iterate(g, P, U, p, check_every);
        it += check_every;
        or_mean_velocity(g, U, qn);
        double ref = fabs(qn[dir]);
        double ch = 0.0;
        for (int d = 0; d < 3; ++d) ch = fmax(ch, fabs(qn[d] - qp[d]));
        delta = ref > 0.0 ? ch / ref : INFINITY;
        if (ch == 0.0) err = 0.0;
        else if (d_prev > 0.0 && delta < d_prev) {
            double r = delta / d_prev;
            err = delta * r / (1.0 - r);
        } else err = INFINITY;
        d_prev = delta;
        memcpy(qp, qn, sizeof qp);
        if (!isfinite(qn[0]) || !isfinite(qn[1]) || !isfinite(qn[2])) break;
        if (delta < tol && err < tol) { conv = 1; break; }
    }
    memcpy(q, qn, sizeof qn);
    double *div = (double *)malloc(sizeof(double) * (size_t)g->N);
    or_divergence(g, U, div);
    double s = 0.0;
    for (int64_t c = 0; c < g->N; ++c) s += div[c] * div[c];
    free(div);
    info[0] = delta;
    info[1] = err;
    info[2] = sqrt(s);
    return conv ? it : -it;
}

/* Percolation (Sec. 5.1 assumes it; the precipitation series loses it): breadth-first
 * search over face-connected fluid cells that records, for each visited cell, how often
 * the path to it crossed each periodic boundary.  Reaching a visited cell with a
 * different crossing count along axis a means a fluid loop that wraps around the
 * domain along a, i.e. flow along a is possible. */
void or_percolation(const or_ctx *g, int32_t out[3]) {
    const int64_t N = g->N;
    out[0] = out[1] = out[2] = 0;
    int16_t *w = (int16_t *)malloc(sizeof(int16_t) * (size_t)(3 * N));
    uint8_t *vis = (uint8_t *)calloc((size_t)N, 1);
    int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    for (int64_t s0 = 0; s0 < N; ++s0) {
        if (!g->cell_fluid[s0] || vis[s0]) continue;
        int64_t head = 0, tail = 0;
        queue[tail++] = s0;
        vis[s0] = 1;
        w[s0] = w[N + s0] = w[2 * N + s0] = 0;
        while (head < tail) {
            int64_t c = queue[head++];
            int64_t co[3];
            or_coords(g, c, &co[0], &co[1], &co[2]);
            for (int a = 0; a < 3; ++a)
                for (int m = -1; m <= 1; m += 2) {
                    int64_t b = or_nb(g, co[0], co[1], co[2], a, m);
                    if (b < 0 || !g->cell_fluid[b]) continue;
                    int16_t wn[3] = {w[c], w[N + c], w[2 * N + c]};
                    int64_t raw = co[a] + m;
                    if (raw < 0) wn[a] -= 1;
                    else if (raw >= g->n[a]) wn[a] += 1;
                    if (!vis[b]) {
                        vis[b] = 1;
                        w[b] = wn[0]; w[N + b] = wn[1]; w[2 * N + b] = wn[2];
                        queue[tail++] = b;
                    } else {
                        for (int k = 0; k < 3; ++k)
                            if (w[k * N + b] != wn[k]) out[k] = 1;
                    }
                }
        }
    }
    if (g->pax >= 0) {
        /* fixed-pressure axis: a path of pore cells from the inlet reservoir layer to the
         * outlet one; reservoir cells carry no cross flow, so a path leaves a reservoir
         * only along the axis */
        const int a = g->pax;
        out[a] = 0;
        memset(vis, 0, (size_t)N);
        int64_t head = 0, tail = 0;
        for (int64_t c = 0; c < N; ++c) {
            int64_t x, y, z;
            or_coords(g, c, &x, &y, &z);
            if (g->cell_fluid[c] && or_reservoir(g, x, y, z) == 0) { vis[c] = 1; queue[tail++] = c; }
        }
        while (head < tail && !out[a]) {
            int64_t c = queue[head++];
            int64_t co[3];
            or_coords(g, c, &co[0], &co[1], &co[2]);
            const int rc = or_reservoir(g, co[0], co[1], co[2]);
            if (rc == 1) { out[a] = 1; break; }
            for (int ax = 0; ax < 3; ++ax)
                for (int m = -1; m <= 1; m += 2) {
                    if (rc == 0 && ax != a) continue;
                    int64_t b = or_nb(g, co[0], co[1], co[2], ax, m);
                    if (b < 0 || !g->cell_fluid[b] || vis[b]) continue;
                    vis[b] = 1;
                    queue[tail++] = b;
                }
        }
    }
    free(w);
    free(vis);
    free(queue);
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
