"""FP64 CPU oracle for the POREMAPS permeability method (arXiv 2407.19868).

TEST INFRASTRUCTURE ONLY: the slow reference the CUDA library is checked against.
Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline and
reference legs may import it.  It shares no code with the CUDA library; the two
meet only through the seeded input generators.

Each function names the passage of the paper it follows; the arithmetic lives in
``poremaps_oracle.c`` (plain loops, FP64), this module only marshals arrays.

Parity pins for every function are in ``tests/test_oracle_*.py``: closed forms
(slit Poiseuille, square ducts), the paper's printed Taylor systems (Appendix B),
a direct sparse solve of the steady system, rotation/shift/tiling invariance,
the tube (Hagen-Poiseuille) and Hasimoto sphere-array limits under refinement,
and, for the adjoint, the dot-product identity and finite differences.
"""
from __future__ import annotations

import ctypes as C
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "poremaps_oracle.c")
_LOCK = threading.Lock()
_LIB = None

PERIODIC = 0
WALL = 1
PRESSURE = 2  # fixed-pressure inlet/outlet reservoirs (first and last layer along the axis)

# Sec. 4, "Simulation parametrization": Re = 0.01, c*^2 = 1.5e6, grad p = 1 / vx.
RE_PAPER = 0.01
C2_PAPER = 1.5e6
DRIVE_PAPER = 1.0


def lib_path() -> str:
    return os.path.join(_HERE, "_build", f"liboracle_{platform.machine()}.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no FP contraction so that x86 and
    Arm give the same bits)."""
    out = lib_path()
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-std=c11", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


class _Params(C.Structure):
    _fields_ = [("Re", C.c_double), ("c2", C.c_double), ("dt", C.c_double),
                ("f", C.c_double * 3), ("alpha", C.POINTER(C.c_double)),
                ("transposed", C.c_int32), ("p_res", C.c_double * 2)]


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            L = C.CDLL(build())
            vp, i64, dp = C.c_void_p, C.c_int64, C.POINTER(C.c_double)
            L.or_ctx_create.restype = vp
            L.or_ctx_create.argtypes = [i64, i64, i64, C.POINTER(C.c_int32), C.POINTER(C.c_uint8)]
            L.or_ctx_destroy.argtypes = [vp]
            L.or_ctx_tables.argtypes = [vp, C.POINTER(C.c_uint8), C.POINTER(C.c_uint8)]
            L.or_classify.restype = C.c_int
            L.or_classify.argtypes = [C.c_int] * 4
            L.or_case_coeffs.argtypes = [C.c_int, dp]
            L.or_momentum_residual.argtypes = [vp, C.POINTER(_Params), dp, dp, dp]
            L.or_divergence.argtypes = [vp, dp, dp]
            L.or_iterate.argtypes = [vp, C.POINTER(_Params), dp, dp, i64]
            L.or_mean_velocity.argtypes = [vp, dp, dp]
            L.or_solve.restype = i64
            L.or_solve.argtypes = [vp, C.POINTER(_Params), C.c_int, C.c_double, i64, i64, dp, dp, dp, dp]
            L.or_percolation.argtypes = [vp, C.POINTER(C.c_int32)]
            L.or_num_threads.restype = C.c_int
            _LIB = L
    return _LIB


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def num_threads() -> int:
    return int(_lib().or_num_threads())


def classify(Fm2: int, Fm1: int, Fp1: int, Fp2: int) -> int:
    """Appendix B / Fig. neighborhoodCases: wall case from the fluid flags of the
    perpendicular neighbours at -2, -1, +1, +2."""
    return int(_lib().or_classify(int(Fm2), int(Fm1), int(Fp1), int(Fp2)))


def case_coeffs(k: int) -> np.ndarray:
    """Appendix B: perpendicular second-derivative coefficients of case k for the
    node values at offsets -2..+2."""
    c = np.zeros(5)
    _lib().or_case_coeffs(int(k), _dptr(c))
    return c


def default_dt(Re: float = RE_PAPER, c2: float = C2_PAPER, safety: float = 0.9) -> float:
    """Pseudo-time step (the paper does not state one): safety x the positive root of
    12 c^2 dt^2 + 40 dt / Re - 4 = 0, combining the acoustic bound of the
    velocity-then-pressure update (the cell Laplacian has eigenvalues <= 12) with the
    viscous Gershgorin bound (<= 20 / Re).  Only the speed depends on it."""
    a, b, c = 12.0 * c2, 40.0 / Re, -4.0
    return safety * (-b + np.sqrt(b * b - 4 * a * c)) / (2 * a)


class Domain:
    """A voxel geometry with its neighbourhood evaluated (Algorithm 1,
    "Evaluate neighborhood").  ``mask`` is uint8 [nz][ny][nx], nonzero = solid;
    ``bc`` per axis (x, y, z): PERIODIC, WALL or PRESSURE (one axis at most, at least 3
    cells: its first and last layer are the inlet and outlet reservoirs, Sec. 4)."""

    def __init__(self, mask: np.ndarray, bc=(PERIODIC, PERIODIC, PERIODIC)):
        m = np.ascontiguousarray(mask, dtype=np.uint8)
        if m.ndim != 3:
            raise ValueError("mask must be 3-D [nz][ny][nx]")
        self.mask = m
        self.shape = m.shape
        nz, ny, nx = m.shape
        self.N = m.size
        self.bc = tuple(int(b) for b in bc)
        pa = [a for a in range(3) if self.bc[a] == PRESSURE]
        if len(pa) > 1:
            raise ValueError("at most one fixed-pressure axis")
        self.pax = pa[0] if pa else None
        if self.pax is not None and (nx, ny, nz)[self.pax] < 3:
            raise ValueError("a fixed-pressure axis needs at least 3 cells")
        bca = (C.c_int32 * 3)(*self.bc)
        self._L = _lib()
        self._ctx = self._L.or_ctx_create(nx, ny, nz, bca, m.ctypes.data_as(C.POINTER(C.c_uint8)))
        if not self._ctx:
            raise MemoryError("oracle context")

    def __del__(self):
        if getattr(self, "_ctx", None):
            self._L.or_ctx_destroy(self._ctx)
            self._ctx = None

    # ------------------------------------------------------------ tables
    def tables(self):
        """(node_fluid [3, nz, ny, nx], perp_case [3, 3, nz, ny, nx])."""
        nf = np.zeros((3,) + self.shape, dtype=np.uint8)
        pc = np.zeros((3, 3) + self.shape, dtype=np.uint8)
        self._L.or_ctx_tables(self._ctx, nf.ctypes.data_as(C.POINTER(C.c_uint8)),
                              pc.ctypes.data_as(C.POINTER(C.c_uint8)))
        return nf, pc

    def _params(self, drive_dir, drive, Re, c2, dt, alpha, transposed):
        f = [0.0, 0.0, 0.0]
        pres = [0.0, 0.0]
        if self.pax is not None:
            # fixed-pressure drive: no body force, p_in - p_out = h (n_a - 1) around 0
            if drive_dir is not None and drive_dir != self.pax:
                raise ValueError("with a fixed-pressure axis the drive is along that axis")
            if transposed:
                raise ValueError("the transposed operator is not defined with fixed pressures")
            if drive_dir is not None:
                L = (self.shape[2], self.shape[1], self.shape[0])[self.pax] - 1
                pres = [0.5 * drive * L, -0.5 * drive * L]
        elif drive_dir is not None:
            f[drive_dir] = drive
        P = _Params(Re, c2, dt if dt is not None else default_dt(Re, c2), (C.c_double * 3)(*f),
                    None, int(transposed), (C.c_double * 2)(*pres))
        if alpha is not None:
            a = np.ascontiguousarray(alpha, dtype=np.float64).reshape(-1)
            assert a.size == self.N
            P.alpha = _dptr(a)
            P._alpha_ref = a  # keep alive
        return P

    def zeros(self):
        return np.zeros((3,) + self.shape), np.zeros(self.shape)

    # ------------------------------------------------------------ operators
    def momentum_residual(self, U, p, drive_dir=None, drive=DRIVE_PAPER, Re=RE_PAPER,
                          alpha=None, transposed=False):
        """Steady momentum residual (Sec. 3, 4): (1/Re)(A + S - alpha_f) u - G p + f."""
        P = self._params(drive_dir, drive, Re, C2_PAPER, 1.0, alpha, transposed)
        U = np.ascontiguousarray(U, dtype=np.float64)
        p = np.ascontiguousarray(p, dtype=np.float64)
        R = np.zeros_like(U)
        self._L.or_momentum_residual(self._ctx, C.byref(P), _dptr(U), _dptr(p), _dptr(R))
        return R

    def divergence(self, U):
        U = np.ascontiguousarray(U, dtype=np.float64)
        div = np.zeros(self.shape)
        self._L.or_divergence(self._ctx, _dptr(U), _dptr(div))
        return div

    def iterate(self, U, p, n, drive_dir=0, drive=DRIVE_PAPER, Re=RE_PAPER, c2=C2_PAPER, dt=None,
                alpha=None, transposed=False):
        """Algorithm 1 loop body, n times, in place: velocity, then pressure from the
        new velocity."""
        assert U.dtype == np.float64 and p.dtype == np.float64
        P = self._params(drive_dir, drive, Re, c2, dt, alpha, transposed)
        self._L.or_iterate(self._ctx, C.byref(P), _dptr(U), _dptr(p), int(n))

    def mean_velocity(self, U):
        """q_d = (1/N) sum u_d: superficial velocity (Fig. perm_computation)."""
        q = np.zeros(3)
        self._L.or_mean_velocity(self._ctx, _dptr(np.ascontiguousarray(U, dtype=np.float64)), _dptr(q))
        return q

    def superficial(self, q):
        """Superficial velocity from the cell means q = (1/N) sum u.  Periodic domains:
        q itself.  Fixed-pressure axis a: the flow crosses the n_a - 1 face planes between
        the layers (q_a n_a / (n_a - 1)); the cross components live in the n_a - 2
        interior layers (q_b n_a / (n_a - 2))."""
        q = np.asarray(q, dtype=np.float64).copy()
        if self.pax is not None:
            n = (self.shape[2], self.shape[1], self.shape[0])[self.pax]
            for d in range(3):
                q[d] *= n / (n - 1) if d == self.pax else n / (n - 2)
        return q

    def percolation(self):
        out = (C.c_int32 * 3)()
        self._L.or_percolation(self._ctx, out)
        return [bool(v) for v in out]

    def solve(self, drive_dir, tol=1e-10, check_every=100, max_iter=2_000_000, drive=DRIVE_PAPER,
              Re=RE_PAPER, c2=C2_PAPER, dt=None, alpha=None, transposed=False, U0=None, p0=None):
        """Pseudo-time iteration to the window criterion.  Returns a dict with the
        fields, q, iteration count (negative if max_iter was hit) and diagnostics."""
        U, p = self.zeros()
        if U0 is not None:
            U[...] = U0
        if p0 is not None:
            p[...] = p0
        P = self._params(drive_dir, drive, Re, c2, dt, alpha, transposed)
        q = np.zeros(3)
        info = np.zeros(3)
        it = self._L.or_solve(self._ctx, C.byref(P), int(drive_dir), float(tol), int(check_every),
                              int(max_iter), _dptr(U), _dptr(p), _dptr(q), _dptr(info))
        return {"U": U, "p": p, "q": q, "iters": int(it), "delta": float(info[0]),
                "err_est": float(info[1]), "div_norm": float(info[2])}


def permeability_from_q(Q: np.ndarray, Re: float = RE_PAPER, drive: float = DRIVE_PAPER,
                        dx: float = 1.0) -> np.ndarray:
    """Eq. darcy / Appendix C: column j of k from the mean velocities q^(j) of the drive
    along e_j.  In iteration units (mu = 1/Re, h_j = drive) k_ij = (1/Re) q_i^(j) / h_j,
    times dx^2 for m^2.  Q[:, j] = q^(j)."""
    return np.asarray(Q, dtype=np.float64) / (Re * drive) * dx * dx


def symmetrise(k: np.ndarray) -> np.ndarray:
    """Sec. 6.4 / Appendix C: k_ij = k_ji = (k_ij + k_ji) / 2."""
    return 0.5 * (k + k.T)


def ktensor(mask, dirs=(0, 1, 2), bc=(PERIODIC, PERIODIC, PERIODIC), tol=1e-10, check_every=100,
            max_iter=2_000_000, dx=1.0, alpha=None, dom: Domain | None = None):
    """Three simulations a) b) c) (Eq. cases_pressure) and the nine Darcy equations
    (Appendix C).  Non-percolating directions give a zero column.  Returns
    (k_sym, k_raw, runs)."""
    dom = dom or Domain(mask, bc)
    perc = dom.percolation()
    if dom.pax is not None:
        dirs = (dom.pax,)  # a fixed-pressure domain is driven along its pressure axis only
    Q = np.zeros((3, 3))
    runs = {}
    for j in dirs:
        if not perc[j]:
            runs[j] = None
            continue
        r = dom.solve(j, tol=tol, check_every=check_every, max_iter=max_iter, alpha=alpha)
        Q[:, j] = dom.superficial(r["q"])
        runs[j] = r
    k_raw = permeability_from_q(Q, dx=dx)
    return symmetrise(k_raw), k_raw, runs


def sensitivity(mask, w, alpha=None, bc=(PERIODIC, PERIODIC, PERIODIC), tol=1e-12, check_every=100,
                dom: Domain | None = None):
    """dJ/d alpha for J = sum_ij w_ij k_ij with a per-cell drag alpha in the momentum
    equation ((1/Re)(L u - alpha_f u), alpha_f = face average; alpha = 0 is the paper).

    Adjoint of the steady system (not in the paper, derived from it): with u^(j) the
    forward solution for drive j and v^(i) the solution of the transposed problem
    (viscous operator L^T) for a unit drive along i,
        dk_ij / d alpha_c = -(1 / (2 Re^2 N)) sum over the six faces F of cell c of v^(i)_F u^(j)_F
    (iteration units, unit drive).  Returns (dJ [nz, ny, nx], J, k_raw)."""
    w = np.asarray(w, dtype=np.float64).reshape(3, 3)
    dom = dom or Domain(mask, bc)
    nz, ny, nx = dom.shape
    fwd, adj = {}, {}
    k = np.zeros((3, 3))
    for j in range(3):
        if np.any(w[:, j] != 0):
            r = dom.solve(j, tol=tol, check_every=check_every, alpha=alpha)
            fwd[j] = r["U"]
            k[:, j] = r["q"] / RE_PAPER
    for i in range(3):
        if np.any(w[i, :] != 0):
            adj[i] = dom.solve(i, tol=tol, check_every=check_every, alpha=alpha, transposed=True)["U"]
    per = [b == PERIODIC for b in bc]
    s = np.zeros(dom.shape)
    for i, V in adj.items():
        for j, U in fwd.items():
            if w[i, j] == 0:
                continue
            for d in range(3):
                prod = V[d] * U[d]  # on the +d face of every cell
                axis = 2 - d        # array axis of direction d ([z][y][x])
                lower = np.roll(prod, 1, axis=axis)  # the -d face of each cell
                if not per[d]:
                    idx = [slice(None)] * 3
                    idx[axis] = 0
                    lower[tuple(idx)] = 0.0
                s += w[i, j] * (prod + lower)
    N = dom.N
    dJ = -s / (2.0 * RE_PAPER * RE_PAPER * N)
    return dJ, float(np.sum(w * k)), k
