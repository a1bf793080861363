"""Python binding of the GB300 permeability solver's C ABI (``include/poremaps_gb.h``).

Argument marshalling only: every step of the solve runs in ``libpm_gb300.so``.
PyTorch supplies device memory and the current CUDA stream.  If the library has not
been built, :func:`load` raises; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

PM_OK = 0
PM_ERR_INVALID_ARG = 1
PM_ERR_NO_FLUID = 2
PM_ERR_NOT_PERCOLATING = 3
PM_ERR_NOT_CONVERGED = 4
PM_ERR_DIVERGED = 5
PM_ERR_OOM = 6
PM_ERR_CUDA = 7
PM_ERR_TIMEOUT = 8
PM_ERR_UNSUPPORTED = 9
PM_ERR_TOO_LARGE = 10

PERIODIC = 0
WALL = 1
PRESSURE = 2  # fixed-pressure inlet/outlet reservoirs: first and last layer along the axis

FP32_RED64 = 0
FP32_DC64 = 1
FP64 = 2
_PRECISION = {"fp32": FP32_RED64, "fp32_red64": FP32_RED64, "fp32_dc64": FP32_DC64, "dc64": FP32_DC64,
              "fp64": FP64}

# every function the header declares (checked by the ABI test)
EXPORTED = ["pm_default_options", "pm_strerror", "pm_version", "pm_time_step", "pm_iterate",
            "pm_iterate_noalloc", "pm_solve_direction", "pm_permeability_tensor", "pm_sensitivity",
            "pm_batch_ktensor", "pm_mirror_mask", "pm_remove_isolated_pores", "pm_principal_axes",
            "pm_anisotropy_class", "pm_release_memory"]


class PMError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {strerror(status)} (status {status})")
        self.status = status


class Domain(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("mask", C.c_void_p),
                ("mask_on_device", C.c_int32), ("voxel_size", C.c_double), ("viscosity", C.c_double),
                ("bc", C.c_int32 * 3)]


class Options(C.Structure):
    _fields_ = [("tol", C.c_double), ("check_every", C.c_int32), ("max_iter", C.c_int64),
                ("precision", C.c_int32), ("dt_safety", C.c_double), ("Re", C.c_double),
                ("c2", C.c_double), ("use_graph", C.c_int32), ("check_percolation", C.c_int32),
                ("dc_switch_tol", C.c_double), ("dc_max_rounds", C.c_int32), ("kernel", C.c_int32),
                ("autotune", C.c_int32), ("schedule", C.c_int32), ("tile", C.c_int32),
                ("sequence", C.c_int32), ("field_memory", C.c_int32), ("schedule_split", C.c_int32),
                ("dc_extrapolate", C.c_int32), ("reserved", C.c_int32 * 1)]


class Stats(C.Structure):
    _fields_ = [("iters", C.c_int64), ("q", C.c_double * 3), ("delta", C.c_double),
                ("err_est", C.c_double), ("div_res", C.c_double), ("seconds", C.c_double),
                ("sweep_ms", C.c_double), ("sweeps_timed", C.c_int64), ("dc_rounds", C.c_int32),
                ("status", C.c_int32), ("percolates", C.c_int32), ("schedule", C.c_int32),
                ("setup_seconds", C.c_double), ("n_fluid", C.c_int64), ("sweep_ms_src", C.c_double),
                ("sweeps_timed_src", C.c_int64), ("kernel_launches", C.c_int64), ("tile", C.c_int32),
                ("schedule_split", C.c_int32)]

    def as_dict(self):
        return {"iters": int(self.iters), "q": [float(v) for v in self.q], "delta": float(self.delta),
                "err_est": float(self.err_est), "div_res": float(self.div_res),
                "seconds": float(self.seconds), "sweep_ms": float(self.sweep_ms),
                "sweeps_timed": int(self.sweeps_timed), "dc_rounds": int(self.dc_rounds),
                "status": int(self.status), "percolates": bool(self.percolates),
                "schedule": int(self.schedule), "setup_seconds": float(self.setup_seconds),
                "n_fluid": int(self.n_fluid), "sweep_ms_src": float(self.sweep_ms_src),
                "sweeps_timed_src": int(self.sweeps_timed_src), "kernel_launches": int(self.kernel_launches),
                "tile": int(self.tile), "schedule_split": int(self.schedule_split)}


_LIB = None
_LOCK = threading.Lock()


def library_path() -> str:
    return _build.lib_path()


def load():
    """Open libpm_gb300.so (built by ``__graft_entry__.build()``); raises if absent."""
    global _LIB
    with _LOCK:
        if _LIB is not None:
            return _LIB
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path} is missing "
                               "(run python -c 'import __graft_entry__ as g; g.build()')")
        L = C.CDLL(path)
        vp, dp = C.c_void_p, C.POINTER(C.c_double)
        L.pm_default_options.argtypes = [C.POINTER(Options)]
        L.pm_strerror.restype = C.c_char_p
        L.pm_strerror.argtypes = [C.c_int]
        L.pm_version.restype = C.c_int
        L.pm_time_step.restype = C.c_double
        L.pm_time_step.argtypes = [C.POINTER(Options)]
        L.pm_iterate.argtypes = [C.POINTER(Domain), C.c_int, C.c_double, C.POINTER(Options), C.c_int64,
                                 vp, vp, vp]
        L.pm_iterate_noalloc.argtypes = L.pm_iterate.argtypes
        L.pm_solve_direction.argtypes = [C.POINTER(Domain), C.c_int, C.c_double, C.POINTER(Options),
                                         vp, vp, vp, vp, dp, C.POINTER(Stats), vp]
        L.pm_permeability_tensor.argtypes = [C.POINTER(Domain), C.c_double, C.POINTER(Options), dp, dp,
                                             C.POINTER(Stats), vp]
        L.pm_sensitivity.argtypes = [C.POINTER(Domain), vp, dp, C.POINTER(Options), vp, dp, dp, C.POINTER(vp),
                                     C.c_int32, vp]
        L.pm_batch_ktensor.argtypes = [C.c_int, C.POINTER(Domain), C.POINTER(C.c_int32), C.POINTER(Options), dp, dp,
                                       C.POINTER(Stats), vp]
        L.pm_principal_axes.argtypes = [dp, dp, dp]
        L.pm_mirror_mask.argtypes = [vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, vp, vp]
        L.pm_remove_isolated_pores.argtypes = [vp, C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_int32), vp,
                                               C.POINTER(C.c_int64)]
        L.pm_anisotropy_class.argtypes = [dp, C.c_double]
        L.pm_release_memory.restype = C.c_int
        _LIB = L
        return L


def release_memory():
    """Hand the scratch the library's memory pool keeps between calls back to the driver
    (pm_release_memory, current device)."""
    _check(load().pm_release_memory(), "pm_release_memory")


def strerror(status: int) -> str:
    try:
        return load().pm_strerror(int(status)).decode()
    except RuntimeError:
        return f"status {status}"


def options(**kw) -> Options:
    o = Options()
    load().pm_default_options(C.byref(o))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = _PRECISION[v]
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def time_step(**kw) -> float:
    o = options(**kw)
    return float(load().pm_time_step(C.byref(o)))


def _stream(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


class _Mask:
    """Keeps the mask alive and describes it as a pm_domain."""

    def __init__(self, mask, dx=1.0, mu=1.0, bc=(PERIODIC, PERIODIC, PERIODIC)):
        import torch
        if isinstance(mask, torch.Tensor):
            m = mask.contiguous()
            if m.dtype != torch.uint8:
                m = (m != 0).to(torch.uint8)
            self._keep = m
            ptr, on_dev = m.data_ptr(), int(m.is_cuda)
            shape = tuple(m.shape)
        else:
            m = np.ascontiguousarray(mask, dtype=np.uint8)
            self._keep = m
            ptr, on_dev = m.ctypes.data, 0
            shape = m.shape
        if len(shape) != 3:
            raise ValueError("mask must be 3-D [nz][ny][nx]")
        nz, ny, nx = shape
        self.shape = shape
        self.N = nx * ny * nz
        self.dom = Domain(nx, ny, nz, ptr, on_dev, float(dx), float(mu), (C.c_int32 * 3)(*bc))


def _check(status: int, what: str, soft=(PM_OK,)):
    if status not in soft:
        raise PMError(status, what)
    return status


def iterate(mask, u, p, n: int, drive_dir: int = 0, drive: float = 1.0, bc=(0, 0, 0), stream=None, **opts):
    """Algorithm 1 loop body n times in place on device fields (iteration units):
    u: (3, nz, ny, nx), p: (nz, ny, nx), float32 (precision fp32) or float64 (fp64)."""
    import torch
    m = _Mask(mask, bc=bc)
    prec = opts.pop("precision", "fp64" if u.dtype == torch.float64 else "fp32")
    o = options(precision=prec, **opts)
    want = torch.float64 if o.precision == FP64 else torch.float32
    if u.dtype != want or p.dtype != want or not (u.is_cuda and p.is_cuda):
        raise TypeError("u, p must be CUDA tensors of the precision's type")
    if not (u.is_contiguous() and p.is_contiguous()) or u.numel() != 3 * m.N or p.numel() != m.N:
        raise ValueError("u, p must be contiguous with 3N and N elements")
    st = load().pm_iterate(C.byref(m.dom), int(drive_dir), float(drive), C.byref(o), int(n),
                           u.data_ptr(), p.data_ptr(), _stream(stream))
    _check(st, "pm_iterate")
    return u, p


def solve_direction(mask, drive_dir: int, drive: float = 1.0, dx: float = 1.0, mu: float = 1.0,
                    bc=(0, 0, 0), fields: bool = True, u0=None, p0=None, stream=None, **opts):
    """One drive direction to convergence.  Returns dict(k_col, u, p, stats, status);
    u, p are Darcy-scaled float32 CUDA tensors (None unless ``fields``)."""
    import torch
    m = _Mask(mask, dx=dx, mu=mu, bc=bc)
    o = options(**opts)
    dev = torch.device("cuda")
    u = torch.empty((3,) + m.shape, dtype=torch.float32, device=dev) if fields else None
    p = torch.empty(m.shape, dtype=torch.float32, device=dev) if fields else None
    k = (C.c_double * 3)()
    s = Stats()
    st = load().pm_solve_direction(C.byref(m.dom), int(drive_dir), float(drive), C.byref(o),
                                   u.data_ptr() if u is not None else None,
                                   p.data_ptr() if p is not None else None,
                                   u0.data_ptr() if u0 is not None else None,
                                   p0.data_ptr() if p0 is not None else None,
                                   k, C.byref(s), _stream(stream))
    _check(st, "pm_solve_direction", soft=(PM_OK, PM_ERR_NOT_PERCOLATING, PM_ERR_NOT_CONVERGED))
    return {"k_col": np.array(k[:]), "u": u, "p": p, "stats": s.as_dict(), "status": st}


def mirror_mask(mask, axes=(True, False, False), stream=None):
    """Mask followed by its mirror image along the chosen axes (x, y, z) -- pre-processing
    for symmetric periodicity (pm_mirror_mask).  numpy in, numpy out (host loop); a CUDA
    uint8 tensor in, a CUDA tensor out (one kernel)."""
    bits = sum(1 << a for a in range(3) if axes[a])
    if hasattr(mask, "is_cuda") and mask.is_cuda:
        import torch
        m = mask.contiguous()
        nz, ny, nx = m.shape
        out = torch.empty((nz << bool(axes[2]), ny << bool(axes[1]), nx << bool(axes[0])), dtype=torch.uint8,
                          device=m.device)
        st = load().pm_mirror_mask(m.data_ptr(), nx, ny, nz, bits, 1, out.data_ptr(), _stream(stream))
    else:
        m = np.ascontiguousarray(mask, dtype=np.uint8)
        nz, ny, nx = m.shape
        out = np.empty((nz << bool(axes[2]), ny << bool(axes[1]), nx << bool(axes[0])), dtype=np.uint8)
        st = load().pm_mirror_mask(m.ctypes.data, nx, ny, nz, bits, 0, out.ctypes.data, None)
    _check(st, "pm_mirror_mask")
    return out


def remove_isolated_pores(mask, bc=(0, 0, 0)):
    """Mask with every pore component that carries no flow through the domain turned solid
    (pm_remove_isolated_pores; host).  Returns (mask, number of cells removed)."""
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    nz, ny, nx = m.shape
    out = np.empty_like(m)
    n = C.c_int64(0)
    _check(load().pm_remove_isolated_pores(m.ctypes.data, nx, ny, nz, (C.c_int32 * 3)(*bc), out.ctypes.data,
                                           C.byref(n)), "pm_remove_isolated_pores")
    return out, int(n.value)


def principal_axes(k):
    """Principal permeabilities (ascending) and axes (columns) of the symmetric part of a
    3x3 tensor (pm_principal_axes; host only)."""
    kk = (C.c_double * 9)(*[float(v) for v in np.asarray(k, dtype=np.float64).reshape(9)])
    lam = (C.c_double * 3)()
    ax = (C.c_double * 9)()
    _check(load().pm_principal_axes(kk, lam, ax), "pm_principal_axes")
    return np.array(lam[:]), np.array(ax[:]).reshape(3, 3)


ISOTROPY, TRANSVERSE_ANISOTROPY, ORTHOTROPY = 0, 1, 2


def anisotropy_class(lam, rel_tol: float = 1e-2) -> int:
    """Sec. 2 material class of three principal permeabilities (pm_anisotropy_class)."""
    v = (C.c_double * 3)(*[float(x) for x in lam])
    c = int(load().pm_anisotropy_class(v, float(rel_tol)))
    if c < 0:
        raise ValueError("invalid principal permeabilities or tolerance")
    return c


def permeability_tensor(mask, dx: float = 1.0, bc=(0, 0, 0), stream=None, **opts):
    """Full tensor, three drives batched per sweep launch.  Returns
    dict(k (symmetrised 3x3), k_raw, stats (3 dicts), status)."""
    m = _Mask(mask, dx=dx, bc=bc)
    o = options(**opts)
    k = (C.c_double * 9)()
    kr = (C.c_double * 9)()
    s = (Stats * 3)()
    st = load().pm_permeability_tensor(C.byref(m.dom), 1.0, C.byref(o), k, kr, s, _stream(stream))
    _check(st, "pm_permeability_tensor", soft=(PM_OK, PM_ERR_NOT_PERCOLATING, PM_ERR_NOT_CONVERGED))
    return {"k": np.array(k[:]).reshape(3, 3), "k_raw": np.array(kr[:]).reshape(3, 3),
            "stats": [s[i].as_dict() for i in range(3)], "status": st}


def sensitivity(mask, w=None, alpha=None, dx: float = 1.0, bc=(0, 0, 0), stream=None, fwd=None,
                keep_fwd=False, grad=True, **opts):
    """Adjoint sensitivity of J = sum w_ij k_ij to a per-cell drag alpha (pm_sensitivity).
    alpha: CUDA float32 tensor (nz, ny, nx) or None.  With w=None only the forward solves
    run and dJ is None.  fwd: forward fields from an earlier call (tensor (3, 3, nz, ny,
    nx): drive, component; those drives are not solved again); keep_fwd: return this
    call's forward fields as "fwd"; grad=False: no gradient, only the forward solves of
    w's nonzero columns (J and those k columns).  Returns dict(dJ, J, k_raw, status, fwd)."""
    import torch
    m = _Mask(mask, dx=dx, bc=bc)
    o = options(**opts)
    a = None
    if alpha is not None:
        a = alpha.detach().to(device="cuda", dtype=torch.float32).contiguous()
        if a.numel() != m.N:
            raise ValueError("alpha must have one value per voxel")
    dJ = torch.empty(m.shape, dtype=torch.float32, device="cuda") if w is not None and grad else None
    wa = (C.c_double * 9)(*np.asarray(w, dtype=np.float64).reshape(-1)) if w is not None else None
    J = C.c_double(0.0)
    kr = (C.c_double * 9)()
    ftype = torch.float64 if o.precision == FP64 else torch.float32
    given = 0
    uf = None
    if fwd is not None:
        if fwd.dtype != ftype or not fwd.is_cuda or fwd.numel() != 9 * m.N:
            raise ValueError("fwd must be a CUDA tensor (3, 3, nz, ny, nx) of the precision's type")
        uf, given = fwd.contiguous(), 1
    elif keep_fwd:
        uf = torch.zeros((3, 3) + tuple(m.shape), dtype=ftype, device="cuda")
    ptrs = (C.c_void_p * 3)(*([uf[j].data_ptr() for j in range(3)] if uf is not None else [None] * 3))
    st = load().pm_sensitivity(C.byref(m.dom), a.data_ptr() if a is not None else None, wa, C.byref(o),
                               dJ.data_ptr() if dJ is not None else None, C.byref(J), kr,
                               ptrs if uf is not None else None, given, _stream(stream))
    _check(st, "pm_sensitivity", soft=(PM_OK, PM_ERR_NOT_CONVERGED))
    return {"dJ": dJ, "J": float(J.value), "k_raw": np.array(kr[:]).reshape(3, 3), "status": st,
            "fwd": uf if keep_fwd else None}


def batch_ktensor(masks, drives=None, dx: float = 1.0, bc=(0, 0, 0), stream=None, **opts):
    """Tensors of many geometries in one solve (pm_batch_ktensor).  masks: list of uint8
    arrays / tensors; drives: per mask a bit mask of drive axes (None = all).  Returns
    dict(k [n, 3, 3], k_raw [n, 3, 3], stats [n][3], status)."""
    ms = [_Mask(m, dx=dx, bc=bc) for m in masks]
    n = len(ms)
    doms = (Domain * n)(*[m.dom for m in ms])
    dr = (C.c_int32 * n)(*(drives if drives is not None else [0] * n))
    o = options(**opts)
    k = (C.c_double * (9 * n))()
    kr = (C.c_double * (9 * n))()
    s = (Stats * (3 * n))()
    st = load().pm_batch_ktensor(n, doms, dr, C.byref(o), k, kr, s, _stream(stream))
    _check(st, "pm_batch_ktensor", soft=(PM_OK, PM_ERR_NOT_PERCOLATING, PM_ERR_NOT_CONVERGED))
    return {"k": np.array(k[:]).reshape(n, 3, 3), "k_raw": np.array(kr[:]).reshape(n, 3, 3),
            "stats": [[s[3 * d + j].as_dict() for j in range(3)] for d in range(n)], "status": st}


def _ktensor_fn():
    import torch

    class KTensorFn(torch.autograd.Function):
        """k_raw(alpha): the 3x3 permeability tensor of the mask with a per-cell drag
        alpha (alpha = 0 is the paper's problem).  forward keeps the three forward fields;
        backward(grad_k) runs only the transposed solves: pm_sensitivity with w = grad_k
        and the kept fields gives d(sum grad_k * k)/d alpha."""

        @staticmethod
        def forward(ctx, alpha, mask, opts):
            r = sensitivity(mask, None, alpha=alpha, keep_fwd=True, **opts)
            ctx.mask, ctx.opts = mask, opts
            ctx.save_for_backward(alpha, r["fwd"])
            return torch.as_tensor(r["k_raw"], dtype=torch.float64, device=alpha.device)

        @staticmethod
        def backward(ctx, grad_k):
            alpha, fwd = ctx.saved_tensors
            w = grad_k.detach().double().cpu().numpy()
            if not np.any(w):
                return torch.zeros_like(alpha), None, None
            r = sensitivity(ctx.mask, w, alpha=alpha, fwd=fwd, **ctx.opts)
            return r["dJ"].to(alpha.dtype), None, None

    return KTensorFn


def __getattr__(name):
    if name == "KTensorFn":
        return _ktensor_fn()
    raise AttributeError(name)
