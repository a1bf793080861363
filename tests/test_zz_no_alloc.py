"""pm_iterate_noalloc: the allocation-free variant of pm_iterate.

Some callers cannot call cudaMalloc (their GPU memory is owned by another allocator,
or an allocation would stall a latency-critical loop); this entry point serves them
from a fixed scratch array inside the library.  Here it is called through the C ABI
and must give pm_iterate's results, on two calls in a row that reuse the shared
scratch.  The file is named to be collected last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2407_19868_gb300 import geometry as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.fixture(scope="module")
def api():
    from paper_2407_19868_gb300 import api as A
    A.load()
    return A


def _run(api, fn, mask, n, drive_dir, precision, bc=(0, 0, 0), **opts):
    dt = torch.float64 if precision == "fp64" else torch.float32
    nz, ny, nx = mask.shape
    g = G.rng(3)
    u = torch.from_numpy(g.standard_normal((3, nz, ny, nx)) * 1e-3).to("cuda", dt).contiguous()
    p = torch.from_numpy(g.standard_normal((nz, ny, nx))).to("cuda", dt).contiguous()
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    dom = api.Domain(nx, ny, nz, m.ctypes.data, 0, 1.0, 1.0, (C.c_int32 * 3)(*bc))
    o = api.options(precision=precision, **opts)
    st = getattr(api.load(), fn)(C.byref(dom), drive_dir, 1.0, C.byref(o), n, u.data_ptr(), p.data_ptr(),
                                 torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return st, u.double().cpu().numpy(), p.double().cpu().numpy()


def test_noalloc_matches_pm_iterate_twice(api):
    """Both entry points launch the same kernels with the same work split, so the fields
    agree bit for bit; the third case is smaller than the first and reuses the scratch
    the larger one left behind."""
    cases = [
        (G.overlapping_spheres((24, 20, 36), 3.0, 0.6, seed=31), 7, 0, "fp32", (0, 0, 0), {"schedule": 5}),
        (G.random_blocks((5, 7, 9), 0.3, seed=32), 4, 2, "fp64", (0, 1, 0), {}),
        (G.overlapping_spheres((6, 10, 12), 2.0, 0.6, seed=33), 5, 1, "fp32", (1, 0, 0), {}),
        (G.overlapping_spheres((9, 11, 16), 2.0, 0.6, seed=34), 3, 0, "fp32", (0, 0, 0), {"kernel": 1}),
    ]
    for mask, n, d, prec, bc, opts in cases:
        st, u_na, p_na = _run(api, "pm_iterate_noalloc", mask, n, d, prec, bc, **opts)
        assert st == api.PM_OK, api.strerror(st)
        st, u_ref, p_ref = _run(api, "pm_iterate", mask, n, d, prec, bc, **opts)
        assert st == api.PM_OK
        assert np.array_equal(u_na, u_ref) and np.array_equal(p_na, p_ref)


def test_noalloc_rejects_domains_beyond_its_scratch(api):
    mask = np.zeros((64, 64, 33), dtype=np.uint8)  # 135168 cells > 131072
    u = torch.zeros((3,) + mask.shape, dtype=torch.float32, device="cuda")
    p = torch.zeros(mask.shape, dtype=torch.float32, device="cuda")
    dom = api.Domain(33, 64, 64, mask.ctypes.data, 0, 1.0, 1.0, (C.c_int32 * 3)(0, 0, 0))
    o = api.options()
    st = api.load().pm_iterate_noalloc(C.byref(dom), 0, 1.0, C.byref(o), 1, u.data_ptr(), p.data_ptr(), None)
    assert st == api.PM_ERR_TOO_LARGE
    assert "131072" in api.strerror(st)


def test_noalloc_rejects_a_fixed_pressure_axis(api):
    mask = np.zeros((4, 4, 8), dtype=np.uint8)
    u = torch.zeros((3,) + mask.shape, dtype=torch.float32, device="cuda")
    p = torch.zeros(mask.shape, dtype=torch.float32, device="cuda")
    dom = api.Domain(8, 4, 4, mask.ctypes.data, 0, 1.0, 1.0, (C.c_int32 * 3)(api.PRESSURE, 0, 0))
    o = api.options()
    st = api.load().pm_iterate_noalloc(C.byref(dom), 0, 1.0, C.byref(o), 1, u.data_ptr(), p.data_ptr(), None)
    assert st == api.PM_ERR_UNSUPPORTED
