"""GPU adjoint sensitivity (pm_sensitivity, KTensorFn) against the oracle's adjoint.

The oracle's adjoint is itself pinned by finite differences and the dot-product
identity (tests/test_oracle_adjoint.py).  Tolerances: FP64 fields 2e-7 of the largest
|dJ| (both sides converged to 1e-12; the ABI returns dJ/d alpha as FP32, whose rounding
is 6e-8 relative); FP32 fields 2e-4 (FP32 solution and a sum of products over six
faces)."""
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


@pytest.fixture(scope="module")
def case():
    mask = G.overlapping_spheres((10, 12, 16), 2.5, 0.62, seed=51)
    alpha = (G.rng(52).random(mask.shape) * 0.3).astype(np.float32)
    w = np.zeros((3, 3))
    w[0, 0], w[1, 0], w[0, 1], w[2, 2] = 1.0, 0.5, -0.3, 0.8
    return mask, alpha, w


@pytest.mark.parametrize("precision,tol,rel", [("fp64", 1e-12, 2e-7), ("fp32", 1e-9, 2e-4)])
def test_sensitivity_matches_oracle(api, oracle_mod, case, precision, tol, rel):
    mask, alpha, w = case
    dJ_o, J_o, k_o = oracle_mod.sensitivity(mask, w, alpha=alpha.astype(np.float64), tol=1e-13)
    r = api.sensitivity(mask, w, alpha=torch.from_numpy(alpha).cuda(), precision=precision, tol=tol)
    assert r["status"] == api.PM_OK
    dJ = r["dJ"].double().cpu().numpy()
    scale = np.abs(dJ_o).max()
    np.testing.assert_allclose(dJ, dJ_o, rtol=0, atol=rel * scale)
    assert r["J"] == pytest.approx(J_o, rel=max(rel, 1e-9))
    # solid voxels with no fluid face have zero sensitivity
    nf, _ = oracle_mod.Domain(mask).tables()
    touch = np.zeros(mask.shape, bool)
    for d in range(3):
        touch |= nf[d].astype(bool) | np.roll(nf[d].astype(bool), 1, axis=2 - d)
    assert np.all(dJ[~touch] == 0.0)


def test_symmetric_identity_on_gpu(api):
    """Channels of width <= 2 voxels: cases 1, 2, 3, 6 only, symmetric stencil, so
    dk_xx/d alpha = -(1/(2 Re^2 N)) sum over faces u_x-solution^2 (face products)."""
    m = np.ones((4, 6, 8), dtype=np.uint8)
    m[:, 1:3, :] = 0
    m[1:3, :, 4] = 0
    w = np.zeros((3, 3))
    w[0, 0] = 1.0
    r = api.sensitivity(m, w, precision="fp64", tol=1e-13)
    s = api.solve_direction(m, 0, precision="fp64", tol=1e-13)
    U = s["u"].double().cpu().numpy() * 0.01  # Darcy-scaled (1/Re) -> iteration units
    ss = np.zeros(m.shape)
    for d in range(3):
        prod = U[d] * U[d]
        ss += prod + np.roll(prod, 1, axis=2 - d)
    expect = -ss / (2 * 0.01**2 * m.size)
    np.testing.assert_allclose(r["dJ"].double().cpu().numpy(), expect, rtol=0, atol=1e-6 * np.abs(expect).max())


def test_ktensor_autograd(api, oracle_mod, case):
    mask, alpha, _ = case
    KTensorFn = api.KTensorFn
    a = torch.from_numpy(alpha).cuda().requires_grad_(True)
    opts = {"precision": "fp64", "tol": 1e-12}
    k = KTensorFn.apply(a, mask, opts)
    _, k_o, _ = oracle_mod.ktensor(mask, tol=1e-13, alpha=alpha.astype(np.float64))
    np.testing.assert_allclose(k.detach().cpu().numpy(), k_o, rtol=0, atol=1e-9 * np.abs(k_o).max())
    g = torch.zeros(3, 3, dtype=torch.float64, device="cuda")
    g[0, 0], g[2, 1] = 1.0, 0.5
    (k * g).sum().backward()
    grad = a.grad.double().cpu().numpy()
    # central differences of the same forward at three pore voxels
    pore = np.argwhere(mask == 0)
    for c in pore[G.rng(53).choice(len(pore), 3, replace=False)]:
        h = 1e-3
        ap, am = alpha.copy(), alpha.copy()
        ap[tuple(c)] += h
        am[tuple(c)] -= h
        kp = KTensorFn.apply(torch.from_numpy(ap).cuda(), mask, opts).cpu().numpy()
        km = KTensorFn.apply(torch.from_numpy(am).cuda(), mask, opts).cpu().numpy()
        fd = (kp[0, 0] - km[0, 0] + 0.5 * (kp[2, 1] - km[2, 1])) / (2 * h)
        assert grad[tuple(c)] == pytest.approx(fd, rel=2e-3, abs=1e-6 * np.abs(grad).max())


@pytest.mark.slow
def test_config4_foam_gradients(api):
    """192^3 open-cell foam (periodic Voronoi edges of 150 seeds, strut radius 3,
    porosity 0.90), the configuration's two objectives at alpha = 0:
    * dk_xx/d alpha against a central difference of the FP64 forward solves along a random
      direction v over all pore voxels (single-voxel changes are ~1e-10 of k, below solver
      noise).  The central difference has an O(h^2) error: measured 6.7e-4, 1.7e-4,
      4.2e-5 relative at h = 1e-3, 5e-4, 2.5e-4, so h = 2.5e-4 with a 1e-4 tolerance.
    * dk_xy/d alpha (forward drive y, transposed solve along x) against a Richardson-
      extrapolated central difference, fd(h/2) + (fd(h/2) - fd(h)) / 3, since k_xy is
      ~1e-2 of k_xx.
    * the whole FP32 gradient of k_xx (FP32 forward and transposed solves on the tiled
      kernels) against the FP64 gradient, within 1e-3 of its largest value."""
    mask, _ = G.voronoi_foam(192, 150, 3.0, 0.90, seed=4)
    dm = torch.from_numpy(mask).cuda()
    v = (G.rng(61).random(mask.shape) * (mask == 0)).astype(np.float32)
    vt = torch.from_numpy(v).cuda()
    # FP64 solves to a window change of 1e-9: their noise in a difference quotient is ~1e-9 / h
    # of k, far below the 1e-4 tolerance
    opts = {"precision": "fp64", "tol": 1e-9}
    wxx, wxy = np.zeros((3, 3)), np.zeros((3, 3))
    wxx[0, 0] = 1.0
    wxy[0, 1] = 1.0

    def fd(w, h):
        # forward solves of w's columns only (no gradient)
        Jp = api.sensitivity(dm, w, alpha=h * vt, grad=False, **opts)["J"]
        Jm = api.sensitivity(dm, w, alpha=-h * vt, grad=False, **opts)["J"]
        return (Jp - Jm) / (2 * h)

    g64 = api.sensitivity(dm, wxx, **opts)["dJ"].double()
    directional = float((g64 * vt.double()).sum())
    assert directional == pytest.approx(fd(wxx, 2.5e-4), rel=1e-4)
    gxy = api.sensitivity(dm, wxy, **opts)["dJ"].double()
    directional = float((gxy * vt.double()).sum())
    f1, f2 = fd(wxy, 1e-3), fd(wxy, 5e-4)
    rich = f2 + (f2 - f1) / 3.0
    assert directional == pytest.approx(rich, rel=1e-4), (directional, f1, f2, rich)
    g32 = api.sensitivity(dm, wxx, precision="fp32", tol=1e-7, max_iter=200000)["dJ"].double()
    assert float((g32 - g64).abs().max()) <= 1e-3 * float(g64.abs().max())


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_forward_fields_handed_over(api, case, precision):
    """Forward fields kept by one call and handed to the next: the second call solves only
    the transposed systems and gives the same gradient (the same converged fields)."""
    mask, alpha, w = case
    a = torch.from_numpy(alpha).cuda()
    tol = 1e-12 if precision == "fp64" else 1e-9
    api.sensitivity(mask, w, alpha=a, precision=precision, tol=tol)  # the shape's tuning runs here
    full = api.sensitivity(mask, w, alpha=a, precision=precision, tol=tol)
    f = api.sensitivity(mask, None, alpha=a, precision=precision, tol=tol, keep_fwd=True)
    part = api.sensitivity(mask, w, alpha=a, precision=precision, tol=tol, fwd=f["fwd"])
    assert torch.equal(part["dJ"], full["dJ"])
    np.testing.assert_allclose(part["k_raw"], f["k_raw"], rtol=1e-12, atol=1e-15)
    assert part["J"] == pytest.approx(full["J"], rel=1e-12)


def test_tiled_transposed_sweep_matches_simple_kernel(api, case):
    """The transposed FP32 solves on the tiled kernel and on the simple kernel (option
    kernel = 1) reach the same gradient within FP32 accuracy."""
    mask, alpha, w = case
    a = torch.from_numpy(alpha).cuda()
    t = api.sensitivity(mask, w, alpha=a, precision="fp32", tol=1e-9)["dJ"].double()
    s = api.sensitivity(mask, w, alpha=a, precision="fp32", tol=1e-9, kernel=1)["dJ"].double()
    assert float((t - s).abs().max()) <= 2e-4 * float(s.abs().max())
