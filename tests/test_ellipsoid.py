"""Benchmark geometries of Sec. 6: the inclined ellipsoid in a periodic box and regular
sphere packings.

CPU: the generator's volume is the ellipsoid's, and a 90 degree rotation about e1 equals
swapping e2 and e3 exactly.  GPU: the full k tensor of a coarse inclined ellipsoid (large
off-diagonal terms) matches the FP64 oracle, and its major principal axis follows the
inclination."""
import numpy as np
import pytest

from paper_2407_19868_gb300 import geometry as G


def test_ellipsoid_volume_and_quarter_turn():
    m0 = G.rotated_ellipsoid(100, (35.0, 10.0, 35.0), 0.0)
    assert abs(m0.sum() / (4.0 / 3.0 * np.pi * 35 * 10 * 35) - 1) < 0.01
    m90 = G.rotated_ellipsoid(100, (35.0, 10.0, 35.0), 90.0)
    assert np.array_equal(m90, np.swapaxes(m0, 0, 1))
    m30 = G.rotated_ellipsoid(100, (35.0, 10.0, 35.0), 30.0)
    assert abs(m30.sum() / m0.sum() - 1) < 0.01


@pytest.mark.gpu
def test_inclined_ellipsoid_ktensor_matches_oracle(oracle_mod):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():  # pragma: no cover
        pytest.skip("no CUDA device")
    from paper_2407_19868_gb300 import api
    m = G.rotated_ellipsoid(24, (8.4, 2.4, 8.4), 30.0)
    _, k_ref, _ = oracle_mod.ktensor(m, tol=1e-11, check_every=200)
    r = api.permeability_tensor(torch.from_numpy(m).cuda(), precision="dc64", tol=1e-9)
    k = np.asarray(r["k_raw"])
    assert np.max(np.abs(k - k_ref)) < 1e-6 * np.max(np.abs(k_ref))
    assert abs(k_ref[1, 2]) > 0.1 * k_ref[1, 1]  # strongly anisotropic, not a trivial case
    k2 = np.zeros((3, 3))
    k2[1:, 1:] = 0.5 * (k[1:, 1:] + k[1:, 1:].T)
    lam, R = api.principal_axes(k2)
    j = int(np.argmax(lam))
    phi = np.degrees(np.arctan2(abs(R[1, j]), abs(R[2, j])))
    assert 15.0 < phi < 40.0  # follows the 30 degree inclination (22 degrees at b = 2.4 voxels)


@pytest.mark.parametrize("kind", ["sc", "bcc", "fcc"])
def test_regular_pack_porosity_and_cubic_symmetry(kind):
    m, r = G.regular_pack(24, kind, 0.5)
    assert abs(G.porosity(m) - 0.5) < 0.02 and r > 0  # ties of equal distance at L = 24
    assert np.array_equal(m, np.transpose(m, (1, 2, 0))) and np.array_equal(m, m[::-1, ::-1, ::-1])


@pytest.mark.gpu
@pytest.mark.parametrize("kind", ["sc", "bcc", "fcc"])
def test_regular_pack_ktensor_is_isotropic(kind):
    """The cubic lattices give k = k_11 I exactly on the discrete grid (axis permutations
    map the geometry onto itself); the GPU tensor shows it to the FP32 floor."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():  # pragma: no cover
        pytest.skip("no CUDA device")
    from paper_2407_19868_gb300 import api
    m, _ = G.regular_pack(32, kind, 0.5)
    r = api.permeability_tensor(torch.from_numpy(m).cuda(), precision="fp32", tol=1e-8)
    k = np.asarray(r["k_raw"])
    kd = np.mean(np.diag(k))
    assert np.max(np.abs(np.diag(k) - kd)) < 1e-5 * kd
    assert np.max(np.abs(k - np.diag(np.diag(k)))) < 1e-5 * kd
    lam, _ = api.principal_axes(k)
    assert api.anisotropy_class(lam, rel_tol=1e-4) == api.ISOTROPY


@pytest.mark.gpu
@pytest.mark.slow
def test_ellipsoid_anisotropy_ratio_of_the_paper():
    """Sec. 6, Table ellipse_allvalues at alpha = 0: k_33 / k_22 = 9.43 / 3.85 = 2.45 and
    k_III / k_II = 9.46 / 3.81 = 2.48 for the 100^3 box with the (35, 10, 35) ellipsoid; the
    paper's absolute values are not comparable (units), its ratio is."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():  # pragma: no cover
        pytest.skip("no CUDA device")
    from paper_2407_19868_gb300 import api
    m = G.rotated_ellipsoid(100, (35.0, 10.0, 35.0), 0.0)
    r = api.permeability_tensor(torch.from_numpy(m).cuda(), precision="fp32", tol=1e-6)
    assert r["status"] == api.PM_OK
    k = np.asarray(r["k"])
    assert 2.43 < k[2, 2] / k[1, 1] < 2.53


def _gpu_api():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():  # pragma: no cover
        pytest.skip("no CUDA device")
    from paper_2407_19868_gb300 import api
    return api, torch


@pytest.mark.gpu
@pytest.mark.parametrize("ny,frame", [(4, 0), (9, 2)], ids=["uniform", "framed"])
def test_thin_medium_cell_matches_oracle(oracle_mod, ny, frame):
    """Thin porous medium of Sec. 6 at a small scale: one cylinder (radius 7 of a 20-voxel
    cell) across e2, uniform along e2 or between 2-voxel solid frames; k_11 of the GPU
    solve (defect-corrected) against the oracle's converged value, and the uniform cell's
    k_22 along the cylinder axis."""
    api, torch = _gpu_api()
    m = G.cylinder_cell(20, 7.0, ny, frame)
    dirs = (0, 1) if frame == 0 else (0,)
    for j in dirs:
        r = api.solve_direction(torch.from_numpy(m).cuda(), j, fields=False, precision="dc64", tol=1e-10)
        q = oracle_mod.Domain(m).solve(j, tol=1e-12, check_every=200)["q"] / oracle_mod.RE_PAPER
        assert r["k_col"][j] == pytest.approx(q[j], rel=1e-7)


@pytest.mark.gpu
@pytest.mark.parametrize("kind", ["sc", "bcc", "fcc"])
def test_regular_pack_matches_oracle_and_kozeny_carman(oracle_mod, kind):
    """Regular sphere packings of Sec. 6 in a 24-voxel unit cell at porosity 0.45: the full
    tensor against the oracle's (each component, defect-corrected), cubic isotropy, and
    the loose Kozeny-Carman agreement the section describes (k_11 within a factor of 2 of
    D^2 phi^3 / (180 (1 - phi)^2))."""
    api, torch = _gpu_api()
    m, rad = G.regular_pack(24, kind, 0.45)
    _, k_ref, _ = oracle_mod.ktensor(m, tol=1e-12, check_every=200)
    r = api.permeability_tensor(torch.from_numpy(m).cuda(), precision="dc64", tol=1e-10)
    k = np.asarray(r["k_raw"])
    kd = np.mean(np.diag(k_ref))
    np.testing.assert_allclose(np.diag(k), np.diag(k_ref), rtol=1e-7)
    assert np.max(np.abs(k - k_ref)) < 1e-7 * kd
    assert np.max(np.abs(np.diag(k) - kd)) < 1e-6 * kd  # cubic lattice: isotropic
    phi = float(1 - m.mean())
    kc = (2 * rad) ** 2 * phi ** 3 / (180.0 * (1 - phi) ** 2)
    assert 0.5 < k[0, 0] / kc < 2.0
