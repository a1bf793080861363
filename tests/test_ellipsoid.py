"""The anisotropy benchmark geometry of Sec. 6 (an inclined ellipsoid in a periodic box).

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
