"""Multi-geometry batches (pm_batch_ktensor): domains of uneven sizes solved together in
one launch per sweep must give each domain's tensor as its own solve does, and the
oracle's; non-percolating drives leave zero columns."""
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


def _masks():
    return [G.overlapping_spheres((12, 20, 36), 3.0, 0.6, seed=81),
            G.overlapping_spheres((8, 16, 24), 2.5, 0.65, seed=82),
            G.slit(32, 3, 6, nz=4),  # flow along x and z only
            G.overlapping_spheres((20, 14, 68), 3.0, 0.62, seed=83)]


def test_batch_matches_single_solves(api, oracle_mod):
    masks = _masks()
    r = api.batch_ktensor(masks, tol=1e-10, precision="fp64")
    assert r["status"] == api.PM_ERR_NOT_PERCOLATING
    for d, m in enumerate(masks):
        single = api.permeability_tensor(m, tol=1e-10, precision="fp64")
        scale = np.abs(np.diag(single["k_raw"])).max()
        np.testing.assert_allclose(r["k_raw"][d], single["k_raw"], rtol=0, atol=1e-8 * scale)
        np.testing.assert_allclose(r["k"][d], single["k"], rtol=0, atol=1e-8 * scale)
    assert np.all(r["k"][2][1, :] == 0) and np.all(r["k"][2][:, 1] == 0)
    assert not r["stats"][2][1]["percolates"]
    # one member against the oracle
    _, k_o, _ = oracle_mod.ktensor(masks[1], tol=1e-12)
    np.testing.assert_allclose(r["k_raw"][1], k_o, rtol=0, atol=1e-8 * np.abs(np.diag(k_o)).max())


def test_batch_fp32_selected_drives(api):
    masks = _masks()[:2]
    r = api.batch_ktensor(masks, drives=[1, 2], tol=1e-9)
    assert r["status"] == api.PM_OK
    for d, j in ((0, 0), (1, 1)):
        single = api.solve_direction(masks[d], j, tol=1e-9, fields=False)
        np.testing.assert_allclose(r["k_raw"][d][:, j], single["k_col"], rtol=0,
                                   atol=2e-5 * abs(single["k_col"][j]))
        others = [c for c in range(3) if c != j]
        assert np.all(r["k_raw"][d][:, others] == 0)
