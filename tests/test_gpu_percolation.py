"""Percolation check on the GPU (device union-find of the pore cells plus a winding
search over the components that meet at the periodic faces) against the oracle's
breadth-first search with winding numbers (Sec. 5.1 assumes percolation; a blocked
drive gives a zero k column).  Random voxel masks near the site-percolation threshold
(pore fraction ~0.31) make many components that touch the faces in different ways."""
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


def _gpu_flags(api, mask, bc):
    r = api.permeability_tensor(torch.from_numpy(mask).cuda(), bc=bc, tol=1e-12, check_every=2, max_iter=2,
                                autotune=0)
    return [bool(s["percolates"]) for s in r["stats"]], r


SHAPES = [((12, 10, 16), (0, 0, 0)), ((6, 20, 9), (0, 0, 0)), ((16, 16, 16), (0, 1, 0)),
          ((1, 24, 20), (0, 0, 0)), ((2, 3, 40), (0, 0, 0)), ((9, 7, 5), (1, 0, 0)), ((20, 6, 6), (0, 0, 1))]


@pytest.mark.parametrize("shape,bc", SHAPES, ids=[f"{s}-{b}" for s, b in SHAPES])
def test_device_percolation_matches_oracle(api, oracle_mod, shape, bc):
    agree = 0
    for seed in range(12):
        solid = 0.62 + 0.01 * (seed % 8)
        mask = G.random_blocks(shape, solid, seed=100 + seed)
        if not np.any(mask == 0):
            continue
        want = oracle_mod.Domain(mask, bc=bc).percolation()
        got, r = _gpu_flags(api, mask, bc)
        assert got == want, (seed, got, want)
        assert all(s["n_fluid"] == int(np.count_nonzero(mask == 0)) for s in r["stats"])
        agree += 1
    assert agree >= 10


def test_blocked_drive_and_wrapping_channel(api, oracle_mod):
    """A channel that only closes through two periodic faces (a staircase across the
    x and y faces) percolates along both; walls across z block that axis."""
    n = 8
    mask = np.ones((3, n, n), dtype=np.uint8)
    for k in range(n):
        mask[1, k, k] = 0
        mask[1, k, (k + 1) % n] = 0
    got, _ = _gpu_flags(api, mask, (0, 0, 0))
    assert got == oracle_mod.Domain(mask).percolation() == [True, True, False]


def test_no_fluid_is_reported(api):
    with pytest.raises(api.PMError) as e:
        api.permeability_tensor(torch.ones((4, 5, 8), dtype=torch.uint8, device="cuda"))
    assert e.value.status == api.PM_ERR_NO_FLUID
