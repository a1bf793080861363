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


def test_batch_any_width(api):
    """Widths that are not a multiple of 4: a periodic x axis is repeated inside the
    library (2 or 4 copies, the same discrete problem), a wall x axis padded with solid;
    each tensor equals the domain's own solve (simple kernel for these widths)."""
    masks = [G.overlapping_spheres((8, 12, 18), 2.5, 0.62, seed=91),   # nx % 4 == 2
             G.overlapping_spheres((9, 10, 17), 2.5, 0.62, seed=92),   # nx odd
             G.overlapping_spheres((6, 14, 24), 2.5, 0.62, seed=93)]   # nx % 4 == 0
    for bc in ((0, 0, 0), (1, 0, 0)):
        r = api.batch_ktensor(masks, bc=bc, tol=1e-10, precision="fp64")
        for d, m in enumerate(masks):
            single = api.permeability_tensor(m, bc=bc, tol=1e-10, precision="fp64")
            scale = np.abs(np.diag(single["k_raw"])).max()
            np.testing.assert_allclose(r["k_raw"][d], single["k_raw"], rtol=0, atol=1e-8 * scale)
            for j in range(3):
                assert r["stats"][d][j]["n_fluid"] == int(np.count_nonzero(m == 0))


def test_sequence_mode_warm_starts(api):
    """Sequence mode: the states of a clogging sequence in order, each from the previous
    one's converged fields; the tensors equal the batch solve's, and the later states need
    fewer iterations than from rest."""
    states = G.clogging_sequence(96, 48, n_states=4, phi0=0.6, phi_end=0.5, seed=7, r_lo=3.0, r_hi=6.0)
    cold = api.batch_ktensor(states, drives=[3] * 4, tol=1e-10, precision="fp64")
    warm = api.batch_ktensor(states, drives=[3] * 4, tol=1e-10, precision="fp64", sequence=1)
    for d in range(4):
        scale = np.abs(np.diag(cold["k_raw"][d])).max()
        np.testing.assert_allclose(warm["k_raw"][d], cold["k_raw"][d], rtol=0, atol=1e-8 * scale)
    it_cold = sum(cold["stats"][d][j]["iters"] for d in range(1, 4) for j in range(2)
                  if cold["stats"][d][j]["percolates"])
    it_warm = sum(warm["stats"][d][j]["iters"] for d in range(1, 4) for j in range(2)
                  if warm["stats"][d][j]["percolates"])
    assert it_warm < it_cold


@pytest.mark.parametrize("name", ["config3_small_s0", "config3_small_s1"])
def test_clogging_states_against_oracle_reference(api, name):
    """Downsized precipitation states (192 x 96 disk image, radii 3 .. 7.5, four fluid
    layers between solid layers) in a batched solve against the oracle's converged
    columns (tests/golden/make_reference.py; the mask hash must match): FP64 fields to
    1e-6 of each component, FP32 fields (the paper's criterion, bounded iterations) to 2e-5
    of the diagonal."""
    import json
    import os
    ref = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "reference_k.json")))
    if name not in ref:
        pytest.skip("oracle reference not generated")
    ref = ref[name]
    s = int(name[-1])
    m = G.clogging_sequence(192, 96, n_states=2, phi0=0.55, phi_end=0.45, seed=3, r_lo=3.0, r_hi=7.5)[s]
    assert G.mask_sha256(m) == ref["sha256"]
    k_o = np.zeros((3, 3))
    for j, col in ref["columns"].items():
        k_o[:, int(j)] = col["k_col"]
    r64 = api.batch_ktensor([m, m[:, :, :190]], drives=[3, 3], tol=1e-11, precision="fp64")
    r32 = api.batch_ktensor([m], drives=[3], tol=1e-6, max_iter=60000)
    for j in (0, 1):
        perc = ref["columns"][str(j)].get("percolates", True)
        assert r64["stats"][0][j]["percolates"] == perc
        if not perc:
            assert np.all(r64["k_raw"][0][:, j] == 0)
            continue
        kj = k_o[:, j]
        # each component against its own value; a component that vanishes by symmetry
        # (below 1e-7 of the diagonal in the reference) against the diagonal
        np.testing.assert_allclose(r64["k_raw"][0][:2, j], kj[:2], rtol=1e-6, atol=1e-7 * abs(kj[j]))
        assert abs(r64["k_raw"][0][2, j]) <= 1e-12 * abs(kj[j])  # solid layers close z
        if r32["stats"][0][j]["status"] == api.PM_OK:
            assert r32["k_raw"][0][j, j] == pytest.approx(kj[j], rel=2e-5)


def test_thin_domains_exchange_axes(api):
    """A thin domain (6 cells along z, 96 along y) is solved inside the batch with y and z
    exchanged; its tensor, statistics and percolation flags are the domain's own, equal to
    its single solve (which marches along z)."""
    states = G.clogging_sequence(64, 96, n_states=2, phi0=0.6, phi_end=0.5, seed=11, r_lo=3.0, r_hi=6.0)
    m = states[1]
    r = api.batch_ktensor([m, states[0]], drives=[3, 7], tol=1e-10, precision="fp64")
    single = api.permeability_tensor(m, tol=1e-10, precision="fp64")
    scale = np.abs(np.diag(single["k_raw"])).max()
    np.testing.assert_allclose(r["k_raw"][0][:, :2], single["k_raw"][:, :2], rtol=0, atol=1e-8 * scale)
    assert np.all(r["k_raw"][0][:, 2] == 0)  # drive z not requested
    for j in range(3):
        assert r["stats"][1][j]["percolates"] == single["stats"][j]["percolates"]
    assert not r["stats"][1][2]["percolates"]  # the solid layers close z
    s0 = api.permeability_tensor(states[0], tol=1e-10, precision="fp64")
    np.testing.assert_allclose(r["k_raw"][1], s0["k_raw"], rtol=0, atol=1e-8 * np.abs(np.diag(s0["k_raw"])).max())
