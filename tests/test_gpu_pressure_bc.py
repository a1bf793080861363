"""GPU parity of the fixed-pressure inlet/outlet boundary (PM_BC_PRESSURE) against the
FP64 oracle, through the C ABI.  Same tolerances as the periodic parity tests:
trajectories 1e-11 (FP64) and 2e-5 (FP32) of the field's maximum; converged k per
component against the oracle at the solve tolerance."""
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


CASES = [
    ("x_periodic", lambda: G.random_blocks((5, 7, 9), 0.25, seed=31), (2, 0, 0), 0),
    ("z_walls", lambda: G.overlapping_spheres((11, 8, 12), 2.0, 0.6, seed=32), (1, 0, 2), 2),
    ("y_thin", lambda: G.random_blocks((1, 6, 8), 0.2, seed=33), (0, 2, 0), 1),
    ("x_min3", lambda: G.random_blocks((4, 5, 3), 0.2, seed=34), (2, 1, 0), 0),
]


@pytest.mark.parametrize("name,make,bc,a", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", 2e-5)])
def test_trajectory_matches_oracle(api, oracle_mod, name, make, bc, a, precision, tol):
    mask = make()
    dt = torch.float64 if precision == "fp64" else torch.float32
    dom = oracle_mod.Domain(mask, bc=bc)
    for n in (1, 2, 10):
        U, p = dom.zeros()
        dom.iterate(U, p, n, drive_dir=a, dt=api.time_step())
        u = torch.zeros((3,) + mask.shape, dtype=dt, device="cuda")
        pg = torch.zeros(mask.shape, dtype=dt, device="cuda")
        api.iterate(torch.from_numpy(mask).cuda(), u, pg, n, drive_dir=a, bc=bc, precision=precision)
        ug, pgn = u.double().cpu().numpy(), pg.double().cpu().numpy()
        su, sp = max(np.max(np.abs(U)), 1e-300), max(np.max(np.abs(p)), 1e-300)
        assert np.max(np.abs(ug - U)) <= tol * su, (n, "u")
        assert np.max(np.abs(pgn - p)) <= tol * sp, (n, "p")
        # non-fluid nodes, including the reservoirs' cross velocities, are exactly 0
        nf, _ = dom.tables()
        assert np.all(ug[nf == 0] == 0)


# Domains that span several tiles of the tiled kernel (64 x 12 cells per tile) with ragged
# last tiles, the reservoirs on every kind of tile edge: x pressure (three tile columns, the
# last 8 wide), y pressure with the outlet reservoir on the +y halo row of the middle tile
# row (ny = 25) and alone in the last one, z pressure with plane chunks that start and end
# next to the reservoirs.  (nz, ny, nx) shapes; x extents are multiples of 4.
TILED = [
    ("x_tiles", lambda: G.overlapping_spheres((6, 27, 136), 3.0, 0.55, seed=41), (2, 0, 0), 0, 0),
    ("y_halo_row", lambda: G.overlapping_spheres((7, 25, 72), 3.0, 0.6, seed=42), (0, 2, 1), 1, 0),
    ("z_chunks", lambda: G.overlapping_spheres((14, 20, 68), 2.5, 0.6, seed=43), (1, 0, 2), 2, 4),
]


@pytest.mark.parametrize("name,make,bc,a,sched", TILED, ids=[c[0] for c in TILED])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", 2e-5)])
def test_tiled_trajectory_matches_oracle(api, oracle_mod, name, make, bc, a, sched, precision, tol):
    """The tiled kernel's fixed-pressure variant (tile shape 1) against the oracle after 1,
    2 and 10 iterations, element by element."""
    mask = make()
    assert mask.shape[2] % 4 == 0
    dt = torch.float64 if precision == "fp64" else torch.float32
    dom = oracle_mod.Domain(mask, bc=bc)
    nf, _ = dom.tables()
    for n in (1, 2, 10):
        U, p = dom.zeros()
        dom.iterate(U, p, n, drive_dir=a, dt=api.time_step())
        u = torch.zeros((3,) + mask.shape, dtype=dt, device="cuda")
        pg = torch.zeros(mask.shape, dtype=dt, device="cuda")
        api.iterate(torch.from_numpy(mask).cuda(), u, pg, n, drive_dir=a, bc=bc, precision=precision,
                    schedule=sched)
        ug, pgn = u.double().cpu().numpy(), pg.double().cpu().numpy()
        su, sp = max(np.max(np.abs(U)), 1e-300), max(np.max(np.abs(p)), 1e-300)
        assert np.max(np.abs(ug - U)) <= tol * su, (n, "u")
        assert np.max(np.abs(pgn - p)) <= tol * sp, (n, "p")
        assert np.all(ug[nf == 0] == 0)


@pytest.mark.parametrize("name,make,bc,a,sched", TILED, ids=[c[0] for c in TILED])
def test_tiled_and_simple_kernels_agree(api, name, make, bc, a, sched):
    """Tiled fixed-pressure sweep against the one-thread-per-cell kernel (kernel=1) over
    200 FP64 iterations: equal up to rounding order."""
    mask = torch.from_numpy(make()).cuda()
    out = []
    for kernel in (0, 1):
        u = torch.zeros((3,) + tuple(mask.shape), dtype=torch.float64, device="cuda")
        p = torch.zeros(tuple(mask.shape), dtype=torch.float64, device="cuda")
        api.iterate(mask, u, p, 200, drive_dir=a, bc=bc, precision="fp64", kernel=kernel, schedule=sched)
        out.append((u.cpu().numpy(), p.cpu().numpy()))
    (u0, p0), (u1, p1) = out
    assert np.max(np.abs(u0 - u1)) <= 1e-12 * np.max(np.abs(u1))
    assert np.max(np.abs(p0 - p1)) <= 1e-12 * np.max(np.abs(p1))


def test_tiled_converged_k_and_statistics(api, oracle_mod):
    """Converged k of a multi-tile fixed-pressure domain on the tiled path (the statistics
    report tile shape 1), against the oracle."""
    mask = G.overlapping_spheres((8, 14, 72), 2.5, 0.6, seed=44)
    bc = (2, 0, 0)
    _, k_raw, _ = oracle_mod.ktensor(mask, bc=bc, tol=1e-13, check_every=100)
    r = api.solve_direction(torch.from_numpy(mask).cuda(), 0, fields=False, bc=bc, tol=1e-12,
                            precision="fp64", check_every=100)
    assert r["status"] == api.PM_OK
    assert r["stats"]["tile"] == 1
    assert r["k_col"][0] == pytest.approx(k_raw[0, 0], rel=1e-8)
    for i in (1, 2):
        assert abs(r["k_col"][i] - k_raw[i, 0]) <= 1e-8 * k_raw[0, 0]


@pytest.mark.parametrize("precision,tol,rel", [("fp64", 1e-12, 1e-8), ("fp32", 1e-8, 1e-5)])
def test_converged_k_matches_oracle(api, oracle_mod, precision, tol, rel):
    mask = G.overlapping_spheres((10, 9, 16), 2.0, 0.55, seed=35)
    bc = (2, 0, 0)
    k_ref, k_raw, _ = oracle_mod.ktensor(mask, bc=bc, tol=1e-13, check_every=100)
    r = api.solve_direction(torch.from_numpy(mask).cuda(), 0, fields=False, bc=bc, tol=tol,
                            precision=precision, check_every=100)
    assert r["status"] == api.PM_OK
    k = r["k_col"]
    assert k[0] == pytest.approx(k_raw[0, 0], rel=rel)
    for i in (1, 2):
        assert abs(k[i] - k_raw[i, 0]) <= rel * k_raw[0, 0]


def test_slit_exact_on_gpu(api):
    h, P = 3, 5
    mask = G.slit(8, h, P, nz=2)
    r = api.solve_direction(torch.from_numpy(mask).cuda(), 0, fields=True, bc=(2, 0, 0), tol=1e-13,
                            precision="fp64", check_every=100)
    assert r["k_col"][0] == pytest.approx(h * (2 * h * h + 1) / (24.0 * P), rel=1e-9)
    p = r["p"].double().cpu().numpy()
    # reservoirs hold p_in / p_out = +-(n - 1) / 2 x drive (Darcy units: dx = 1, drive 1)
    assert np.allclose(p[:, :h, 0], 3.5) and np.allclose(p[:, :h, -1], -3.5)


def test_blocked_axis_reports_not_percolating(api):
    mask = np.zeros((3, 4, 6), dtype=np.uint8)
    mask[:, :, 3] = 1
    r = api.solve_direction(torch.from_numpy(mask).cuda(), 0, fields=False, bc=(2, 0, 0), tol=1e-8)
    assert r["status"] == api.PM_ERR_NOT_PERCOLATING
    assert np.all(r["k_col"] == 0)
