"""GPU parity: the CUDA library (through its C ABI) against the FP64 CPU oracle.

Trajectories are compared element by element after 1, 2 and 10 iterations of
Algorithm 1 (same inputs, same order of updates); converged permeabilities are
compared per component.

Tolerances (derived from the arithmetic):
* FP64 fields: the GPU contracts a*b+c into FMAs and sums in another order, so each
  value differs by a few ulp per iteration -> 1e-11 relative to the field's max.
* FP32 fields: one FP32 rounding per operation, ~30 operations per update, errors do
  not grow within a few iterations -> 2e-5 relative to the field's max.
* Converged k, forms with FP64 accuracy (FP64 fields, FP32 sweeps + FP64 defect
  correction): every k_ij within its tolerance of its own oracle value, off-diagonal
  components included.
* Converged k, plain FP32 sweeps: the iteration stalls at the FP32 floor, about 1e-7 of
  the driven component's mean velocity; an off-diagonal component (1e-3 .. 1e-2 of the
  diagonal on these packs) carries that absolute error, so it is held to 1e-5 x max
  |k_ii| and the diagonal to 1e-5 of its own value.  Meeting 1e-5 on each off-diagonal
  needs the defect correction.
"""
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


def _gpu_iterate(api, mask, n, drive_dir, precision, bc=(0, 0, 0), U0=None, p0=None, **kw):
    dt = torch.float64 if precision == "fp64" else torch.float32
    nz, ny, nx = mask.shape
    u = torch.zeros((3, nz, ny, nx), dtype=dt, device="cuda")
    p = torch.zeros((nz, ny, nx), dtype=dt, device="cuda")
    if U0 is not None:
        u.copy_(torch.from_numpy(U0))
        p.copy_(torch.from_numpy(p0))
    api.iterate(torch.from_numpy(mask).cuda(), u, p, n, drive_dir=drive_dir, bc=bc, precision=precision, **kw)
    torch.cuda.synchronize()
    return u.double().cpu().numpy(), p.double().cpu().numpy()


def _oracle_iterate(oracle_mod, mask, n, drive_dir, bc=(0, 0, 0), U0=None, p0=None, dt=None):
    dom = oracle_mod.Domain(mask, bc=bc)
    U, p = dom.zeros()
    if U0 is not None:
        U[...] = U0
        p[...] = p0
    dom.iterate(U, p, n, drive_dir=drive_dir, dt=dt)
    return U, p


# shapes are (nz, ny, nx); the tiled kernel takes nx % 4 == 0 (ragged tiles included),
# the simple kernel every other shape
CASES = [
    ("odd_random", lambda: G.random_blocks((5, 7, 9), 0.3, seed=1), (0, 0, 0)),
    ("spheres_ragged", lambda: G.overlapping_spheres((11, 13, 36), 2.5, 0.6, seed=2), (0, 0, 0)),
    ("spheres_2tiles", lambda: G.overlapping_spheres((9, 21, 68), 3.0, 0.6, seed=9), (0, 0, 0)),
    ("walls_y", lambda: G.overlapping_spheres((8, 10, 12), 2.0, 0.7, seed=3), (0, 1, 0)),
    ("walls_xz", lambda: G.random_blocks((6, 9, 44), 0.25, seed=4), (1, 0, 1)),
    ("walls_xyz", lambda: G.random_blocks((7, 10, 40), 0.2, seed=10), (1, 1, 1)),
    ("thin_n1", lambda: G.random_blocks((1, 12, 40), 0.3, seed=5), (0, 0, 0)),
    ("thin_n2", lambda: G.random_blocks((2, 3, 16), 0.2, seed=6), (0, 0, 0)),
    ("odd_walls", lambda: G.random_blocks((4, 5, 17), 0.2, seed=7), (0, 1, 1)),
]


@pytest.mark.parametrize("name,make,bc", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("kernel", [1, 0], ids=["simple", "default"])
def test_trajectory_matches_oracle(api, oracle_mod, name, make, bc, precision, kernel):
    mask = make()
    dt = api.time_step()
    for n in (1, 2, 10):
        for drive_dir in (0, 2):
            Ug, pg = _gpu_iterate(api, mask, n, drive_dir, precision, bc=bc, kernel=kernel)
            Uo, po = _oracle_iterate(oracle_mod, mask, n, drive_dir, bc=bc, dt=dt)
            tol = 1e-11 if precision == "fp64" else 2e-5
            su, sp = max(np.abs(Uo).max(), 1e-300), max(np.abs(po).max(), 1e-300)
            np.testing.assert_allclose(Ug, Uo, rtol=0, atol=tol * su, err_msg=f"u n={n} dir={drive_dir}")
            np.testing.assert_allclose(pg, po, rtol=0, atol=tol * sp, err_msg=f"p n={n} dir={drive_dir}")
            nf, _ = oracle_mod.Domain(mask, bc=bc).tables()
            assert np.all(Ug[nf == 0] == 0.0)


def test_warm_start_trajectory(api, oracle_mod):
    mask = G.overlapping_spheres((10, 12, 14), 2.5, 0.65, seed=8)
    rng = G.rng(9)
    U0 = rng.standard_normal((3,) + mask.shape) * 1e-3
    p0 = rng.standard_normal(mask.shape)
    Ug, pg = _gpu_iterate(api, mask, 3, 1, "fp64", U0=U0, p0=p0)
    Uo, po = _oracle_iterate(oracle_mod, mask, 3, 1, U0=np.where(oracle_mod.Domain(mask).tables()[0] == 1, U0, 0.0),
                             p0=np.where(mask == 0, p0, 0.0), dt=api.time_step())
    np.testing.assert_allclose(Ug, Uo, rtol=0, atol=1e-11 * np.abs(Uo).max())
    np.testing.assert_allclose(pg, po, rtol=0, atol=1e-11 * np.abs(po).max())


@pytest.fixture(scope="module")
def config1():
    # 32^3 periodic, overlapping spheres r = 4 to porosity 0.70, seed 1
    return G.overlapping_spheres((32, 32, 32), 4.0, 0.70, seed=1)


@pytest.fixture(scope="module")
def config1_oracle(oracle_mod, config1):
    r = oracle_mod.Domain(config1).solve(0, tol=1e-11, check_every=100)
    assert r["iters"] > 0
    return r["q"] / oracle_mod.RE_PAPER


@pytest.mark.parametrize("precision,tol,rel", [("fp64", 1e-11, 1e-9), ("fp32", 1e-9, 1e-5)])
def test_config1_kxx_converged(api, config1, config1_oracle, precision, tol, rel):
    r = api.solve_direction(config1, 0, tol=tol, precision=precision, check_every=100)
    assert r["status"] == api.PM_OK
    k = r["k_col"]
    ko = config1_oracle
    assert k[0] == pytest.approx(ko[0], rel=rel)
    np.testing.assert_allclose(k[1:], ko[1:], rtol=0, atol=rel * abs(ko[0]))
    if precision == "fp64":
        np.testing.assert_allclose(k, ko, rtol=1e-6)  # each component against its own value
    # returned fields: Darcy-scaled (drive = dx = mu = 1 -> mean u_x = k_xx)
    u = r["u"].double()
    assert float(u[0].mean()) == pytest.approx(k[0], rel=1e-6)


def test_full_tensor_batched(api, oracle_mod):
    mask = G.overlapping_spheres((20, 24, 28), 3.0, 0.6, seed=12)
    k_sym_o, k_raw_o, _ = oracle_mod.ktensor(mask, tol=1e-11)
    scale = np.abs(np.diag(k_raw_o)).max()
    for prec, tol, rel in (("fp64", 1e-11, 1e-9), ("fp32", 1e-9, 1e-5)):
        r = api.permeability_tensor(mask, tol=tol, precision=prec)
        assert r["status"] == api.PM_OK
        np.testing.assert_allclose(r["k_raw"], k_raw_o, rtol=0, atol=rel * scale)
        np.testing.assert_allclose(r["k"], k_sym_o, rtol=0, atol=rel * scale)
        np.testing.assert_allclose(np.diag(r["k"]), np.diag(k_sym_o), rtol=rel)
        if prec == "fp64":
            np.testing.assert_allclose(r["k_raw"], k_raw_o, rtol=1e-6)  # each against its own value


def test_non_percolating_axis(api):
    m = G.slit(8, 3, 6, nz=4)  # walls normal to y: no flow along y
    r = api.permeability_tensor(m, tol=1e-10, precision="fp64")
    assert r["status"] == api.PM_ERR_NOT_PERCOLATING
    assert not r["stats"][1]["percolates"]
    assert np.all(r["k"][1, :] == 0) and np.all(r["k"][:, 1] == 0)
    assert r["k"][0, 0] == pytest.approx(3 * (2 * 9 + 1) / (24 * 6), rel=1e-9)


def test_slit_exact_on_gpu(api):
    for h, P in ((1, 3), (2, 4), (5, 8)):
        m = G.slit(32, h, P, nz=3)
        r = api.solve_direction(m, 0, tol=1e-13, precision="fp64", check_every=100)
        assert r["k_col"][0] == pytest.approx(h * (2 * h * h + 1) / (24 * P), rel=1e-10)


def test_no_fluid_is_an_error(api):
    with pytest.raises(api.PMError) as e:
        api.solve_direction(np.ones((4, 4, 4), dtype=np.uint8), 0)
    assert e.value.status == api.PM_ERR_NO_FLUID


@pytest.mark.slow
def test_config2_full_size_batched_launch(api, oracle_mod):
    """256^3 benchmark geometry in the benchmark's launch configuration (three drives
    batched per sweep, FP32 fields, graph windows): after exactly 21 iterations
    (max_iter stops it) the mean velocities of each drive match the oracle's after the
    same 21 iterations."""
    mask, _ = G.rsa_sphere_pack((256, 256, 256), 10.0, 0.3, 4.0, 25.0, 0.38, seed=2)
    r = api.permeability_tensor(torch.from_numpy(mask).cuda(), tol=1e-12, check_every=10, max_iter=21, autotune=0)
    assert r["status"] == api.PM_ERR_NOT_CONVERGED
    assert all(s["iters"] == 21 for s in r["stats"])
    dom = oracle_mod.Domain(mask)
    dt = api.time_step()
    K = np.zeros((3, 3))
    for j in range(3):
        U, p = dom.zeros()
        dom.iterate(U, p, 21, drive_dir=j, dt=dt)
        K[:, j] = dom.mean_velocity(U) / oracle_mod.RE_PAPER
    scale = np.abs(np.diag(K)).max()
    np.testing.assert_allclose(r["k_raw"], K, rtol=0, atol=1e-5 * scale)
    np.testing.assert_allclose(np.diag(r["k_raw"]), np.diag(K), rtol=1e-5)


def test_defect_correction_config1(api, config1, config1_oracle):
    """FP32 sweeps + FP64 defect correction reach the oracle's converged k far below the
    FP32 floor: 1e-8 relative on k_xx, off-diagonals within 1e-8 of k_xx."""
    r = api.solve_direction(config1, 0, tol=1e-11, precision="fp32_dc64", check_every=100)
    assert r["status"] == api.PM_OK
    assert r["stats"]["dc_rounds"] >= 1
    k, ko = r["k_col"], config1_oracle
    assert k[0] == pytest.approx(ko[0], rel=1e-8)
    np.testing.assert_allclose(k[1:], ko[1:], rtol=0, atol=1e-8 * abs(ko[0]))
    np.testing.assert_allclose(k, ko, rtol=1e-6)  # each component against its own value


def test_defect_correction_full_tensor(api, oracle_mod):
    mask = G.overlapping_spheres((20, 24, 28), 3.0, 0.6, seed=12)
    _, k_raw_o, _ = oracle_mod.ktensor(mask, tol=1e-12)
    r = api.permeability_tensor(mask, tol=1e-11, precision="fp32_dc64")
    assert r["status"] == api.PM_OK
    scale = np.abs(np.diag(k_raw_o)).max()
    np.testing.assert_allclose(r["k_raw"], k_raw_o, rtol=0, atol=1e-8 * scale)
    np.testing.assert_allclose(r["k_raw"], k_raw_o, rtol=1e-6)  # each component against its own value


@pytest.mark.slow
def test_config2_ktensor_against_oracle_reference(api):
    """256^3 benchmark geometry, full tensor in the benchmark's launch configuration with
    defect correction, against the oracle's converged columns stored by
    tests/golden/make_reference.py (the mask hash must match): 1e-5 relative on every
    component, off-diagonals included."""
    import json
    import os
    ref = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "reference_k.json")))
    if "config2" not in ref:
        pytest.skip("oracle reference for the 256^3 geometry not generated yet")
    ref = ref["config2"]
    mask, _ = G.rsa_sphere_pack((256, 256, 256), 10.0, 0.3, 4.0, 25.0, 0.38, seed=2)
    assert G.mask_sha256(mask) == ref["sha256"]
    r = api.permeability_tensor(torch.from_numpy(mask).cuda(), tol=1e-8, precision="fp32_dc64")
    assert r["status"] == api.PM_OK
    for j, col in ref["columns"].items():
        ko = np.array(col["k_col"])
        kg = r["k_raw"][:, int(j)]
        np.testing.assert_allclose(kg, ko, rtol=1e-5, atol=0)


def test_divergence_and_iteration_limit_are_reported(api):
    """Failure detection on the host: a pseudo-time step five times the stability bound
    blows the iteration up (a finite overflow to Inf/NaN, no device fault) and comes back
    as PM_ERR_DIVERGED; an iteration limit gives PM_ERR_NOT_CONVERGED with valid fields."""
    mask = G.overlapping_spheres((16, 16, 16), 3.0, 0.6, seed=71)
    with pytest.raises(api.PMError) as e:
        api.solve_direction(mask, 0, dt_safety=5.0, check_every=50, max_iter=20000)
    assert e.value.status == api.PM_ERR_DIVERGED
    r = api.solve_direction(mask, 0, tol=1e-14, check_every=10, max_iter=51, autotune=0)
    assert r["status"] == api.PM_ERR_NOT_CONVERGED
    assert r["stats"]["iters"] == 51
    assert bool(torch.isfinite(r["u"]).all())


@pytest.mark.parametrize("tile", [1, 2, 3])
@pytest.mark.parametrize("schedule", [-1, 1, 2, 5, 13, 40])
@pytest.mark.parametrize("bc", [(0, 0, 0), (1, 0, 1), (0, 1, 0)], ids=["periodic", "walls_xz", "walls_y"])
def test_tiles_and_schedules_give_identical_fields(api, tile, schedule, bc):
    """Every tile shape (64 x 12 cells with two or four cells per thread, 64 x 8 with four)
    and every work split (persistent CTAs, plane chunks of any length, including chunks
    shorter than the kernel's pipeline) does the same arithmetic per cell: the fields
    after 11 iterations are bit-identical to the default shape and split.  The domain has
    ragged tiles in x and y."""
    mask = G.overlapping_spheres((27, 19, 72), 3.0, 0.6, seed=21)
    ref = _gpu_iterate(api, mask, 11, 1, "fp32", bc=bc)
    got = _gpu_iterate(api, mask, 11, 1, "fp32", bc=bc, schedule=schedule, tile=tile)
    assert np.array_equal(ref[0], got[0]) and np.array_equal(ref[1], got[1])


@pytest.mark.parametrize("tile", [1, 2, 3])
@pytest.mark.parametrize("schedule,split", [(5, 2), (5, 4), (10, 3), (10, 4), (40, 2), (40, 4), (40, 7)])
@pytest.mark.parametrize("bc", [(0, 0, 0), (1, 0, 1)], ids=["periodic", "walls_xz"])
def test_split_last_chunk_gives_identical_fields(api, tile, schedule, split, bc):
    """Plane chunks whose last chunk per column is cut into shorter pieces (27 planes:
    chunks of 5 with a last chunk of 2, chunks of 10 with a last one of 7, one chunk of
    27 cut into up to 7 pieces) give fields bit-identical to the unsplit schedule."""
    mask = G.overlapping_spheres((27, 19, 72), 3.0, 0.6, seed=21)
    ref = _gpu_iterate(api, mask, 11, 1, "fp32", bc=bc)
    got = _gpu_iterate(api, mask, 11, 1, "fp32", bc=bc, schedule=schedule, schedule_split=split, tile=tile)
    assert np.array_equal(ref[0], got[0]) and np.array_equal(ref[1], got[1])


def test_split_last_chunk_fp64_and_reported(api):
    """FP64 fields with a split last chunk are bit-identical too; a solve reports the
    split it ran with and converges to the same k."""
    mask = G.overlapping_spheres((27, 19, 72), 3.0, 0.6, seed=21)
    ref = _gpu_iterate(api, mask, 7, 0, "fp64")
    got = _gpu_iterate(api, mask, 7, 0, "fp64", schedule=10, schedule_split=4)
    assert np.array_equal(ref[0], got[0]) and np.array_equal(ref[1], got[1])
    d = torch.from_numpy(mask).cuda()
    a = api.solve_direction(d, 0, fields=False, tol=1e-7, schedule=10, tile=1)
    b = api.solve_direction(d, 0, fields=False, tol=1e-7, schedule=10, schedule_split=4, tile=1)
    assert a["stats"]["schedule_split"] == 1 and b["stats"]["schedule_split"] == 4
    assert a["stats"]["iters"] == b["stats"]["iters"]
    # the FP64 block sums group the cells by CTA: equal up to summation order
    np.testing.assert_allclose(a["k_col"], b["k_col"], rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("tile", [2, 3])
def test_tiles_with_source_and_drag_terms(api, tile):
    """The source (defect-correction) and drag (adjoint) variants of the wide shapes
    against the first shape: the defect-corrected tensor and the tensor with a drag field
    agree to the convergence noise of the window criterion."""
    mask = G.overlapping_spheres((20, 24, 28), 3.0, 0.6, seed=12)
    a = api.permeability_tensor(mask, tol=1e-11, precision="dc64", tile=1)
    b = api.permeability_tensor(mask, tol=1e-11, precision="dc64", tile=tile)
    assert b["stats"][0]["tile"] == tile
    np.testing.assert_allclose(b["k_raw"], a["k_raw"], rtol=1e-7, atol=1e-12)
    alpha = torch.from_numpy(G.rng(5).random(mask.shape) * 0.5).float().cuda()
    ka = api.sensitivity(mask, None, alpha=alpha, tol=1e-9, tile=1)["k_raw"]
    kb = api.sensitivity(mask, None, alpha=alpha, tol=1e-9, tile=tile)["k_raw"]
    np.testing.assert_allclose(kb, ka, rtol=1e-6, atol=1e-10)


def test_schedule_reported_and_converged_k_unchanged(api):
    mask = G.overlapping_spheres((40, 24, 32), 3.0, 0.6, seed=22)
    d = torch.from_numpy(mask).cuda()
    a = api.solve_direction(d, 0, fields=False, tol=1e-7, schedule=-1, tile=1)
    b = api.solve_direction(d, 0, fields=False, tol=1e-7, schedule=7, tile=1)
    assert a["stats"]["schedule"] == -1 and b["stats"]["schedule"] == 7
    assert a["stats"]["tile"] == 1 and b["stats"]["tile"] == 1
    assert a["stats"]["iters"] == b["stats"]["iters"]
    np.testing.assert_allclose(a["k_col"], b["k_col"], rtol=1e-12, atol=1e-14)


def test_defect_correction_on_a_slowly_converging_geometry(api):
    """A dilute obstacle converges slowly (each window shrinks the change by only a few
    per cent); the defect correction must not mistake that for the FP32 floor."""
    m = G.sc_sphere(32, 4.0)
    d = torch.from_numpy(m).cuda()
    r64 = api.solve_direction(d, 0, fields=False, precision="fp64", tol=1e-10, check_every=100)
    rdc = api.solve_direction(d, 0, fields=False, precision="dc64", tol=1e-9, check_every=100)
    assert r64["status"] == api.PM_OK and rdc["status"] == api.PM_OK
    assert rdc["k_col"][0] == pytest.approx(r64["k_col"][0], rel=1e-7)


@pytest.mark.parametrize("geo", ["pack", "dilute"])
def test_defect_correction_from_the_extrapolated_error(api, oracle_mod, geo):
    """Starting the first correction solve from the FP32 phase's geometric-tail error
    estimate changes only the starting point: the tensor meets the same criterion and
    agrees with the oracle (and with the zero start) per component."""
    if geo == "pack":
        mask = G.overlapping_spheres((20, 24, 28), 3.0, 0.6, seed=12)
        _, k_ref, _ = oracle_mod.ktensor(mask, tol=1e-11)
        a = api.permeability_tensor(mask, tol=1e-9, precision="dc64", dc_extrapolate=0)
        b = api.permeability_tensor(mask, tol=1e-9, precision="dc64", dc_extrapolate=1)
        ka, kb = np.asarray(a["k_raw"]), np.asarray(b["k_raw"])
    else:
        mask = G.sc_sphere(32, 4.0)
        k_ref = api.solve_direction(mask, 0, fields=False, precision="fp64", tol=1e-10, check_every=100)["k_col"]
        a = api.solve_direction(mask, 0, fields=False, precision="dc64", tol=1e-9, check_every=100, dc_extrapolate=0)
        b = api.solve_direction(mask, 0, fields=False, precision="dc64", tol=1e-9, check_every=100, dc_extrapolate=1)
        ka, kb = np.asarray(a["k_col"]), np.asarray(b["k_col"])
    assert a["status"] == api.PM_OK and b["status"] == api.PM_OK
    scale = np.abs(k_ref).max()
    np.testing.assert_allclose(kb, k_ref, rtol=0, atol=1e-7 * scale)
    np.testing.assert_allclose(kb, ka, rtol=0, atol=1e-7 * scale)


@pytest.mark.slow
@pytest.mark.parametrize("drive_dir", [0, 2])
def test_config2_full_size_fields_after_21_iterations(api, oracle_mod, drive_dir):
    """256^3 benchmark geometry in the benchmark's work split (chunks of 64 planes): the
    FP32 fields after 21 iterations match the oracle's element by element."""
    mask, _ = G.rsa_sphere_pack((256, 256, 256), 10.0, 0.3, 4.0, 25.0, 0.38, seed=2)
    Ug, pg = _gpu_iterate(api, mask, 21, drive_dir, "fp32", schedule=64)
    Uo, po = _oracle_iterate(oracle_mod, mask, 21, drive_dir, dt=api.time_step())
    np.testing.assert_allclose(Ug, Uo, rtol=0, atol=2e-5 * np.abs(Uo).max())
    np.testing.assert_allclose(pg, po, rtol=0, atol=2e-5 * np.abs(po).max())


@pytest.mark.parametrize("precision,tile", [("fp32", 1), ("fp32", 2), ("fp32", 3), ("fp64", 1)])
def test_persistent_rounds_trajectory(api, oracle_mod, precision, tile):
    """1024 x 640 x 6 cells make 16 x 54 = 864 tile columns, more than the persistent
    grid (2 CTAs per SM for FP32, 1 for FP64): whole-column rounds in lockstep run
    before the equal plane ranges of the remaining columns.  Element-wise parity with
    the oracle after 1, 2 and 10 iterations."""
    mask = G.random_blocks((6, 640, 1024), 0.3, seed=41)
    dt = api.time_step()
    tol = 1e-11 if precision == "fp64" else 2e-5
    for n in (1, 2, 10):
        for drive_dir in (0, 1):
            Ug, pg = _gpu_iterate(api, mask, n, drive_dir, precision, schedule=-1, tile=tile)
            Uo, po = _oracle_iterate(oracle_mod, mask, n, drive_dir, dt=dt)
            np.testing.assert_allclose(Ug, Uo, rtol=0, atol=tol * np.abs(Uo).max(), err_msg=f"u n={n}")
            np.testing.assert_allclose(pg, po, rtol=0, atol=tol * np.abs(po).max(), err_msg=f"p n={n}")


@pytest.mark.slow
def test_beyond_2_31_cells_replicates_the_unit_cell(api, oracle_mod):
    """A periodic 64^3 cell (checked against the oracle) tiled 21 x 21 x 19 times gives
    1344 x 1344 x 1216 = 2.2e9 cells, beyond 32-bit cell indices.  Every cell does the
    same arithmetic as its image in the unit cell, so after 10 FP32 iterations each
    replica of the large fields is bit-identical to the unit cell's fields."""
    cell = G.overlapping_spheres((64, 64, 64), 4.0, 0.6, seed=51)
    n = 10
    u1, p1 = _gpu_iterate(api, cell, n, 0, "fp32")
    Uo, po = _oracle_iterate(oracle_mod, cell, n, 0, dt=api.time_step())
    np.testing.assert_allclose(u1, Uo, rtol=0, atol=2e-5 * np.abs(Uo).max())
    reps = (19, 21, 21)
    big = torch.from_numpy(cell).cuda().repeat(reps)
    assert big.numel() > 2 ** 31
    u = torch.zeros((3,) + tuple(big.shape), dtype=torch.float32, device="cuda")
    p = torch.zeros(tuple(big.shape), dtype=torch.float32, device="cuda")
    api.iterate(big, u, p, n, drive_dir=0, precision="fp32")
    torch.cuda.synchronize()
    del big
    ref_u = torch.from_numpy(u1).float().cuda()
    ref_p = torch.from_numpy(p1).float().cuda()
    for d in range(3):
        v = u[d].view(19, 64, 21, 64, 21, 64)
        assert bool((v == ref_u[d][None, :, None, :, None, :]).all()), d
    v = p.view(19, 64, 21, 64, 21, 64)
    assert bool((v == ref_p[None, :, None, :, None, :]).all())


@pytest.mark.parametrize("field_memory", [1, 2])
def test_fields_in_host_memory_bit_identical(api, field_memory):
    """Ping-pong field buffers in pinned host memory (one or both), which the kernels read
    and write directly: the same fields bit for bit as in device memory, and the same
    defect-corrected tensor."""
    mask = G.overlapping_spheres((20, 36, 64), 3.0, 0.6, seed=23)
    ref = _gpu_iterate(api, mask, 9, 0, "fp32")
    got = _gpu_iterate(api, mask, 9, 0, "fp32", field_memory=field_memory)
    assert np.array_equal(ref[0], got[0]) and np.array_equal(ref[1], got[1])
    api.permeability_tensor(mask, tol=1e-9, precision="dc64")  # the shape's tuning runs here
    a = api.permeability_tensor(mask, tol=1e-9, precision="dc64")
    b = api.permeability_tensor(mask, tol=1e-9, precision="dc64", field_memory=field_memory)
    assert a["stats"][0]["iters"] == b["stats"][0]["iters"]
    np.testing.assert_array_equal(a["k_raw"], b["k_raw"])


@pytest.mark.slow
def test_large_domain_generator_at_192_against_oracle_reference(api):
    """The large-domain workload (periodic Boolean model of spheres, radii U[15, 25],
    porosity 0.35, seed 5) at 192^3, generated on the GPU, in the large-domain launch
    configuration (one drive, no percolation search), against the oracle's converged k
    column (tests/golden/make_reference.py, the same mask rasterised on the CPU):
    defect-corrected to 1e-6 of each component, plain FP32 to 1e-5 of k_xx."""
    import json
    import os
    ref = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "reference_k.json")))
    if "config5_192" not in ref:
        pytest.skip("oracle reference not generated")
    ref = ref["config5_192"]
    mask, _ = G.boolean_spheres_gpu(192, 15.0, 25.0, 0.35, seed=5)
    assert G.mask_sha256(mask.cpu().numpy()) == ref["sha256"]
    ko = np.array(ref["columns"]["0"]["k_col"])
    dc = api.solve_direction(mask, 0, fields=False, tol=1e-9, check_percolation=0, precision="dc64")
    assert dc["status"] == api.PM_OK
    np.testing.assert_allclose(dc["k_col"], ko, rtol=1e-6)
    fp = api.solve_direction(mask, 0, fields=False, tol=1e-7, check_percolation=0, precision="fp32")
    assert fp["k_col"][0] == pytest.approx(ko[0], rel=1e-5)
