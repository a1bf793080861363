"""Pins of the oracle's fixed-pressure inlet/outlet boundary (CPU only).

Sec. 4 names a fixed pressure in the main flow direction but gives no discrete form.
Reading used here: the first and last cell layers along the pressure axis are
reservoirs with fixed pressures and no cross flow; the inlet and outlet faces take a
zero-gradient axial neighbour.  What fixes it independently of the code:

* fully developed flows (slit, square ducts) are uniform along the axis, so the
  reading must reproduce their exact periodic results (closed forms);
* the iteration's fixed point equals a dense solve of the steady equations;
* mirroring the geometry along the axis keeps k_aa and flips the sign of the cross
  components (mirror, then Stokes reversibility; the discrete operator maps wall case
  4 onto 5 and 2 onto 3);
* continuity: equal flux through every face plane at the fixed point;
* a long chain of periodic cells approaches the periodic k as the entrance and exit
  regions become a smaller share of the length.
"""
import numpy as np
import pytest

from paper_2407_19868_gb300 import geometry as G

from test_oracle_solver import _solve_direct


def _k_slit(h, P):
    return h * (2 * h * h + 1) / (24.0 * P)


def _kcol(oracle_mod, m, bc, tol=1e-13, check_every=50):
    dom = oracle_mod.Domain(m, bc=bc)
    k, k_raw, runs = oracle_mod.ktensor(m, dom=dom, tol=tol, check_every=check_every)
    return k_raw[:, dom.pax], runs[dom.pax], dom


@pytest.mark.parametrize("h,P", [(1, 3), (2, 4), (3, 5), (5, 7)])
def test_slit_exact_with_fixed_pressure(oracle_mod, h, P):
    m = G.slit(6, h, P, nz=2)  # flow along x between walls normal to y
    k, r, _ = _kcol(oracle_mod, m, (oracle_mod.PRESSURE, 0, 0))
    assert r["iters"] > 0
    assert k[0] == pytest.approx(_k_slit(h, P), rel=1e-10)
    assert abs(k[1]) < 1e-13 and abs(k[2]) < 1e-13


def test_slit_exact_along_z_with_side_walls(oracle_mod):
    # flow along z, slit normal along x, the slit walls are the outer walls (P = h)
    h = 4
    m = np.zeros((5, 3, h), dtype=np.uint8)
    k, _, _ = _kcol(oracle_mod, m, (oracle_mod.WALL, 0, oracle_mod.PRESSURE))
    assert k[2] == pytest.approx(_k_slit(h, h), rel=1e-10)


def test_square_ducts_exact_with_fixed_pressure(oracle_mod):
    P = 4
    k, _, _ = _kcol(oracle_mod, G.square_duct(5, 1, P), (oracle_mod.PRESSURE, 0, 0))
    assert k[0] == pytest.approx(1.0 / 16.0 / (P * P), rel=1e-10)
    k, _, _ = _kcol(oracle_mod, G.square_duct(5, 2, P), (oracle_mod.PRESSURE, 0, 0))
    assert k[0] == pytest.approx(4 * 3.0 / 16.0 / (P * P), rel=1e-10)


@pytest.mark.parametrize("bc", [(2, 0, 0), (0, 1, 2)], ids=["x_periodic", "z_wall_y"])
def test_fixed_point_equals_direct_solve(oracle_mod, bc):
    m = G.random_blocks((5, 4, 6), 0.25, seed=13)
    dom = oracle_mod.Domain(m, bc=bc)
    j = dom.pax
    U_ref = _solve_direct(dom, j)
    r = dom.solve(j, tol=1e-14, check_every=100)
    assert r["iters"] > 0
    scale = np.max(np.abs(U_ref))
    assert scale > 0
    assert np.max(np.abs(r["U"] - U_ref)) < 1e-9 * scale


def test_reservoirs_hold_fixed_pressure_and_no_cross_flow(oracle_mod):
    m = G.random_blocks((6, 5, 7), 0.2, seed=3)
    dom = oracle_mod.Domain(m, bc=(oracle_mod.PRESSURE, 0, 0))
    U, p = dom.zeros()
    dom.iterate(U, p, 40, drive_dir=0, drive=2.0)
    nx = m.shape[2]
    open0, open1 = m[:, :, 0] == 0, m[:, :, -1] == 0
    assert np.all(p[:, :, 0][open0] == 2.0 * (nx - 1) / 2)
    assert np.all(p[:, :, -1][open1] == -2.0 * (nx - 1) / 2)
    for d in (1, 2):  # no cross flow in the reservoir layers
        assert np.all(U[d][:, :, 0] == 0) and np.all(U[d][:, :, -1] == 0)
    assert np.all(U[0][:, :, -1] == 0)  # outlet layer's +x face lies outside the box


def test_equal_flux_through_every_face_plane(oracle_mod):
    m = G.overlapping_spheres((6, 6, 10), 1.5, 0.6, seed=8)
    _, r, dom = _kcol(oracle_mod, m, (oracle_mod.PRESSURE, 0, 0))
    flux = r["U"][0].sum(axis=(0, 1))[:-1]  # the nx - 1 face planes between the layers
    assert np.max(np.abs(flux - flux.mean())) < 1e-9 * abs(flux.mean())


def test_mirror_along_the_axis(oracle_mod):
    m = G.random_blocks((6, 6, 8), 0.25, seed=21)
    bc = (oracle_mod.PRESSURE, 0, 0)
    k1, _, _ = _kcol(oracle_mod, m, bc)
    k2, _, _ = _kcol(oracle_mod, np.ascontiguousarray(m[:, :, ::-1]), bc)
    assert abs(k1[1]) > 1e-4 * k1[0]  # the cross term is not trivially zero
    assert k2[0] == pytest.approx(k1[0], rel=1e-9)
    for d in (1, 2):
        assert k2[d] == pytest.approx(-k1[d], abs=1e-9 * abs(k1[0]))


def test_long_chain_approaches_periodic_k(oracle_mod):
    unit = G.random_blocks((4, 4, 6), 0.2, seed=5)
    kp = oracle_mod.ktensor(unit, dirs=(0,), tol=1e-13)[1][0, 0]
    errs = []
    for R in (2, 4, 8):
        k, _, _ = _kcol(oracle_mod, np.ascontiguousarray(np.tile(unit, (1, 1, R))), (oracle_mod.PRESSURE, 0, 0))
        errs.append(abs(k[0] / kp - 1))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.5 * errs[0]


def test_k_independent_of_drive(oracle_mod):
    m = G.random_blocks((4, 5, 6), 0.2, seed=9)
    dom = oracle_mod.Domain(m, bc=(oracle_mod.PRESSURE, 0, 0))
    q1 = dom.solve(0, tol=1e-13, check_every=50, drive=1.0)["q"]
    q3 = dom.solve(0, tol=1e-13, check_every=50, drive=3.0)["q"]
    np.testing.assert_allclose(q3, 3.0 * q1, rtol=1e-9, atol=1e-15)


def test_percolation_along_the_pressure_axis(oracle_mod):
    m = np.zeros((3, 3, 6), dtype=np.uint8)
    assert oracle_mod.Domain(m, bc=(2, 0, 0)).percolation()[0]
    b = m.copy()
    b[:, :, 3] = 1  # a closed plane
    assert not oracle_mod.Domain(b, bc=(2, 0, 0)).percolation()[0]
    # open only through a sideways move inside the inlet reservoir: not a path
    c = np.ones((1, 4, 5), dtype=np.uint8)
    c[0, 0, 0] = c[0, 1, 0] = 0
    c[0, 1, 1:] = 0
    c[0, 1, 1] = 1
    c[0, 0, 1] = 0
    c[0, 0, 2] = 1
    assert not oracle_mod.Domain(c, bc=(2, 0, 0)).percolation()[0]


def test_invalid_fixed_pressure_setups(oracle_mod):
    m = np.zeros((4, 4, 4), dtype=np.uint8)
    with pytest.raises(ValueError):
        oracle_mod.Domain(m, bc=(2, 2, 0))
    with pytest.raises(ValueError):
        oracle_mod.Domain(np.zeros((4, 4, 2), dtype=np.uint8), bc=(2, 0, 0))
    dom = oracle_mod.Domain(m, bc=(2, 0, 0))
    with pytest.raises(ValueError):
        dom.solve(1)
