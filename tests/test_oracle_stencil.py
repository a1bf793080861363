"""Pins of the oracle's wall stencil against the paper and closed forms (CPU only).

* Appendix B prints, for each wall case, a Taylor system: node values (or a wall,
  value 0) at given offsets from the node.  Here each system is solved symbolically
  from its offsets alone and compared with the oracle's coefficient table.
* Plane-channel (slit) and square-duct flows are exact on the grid: every node's
  stencil is exact for the quadratic profile, so k has a closed form.
"""
import numpy as np
import pytest
import sympy as sp

from paper_2407_19868_gb300 import geometry as G

# Appendix B, per case: the offsets (in grid spacings, along the perpendicular axis
# e_i, relative to the node whose second derivative is taken) of the points in the
# printed Taylor system, each tagged "wall" (value 0) or with the node offset whose
# value it is, and the highest derivative order kept in the expansion.
TAYLOR_SYSTEMS = {
    1: ([(-0.5, "wall"), (0.5, "wall")], 3),
    2: ([(-0.5, "wall"), (1, 1), (1.5, "wall")], 3),
    3: ([(-1.5, "wall"), (-1, -1), (0.5, "wall")], 3),
    4: ([(-0.5, "wall"), (1, 1), (2, 2)], 3),
    5: ([(-2, -2), (-1, -1), (0.5, "wall")], 3),
    6: ([(-1, -1), (1, 1)], 3),
    7: ([(-0.5, "wall"), (1, 1)], 2),
    8: ([(-1, -1), (0.5, "wall")], 2),
}


def _second_derivative_from_taylor(points, order):
    """Solve the Taylor system for d2v/dx2 as a linear combination of node values."""
    v = {m: sp.Symbol(f"v{m}") for m in (-2, -1, 0, 1, 2)}
    D = sp.symbols("D1:%d" % (order + 1))
    eqs = []
    for s, tag in points:
        s = sp.Rational(s).limit_denominator(4)
        expansion = v[0] + sum(D[k - 1] * s**k / sp.factorial(k) for k in range(1, order + 1))
        rhs = 0 if tag == "wall" else v[tag]
        eqs.append(sp.Eq(expansion, rhs))
    sol = sp.solve(eqs, D, dict=True)
    assert len(sol) == 1
    d2 = sp.expand(sol[0][D[1]])
    # D2 must not depend on the other (free) derivatives
    assert not (d2.free_symbols & set(D))
    return np.array([float(d2.coeff(v[m])) for m in (-2, -1, 0, 1, 2)])


@pytest.mark.parametrize("case", sorted(TAYLOR_SYSTEMS))
def test_case_coefficients_match_printed_taylor_systems(oracle_mod, case):
    pts, order = TAYLOR_SYSTEMS[case]
    expected = _second_derivative_from_taylor(pts, order)
    np.testing.assert_allclose(oracle_mod.case_coeffs(case), expected, rtol=0, atol=1e-15)


def test_classification_matches_case_geometry(oracle_mod):
    """Fig. neighborhoodCases: the case of a node is the one whose Taylor system uses
    exactly the fluid neighbours present (walls at +-1/2 where a neighbour is missing,
    one-sided systems use +-2 when it is fluid)."""
    for Fm2 in (0, 1):
        for Fm1 in (0, 1):
            for Fp1 in (0, 1):
                for Fp2 in (0, 1):
                    k = oracle_mod.classify(Fm2, Fm1, Fp1, Fp2)
                    pts, _ = TAYLOR_SYSTEMS[k]
                    used = {tag for _, tag in pts if tag != "wall"}
                    walls = {s for s, tag in pts if tag == "wall"}
                    # walls at -1/2 / +1/2 exactly when the -1 / +1 neighbour is not fluid
                    assert (-0.5 in walls) == (not Fm1)
                    assert (0.5 in walls) == (not Fp1)
                    # every node value used is a fluid neighbour
                    flags = {-2: Fm2, -1: Fm1, 1: Fp1, 2: Fp2}
                    assert all(flags[m] for m in used)
                    # a one-sided system uses the +-2 node iff it is fluid
                    if Fm1 and not Fp1:
                        assert (-2 in used) == bool(Fm2)
                    if Fp1 and not Fm1:
                        assert (2 in used) == bool(Fp2)


def _k_slit(h, P):
    # exact discrete k_xx of a slit with h fluid layers per period P (midpoint sum of
    # the parabola u = (Re f / 2) eta (h - eta) at eta = y + 1/2)
    return h * (2 * h * h + 1) / (24.0 * P)


@pytest.mark.parametrize("h,P", [(1, 2), (1, 3), (2, 4), (3, 5), (4, 7), (6, 9)])
def test_slit_poiseuille_exact(oracle_mod, h, P):
    m = G.slit(3, h, P, nz=2)  # slit normal along y, uniform along x and z
    dom = oracle_mod.Domain(m)
    r = dom.solve(0, tol=1e-14, check_every=200)
    k = r["q"][0] / oracle_mod.RE_PAPER
    assert r["iters"] > 0
    assert k == pytest.approx(_k_slit(h, P), rel=1e-11)
    assert abs(r["q"][1]) < 1e-15 and abs(r["q"][2]) < 1e-15


@pytest.mark.parametrize("flow,normal", [(0, 2), (1, 0), (1, 2), (2, 0), (2, 1)])
def test_slit_exact_all_orientations(oracle_mod, flow, normal):
    h, P = 3, 5
    prof = np.zeros(P, dtype=np.uint8)
    prof[h:] = 1
    shape = [3, 3, 3]
    shape[2 - normal] = P
    m = np.zeros(shape, dtype=np.uint8)
    idx = [None, None, None]
    idx[2 - normal] = slice(None)
    m[...] = prof[tuple(idx)]
    dom = oracle_mod.Domain(m)
    r = dom.solve(flow, tol=1e-14, check_every=200)
    assert r["q"][flow] / oracle_mod.RE_PAPER == pytest.approx(_k_slit(h, P), rel=1e-11)


def test_square_ducts_exact(oracle_mod):
    # 1x1 duct: case 1 in both perpendicular directions -> u = Re f / 16
    P = 3
    dom = oracle_mod.Domain(G.square_duct(2, 1, P))
    r = dom.solve(0, tol=1e-14, check_every=100)
    assert r["q"][0] / oracle_mod.RE_PAPER == pytest.approx(1.0 / (16 * P * P), rel=1e-12)
    # 2x2 duct: cases 2/3 in both directions -> u = 3 Re f / 16 on 4 nodes
    P = 4
    dom = oracle_mod.Domain(G.square_duct(2, 2, P))
    r = dom.solve(0, tol=1e-14, check_every=100)
    assert r["q"][0] / oracle_mod.RE_PAPER == pytest.approx(4 * 3.0 / (16 * P * P), rel=1e-12)


def test_wall_boundary_equals_solid_layer(oracle_mod):
    """An outer no-slip wall (Sec. 4) behaves like a solid layer outside the box: a slit
    whose two walls are the outer boundary gives the slit result with P = h."""
    h = 4
    m = np.zeros((2, h, 3), dtype=np.uint8)
    dom = oracle_mod.Domain(m, bc=(oracle_mod.PERIODIC, oracle_mod.WALL, oracle_mod.PERIODIC))
    r = dom.solve(0, tol=1e-14, check_every=200)
    assert r["q"][0] / oracle_mod.RE_PAPER == pytest.approx(_k_slit(h, h), rel=1e-11)
