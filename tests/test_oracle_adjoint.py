"""Pins of the oracle's adjoint (CPU only): the transposed viscous operator is the
transpose (dot-product identity), the adjoint sensitivity equals finite differences of
k with respect to the drag alpha, and for a symmetric stencil dk_ii/d alpha reduces to
-(1/(2 Re^2 N)) sum u^(i) . u^(i) over the faces of each cell."""
import numpy as np
import pytest

from paper_2407_19868_gb300 import geometry as G


def test_transposed_operator_is_the_transpose(oracle_mod):
    m = G.random_blocks((5, 6, 7), 0.3, seed=41)
    dom = oracle_mod.Domain(m)
    nf, _ = dom.tables()
    g = G.rng(42)
    a = np.where(nf == 1, g.standard_normal(nf.shape), 0.0)
    b = np.where(nf == 1, g.standard_normal(nf.shape), 0.0)
    p0 = np.zeros(m.shape)
    La = dom.momentum_residual(a, p0, drive_dir=None)
    LTb = dom.momentum_residual(b, p0, drive_dir=None, transposed=True)
    lhs, rhs = float(np.sum(b * La)), float(np.sum(LTb * a))
    assert lhs == pytest.approx(rhs, rel=1e-13)
    # the operator is not symmetric (one-sided wall cases), so the test has teeth
    Lb = dom.momentum_residual(b, p0, drive_dir=None)
    assert abs(np.sum(LTb * a) - np.sum(Lb * a)) > 1e-6 * abs(rhs)


def _k(oracle_mod, dom, j, alpha):
    return dom.solve(j, tol=1e-13, check_every=100, alpha=alpha)["q"] / oracle_mod.RE_PAPER


@pytest.mark.slow
def test_adjoint_matches_finite_differences(oracle_mod):
    m = G.overlapping_spheres((8, 9, 10), 2.2, 0.65, seed=43)
    dom = oracle_mod.Domain(m)
    alpha = G.rng(44).random(m.shape) * 0.3
    w = np.zeros((3, 3))
    w[0, 0], w[1, 0], w[2, 1] = 1.0, 0.7, -0.4
    dJ, J, k = oracle_mod.sensitivity(m, w, alpha=alpha, dom=dom)
    fluid = np.argwhere(m == 0)
    pick = fluid[G.rng(45).choice(len(fluid), 5, replace=False)]
    h = 1e-3
    for c in pick:
        ap, am = alpha.copy(), alpha.copy()
        ap[tuple(c)] += h
        am[tuple(c)] -= h
        Jp = sum(w[i, j] * _k(oracle_mod, dom, j, ap)[i] for i in range(3) for j in range(3) if w[i, j])
        Jm = sum(w[i, j] * _k(oracle_mod, dom, j, am)[i] for i in range(3) for j in range(3) if w[i, j])
        fd = (Jp - Jm) / (2 * h)
        assert dJ[tuple(c)] == pytest.approx(fd, rel=1e-5, abs=1e-9 * np.abs(dJ).max())


def test_symmetric_stencil_identity(oracle_mod):
    """Channels at most two voxels wide use only cases 1, 2, 3, 6, whose stencil is
    symmetric: the adjoint field equals the forward one."""
    m = np.ones((4, 6, 6), dtype=np.uint8)
    m[:, 1:3, :] = 0      # a 2-voxel channel along x ...
    m[1:3, :, 4] = 0      # ... joined by a 2-voxel channel along y
    dom = oracle_mod.Domain(m)
    _, pc = dom.tables()
    assert not np.any((pc == 4) | (pc == 5))
    w = np.zeros((3, 3))
    w[0, 0] = 1.0
    dJ, _, _ = oracle_mod.sensitivity(m, w, dom=dom)
    U = dom.solve(0, tol=1e-13)["U"]
    s = np.zeros(m.shape)
    for d in range(3):
        prod = U[d] * U[d]
        s += prod + np.roll(prod, 1, axis=2 - d)
    np.testing.assert_allclose(dJ, -s / (2 * oracle_mod.RE_PAPER**2 * dom.N), rtol=1e-8,
                               atol=1e-10 * np.abs(dJ).max())
