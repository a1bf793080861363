"""Input pre-processing of Sec. 5 ("Processing input data") through the C ABI, host paths
(no GPU): mirroring for symmetric periodicity and the elimination of disconnected pore
spaces.  Pins: the mirror is numpy's reflection; the mirrored domain has no coupling
between the mirrored axis and the others (oracle k); removing closed pores leaves the
oracle's k unchanged and removes nothing from a flowing component."""
import numpy as np
import pytest

from paper_2407_19868_gb300 import geometry as G


@pytest.fixture(scope="module")
def api():
    from paper_2407_19868_gb300 import api as A
    A.load()
    return A


@pytest.mark.parametrize("axes", [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 1, 1)])
def test_mirror_matches_reflection(api, axes):
    m = G.random_blocks((3, 4, 5), 0.4, seed=2)
    ref = m
    for a in range(3):
        if axes[a]:
            ax = 2 - a
            ref = np.concatenate([ref, np.flip(ref, axis=ax)], axis=ax)
    assert np.array_equal(api.mirror_mask(m, axes), ref)


def test_mirrored_domain_decouples_the_mirrored_axis(api, oracle_mod):
    m = G.random_blocks((6, 6, 6), 0.3, seed=4)
    mm = api.mirror_mask(m, (1, 0, 0))
    _, k, _ = oracle_mod.ktensor(mm, tol=1e-12, check_every=100)
    for i, j in ((0, 1), (0, 2), (1, 0), (2, 0)):
        assert abs(k[i, j]) < 1e-9 * max(abs(k[0, 0]), abs(k[1, 1]))
    _, k0, _ = oracle_mod.ktensor(m, tol=1e-12, check_every=100)
    assert abs(k0[0, 1]) > 1e-4 * k0[0, 0]  # the original sample does couple x and y


def test_closed_cavity_removed_flowing_pores_kept(api):
    m = np.ones((6, 6, 8), dtype=np.uint8)
    m[2, 2, :] = 0          # channel along x (wraps: flows)
    m[4, 4, 3:5] = 0        # closed cavity
    out, n = api.remove_isolated_pores(m, (0, 0, 0))
    assert n == 2 and np.all(out[4, 4, 3:5] == 1) and np.all(out[2, 2, :] == 0)
    # with walls along x the channel no longer flows anywhere and goes too
    out, n = api.remove_isolated_pores(m, (1, 0, 0))
    assert n == 10
    # a fixed-pressure axis keeps what joins its first and last layer
    out, n = api.remove_isolated_pores(m, (2, 0, 0))
    assert n == 2 and np.all(out[2, 2, :] == 0)


def test_removal_leaves_the_oracle_k_unchanged(api, oracle_mod):
    m = G.random_blocks((8, 8, 8), 0.45, seed=12)
    out, n = api.remove_isolated_pores(m, (0, 0, 0))
    assert n > 0 and np.all(out >= m)
    _, k1, _ = oracle_mod.ktensor(m, tol=1e-12, check_every=100)
    _, k2, _ = oracle_mod.ktensor(out, tol=1e-12, check_every=100)
    np.testing.assert_allclose(k2, k1, rtol=0, atol=1e-9 * np.max(np.abs(np.diag(k1))))


@pytest.mark.gpu
def test_mirror_on_the_device_matches_the_host(api):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():  # pragma: no cover
        pytest.skip("no CUDA device")
    m = G.random_blocks((5, 6, 7), 0.4, seed=3)
    for axes in ((1, 0, 0), (0, 1, 1), (1, 1, 1)):
        d = api.mirror_mask(torch.from_numpy(m).cuda(), axes)
        assert np.array_equal(d.cpu().numpy(), api.mirror_mask(m, axes))
