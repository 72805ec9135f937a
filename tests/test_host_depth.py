"""The library's usable-depth decision (a host computation, no GPU) against
the oracle's, on the same blocks: eigenvalue ranges from LAPACK, planted
near-singular levels, the exemption of the last Gamma_k and the rule that
keeps at least one level."""
import numpy as np
import pytest

import sfm_inputs as inputs
from oracle import pipeline, sfrac
from paper_1406_6923_gb300 import sfm


def _ranges(Gam_list, Gh_list, kmax):
    """[nsub][2*kmax][2] (lambda_min, lambda_max) in the sfm_set_coeffs block
    order: Gamma_1..k then Gammahat_1..k."""
    out = np.zeros((len(Gam_list), 2 * kmax, 2))
    for s, (G, H) in enumerate(zip(Gam_list, Gh_list)):
        k = len(G)
        for j, B in enumerate(list(G) + list(H)):
            w = np.linalg.eigvalsh(0.5 * (B + B.T))
            out[s, j] = (w[0], w[-1])
    return out


def _spd(rng, b, lam_min=None):
    Q, _ = np.linalg.qr(rng.standard_normal((b, b)))
    w = np.exp(rng.uniform(-3, 3, b))
    if lam_min is not None:
        w[0] = lam_min * w.max()
    return (Q * w) @ Q.T


def test_well_conditioned_roms_keep_every_level():
    p = inputs.small_problem(ncell=(8, 8, 8), cuts=(4, 4, 4), m=3, k=3, model="layers")
    rs = pipeline.build(p)
    kmax = int(max(rs.k))
    depth = sfm.sfm_usable_depths(rs.k, _ranges(rs.Gamma, rs.Gammahat, kmax), 1e-13)
    want = [sfrac.usable_depth(rs.Gamma[s], rs.Gammahat[s], 1e-13) for s in range(rs.nsub)]
    np.testing.assert_array_equal(depth, want)
    np.testing.assert_array_equal(depth, rs.k)


def test_planted_levels_cut_where_the_oracle_cuts():
    rng = np.random.default_rng(11)
    kmax, b = 6, 5
    Gams, Ghs, ks = [], [], []
    for case in range(60):
        k = int(rng.integers(1, kmax + 1))
        G = [_spd(rng, b) for _ in range(k)]
        H = [_spd(rng, b) for _ in range(k)]
        kind = case % 5
        j = int(rng.integers(0, k))
        if kind == 1:                                  # Gammahat_j at the rounding level
            H[j] = _spd(rng, b, 1e-16)
        elif kind == 2:                                # Gamma_j (exempt when j = k - 1)
            G[j] = _spd(rng, b, 1e-15)
        elif kind == 3:                                # indefinite Gammahat_j
            H[j] = _spd(rng, b, -1e-14)
        elif kind == 4:                                # just either side of tau
            H[j] = _spd(rng, b, 1e-13 * (2.0 if rng.uniform() < 0.5 else 0.5))
        Gams.append(G)
        Ghs.append(H)
        ks.append(k)
    depth = sfm.sfm_usable_depths(ks, _ranges(Gams, Ghs, kmax), 1e-13)
    want = [sfrac.usable_depth(G, H, 1e-13) for G, H in zip(Gams, Ghs)]
    np.testing.assert_array_equal(depth, want)
    assert min(want) == 1 and any(w < k for w, k in zip(want, ks))


def test_last_gamma_is_exempt_and_one_level_is_kept():
    rng = np.random.default_rng(2)
    b = 4
    G = [_spd(rng, b) for _ in range(3)]
    H = [_spd(rng, b) for _ in range(3)]
    G[2] = _spd(rng, b, 0.0)                           # semidefinite last level
    assert list(sfm.sfm_usable_depths([3], _ranges([G], [H], 3))) == [3]
    H[0] = _spd(rng, b, -1.0)                          # level 1 itself fails
    assert list(sfm.sfm_usable_depths([3], _ranges([G], [H], 3))) == [1]


def test_bad_arguments_are_rejected():
    r = np.zeros((1, 4, 2))
    with pytest.raises(sfm.SfmError):
        sfm.sfm_usable_depths([2], r, 1.5)
    with pytest.raises(sfm.SfmError):
        sfm.sfm_usable_depths([3], r, 1e-13)           # k above kmax = 2


def test_cut_depth_rejects_a_null_handle_without_device_work():
    lib = sfm.load()
    assert lib.sfm_cut_depth(None, 1e-13, None, 0, None) == sfm.SFM_ERR_ARG
