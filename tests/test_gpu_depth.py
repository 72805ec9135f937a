"""GPU parity of the usable-depth cut (sfm_cut_depth) against the oracle's
(reading of Eqs. 12-13: a fraction cut after its last usable level and
terminated with U_{d+1} = 0), through the C ABI."""
import numpy as np
import pytest

import sfm_inputs as inputs
from oracle import coupled, pipeline, sfrac

from rom_abi import load_into

pytestmark = pytest.mark.gpu

TAU = 1e-13


def cut_tol(nsteps, tau=TAU):
    """FP64 trace tolerance for a fraction cut at tau: every kept block has
    lambda_min / lambda_max >= tau, so cond(G_j) <= tau^{-1/2}, and the
    U-form stepping amplifies a rounding of relative size eps by up to
    cond(G_j) per step; a stable leapfrog accumulates such perturbations at
    most linearly in the step count.  Two summation orders of the same
    recurrence may therefore differ by nsteps * eps * tau^{-1/2}."""
    return nsteps * np.finfo(np.float64).eps * tau ** -0.5


@pytest.fixture(scope="module")
def sfm():
    import os
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1406_6923_gb300 import _build, sfm as mod
    if not os.path.exists(mod.LIB_PATH):
        _build.build()
    mod.load()
    return mod


@pytest.fixture(scope="module")
def deep_pair():
    """Two 16^3-cell subdomains (one shared face) at m = 8, k = 24,
    sigma = (2 pi 8 f)^2: deep levels past FP64's range (the oracle pin of
    the usable depth), one source and three receivers."""
    n = 16
    p = inputs.small_problem(ncell=(2 * n, n, n), cuts=([0, n, 2 * n], [0, n], [0, n]), m=8,
                             k=24, model="two_layer", f_peak=20.0,
                             sigma=inputs.default_sigma(20.0, 8), nsteps=300)
    full = pipeline.build(p)
    cut = pipeline.build(p, depth_tau=TAU)
    return p, full, cut


def _ratio_at(G, H, j, k):
    """Smallest lambda_min / lambda_max of the blocks that decide level j."""
    blocks = [H[j]] + ([G[j]] if j < k - 1 else [])
    r = []
    for B in blocks:
        w = np.linalg.eigvalsh(0.5 * (B + B.T))
        r.append(w[0] / w[-1])
    return min(r)


def test_cut_depths_match_the_oracle(sfm, deep_pair):
    p, full, cut = deep_pair
    h = sfm.sfm_create(0)
    try:
        load_into(sfm, h, full)
        depth, ncut = sfm.sfm_cut_depth(h, full.nsub, TAU)
    finally:
        sfm.sfm_destroy(h)
    want = np.asarray(cut.k)
    assert ncut == int((np.asarray(full.k) - depth).sum()) > 0
    for s in range(full.nsub):
        if depth[s] != want[s]:
            # a different decision is valid only at a level whose ratio sits
            # within rounding of tau (Jacobi vs LAPACK eigenvalues)
            j = min(depth[s], want[s])
            r = _ratio_at(full.Gamma[s], full.Gammahat[s], j, full.k[s])
            assert 0.5 * TAU < r < 2.0 * TAU, (s, depth[s], want[s], r)


def test_cut_keeps_the_leading_levels_and_steps_like_the_oracle(sfm, deep_pair):
    p, full, cut = deep_pair
    h = sfm.sfm_create(0)
    try:
        load_into(sfm, h, full)
        depth, _ = sfm.sfm_cut_depth(h, full.nsub, TAU)
        if not np.array_equal(depth, cut.k):
            pytest.skip("depth decided differently within rounding of tau")
        got = sfm.sfm_get_coeffs(h)
        want = np.concatenate([np.concatenate([cut.Gamma[s].ravel(), cut.Gammahat[s].ravel()])
                               for s in range(cut.nsub)])
        np.testing.assert_array_equal(got, want)
        dt = pipeline.rom_dt(cut)
        w = inputs.wavelet_samples(p, dt)
        traces, _ = sfm.sfm_run(h, sfm.SFM_FP64, dt, p.nsteps, w, cut.nshots, cut.nrec)
    finally:
        sfm.sfm_destroy(h)
    ref = coupled.step_structured(cut, dt, p.nsteps, w)
    assert pipeline.rel_l2(traces, ref) < cut_tol(p.nsteps)


def test_nothing_to_cut_leaves_the_handle_alone(sfm):
    p = inputs.small_problem(ncell=(8, 8, 8), cuts=(4, 4, 4), m=3, k=3, model="layers")
    rs = pipeline.build(p)
    assert all(sfrac.usable_depth(rs.Gamma[s], rs.Gammahat[s], TAU) == rs.k[s]
               for s in range(rs.nsub))
    h = sfm.sfm_create(0)
    try:
        load_into(sfm, h, rs)
        before = sfm.sfm_get_coeffs(h)
        depth, ncut = sfm.sfm_cut_depth(h, rs.nsub, TAU)
        assert ncut == 0 and np.array_equal(depth, rs.k)
        np.testing.assert_array_equal(sfm.sfm_get_coeffs(h), before)
    finally:
        sfm.sfm_destroy(h)
