"""Pins of the oracle at the paper's own face width (section "Numerical
experiments": 25 modes per face, so b = 6m = 150), the width the GPU
path's wide-block tests compare against: moment matching of the Krylov ROM
(Eqs. 5-7), agreement of the transfer-function forms (Eqs. 4, 9, 15), the
level-one closed form on a uniform cube with all 25 modes of every face,
positive definiteness below the last level (Eq. 13), and the coupled
stepping against a generic leapfrog of the assembled system."""
import numpy as np
import pytest

import sfm_inputs as inputs
from oracle import coupled, faces, pipeline, sfrac


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def wide_sub():
    """One 8^3-cell subdomain (7 x 7 open-face nodes per face), m = 25,
    k = 2, random cell velocities."""
    n = 8
    p = inputs.small_problem(ncell=(n, n, n), cuts=(n, n, n), m=25, k=2, model="random", seed=5,
                             src=[[31.0, 37.0, 41.0]], rec=[[40.0, 40.0, 40.0]])
    topo = faces.Topology(p)
    return p, topo, pipeline.SubdomainROM(p, topo, 0, keep_basis=True)


def test_wide_block_has_the_papers_width(wide_sub):
    p, topo, sr = wide_sub
    assert sr.Gammahat[0].shape == (150, 150)
    assert sr.V.shape[1] == 150 * sr.k


def test_wide_moment_matching(wide_sub):
    """F~^T (L~+s)^{-j} F~ = F^T (L+s)^{-j} F for j = 0..2k-2, with the
    fine side from dense solves of K + sigma M (not the ROM's factors)."""
    p, topo, sr = wide_sub
    K = sr.K.toarray()
    M = sr.mass
    A = K + sr.sigma * np.diag(M)
    At = sr.Lt + sr.sigma * np.eye(sr.Lt.shape[0])
    Ai = np.linalg.inv(At)
    X = sr.B / M[:, None]
    for j in range(0, 2 * sr.k - 1):
        fine_m = sr.B.T @ X
        rom_m = sr.Ft.T @ np.linalg.matrix_power(Ai, j) @ sr.Ft
        assert _rel(rom_m, fine_m) < 1e-9, j
        X = np.linalg.solve(A, M[:, None] * X)


@pytest.mark.parametrize("lam_kind", ["s", "10s", "complex"])
def test_wide_transfer_function_forms_agree(wide_sub, lam_kind):
    p, topo, sr = wide_sub
    s = sr.sigma
    lam = {"s": s, "10s": 10 * s, "complex": (2 * np.pi * 3.0 + 1j * 2 * np.pi * 40.0) ** 2}[lam_kind]
    a = sfrac.transfer_rom(sr.Lt, sr.Ft, lam)
    b = sfrac.transfer_tridiag(sr.alpha, sr.C, sr.R1, lam)
    c = sfrac.transfer_sfraction(sr.Gamma, sr.Gammahat, lam)
    assert _rel(b, a) < 1e-9 and _rel(c, a) < 1e-9


def test_wide_blocks_are_spd_below_the_last_level(wide_sub):
    p, topo, sr = wide_sub
    for j in range(sr.k):
        assert np.linalg.eigvalsh(0.5 * (sr.Gammahat[j] + sr.Gammahat[j].T)).min() > 0.0, j
    for j in range(sr.k - 1):
        assert np.linalg.eigvalsh(0.5 * (sr.Gamma[j] + sr.Gamma[j].T)).min() > 0.0, j


def test_wide_uniform_cube_level_one_closed_form():
    """Uniform c with the 25 modes of every face (the lowest p^2 + q^2,
    up to p = 5):
    [Gammahat_1]_f = 2 h c^2 n_f^2 diag(w_p w_q), w_0 = 1, w_{>0} = 1/2,
    and no coupling between faces."""
    n, m = 8, 25
    p = inputs.small_problem(ncell=(n, n, n), cuts=(n, n, n), m=m, k=2, model="uniform",
                             src=[[31.0, 37.0, 41.0]], rec=[[40.0, 40.0, 40.0]])
    sr = pipeline.SubdomainROM(p, faces.Topology(p), 0)
    c0, h, nf = 2000.0, p.h, n - 1
    modes = faces.mode_list(nf, nf, m)
    assert len(modes) == 25 and (5, 0) in modes and (4, 4) not in modes
    w = lambda q: 1.0 if q == 0 else 0.5
    expect = np.diag([2 * h * c0 ** 2 * nf * nf * w(a) * w(b) for a, b in modes])
    for f in range(6):
        sl = slice(f * m, (f + 1) * m)
        np.testing.assert_allclose(sr.Gammahat[0][sl, sl], expect, rtol=1e-11,
                                   atol=1e-11 * expect.max())
        for g in range(6):
            if g != f:
                assert np.abs(sr.Gammahat[0][sl, g * m:(g + 1) * m]).max() < 1e-11 * expect.max()


def test_wide_structured_stepping_equals_the_assembled_leapfrog():
    """Two subdomains of 8^3 cells at m = 25, k = 2: the structured
    a1-a7 recurrence against a generic leapfrog of the assembled (M, K)."""
    p = inputs.small_problem(ncell=(16, 8, 8), cuts=([0, 8, 16], [0, 8], [0, 8]), m=25, k=2,
                             model="random", rec=[[40.0, 40.0, 40.0], [120.0, 40.0, 40.0]])
    rs = pipeline.build(p)
    A = coupled.Assembled(rs)
    dt = 0.9 * A.cfl_dt()
    n = 120
    w = np.stack([inputs.ricker(np.arange(n) * dt, p.f_peak) for _ in range(rs.nshots)])
    a = coupled.step_structured(rs, dt, n, w)
    b = A.leapfrog(dt, n, w)
    assert np.abs(a).max() > 0
    assert pipeline.rel_l2(a, b) < 1e-12
