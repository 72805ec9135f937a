"""Pins of the oracle's Krylov subspace with distinct finite shifts (Eq. 6
with sigma_1..sigma_{k-1} distinct): the Galerkin ROM interpolates the
subdomain's NtD map and its derivative at every shift, the S-fraction of
that ROM is exact (Eqs. 4, 9 and 15 agree), and repeated shifts give back
the single-shift ROM."""
import numpy as np
import pytest

import sfm_inputs as inputs
from oracle import faces, pipeline, sfrac


def _sub(sigma, m=3, k=4, model="random", ncell=(6, 5, 7), seed=3):
    p = inputs.small_problem(ncell=ncell, cuts=ncell, m=m, k=k, model=model, seed=seed,
                             src=[[21.0, 17.0, 33.0]], rec=[[30.0, 20.0, 40.0]])
    p.sigma = sigma
    topo = faces.Topology(p)
    return p, pipeline.SubdomainROM(p, topo, 0, keep_basis=True)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _fine_S(sr, lam, power=1):
    """F^T (L + lam)^{-power} F from dense solves with K + lam M:
    (L + lam)^{-1} = M^{1/2} (K + lam M)^{-1} M^{1/2}."""
    A = sr.K.toarray() + lam * np.diag(sr.mass)
    X = np.linalg.solve(A, sr.B)
    for _ in range(power - 1):
        X = np.linalg.solve(A, sr.mass[:, None] * X)
    return sr.B.T @ X


def _rom_S(sr, lam, power=1):
    Ai = np.linalg.inv(sr.Lt + lam * np.eye(sr.Lt.shape[0]))
    return sr.Ft.T @ np.linalg.matrix_power(Ai, power) @ sr.Ft


@pytest.fixture(scope="module")
def multi():
    base = inputs.small_problem(ncell=(6, 5, 7), cuts=(6, 5, 7), model="random", seed=3).sigma
    shifts = [0.05 * base, 0.6 * base, 4.0 * base]
    return shifts, _sub(shifts)


def test_interpolates_the_ntd_map_and_its_derivative_at_every_shift(multi):
    shifts, (p, sr) = multi
    for s in shifts:
        assert _rel(_rom_S(sr, s), _fine_S(sr, s)) < 1e-10, s
        assert _rel(_rom_S(sr, s, 2), _fine_S(sr, s, 2)) < 1e-9, s
    # and only there: halfway between two shifts the ROM is an approximation
    mid = 0.5 * (shifts[0] + shifts[1])
    assert _rel(_rom_S(sr, mid), _fine_S(sr, mid)) > 1e-12


def test_first_level_closed_form_holds(multi):
    """F is in the subspace, so Gammahat_1 = F^T F as with one shift."""
    shifts, (p, sr) = multi
    assert _rel(sr.Gammahat[0], sr.F.T @ sr.F) < 1e-10


@pytest.mark.parametrize("lam_kind", ["between", "above", "complex"])
def test_transfer_function_forms_agree(multi, lam_kind):
    shifts, (p, sr) = multi
    lam = {"between": 0.3 * shifts[1], "above": 10 * shifts[2],
           "complex": (2 * np.pi * 3.0 + 1j * 2 * np.pi * 40.0) ** 2}[lam_kind]
    a = sfrac.transfer_rom(sr.Lt, sr.Ft, lam)
    b = sfrac.transfer_tridiag(sr.alpha, sr.C, sr.R1, lam)
    c = sfrac.transfer_sfraction(sr.Gamma, sr.Gammahat, lam)
    assert _rel(b, a) < 1e-10 and _rel(c, a) < 1e-10


def test_repeated_shifts_give_the_single_shift_rom():
    s = inputs.small_problem(ncell=(6, 5, 7), cuts=(6, 5, 7), model="random", seed=3).sigma
    _, sr1 = _sub(s)
    _, srl = _sub([s, s, s])
    for j in range(sr1.k):
        assert _rel(srl.Gamma[j], sr1.Gamma[j]) < 1e-8, j
        assert _rel(srl.Gammahat[j], sr1.Gammahat[j]) < 1e-8, j
