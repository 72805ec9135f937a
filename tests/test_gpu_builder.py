"""GPU offline builder (Algorithm 1 stage 1, FP64) against the oracle: the
S-fraction coefficients, their transfer function, and end-to-end traces
(GPU-built ROMs stepped on the GPU vs oracle-built ROMs stepped by the
oracle)."""
import numpy as np
import pytest

import sfm_inputs as inputs
from oracle import coupled, pipeline, sfrac

from rom_abi import abi_arrays

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sfm():
    import os
    from paper_1406_6923_gb300 import _build, sfm as mod
    if not os.path.exists(mod.LIB_PATH):
        _build.build()
    mod.load()
    return mod


def _gpu_build(sfm, p, cg_tol=1e-14):
    h = sfm.sfm_create(0)
    sfm.sfm_set_model(h, p.c, p.h, p.xcuts, p.ycuts, p.zcuts)
    rep = sfm.sfm_build_roms(h, p.m_sub, p.k_sub, p.sigma, cg_tol)
    sfm.sfm_project_sources(h, p.src_xyz, p.src_width)
    sfm.sfm_project_receivers(h, p.rec_xyz)
    return h, rep


def _split(coeffs, rs):
    out, o = [], 0
    for s in range(rs.nsub):
        k, b = rs.k[s], rs.b[s]
        G = coeffs[o:o + k * b * b].reshape(k, b, b)
        o += k * b * b
        Gh = coeffs[o:o + k * b * b].reshape(k, b, b)
        o += k * b * b
        out.append((G, Gh))
    return out


@pytest.fixture(scope="module")
def uneven_problem():
    p = inputs.small_problem(ncell=(10, 9, 8), cuts=([0, 5, 10], [0, 4, 9], [0, 4, 8]),
                             m=None, k=None, m_sub=[4, 3, 4, 2, 3, 4, 4, 3],
                             k_sub=[3, 2, 3, 1, 2, 3, 4, 3], model="random",
                             src=[[41.0, 37.0, 39.0], [12.0, 70.0, 20.0]],
                             rec=[[20.0, 20.0, 20.0], [50.0, 45.0, 40.0], [80.0, 80.0, 70.0],
                                  [50.0, 40.0, 40.0]])
    return p, pipeline.build(p)


def test_builder_coefficients_match_oracle(sfm, uneven_problem):
    p, rs = uneven_problem
    h, rep = _gpu_build(sfm, p)
    try:
        got = _split(sfm.sfm_get_coeffs(h), rs)
    finally:
        sfm.sfm_destroy(h)
    assert rep["cg_residual_max"] < 1e-13
    # well-conditioned ROMs need no diagonal shift
    assert rep["nregularized"] == 0
    for s in range(rs.nsub):
        G, Gh = got[s]
        for j in range(rs.k[s]):
            rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
            assert rel(Gh[j], rs.Gammahat[s][j]) < 1e-9, (s, j)
            assert rel(G[j], rs.Gamma[s][j]) < 1e-8, (s, j)


def test_builder_transfer_function_matches_oracle(sfm, uneven_problem):
    p, rs = uneven_problem
    h, rep = _gpu_build(sfm, p)
    try:
        got = _split(sfm.sfm_get_coeffs(h), rs)
    finally:
        sfm.sfm_destroy(h)
    for s in range(rs.nsub):
        for lam in (0.3 * p.sigma, p.sigma, (2 * np.pi * 5 + 2j * np.pi * p.f_peak) ** 2):
            a = sfrac.transfer_sfraction(list(got[s][0]), list(got[s][1]), lam)
            b = sfrac.transfer_sfraction(list(rs.Gamma[s]), list(rs.Gammahat[s]), lam)
            assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-10


def test_builder_end_to_end_traces_match_oracle(sfm, uneven_problem):
    p, rs = uneven_problem
    dt = pipeline.rom_dt(rs)
    n = 300
    w = inputs.wavelet_samples(p, dt, n)
    ref = coupled.step_structured(rs, dt, n, w)
    h, rep = _gpu_build(sfm, p)
    try:
        got, _ = sfm.sfm_run(h, sfm.SFM_FP64, dt, n, w, rs.nshots, rs.nrec)
    finally:
        sfm.sfm_destroy(h)
    assert pipeline.rel_l2(got, ref) < 1e-8


def test_builder_config1_end_to_end(sfm):
    p = inputs.config1()
    rs = pipeline.build(p)
    dt = pipeline.rom_dt(rs)
    w = inputs.wavelet_samples(p, dt)
    ref = coupled.step_structured(rs, dt, p.nsteps, w)
    h, rep = _gpu_build(sfm, p)
    try:
        got, _ = sfm.sfm_run(h, sfm.SFM_FP64, dt, p.nsteps, w, rs.nshots, rs.nrec)
        lam, dtc = sfm.sfm_cfl_dt(h, 1000)
    finally:
        sfm.sfm_destroy(h)
    assert pipeline.rel_l2(got, ref) < 1e-8
    assert abs(0.9 * dtc / dt - 1.0) < 1e-4


def test_builder_rejects_bad_input(sfm):
    p = inputs.small_problem(ncell=(8, 8, 8), cuts=(4, 4, 4), m=3, k=2)
    h = sfm.sfm_create(0)
    try:
        with pytest.raises(sfm.SfmError) as e:
            sfm.sfm_build_roms(h, p.m_sub, p.k_sub, p.sigma)
        assert e.value.code == sfm.SFM_ERR_STATE
        with pytest.raises(sfm.SfmError) as e:
            sfm.sfm_set_model(h, p.c, p.h, [0, 1, 8], p.ycuts, p.zcuts)   # 1-cell subdomain
        assert e.value.code == sfm.SFM_ERR_ARG
        sfm.sfm_set_model(h, p.c, p.h, p.xcuts, p.ycuts, p.zcuts)
        with pytest.raises(sfm.SfmError) as e:
            sfm.sfm_build_roms(h, np.full(p.nsub, 10), p.k_sub, p.sigma)  # 10 > 3x3 open nodes
        assert e.value.code == sfm.SFM_ERR_ARG
    finally:
        sfm.sfm_destroy(h)


@pytest.mark.slow
def test_builder_full_config2_sampled_against_oracle(sfm):
    """The full 192^3 layered-lens model with 512 subdomains, m = 8, k = 16,
    built on the GPU; a sample of subdomains (the source's, a central one, a
    deep one and a corner) built by the oracle alone.  The transfer
    functions S(lambda) of the two S-fractions agree at shifts across the
    source band.  Evaluating S from deep coefficients inverts blocks with
    condition numbers up to ~1e10 on both sides, so the bound is 1e-6: a
    wrong block, sign or level gives O(1)."""
    p = inputs.config2()
    ncx = len(p.xcuts) - 1
    sample = [4 + ncx * (4 + ncx * 0), 4 + ncx * (4 + ncx * 4), 2 + ncx * (6 + ncx * 5), 0]
    topo, Gam, Gh, kept = pipeline.build(p, subs=sample)
    h = sfm.sfm_create(0)
    try:
        sfm.sfm_set_model(h, p.c, p.h, p.xcuts, p.ycuts, p.zcuts)
        sfm.sfm_build_roms(h, p.m_sub, p.k_sub, p.sigma)
        coeffs = sfm.sfm_get_coeffs(h)
    finally:
        sfm.sfm_destroy(h)
    b, k = 48, 16
    per = 2 * k * b * b
    for s in sample:
        G = coeffs[s * per:s * per + k * b * b].reshape(k, b, b)
        H = coeffs[s * per + k * b * b:(s + 1) * per].reshape(k, b, b)
        for lam in (0.1 * p.sigma, p.sigma, (2 * np.pi * 5 + 2j * np.pi * p.f_peak) ** 2):
            a = sfrac.transfer_sfraction(list(G), list(H), lam)
            r = sfrac.transfer_sfraction(list(Gam[s]), list(Gh[s]), lam)
            assert np.linalg.norm(a - r) / np.linalg.norm(r) < 1e-6, (s, lam)


def test_builder_with_distinct_shifts_matches_oracle(sfm):
    """Distinct finite shifts (Eq. 6): the GPU build against the oracle's
    build with the same three shifts, coefficient by coefficient and through
    the transfer function, which interpolates the subdomain's NtD map at
    every shift."""
    p = inputs.small_problem(ncell=(10, 9, 8), cuts=([0, 5, 10], [0, 4, 9], [0, 4, 8]), m=3, k=4,
                             model="random")
    base = p.sigma
    shifts = [0.05 * base, 0.6 * base, 4.0 * base]
    p.sigma = shifts
    rs = pipeline.build(p)
    h = sfm.sfm_create(0)
    try:
        sfm.sfm_set_model(h, p.c, p.h, p.xcuts, p.ycuts, p.zcuts)
        rep = sfm.sfm_build_roms_shifts(h, p.m_sub, p.k_sub, shifts)
        got = _split(sfm.sfm_get_coeffs(h), rs)
    finally:
        sfm.sfm_destroy(h)
    assert rep["cg_residual_max"] < 1e-13
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    for s in range(rs.nsub):
        G, Gh = got[s]
        for j in range(rs.k[s]):
            assert rel(Gh[j], rs.Gammahat[s][j]) < 1e-8, (s, j)
            assert rel(G[j], rs.Gamma[s][j]) < 1e-7, (s, j)
        for lam in (shifts[0], shifts[2], 0.3 * base * (1 + 1j)):
            a = sfrac.transfer_sfraction(list(G), list(Gh), lam)
            r = sfrac.transfer_sfraction(list(rs.Gamma[s]), list(rs.Gammahat[s]), lam)
            assert rel(a, r) < 1e-9, (s, lam)
