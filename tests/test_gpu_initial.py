"""GPU parity of the initial-value form (Algorithm 1 step 1.4 for initial
conditions) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import sfm_inputs as inputs
from oracle import coupled, pipeline

from rom_abi import load_into

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-11
FP32X2_TOL = 1e-5
FP32F_GATE = 1e-3


@pytest.fixture(scope="module")
def sfm():
    import os
    from paper_1406_6923_gb300 import _build, sfm as mod
    if not os.path.exists(mod.LIB_PATH):
        _build.build()
    mod.load()
    return mod


def _fields(p, seed, shots):
    """Smooth seeded nodal fields [shots][nz+1][ny+1][nx+1]."""
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(np.arange(p.nz + 1), np.arange(p.ny + 1), np.arange(p.nx + 1),
                          indexing="ij")
    out = []
    for _ in range(shots):
        c = rng.uniform(0.3, 0.7, 3) * np.array([p.nx, p.ny, p.nz])
        w = 0.2 * min(p.nx, p.ny, p.nz)
        out.append(np.exp(-((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) / (2 * w * w)))
    return np.stack(out)


@pytest.fixture(scope="module")
def initial():
    """Uneven boxes and m, k; two shots, each with a source and its own
    initial displacement and velocity."""
    p = inputs.small_problem(ncell=(10, 9, 8), cuts=([0, 5, 10], [0, 4, 9], [0, 4, 8]),
                             m=None, k=None, m_sub=[4, 3, 4, 2, 3, 4, 4, 3],
                             k_sub=[3, 2, 3, 1, 2, 3, 4, 3], model="random",
                             src=[[41.0, 37.0, 39.0], [12.0, 70.0, 20.0]],
                             rec=[[20.0, 20.0, 20.0], [50.0, 45.0, 40.0], [80.0, 80.0, 70.0],
                                  [50.0, 40.0, 40.0]])
    u0 = _fields(p, 31, 2)
    v0 = 2e3 * _fields(p, 32, 2)
    rs = pipeline.build(p, u0=u0, v0=v0)
    dt = pipeline.rom_dt(rs)
    n = 300
    w = np.stack([inputs.ricker(np.arange(n) * dt, p.f_peak),
                  inputs.ricker(np.arange(n) * dt - 0.01, p.f_peak)])
    ref = coupled.step_structured(rs, dt, n, w, U0=rs.U0, V0=rs.V0)
    return p, rs, dt, n, w, ref


def _set_initial(sfm, h, rs, with_velocity=True):
    shots, subs, u, v = [], [], [], []
    for q in range(len(rs.U0)):
        for s in sorted(rs.U0[q]):
            shots.append(q)
            subs.append(s)
            u.append(rs.U0[q][s].ravel())
            v.append(rs.V0[q][s].ravel())
    sfm.sfm_set_initial(h, rs.nshots, shots, subs, np.concatenate(u),
                        np.concatenate(v) if with_velocity else None)


def _run(sfm, rs, dt, n, w, precision, init=True):
    h = sfm.sfm_create(0)
    try:
        load_into(sfm, h, rs)
        if init:
            _set_initial(sfm, h, rs)
        tr, _ = sfm.sfm_run(h, precision, dt, n, w, rs.nshots, rs.nrec)
        return tr
    finally:
        sfm.sfm_destroy(h)


def test_initial_state_fp64_matches_oracle(sfm, initial):
    p, rs, dt, n, w, ref = initial
    got = _run(sfm, rs, dt, n, w, sfm.SFM_FP64)
    assert pipeline.rel_l2(got, ref) <= FP64_TOL
    assert np.abs(got[:, :, 0] - ref[:, :, 0]).max() <= 10 * FP64_TOL * np.abs(ref).max()


def test_initial_state_fp32x2_matches_oracle(sfm, initial):
    p, rs, dt, n, w, ref = initial
    got = _run(sfm, rs, dt, n, w, sfm.SFM_FP32X2)
    assert pipeline.rel_l2(got, ref) <= FP32X2_TOL


def test_initial_state_fp32fx2_matches_oracle(sfm, initial):
    p, rs, dt, n, w, ref = initial
    got = _run(sfm, rs, dt, n, w, sfm.SFM_FP32FX2)
    assert pipeline.rel_l2(got, ref) <= FP32X2_TOL


def test_initial_state_fp32f_matches_oracle(sfm, initial):
    p, rs, dt, n, w, ref = initial
    got = _run(sfm, rs, dt, n, w, sfm.SFM_FP32F)
    assert pipeline.rel_l2(got, ref) <= FP32F_GATE


def test_pure_initial_value_problem_and_clearing(sfm, initial):
    """Zero source: the traces come from the initial data alone; without
    velocity the start uses V^0 = 0; npairs = 0 returns to rest."""
    p, rs, dt, n, w, ref = initial
    w0 = np.zeros_like(w)
    V0zero = [{s: np.zeros_like(r) for s, r in d.items()} for d in rs.U0]
    ref0 = coupled.step_structured(rs, dt, n, w0, U0=rs.U0, V0=V0zero)
    h = sfm.sfm_create(0)
    try:
        load_into(sfm, h, rs)
        _set_initial(sfm, h, rs, with_velocity=False)
        got, _ = sfm.sfm_run(h, sfm.SFM_FP64, dt, n, w0, rs.nshots, rs.nrec)
        assert np.abs(ref0).max() > 0
        assert pipeline.rel_l2(got, ref0) <= FP64_TOL
        sfm.sfm_set_initial(h, rs.nshots, [], [], np.zeros(0))
        got, _ = sfm.sfm_run(h, sfm.SFM_FP64, dt, n, w0, rs.nshots, rs.nrec)
        assert np.abs(got).max() == 0.0
    finally:
        sfm.sfm_destroy(h)
