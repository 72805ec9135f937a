"""Blocks wider than 64: the paper's own 25 cosine modes per face
(b = 6m = 150; section "Numerical experiments") on the GPU.  The offline
builder (Algorithm 1 stage 1, Eqs. 5-13) and the FP64, two-float and FP32
stepping (stage 2, Eqs. 12, 18, 19) against the oracle, and the modes that
keep a block's tiles in one warp's registers refusing such blocks."""
import numpy as np
import pytest

import sfm_inputs as inputs
from oracle import coupled, pipeline

from rom_abi import load_into

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-11
FP32X2_TOL = 1e-5
FP32_GATE = 1e-3


@pytest.fixture(scope="module")
def sfm():
    import os
    from paper_1406_6923_gb300 import _build, sfm as mod
    if not os.path.exists(mod.LIB_PATH):
        _build.build()
    mod.load()
    return mod


@pytest.fixture(scope="module")
def wide():
    """2 x 2 x 1 subdomains of 8^3 cells (7 x 7 open-face nodes carry the
    25 lowest cosine modes), m = 25 on every face, k = 3, random cell
    velocities."""
    p = inputs.small_problem(ncell=(16, 16, 8), cuts=([0, 8, 16], [0, 8, 16], [0, 8]), m=25, k=3,
                             model="random",
                             rec=[[30.0, 40.0, 40.0], [120.0, 100.0, 40.0], [80.0, 80.0, 0.0]])
    rs = pipeline.build(p)
    dt = pipeline.rom_dt(rs)
    n = 400
    w = np.stack([inputs.ricker(np.arange(n) * dt, p.f_peak) for _ in range(rs.nshots)])
    ref = coupled.step_structured(rs, dt, n, w)
    return p, rs, dt, n, w, ref


def _run(sfm, rs, prec, dt, n, w):
    h = sfm.sfm_create(0)
    try:
        load_into(sfm, h, rs)
        got, _ = sfm.sfm_run(h, prec, dt, n, w, rs.nshots, rs.nrec)
    finally:
        sfm.sfm_destroy(h)
    return got


def test_wide_blocks_build_like_the_oracle(sfm, wide):
    p, rs, dt, n, w, ref = wide
    assert max(rs.b) == 150
    h = sfm.sfm_create(0)
    try:
        sfm.sfm_set_model(h, p.c, p.h, p.xcuts, p.ycuts, p.zcuts)
        sfm.sfm_build_roms(h, p.m_sub, p.k_sub, p.sigma, 1e-14)
        coeffs = sfm.sfm_get_coeffs(h)
    finally:
        sfm.sfm_destroy(h)
    o = 0
    worst = 0.0
    for s in range(rs.nsub):
        k, b = rs.k[s], rs.b[s]
        G = coeffs[o:o + k * b * b].reshape(k, b, b)
        Gh = coeffs[o + k * b * b:o + 2 * k * b * b].reshape(k, b, b)
        o += 2 * k * b * b
        for j in range(k):
            eg = np.linalg.norm(G[j] - rs.Gamma[s][j]) / np.linalg.norm(rs.Gamma[s][j])
            eh = np.linalg.norm(Gh[j] - rs.Gammahat[s][j]) / np.linalg.norm(rs.Gammahat[s][j])
            worst = max(worst, eg, eh)
            assert eh < 1e-9, (s, j, eh)
            assert eg < 1e-8, (s, j, eg)
    print(f"wide blocks (b = 150): coefficients within {worst:.2e} of the oracle")


def test_wide_blocks_step_like_the_oracle(sfm, wide):
    p, rs, dt, n, w, ref = wide
    e64 = pipeline.rel_l2(_run(sfm, rs, sfm.SFM_FP64, dt, n, w), ref)
    ex2 = pipeline.rel_l2(_run(sfm, rs, sfm.SFM_FP32X2, dt, n, w), ref)
    print(f"wide blocks: FP64 {e64:.2e}, FP32X2 {ex2:.2e}")
    assert e64 <= FP64_TOL
    assert ex2 <= FP32X2_TOL
    try:
        e32 = pipeline.rel_l2(_run(sfm, rs, sfm.SFM_FP32, dt, n, w), ref)
        print(f"wide blocks: FP32 {e32:.2e}")
        assert e32 <= FP32_GATE
    except sfm.SfmError as e:
        # plain FP32 blocks may turn indefinite under rounding
        assert e.code == sfm.SFM_ERR_UNSTABLE


@pytest.mark.parametrize("mode", ["SFM_FP32F", "SFM_FP32FX2", "SFM_TF32X3", "SFM_FP32X2P"])
def test_register_tiled_modes_refuse_wide_blocks(sfm, wide, mode):
    p, rs, dt, n, w, ref = wide
    with pytest.raises(sfm.SfmError) as e:
        _run(sfm, rs, getattr(sfm, mode), dt, 20, np.ascontiguousarray(w[:, :20]))
    assert e.value.code == sfm.SFM_ERR_ARG
