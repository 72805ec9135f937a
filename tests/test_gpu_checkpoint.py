"""Checkpoint and restore of the stepping state (sfm_checkpoint,
sfm_restore) through the C ABI: an N-step run, its checkpoint and an M-step
run from the restored state give the traces of one N+M-step run, which
matches the oracle's stepping.

"""
import numpy as np
import pytest

import sfm_inputs as inputs
from oracle import coupled, pipeline

from rom_abi import load_into

pytestmark = pytest.mark.gpu

N, M = 120, 180


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
def small():
    p = inputs.small_problem(ncell=(12, 8, 8), cuts=([0, 4, 8, 12], [0, 4, 8], [0, 8]), m=3, k=3,
                             model="layers", nsteps=N + M,
                             src=[[41.0, 37.0, 33.0], [83.0, 45.0, 52.0]])
    rs = pipeline.build(p)
    dt = pipeline.rom_dt(rs)
    w = np.tile(inputs.ricker(np.arange(N + M) * dt, p.f_peak), (rs.nshots, 1))
    return p, rs, dt, w


def _split_run(sfm, rs, dt, w, precision):
    h = sfm.sfm_create(0)
    try:
        load_into(sfm, h, rs)
        whole, _ = sfm.sfm_run(h, precision, dt, N + M, w, rs.nshots, rs.nrec)
        first, _ = sfm.sfm_run(h, precision, dt, N, np.ascontiguousarray(w[:, :N]), rs.nshots,
                               rs.nrec)
        blob = sfm.sfm_checkpoint(h)
        sfm.sfm_restore(h, blob)
        second, _ = sfm.sfm_run(h, precision, dt, M, np.ascontiguousarray(w[:, N:]), rs.nshots,
                                rs.nrec)
    finally:
        sfm.sfm_destroy(h)
    return whole, first, second, blob


@pytest.mark.parametrize("prec_name", ["SFM_FP64", "SFM_FP32F"])
def test_restored_run_continues_bitwise(sfm, small, prec_name):
    p, rs, dt, w = small
    whole, first, second, _ = _split_run(sfm, rs, dt, w, getattr(sfm, prec_name))
    np.testing.assert_array_equal(first, whole[..., :N + 1])
    np.testing.assert_array_equal(second, whole[..., N:])


@pytest.mark.parametrize("prec_name", ["SFM_FP32X2", "SFM_FP32FX2"])
def test_restored_two_float_run_continues(sfm, small, prec_name):
    p, rs, dt, w = small
    whole, first, second, _ = _split_run(sfm, rs, dt, w, getattr(sfm, prec_name))
    assert pipeline.rel_l2(second, whole[..., N:]) < 1e-13


def test_continued_fp64_run_matches_the_oracle(sfm, small):
    p, rs, dt, w = small
    _, first, second, _ = _split_run(sfm, rs, dt, w, sfm.SFM_FP64)
    ref = coupled.step_structured(rs, dt, N + M, w)
    got = np.concatenate([first, second[..., 1:]], axis=-1)
    assert pipeline.rel_l2(got, ref) < 1e-11


def test_checkpoint_blob_and_topology_check(sfm, small):
    p, rs, dt, w = small
    _, _, _, blob = _split_run(sfm, rs, dt, w, sfm.SFM_FP64)
    head = np.frombuffer(blob[:64], dtype=np.int64)
    nstate = int(sum(rs.k * rs.b))
    assert head[2] == rs.nshots and head[3] == nstate and head[4] == rs.nsub and head[6] == N
    assert len(blob) == 64 + 2 * rs.nshots * nstate * 8
    other = pipeline.build(inputs.small_problem(ncell=(8, 8, 8), cuts=(4, 4, 4), m=3, k=3,
                                                model="layers"))
    h = sfm.sfm_create(0)
    try:
        load_into(sfm, h, other)
        with pytest.raises(sfm.SfmError):
            sfm.sfm_restore(h, blob)
        with pytest.raises(sfm.SfmError):
            sfm.sfm_checkpoint(h)                      # nothing stepped yet
    finally:
        sfm.sfm_destroy(h)
