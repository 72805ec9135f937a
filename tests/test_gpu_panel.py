"""GPU parity of the multi-shot panel modes (shots stepped 16 at a time with
tensor-core factor products, Algorithm 1 stage 2; Eqs. 12, 18, 19) through
the C ABI against the FP64 oracle, on uneven subdomains with uneven (m, k):
the whole-trace relative L2 and every (shot, receiver) trace."""
import numpy as np
import pytest

import sfm_inputs as inputs
from oracle import coupled, pipeline

from rom_abi import load_into

pytestmark = pytest.mark.gpu

# SFM_TF32X3 computes every product with FP32 accuracy (head/tail TF32
# splits of both operands, FP32 accumulation) through FP32 Cholesky
# factors, like SFM_FP32F: it is held to the throughput metric's gate.
GATE = 1e-3


@pytest.fixture(scope="module")
def sfm():
    import os
    from paper_1406_6923_gb300 import _build, sfm as mod
    if not os.path.exists(mod.LIB_PATH):
        _build.build()
    mod.load()
    return mod


def per_trace_errors(got, ref):
    """Error of every (shot, receiver) trace relative to the RMS trace norm
    of its shot.  Rounding errors scale with the state, not with one
    trace's amplitude, so this is the per-receiver form of the whole-trace
    measure; a wrong receiver row or a wrong segment of one trace shows up
    at order one."""
    num = np.linalg.norm(got - ref, axis=2)
    rms = np.sqrt(np.mean(np.linalg.norm(ref, axis=2) ** 2, axis=1, keepdims=True))
    return num / rms


def surface_shots(p, nx, ny, z):
    xs = (np.arange(nx) + 0.5) * p.nx * p.h / nx
    ys = (np.arange(ny) + 0.5) * p.ny * p.h / ny
    return np.array([[x, y, z] for y in ys for x in xs])


@pytest.fixture(scope="module")
def uneven20():
    """Uneven boxes and (m, k) (k = 1 in one subdomain), 20 shots: one full
    16-shot group and a ragged one of 4."""
    p = inputs.small_problem(ncell=(10, 9, 8), cuts=([0, 5, 10], [0, 4, 9], [0, 4, 8]),
                             m=None, k=None, m_sub=[4, 3, 4, 2, 3, 4, 4, 3],
                             k_sub=[3, 2, 3, 1, 2, 3, 4, 3], model="random",
                             rec=[[20.0, 20.0, 20.0], [50.0, 45.0, 40.0], [80.0, 80.0, 70.0],
                                  [50.0, 40.0, 40.0]])
    p.src_xyz = surface_shots(p, 5, 4, 35.0)
    rs = pipeline.build(p)
    dt = pipeline.rom_dt(rs)
    n = 400
    w = np.stack([inputs.ricker(np.arange(n) * dt - 0.002 * q, p.f_peak) for q in range(rs.nshots)])
    ref = coupled.step_structured(rs, dt, n, w)
    return p, rs, dt, n, w, ref


@pytest.fixture(scope="module")
def crop64():
    """A 64-shot uneven crop in the manner of the batched workload: cut
    lengths from {4, 5, 6, 8} cells, m in {2, 3} per subdomain (a shared
    face takes the smaller), k in 2..4, 64 shots on an 8 x 8 surface grid,
    16 receivers on a 4 x 4 surface grid, layered velocity."""
    rng = np.random.default_rng(1406)
    cuts = ([0, 4, 10, 16, 24], [0, 5, 10, 16, 20], [0, 6, 12])
    nsub = 4 * 4 * 2
    p = inputs.small_problem(ncell=(24, 20, 12), cuts=cuts, m=None, k=None,
                             m_sub=rng.integers(2, 4, nsub), k_sub=rng.integers(2, 5, nsub),
                             model="layers")
    p.src_xyz = surface_shots(p, 8, 8, 10.0)
    xs = (np.arange(4) + 0.5) * p.nx * p.h / 4
    ys = (np.arange(4) + 0.5) * p.ny * p.h / 4
    p.rec_xyz = np.array([[x, y, 0.0] for y in ys for x in xs])
    rs = pipeline.build(p)
    dt = pipeline.rom_dt(rs)
    n = 300
    w = np.stack([inputs.ricker(np.arange(n) * dt - 0.001 * (q % 7), p.f_peak)
                  for q in range(rs.nshots)])
    ref = coupled.step_structured(rs, dt, n, w)
    return p, rs, dt, n, w, ref


def run(sfm, rs, prec, dt, n, w, shape=None):
    h = sfm.sfm_create(0)
    try:
        load_into(sfm, h, rs)
        if shape:
            sfm.sfm_debug_set(h, 3, shape[0])
            sfm.sfm_debug_set(h, 4, shape[1])
        got, ms = sfm.sfm_run(h, prec, dt, n, w, rs.nshots, rs.nrec)
    finally:
        sfm.sfm_destroy(h)
    return got


def test_tf32x3_uneven_ragged_group_matches_oracle(sfm, uneven20):
    p, rs, dt, n, w, ref = uneven20
    got = run(sfm, rs, sfm.SFM_TF32X3, dt, n, w)
    err = pipeline.rel_l2(got, ref)
    per = per_trace_errors(got, ref)
    print(f"TF32X3 uneven, 20 shots: rel L2 {err:.3e}, worst trace {per.max():.3e}")
    assert err < GATE
    assert per.max() < GATE


def test_tf32x3_agrees_with_factored_fp32(sfm, uneven20):
    """Both modes apply the same FP32 factors in FP32-accurate arithmetic:
    their traces differ by rounding only, far inside the gate."""
    p, rs, dt, n, w, ref = uneven20
    a = run(sfm, rs, sfm.SFM_TF32X3, dt, n, w)
    b = run(sfm, rs, sfm.SFM_FP32F, dt, n, w)
    d = pipeline.rel_l2(a, b)
    print(f"TF32X3 vs FP32F: {d:.3e}; FP32F vs oracle {pipeline.rel_l2(b, ref):.3e}")
    assert d < 0.1 * GATE


def test_tf32x3_64_shot_uneven_crop_matches_oracle(sfm, crop64):
    p, rs, dt, n, w, ref = crop64
    got = run(sfm, rs, sfm.SFM_TF32X3, dt, n, w)
    err = pipeline.rel_l2(got, ref)
    per = per_trace_errors(got, ref)
    print(f"TF32X3 64-shot crop: rel L2 {err:.3e}, worst trace {per.max():.3e}")
    assert err < GATE
    assert per.max() < GATE


def test_panel_traces_do_not_depend_on_the_block_shape(sfm, crop64):
    p, rs, dt, n, w, ref = crop64
    runs = [run(sfm, rs, sfm.SFM_TF32X3, dt, n, w, shape=s) for s in ((1, 2), (2, 3), (4, 4), (4, 8))]
    for r in runs[1:]:
        np.testing.assert_array_equal(r, runs[0])


def test_single_word_tf32_is_coarser(sfm, uneven20):
    """1xTF32 keeps 11 significant bits of each operand: it either diverges
    or lands well behind the split form."""
    p, rs, dt, n, w, ref = uneven20
    e3 = pipeline.rel_l2(run(sfm, rs, sfm.SFM_TF32X3, dt, n, w), ref)
    try:
        e1 = pipeline.rel_l2(run(sfm, rs, sfm.SFM_TF32, dt, n, w), ref)
    except sfm.SfmError as e:
        assert e.code == sfm.SFM_ERR_UNSTABLE
        return
    print(f"1xTF32 {e1:.3e} vs 3xTF32 {e3:.3e}")
    assert e1 > 10 * e3


def test_bf16_is_reported_unavailable(sfm, uneven20):
    p, rs, dt, n, w, ref = uneven20
    with pytest.raises(sfm.SfmError) as e:
        run(sfm, rs, sfm.SFM_BF16, dt, n, w)
    assert e.value.code == sfm.SFM_ERR_ARG


def test_panel_checkpoint_continues_bitwise(sfm, uneven20):
    """FP32 panel state converts to FP64 and back exactly: an N-step run, its
    checkpoint and an M-step run from it give the N+M-step traces."""
    p, rs, dt, n, w, ref = uneven20
    n1 = n // 2
    h = sfm.sfm_create(0)
    try:
        load_into(sfm, h, rs)
        whole, _ = sfm.sfm_run(h, sfm.SFM_TF32X3, dt, n, w, rs.nshots, rs.nrec)
        first, _ = sfm.sfm_run(h, sfm.SFM_TF32X3, dt, n1, np.ascontiguousarray(w[:, :n1]),
                               rs.nshots, rs.nrec)
        blob = sfm.sfm_checkpoint(h)
        sfm.sfm_restore(h, blob)
        second, _ = sfm.sfm_run(h, sfm.SFM_TF32X3, dt, n - n1, np.ascontiguousarray(w[:, n1:]),
                                rs.nshots, rs.nrec)
    finally:
        sfm.sfm_destroy(h)
    np.testing.assert_array_equal(first, whole[:, :, :n1 + 1])
    np.testing.assert_array_equal(second, whole[:, :, n1:])


# SFM_FP32X2P: the panels in two-float form (blocks, state, face data and
# the compensated products of SFM_FP32X2), held to the FP32-class target.
FP32X2_TOL = 1e-5


def test_fp32x2p_uneven_ragged_group_matches_oracle(sfm, uneven20):
    p, rs, dt, n, w, ref = uneven20
    got = run(sfm, rs, sfm.SFM_FP32X2P, dt, n, w)
    err = pipeline.rel_l2(got, ref)
    per = per_trace_errors(got, ref)
    print(f"FP32X2P uneven, 20 shots: rel L2 {err:.3e}, worst trace {per.max():.3e}")
    assert err < FP32X2_TOL
    assert per.max() < FP32X2_TOL


def test_fp32x2p_64_shot_uneven_crop_matches_oracle(sfm, crop64):
    p, rs, dt, n, w, ref = crop64
    got = run(sfm, rs, sfm.SFM_FP32X2P, dt, n, w)
    err = pipeline.rel_l2(got, ref)
    per = per_trace_errors(got, ref)
    print(f"FP32X2P 64-shot crop: rel L2 {err:.3e}, worst trace {per.max():.3e}")
    assert err < FP32X2_TOL
    assert per.max() < FP32X2_TOL


def test_fp32x2p_agrees_with_the_single_shot_two_float_mode(sfm, crop64):
    """The same two-float blocks and state as SFM_FP32X2, summed in another
    order: the two differ by two-float rounding only."""
    p, rs, dt, n, w, ref = crop64
    a = run(sfm, rs, sfm.SFM_FP32X2P, dt, n, w)
    b = run(sfm, rs, sfm.SFM_FP32X2, dt, n, w)
    d = pipeline.rel_l2(a, b)
    print(f"FP32X2P vs FP32X2: {d:.3e}; FP32X2 vs oracle {pipeline.rel_l2(b, ref):.3e}")
    assert d < 0.1 * FP32X2_TOL


def test_fp32x2p_traces_do_not_depend_on_the_block_shape(sfm, crop64):
    p, rs, dt, n, w, ref = crop64
    runs = [run(sfm, rs, sfm.SFM_FP32X2P, dt, n, w, shape=s) for s in ((1, 2), (2, 3), (4, 4), (4, 8))]
    for r in runs[1:]:
        np.testing.assert_array_equal(r, runs[0])


def test_fp32x2p_checkpoint_continues(sfm, uneven20):
    """The two-float panel state goes through the FP64 checkpoint (hi + lo
    rounded to FP64 and split again): a restored run continues the N+M-step
    traces to far below the mode's own error."""
    p, rs, dt, n, w, ref = uneven20
    n1 = n // 2
    h = sfm.sfm_create(0)
    try:
        load_into(sfm, h, rs)
        whole, _ = sfm.sfm_run(h, sfm.SFM_FP32X2P, dt, n, w, rs.nshots, rs.nrec)
        first, _ = sfm.sfm_run(h, sfm.SFM_FP32X2P, dt, n1, np.ascontiguousarray(w[:, :n1]),
                               rs.nshots, rs.nrec)
        blob = sfm.sfm_checkpoint(h)
        sfm.sfm_restore(h, blob)
        second, _ = sfm.sfm_run(h, sfm.SFM_FP32X2P, dt, n - n1, np.ascontiguousarray(w[:, n1:]),
                                rs.nshots, rs.nrec)
    finally:
        sfm.sfm_destroy(h)
    np.testing.assert_array_equal(first, whole[:, :, :n1 + 1])
    assert pipeline.rel_l2(second, whole[:, :, n1:]) < 1e-9
