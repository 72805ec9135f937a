"""GPU parity of the coupled stepping (Algorithm 1 stage 2) through the C ABI
against the FP64 oracle, plus the failure paths (bounded barrier timeout,
instability) and determinism."""
import numpy as np
import pytest

import sfm_inputs as inputs
from oracle import coupled, pipeline

from rom_abi import load_into

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-11
# The k = 16 ROMs of the 192^3 workload have cond(Gammahat_j) ~ 1e10, which
# amplifies the rounding-order differences between two FP64 evaluations of
# the same recurrence by ~1e6 (measured: 9e-11); their FP64 tolerance is
# scaled accordingly.
FP64_TOL_DEEP = 1e-9
# Plain FP32 stepping of the U-form: the same recurrence evaluated exactly in
# FP32 (coefficients, state and sums rounded to FP32) already lies 3e-5 to
# 2e-4 from FP64 on these problems, because the S-fraction coefficients of an
# accurate ROM are ill-conditioned (cond(Gammahat_j) ~ 1e4-1e5 here).  Plain
# FP32 is therefore held to the throughput metric's gate, 1e-3 vs FP64.
FP32_GATE = 1e-3
# Two-float stepping (hi + lo FP32 words, compensated FP32 arithmetic) carries
# the FP32-class accuracy target.
FP32X2_TOL = 1e-5
# FP32 stepping through FP32 Cholesky factors of the blocks: stable on every
# ROM, with the error of plain FP32 sums over ill-conditioned blocks (a CPU
# emulation of a 64-subdomain k = 16 crop of the 192^3 model gave 8e-5 after
# 4000 steps); held to the throughput metric's gate.
FP32F_GATE = 1e-3
# The same FP32 factors with a two-float state, two-float vectors and
# compensated sums: the factors' rounding is the only FP32 rounding left (the
# crop emulation: 5.2e-6 after 4000 steps); held to the FP32 target.
FP32FX2_TOL = 1e-5


@pytest.fixture(scope="module")
def sfm():
    import os
    from paper_1406_6923_gb300 import _build, sfm as mod
    if not os.path.exists(mod.LIB_PATH):
        _build.build()
    mod.load()
    return mod


@pytest.fixture(scope="module")
def uneven():
    """Uneven boxes, uneven m and k (one subdomain with k = 1, a face count
    mismatch resolved to the smaller m), two shots."""
    p = inputs.small_problem(ncell=(10, 9, 8), cuts=([0, 5, 10], [0, 4, 9], [0, 4, 8]),
                             m=None, k=None, m_sub=[4, 3, 4, 2, 3, 4, 4, 3],
                             k_sub=[3, 2, 3, 1, 2, 3, 4, 3], model="random",
                             src=[[41.0, 37.0, 39.0], [12.0, 70.0, 20.0]],
                             rec=[[20.0, 20.0, 20.0], [50.0, 45.0, 40.0], [80.0, 80.0, 70.0],
                                  [50.0, 40.0, 40.0]])
    rs = pipeline.build(p)
    dt = pipeline.rom_dt(rs)
    n = 400
    w = np.stack([inputs.ricker(np.arange(n) * dt, p.f_peak),
                  inputs.ricker(np.arange(n) * dt - 0.01, p.f_peak)])
    ref = coupled.step_structured(rs, dt, n, w)
    return p, rs, dt, n, w, ref


def _run(sfm, rs, dt, n, w, precision):
    h = sfm.sfm_create(0)
    try:
        load_into(sfm, h, rs)
        tr, ms = sfm.sfm_run(h, precision, dt, n, w, rs.nshots, rs.nrec)
        return tr
    finally:
        sfm.sfm_destroy(h)


def test_uneven_fp64_matches_oracle(sfm, uneven):
    p, rs, dt, n, w, ref = uneven
    got = _run(sfm, rs, dt, n, w, sfm.SFM_FP64)
    assert pipeline.rel_l2(got, ref) <= FP64_TOL
    # every receiver, every shot, element by element
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 10 * FP64_TOL * scale


def test_uneven_fp32_matches_oracle(sfm, uneven):
    p, rs, dt, n, w, ref = uneven
    got = _run(sfm, rs, dt, n, w, sfm.SFM_FP32)
    assert pipeline.rel_l2(got, ref) <= FP32_GATE


def test_uneven_fp32x2_matches_oracle(sfm, uneven):
    p, rs, dt, n, w, ref = uneven
    got = _run(sfm, rs, dt, n, w, sfm.SFM_FP32X2)
    assert pipeline.rel_l2(got, ref) <= FP32X2_TOL


def test_uneven_fp32f_matches_oracle(sfm, uneven):
    p, rs, dt, n, w, ref = uneven
    got = _run(sfm, rs, dt, n, w, sfm.SFM_FP32F)
    assert pipeline.rel_l2(got, ref) <= FP32F_GATE


def test_uneven_fp32fx2_matches_oracle(sfm, uneven):
    p, rs, dt, n, w, ref = uneven
    got = _run(sfm, rs, dt, n, w, sfm.SFM_FP32FX2)
    f32f = _run(sfm, rs, dt, n, w, sfm.SFM_FP32F)
    print(f"uneven FP32FX2 {pipeline.rel_l2(got, ref):.3e}, FP32F {pipeline.rel_l2(f32f, ref):.3e}")
    assert pipeline.rel_l2(got, ref) <= FP32FX2_TOL
    assert np.abs(got - ref).max() <= 10 * FP32FX2_TOL * np.abs(ref).max()


def test_runs_are_bitwise_deterministic(sfm, uneven):
    p, rs, dt, n, w, ref = uneven
    a = _run(sfm, rs, dt, n, w, sfm.SFM_FP32)
    b = _run(sfm, rs, dt, n, w, sfm.SFM_FP32)
    assert np.array_equal(a, b)


def test_device_pointer_path_matches_host_path(sfm, uneven):
    torch = pytest.importorskip("torch")
    p, rs, dt, n, w, ref = uneven
    h = sfm.sfm_create(0)
    try:
        load_into(sfm, h, rs)
        host, _ = sfm.sfm_run(h, sfm.SFM_FP64, dt, n, w, rs.nshots, rs.nrec)
        wd = torch.tensor(w, dtype=torch.float64, device="cuda")
        td = torch.empty((rs.nshots, rs.nrec, n + 1), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        sfm.sfm_run(h, sfm.SFM_FP64, dt, n, None, rs.nshots, rs.nrec,
                    device_ptrs=(wd.data_ptr(), td.data_ptr()))
        assert np.array_equal(td.cpu().numpy(), host)
        assert sfm.sfm_last_launches(h) >= 2
    finally:
        sfm.sfm_destroy(h)


@pytest.mark.parametrize("precision", [0, 2, 3, 7])
def test_block_shapes_give_identical_traces(sfm, uneven, precision):
    """Consumer warps and ring stages change the grid, the per-block pieces
    (units cut at different levels) and which warp runs a tile row, never the
    order of any sum: traces are bitwise equal across shapes, and the shape
    the autotuner picks is one of its candidates."""
    p, rs, dt, n, w, ref = uneven
    h = sfm.sfm_create(0)
    try:
        load_into(sfm, h, rs)
        base, _ = sfm.sfm_run(h, precision, dt, n, w, rs.nshots, rs.nrec)
        for ncw, nst in ((1, 2), (2, 3), (6, 4), (8, 8), (3, 16)):
            sfm.sfm_debug_set(h, 3, ncw)
            sfm.sfm_debug_set(h, 4, nst)
            got, _ = sfm.sfm_run(h, precision, dt, n, w, rs.nshots, rs.nrec)
            assert np.array_equal(got, base), (ncw, nst)
        ncw, nst, us = sfm.sfm_autotune(h, precision, 50)
        assert ncw in (2, 4, 6, 8) and nst in (2, 3, 4, 6, 8, 12, 16) and us > 0
        if precision in (sfm.SFM_FP32F, sfm.SFM_FP32FX2):
            assert nst % ncw == 0
        got, _ = sfm.sfm_run(h, precision, dt, n, w, rs.nshots, rs.nrec)
        assert np.array_equal(got, base)
    finally:
        sfm.sfm_destroy(h)


def test_coefficients_round_trip(sfm, uneven):
    p, rs, dt, n, w, ref = uneven
    h = sfm.sfm_create(0)
    try:
        a = load_into(sfm, h, rs)
        assert np.array_equal(sfm.sfm_get_coeffs(h), a["coeffs"])
    finally:
        sfm.sfm_destroy(h)


def test_gpu_cfl_matches_oracle(sfm, uneven):
    p, rs, dt, n, w, ref = uneven
    lam_ref = coupled.lambda_max(rs)
    h = sfm.sfm_create(0)
    try:
        load_into(sfm, h, rs)
        lam, dtc = sfm.sfm_cfl_dt(h, 1000)
    finally:
        sfm.sfm_destroy(h)
    assert lam <= lam_ref * (1 + 1e-9)          # a Rayleigh quotient: from below
    assert abs(lam / lam_ref - 1.0) < 1e-4
    assert abs(dtc - 2.0 / np.sqrt(lam)) < 1e-15 * dtc + 1e-300


def test_unstable_step_is_reported(sfm, uneven):
    p, rs, dt, n, w, ref = uneven
    h = sfm.sfm_create(0)
    try:
        load_into(sfm, h, rs)
        big = 1.5 * dt / 0.9
        with pytest.raises(sfm.SfmError) as e:
            sfm.sfm_run(h, sfm.SFM_FP64, big, 20000,
                        np.zeros((rs.nshots, 20000)) + 1.0, rs.nshots, rs.nrec)
        assert e.value.code == sfm.SFM_ERR_UNSTABLE
    finally:
        sfm.sfm_destroy(h)


def test_barrier_timeout_is_bounded_and_recoverable(sfm, uneven):
    """One block skips its barrier arrival: every block's bounded wait runs
    out, the run returns SFM_ERR_TIMEOUT and the next run on the same handle
    is correct again."""
    p, rs, dt, n, w, ref = uneven
    h = sfm.sfm_create(0)
    try:
        load_into(sfm, h, rs)
        sfm.sfm_debug_set(h, 1, 200_000_000)     # 0.2 s limit
        sfm.sfm_debug_set(h, 2, 0)               # block 0 never arrives
        with pytest.raises(sfm.SfmError) as e:
            sfm.sfm_run(h, sfm.SFM_FP64, dt, 10, w[:, :10], rs.nshots, rs.nrec)
        assert e.value.code == sfm.SFM_ERR_TIMEOUT
        sfm.sfm_debug_set(h, 2, -1)
        got, _ = sfm.sfm_run(h, sfm.SFM_FP64, dt, n, w, rs.nshots, rs.nrec)
        assert pipeline.rel_l2(got, ref) <= FP64_TOL
    finally:
        sfm.sfm_destroy(h)


def test_argument_errors(sfm, uneven):
    p, rs, dt, n, w, ref = uneven
    h = sfm.sfm_create(0)
    try:
        with pytest.raises(sfm.SfmError) as e:
            sfm.sfm_run(h, sfm.SFM_FP64, dt, 5, w[:, :5], rs.nshots, rs.nrec)
        assert e.value.code == sfm.SFM_ERR_STATE
        a = load_into(sfm, h, rs)
        with pytest.raises(sfm.SfmError) as e:
            sfm.sfm_set_coeffs(h, a["coeffs"][:-1])
        assert e.value.code == sfm.SFM_ERR_ARG
        bad = a["nbr"].copy()
        bad[0, 1] = -1                            # breaks the neighbour symmetry
        with pytest.raises(sfm.SfmError) as e:
            sfm.sfm_set_topology(h, a["k_sub"], a["m_face"], bad)
        assert e.value.code == sfm.SFM_ERR_ARG
    finally:
        sfm.sfm_destroy(h)


def test_not_spd_face_block_is_rejected(sfm, uneven):
    p, rs, dt, n, w, ref = uneven
    h = sfm.sfm_create(0)
    try:
        from rom_abi import abi_arrays
        a = abi_arrays(rs)
        sfm.sfm_set_topology(h, a["k_sub"], a["m_face"], a["nbr"])
        c = a["coeffs"].copy()
        b0, k0 = rs.b[0], rs.k[0]
        gh1 = k0 * b0 * b0                        # Gammahat_1 of subdomain 0
        c[gh1] = -abs(c[gh1])                     # first diagonal entry negative
        with pytest.raises(sfm.SfmError) as e:
            sfm.sfm_set_coeffs(h, c)
        assert e.value.code == sfm.SFM_ERR_NOT_SPD
    finally:
        sfm.sfm_destroy(h)


def test_factored_mode_rejects_indefinite_block(sfm, uneven):
    """A Gamma_2 block that is not positive definite has no Cholesky factor:
    the factored FP32 mode reports it instead of stepping."""
    p, rs, dt, n, w, ref = uneven
    h = sfm.sfm_create(0)
    try:
        a = load_into(sfm, h, rs)
        c = a["coeffs"].copy()
        b0 = rs.b[0]
        c[b0 * b0] = -abs(c[b0 * b0])           # Gamma_2 of subdomain 0, entry (0, 0)
        sfm.sfm_set_coeffs(h, c)
        with pytest.raises(sfm.SfmError) as e:
            sfm.sfm_run(h, sfm.SFM_FP32F, dt, 10, w[:, :10], rs.nshots, rs.nrec)
        assert e.value.code == sfm.SFM_ERR_NOT_SPD
        sfm.sfm_set_coeffs(h, a["coeffs"])      # valid blocks again: the mode runs
        got, _ = sfm.sfm_run(h, sfm.SFM_FP32F, dt, n, w, rs.nshots, rs.nrec)
        assert pipeline.rel_l2(got, ref) <= FP32F_GATE
    finally:
        sfm.sfm_destroy(h)


@pytest.fixture(scope="module")
def cfg1():
    p = inputs.config1()
    rs = pipeline.build(p)
    dt = pipeline.rom_dt(rs)
    w = inputs.wavelet_samples(p, dt)
    ref = coupled.step_structured(rs, dt, p.nsteps, w)
    return p, rs, dt, w, ref


def test_config1_fp64_matches_oracle(sfm, cfg1):
    """48^3 cells in 2x2x2 subdomains, m = 4, k = 8, 500 steps, FP64."""
    p, rs, dt, w, ref = cfg1
    got = _run(sfm, rs, dt, p.nsteps, w, sfm.SFM_FP64)
    assert pipeline.rel_l2(got, ref) <= FP64_TOL


def test_config1_fp32x2_matches_oracle(sfm, cfg1):
    p, rs, dt, w, ref = cfg1
    got = _run(sfm, rs, dt, p.nsteps, w, sfm.SFM_FP32X2)
    assert pipeline.rel_l2(got, ref) <= FP32X2_TOL


def test_config1_fp32_matches_oracle(sfm, cfg1):
    p, rs, dt, w, ref = cfg1
    got = _run(sfm, rs, dt, p.nsteps, w, sfm.SFM_FP32)
    assert pipeline.rel_l2(got, ref) <= FP32_GATE


def test_config1_fp32f_matches_oracle(sfm, cfg1):
    p, rs, dt, w, ref = cfg1
    got = _run(sfm, rs, dt, p.nsteps, w, sfm.SFM_FP32F)
    assert pipeline.rel_l2(got, ref) <= FP32F_GATE


def test_config1_fp32fx2_matches_oracle(sfm, cfg1):
    p, rs, dt, w, ref = cfg1
    got = _run(sfm, rs, dt, p.nsteps, w, sfm.SFM_FP32FX2)
    assert pipeline.rel_l2(got, ref) <= FP32FX2_TOL


def per_trace_errors(got, ref):
    """Error of every (shot, receiver) trace relative to the RMS trace norm
    of its shot (rounding errors scale with the state, not with one trace's
    amplitude; a wrong receiver row or segment shows up at order one)."""
    num = np.linalg.norm(got - ref, axis=2)
    rms = np.sqrt(np.mean(np.linalg.norm(ref, axis=2) ** 2, axis=1, keepdims=True))
    return num / rms


def deep_fp64_tol(rs, nsteps):
    """FP64 tolerance of two summation orders of the same recurrence on deep
    ROMs: the U-form stepping amplifies a relative rounding eps by up to
    cond(G_j) = cond(Gammahat_j)^{1/2} per step (Eq. 13, Gammahat_j =
    G_j G_j^T), accumulated at most linearly by the stable leapfrog."""
    kappa = 1.0
    for s in range(rs.nsub):
        for B in rs.Gammahat[s][1:]:
            w = np.linalg.eigvalsh(0.5 * (B + B.T))
            kappa = max(kappa, w[-1] / max(w[0], w[-1] * 1e-300))
    return nsteps * np.finfo(np.float64).eps * np.sqrt(kappa)


@pytest.fixture(scope="module")
def cfg2_layered():
    """The 192^3, 8x8x8-subdomain geometry with m = 8, k = 16, one shot and
    the 1024-receiver line, on a laterally invariant layered model (layer
    jumps inside subdomains) so the oracle builds one ROM per subdomain
    layer; the workload's full 4000 steps."""
    p = inputs.config2()
    rng = np.random.default_rng(inputs.SEED)
    p.c = inputs.layered_lens(p.nx, p.ny, p.nz, p.h, rng, lens_amp=0.0)
    rs = pipeline.build(p)
    dt = pipeline.rom_dt(rs)
    w = inputs.wavelet_samples(p, dt)
    ref = coupled.step_structured(rs, dt, p.nsteps, w)
    return p, rs, dt, w, ref


def test_config2_geometry_fp64_matches_oracle(sfm, cfg2_layered):
    p, rs, dt, w, ref = cfg2_layered
    got = _run(sfm, rs, dt, p.nsteps, w, sfm.SFM_FP64)
    tol = deep_fp64_tol(rs, p.nsteps)
    print(f"config-2 geometry FP64, {p.nsteps} steps: {pipeline.rel_l2(got, ref):.3e} "
          f"(tolerance {tol:.3e}), worst trace {per_trace_errors(got, ref).max():.3e}")
    assert pipeline.rel_l2(got, ref) <= tol
    assert per_trace_errors(got, ref).max() <= tol


def test_config2_geometry_fp32x2_matches_oracle(sfm, cfg2_layered):
    """k = 16 levels: the S-fraction coefficients span ~1e10 in one block, out
    of reach of plain FP32 but not of the two-float mode."""
    p, rs, dt, w, ref = cfg2_layered
    got = _run(sfm, rs, dt, p.nsteps, w, sfm.SFM_FP32X2)
    print(f"config-2 geometry FP32x2: {pipeline.rel_l2(got, ref):.3e}, "
          f"worst trace {per_trace_errors(got, ref).max():.3e}")
    assert pipeline.rel_l2(got, ref) <= FP32X2_TOL
    assert per_trace_errors(got, ref).max() <= FP32X2_TOL


def test_config2_geometry_plain_fp32_is_unstable(sfm, cfg2_layered):
    """Plain FP32 coefficients of these k = 16 blocks turn indefinite (the
    factored modes exist for this): the run must end with SFM_ERR_UNSTABLE,
    not with finite wrong traces."""
    p, rs, dt, w, ref = cfg2_layered
    with pytest.raises(sfm.SfmError) as e:
        _run(sfm, rs, dt, p.nsteps, w, sfm.SFM_FP32)
    assert e.value.code == sfm.SFM_ERR_UNSTABLE


def test_config2_geometry_tf32x3_matches_oracle(sfm, cfg2_layered):
    p, rs, dt, w, ref = cfg2_layered
    got = _run(sfm, rs, dt, p.nsteps, w, sfm.SFM_TF32X3)
    print(f"config-2 geometry TF32X3: {pipeline.rel_l2(got, ref):.3e}, "
          f"worst trace {per_trace_errors(got, ref).max():.3e}")
    assert pipeline.rel_l2(got, ref) <= FP32F_GATE
    assert per_trace_errors(got, ref).max() <= FP32F_GATE


def test_config2_geometry_fp32f_matches_oracle(sfm, cfg2_layered):
    p, rs, dt, w, ref = cfg2_layered
    got = _run(sfm, rs, dt, p.nsteps, w, sfm.SFM_FP32F)
    print(f"config-2 geometry FP32F: {pipeline.rel_l2(got, ref):.3e}, "
          f"worst trace {per_trace_errors(got, ref).max():.3e}")
    assert pipeline.rel_l2(got, ref) <= FP32F_GATE
    assert per_trace_errors(got, ref).max() <= FP32F_GATE


def test_config2_geometry_fp32fx2_matches_oracle(sfm, cfg2_layered):
    """FP32 factor bytes at the FP32 target: every trace of the 4000-step
    run within 1e-5 of the oracle."""
    p, rs, dt, w, ref = cfg2_layered
    got = _run(sfm, rs, dt, p.nsteps, w, sfm.SFM_FP32FX2)
    print(f"config-2 geometry FP32FX2: {pipeline.rel_l2(got, ref):.3e}, "
          f"worst trace {per_trace_errors(got, ref).max():.3e}")
    assert pipeline.rel_l2(got, ref) <= FP32FX2_TOL
    assert per_trace_errors(got, ref).max() <= FP32FX2_TOL
