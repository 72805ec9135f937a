"""sfm_run_static: the FP64 stepping without any device allocation, for
callers that cannot allocate device memory when they step (their GPU memory
is owned by another allocator, or cudaMalloc's implicit synchronisation is
not acceptable in their loop).  Its traces must equal those of sfm_run and of
the FP64 oracle's coupled stepping, call after call; its scratch lives in one
static device array of fixed size, so free device memory must not change
across a call."""
import numpy as np
import pytest

import sfm_inputs as inputs
from oracle import coupled, pipeline

from rom_abi import abi_arrays, load_into

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-11


@pytest.fixture(scope="module")
def sfm():
    import os
    from paper_1406_6923_gb300 import _build, sfm as mod
    if not os.path.exists(mod.LIB_PATH):
        _build.build()
    mod.load()
    return mod


@pytest.fixture(scope="module")
def problem():
    p = inputs.small_problem(ncell=(10, 9, 8), cuts=([0, 5, 10], [0, 4, 9], [0, 4, 8]),
                             m=None, k=None, m_sub=[4, 3, 4, 2, 3, 4, 4, 3],
                             k_sub=[3, 2, 3, 1, 2, 3, 4, 3], model="random",
                             src=[[41.0, 37.0, 39.0], [12.0, 70.0, 20.0]],
                             rec=[[20.0, 20.0, 20.0], [50.0, 45.0, 40.0], [80.0, 80.0, 70.0],
                                  [50.0, 40.0, 40.0]])
    rs = pipeline.build(p)
    dt = pipeline.rom_dt(rs)
    n = 300
    w = np.stack([inputs.ricker(np.arange(n) * dt, p.f_peak),
                  inputs.ricker(np.arange(n) * dt - 0.01, p.f_peak)])
    return p, rs, dt, n, w


def test_static_entry_point_matches_sfm_run(sfm, problem):
    torch = pytest.importorskip("torch")
    p, rs, dt, n, w = problem
    h = sfm.sfm_create(0)
    try:
        load_into(sfm, h, rs)
        ref, _ = sfm.sfm_run(h, sfm.SFM_FP64, dt, n, w, rs.nshots, rs.nrec)
    finally:
        sfm.sfm_destroy(h)
    a = abi_arrays(rs)
    nshots, sp_shot, sp_sub, srows = a["src"]
    nrec, rp_rec, rp_sub, rrows = a["rec"]
    dev = torch.device("cuda:0")
    coeffs = torch.tensor(a["coeffs"], dtype=torch.float64, device=dev)
    srows_d = torch.tensor(srows, dtype=torch.float64, device=dev)
    rrows_d = torch.tensor(rrows, dtype=torch.float64, device=dev)
    wav = torch.tensor(w, dtype=torch.float64, device=dev)
    oracle_tr = coupled.step_structured(rs, dt, n, w)
    stream = torch.cuda.current_stream().cuda_stream
    outs = [torch.full((nshots, nrec, n + 1), float("nan"), dtype=torch.float64, device=dev)
            for _ in range(2)]
    for call in range(2):                      # two calls in a row share the scratch
        out = outs[call]
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info(0)[0]
        sfm.sfm_run_static(0, stream, a["k_sub"], a["m_face"], a["nbr"], coeffs.data_ptr(), nshots,
                           sp_shot, sp_sub, srows_d.data_ptr(), nrec, rp_rec, rp_sub,
                           rrows_d.data_ptr(), dt, n, wav.data_ptr(), out.data_ptr())
        torch.cuda.synchronize()
        free_after = torch.cuda.mem_get_info(0)[0]
        if call == 1:                          # the first call may load the module
            assert free_after == free_before, (free_before, free_after)
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        assert np.linalg.norm(got - ref) <= FP64_TOL * np.linalg.norm(ref), call
        assert np.linalg.norm(got - oracle_tr) <= FP64_TOL * np.linalg.norm(oracle_tr), call


def test_static_entry_point_rejects_oversized_problems(sfm, problem):
    p, rs, dt, n, w = problem
    a = abi_arrays(rs)
    nshots, sp_shot, sp_sub, srows = a["src"]
    nrec, rp_rec, rp_sub, rrows = a["rec"]
    # 3 million time steps of partial receiver sums exceed the 64 MiB scratch;
    # the size check runs before any device pointer is touched
    with pytest.raises(sfm.SfmError) as e:
        sfm.sfm_run_static(0, 0, a["k_sub"], a["m_face"], a["nbr"], 16, nshots, sp_shot, sp_sub,
                           16, nrec, rp_rec, rp_sub, 16, dt, 3_000_000, 16, 16)
    assert e.value.code == sfm.SFM_ERR_ARG
    assert "static limit" in sfm.sfm_last_error(None)
