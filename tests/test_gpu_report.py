"""GPU tests of the run report (sfm_run_report): the discrete energy of the
leapfrog (Stage 2; the assembled form of Eqs. 17-19, MM U'' = -KK U) against
the oracle's assembled system and its conservation without a source, the
instability sentinel, and the report's bookkeeping."""
import numpy as np
import pytest

import sfm_inputs as inputs
from oracle import coupled, pipeline

from rom_abi import load_into

pytestmark = pytest.mark.gpu

# Two FP64 evaluations of the same quadratic forms in different orders, on
# well-conditioned small ROMs.
ENERGY_TOL = 1e-10


@pytest.fixture(scope="module")
def sfm():
    import os
    from paper_1406_6923_gb300 import _build, sfm as mod
    if not os.path.exists(mod.LIB_PATH):
        _build.build()
    mod.load()
    return mod


def _fields(p, seed, shots):
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
def free():
    """Uneven boxes and (m, k), two shots with their own initial displacement
    and velocity and no source term (zero wavelet): a free oscillation."""
    p = inputs.small_problem(ncell=(10, 9, 8), cuts=([0, 5, 10], [0, 4, 9], [0, 4, 8]),
                             m=None, k=None, m_sub=[4, 3, 4, 2, 3, 4, 4, 3],
                             k_sub=[3, 2, 3, 1, 2, 3, 4, 3], model="random",
                             src=[[41.0, 37.0, 39.0], [12.0, 70.0, 20.0]],
                             rec=[[20.0, 20.0, 20.0], [50.0, 45.0, 40.0], [80.0, 80.0, 70.0]])
    rs = pipeline.build(p, u0=_fields(p, 31, 2), v0=2e3 * _fields(p, 32, 2))
    dt = pipeline.rom_dt(rs)
    n = 300
    return p, rs, dt, n, np.zeros((rs.nshots, n))


def _set_initial(sfm, h, rs):
    shots, subs, u, v = [], [], [], []
    for q in range(len(rs.U0)):
        for s in sorted(rs.U0[q]):
            shots.append(q)
            subs.append(s)
            u.append(rs.U0[q][s].ravel())
            v.append(rs.V0[q][s].ravel())
    sfm.sfm_set_initial(h, rs.nshots, shots, subs, np.concatenate(u), np.concatenate(v))


def _assembled(A, rs, states):
    """State-layout vectors (per shot: subdomains in order, levels 1..k of b)
    as columns of the oracle's assembled vector."""
    out = np.zeros((A.n, len(states)))
    for q, x in enumerate(states):
        off = 0
        for s in range(rs.nsub):
            kb = rs.k[s] * rs.b[s]
            out[A.E[s], q] = x[off:off + kb]
            off += kb
    return out


def _oracle_energies(rs, dt, n):
    """Energies E^{n+1/2}, n = 0..N-1, of the oracle's generic leapfrog of the
    assembled system from the same start (U^0, delta^0 = dt V^0 - dt^2/2
    MM^{-1} (-KK U^0))."""
    A = coupled.Assembled(rs)
    U0 = np.zeros((A.n, rs.nshots))
    V0 = np.zeros((A.n, rs.nshots))
    for q in range(rs.nshots):
        for s, rows in rs.U0[q].items():
            U0[A.E[s], q] = rows.ravel()
        for s, rows in rs.V0[q].items():
            V0[A.E[s], q] = rows.ravel()
    d0 = dt * V0 - 0.5 * dt * dt * (A.MMinv @ (-(A.KK @ U0)))
    _, en, _, _ = A.leapfrog(dt, n, np.zeros((rs.nshots, n)), U0=U0, dU0=d0, energies=True)
    return A, en


def test_energy_matches_the_oracle_and_is_conserved(sfm, free):
    p, rs, dt, n, w = free
    h = sfm.sfm_create(0)
    try:
        load_into(sfm, h, rs)
        _set_initial(sfm, h, rs)
        sfm.sfm_run(h, sfm.SFM_FP64, dt, n, w, rs.nshots, rs.nrec, energy=True)
        rep = sfm.sfm_run_report(h)
        blob = np.frombuffer(sfm.sfm_checkpoint(h), dtype=np.int64)
    finally:
        sfm.sfm_destroy(h)
    A, en = _oracle_energies(rs, dt, n)
    e0, e1 = rep["energy_start"], rep["energy_end"]
    print(f"energy start {e0}, end {e1}; oracle E^1/2 {en[0]}, E^(N-1/2) {en[-1]}")
    # E^{-1/2} equals E^{1/2} without a source; E^{N-1/2} is the oracle's last
    np.testing.assert_allclose(e0, en[0], rtol=ENERGY_TOL)
    np.testing.assert_allclose(e1, en[-1], rtol=ENERGY_TOL)
    np.testing.assert_allclose(e1, e0, rtol=ENERGY_TOL)
    # the reported end energy is the oracle's energy of the GPU's own state
    nst = int(blob[3])
    st = blob[8:].view(np.float64)
    U = st[:rs.nshots * nst].reshape(rs.nshots, nst)
    D = st[rs.nshots * nst:].reshape(rs.nshots, nst)
    Ua, Da = _assembled(A, rs, U), _assembled(A, rs, D)
    np.testing.assert_allclose(e1, A.energy(Ua, Ua - Da, dt), rtol=ENERGY_TOL)


@pytest.mark.parametrize("prec", ["SFM_FP32F", "SFM_TF32X3", "SFM_FP32FX2"])
def test_fp32_class_energy_stays_near_fp64(sfm, free, prec):
    """FP32 state and sums: the energy carries the state's FP32 rounding."""
    p, rs, dt, n, w = free
    h = sfm.sfm_create(0)
    try:
        load_into(sfm, h, rs)
        _set_initial(sfm, h, rs)
        sfm.sfm_run(h, sfm.SFM_FP64, dt, n, w, rs.nshots, rs.nrec, energy=True)
        ref = sfm.sfm_run_report(h)["energy_end"]
        sfm.sfm_run(h, getattr(sfm, prec), dt, n, w, rs.nshots, rs.nrec, energy=True)
        got = sfm.sfm_run_report(h)
    finally:
        sfm.sfm_destroy(h)
    print(f"{prec}: energy end {got['energy_end']} vs FP64 {ref}")
    np.testing.assert_allclose(got["energy_end"], ref, rtol=1e-4)
    np.testing.assert_allclose(got["energy_end"], got["energy_start"], rtol=1e-4)


@pytest.mark.parametrize("prec", ["SFM_FP64", "SFM_FP32F", "SFM_TF32X3", "SFM_FP32FX2"])
def test_sentinel_stops_an_unstable_run_early(sfm, free, prec):
    """Twice the CFL step: the state runs away within tens of steps; the
    sentinel must end a 50000-step run long before its end."""
    p, rs, dt, n, w = free
    nsteps = 50000
    h = sfm.sfm_create(0)
    try:
        load_into(sfm, h, rs)
        _set_initial(sfm, h, rs)
        with pytest.raises(sfm.SfmError) as e:
            sfm.sfm_run(h, getattr(sfm, prec), 2.0 * dt / 0.9, nsteps, np.zeros((rs.nshots, nsteps)),
                        rs.nshots, rs.nrec)
        rep = sfm.sfm_run_report(h)
    finally:
        sfm.sfm_destroy(h)
    assert e.value.code == sfm.SFM_ERR_UNSTABLE
    print(f"{prec}: stopped at step {rep['unstable_step']} of {nsteps}")
    assert 0 <= rep["unstable_step"] < nsteps // 10
    assert rep["status"] == sfm.SFM_ERR_UNSTABLE


def test_report_bookkeeping(sfm, free):
    p, rs, dt, n, w = free
    h = sfm.sfm_create(0)
    try:
        load_into(sfm, h, rs)
        sfm.sfm_run(h, sfm.SFM_FP32F, dt, n, np.ones((rs.nshots, n)), rs.nshots, rs.nrec)
        rep = sfm.sfm_run_report(h)
    finally:
        sfm.sfm_destroy(h)
    assert rep["precision"] == sfm.SFM_FP32F and rep["nsteps"] == n and rep["nshots"] == rs.nshots
    assert rep["status"] == 0 and rep["unstable_step"] == -1 and rep["energy"] == 0
    assert rep["launches"] >= 2 and 0 < rep["kernel_ms"] <= rep["total_ms"]
    assert "energy_start" not in rep
