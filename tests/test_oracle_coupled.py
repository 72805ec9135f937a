"""Pins of the oracle's online stage: Algorithm 1 stage 2 (Eqs. 17-19) with
leapfrog, against the assembled system, energy, CFL, symmetry and the fine
grid it converges to."""
import numpy as np
import pytest

import sfm_inputs as inputs
from oracle import coupled, faces, fine, pipeline


@pytest.fixture(scope="module")
def uneven():
    """Uneven boxes, uneven m (so shared faces take the smaller m) and k, two shots."""
    p = inputs.small_problem(ncell=(10, 9, 8), cuts=([0, 5, 10], [0, 4, 9], [0, 4, 8]),
                             m=None, k=None, m_sub=[4, 3, 4, 2, 3, 4, 4, 3],
                             k_sub=[3, 2, 3, 3, 2, 3, 4, 3], model="random",
                             src=[[41.0, 37.0, 39.0], [12.0, 70.0, 20.0]],
                             rec=[[20.0, 20.0, 20.0], [50.0, 45.0, 40.0], [80.0, 80.0, 70.0]])
    return p, pipeline.build(p)


def test_structured_stepping_equals_the_assembled_leapfrog(uneven):
    p, rs = uneven
    A = coupled.Assembled(rs)
    dt = 0.9 * A.cfl_dt()
    w = np.stack([inputs.ricker(np.arange(400) * dt, p.f_peak),
                  inputs.ricker(np.arange(400) * dt - 0.01, p.f_peak)])
    d1 = coupled.step_structured(rs, dt, 400, w)
    d2 = A.leapfrog(dt, 400, w)
    assert pipeline.rel_l2(d1, d2) < 1e-12
    assert np.abs(d1).max() > 0


def test_outer_face_coupling_is_the_own_block(uneven):
    p, rs = uneven
    topo = rs.topo
    for g, sides in enumerate(topo.face_sides):
        if len(sides) == 1:
            s, f = sides[0]
            sl = topo.face_slices(s)[f]
            np.testing.assert_allclose(rs.H[g], rs.Gammahat[s][0][sl, sl], rtol=1e-12)
        else:
            (a, fa), (b, fb) = sides
            Ha = rs.Gammahat[a][0][topo.face_slices(a)[fa]][:, topo.face_slices(a)[fa]]
            Hb = rs.Gammahat[b][0][topo.face_slices(b)[fb]][:, topo.face_slices(b)[fb]]
            # H^{-1} = Ha^{-1} + Hb^{-1}
            np.testing.assert_allclose(np.linalg.inv(rs.H[g]),
                                       np.linalg.inv(Ha) + np.linalg.inv(Hb), rtol=1e-10)


def test_discrete_energy_is_conserved_after_the_source(uneven):
    p, rs = uneven
    A = coupled.Assembled(rs)
    dt = 0.9 * A.cfl_dt()
    n_on = 60
    w = np.zeros((2, 2000))
    w[:, :n_on] = np.sin(np.arange(n_on) * 0.3)
    _, en, _, _ = A.leapfrog(dt, 2000, w, energies=True)
    e = en[n_on:]
    # any inconsistency of the scheme shows at O(dt^2) ~ 1e-3; rounding through
    # the badly conditioned mass blocks Gammahat_j^{-1} leaves ~1e-12
    assert np.abs(e - e[0]).max() < 1e-10 * np.abs(e[0]).max()
    assert np.all(e > 0)


def test_rom_cfl_limit_is_sharp(uneven):
    p, rs = uneven
    A = coupled.Assembled(rs)
    dtc = A.cfl_dt()
    rng = np.random.default_rng(5)
    U0 = 1e-6 * rng.standard_normal((A.n, 2))
    out = {}
    for f in (0.99, 1.01):
        U, dU = U0.copy(), np.zeros_like(U0)
        dt = f * dtc
        for _ in range(10000):
            dU = dU + dt * dt * (A.MMinv @ (-(A.KK @ U)))
            U = U + dU
            if np.abs(U).max() > 1e3:
                break
        out[f] = np.abs(U).max()
    assert out[0.99] < 1e-4 and out[1.01] > 1e3


def test_symmetric_problem_gives_symmetric_traces():
    """Uniform medium, source at the centre of a 2x2x2 split, six receivers at
    mirror/rotation images of each other: all traces agree."""
    n, h = 12, 10.0
    ctr = n * h / 2
    rec = [[ctr - 30, ctr, ctr], [ctr + 30, ctr, ctr], [ctr, ctr - 30, ctr],
           [ctr, ctr + 30, ctr], [ctr, ctr, ctr - 30], [ctr, ctr, ctr + 30]]
    p = inputs.small_problem(ncell=(n, n, n), cuts=(6, 6, 6), m=4, k=3, model="uniform",
                             src=[[ctr, ctr, ctr]], rec=rec)
    rs = pipeline.build(p)
    dt = 0.9 * coupled.Assembled(rs).cfl_dt()
    d = coupled.step_structured(rs, dt, 300, inputs.wavelet_samples(p, dt, 300))[0]
    scale = np.abs(d).max()
    assert scale > 0
    for r in range(1, 6):
        assert np.abs(d[r] - d[0]).max() < 1e-10 * scale


def test_identical_blocks_give_identical_coefficients():
    p = inputs.small_problem(ncell=(8, 8, 8), cuts=(4, 4, 4), m=3, k=3, model="uniform")
    rs = pipeline.build(p)
    for s in range(1, p.nsub):
        np.testing.assert_allclose(rs.Gamma[s], rs.Gamma[0], rtol=0, atol=1e-12 * np.abs(rs.Gamma[0]).max())
        np.testing.assert_allclose(rs.Gammahat[s], rs.Gammahat[0], rtol=0,
                                   atol=1e-12 * np.abs(rs.Gammahat[0]).max())


@pytest.mark.slow
def test_rom_converges_to_the_slit_fine_grid():
    """With the open-face reading the ROM's limit is the fine grid with only
    open-face nodes shared; the trace error to it falls as m and k grow."""
    base = inputs.small_problem(ncell=(16, 16, 16), cuts=(8, 8, 8), m=4, k=2, model="layers")
    ss = pipeline.slit_system(base)
    dtf = 0.9 * fine.cfl_dt(ss[0], ss[1])
    nf = 400
    T = nf * dtf
    ref = pipeline.fine_traces(ss, dtf, nf, inputs.ricker(np.arange(nf) * dtf, base.f_peak)[None])
    tf = np.arange(nf + 1) * dtf
    errs = []
    for m, k in [(4, 2), (4, 4), (9, 5), (16, 5)]:
        p = inputs.small_problem(ncell=(16, 16, 16), cuts=(8, 8, 8), m=m, k=k, model="layers")
        rs = pipeline.build(p)
        dt = 0.9 * coupled.Assembled(rs).cfl_dt()
        n = int(T / dt) + 1
        d = coupled.step_structured(rs, dt, n, inputs.ricker(np.arange(n) * dt, p.f_peak)[None])
        tr = np.arange(n + 1) * dt
        di = np.stack([[np.interp(tf, tr, d[0, r]) for r in range(d.shape[1])]])
        errs.append(pipeline.rel_l2(di, ref))
    assert all(a > b for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-2, errs


def test_lanczos_max_matches_dense_eigvalsh():
    """The stability limits use a Lanczos iteration; pin it to LAPACK's
    dense eigenvalues on the assembled ROM system and a random SPD matrix."""
    from oracle.eig import lanczos_max
    rng = np.random.default_rng(3)
    X = rng.standard_normal((300, 300))
    A = X @ X.T
    assert abs(lanczos_max(lambda v: A @ v, 300) / np.linalg.eigvalsh(A)[-1] - 1) < 1e-10
    p = inputs.small_problem(ncell=(8, 8, 8), cuts=(4, 4, 4), m=4, k=3, model="random")
    rs = pipeline.build(p)
    A = coupled.Assembled(rs)
    assert abs(coupled.lambda_max(rs) / A.lambda_max() - 1) < 1e-10
