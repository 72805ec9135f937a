"""Pins of the initial-value form (Algorithm 1 step 1.4 for u|t=0 and
du/dt|t=0, Eq. 16): the projection, face continuity, and the time
integrator's start against closed forms of the leapfrog recurrence."""
import numpy as np
import pytest

import sfm_inputs as inputs
from oracle import coupled, pipeline


def _smooth_field(p, seed, shots=1):
    """Smooth random nodal fields [shots][nz+1][ny+1][nx+1]: a Gaussian bump
    plus low-order polynomial terms (no method arithmetic)."""
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(np.arange(p.nz + 1), np.arange(p.ny + 1), np.arange(p.nx + 1),
                          indexing="ij")
    out = []
    for _ in range(shots):
        c = rng.uniform(0.3, 0.7, 3) * np.array([p.nx, p.ny, p.nz])
        w = 0.25 * min(p.nx, p.ny, p.nz)
        f = np.exp(-((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) / (2 * w * w))
        f = f + 0.1 * rng.standard_normal() * x / p.nx + 0.05 * rng.standard_normal() * y * z / (p.ny * p.nz)
        out.append(f)
    return np.stack(out)


def test_state_projection_inverts_the_reconstruction():
    """A field in the ROM subspace, u = M^{-1/2} V Qh z, projects to
    U_j = G_j z_j, and the receiver-side reconstruction z_j = G_j^{-1} U_j
    returns it (a transposed or inverted G fails)."""
    p = inputs.small_problem(ncell=(6, 5, 4), cuts=([0, 6], [0, 5], [0, 4]), m=3, k=3)
    rs = pipeline.build(p, keep=True)
    sr = rs.subroms[0]
    rng = np.random.default_rng(3)
    z = rng.standard_normal(sr.Qh.shape[1])
    u = (sr.V @ (sr.Qh @ z)) / np.sqrt(sr.mass)
    U = sr.state_rows(u)
    b = U.shape[1]
    for j in range(U.shape[0]):
        np.testing.assert_allclose(U[j], sr.G[j] @ z[j * b:(j + 1) * b], rtol=0, atol=1e-11 * np.abs(U).max())
    back = np.concatenate([np.linalg.solve(sr.G[j], U[j]) for j in range(U.shape[0])])
    np.testing.assert_allclose(back, z, rtol=0, atol=1e-10 * np.abs(z).max())


def test_face_blocks_of_a_projected_field_agree_across_shared_faces():
    """On level 1 the projection is B^T u, so both sides of a shared face
    carry the same face data (the continuity condition of Eq. 17)."""
    p = inputs.small_problem(ncell=(8, 6, 5), cuts=([0, 4, 8], [0, 6], [0, 5]), m=3, k=3,
                             model="random")
    u0 = _smooth_field(p, 5)
    rs = pipeline.build(p, u0=u0)
    a, b = rs.U0[0][0][0], rs.U0[0][1][0]
    fa = rs.topo.face_slices(0)[1]          # +x face of subdomain 0
    fb = rs.topo.face_slices(1)[0]          # -x face of subdomain 1
    np.testing.assert_allclose(a[fa], b[fb], rtol=0, atol=1e-12 * np.abs(a[fa]).max())
    assert np.abs(a[fa]).max() > 1e-6


@pytest.fixture(scope="module")
def coupled_small():
    p = inputs.small_problem(ncell=(8, 8, 6), cuts=(4, 4, 3), m=3, k=3, model="random",
                             rec=[[20.0, 20.0, 20.0], [55.0, 45.0, 30.0], [70.0, 10.0, 50.0]])
    rs = pipeline.build(p)
    asm = coupled.Assembled(rs)
    return p, rs, asm


def _rows_from_flat(rs, asm, x):
    """Per-subdomain (k, b) rows of an assembled state vector (one shot)."""
    return [{s: x[asm.E[s]].reshape(rs.k[s], rs.b[s]) for s in range(rs.nsub)}]


def test_eigenmode_start_follows_the_discrete_cosine_and_sine(coupled_small):
    """For an eigenvector phi of MM^{-1} KK (eigenvalue lam) the leapfrog with
    U^0 = phi, V^0 = 0 and the second-order start gives U^n = phi cos(n th)
    with 2 (1 - cos th) = dt^2 lam; with U^0 = 0, V^0 = phi it gives
    U^n = dt phi sin(n th) / sin th.  Checked on the receiver traces."""
    p, rs, asm = coupled_small
    cs = []
    for m in asm.minv_blocks:
        w, U = np.linalg.eigh(0.5 * (m + m.T))
        cs.append(U * np.sqrt(np.maximum(w, 0.0)))
    from scipy.linalg import block_diag
    C = block_diag(*cs)
    lam_all, Y = np.linalg.eigh(C.T @ asm.KK.toarray() @ C)
    dt = 0.9 * 2.0 / np.sqrt(lam_all[-1])
    nsteps = 200
    w = np.zeros((1, nsteps))
    for idx in (len(lam_all) // 2, len(lam_all) - 3):
        lam = lam_all[idx]
        phi = C @ Y[:, idx]
        th = np.arccos(1.0 - 0.5 * dt * dt * lam)
        n = np.arange(nsteps + 1)
        ref_rows = asm.R @ phi
        got = coupled.step_structured(rs, dt, nsteps, w, U0=_rows_from_flat(rs, asm, phi))[0]
        ref = ref_rows[:, None] * np.cos(n * th)[None, :]
        assert pipeline.rel_l2(got, ref) < 1e-9, idx
        got = coupled.step_structured(rs, dt, nsteps, w, V0=_rows_from_flat(rs, asm, phi))[0]
        ref = dt * ref_rows[:, None] * (np.sin(n * th) / np.sin(th))[None, :]
        assert pipeline.rel_l2(got, ref) < 1e-9, idx


def test_initial_value_stepping_equals_the_assembled_leapfrog(coupled_small):
    """Projected initial displacement and velocity (plus the source): the
    structured scheme equals a generic leapfrog of the assembled system
    started with delta^0 = dt V^0 - dt^2/2 MM^{-1}(-KK U^0)."""
    p, rs0, asm = coupled_small
    u0 = _smooth_field(p, 11)
    v0 = 1e3 * _smooth_field(p, 12)
    rs = pipeline.build(p, u0=u0, v0=v0)
    dt = 0.9 * asm.cfl_dt()
    nsteps = 150
    w = inputs.ricker(np.arange(nsteps) * dt, p.f_peak)[None, :]
    got = coupled.step_structured(rs, dt, nsteps, w, U0=rs.U0, V0=rs.V0)
    X0 = np.zeros((asm.n, 1))
    V = np.zeros((asm.n, 1))
    for s in range(rs.nsub):
        X0[asm.E[s], 0] = rs.U0[0][s].ravel()
        V[asm.E[s], 0] = rs.V0[0][s].ravel()
    d0 = dt * V - 0.5 * dt * dt * (asm.MMinv @ (-(asm.KK @ X0)))
    ref = asm.leapfrog(dt, nsteps, w, U0=X0, dU0=d0)
    assert np.abs(ref).max() > 0
    assert pipeline.rel_l2(got, ref) < 1e-12


def test_energy_is_conserved_from_initial_data(coupled_small):
    """No source: the discrete energy of the assembled leapfrog started from
    projected initial data stays constant."""
    p, rs0, asm = coupled_small
    rs = pipeline.build(p, u0=_smooth_field(p, 21), v0=1e3 * _smooth_field(p, 22))
    X0 = np.zeros((asm.n, 1))
    V = np.zeros((asm.n, 1))
    for s in range(rs.nsub):
        X0[asm.E[s], 0] = rs.U0[0][s].ravel()
        V[asm.E[s], 0] = rs.V0[0][s].ravel()
    dt = 0.9 * asm.cfl_dt()
    d0 = dt * V - 0.5 * dt * dt * (asm.MMinv @ (-(asm.KK @ X0)))
    out, en, U, dU = asm.leapfrog(dt, 2000, np.zeros((1, 2000)), U0=X0, dU0=d0, energies=True)
    assert abs(en).max() > 0
    assert np.abs(en - en[0]).max() / abs(en[0]) < 1e-10
