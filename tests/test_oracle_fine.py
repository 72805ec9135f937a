"""Pins of the oracle's fine-grid operator (Eq. 1 reading) and face basis."""
import numpy as np
import scipy.sparse as sp
import pytest

import sfm_inputs as inputs
from oracle import fine, faces, pipeline


def _problem(**kw):
    args = dict(ncell=(9, 7, 8), cuts=([0, 4, 9], [0, 3, 7], [0, 5, 8]), m=2, k=2,
                model="random")
    args.update(kw)
    return inputs.small_problem(**args)


def test_subdomain_operators_sum_to_global():
    """sum_a E_a^T K^a E_a = K and sum_a E_a^T M^a = M (per-cell assembly)."""
    p = _problem()
    K, M = fine.assemble_global(p)
    gbox = fine.global_box(p)
    Ks = sp.csr_matrix(K.shape)
    Ms = np.zeros_like(M)
    for s in range(p.nsub):
        box = p.sub_box(s)
        Ka, Ma = fine.assemble(p.c, p.h, box)
        g = fine.node_index(gbox, *fine.node_coords(box))
        P = sp.csr_matrix((np.ones(len(g)), (g, np.arange(len(g)))), shape=(K.shape[0], len(g)))
        Ks = Ks + P @ Ka @ P.T
        np.add.at(Ms, g, Ma)
    assert abs(Ks - K).max() == 0.0          # conductances are multiples of h/4
    np.testing.assert_allclose(Ms, M, rtol=1e-14)   # up to the order of the sums


def test_uniform_interior_rows_are_7_point_laplacian():
    c0, h = 1800.0, 7.0
    p = _problem(model="uniform")
    p.c[:] = c0
    p.h = h
    K, M = fine.assemble_global(p)
    A = sp.diags(1.0 / M) @ K          # = -c^2 Lap_h on interior nodes
    box = fine.global_box(p)
    i, j, k = 4, 3, 5
    r = int(fine.node_index(box, i, j, k))
    row = A.getrow(r).toarray().ravel()
    expect = np.zeros_like(row)
    expect[r] = 6.0 * c0 ** 2 / h ** 2
    for d in [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]:
        expect[int(fine.node_index(box, i + d[0], j + d[1], k + d[2]))] = -c0 ** 2 / h ** 2
    np.testing.assert_allclose(row, expect, rtol=1e-13, atol=1e-9)
    assert np.isclose(M[r], h ** 3 / c0 ** 2, rtol=1e-14)


def test_neumann_null_space_and_psd():
    p = _problem()
    K, M = fine.assemble(p.c, p.h, p.sub_box(3))
    assert np.abs(K @ np.ones(K.shape[0])).max() < 1e-12
    w = np.linalg.eigvalsh(K.toarray())
    assert w.min() > -1e-12 * w.max() and abs(w[0]) < 1e-10 * w.max()
    assert w[1] > 1e-8 * w.max()          # one connected box: one null vector


def test_fine_energy_is_conserved():
    p = _problem()
    K, M = fine.assemble_global(p)
    dt = 0.9 * fine.cfl_dt(K, M)
    rng = np.random.default_rng(0)
    u_old = rng.standard_normal(K.shape[0])
    u = u_old + 0.01 * rng.standard_normal(K.shape[0])
    e0 = fine.energy(K, M, u, u_old, dt)
    for _ in range(500):
        v = (u - u_old) + dt * dt * (-(K @ u)) / M
        u_old, u = u, u + v
    assert abs(fine.energy(K, M, u, u_old, dt) - e0) < 1e-12 * abs(e0)


def test_fine_cfl_is_sharp():
    p = _problem()
    K, M = fine.assemble_global(p)
    dtc = fine.cfl_dt(K, M)
    rng = np.random.default_rng(1)
    grow = {}
    for f in (0.99, 1.01):
        dt = f * dtc
        u_old = np.zeros(K.shape[0])
        u = 1e-6 * rng.standard_normal(K.shape[0])
        for _ in range(3000):
            u_old, u = u, 2 * u - u_old - dt * dt * (K @ u) / M
            if np.abs(u).max() > 1e6:
                break
        grow[f] = np.abs(u).max()
    assert grow[0.99] < 1e-3 and grow[1.01] > 1e3


def test_fine_fdtd_matches_3d_greens_function():
    """A point force in a homogeneous medium: ``(1/c^2) u_tt = Lap u + delta f``
    gives ``u = f(t - r/c) / (4 pi r)``; the fine FDTD reproduces it up to grid
    dispersion before any boundary reflection arrives."""
    n, h, c0, f0 = 60, 10.0, 2000.0, 10.0
    p = inputs.small_problem(ncell=(n, n, n), cuts=(n, n, n), model="uniform",
                             src=[[300.0, 300.0, 300.0]], rec=[[360.0, 300.0, 300.0],
                                                               [300.0, 370.0, 300.0]])
    p.c[:] = c0
    p.src_sigma = 1e-3 * h                      # a single-node force
    p.f_peak = f0
    K, M, force, R = pipeline.fine_system(p)
    dt = 0.5 * fine.cfl_dt(K, M)
    nt = int(0.3 / dt)
    t = np.arange(nt + 1) * dt
    w = inputs.ricker(t, f0)
    d = fine.leapfrog(K, M, dt, nt, force[:, 0], w, R)
    for r, dist in enumerate([60.0, 70.0]):
        g = inputs.ricker(t - dist / c0, f0) / (4 * np.pi * dist)
        err = np.linalg.norm(d[r] - g) / np.linalg.norm(g)
        assert err < 2e-2, err                                 # 20 points per wavelength
        assert abs(np.dot(d[r], g) / np.dot(g, g) - 1.0) < 1e-2  # amplitude scale


def test_face_mode_order():
    assert faces.mode_list(23, 23, 8) == [(0, 0), (1, 0), (0, 1), (1, 1), (2, 0), (0, 2),
                                          (2, 1), (1, 2)]


def test_face_supports_are_open_and_disjoint():
    p = _problem()
    box = p.sub_box(0)
    seen = set()
    nxl, nyl, nzl = fine.box_shape(box)
    for f in range(6):
        idx, s, t, (ns, nt) = faces.open_face_nodes(box, f)
        assert len(idx) == ns * nt
        assert not (seen & set(idx.tolist()))
        seen |= set(idx.tolist())
        i, j, k = fine.node_coords(box)
        on_edge = 0
        for li in idx:
            q = np.array([i[li] - box[0], j[li] - box[2], k[li] - box[4]])
            ext = np.array([nxl - 1, nyl - 1, nzl - 1])
            on_edge += int(np.sum((q == 0) | (q == ext)) >= 2)
        assert on_edge == 0


def test_shared_face_basis_agrees_on_both_sides():
    """Both sides of a shared face put the same function on the same node."""
    p = _problem()
    topo = faces.Topology(p)
    for s in range(p.nsub):
        for f in range(6):
            t = topo.nbr[s, f]
            if t < 0:
                continue
            m = topo.mf[s, f]
            ia, va = faces.face_B(p.sub_box(s), f, m, p.h)
            ib, vb = faces.face_B(p.sub_box(t), f ^ 1, m, p.h)
            ga = fine.node_coords(p.sub_box(s))
            gb = fine.node_coords(p.sub_box(t))
            ka = [(ga[0][q], ga[1][q], ga[2][q]) for q in ia]
            kb = [(gb[0][q], gb[1][q], gb[2][q]) for q in ib]
            assert ka == kb
            assert np.array_equal(va, vb)


def test_fine_initial_value_start_follows_the_discrete_cosine_and_sine():
    """The fine leapfrog's initial-value start: for an eigenvector phi of
    M^{-1} K (K phi = lam M phi), u0 = phi gives u^n = phi cos(n th) with
    2 (1 - cos th) = dt^2 lam, and v0 = phi gives dt phi sin(n th) / sin th."""
    p = inputs.small_problem(ncell=(5, 4, 3), cuts=(5, 4, 3), model="random")
    K, mass = fine.assemble(p.c, p.h, fine.global_box(p))
    s = 1.0 / np.sqrt(mass)
    lam_all, Y = np.linalg.eigh((s[:, None] * K.toarray()) * s[None, :])
    dt = 0.9 * 2.0 / np.sqrt(lam_all[-1])
    nsteps = 300
    R = sp.identity(K.shape[0], format="csr")[::7]
    zero = np.zeros(K.shape[0])
    n = np.arange(nsteps + 1)
    for idx in (1, K.shape[0] // 2, K.shape[0] - 2):
        phi = s * Y[:, idx]
        th = np.arccos(1.0 - 0.5 * dt * dt * lam_all[idx])
        got = fine.leapfrog(K, mass, dt, nsteps, zero, np.zeros(nsteps), R, u0=phi)
        ref = (R @ phi)[:, None] * np.cos(n * th)[None, :]
        assert pipeline.rel_l2(got, ref) < 1e-9, idx
        got = fine.leapfrog(K, mass, dt, nsteps, zero, np.zeros(nsteps), R, v0=phi)
        ref = dt * (R @ phi)[:, None] * (np.sin(n * th) / np.sin(th))[None, :]
        assert pipeline.rel_l2(got, ref) < 1e-9, idx


def test_slit_field_copies_every_node_value():
    """Every slit unknown of a node carries the node's value, and a field
    that is constant stays constant; the slit grid has one extra copy per
    extra subdomain sharing an edge or corner node."""
    p = inputs.small_problem(ncell=(8, 8, 8), cuts=(4, 4, 4), model="random")
    pieces, n = pipeline.slit_nodes(p)
    rng = np.random.default_rng(5)
    field = rng.standard_normal((p.nz + 1, p.ny + 1, p.nx + 1))
    u = pipeline.slit_field(p, field)
    for box, gidx in pieces:
        i, j, k = fine.node_coords(box)
        np.testing.assert_array_equal(u[gidx], field[k, j, i])
    assert np.all(pipeline.slit_field(p, np.ones_like(field)) == 1.0)
    K, mass, _, _ = pipeline.slit_system(p)
    assert K.shape == (n, n) and n > (p.nx + 1) * (p.ny + 1) * (p.nz + 1)
    assert abs(mass.sum() - fine.global_mass_ijk(p).sum()) < 1e-9 * mass.sum()
