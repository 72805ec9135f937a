"""Pins of the oracle's offline stage: Krylov ROM (Eqs. 5-7), block Lanczos
(Eq. 8), S-fraction transform (Eq. 13), transfer functions (Eqs. 4, 9, 15)
and the source/receiver rows of Eq. (16)."""
import numpy as np
import pytest

import sfm_inputs as inputs
from oracle import coupled, faces, fine, pipeline, rom, sfrac


def _single(m=3, k=4, model="random", ncell=(6, 5, 7), seed=3):
    p = inputs.small_problem(ncell=ncell, cuts=ncell, m=m, k=k, model=model, seed=seed,
                             src=[[21.0, 17.0, 33.0]], rec=[[30.0, 20.0, 40.0], [12.5, 31.0, 22.0]])
    topo = faces.Topology(p)
    return p, topo, pipeline.SubdomainROM(p, topo, 0, keep_basis=True)


@pytest.fixture(scope="module")
def sub():
    return _single()


def _fine_moment(sr, j):
    """F^T (L+sigma)^{-j} F from dense solves with K + sigma M (not the ROM's
    factorisation): (L+s)^{-1} = M^{1/2} (K+sM)^{-1} M^{1/2}."""
    K = sr.K.toarray()
    M = sr.mass
    A = K + sr.sigma * np.diag(M)
    if j == -1:
        return sr.B.T @ (A @ (sr.B / M[:, None]) / M[:, None])
    if j == 0:
        return sr.B.T @ (sr.B / M[:, None])
    X = np.linalg.solve(A, sr.B)
    for _ in range(j - 1):
        X = np.linalg.solve(A, M[:, None] * X)
    return sr.B.T @ X


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_basis_is_orthonormal(sub):
    p, topo, sr = sub
    V = sr.V
    assert np.abs(V.T @ V - np.eye(V.shape[1])).max() < 1e-12


def test_moment_matching(sub):
    """F~^T (L~+s)^{-j} F~ = F^T (L+s)^{-j} F for j = -1, 0, ..., 2k-2."""
    p, topo, sr = sub
    At = sr.Lt + sr.sigma * np.eye(sr.Lt.shape[0])
    for j in range(-1, 2 * sr.k - 1):
        if j == -1:
            rom_m = sr.Ft.T @ At @ sr.Ft
        else:
            rom_m = sr.Ft.T @ np.linalg.matrix_power(np.linalg.inv(At), j) @ sr.Ft
        assert _rel(rom_m, _fine_moment(sr, j)) < 1e-10, j


@pytest.mark.parametrize("lam_kind", ["s/10", "s", "10s", "lmax/10", "complex"])
def test_transfer_function_forms_agree(sub, lam_kind):
    p, topo, sr = sub
    s = sr.sigma
    lmax = np.linalg.eigvalsh(sr.Lt)[-1]
    lam = {"s/10": s / 10, "s": s, "10s": 10 * s, "lmax/10": lmax / 10,
           "complex": (2 * np.pi * 3.0 + 1j * 2 * np.pi * 40.0) ** 2}[lam_kind]
    a = sfrac.transfer_rom(sr.Lt, sr.Ft, lam)
    b = sfrac.transfer_tridiag(sr.alpha, sr.C, sr.R1, lam)
    c = sfrac.transfer_sfraction(sr.Gamma, sr.Gammahat, lam)
    assert _rel(b, a) < 1e-10 and _rel(c, a) < 1e-10


def test_rom_transfer_matches_fine_at_shift_and_nearby(sub):
    p, topo, sr = sub
    A = sr.K.toarray() + sr.sigma * np.diag(sr.mass)
    fine_s = sr.B.T @ np.linalg.solve(A, sr.B)
    assert _rel(sfrac.transfer_sfraction(sr.Gamma, sr.Gammahat, sr.sigma), fine_s) < 1e-10
    lam = 0.5 * sr.sigma
    fine_l = sr.B.T @ np.linalg.solve(sr.K.toarray() + lam * np.diag(sr.mass), sr.B)
    assert _rel(sfrac.transfer_sfraction(sr.Gamma, sr.Gammahat, lam), fine_l) < 1e-6


def test_similarity_to_the_u_form(sub):
    """``G T_L G^{-1} = blockdiag(Gammahat) D^T Gamma D`` (Eq. 12 from Eq. 10)."""
    p, topo, sr = sub
    k, b = sr.k, sr.Gamma[0].shape[0]
    T = sfrac.tridiag_matrix(sr.alpha, sr.C)
    Gb = np.zeros((k * b, k * b))
    Ghb = np.zeros_like(Gb)
    DGD = np.zeros_like(Gb)
    for j in range(k):
        sl = slice(j * b, (j + 1) * b)
        Gb[sl, sl] = sr.G[j]
        Ghb[sl, sl] = sr.Gammahat[j]
        DGD[sl, sl] += sr.Gamma[j]
        if j + 1 < k:
            sn = slice((j + 1) * b, (j + 2) * b)
            DGD[sn, sn] += sr.Gamma[j]
            DGD[sl, sn] -= sr.Gamma[j]
            DGD[sn, sl] -= sr.Gamma[j]
    lhs = Gb @ T @ np.linalg.inv(Gb)
    assert _rel(lhs, Ghb @ DGD) < 1e-10


def test_closed_forms_of_level_one(sub):
    """``Gammahat_1 = F^T F`` and ``Gamma_1 = Gh_1^{-1} F^T L F Gh_1^{-1}``."""
    p, topo, sr = sub
    FtF = sr.F.T @ sr.F
    assert _rel(sr.Gammahat[0], FtF) < 1e-12
    FLF = sr.F.T @ (sr.L @ sr.F)
    Gi = np.linalg.inv(FtF)
    assert _rel(sr.Gamma[0], Gi @ FLF @ Gi) < 1e-10


def test_gammas_are_invariant_under_block_rotations(sub):
    p, topo, sr = sub
    rng = np.random.default_rng(7)
    b = sr.R1.shape[0]
    Om = [np.linalg.qr(rng.standard_normal((b, b)))[0] for _ in range(sr.k)]
    alpha = [O.T @ a @ O for O, a in zip(Om, sr.alpha)]
    C = [Om[j + 1].T @ sr.C[j] @ Om[j] for j in range(sr.k - 1)]
    R1 = Om[0].T @ sr.R1
    Gam, Gh, _, _ = sfrac.gamma_transform(alpha, C, R1)
    for j in range(sr.k):
        assert _rel(Gam[j], sr.Gamma[j]) < 1e-10 and _rel(Gh[j], sr.Gammahat[j]) < 1e-10


def test_gammas_are_spd_below_the_last_level(sub):
    p, topo, sr = sub
    for j in range(sr.k):
        assert np.linalg.eigvalsh(sr.Gammahat[j]).min() > 0
        if j < sr.k - 1:
            assert np.linalg.eigvalsh(sr.Gamma[j]).min() > 0
    assert np.linalg.eigvalsh(sr.Gamma[-1]).min() >= 0


def _chain_L_F(Gh, Gam):
    """Symmetrised operator and input of a block chain with masses Gh_j^{-1},
    stiffness D^T Gamma D (last level grounded), input on level 1."""
    k, b = len(Gam), Gam[0].shape[0]
    MMinv_half = np.zeros((k * b, k * b))
    KK = np.zeros((k * b, k * b))
    for j in range(k):
        sl = slice(j * b, (j + 1) * b)
        w, U = np.linalg.eigh(Gh[j])
        MMinv_half[sl, sl] = (U * np.sqrt(w)) @ U.T
        KK[sl, sl] += Gam[j]
        if j + 1 < k:
            sn = slice((j + 1) * b, (j + 2) * b)
            KK[sn, sn] += Gam[j]
            KK[sl, sn] -= Gam[j]
            KK[sn, sl] -= Gam[j]
    L = MMinv_half @ KK @ MMinv_half
    F = MMinv_half[:, :b]
    return L, F


def _run_offline(L, F, k, sigma):
    solve = lambda X: np.linalg.solve(L + sigma * np.eye(L.shape[0]), X)
    V = rom.krylov_basis(solve, F, k)
    Lt, Ft = rom.galerkin(L, V, F)
    alpha, C, R1, _ = sfrac.block_lanczos(Lt, Ft, k)
    Gam, Gh, _, _ = sfrac.gamma_transform(alpha, C, R1)
    return Gam, Gh


def test_scalar_chain_gives_back_its_masses_and_conductances():
    """The 1D spring-mass chain (node k+1 grounded): the S-fraction of its
    input admittance returns ``Gammahat_j = 1/m_j``, ``Gamma_j = gamma_j``, the
    grid steps of the paper's remark after Eq. (15)."""
    rng = np.random.default_rng(11)
    k = 7
    m = rng.uniform(0.5, 2.0, k)
    g = rng.uniform(0.5, 2.0, k)
    Gam, Gh = _run_offline(*_chain_L_F([np.array([[1 / x]]) for x in m],
                                       [np.array([[x]]) for x in g]), k, 0.3)
    np.testing.assert_allclose([x[0, 0] for x in Gh], 1 / m, rtol=1e-12)
    np.testing.assert_allclose([x[0, 0] for x in Gam], g, rtol=1e-11)


def test_block_chain_gives_back_its_blocks():
    rng = np.random.default_rng(12)
    b, k = 3, 4

    def spd():
        X = rng.standard_normal((b, b))
        return X @ X.T + b * np.eye(b)
    Gh0 = [spd() for _ in range(k)]
    Gam0 = [spd() for _ in range(k)]
    Gam, Gh = _run_offline(*_chain_L_F(Gh0, Gam0), k, 0.7)
    for j in range(k):
        assert _rel(Gh[j], Gh0[j]) < 1e-11 and _rel(Gam[j], Gam0[j]) < 1e-10


def test_uniform_cube_level_one_closed_form():
    """Uniform c: ``[Gammahat_1]_f = 2 h c^2 n_s n_t diag(w_p w_q)``,
    w_0 = 1, w_{>0} = 1/2, identical on all six faces."""
    n, m = 6, 5
    p, topo, sr = _single(m=m, k=2, model="uniform", ncell=(n, n, n))
    c0, h = 2000.0, p.h
    nf = n - 1
    modes = faces.mode_list(nf, nf, m)
    w = lambda q: 1.0 if q == 0 else 0.5
    expect = np.diag([2 * h * c0 ** 2 * nf * nf * w(a) * w(b) for a, b in modes])
    for f in range(6):
        sl = slice(f * m, (f + 1) * m)
        np.testing.assert_allclose(sr.Gammahat[0][sl, sl], expect, rtol=1e-12,
                                   atol=1e-12 * expect.max())
        for g in range(6):
            if g != f:
                assert np.abs(sr.Gammahat[0][sl, g * m:(g + 1) * m]).max() < 1e-12 * expect.max()


def test_breakdown_is_raised_for_a_rank_deficient_face_basis():
    p, topo, sr = _single()
    F = np.hstack([sr.F, sr.F[:, :1]])
    solve = rom.shifted_solver(sr.K, sr.mass, sr.sigma)
    with pytest.raises(rom.Breakdown):
        rom.krylov_basis(solve, F, 3)


# ----------------------------------------------------------------------------
# Algorithm 1 step 1.4: source and receiver rows
# ----------------------------------------------------------------------------

def _u_form_solve(sr, lam, rhs):
    """Solve ``(lam blockdiag(Gh^{-1}) + D^T Gamma D) U = rhs`` (the Laplace
    transform of the level equations with U_{k+1} = 0)."""
    k, b = sr.k, sr.Gamma[0].shape[0]
    S = np.zeros((k * b, k * b), dtype=complex)
    for j in range(k):
        sl = slice(j * b, (j + 1) * b)
        S[sl, sl] += lam * np.linalg.inv(sr.Gammahat[j]) + sr.Gamma[j]
        if j + 1 < k:
            sn = slice((j + 1) * b, (j + 2) * b)
            S[sn, sn] += sr.Gamma[j]
            S[sl, sn] -= sr.Gamma[j]
            S[sn, sl] -= sr.Gamma[j]
    return np.linalg.solve(S, rhs).reshape(k, b)


def _node_vector(p, sr, nodes, w):
    from oracle import project
    return project.local_share(sr.box, fine.global_mass_ijk(p), sr.mass, nodes, w)


@pytest.mark.parametrize("lam", [30.0, 300.0, (12.0 + 150j) ** 2])
def test_source_rows_reproduce_the_galerkin_source_response(sub, lam):
    """Face response U_1 to the projected force equals
    ``F~^T (L~+lam)^{-1} V^T M^{-1/2} s`` for every lam (Eq. 16)."""
    p, topo, sr = sub
    nodes, w = inputs.gaussian_node_weights(p.src_xyz[0], p.h, p.h, p.nx, p.ny, p.nz)
    s = _node_vector(p, sr, nodes, w)
    P = sr.rows(s)
    U = _u_form_solve(sr, lam, P.ravel().astype(complex))
    n = sr.Lt.shape[0]
    ref = sr.Ft.T @ np.linalg.solve(sr.Lt + lam * np.eye(n), sr.V.T @ (s / np.sqrt(sr.mass)))
    assert _rel(U[0], ref) < 1e-10


def test_source_moments_match_the_fine_grid(sub):
    """``F^T (L+s)^{-j} M^{-1/2} s = F~^T (L~+s)^{-j} V^T M^{-1/2} s``, j < k."""
    p, topo, sr = sub
    nodes, w = inputs.gaussian_node_weights(p.src_xyz[0], p.h, p.h, p.nx, p.ny, p.nz)
    s = _node_vector(p, sr, nodes, w)
    M = sr.mass
    A = sr.K.toarray() + sr.sigma * np.diag(M)
    At = sr.Lt + sr.sigma * np.eye(sr.Lt.shape[0])
    x = s.copy()                               # (L+s)^{-j} M^{-1/2} s = M^{1/2} y_j
    y_rom = sr.V.T @ (s / np.sqrt(M))
    for j in range(sr.k):
        fine_m = sr.B.T @ (x / M)                # F^T M^{-1/2} ... = B^T M^{-1} x
        rom_m = sr.Ft.T @ y_rom
        assert _rel(rom_m, fine_m) < 1e-10, j
        x = M * np.linalg.solve(A, x)
        y_rom = np.linalg.solve(At, y_rom)


def test_receiver_rows_reproduce_the_galerkin_field(sub):
    """``sum_j rho_j^T U_j(lam) = e^T M^{-1/2} V (L~+lam)^{-1} F~`` for a face
    input, and its moments match the fine grid exactly for j < k."""
    p, topo, sr = sub
    nodes, w = inputs.trilinear_node_weights(p.rec_xyz[1], p.h, p.nx, p.ny, p.nz)
    e = _node_vector(p, sr, nodes, w)
    rho = sr.rows(e)
    k, b = sr.k, sr.Gamma[0].shape[0]
    n = sr.Lt.shape[0]
    for lam in (sr.sigma, 5e3, (20.0 + 300j) ** 2):
        got = np.zeros(b, dtype=complex)
        for i in range(b):
            rhs = np.zeros(k * b, dtype=complex)
            rhs[i] = 1.0
            U = _u_form_solve(sr, lam, rhs)
            got[i] = np.sum(rho * U)
        ref = (e / np.sqrt(sr.mass)) @ sr.V @ np.linalg.solve(sr.Lt + lam * np.eye(n), sr.Ft)
        assert _rel(got, ref) < 1e-10
    # moments: e^T M^{-1/2} (L+s)^{-j} F, j < k, are reproduced by the ROM
    M = sr.mass
    A = sr.K.toarray() + sr.sigma * np.diag(M)
    At = sr.Lt + sr.sigma * np.eye(n)
    X = sr.B.copy()                         # M^{1/2} (L+s)^{-j} F  (j=0: B)
    Y = sr.Ft.copy()
    for j in range(k):
        fine_m = e @ (X / M[:, None])
        rom_m = (e / np.sqrt(M)) @ sr.V @ Y
        scale = np.linalg.norm(e / np.sqrt(M)) * np.linalg.norm(Y, 2)   # |V| = 1
        assert np.linalg.norm(rom_m - fine_m) < 1e-10 * scale, j
        X = M[:, None] * np.linalg.solve(A, X)
        Y = np.linalg.solve(At, Y)


def test_usable_depth_keeps_well_conditioned_fractions_whole():
    p = inputs.small_problem(ncell=(8, 8, 8), cuts=([0, 8], [0, 8], [0, 8]), m=2, k=4)
    rs = pipeline.build(p)
    assert sfrac.usable_depth(rs.Gamma[0], rs.Gammahat[0]) == 4
    rs2 = pipeline.build(p, depth_tau=1e-13)
    assert rs2.k[0] == 4


@pytest.mark.slow
def test_usable_depth_cuts_a_fraction_past_fp64_range():
    """A 16^3-cell subdomain with m = 8 and k = 24 at sigma = (2 pi 8 f)^2:
    its deep Gammahat blocks are indefinite at rounding level and the
    fraction's lambda_max exceeds the Galerkin ROM's; cut at its usable
    depth every block is positive definite and lambda_max is the Galerkin
    ROM's again (to 1e-3)."""
    n = 16
    p = inputs.small_problem(ncell=(n, n, n), cuts=([0, n], [0, n], [0, n]), m=8, k=24,
                             model="two_layer", f_peak=20.0, sigma=inputs.default_sigma(20.0, 8))
    full = pipeline.build(p, keep=True)
    lam_rom = np.linalg.eigvalsh(full.subroms[0].Lt).max()
    assert coupled.lambda_max(full) > 2.0 * lam_rom
    cut = pipeline.build(p, depth_tau=1e-13)
    kk = cut.k[0]
    assert 1 <= kk < 24
    for G in list(cut.Gammahat[0]) + list(cut.Gamma[0][:-1]):
        ev = np.linalg.eigvalsh(G)
        assert ev.min() > 0
    assert abs(coupled.lambda_max(cut) / lam_rom - 1.0) < 1e-3
