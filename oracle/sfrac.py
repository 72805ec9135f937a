"""Algorithm 1 steps (1.2)-(1.3): block Lanczos to block-tridiagonal form
(Eq. 8) and the S-fraction transform (Eq. 13); transfer functions of Eqs.
(4), (9) and (15).

Sign convention.  The paper writes ``u_tt = A u`` (Eq. 1) with ``A <= 0`` and
transfer functions in ``omega^2``.  Here ``L = -A >= 0`` and ``lambda`` takes
the place of ``omega^2``: ``S(lambda) = F^T (L + lambda)^{-1} F``.

Block Lanczos on ``(L~, F~)`` gives ``F~ = Qh_1 R_1`` and a block tridiagonal
``T_L = Qh^T L~ Qh`` with diagonal blocks ``alpha_j`` and sub-diagonal blocks
``C_{j+1}`` (block (j+1, j)); the super-diagonal block (j, j+1) is
``C_{j+1}^T``.  In the paper's notation ``A_j = -alpha_j``, ``B_1 = R_1^T`` and
the off-diagonal ``B_{j+1} = -C_{j+1}^T``.  (The paper writes B_j on both
sides of the diagonal, which is Hermitian only if B_j is symmetric; taking
the transpose below the diagonal is the reading under which the recursion of
Eq. (13) follows from Eq. (10).)

S-fraction transform (Eq. 13 in L convention).  With ``U_j = G_j z_j`` where
``z`` are the Lanczos coordinates, the Lanczos equations become Eq. (12) if

    G_1 = R_1^T,  Gamma_0 = 0,  Gammahat_j = G_j G_j^T,
    Gamma_j   = G_j^{-T} alpha_j G_j^{-1} - Gamma_{j-1},
    G_{j+1}   = -(G_j^T Gamma_j)^{-1} C_{j+1}^T.

Derivation: multiplying the j-th Lanczos row
``z_j'' = -(C_j z_{j-1} + alpha_j z_j + C_{j+1}^T z_{j+1})`` by G_j and
asking for ``Gammahat_j (Gamma_j (U_{j+1}-U_j) - Gamma_{j-1}(U_j-U_{j-1}))``
gives, coefficient by coefficient, ``G_j^T Gamma_j G_{j+1} = -C_{j+1}^T`` and
``Gamma_j + Gamma_{j-1} = G_j^{-T} alpha_j G_j^{-1}``; the third coefficient
``G_j^T Gamma_{j-1} G_{j-1} = -C_j`` is the transpose of the first at j-1,
so the system is consistent exactly when every Gamma_j is symmetric.

Reading where the paper is silent: the last ``Gamma_k`` can be numerically
semidefinite (the constant mode is a near-pole at lambda = 0 for Neumann
faces); after symmetrising, eigenvalues of Gamma_k below zero are clipped to
zero.  An eigenvalue below ``-1e-12 |Gamma_j|`` for j < k raises ``NotSPD``.
"""
from __future__ import annotations

import numpy as np


class NotSPD(RuntimeError):
    pass


def sym(X):
    return 0.5 * (X + X.T)


def block_lanczos(Lt, Ft, k):
    """Block Lanczos with full reorthogonalisation.  Returns
    ``(alpha[k], C[k-1], R1, Qh)`` with ``Qh`` the (n x b*k) Lanczos basis and
    ``C[j]`` the block (j+2, j+1) of T_L (1-based)."""
    Q, R1 = np.linalg.qr(Ft)
    Qs = [Q]
    alpha, C = [], []
    for j in range(k):
        Qj = Qs[-1]
        W = Lt @ Qj
        a = sym(Qj.T @ W)
        alpha.append(a)
        if j == k - 1:
            break
        W = W - Qj @ a
        if j > 0:
            W = W - Qs[-2] @ C[-1].T
        for _ in range(2):
            for Qi in Qs:
                W = W - Qi @ (Qi.T @ W)
        Qn, Cn = np.linalg.qr(W)
        C.append(Cn)
        Qs.append(Qn)
    return alpha, C, R1, np.hstack(Qs)


def tridiag_matrix(alpha, C):
    """Assemble T_L (b*k x b*k) from its blocks."""
    b = alpha[0].shape[0]
    k = len(alpha)
    T = np.zeros((b * k, b * k))
    for j in range(k):
        T[j * b:(j + 1) * b, j * b:(j + 1) * b] = alpha[j]
    for j in range(k - 1):
        T[(j + 1) * b:(j + 2) * b, j * b:(j + 1) * b] = C[j]
        T[j * b:(j + 1) * b, (j + 1) * b:(j + 2) * b] = C[j].T
    return T


def gamma_transform(alpha, C, R1, spd_tol=1e-12):
    """Eq. (13).  Returns ``(Gamma[k], Gammahat[k], G[k], min_eigs)``."""
    k = len(alpha)
    G = R1.T.copy()
    Gam, Gh, Gs = [], [], []
    prev = np.zeros_like(alpha[0])
    mins = []
    for j in range(k):
        Gs.append(G)
        Gh.append(sym(G @ G.T))
        Gi = np.linalg.inv(G)
        Gj = sym(Gi.T @ alpha[j] @ Gi - prev)
        w, U = np.linalg.eigh(Gj)
        mins.append((float(w.min()), float(np.linalg.eigvalsh(Gh[-1]).min())))
        scale = max(np.abs(w).max(), 1e-300)
        if j < k - 1:
            if w.min() < -spd_tol * scale:
                raise NotSPD(f"Gamma_{j + 1} has eigenvalue {w.min():.3e}")
        elif w.min() < 0:
            Gj = sym((U * np.maximum(w, 0.0)) @ U.T)
        Gam.append(Gj)
        prev = Gj
        if j < k - 1:
            G = -np.linalg.solve(G.T @ Gj, C[j].T)
    return Gam, Gh, Gs, mins


def usable_depth(Gam, Gh, tau=1e-13):
    """Number of leading levels whose blocks are positive definite beyond the
    rounding level: the first level j with ``lambda_min < tau * lambda_max``
    in Gammahat_j, or in Gamma_j below the last level, ends the usable
    fraction (at least one level is kept).  Deep levels of an accurate ROM
    at a small shift run past FP64's dynamic range (their smallest
    eigenvalues sit at rounding level, some rounded below zero, and the
    coupled lambda_max of the fraction exceeds the Galerkin ROM's); the
    fraction truncated there, terminated with U_{j+1} = 0 like the full one,
    stays a positive definite S-fraction."""
    k = len(Gam)
    for j in range(k):
        eh = np.linalg.eigvalsh(sym(Gh[j]))
        ok = eh.min() > tau * eh.max()
        if j < k - 1:
            eg = np.linalg.eigvalsh(sym(Gam[j]))
            ok = ok and eg.min() > tau * eg.max()
        if not ok:
            return max(j, 1)
    return k


# ----------------------------------------------------------------------------
# transfer functions S(lambda) = F^T (L + lambda)^{-1} F in its four forms
# ----------------------------------------------------------------------------

def transfer_rom(Lt, Ft, lam):
    """Eq. (4): ``F~^T (L~ + lambda)^{-1} F~``."""
    n = Lt.shape[0]
    return Ft.T @ np.linalg.solve(Lt + lam * np.eye(n), Ft)


def transfer_tridiag(alpha, C, R1, lam):
    """Eq. (9): ``R^T (T + lambda)^{-1} R`` with ``R = [R_1; 0; ...]``."""
    T = tridiag_matrix(alpha, C)
    b = R1.shape[0]
    E = np.zeros((T.shape[0], b))
    E[:b] = R1
    return E.T @ np.linalg.solve(T + lam * np.eye(T.shape[0]), E)


def transfer_sfraction(Gam, Gh, lam):
    """Eq. (15), the matrix S-fraction, evaluated from the bottom level up:
    ``Y_k = lambda Gh_k^{-1} + Gamma_k``,
    ``Y_j = lambda Gh_j^{-1} + (Gamma_j^{-1} + Y_{j+1}^{-1})^{-1}``, and
    ``S = Y_1^{-1}``.  (The printed 1D formula is garbled; this is its matrix
    form, read off Eq. (12) with U_{k+1} = 0.)"""
    k = len(Gam)
    Y = lam * np.linalg.inv(Gh[k - 1]) + Gam[k - 1]
    for j in range(k - 2, -1, -1):
        Y = lam * np.linalg.inv(Gh[j]) + np.linalg.inv(np.linalg.inv(Gam[j]) + np.linalg.inv(Y))
    return np.linalg.inv(Y)
