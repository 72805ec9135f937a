"""Algorithm 1 step (1.1): projection subspace and Galerkin ROM (Eqs. 5-7).

Reading of the paper: with Neumann faces the subdomain operator is singular
(constants are in its null space), so the paper's ``K_n(0)`` of Eq. (7),
built from ``A^{-1}``, does not exist.  We take the paper's own rational
Krylov family (Eq. 6) with ONE repeated finite shift ``sigma > 0`` and, as the
discussion before Eq. (18) requires, F itself as the first block:

    V = orth[ F, (L+sigma)^{-1} F, ..., (L+sigma)^{-(k-1)} F ]   (dim b*k)

which is what block Lanczos on ``((L+sigma)^{-1}, F)`` started from F spans.
The shifted matrix is factored once per subdomain and the factor reused for
every block solve, as the paper recommends.  The factorisation is SuperLU with
a symmetric fill-reducing ordering and no pivoting, i.e. the LDL^T form of the
Cholesky factor of the SPD matrix ``K + sigma M``.

Block Gram-Schmidt against all previous blocks is done twice (full
reorthogonalisation); a numerically rank-deficient new block raises
``Breakdown`` (deflation would make the Lanczos blocks rectangular).

Eq. 6 also allows distinct finite shifts sigma_1..sigma_{k-1}: block j+1 is
then ``(L + sigma_j)^{-1}`` applied to block j, which for distinct shifts
spans ``F, (L+sigma_1)^{-1}F, ..., (L+sigma_{k-1})^{-1}F`` (partial
fractions) and for repeated ones the powers above.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


class Breakdown(RuntimeError):
    pass


def shifted_solver(K, mass, sigma):
    """Returns ``x -> (L + sigma I)^{-1} x`` with ``L = M^{-1/2} K M^{-1/2}``,
    using ``(L+sigma)^{-1} = M^{1/2} (K + sigma M)^{-1} M^{1/2}``."""
    A = (K + sigma * sp.diags(mass)).tocsc()
    lu = spla.splu(A, permc_spec="MMD_AT_PLUS_A", diag_pivot_thresh=0.0,
                   options=dict(SymmetricMode=True))
    ms = np.sqrt(mass)

    def solve(X):
        X = np.asarray(X)
        sh = ms[:, None] if X.ndim == 2 else ms
        return sh * lu.solve(sh * X)
    return solve


def _qr(W, tol, what):
    Q, R = np.linalg.qr(W)
    d = np.abs(np.diag(R))
    if d.min() < tol * max(np.linalg.norm(W), 1e-300):
        raise Breakdown(f"rank-deficient block in {what}: min|diag R| = {d.min():.3e}")
    return Q, R


def krylov_basis(solve, F, k, tol=1e-12):
    """Orthonormal ``V = [Q_1 .. Q_k]`` of the shifted block Krylov space.
    ``solve``: one resolvent ``x -> (L + sigma)^{-1} x`` for every block, or
    a list of k-1 of them, the j-th making block j+1."""
    solves = list(solve) if isinstance(solve, (list, tuple)) else [solve] * (k - 1)
    if len(solves) != k - 1:
        raise ValueError("one resolvent per block after the first")
    Q, _ = _qr(F, tol, "F")
    blocks = [Q]
    for j in range(1, k):
        W = solves[j - 1](blocks[-1])
        for _ in range(2):
            for Qi in blocks:
                W = W - Qi @ (Qi.T @ W)
        Q, _ = _qr(W, tol, "Krylov block")
        blocks.append(Q)
    return np.hstack(blocks)


def galerkin(L, V, F):
    """Eq. (5) in symmetrised form: ``L~ = V^T L V`` (symmetrised), ``F~ = V^T F``."""
    Lt = V.T @ (L @ V)
    Lt = 0.5 * (Lt + Lt.T)
    return Lt, V.T @ F
