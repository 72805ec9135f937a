"""Largest eigenvalue of a symmetric operator by the Lanczos iteration with
full reorthogonalisation (used for leapfrog stability limits).

Plain NumPy: the Krylov basis is kept as the rows of one array, every new
vector is orthogonalised twice against all previous ones, and the largest
Ritz value of the tridiagonal matrix is tracked until it settles."""
from __future__ import annotations

import numpy as np


def lanczos_max(matvec, n, tol=1e-11, max_iter=400, seed=0):
    rng = np.random.default_rng(seed)
    m = min(max_iter, n)
    Q = np.empty((m, n))
    q = rng.standard_normal(n)
    Q[0] = q / np.linalg.norm(q)
    alpha, beta = [], []
    prev = None
    for j in range(m):
        w = matvec(Q[j])
        alpha.append(float(np.dot(Q[j], w)))
        for _ in range(2):
            w = w - Q[:j + 1].T @ (Q[:j + 1] @ w)
        T = np.diag(alpha) + np.diag(beta, 1) + np.diag(beta, -1)
        lam = float(np.linalg.eigvalsh(T)[-1])
        if prev is not None and abs(lam - prev) <= tol * abs(lam):
            return lam
        prev = lam
        bnorm = float(np.linalg.norm(w))
        if bnorm <= 1e-14 * max(abs(lam), 1e-300) or j == m - 1:
            return lam
        beta.append(bnorm)
        Q[j + 1] = w / bnorm
    return prev
