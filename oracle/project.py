"""Algorithm 1 step (1.4): sources and receivers in the S-fraction coordinates.

The change of variables is Eq. (16), ``U_j = G_j [Qh^T V^T w]_j`` with
``w = M^{1/2} u`` the symmetrised fine field.  Its consequences used here:

* a nodal force ``s f(t)`` (``M u'' = -K u + s f``) enters the symmetrised
  equation as ``M^{-1/2} s f``; Galerkin projection and the Lanczos/G change
  of variables turn it into ``Gammahat_j p_j f(t)`` on level j with
  ``p_j = G_j^{-T} Qh_j^T V^T M^{-1/2} s``;
* the field at a node is ``u = M^{-1/2} V Qh z`` with ``z_j = G_j^{-1} U_j``,
  so a receiver that reads ``e^T u`` reads ``sum_j rho_j^T U_j`` with
  ``rho_j = G_j^{-T} Qh_j^T V^T M^{-1/2} e``.

Initial conditions (Algorithm 1 step 1.4 as the paper states it): a nodal
field u (a displacement, or a velocity for the time derivative) maps to
``U_j = G_j [Qh^T V^T M^{1/2} u]_j`` (``project_state``).  On the level-1
face blocks this is ``B^T u`` (the first Krylov block is F and
``G_1 = R_1^T``), so the two sides of a shared face agree.

Readings where the paper is silent (its experiment uses an initial pulse,
Algorithm 1 step 1.4; the workloads here use a point force):

* the source is a FORCE with a normalised Gaussian spatial density (width h,
  cut at 3 widths, weights summing to one);
* a node shared by several subdomains gives each copy the share
  ``M^a_node / M_node`` of its force, so every copy accelerates alike;
* a receiver reads the trilinear interpolation of nodal u, where the value
  at a shared node is the mass-weighted average ``sum_a (M^a/M) u^a`` over its
  copies.
"""
from __future__ import annotations

import numpy as np

from .fine import node_index


def local_share(box, global_mass, sub_mass, nodes, weights):
    """Vector over the box's nodes holding ``weight * M^a/M`` for each of the
    given global nodes that lie in the box (zero elsewhere)."""
    x0, x1, y0, y1, z0, z1 = box
    out = np.zeros(sub_mass.shape[0])
    i, j, k = nodes[:, 0], nodes[:, 1], nodes[:, 2]
    inside = (i >= x0) & (i <= x1) & (j >= y0) & (j <= y1) & (k >= z0) & (k <= z1)
    if not inside.any():
        return None
    loc = node_index(box, i[inside], j[inside], k[inside])
    gm = global_mass[i[inside], j[inside], k[inside]]
    np.add.at(out, loc, weights[inside] * sub_mass[loc] / gm)
    return out


def project(V, Qh, G, sub_mass, vec):
    """``p_j = G_j^{-T} Qh_j^T V^T M^{-1/2} vec`` for j = 1..k; returns (k, b).
    ``vec`` may also be a matrix of column vectors (N, n): returns (n, k, b)."""
    one = vec.ndim == 1
    X = vec[:, None] if one else vec
    Y = Qh.T @ (V.T @ (X / np.sqrt(sub_mass)[:, None]))
    b = G[0].shape[0]
    k = len(G)
    out = np.stack([np.linalg.solve(G[j].T, Y[j * b:(j + 1) * b]) for j in range(k)])  # (k,b,n)
    out = np.moveaxis(out, 2, 0)
    return out[0] if one else out


def project_state(V, Qh, G, sub_mass, u):
    """Eq. (16) applied to a nodal field: ``U_j = G_j [Qh^T V^T M^{1/2} u]_j``
    for j = 1..k; returns (k, b).  ``u`` may be a matrix of columns (N, n):
    returns (n, k, b)."""
    one = u.ndim == 1
    X = u[:, None] if one else u
    Y = Qh.T @ (V.T @ (X * np.sqrt(sub_mass)[:, None]))
    b = G[0].shape[0]
    out = np.stack([G[j] @ Y[j * b:(j + 1) * b] for j in range(len(G))])    # (k, b, n)
    out = np.moveaxis(out, 2, 0)
    return out[0] if one else out

