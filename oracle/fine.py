"""Fine-grid operator of Eq. (1) and the reference fine-grid FDTD.

Reading of the paper (it leaves the fine operator generic, Eq. 1):
vertex-centred finite volumes with per-cell assembly for the constant-density
acoustic equation ``u_tt = c^2 Laplacian(u)`` (the experiment's Eq. 20).  Each
cell of side h and velocity c adds

* conductance ``h/4`` to each of its 12 edges (stiffness K), and
* lumped mass ``h^3 / (8 c^2)`` to each of its 8 corner nodes (mass M).

A subdomain's ``K^a, M^a`` are the sums over its own cells, so the global
matrices are exactly the sums over subdomains, and the outer boundary of any
box is natural (homogeneous Neumann).  With these, ``M u'' = -K u`` is the
semi-discrete wave equation, i.e. ``A = -M^{-1}K`` in Eq. (1); the symmetrised
form used by the ROM is ``L = M^{-1/2} K M^{-1/2}`` (so ``L = -A`` up to the
similarity by ``M^{1/2}``).  Node numbering inside a box is lexicographic with
x fastest.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .eig import lanczos_max


def box_shape(box):
    x0, x1, y0, y1, z0, z1 = box
    return (x1 - x0 + 1, y1 - y0 + 1, z1 - z0 + 1)


def node_index(box, i, j, k):
    """Local index of global node(s) (i, j, k) inside ``box``."""
    x0, _, y0, _, z0, _ = box
    nxl, nyl, _ = box_shape(box)
    return (np.asarray(i) - x0) + nxl * ((np.asarray(j) - y0) + nyl * (np.asarray(k) - z0))


def node_coords(box):
    """Global (i, j, k) of every local node of ``box`` (x fastest)."""
    x0, x1, y0, y1, z0, z1 = box
    k, j, i = np.meshgrid(np.arange(z0, z1 + 1), np.arange(y0, y1 + 1),
                          np.arange(x0, x1 + 1), indexing="ij")
    return i.ravel(), j.ravel(), k.ravel()


def assemble(c, h, box, mass_only=False):
    """Per-cell assembly of ``(K, Mdiag)`` over the cells inside ``box``.

    ``c`` is the global cell velocity array ``[nz, ny, nx]``; ``box`` a node
    box ``(x0, x1, y0, y1, z0, z1)``.  Returns a CSR stiffness and the lumped
    mass diagonal over the box's nodes."""
    x0, x1, y0, y1, z0, z1 = box
    nxl, nyl, nzl = box_shape(box)
    n = nxl * nyl * nzl
    ck, cj, ci = np.meshgrid(np.arange(z0, z1), np.arange(y0, y1), np.arange(x0, x1),
                             indexing="ij")
    ci, cj, ck = ci.ravel(), cj.ravel(), ck.ravel()
    cv = c[ck, cj, ci]
    # corner nodes of every cell
    corner = {}
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                corner[(dx, dy, dz)] = node_index(box, ci + dx, cj + dy, ck + dz)
    mass = np.zeros(n)
    for idx in corner.values():
        np.add.at(mass, idx, h ** 3 / (8.0 * cv * cv))
    if mass_only:
        return mass
    rows, cols, vals = [], [], []
    g = np.full(ci.shape, h / 4.0)
    # the 12 edges: 4 along each axis
    for (a, b) in [((0, y, z), (1, y, z)) for y in (0, 1) for z in (0, 1)] + \
                  [((x, 0, z), (x, 1, z)) for x in (0, 1) for z in (0, 1)] + \
                  [((x, y, 0), (x, y, 1)) for x in (0, 1) for y in (0, 1)]:
        p, q = corner[a], corner[b]
        rows += [p, q, p, q]
        cols += [p, q, q, p]
        vals += [g, g, -g, -g]
    K = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n)).tocsr()
    K.sum_duplicates()
    return K, mass


def lumped_mass(c, h, box):
    """Lumped mass diagonal of ``box`` (the M part of :func:`assemble`)."""
    return assemble(c, h, box, mass_only=True)


def global_mass_ijk(problem):
    """Global lumped mass as an array indexed ``[i, j, k]`` (x, y, z)."""
    m = lumped_mass(problem.c, problem.h, global_box(problem))
    return m.reshape(problem.nz + 1, problem.ny + 1, problem.nx + 1).transpose(2, 1, 0)


def global_box(problem):
    return (0, problem.nx, 0, problem.ny, 0, problem.nz)


def assemble_global(problem):
    return assemble(problem.c, problem.h, global_box(problem))


def symmetrised(K, mass):
    """``L = M^{-1/2} K M^{-1/2}`` (the SPD form of ``-A`` in Eq. 1)."""
    s = 1.0 / np.sqrt(mass)
    return sp.diags(s) @ K @ sp.diags(s)


def lambda_max(K, mass):
    """Largest eigenvalue of ``M^{-1} K``."""
    L = symmetrised(K, mass)
    if L.shape[0] <= 400:
        return float(np.linalg.eigvalsh(L.toarray())[-1])
    return lanczos_max(lambda v: L @ v, L.shape[0])


def cfl_dt(K, mass):
    """Leapfrog stability limit ``2 / sqrt(lambda_max(M^{-1}K))``."""
    return 2.0 / np.sqrt(lambda_max(K, mass))


def leapfrog(K, mass, dt, nsteps, force, wavelet, rec_rows, u0=None, v0=None):
    """Fine-grid explicit leapfrog
    ``M (u^{n+1} - 2u^n + u^{n-1}) = dt^2 (-K u^n + force * f(t_n))`` from rest,
    in increment form ``v^{n+1} = v^n + dt^2 M^{-1}(...)``, ``u^{n+1} = u^n + v^{n+1}``.

    ``force``: [N] nodal force density; ``wavelet``: samples f(t_n), n < nsteps;
    ``rec_rows``: sparse [nrec, N].  Returns traces ``[nrec, nsteps+1]`` at
    ``t_n = n dt``.

    ``u0``, ``v0``: optional initial displacement and velocity [N]; the start
    is the second-order Taylor step of the ROM stepping,
    ``v^0 = dt v0 - dt^2/2 M^{-1}(-K u0)``, so that
    ``u^1 = u0 + dt v0 + dt^2/2 M^{-1}(-K u0) + dt^2 M^{-1} force f(t_0)``."""
    n = K.shape[0]
    minv = 1.0 / mass
    u = np.zeros(n) if u0 is None else np.array(u0, dtype=np.float64)
    v = np.zeros(n)
    if u0 is not None:
        v -= 0.5 * dt * dt * minv * (-(K @ u))
    if v0 is not None:
        v += dt * np.asarray(v0, dtype=np.float64)
    out = np.zeros((rec_rows.shape[0], nsteps + 1))
    for it in range(nsteps):
        out[:, it] = rec_rows @ u
        v += dt * dt * minv * (-(K @ u) + force * wavelet[it])
        u += v
    out[:, nsteps] = rec_rows @ u
    return out


def energy(K, mass, u_new, u_old, dt):
    """Conserved leapfrog energy ``1/2 |v|_M^2 / dt^2 + 1/2 u_new^T K u_old``."""
    v = u_new - u_old
    return 0.5 * np.dot(v, mass * v) / dt ** 2 + 0.5 * np.dot(u_new, K @ u_old)
