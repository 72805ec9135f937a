"""Face basis F^alpha (section "Stage 1: reduced order models") and the
subdomain topology (faces shared by two subdomains, outer faces).

Readings of the paper:

* Non-overlap.  The paper asks that basis functions of different faces do not
  overlap (discussion before Eq. 18), which closed faces of a box cannot
  satisfy: edges and corners touch two or three faces.  Each face's functions
  are therefore supported on its OPEN face: the nodes of the face that lie on
  no edge of the subdomain box.  Subdomain edges and corners are then not part
  of any exchange.
* Functions.  ``m`` cosine modes per face,
  ``phi_pq(s, t) = cos(pi p (s - 1/2)/n_s) cos(pi q (t - 1/2)/n_t)`` for the
  open-face node numbers ``s = 1..n_s``, ``t = 1..n_t`` counted along the two
  in-plane axes in increasing global coordinate (x-face: (y, z); y-face:
  (x, z); z-face: (x, y)), so both sides of a shared face use the same
  functions in the same order.  Modes are taken by ascending ``p^2 + q^2``,
  ties by ascending q, then p.
* Scaling.  ``B[node, (f, pq)] = h^2 phi_pq(node)`` (a flux times a face
  area), and ``F = M^{-1/2} B`` in the symmetrised variables.
* Face count per face: a shared face carries ``min(m_a, m_b)`` modes, an outer
  face the subdomain's own m.  Outer faces are homogeneous Neumann.

Faces of a subdomain are numbered ``0..5 = -x, +x, -y, +y, -z, +z``.
"""
from __future__ import annotations

import numpy as np

from .fine import box_shape, node_index


def mode_list(ns, nt, m):
    """The first ``m`` modes (p, q), 0 <= p < ns, 0 <= q < nt."""
    modes = [(p, q) for p in range(ns) for q in range(nt)]
    modes.sort(key=lambda pq: (pq[0] ** 2 + pq[1] ** 2, pq[1], pq[0]))
    if m > len(modes):
        raise ValueError(f"face has only {len(modes)} open-face modes, asked for {m}")
    return modes[:m]


def face_axes(f):
    """Normal axis and the two in-plane axes (in order s, t) of face ``f``."""
    a = f // 2
    inplane = [x for x in range(3) if x != a]
    return a, inplane[0], inplane[1]


def open_face_nodes(box, f):
    """Local indices of the open-face nodes of face ``f`` of ``box`` and their
    1-based in-plane numbers ``(s, t)``; also returns ``(n_s, n_t)``."""
    lo = np.array(box[0::2])
    hi = np.array(box[1::2])
    a, u, v = face_axes(f)
    ns = hi[u] - lo[u] - 1
    nt = hi[v] - lo[v] - 1
    s, t = np.meshgrid(np.arange(1, ns + 1), np.arange(1, nt + 1), indexing="ij")
    s, t = s.ravel(), t.ravel()
    g = [None, None, None]
    g[a] = np.full(s.shape, hi[a] if f % 2 else lo[a])
    g[u] = lo[u] + s
    g[v] = lo[v] + t
    return node_index(box, g[0], g[1], g[2]), s, t, (ns, nt)


def face_B(box, f, m, h):
    """Columns of B for face ``f``: returns ``(local_nodes, values[nodes, m])``."""
    idx, s, t, (ns, nt) = open_face_nodes(box, f)
    vals = np.empty((idx.size, m))
    for c, (p, q) in enumerate(mode_list(ns, nt, m)):
        vals[:, c] = h * h * np.cos(np.pi * p * (s - 0.5) / ns) * np.cos(np.pi * q * (t - 0.5) / nt)
    return idx, vals


def B_matrix(box, mf, h):
    """Dense ``B`` (N x b) of a subdomain with per-face mode counts ``mf[6]``."""
    n = int(np.prod(box_shape(box)))
    b = int(sum(mf))
    B = np.zeros((n, b))
    col = 0
    for f in range(6):
        if mf[f] == 0:
            continue
        idx, vals = face_B(box, f, int(mf[f]), h)
        B[idx, col:col + mf[f]] = vals
        col += mf[f]
    return B


class Topology:
    """Subdomain adjacency and global face numbering.

    ``nbr[s, f]``: neighbour across face f (or -1 for an outer face);
    ``face_id[s, f]``: global face index; ``mf[s, f]``: modes on that face;
    ``face_sides[g]``: list of (s, f) sharing global face g; ``face_m[g]``.
    """

    def __init__(self, problem):
        ncx, ncy, ncz = problem.ncuts
        nsub = problem.nsub
        self.nsub = nsub
        self.nbr = -np.ones((nsub, 6), dtype=int)
        for s in range(nsub):
            ix, iy, iz = s % ncx, (s // ncx) % ncy, s // (ncx * ncy)
            pos = [ix, iy, iz]
            lim = [ncx, ncy, ncz]
            for f in range(6):
                a = f // 2
                q = list(pos)
                q[a] += 1 if f % 2 else -1
                if 0 <= q[a] < lim[a]:
                    self.nbr[s, f] = problem.sub_index(*q)
        msub = np.asarray(problem.m_sub)
        self.mf = np.zeros((nsub, 6), dtype=int)
        self.face_id = -np.ones((nsub, 6), dtype=int)
        self.face_sides = []
        self.face_m = []
        for s in range(nsub):
            for f in range(6):
                t = self.nbr[s, f]
                self.mf[s, f] = msub[s] if t < 0 else min(msub[s], msub[t])
                if t < 0:
                    self.face_id[s, f] = len(self.face_sides)
                    self.face_sides.append([(s, f)])
                    self.face_m.append(self.mf[s, f])
                elif t > s:
                    g = len(self.face_sides)
                    self.face_id[s, f] = g
                    self.face_id[t, f ^ 1] = g
                    self.face_sides.append([(s, f), (t, f ^ 1)])
                    self.face_m.append(self.mf[s, f])
        self.face_m = np.array(self.face_m, dtype=int)
        self.nface = len(self.face_sides)
        self.face_off = np.concatenate([[0], np.cumsum(self.face_m)]).astype(int)
        self.b = self.mf.sum(axis=1)

    def level1_index(self, s):
        """Positions of subdomain s's level-1 entries in the flat face array."""
        out = []
        for f in range(6):
            g = self.face_id[s, f]
            out.append(self.face_off[g] + np.arange(self.mf[s, f]))
        return np.concatenate(out)

    def face_slices(self, s):
        """Slices of subdomain s's b-vector per face."""
        off = np.concatenate([[0], np.cumsum(self.mf[s])])
        return [slice(off[f], off[f + 1]) for f in range(6)]
