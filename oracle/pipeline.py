"""The offline stage of Algorithm 1 (steps 1.1-1.4) for every subdomain of a
problem from ``sfm_inputs``, plus helpers shared by the oracle's tests: the
global and "slit" fine grids and the trace error metric."""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

import sfm_inputs as inputs

from . import fine, faces, rom, sfrac, project, coupled


class SubdomainROM:
    """Everything the oracle computes for one subdomain."""

    def __init__(self, problem, topo, s, keep_basis=False):
        self.box = problem.sub_box(s)
        self.K, self.mass = fine.assemble(problem.c, problem.h, self.box)
        self.B = faces.B_matrix(self.box, topo.mf[s], problem.h)
        self.F = self.B / np.sqrt(self.mass)[:, None]
        self.sigma = problem.sigma
        self.k = int(problem.k_sub[s])
        if np.ndim(self.sigma) == 0:
            solve = rom.shifted_solver(self.K, self.mass, self.sigma)
        else:
            # distinct shifts (Eq. 6): one per block after F, the first k-1
            # of the problem's list
            shifts = [float(x) for x in self.sigma[:self.k - 1]]
            if len(shifts) < self.k - 1:
                raise ValueError("fewer shifts than blocks after the first")
            cache = {x: rom.shifted_solver(self.K, self.mass, x) for x in set(shifts)}
            solve = [cache[x] for x in shifts]
        V = rom.krylov_basis(solve, self.F, self.k)
        L = fine.symmetrised(self.K, self.mass)
        self.Lt, self.Ft = rom.galerkin(L, V, self.F)
        self.alpha, self.C, self.R1, Qh = sfrac.block_lanczos(self.Lt, self.Ft, self.k)
        self.Gamma, self.Gammahat, self.G, self.min_eigs = sfrac.gamma_transform(
            self.alpha, self.C, self.R1)
        self._V, self._Qh = V, Qh
        if keep_basis:
            self.V, self.Qh, self.L = V, Qh, L

    def rows(self, vec):
        """Projected rows (k, b) of a nodal vector (Algorithm 1 step 1.4)."""
        return project.project(self._V, self._Qh, self.G, self.mass, vec)

    def state_rows(self, u):
        """S-fraction coordinates (k, b) of a nodal field on the box
        (Algorithm 1 step 1.4, Eq. 16)."""
        return project.project_state(self._V, self._Qh, self.G, self.mass, u)



def build(problem, keep=False, subs=None, u0=None, v0=None, depth_tau=None):
    """Build the ROM set of ``problem``.  ``keep`` keeps every subdomain's
    ``SubdomainROM`` (with V) in ``.subroms``; ``subs`` restricts the build
    to a list of subdomains (their coefficients only, for sampling).
    ``depth_tau``: when given, each subdomain's fraction is cut at
    ``sfrac.usable_depth(..., depth_tau)`` levels (its source, receiver and
    initial rows with it; ``rs.k`` then holds the kept depths).
    ``u0``, ``v0``: initial displacement and velocity, nodal arrays
    [shot][nz+1][ny+1][nx+1] (or without the shot axis for one shot);
    their S-fraction coordinates go to ``rs.U0``, ``rs.V0`` (per shot, a
    dict subdomain -> (k, b)).

    Subdomains whose operator inputs are identical (same box shape, same
    velocity block, same face mode counts, same k) have identical ROMs; the
    build is done once for each distinct input and reused."""
    topo = faces.Topology(problem)
    gmass = fine.global_mass_ijk(problem)
    h = problem.h
    src_w = [inputs.gaussian_node_weights(x, problem.src_width, h, problem.nx, problem.ny,
                                          problem.nz) for x in problem.src_xyz]
    rec_w = [inputs.trilinear_node_weights(x, h, problem.nx, problem.ny, problem.nz)
             for x in problem.rec_xyz]
    Gam, Gh = [None] * problem.nsub, [None] * problem.nsub
    src = [dict() for _ in src_w]
    rec = [dict() for _ in rec_w]
    kept = {}
    built = {}
    inits = []
    for field in (u0, v0):
        if field is None:
            inits.append(None)
            continue
        f = np.asarray(field, dtype=np.float64)
        inits.append(f[None] if f.ndim == 3 else f)
    ninit = max((x.shape[0] for x in inits if x is not None), default=0)
    U0 = [dict() for _ in range(ninit)]
    V0 = [dict() for _ in range(ninit)]
    for s in (range(problem.nsub) if subs is None else subs):
        box = problem.sub_box(s)
        x0, x1, y0, y1, z0, z1 = box
        key = (x1 - x0, y1 - y0, z1 - z0, tuple(int(v) for v in topo.mf[s]),
               int(problem.k_sub[s]), problem.c[z0:z1, y0:y1, x0:x1].tobytes())
        if key not in built:
            built[key] = SubdomainROM(problem, topo, s, keep_basis=keep)
        sr = built[key]
        Gam[s] = np.stack(sr.Gamma)
        Gh[s] = np.stack(sr.Gammahat)
        vecs, where = [], []
        for q, (nodes, w) in enumerate(src_w):
            v = project.local_share(box, gmass, sr.mass, nodes, w)
            if v is not None:
                vecs.append(v)
                where.append((src, q))
        for r, (nodes, w) in enumerate(rec_w):
            v = project.local_share(box, gmass, sr.mass, nodes, w)
            if v is not None:
                vecs.append(v)
                where.append((rec, r))
        if vecs:
            rows = sr.rows(np.stack(vecs, axis=1))
            for (dst, i), row in zip(where, rows):
                dst[i][s] = row
        for field, dst in zip(inits, (U0, V0)):
            if field is None:
                continue
            for q in range(field.shape[0]):
                dst[q][s] = sr.state_rows(field[q, z0:z1 + 1, y0:y1 + 1, x0:x1 + 1].ravel())
        if keep:
            kept[s] = sr
    if subs is not None:
        return topo, Gam, Gh, kept
    if depth_tau is not None:
        depth = [sfrac.usable_depth(Gam[s], Gh[s], depth_tau) for s in range(problem.nsub)]
        Gam = [Gam[s][:depth[s]] for s in range(problem.nsub)]
        Gh = [Gh[s][:depth[s]] for s in range(problem.nsub)]
        cut = lambda rows: [{s: r[:depth[s]] for s, r in d.items()} for d in rows]
        src, rec, U0, V0 = cut(src), cut(rec), cut(U0), cut(V0)
    rs = coupled.RomSet(topo, Gam, Gh, src, rec)
    rs.U0, rs.V0 = U0, V0
    rs.subroms = kept
    rs.distinct = len(built)
    return rs


def rom_dt(rs, safety=0.9, tol=1e-9):
    """``safety * dt_CFL`` of the coupled ROM system (0.9 by default)."""
    return safety * 2.0 / np.sqrt(coupled.lambda_max(rs, tol=tol))


# ----------------------------------------------------------------------------
# reference fine grids
# ----------------------------------------------------------------------------

def fine_system(problem):
    """Global fine grid: ``(K, M, force[N, nshots], rec_rows[nrec, N])``."""
    K, mass = fine.assemble_global(problem)
    box = fine.global_box(problem)
    return (K, mass) + _point_vectors(problem, box, [(box, np.arange(K.shape[0]))], K.shape[0])


def _point_vectors(problem, box, pieces, n):
    h = problem.h
    gmass = fine.global_mass_ijk(problem)
    force = np.zeros((n, problem.nshots))
    R = np.zeros((problem.nrec, n))
    for q, x in enumerate(problem.src_xyz):
        nodes, w = inputs.gaussian_node_weights(x, problem.src_width, h, problem.nx,
                                                problem.ny, problem.nz)
        for pbox, gidx in pieces:
            m = fine.lumped_mass(problem.c, h, pbox)
            v = project.local_share(pbox, gmass, m, nodes, w)
            if v is not None:
                np.add.at(force[:, q], gidx, v)
    for r, x in enumerate(problem.rec_xyz):
        nodes, w = inputs.trilinear_node_weights(x, h, problem.nx, problem.ny, problem.nz)
        for pbox, gidx in pieces:
            m = fine.lumped_mass(problem.c, h, pbox)
            v = project.local_share(pbox, gmass, m, nodes, w)
            if v is not None:
                np.add.at(R[r], gidx, v)
    return force, sp.csr_matrix(R)


def slit_system(problem):
    """The fine grid the ROM converges to under the open-face reading: the
    subdomain operators ``K^a, M^a`` assembled with only the OPEN-face nodes
    of shared faces identified; subdomain edge and corner nodes keep one copy
    per subdomain.  Returns ``(K, M, force, rec_rows)``."""
    pieces, n = slit_nodes(problem)
    Kg = sp.csr_matrix((n, n))
    Mg = np.zeros(n)
    for box, gidx in pieces:
        K, m = fine.assemble(problem.c, problem.h, box)
        P = sp.csr_matrix((np.ones(len(gidx)), (gidx, np.arange(len(gidx)))), shape=(n, len(gidx)))
        Kg = Kg + P @ K @ P.T
        np.add.at(Mg, gidx, m)
    return (Kg.tocsr(), Mg) + _point_vectors(problem, None, pieces, n)


def slit_field(problem, field):
    """A nodal field [nz+1, ny+1, nx+1] on the slit grid's unknowns (every
    copy of a node takes the node's value)."""
    pieces, n = slit_nodes(problem)
    out = np.zeros(n)
    f = np.asarray(field, dtype=np.float64)
    for box, gidx in pieces:
        x0, x1, y0, y1, z0, z1 = box
        out[gidx] = f[z0:z1 + 1, y0:y1 + 1, x0:x1 + 1].ravel()
    return out


def slit_nodes(problem):
    """Numbering of the slit grid: per subdomain ``(box, gidx)``, the slit
    unknown of each local node; open-face nodes of shared faces are numbered
    once, every other node once per subdomain.  Returns ``(pieces, n)``."""
    topo = faces.Topology(problem)
    gid_of = {}
    pieces = []
    nxt = 0
    for s in range(problem.nsub):
        box = problem.sub_box(s)
        gidx = -np.ones(int(np.prod(fine.box_shape(box))), dtype=int)
        for f in range(6):
            if topo.nbr[s, f] < 0:
                continue
            idx, _, _, _ = faces.open_face_nodes(box, f)
            ii, jj, kk = fine.node_coords(box)
            for li in idx:
                key = (ii[li], jj[li], kk[li])
                if key not in gid_of:
                    gid_of[key] = nxt
                    nxt += 1
                gidx[li] = gid_of[key]
        free = gidx < 0
        gidx[free] = nxt + np.arange(free.sum())
        nxt += int(free.sum())
        pieces.append((box, gidx))
    return pieces, nxt


def fine_traces(system, dt, nsteps, wavelet, u0=None, v0=None):
    """Fine-grid leapfrog traces ``[nshots, nrec, nsteps+1]`` of a system from
    :func:`fine_system` / :func:`slit_system`; ``u0``, ``v0``: optional
    initial fields in the system's own unknowns, shared by every shot."""
    K, mass, force, R = system
    wavelet = np.asarray(wavelet).reshape(force.shape[1], -1)
    return np.stack([fine.leapfrog(K, mass, dt, nsteps, force[:, q], wavelet[q], R, u0, v0)
                     for q in range(force.shape[1])])


def rel_l2(d, ref):
    """Relative L2 error over all receivers and samples concatenated."""
    d, ref = np.asarray(d, np.float64), np.asarray(ref, np.float64)
    return float(np.linalg.norm(d - ref) / np.linalg.norm(ref))
