"""Algorithm 1 stage 2: coupled explicit time stepping of the subdomain ROMs.

State.  Each subdomain holds levels ``U_1..U_k`` (each in R^b, b = sum of its
face mode counts).  Level 1 is split into the face blocks of its 6 faces; a
face shared by two subdomains has ONE level-1 block, which is the continuity
condition ``[U_1^a]_b = [U_1^b]_a`` of Eq. (17).

Right-hand sides, evaluated at the current step (end of section "Stage 2"):

* level flux ``phi_j = Gamma_j (U_{j+1} - U_j)``, ``U_{k+1} = 0`` (Eq. 12);
* interior levels j >= 2 (Eq. 19 with the source of Algorithm 1 step 1.4):
  ``U_j'' = Gammahat_j (phi_j - phi_{j-1} + p_j f(t))``;
* a face shared by a and b (Eq. 18):
  ``U_f'' = H_f ([phi_1^a + p_1^a f]_f + [phi_1^b + p_1^b f]_f)`` with
  ``H_f = ([Gammahat_1^a]_f^{-1} + [Gammahat_1^b]_f^{-1})^{-1}``;
  an outer face (homogeneous Neumann, no neighbour) has the single term,
  ``H_f = [Gammahat_1^a]_f``.

Eq. (18) needs ``Gammahat_1`` block diagonal over faces; with ``F`` in the
subspace, ``Gammahat_1 = F^T F = B^T M^{-1} B``, which is block diagonal
because the open-face supports are disjoint.

Time integrator.  The paper allows any standard scheme; here leapfrog
``U^{n+1} = 2U^n - U^{n-1} + dt^2 a^n`` in the two-level increment form
``delta^{n+1} = delta^n + dt^2 a^n``, ``U^{n+1} = U^n + delta^{n+1}``, from rest
(U = delta = 0).  Traces are ``d_r(t_n) = sum_j rho_{r,j}^T U_j^n`` at
``t_n = n dt``, n = 0..nsteps.  Per step, the order of Algorithm 1 is kept:
(2.1) face data ``[phi_1 + p_1 f]_f`` is published, (2.2) interior levels are
updated, (2.3) faces are updated from both sides' data.

``assembled`` writes the same scheme as one mass/stiffness system
``MM U'' = -KK U + f`` (used for the CFL limit, the conserved energy and as an
independent check of the structured stepping).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .eig import lanczos_max


class RomSet:
    """All subdomain ROMs of a problem in S-fraction form plus the projected
    sources and receivers.

    ``Gamma[s], Gammahat[s]``: arrays (k_s, b_s, b_s), levels 1..k;
    ``src[q]``: dict subdomain -> (k_s, b_s) rows of shot q;
    ``rec[r]``: dict subdomain -> (k_s, b_s) rows of receiver r."""

    def __init__(self, topo, Gamma, Gammahat, src, rec):
        self.topo = topo
        self.Gamma = Gamma
        self.Gammahat = Gammahat
        self.src = src
        self.rec = rec
        self.nsub = topo.nsub
        self.b = np.array([g.shape[1] for g in Gamma])
        self.k = np.array([g.shape[0] for g in Gamma])
        self.H = face_H(self)

    @property
    def nshots(self):
        return len(self.src)

    @property
    def nrec(self):
        return len(self.rec)


def face_H(rs):
    """``H_f = (sum over the face's sides of [Gammahat_1]_f^{-1})^{-1}`` (Eq. 18)."""
    topo = rs.topo
    H = []
    for sides in topo.face_sides:
        acc = 0.0
        for (s, f) in sides:
            sl = topo.face_slices(s)[f]
            acc = acc + np.linalg.inv(rs.Gammahat[s][0][sl, sl])
        H.append(np.linalg.inv(acc))
    return H


# ----------------------------------------------------------------------------
# the structured scheme (what the GPU path computes)
# ----------------------------------------------------------------------------

def _groups(rs):
    keys = {}
    for s in range(rs.nsub):
        keys.setdefault((int(rs.b[s]), int(rs.k[s])), []).append(s)
    return [(np.array(v), b, k) for (b, k), v in keys.items()]


def step_structured(rs, dt, nsteps, wavelet, U0=None, V0=None):
    """Coupled leapfrog of all subdomain ROMs (Algorithm 1 stage 2).

    ``wavelet``: [nshots, nsteps] samples ``f(t_n)``.  Returns traces
    ``[nshots, nrec, nsteps+1]`` (float64).  The state is one flat array:
    the face blocks first, then the levels 2..k of every subdomain, grouped
    by (b, k) so each group's levels are a (S, k-1, b, shots) view.

    ``U0``, ``V0``: optional initial state and time derivative (Algorithm 1
    step 1.4), per shot a dict subdomain -> (k, b) rows (``rs.U0``/``rs.V0``
    of ``pipeline.build``); missing entries are zero.  The start is the
    second-order Taylor step ``U^1 = U^0 + dt V^0 + dt^2/2 a_hom(U^0) +
    dt^2 p f(t_0)``, i.e. ``delta^0 = dt V^0 - dt^2/2 a_hom(U^0)`` in the
    increment form (``a_hom``: the right-hand side without the source)."""
    topo = rs.topo
    nsh = rs.nshots
    wavelet = np.asarray(wavelet, dtype=np.float64).reshape(nsh, -1)
    nfm = int(topo.face_off[-1])
    groups = []
    pos = nfm
    where = {}                                  # subdomain -> (group, index in group)
    for gi, (subs, b, k) in enumerate(_groups(rs)):
        n = len(subs) * (k - 1) * b
        groups.append(dict(subs=subs, b=b, k=k, lo=pos, hi=pos + n,
                           G=np.stack([rs.Gamma[s] for s in subs]),
                           Gh=np.stack([rs.Gammahat[s][1:] for s in subs]),
                           idx1=np.stack([topo.level1_index(s) for s in subs]),
                           P=np.zeros((len(subs), k, b, nsh))))
        for i, s in enumerate(subs):
            where[s] = (gi, i)
        pos += n
    ndof = pos
    for q in range(nsh):
        for s, row in rs.src[q].items():
            gi, i = where[s]
            groups[gi]["P"][i, :, :, q] = row
    # sparse receiver matrix over the flat state
    rr, cc, vv = [], [], []
    for r in range(rs.nrec):
        for s, row in rs.rec[r].items():
            g = groups[where[s][0]]
            i, b, k = where[s][1], g["b"], g["k"]
            cols = np.concatenate([g["idx1"][i],
                                   g["lo"] + i * (k - 1) * b + np.arange((k - 1) * b)])
            rr.append(np.full(k * b, r))
            cc.append(cols)
            vv.append(row.ravel())
    R = sp.csr_matrix((np.concatenate(vv) if vv else [], (np.concatenate(rr) if rr else [],
                       np.concatenate(cc) if cc else [])), shape=(rs.nrec, ndof))
    Hblk = sp.block_diag([sp.csr_matrix(x) for x in rs.H], format="csr")

    def accel(X, w):
        """Right-hand sides of Eqs. 18-19 at state X with source samples w."""
        a = np.zeros_like(X)
        Uf = X[:nfm]
        face_sum = np.zeros((nfm, nsh))
        for g in groups:
            S, b, k = len(g["subs"]), g["b"], g["k"]
            Ui = X[g["lo"]:g["hi"]].reshape(S, k - 1, b, nsh)
            U = np.concatenate([Uf[g["idx1"]][:, None], Ui], axis=1)          # (S,k,b,q)
            Up = np.concatenate([U, np.zeros_like(U[:, :1])], axis=1)
            delta = Up[:, 1:] - Up[:, :-1]                                    # U_{j+1}-U_j
            phi = np.matmul(g["G"], delta)                                    # Eq. (12)
            src = g["P"] * w
            # (2.1) face data [phi_1 + p_1 f]_f, summed over both sides of a face
            np.add.at(face_sum, g["idx1"], phi[:, 0] + src[:, 0])
            # (2.2) interior levels, Eq. (19)
            ai = np.matmul(g["Gh"], phi[:, 1:] - phi[:, :-1] + src[:, 1:])
            a[g["lo"]:g["hi"]] = ai.reshape(-1, nsh)
        # (2.3) faces, Eq. (18)
        a[:nfm] = Hblk @ face_sum
        return a

    def flat(rows):
        """Per-shot dicts of (k, b) rows -> the flat state (face blocks are
        shared: both sides carry the same values)."""
        X = np.zeros((ndof, nsh))
        for q in range(min(nsh, len(rows))):
            for s, row in rows[q].items():
                g = groups[where[s][0]]
                i, b, k = where[s][1], g["b"], g["k"]
                X[g["idx1"][i], q] = row[0]
                X[g["lo"] + i * (k - 1) * b:g["lo"] + (i + 1) * (k - 1) * b, q] = row[1:].ravel()
        return X

    X = np.zeros((ndof, nsh)) if U0 is None else flat(U0)         # U
    dX = np.zeros((ndof, nsh))                                     # delta
    if V0 is not None:
        dX += dt * flat(V0)
    if U0 is not None:
        dX -= 0.5 * dt * dt * accel(X, np.zeros(nsh))
    out = np.zeros((nsh, rs.nrec, nsteps + 1))
    for it in range(nsteps):
        out[:, :, it] = (R @ X).T
        dX += dt * dt * accel(X, wavelet[:, it])
        X += dX
    out[:, :, nsteps] = (R @ X).T
    return out


def lambda_max(rs, tol=1e-12):
    """Largest eigenvalue of ``MM^{-1} KK`` without assembling KK: Lanczos on
    the symmetric ``C^T KK C``, ``C C^T = MM^{-1}`` blockwise, with ``KK x``
    evaluated subdomain by subdomain as ``E^T D^T Gamma D E x``."""
    topo = rs.topo
    nfm = int(topo.face_off[-1])
    int_off = np.zeros(rs.nsub + 1, dtype=int)
    int_off[0] = nfm
    for s in range(rs.nsub):
        int_off[s + 1] = int_off[s] + (rs.k[s] - 1) * rs.b[s]
    n = int(int_off[-1])

    def sqrt_psd(m):
        w, U = np.linalg.eigh(0.5 * (m + m.T))
        return U * np.sqrt(np.maximum(w, 0.0))
    cs = [sqrt_psd(H) for H in rs.H]
    for s in range(rs.nsub):
        cs += [sqrt_psd(rs.Gammahat[s][j]) for j in range(1, rs.k[s])]
    C = sp.block_diag([sp.csr_matrix(x) for x in cs], format="csr")
    groups = []
    for subs, b, k in _groups(rs):
        E = np.stack([np.concatenate([topo.level1_index(s),
                                      int_off[s] + np.arange((k - 1) * b)]) for s in subs])
        groups.append((E, np.stack([rs.Gamma[s] for s in subs]), b, k))

    def KK(x):
        y = np.zeros_like(x)
        for E, G, b, k in groups:
            U = x[E].reshape(len(E), k, b)
            Up = np.concatenate([U, np.zeros_like(U[:, :1])], axis=1)
            D = Up[:, :-1] - Up[:, 1:]                    # (D U)_j = U_j - U_{j+1}
            GD = np.einsum("sjab,sjb->sja", G, D)
            out = GD.copy()
            out[:, 1:] -= GD[:, :-1]                      # D^T
            np.add.at(y, E.ravel(), out.reshape(-1))
        return y

    return lanczos_max(lambda v: C.T @ KK(C @ v), n, tol=tol)


# ----------------------------------------------------------------------------
# the same scheme as one assembled system
# ----------------------------------------------------------------------------

class Assembled:
    """``MM U'' = -KK U + sum_q f_q w_q(t)``; dofs = face blocks, then the
    levels 2..k of every subdomain.  The inverse mass is block diagonal and
    known without inversion: ``MM^{-1} = blockdiag(H_f, Gammahat_j (j >= 2))``."""

    def __init__(self, rs):
        topo = rs.topo
        nfm = int(topo.face_off[-1])
        self.int_off = np.zeros(rs.nsub + 1, dtype=int)
        self.int_off[0] = nfm
        for s in range(rs.nsub):
            self.int_off[s + 1] = self.int_off[s] + (rs.k[s] - 1) * rs.b[s]
        n = int(self.int_off[-1])
        self.n = n
        minv = list(rs.H)
        for s in range(rs.nsub):
            for j in range(1, rs.k[s]):
                minv.append(rs.Gammahat[s][j])
        self.minv_blocks = minv
        self.MMinv = sp.block_diag([sp.csr_matrix(x) for x in minv], format="csr")
        rows, cols, vals = [], [], []
        self.E = []
        for s in range(rs.nsub):
            b, k = rs.b[s], rs.k[s]
            e = np.concatenate([topo.level1_index(s),
                                self.int_off[s] + np.arange((k - 1) * b)])
            self.E.append(e)
            Ks = np.zeros((k * b, k * b))
            for j in range(k):
                # (D U)_j = U_j - U_{j+1};  D^T Gamma D
                Gj = rs.Gamma[s][j]
                sl = slice(j * b, (j + 1) * b)
                Ks[sl, sl] += Gj
                if j + 1 < k:
                    sn = slice((j + 1) * b, (j + 2) * b)
                    Ks[sn, sn] += Gj
                    Ks[sl, sn] -= Gj
                    Ks[sn, sl] -= Gj
            r, c = np.meshgrid(e, e, indexing="ij")
            rows.append(r.ravel())
            cols.append(c.ravel())
            vals.append(Ks.ravel())
        self.KK = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows),
                                 np.concatenate(cols))), shape=(n, n)).tocsr()
        self.f = np.zeros((n, rs.nshots))
        for q in range(rs.nshots):
            for s, row in rs.src[q].items():
                np.add.at(self.f[:, q], self.E[s], row.ravel())
        self.R = np.zeros((rs.nrec, n))
        for r in range(rs.nrec):
            for s, row in rs.rec[r].items():
                np.add.at(self.R[r], self.E[s], row.ravel())

    def lambda_max(self):
        """Largest eigenvalue of ``MM^{-1} KK``, computed on the symmetric
        ``C^T KK C`` with ``C C^T = MM^{-1}`` blockwise."""
        cs = []
        for m in self.minv_blocks:
            w, U = np.linalg.eigh(0.5 * (m + m.T))
            cs.append(U * np.sqrt(np.maximum(w, 0.0)))
        C = sp.block_diag([sp.csr_matrix(x) for x in cs], format="csr")
        S = C.T @ self.KK @ C
        if self.n <= 3000:
            return float(np.linalg.eigvalsh(S.toarray())[-1])
        return lanczos_max(lambda v: S @ v, self.n)

    def cfl_dt(self):
        """Leapfrog limit ``2 / sqrt(lambda_max(MM^{-1} KK))``."""
        return 2.0 / np.sqrt(self.lambda_max())

    def leapfrog(self, dt, nsteps, wavelet, U0=None, dU0=None, energies=False):
        """Generic leapfrog of the assembled system (increment form)."""
        nsh = self.f.shape[1]
        wavelet = np.asarray(wavelet, dtype=np.float64).reshape(nsh, -1)
        U = np.zeros((self.n, nsh)) if U0 is None else U0.copy()
        dU = np.zeros((self.n, nsh)) if dU0 is None else dU0.copy()
        out = np.zeros((nsh, self.R.shape[0], nsteps + 1))
        en = []
        for it in range(nsteps):
            out[:, :, it] = (self.R @ U).T
            w = wavelet[:, it] if it < wavelet.shape[1] else np.zeros(nsh)
            a = self.MMinv @ (-(self.KK @ U) + self.f * w)
            dU = dU + dt * dt * a
            Un = U + dU
            if energies:
                en.append(self.energy(Un, U, dt))
            U = Un
        out[:, :, nsteps] = (self.R @ U).T
        if energies:
            return out, np.array(en), U, dU
        return out

    def energy(self, U_new, U_old, dt):
        """``1/2 (dU/dt)^T MM (dU/dt) + 1/2 U_new^T KK U_old`` per shot."""
        if not hasattr(self, "_mlu"):
            self._mlu = spla.splu(self.MMinv.tocsc())
        d = U_new - U_old
        return 0.5 * np.sum(d * self._mlu.solve(d), axis=0) / dt ** 2 + \
            0.5 * np.sum(U_new * (self.KK @ U_old), axis=0)
