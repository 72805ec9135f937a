"""Learned surrogate of the offline stage: the CPU reference (test
infrastructure only; the GPU path never imports it) for a network that maps
a subdomain's velocity block to its S-fraction coefficients, replacing the
Krylov/Lanczos build when the model changes between inversion iterations.

Pieces, in the order the data flows:

* input: log(c / c_ref) on the block's cells, one channel;
* three 3x3x3 convolutions of stride 2 with ReLU (n -> n/2 -> n/4 -> n/8);
* a two-layer MLP (ReLU between) to a code z of dimension d;
* a fixed low-rank decoder r = mu + P z (mean and leading principal
  directions of the training targets, not trained);
* r -> factors of Gamma_j and Gammahat_j for j >= 2, one (unit lower
  triangular) x diag(exp(g)) factor per block, scaled per level: every
  decoded block is positive definite, so the ROM it gives is a passive
  S-fraction (Eqs. 12-13) whatever the network outputs;
* level 1 from its closed forms, Gammahat_1 = F^T F and
  Gamma_1 = Gammahat_1^{-1} F^T L F Gammahat_1^{-1} (no solves);
* measured by the NtD map S(lambda) = F^T (L + lambda)^{-1} F, the transfer
  function of the S-fraction (Eq. 15), at complex lambda = (eta + i w)^2;
* fallback: the block solve F^T (L + sigma)^{-1} F at one shift against the
  decoded S(sigma); above the tolerance the exact build is used.

Everything is plain FP64 NumPy, layer by layer, forward and backward
written out; the training loss is the squared error of the code against
the projection of the target on the decoder's basis."""
from __future__ import annotations

import numpy as np

from . import sfrac


# ----------------------------------------------------------------------------
# layers
# ----------------------------------------------------------------------------

def conv3d_forward(x, W, bias, stride=2):
    """3D cross-correlation with zero padding 1: x (Cin, n, n, n), W (Cout,
    Cin, 3, 3, 3) -> (Cout, m, m, m), m = (n - 1) // stride + 1."""
    cin, n = x.shape[0], x.shape[1]
    m = (n - 1) // stride + 1
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1)))
    cols = []
    for a in range(3):
        for b in range(3):
            for c in range(3):
                cols.append(xp[:, a:a + stride * m:stride, b:b + stride * m:stride,
                               c:c + stride * m:stride].reshape(cin, -1))
    P = np.stack(cols, axis=1).reshape(cin * 27, -1)          # (ci, offset) rows
    out = W.reshape(W.shape[0], -1) @ P + bias[:, None]
    return out.reshape(W.shape[0], m, m, m), (P, x.shape, stride)


def conv3d_backward(dout, cache, W):
    """Gradients of conv3d_forward: (dx, dW, dbias)."""
    P, xshape, stride = cache
    cout = W.shape[0]
    cin, n = xshape[0], xshape[1]
    m = dout.shape[1]
    D = dout.reshape(cout, -1)
    dW = (D @ P.T).reshape(W.shape)
    db = D.sum(axis=1)
    dP = (W.reshape(cout, -1).T @ D).reshape(cin, 27, m, m, m)
    dxp = np.zeros((cin, n + 2, n + 2, n + 2))
    o = 0
    for a in range(3):
        for b in range(3):
            for c in range(3):
                dxp[:, a:a + stride * m:stride, b:b + stride * m:stride,
                    c:c + stride * m:stride] += dP[:, o]
                o += 1
    return dxp[:, 1:-1, 1:-1, 1:-1], dW, db


def relu(x):
    return np.maximum(x, 0.0)


# ----------------------------------------------------------------------------
# the network: convolutions + MLP -> code
# ----------------------------------------------------------------------------

class SurrogateNet:
    """Parameters in ``self.p``: conv weights/biases c1..c3, MLP W1, b1, W2,
    b2.  ``forward`` maps an input (1, n, n, n) to the code (d,)."""

    def __init__(self, n=24, channels=(8, 16, 32), hidden=256, code=64, seed=0):
        rng = np.random.default_rng(seed)
        self.n = n
        self.channels = channels
        p = {}
        cin = 1
        m = n
        for i, c in enumerate(channels, start=1):
            p[f"c{i}w"] = rng.standard_normal((c, cin, 3, 3, 3)) * np.sqrt(2.0 / (27 * cin))
            p[f"c{i}b"] = np.zeros(c)
            cin = c
            m = (m - 1) // 2 + 1
        self.flat = cin * m ** 3
        p["W1"] = rng.standard_normal((hidden, self.flat)) * np.sqrt(2.0 / self.flat)
        p["b1"] = np.zeros(hidden)
        p["W2"] = rng.standard_normal((code, hidden)) * np.sqrt(1.0 / hidden)
        p["b2"] = np.zeros(code)
        self.p = p

    def forward(self, x):
        caches = []
        h = x
        for i in range(1, len(self.channels) + 1):
            a, cache = conv3d_forward(h, self.p[f"c{i}w"], self.p[f"c{i}b"], 2)
            caches.append((cache, a))
            h = relu(a)
        f = h.reshape(-1)
        a1 = self.p["W1"] @ f + self.p["b1"]
        h1 = relu(a1)
        z = self.p["W2"] @ h1 + self.p["b2"]
        return z, (caches, h.shape, f, a1, h1)

    def backward(self, dz, state):
        """Gradients of every parameter (dict) and of the input."""
        caches, hshape, f, a1, h1 = state
        g = {"W2": np.outer(dz, h1), "b2": dz.copy()}
        dh1 = self.p["W2"].T @ dz
        da1 = dh1 * (a1 > 0)
        g["W1"] = np.outer(da1, f)
        g["b1"] = da1
        dh = (self.p["W1"].T @ da1).reshape(hshape)
        for i in range(len(self.channels), 0, -1):
            cache, a = caches[i - 1]
            da = dh * (a > 0)
            dh, g[f"c{i}w"], g[f"c{i}b"] = conv3d_backward(da, cache, self.p[f"c{i}w"])
        return g, dh


def features(c, c_ref=2500.0):
    """Network input of a velocity block c[nz][ny][nx]: log(c / c_ref)."""
    return np.log(np.asarray(c, dtype=np.float64) / c_ref)[None]


# ----------------------------------------------------------------------------
# the decoder: code -> factors of Gamma_j, Gammahat_j (j >= 2)
# ----------------------------------------------------------------------------

class FactorDecoder:
    """Block layout: levels 2..k, each with Gamma_j and Gammahat_j written as
    B = s^2 (U D)(U D)^T, U unit lower triangular, D = diag(exp(g)), s a
    per-(level, kind) constant; a block's raw numbers are U's entries below
    the diagonal (row by row) followed by g.  Every raw vector decodes to a
    positive definite block, and errors are relative per direction (a raw
    error e moves a pivot by the factor exp(e)), which keeps the NtD map
    well conditioned in the raw numbers; entrywise errors in the factor
    itself are not (a 1e-3 error in one Gamma_j factor, relative to its
    largest entry, can move the NtD map by O(1))."""

    def __init__(self, b, k):
        self.b, self.k = b, k
        self.low = np.tril_indices(b, -1)
        self.nlow = len(self.low[0])
        self.nper = self.nlow + b
        self.nblocks = 2 * (k - 1)
        self.scale = np.ones(self.nblocks)
        self.mu = None
        self.P = None

    def _blocks(self, Gam, Gh):
        return [Gam[j] for j in range(1, self.k)] + [Gh[j] for j in range(1, self.k)]

    def encode(self, Gam, Gh):
        """Raw vector of a coefficient set (from exact Cholesky factors)."""
        out = []
        for i, B in enumerate(self._blocks(Gam, Gh)):
            L = np.linalg.cholesky(0.5 * (B + B.T)) / self.scale[i]
            d = np.diag(L).copy()
            U = L / d[None, :]
            out.append(np.concatenate([U[self.low], np.log(d)]))
        return np.concatenate(out)

    def blocks(self, r):
        """Raw vector -> (Gamma_2..k, Gammahat_2..k)."""
        mats = []
        for i in range(self.nblocks):
            v = r[i * self.nper:(i + 1) * self.nper]
            U = np.eye(self.b)
            U[self.low] = v[:self.nlow]
            L = U * (np.exp(v[self.nlow:]) * self.scale[i])[None, :]
            mats.append(L @ L.T)
        return mats[:self.k - 1], mats[self.k - 1:]

    def fit(self, targets_Gam, targets_Gh, d):
        """Per-block scales (geometric mean of the factors' diagonals over
        the data), then the mean and the d leading principal directions of
        the raw targets."""
        for i in range(self.nblocks):
            logs = []
            for Gam, Gh in zip(targets_Gam, targets_Gh):
                B = self._blocks(Gam, Gh)[i]
                logs.append(np.mean(np.log(np.diag(np.linalg.cholesky(0.5 * (B + B.T))))))
            self.scale[i] = np.exp(np.mean(logs))
        R = np.stack([self.encode(G, H) for G, H in zip(targets_Gam, targets_Gh)], axis=1)
        self.mu = R.mean(axis=1)
        U, s, _ = np.linalg.svd(R - self.mu[:, None], full_matrices=False)
        self.P = U[:, :d]
        return R

    def code_of(self, r):
        """Projection of a raw target on the decoder's basis."""
        return self.P.T @ (r - self.mu)

    def decode(self, z):
        return self.blocks(self.mu + self.P @ z)


# ----------------------------------------------------------------------------
# level 1, the NtD map and the fallback test
# ----------------------------------------------------------------------------

def level_one(F, L):
    """Closed forms ``Gammahat_1 = F^T F``,
    ``Gamma_1 = Gammahat_1^{-1} F^T L F Gammahat_1^{-1}``."""
    Gh1 = F.T @ F
    Gi = np.linalg.inv(Gh1)
    G1 = Gi @ (F.T @ (L @ F)) @ Gi
    return 0.5 * (G1 + G1.T), 0.5 * (Gh1 + Gh1.T)


def frequencies(f_peak, count=16, eta_hz=4.0, band=2.5):
    """``lambda_i = (eta + i w_i)^2``, ``w_i = 2 pi f_i``, f_i evenly spaced
    in (0, band * f_peak], ``eta = 2 pi eta_hz``."""
    f = band * f_peak * np.arange(1, count + 1) / count
    return (2 * np.pi * eta_hz + 2j * np.pi * f) ** 2


def ntd_error(Gam, Gh, Gam_ref, Gh_ref, lams):
    """Largest relative Frobenius error of the S-fraction's NtD map over the
    given lambdas."""
    worst = 0.0
    for lam in lams:
        a = sfrac.transfer_sfraction(list(Gam), list(Gh), lam)
        r = sfrac.transfer_sfraction(list(Gam_ref), list(Gh_ref), lam)
        worst = max(worst, float(np.linalg.norm(a - r) / np.linalg.norm(r)))
    return worst


def needs_fallback(Gam, Gh, S_sigma, sigma, tol):
    """True when the decoded S(sigma) is further than ``tol`` (relative) from
    the block solve ``S_sigma = F^T (L + sigma)^{-1} F``."""
    a = sfrac.transfer_sfraction(list(Gam), list(Gh), sigma)
    return bool(np.linalg.norm(a - S_sigma) / np.linalg.norm(S_sigma) > tol)


# ----------------------------------------------------------------------------
# training
# ----------------------------------------------------------------------------

def code_loss(z, z_target):
    """Mean squared error of the code and its gradient."""
    e = z - z_target
    return float(e @ e) / len(e), 2.0 * e / len(e)


def adam_update(w, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma and Ba): returns the new (w, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v
