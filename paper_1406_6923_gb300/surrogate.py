"""Training and evaluation workflow of the learned surrogate of the offline
stage (Algorithm 1 stage 1 replaced by a network for blocks of a fixed size;
the exact build stays as fallback).

Only orchestration and marshalling live here: the ROM builds, the encoding
of the targets, the decoder fit, the network's forward and backward passes,
Adam, decoding and the NtD-map errors all run in ``libsfm``'s kernels
(``include/sfm.h``).  Device buffers are torch tensors (plumbing only)."""
from __future__ import annotations

import time

import numpy as np

from . import sfm


def tile_blocks(blocks):
    """A velocity model made of ``count`` n^3 blocks side by side, so that one
    offline build gives every block's ROM: each subdomain's ROM depends only
    on its own cells and its face basis (the same m on every face), not on
    its neighbours.  Returns (c [nz][ny][nx], xcuts, ycuts, zcuts, order)
    with order[s] the block of subdomain s."""
    blocks = np.asarray(blocks)
    count, n = blocks.shape[0], blocks.shape[1]
    ax = int(np.ceil(count ** (1 / 3)))
    ay = int(np.ceil(np.sqrt(count / ax)))
    az = int(np.ceil(count / (ax * ay)))
    c = np.empty((az * n, ay * n, ax * n))
    order = []
    for s in range(ax * ay * az):
        i, j, kk = s % ax, (s // ax) % ay, s // (ax * ay)
        b = s % count                   # pad the last layer with repeats
        c[kk * n:(kk + 1) * n, j * n:(j + 1) * n, i * n:(i + 1) * n] = blocks[b]
        order.append(b)
    cuts = lambda a: np.arange(a + 1) * n
    return c, cuts(ax), cuts(ay), cuts(az), np.asarray(order)


def build_sets(h, blocks, h_grid, m, k, sigma, cg_tol=1e-14, chunk=512):
    """Exact ROMs (GPU builder) of every block: FP64 coefficient sets
    [count][2k][b][b] (Gamma_1..k, Gammahat_1..k) and the build's wall time
    per block.  Blocks are built ``chunk`` at a time (the builder keeps each
    subdomain's Krylov basis until sfm_free_build, ~0.1 GB per 24^3 block at
    k = 16, m = 8)."""
    b = 6 * m
    out = []
    secs = 0.0
    for c0 in range(0, len(blocks), chunk):
        part = np.asarray(blocks[c0:c0 + chunk])
        c, xc, yc, zc, order = tile_blocks(part)
        sfm.sfm_set_model(h, c, h_grid, xc, yc, zc)
        nsub = len(order)
        t0 = time.perf_counter()
        sfm.sfm_build_roms(h, np.full(nsub, m), np.full(nsub, k), sigma, cg_tol)
        secs += time.perf_counter() - t0
        coef = sfm.sfm_get_coeffs(h).reshape(nsub, 2 * k, b, b)
        sfm.sfm_free_build(h)
        first = {}
        for s, blk in enumerate(order):
            first.setdefault(int(blk), s)
        out.append(np.stack([coef[first[i]] for i in range(len(part))]))
    return np.concatenate(out), secs / len(blocks)


def train(torch, net, c_dev, codes_dev, epochs, batch, lr, seed=0, log=None):
    """Mini-batch Adam on the code loss; returns the per-epoch mean losses."""
    n = c_dev.shape[0]
    rng = np.random.default_rng(seed)
    losses = []
    for ep in range(epochs):
        perm = torch.as_tensor(rng.permutation(n), device=c_dev.device)
        tot, cnt = 0.0, 0
        for i0 in range(0, n - batch + 1, batch):
            idx = perm[i0:i0 + batch]
            cb = c_dev.index_select(0, idx).contiguous()
            zb = codes_dev.index_select(0, idx).contiguous()
            loss, _ = sfm.sfm_net_grad(net, cb.data_ptr(), zb.data_ptr(), batch)
            sfm.sfm_net_adam(net, lr)
            tot += loss
            cnt += 1
        losses.append(tot / max(cnt, 1))
        if log:
            log(f"epoch {ep}: loss {losses[-1]:.4e}")
    return losses


def predict_sets(torch, net, code, c_dev, exact_sets_dev, bf16=True):
    """Coefficient sets of the network (code size ``code``) for the blocks
    c_dev: levels 2..k decoded from its codes, level 1 copied from
    exact_sets_dev (its closed forms need no network)."""
    B = c_dev.shape[0]
    z = torch.empty((B, code), dtype=torch.float32, device=c_dev.device)
    sfm.sfm_net_forward(net, c_dev.data_ptr(), B, z.data_ptr(), bf16=bf16)
    out = exact_sets_dev.clone()
    sfm.sfm_net_decode(net, z.data_ptr(), B, out.data_ptr())
    return out
