"""Pins of the learned-surrogate reference (oracle/surrogate.py): its layers
against library definitions and finite differences, the factor decoder
against the exact S-fraction, the closed forms of level 1, the NtD-map
error and the fallback test."""
import numpy as np
import pytest
from scipy import signal

import sfm_inputs as inputs
from oracle import pipeline, surrogate as sg


def _rom_of_block(c, m=2, k=3, h=10.0, f_peak=20.0):
    """Exact ROM (oracle build) of one velocity block c[n][n][n]."""
    n = c.shape[0]
    cuts = np.array([0, n])
    p = inputs.Problem("block", n, n, n, h, c, cuts, cuts.copy(), cuts.copy(),
                       np.array([m]), np.array([k]), inputs.default_sigma(f_peak, 2.5), f_peak,
                       np.zeros((0, 3)), np.zeros((0, 3)), 1)
    rs = pipeline.build(p, keep=True)
    return p, rs, rs.subroms[0]


def test_conv3d_matches_library_correlation():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 7, 7, 7))
    W = rng.standard_normal((3, 2, 3, 3, 3))
    b = rng.standard_normal(3)
    for stride in (1, 2):
        got, _ = sg.conv3d_forward(x, W, b, stride)
        xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1)))
        for o in range(3):
            full = sum(signal.correlate(xp[c], W[o, c], mode="valid") for c in range(2)) + b[o]
            np.testing.assert_allclose(got[o], full[::stride, ::stride, ::stride], rtol=0, atol=1e-12)


def test_network_gradients_match_finite_differences():
    """Loss 0.5 |z - t|^2 on a small net: every parameter block (sampled
    entries) and the input against central differences."""
    net = sg.SurrogateNet(n=8, channels=(2, 3, 2), hidden=6, code=4, seed=2)
    rng = np.random.default_rng(3)
    for k in net.p:                          # non-zero biases exercise every path
        net.p[k] = net.p[k] + 0.1 * rng.standard_normal(net.p[k].shape)
    x = rng.standard_normal((1, 8, 8, 8))
    t = rng.standard_normal(4)

    def loss():
        z, _ = net.forward(x)
        return 0.5 * float((z - t) @ (z - t))

    z, st = net.forward(x)
    g, gx = net.backward(z - t, st)
    eps = 1e-6
    for name, w in net.p.items():
        flat = w.reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + eps
            lp = loss()
            flat[idx] = old - eps
            lm = loss()
            flat[idx] = old
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - g[name].reshape(-1)[idx]) <= 1e-6 * max(1.0, abs(fd)), (name, idx)
    xf = x.reshape(-1)
    for idx in rng.choice(xf.size, size=8, replace=False):
        old = xf[idx]
        xf[idx] = old + eps
        lp = loss()
        xf[idx] = old - eps
        lm = loss()
        xf[idx] = old
        assert abs((lp - lm) / (2 * eps) - gx.reshape(-1)[idx]) <= 1e-6 * max(1.0, abs(lp - lm) / (2 * eps))


@pytest.fixture(scope="module")
def block_rom():
    rng = np.random.default_rng(11)
    c = inputs.lognormal_block(6, 10.0, rng)
    return _rom_of_block(c)


def test_decoder_round_trip_reproduces_the_exact_rom(block_rom):
    """Encoding the exact coefficients and decoding them through an identity
    basis returns them, and with them the exact NtD map."""
    p, rs, sr = block_rom
    b, k = rs.b[0], rs.k[0]
    dec = sg.FactorDecoder(b, k)
    r = dec.encode(rs.Gamma[0], rs.Gammahat[0])
    dec.mu, dec.P = np.zeros_like(r), np.eye(len(r))
    G, H = dec.decode(r)
    for j in range(1, k):
        np.testing.assert_allclose(G[j - 1], rs.Gamma[0][j], rtol=0, atol=1e-11 * np.abs(rs.Gamma[0][j]).max())
        np.testing.assert_allclose(H[j - 1], rs.Gammahat[0][j], rtol=0, atol=1e-11 * np.abs(rs.Gammahat[0][j]).max())
    G1, H1 = sg.level_one(sr.F, sr.L)
    Gam = [G1] + G
    Gh = [H1] + H
    lams = sg.frequencies(p.f_peak)
    assert sg.ntd_error(Gam, Gh, rs.Gamma[0], rs.Gammahat[0], lams) < 1e-9


def test_level_one_closed_forms(block_rom):
    p, rs, sr = block_rom
    G1, H1 = sg.level_one(sr.F, sr.L)
    np.testing.assert_allclose(H1, rs.Gammahat[0][0], rtol=0, atol=1e-11 * np.abs(H1).max())
    np.testing.assert_allclose(G1, rs.Gamma[0][0], rtol=0, atol=1e-9 * np.abs(G1).max())


def test_decoded_blocks_are_positive_definite(block_rom):
    """Every raw vector decodes to (U D)(U D)^T with U unit lower triangular
    and D = diag(exp(g)) > 0, i.e. a positive definite block; checked by
    eigenvalues where the factor is well conditioned and by a Cholesky
    factorisation with the expected diagonal."""
    p, rs, sr = block_rom
    b, k = rs.b[0], rs.k[0]
    dec = sg.FactorDecoder(b, k)
    rng = np.random.default_rng(5)
    for _ in range(5):
        raw = rng.standard_normal(dec.nblocks * dec.nper)
        for i in range(dec.nblocks):
            raw[i * dec.nper:i * dec.nper + dec.nlow] *= 0.1      # well-conditioned factors
        G, H = dec.blocks(raw)
        for i, B in enumerate(G + H):
            ev = np.linalg.eigvalsh(B)
            assert ev.min() > 1e-6 * ev.max()
            g = raw[i * dec.nper + dec.nlow:(i + 1) * dec.nper]
            np.testing.assert_allclose(np.diag(np.linalg.cholesky(B)), np.exp(g), rtol=1e-10)


def test_decoder_raw_errors_are_relative_per_direction(block_rom):
    """A raw error of 1e-3 in one block (its unit-lower part and its log
    pivots) moves the NtD map by about that much, not by O(1)."""
    p, rs, sr = block_rom
    b, k = rs.b[0], rs.k[0]
    dec = sg.FactorDecoder(b, k)
    r0 = dec.encode(rs.Gamma[0], rs.Gammahat[0])
    rng = np.random.default_rng(9)
    G1, H1 = sg.level_one(sr.F, sr.L)
    for i in range(dec.nblocks):
        r = r0.copy()
        r[i * dec.nper:(i + 1) * dec.nper] += 1e-3 * rng.standard_normal(dec.nper)
        G, H = dec.blocks(r)
        err = sg.ntd_error([G1] + G, [H1] + H, rs.Gamma[0], rs.Gammahat[0], sg.frequencies(p.f_peak))
        assert 1e-6 < err < 5e-2, (i, err)


def test_fallback_flags_a_wrong_rom_and_passes_the_exact_one(block_rom):
    """The block solve F^T (L + sigma)^{-1} F against the decoded S(sigma):
    the exact coefficients pass, a coefficient set with one level off by 50%
    is flagged, and its NtD error shows it."""
    p, rs, sr = block_rom
    sigma = p.sigma
    S_sigma = sr.F.T @ np.linalg.solve(sr.L.toarray() + sigma * np.eye(sr.L.shape[0]), sr.F)
    Gam, Gh = list(rs.Gamma[0]), list(rs.Gammahat[0])
    assert not sg.needs_fallback(Gam, Gh, S_sigma, sigma, 1e-8)
    bad = [x.copy() for x in Gh]
    bad[1] = 1.5 * bad[1]
    assert sg.needs_fallback(Gam, bad, S_sigma, sigma, 1e-3)
    assert sg.ntd_error(Gam, bad, Gam, Gh, sg.frequencies(p.f_peak)) > 1e-3


def test_adam_step_matches_its_definition():
    w, g = np.array([1.0, -2.0]), np.array([0.5, -0.25])
    w1, m, v = sg.adam_update(w, g, np.zeros(2), np.zeros(2), 1, lr=0.1, eps=0.0)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)
    np.testing.assert_allclose(w1, w - 0.1 * np.sign(g))   # bias-corrected first step


@pytest.mark.slow
def test_training_reduces_the_code_loss():
    """Targets from exact ROMs of a few seeded blocks, the decoder fitted to
    them, Adam on the code loss: the loss falls."""
    rng = np.random.default_rng(21)
    blocks = [inputs.lognormal_block(8, 10.0, rng) for _ in range(4)]
    roms = [_rom_of_block(c) for c in blocks]
    b, k = roms[0][1].b[0], roms[0][1].k[0]
    dec = sg.FactorDecoder(b, k)
    R = dec.fit([r[1].Gamma[0] for r in roms], [r[1].Gammahat[0] for r in roms], d=3)
    codes = [dec.code_of(R[:, i]) for i in range(R.shape[1])]
    net = sg.SurrogateNet(n=8, channels=(2, 3, 2), hidden=16, code=3, seed=4)
    state = {k2: (np.zeros_like(w), np.zeros_like(w)) for k2, w in net.p.items()}

    def total():
        return sum(sg.code_loss(net.forward(sg.features(c))[0], z)[0] for c, z in zip(blocks, codes))

    first = total()
    for t in range(1, 101):
        grads = {k2: np.zeros_like(w) for k2, w in net.p.items()}
        for c, z in zip(blocks, codes):
            zz, st = net.forward(sg.features(c))
            g, _ = net.backward(sg.code_loss(zz, z)[1], st)
            for k2 in grads:
                grads[k2] += g[k2]
        for k2 in net.p:
            m, v = state[k2]
            net.p[k2], m, v = sg.adam_update(net.p[k2], grads[k2], m, v, t, lr=3e-2)
            state[k2] = (m, v)
    assert total() < 0.5 * first
