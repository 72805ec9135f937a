"""GPU kernels of the learned surrogate (forward, backward, Adam, BF16
inference) against the FP64 CPU reference ``oracle/surrogate.py``, through
the C ABI."""
import numpy as np
import pytest

import sfm_inputs as inputs
from oracle import surrogate as osur

pytestmark = pytest.mark.gpu

# FP32 forward/backward against FP64: sums of up to a few thousand terms
# (dense layer of 1728 inputs) in FP32, compared tensor by tensor in norm.
GRAD_TOL = 1e-5


@pytest.fixture(scope="module")
def env():
    import os
    torch = pytest.importorskip("torch")
    from paper_1406_6923_gb300 import _build, sfm as mod
    if not os.path.exists(mod.LIB_PATH):
        _build.build()
    mod.load()
    return mod, torch


NAMES = ["c1w", "c1b", "c2w", "c2b", "c3w", "c3b", "W1", "b1", "W2", "b2"]


def flat_params(onet):
    return np.concatenate([onet.p[k].ravel() for k in NAMES]).astype(np.float32)


def oracle_batch(onet, blocks, zt):
    """Mean loss over the batch and the mean gradient (oracle, FP64)."""
    B = len(blocks)
    loss = 0.0
    grads = {k: np.zeros_like(v) for k, v in onet.p.items()}
    zs = []
    for c, t in zip(blocks, zt):
        z, state = onet.forward(osur.features(c))
        l, dz = osur.code_loss(z, t)
        g, _ = onet.backward(dz / B, state)
        for k in grads:
            grads[k] += g[k]
        loss += l / B
        zs.append(z)
    return loss, grads, np.stack(zs)


def make_net(sfm, onet, n, channels, hidden, code):
    net = sfm.sfm_net_create(0, n, *channels, hidden, code, 1)
    sfm.sfm_net_params(net, flat_params(onet))
    return net


@pytest.mark.parametrize("shape", [(8, (2, 3, 4), 16, 5), (24, (16, 32, 64), 1024, 64)])
def test_forward_and_gradients_match_the_oracle(env, shape):
    sfm, torch = env
    n, channels, hidden, code = shape
    onet = osur.SurrogateNet(n=n, channels=channels, hidden=hidden, code=code, seed=3)
    rng = np.random.default_rng(5)
    blocks = inputs.surrogate_blocks(3, n=n, seed=11)
    zt = rng.standard_normal((3, code))
    loss_ref, g_ref, z_ref = oracle_batch(onet, blocks, zt)
    net = make_net(sfm, onet, n, channels, hidden, code)
    try:
        c = torch.tensor(np.asarray(blocks, np.float32), device="cuda")
        t = torch.tensor(zt.astype(np.float32), device="cuda")
        z = torch.empty((3, code), dtype=torch.float32, device="cuda")
        sfm.sfm_net_forward(net, c.data_ptr(), 3, z.data_ptr(), bf16=False)
        loss, grad = sfm.sfm_net_grad(net, c.data_ptr(), t.data_ptr(), 3, want_grad=True)
    finally:
        sfm.sfm_net_destroy(net)
    zg = z.cpu().numpy()
    assert np.linalg.norm(zg - z_ref) <= GRAD_TOL * np.linalg.norm(z_ref)
    assert abs(loss - loss_ref) <= GRAD_TOL * loss_ref
    off = 0
    for k in NAMES:
        ref = g_ref[k].ravel()
        got = grad[off:off + ref.size]
        off += ref.size
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        print(f"{shape[0]}^3 net, d{k}: rel err {err:.2e}")
        assert err <= GRAD_TOL, k


def test_bf16_inference_stays_near_fp32(env):
    sfm, torch = env
    onet = osur.SurrogateNet(n=24, channels=(16, 32, 64), hidden=1024, code=64, seed=3)
    blocks = inputs.surrogate_blocks(4, n=24, seed=12)
    net = make_net(sfm, onet, 24, (16, 32, 64), 1024, 64)
    try:
        c = torch.tensor(np.asarray(blocks, np.float32), device="cuda")
        z32 = torch.empty((4, 64), dtype=torch.float32, device="cuda")
        z16 = torch.empty_like(z32)
        sfm.sfm_net_forward(net, c.data_ptr(), 4, z32.data_ptr(), bf16=False)
        sfm.sfm_net_forward(net, c.data_ptr(), 4, z16.data_ptr(), bf16=True)
    finally:
        sfm.sfm_net_destroy(net)
    a, b = z32.cpu().numpy(), z16.cpu().numpy()
    err = np.linalg.norm(a - b) / np.linalg.norm(a)
    print(f"BF16 vs FP32 codes: {err:.2e}")
    # 8 significant bits per stored weight and activation over five layers
    assert err < 5e-2


def test_adam_step_matches_its_definition(env):
    sfm, torch = env
    onet = osur.SurrogateNet(n=8, channels=(2, 3, 4), hidden=16, code=5, seed=4)
    blocks = inputs.surrogate_blocks(2, n=8, seed=13)
    zt = np.random.default_rng(6).standard_normal((2, 5))
    net = make_net(sfm, onet, 8, (2, 3, 4), 16, 5)
    try:
        c = torch.tensor(np.asarray(blocks, np.float32), device="cuda")
        t = torch.tensor(zt.astype(np.float32), device="cuda")
        _, g = sfm.sfm_net_grad(net, c.data_ptr(), t.data_ptr(), 2, want_grad=True)
        w0 = sfm.sfm_net_params(net)
        sfm.sfm_net_adam(net, 1e-3)
        w1 = sfm.sfm_net_params(net)
    finally:
        sfm.sfm_net_destroy(net)
    want, _, _ = osur.adam_update(w0.astype(np.float64), g.astype(np.float64), 0.0, 0.0, 1, lr=1e-3)
    np.testing.assert_allclose(w1, want, rtol=1e-5, atol=1e-7)


def test_training_fits_a_seeded_set(env):
    """A few hundred Adam steps on 8 blocks with random target codes drive
    the loss far down (the network can fit a small set)."""
    sfm, torch = env
    blocks = inputs.surrogate_blocks(8, n=24, seed=14)
    zt = np.random.default_rng(7).standard_normal((8, 16)).astype(np.float32)
    net = sfm.sfm_net_create(0, 24, 8, 16, 32, 256, 16, 2)
    try:
        c = torch.tensor(np.asarray(blocks, np.float32), device="cuda")
        t = torch.tensor(zt, device="cuda")
        first, _ = sfm.sfm_net_grad(net, c.data_ptr(), t.data_ptr(), 8)
        for _ in range(300):
            loss, _ = sfm.sfm_net_grad(net, c.data_ptr(), t.data_ptr(), 8)
            sfm.sfm_net_adam(net, 2e-3)
    finally:
        sfm.sfm_net_destroy(net)
    print(f"loss {first:.3e} -> {loss:.3e}")
    assert loss < 1e-2 * first


@pytest.fixture(scope="module")
def rom_sets():
    """Eight oracle-built S-fractions of one width (m = 2 on every face,
    b = 12) and depth (k = 4): 4^3-cell subdomains of a random medium."""
    from oracle import pipeline
    p = inputs.small_problem(ncell=(8, 8, 8), cuts=(4, 4, 4), m=2, k=4, model="random")
    rs = pipeline.build(p)
    b, k = int(rs.b[0]), int(rs.k[0])
    sets = np.stack([np.concatenate([np.stack(rs.Gamma[s]).ravel(), np.stack(rs.Gammahat[s]).ravel()])
                     for s in range(rs.nsub)])
    return rs, b, k, sets


def test_encode_matches_the_oracle(env, rom_sets):
    sfm, torch = env
    rs, b, k, sets = rom_sets
    dec = osur.FactorDecoder(b, k)
    want = np.stack([dec.encode(rs.Gamma[s], rs.Gammahat[s]) for s in range(rs.nsub)])
    coef = torch.tensor(sets, device="cuda")
    raw = torch.empty((rs.nsub, sfm.raw_size(b, k)), dtype=torch.float64, device="cuda")
    sfm.sfm_raw_encode(0, rs.nsub, b, k, coef.data_ptr(), raw.data_ptr())
    got = raw.cpu().numpy()
    np.testing.assert_allclose(got, want, rtol=1e-9, atol=1e-9)


def test_decoder_round_trip_is_exact(env, rom_sets):
    """With code = N - 1 the fitted subspace holds every centred target, so
    encode -> fit -> code -> decode returns the blocks of levels 2..k (and
    the NtD map) to rounding."""
    sfm, torch = env
    rs, b, k, sets = rom_sets
    N = rs.nsub
    coef = torch.tensor(sets, device="cuda")
    raw = torch.empty((N, sfm.raw_size(b, k)), dtype=torch.float64, device="cuda")
    sfm.sfm_raw_encode(0, N, b, k, coef.data_ptr(), raw.data_ptr())
    net = sfm.sfm_net_create(0, 8, 2, 2, 2, 8, N - 1, 1)
    try:
        codes = torch.empty((N, N - 1), dtype=torch.float32, device="cuda")
        sfm.sfm_net_fit_decoder(net, b, k, raw.data_ptr(), N, iters=2, seed=3, codes_ptr=codes.data_ptr())
        # decode the codes (FP32, the network's output type) over a copy that
        # keeps level 1
        out = coef.clone()
        sfm.sfm_net_decode(net, codes.data_ptr(), N, out.data_ptr())
    finally:
        sfm.sfm_net_destroy(net)
    got = out.cpu().numpy().reshape(N, 2, k, b, b)
    ref = sets.reshape(N, 2, k, b, b)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    print(f"decoder round trip through FP32 codes: rel err {err:.2e}")
    # the codes are FP32 (the network's output precision): 1e-6 relative per
    # raw number, amplified by exp() on the pivots
    assert err < 1e-5
    lams = osur.frequencies(20.0)
    e = sfm.sfm_ntd_error(0, N, b, k, out.data_ptr(), coef.data_ptr(), lams)
    print(f"decoder round trip NtD error: {e.max():.2e}")
    assert e.max() < 1e-4


def test_ntd_map_matches_the_oracle(env, rom_sets):
    """The GPU transfer function of an S-fraction against the oracle's
    continued fraction, through the relative error of two different sets."""
    from oracle import sfrac
    sfm, torch = env
    rs, b, k, sets = rom_sets
    lams = osur.frequencies(20.0)
    a = torch.tensor(sets[:4], device="cuda")
    r = torch.tensor(sets[4:8], device="cuda")
    got = sfm.sfm_ntd_error(0, 4, b, k, a.data_ptr(), r.data_ptr(), lams)
    for i in range(4):
        for li, lam in enumerate(lams):
            Sa = sfrac.transfer_sfraction(list(rs.Gamma[i]), list(rs.Gammahat[i]), lam)
            Sr = sfrac.transfer_sfraction(list(rs.Gamma[4 + i]), list(rs.Gammahat[4 + i]), lam)
            want = np.linalg.norm(Sa - Sr) / np.linalg.norm(Sr)
            assert abs(got[i, li] - want) <= 1e-8 * max(want, 1e-3), (i, li, got[i, li], want)


@pytest.fixture(scope="module")
def trained(env):
    """A small surrogate trained on the GPU end to end: 8^3-cell blocks of
    the surrogate recipe (log-normal background, 1-3 interfaces), m = 2
    (b = 12), k = 4, exact ROMs from the GPU builder (128 training and 32
    test blocks), decoder fitted on the training targets, 40 epochs of
    Adam."""
    sfm, torch = env
    from paper_1406_6923_gb300 import surrogate as sur
    n, m, k, f = 8, 2, 4, 40.0
    sigma = inputs.default_sigma(f, 8.0)
    blocks = inputs.surrogate_blocks(160, n=n, seed=21)
    h = sfm.sfm_create(0)
    try:
        sets, per_block = sur.build_sets(h, blocks, 10.0, m, k, sigma)
    finally:
        sfm.sfm_destroy(h)
    b, code = 6 * m, 24
    dev = "cuda"
    sets_d = torch.tensor(sets.reshape(len(blocks), -1), device=dev)
    raw = torch.empty((len(blocks), sfm.raw_size(b, k)), dtype=torch.float64, device=dev)
    sfm.sfm_raw_encode(0, len(blocks), b, k, sets_d.data_ptr(), raw.data_ptr())
    net = sfm.sfm_net_create(0, n, 8, 16, 32, 128, code, 5)
    codes = torch.empty((128, code), dtype=torch.float32, device=dev)
    sfm.sfm_net_fit_decoder(net, b, k, raw.data_ptr(), 128, iters=4, seed=9, codes_ptr=codes.data_ptr())
    c = torch.tensor(np.asarray(blocks, np.float32), device=dev)
    losses = sur.train(torch, net, c[:128].contiguous(), codes, epochs=40, batch=16, lr=1e-3, seed=2)
    yield dict(sfm=sfm, torch=torch, sur=sur, net=net, n=n, m=m, k=k, b=b, code=code, sigma=sigma,
               f=f, blocks=blocks, sets=sets, sets_d=sets_d, c=c, losses=losses, per_block=per_block)
    sfm.sfm_net_destroy(net)


def test_trained_surrogate_beats_the_mean_rom(trained):
    """NtD error at 16 frequencies on the 32 held-out blocks: the network's
    ROMs against the exact ones, and the decoder's mean ROM (code 0) as the
    baseline a network must beat to be worth anything."""
    t = trained
    sfm, torch, sur = t["sfm"], t["torch"], t["sur"]
    test_c = t["c"][128:].contiguous()
    exact = t["sets_d"][128:].contiguous()
    pred = sur.predict_sets(torch, t["net"], t["code"], test_c, exact, bf16=True)
    zero = torch.zeros((32, t["code"]), dtype=torch.float32, device="cuda")
    mean = exact.clone()
    sfm.sfm_net_decode(t["net"], zero.data_ptr(), 32, mean.data_ptr())
    lams = osur.frequencies(t["f"])
    e_net = sfm.sfm_ntd_error(0, 32, t["b"], t["k"], pred.data_ptr(), exact.data_ptr(), lams).max(axis=1)
    e_mean = sfm.sfm_ntd_error(0, 32, t["b"], t["k"], mean.data_ptr(), exact.data_ptr(), lams).max(axis=1)
    print(f"loss {t['losses'][0]:.3e} -> {t['losses'][-1]:.3e}; NtD error on held-out blocks: "
          f"network median {np.median(e_net):.3e} (max {e_net.max():.3e}), mean ROM median "
          f"{np.median(e_mean):.3e}")
    assert t["losses"][-1] < 0.5 * t["losses"][0]
    assert np.median(e_net) < np.median(e_mean)


def _tiled(t, idx):
    c, xc, yc, zc, order = t["sur"].tile_blocks(t["blocks"][idx])
    return c, xc, yc, zc, len(order)


def test_surrogate_build_falls_back_exactly(trained):
    """nt_tol = 0: every served subdomain fails the S(sigma) test and is
    rebuilt exactly, so the coefficients equal the plain build's bitwise;
    nt_tol = inf: every served subdomain keeps the network's ROM (level 1
    exact), and the coupled stepping of that ROM set stays stable."""
    t = trained
    sfm = t["sfm"]
    idx = np.arange(128, 136)                # eight held-out blocks, 2 x 2 x 2
    c, xc, yc, zc, nsub = _tiled(t, idx)
    msub, ksub = np.full(nsub, t["m"]), np.full(nsub, t["k"])
    h = sfm.sfm_create(0)
    try:
        sfm.sfm_set_model(h, c, 10.0, xc, yc, zc)
        sfm.sfm_build_roms(h, msub, ksub, t["sigma"])
        plain = sfm.sfm_get_coeffs(h)
        srep, _ = sfm.sfm_build_roms_surrogate(h, t["net"], msub, ksub, t["sigma"], 0.0)
        assert srep["eligible"] == nsub and srep["accepted"] == 0 and srep["fallback"] == nsub
        np.testing.assert_array_equal(sfm.sfm_get_coeffs(h), plain)
        srep, _ = sfm.sfm_build_roms_surrogate(h, t["net"], msub, ksub, t["sigma"], np.inf)
        assert srep["accepted"] == nsub
        sur_coef = sfm.sfm_get_coeffs(h)
        print(f"S(sigma) error of the network's ROMs: median {srep['sigma_err_median']:.3e}; "
              f"surrogate pass {srep['seconds_surrogate']:.3f} s for {nsub} blocks")
        lam, dtc = sfm.sfm_cfl_dt(h, 500)
        assert np.isfinite(dtc) and dtc > 0
    finally:
        sfm.sfm_destroy(h)
    assert not np.array_equal(sur_coef, plain)
