"""The learned encoder aid's kernels through the C ABI, against the CPU
oracle: the (shift, mode) search and the block statistics, the encoder's
per-block modes and training-data outputs, the network's gradients (FP32 on
BF16 inputs against the FP64 oracle), Adam, inference, and what a trained
network gains over the plain method."""
import numpy as np
import pytest
import torch

import lf_synth
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rl():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1805_06019_gb300 import learned, rlfc
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return rlfc, learned


def to_bf16_bits(x):
    """Round to the nearest BF16 (ties to even): uint16 bit patterns."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    return ((b + 0x7FFF + ((b >> 16) & 1)) >> 16).astype(np.uint16)


def bf16_value(bits):
    return (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def _blocks(n, seed):
    rng = np.random.default_rng(seed)
    out = np.empty((n, 16), dtype=np.int16)
    for i in range(n):
        sc = [3, 12, 60, 400][i % 4]
        v = rng.integers(-sc, sc + 1, 16)
        if i % 5 == 1:
            v = 2 * (v // 2)
        if i % 7 == 3:
            v[:] = v[0]
        out[i] = v
    return out


@pytest.mark.parametrize("q,tau_err,lam", [(0, 4, 256), (0, 1, 64), (1, 3, 1024), (0, 0, 0), (2, 8, 16)])
def test_search_matches_the_oracle(rl, q, tau_err, lam):
    _, learned = rl
    blocks = _blocks(3000, seed=q * 7 + tau_err)
    got = learned.search(torch.from_numpy(blocks).cuda(), q, tau_err, lam).cpu().numpy()
    for i, b in enumerate(blocks):
        r = oracle.ks_search(b, q, tau_err, lam)
        assert got[i] == (0xFF if r is None else (r[0] | r[1] << 5)), (i, b)


def test_statistics_match_the_oracle(rl):
    _, learned = rl
    blocks = _blocks(2000, seed=5)
    x, _ = learned.features(torch.from_numpy(blocks).cuda(), None, None, len(blocks))
    got = x.view(torch.int16).cpu().numpy().view(np.uint16)
    want = to_bf16_bits(np.stack([oracle.ks_features(b) for b in blocks]))
    diff = np.abs(got.astype(np.int32) - want.astype(np.int32))
    # exact except where FP32 and FP64 straddle a BF16 rounding boundary
    # (standard deviation and log2): one unit in the last place at most
    assert diff.max() <= 1
    assert np.all(diff[:, [i for i in range(48) if i not in (33, 47)]] == 0)


def test_compaction_keeps_order(rl):
    rlfc, learned = rl
    rng = np.random.default_rng(6)
    lab = rng.integers(0, 256, 100003).astype(np.uint8)
    lab[rng.random(lab.size) < 0.6] = 0xFF
    idx, n = learned.compact(torch.from_numpy(lab).cuda())
    assert np.array_equal(idx.cpu().numpy(), np.nonzero(lab != 0xFF)[0])


# (U, V, W, H, L, c, tau_p, tau_b, q, tau_err, lam_q8)
ENC = [
    (5, 5, 40, 24, 3, [0, 2, 3], 2, 32, 0, 4, 256),
    (6, 5, 30, 21, 2, [0, 3], 0, 0, 0, 2, 64),
    (4, 4, 16, 16, 3, [0, 2, 2], 1, 8, 1, 3, 512),
]


@pytest.mark.parametrize("case", range(len(ENC)))
def test_encoder_modes_and_dataset_match_the_oracle(rl, case):
    rlfc, learned = rl
    U, V, W, H, L, c, tp, tb, q, te, lam = ENC[case]
    lf = lf_synth.make_lightfield(U, V, W, H, [0.0, 0.8, 1.7], 1.0, preset_id=800 + case)
    d = torch.from_numpy(lf).cuda()
    out = {}
    want = oracle.encode(lf, U, V, B=4, L=L, c=c, tau_p=tp, tau_b=tb, q=q, mode_space=1, tau_err=te,
                         lam_q8=lam, leaf_out=out)
    got, resid, label, index, n = learned.leaf_dataset(d, U, V, L, c, tp, tb, q, te, lam)
    assert got == want
    nloc = ((W + 3) // 4) * ((H + 3) // 4)
    assert np.array_equal(resid.cpu().numpy(), out["resid"].reshape(-1, 16))
    assert np.array_equal(label.cpu().numpy(), out["label"].reshape(-1))
    # given level-0 modes, feasible or not, with the search as fallback
    rng = np.random.default_rng(case)
    modes = rng.integers(0, 128, U * V * 3 * nloc).astype(np.uint8)
    modes[rng.random(modes.size) < 0.2] = 0xFF
    want2 = oracle.encode(lf, U, V, B=4, L=L, c=c, tau_p=tp, tau_b=tb, q=q, mode_space=1, tau_err=te,
                          lam_q8=lam, leaf_modes=modes)
    got2 = rlfc.encode(d, U, V, L, c, tau_p=tp, tau_b=tb, q=q, mode_space=1, tau_err=te, lam_q8=lam,
                       leaf_modes=torch.from_numpy(modes).cuda())
    assert got2 == want2
    # the GPU decoder reads the shift field: bit-exact to the oracle's decode
    for data in (got, got2):
        assert np.array_equal(rlfc.Stream(data).decode_all().cpu().numpy(), oracle.Stream(data).decode_all())


def _net_inputs(seed, n=96):
    rng = np.random.default_rng(seed)
    wb = to_bf16_bits(rng.normal(0, 0.15, oracle.mlp_nparams()))
    xb = to_bf16_bits(rng.normal(0, 1.0, (n, 48)))
    y = rng.integers(0, 112, n)
    labels = ((y % 28) | ((y // 28) << 5)).astype(np.uint8)
    return wb, xb, y, labels


def _dev_bf16(bits):
    return torch.from_numpy(bits.view(np.int16)).cuda().view(torch.bfloat16)


def test_gradients_match_the_fp64_oracle(rl):
    _, learned = rl
    wb, xb, y, labels = _net_inputs(7)
    labels[5] = 0x1F            # mode 31 does not exist: the sample is skipped
    keep = np.ones(len(y), bool)
    keep[5] = False
    aid = learned.Aid()
    aid.w = _dev_bf16(wb)
    aid.grad.zero_()
    aid.loss.zero_()
    aid.loss_grad(_dev_bf16(xb), torch.from_numpy(labels).cuda())
    g = aid.grad.cpu().numpy().astype(np.float64)
    loss = float(aid.loss.item())
    ref_loss, ref = oracle.mlp_loss_grad(bf16_value(wb), bf16_value(xb)[keep], y[keep])
    assert loss == pytest.approx(ref_loss, rel=1e-5)
    assert np.abs(g - ref).max() <= 1e-4 * np.abs(ref).max() + 1e-6
    # a permuted subset through the order argument
    order = np.array([3, 17, 40, 2, 95, 64], dtype=np.int32)
    aid.grad.zero_()
    aid.loss.zero_()
    aid.loss_grad(_dev_bf16(xb), torch.from_numpy(labels).cuda(), torch.from_numpy(order).cuda(), len(order))
    _, ref2 = oracle.mlp_loss_grad(bf16_value(wb), bf16_value(xb)[order], y[order])
    assert np.abs(aid.grad.cpu().numpy() - ref2).max() <= 1e-4 * np.abs(ref2).max() + 1e-6


def test_adam_and_prediction(rl):
    _, learned = rl
    wb, xb, y, labels = _net_inputs(8, n=200)
    aid = learned.Aid(seed=3)
    master0 = aid.master.cpu().numpy().copy()
    grad = np.random.default_rng(9).normal(0, 1, master0.size).astype(np.float32)
    aid.grad.copy_(torch.from_numpy(grad))
    aid.adam(lr=1e-2, scale=0.5)
    # Adam, first step, in plain float32 numpy
    g = grad * np.float32(0.5)
    m = np.float32(0.1) * g
    v = np.float32(0.001) * g * g
    want = master0 - np.float32(1e-2) * (m / np.float32(0.1)) / (np.sqrt(v / np.float32(0.001)) + np.float32(1e-8))
    assert np.allclose(aid.master.cpu().numpy(), want, rtol=1e-5, atol=1e-6)
    assert np.array_equal(aid.w.view(torch.int16).cpu().numpy().view(np.uint16),
                          to_bf16_bits(aid.master.cpu().numpy()))
    assert not aid.grad.any()
    # inference: the oracle's argmax wherever the top two logits are apart
    aid.w = _dev_bf16(wb)
    pred = aid.predict(_dev_bf16(xb)).cpu().numpy()
    z = oracle.mlp_forward(bf16_value(wb), bf16_value(xb))
    top2 = np.sort(z, axis=1)[:, -2:]
    clear = top2[:, 1] - top2[:, 0] > 1e-3
    arg = z.argmax(1)
    assert clear.sum() > 150
    assert np.array_equal(pred[clear], ((arg % 28) | ((arg // 28) << 5)).astype(np.uint8)[clear])


def test_trained_network_gains_over_the_plain_method(rl):
    rlfc, learned = rl
    U, V, W, H, L, c = 9, 9, 96, 64, 3, [0, 3, 3]
    tau = 4
    lf = lf_synth.make_lightfield(U, V, W, H, [-0.8, 0.0, 0.7], 2.0, preset_id=900)
    d = torch.from_numpy(lf).cuda()
    plain = rlfc.encode(d, U, V, L, c, tau_p=tau, tau_b=16 * tau)
    searched, resid, label, index, n = learned.leaf_dataset(d, U, V, L, c, tau, 16 * tau, 0, tau, 256)
    x, y = learned.features(resid, label, index, n)
    split = int(0.8 * n)
    aid = learned.Aid(seed=1)
    hist = aid.train(x[:split], y[:split], epochs=6, batch=1024, lr=3e-3)
    assert hist[-1] < 0.8 * hist[0]
    pred = aid.predict(x[split:]).cpu().numpy()
    truth = y[split:].cpu().numpy()
    agree = float(np.mean(pred == truth))
    majority = float(np.bincount(y[:split].cpu().numpy(), minlength=256).max()) / split
    assert agree > majority + 0.05, (agree, majority)
    aided = learned.encode_aided(d, U, V, L, c, tau, 16 * tau, aid, x, index, resid.shape[0], 0, tau, 256)
    # an ordinary stream: the GPU decoder matches the oracle bit for bit
    dec = rlfc.Stream(aided).decode_all().cpu().numpy()
    assert np.array_equal(dec, oracle.Stream(aided).decode_all())
    # the gain over the method without the aid: fewer bits, bounded loss
    p_plain = learned.psnr_ycocg(lf, oracle.Stream(plain).decode_all())
    p_aided = learned.psnr_ycocg(lf, dec)
    assert len(aided) < 0.97 * len(plain)
    assert p_aided > p_plain - 3.0
    # every level-0 value stays within the search's error budget of the
    # value the plain method would have stored: not more than the search
    assert len(aided) <= 1.03 * len(searched)
