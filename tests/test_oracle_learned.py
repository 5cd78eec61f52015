"""Pins of the oracle's learned-encoder-aid pieces: the (mode, shift) search
and the encoder's use of the header's shift field, the 48 block statistics,
and the FP64 network's forward and backward passes."""
import numpy as np
import pytest

import lf_synth
import oracle


def _blocks(n, seed, scale=40):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        kind = i % 4
        if kind == 0:
            b = rng.integers(-scale, scale + 1, 16)
        elif kind == 1:
            b = 2 * rng.integers(-scale // 2, scale // 2 + 1, 16)      # all even
        elif kind == 2:
            b = 4 * rng.integers(-scale // 4, scale // 4 + 1, 16)      # multiples of 4
        else:
            b = np.round(rng.normal(0, scale / 4, 16)).astype(int)
        out.append(b.astype(np.int32))
    return out


def _quantise_np(r, t):
    # round half away from zero of r / 2^t, written with floats
    r = np.asarray(r, dtype=np.float64)
    return (np.sign(r) * np.floor(np.abs(r) / 2.0 ** t + 0.5)).astype(np.int64)


def test_quantiser_matches_round_half_away_from_zero():
    rng = np.random.default_rng(1)
    for t in range(0, 6):
        r = rng.integers(-700, 701, 64)
        got = oracle.ks_quantise(r, q=t, s=0)
        assert np.array_equal(got, _quantise_np(r, t))
        assert np.array_equal(oracle.ks_quantise(r, q=max(t - 1, 0), s=min(t, 1)), _quantise_np(r, t))


def test_zero_error_budget_is_the_plain_method_unless_a_shift_is_exact():
    for r in _blocks(400, seed=2):
        k, s = oracle.ks_search(r, q=0, tau_err=0, lam_q8=256)
        if np.any(r % 2 != 0):
            # no exact shift: the plain method's cheapest range
            assert s == 0 and k == oracle.choose_mode(16, int(r.max() - r.min()))
        else:
            assert s >= 1
            assert np.all(r % (1 << s) == 0)


def test_search_without_distortion_weight_takes_the_largest_allowed_shift():
    # with lam = 0 only the bits count, and a larger shift never widens the
    # range: the result is the largest shift within the error budget, with the
    # cheapest range for its quantised values
    for tau in (1, 2, 4, 8):
        for r in _blocks(200, seed=3 + tau):
            k, s = oracle.ks_search(r, q=0, tau_err=tau, lam_q8=0)
            best_s = 0
            for t in range(1, 4):
                qv = _quantise_np(r, t)
                if np.abs(r - qv * 2 ** t).max() <= tau:
                    best_s = t
            qv = _quantise_np(r, best_s)
            want_k = oracle.choose_mode(16, int(qv.max() - qv.min()))
            bits = oracle.bise_bits(16, want_k)
            assert oracle.bise_bits(16, k) == bits
            if s != best_s:
                # only a tie in bits may pick a smaller shift
                assert s < best_s


def test_search_result_is_never_worse_than_the_plain_choice():
    for lam in (0, 64, 256, 1024, 10 ** 6):
        for r in _blocks(200, seed=10 + lam % 97):
            k, s = oracle.ks_search(r, q=0, tau_err=4, lam_q8=lam)
            plain = oracle.ks_cost(r, 0, 0, oracle.choose_mode(16, int(r.max() - r.min())), 4, lam)
            assert oracle.ks_cost(r, 0, s, k, 4, lam) <= plain
            # the range is the smallest that holds the quantised span
            qv = _quantise_np(r, s)
            assert k == oracle.choose_mode(16, int(qv.max() - qv.min()))
            if lam == 10 ** 6:
                assert s == 0 or np.all(qv * 2 ** s == r)


def _small_lf(seed):
    return lf_synth.make_lightfield(5, 5, 24, 20, [0.0, 0.9], 1.0, preset_id=600 + seed)


def test_exact_shifts_keep_a_lossless_encode_lossless():
    lf = _small_lf(1)
    plain = oracle.encode(lf, 5, 5, B=4, L=3, c=[0, 2, 3])
    ks = oracle.encode(lf, 5, 5, B=4, L=3, c=[0, 2, 3], mode_space=1, tau_err=0, lam_q8=256)
    assert np.array_equal(oracle.Stream(ks).decode_all(), lf)
    assert len(ks) <= len(plain)


def test_leaf_error_stays_within_the_budget_and_bits_drop():
    # closed loop: every level is re-coded against the parent's reconstruction,
    # so only the leaves' own shifts remain, each within tau_err
    lf = _small_lf(2)
    ycc = oracle.ycocg_fwd(lf)
    for tau in (1, 2, 4):
        data = oracle.encode(lf, 5, 5, B=4, L=3, c=[0, 2, 3], mode_space=1, tau_err=tau, lam_q8=64)
        st = oracle.Stream(data)
        worst = 0
        for view in range(25):
            for loc in range(st.nloc):
                bx, by = loc % st.nlx, loc // st.nlx
                got = st.decode_block_ycc(view, loc).transpose(1, 2, 0)
                want = ycc[view, by * 4:by * 4 + 4, bx * 4:bx * 4 + 4]
                worst = max(worst, int(np.abs(got - want).max()))
        assert worst <= tau
        assert len(data) < len(oracle.encode(lf, 5, 5, B=4, L=3, c=[0, 2, 3]))


def test_given_leaf_modes_are_used_and_infeasible_ones_fall_back():
    lf = _small_lf(3)
    U = V = 5
    out = {}
    ref = oracle.encode(lf, U, V, B=4, L=3, c=[0, 2, 3], mode_space=1, tau_err=2, lam_q8=128, leaf_out=out)
    # the search's own labels as given modes reproduce the search's stream
    same = oracle.encode(lf, U, V, B=4, L=3, c=[0, 2, 3], mode_space=1, tau_err=2, lam_q8=128,
                         leaf_modes=out["label"])
    assert same == ref
    # mode 0 (one value) with no shift is infeasible wherever a block varies:
    # those fall back to the search; the stream still decodes within budget
    bad = np.where(out["label"] == 0xFF, 0xFF, 0).astype(np.uint8)
    fb = oracle.encode(lf, U, V, B=4, L=3, c=[0, 2, 3], mode_space=1, tau_err=2, lam_q8=128, leaf_modes=bad)
    assert fb == ref
    # all-0xFF means "search" everywhere
    assert oracle.encode(lf, U, V, B=4, L=3, c=[0, 2, 3], mode_space=1, tau_err=2, lam_q8=128,
                         leaf_modes=np.full_like(out["label"], 0xFF)) == ref


def test_leaf_dataset_matches_the_encoder_residuals():
    lf = _small_lf(4)
    out = {}
    oracle.encode(lf, 5, 5, B=4, L=2, c=[0, 5], tau_p=2, tau_b=16, mode_space=0, tau_err=3, lam_q8=128,
                  leaf_out=out)
    lab, res = out["label"], out["resid"]
    kept = lab != 0xFF
    assert kept.any() and (~kept).any()
    # labels are the search result of the stored residuals; dropped blocks
    # carry energy below the threshold
    idx = np.argwhere(kept)
    for (v, c, l) in idx[:: max(1, len(idx) // 200)]:
        k, s = oracle.ks_search(res[v, c, l], 0, 3, 128)
        assert lab[v, c, l] == (k | s << 5)
    for (v, c, l) in np.argwhere(~kept)[:200]:
        assert np.abs(res[v, c, l]).sum() < 16
        assert np.all((res[v, c, l] == 0) | (np.abs(res[v, c, l]) >= 2))


def test_block_statistics_match_numpy():
    for r in _blocks(100, seed=20, scale=300):
        f = oracle.ks_features(r)
        rd = r.astype(np.float64)
        a = np.abs(r)
        want = np.concatenate([np.sort(rd) / 32, rd / 32, [
            rd.mean() / 32, rd.std() / 32, rd.min() / 32, rd.max() / 32, (rd.max() - rd.min()) / 64,
            a.max() / 32, a.sum() / 256, np.count_nonzero(r) / 16, np.count_nonzero(a % 2) / 16,
            np.count_nonzero(a % 4 == 2) / 16, np.count_nonzero(a % 8 == 4) / 16,
            np.count_nonzero(a <= 1) / 16, np.count_nonzero(a <= 2) / 16, np.count_nonzero(a <= 4) / 16,
            np.count_nonzero(a <= 8) / 16, np.log2(rd.max() - rd.min() + 1) / 10]])
        assert np.allclose(f, want, rtol=1e-12, atol=1e-12)


def _params(seed, scale=0.2):
    rng = np.random.default_rng(seed)
    return rng.normal(0, scale, oracle.mlp_nparams())


def _split(w):
    s = [64 * 48, 64, 64 * 64, 64, 112 * 64, 112]
    o = np.cumsum([0] + s)
    W1, b1, W2, b2, W3, b3 = (w[o[i]:o[i + 1]] for i in range(6))
    return W1.reshape(64, 48), b1, W2.reshape(64, 64), b2, W3.reshape(112, 64), b3


def test_network_forward_matches_numpy_and_uniform_loss():
    w = _params(1)
    x = np.random.default_rng(2).normal(0, 1, (37, 48))
    W1, b1, W2, b2, W3, b3 = _split(w)
    h1 = np.maximum(x @ W1.T + b1, 0)
    h2 = np.maximum(h1 @ W2.T + b2, 0)
    assert np.allclose(oracle.mlp_forward(w, x), h2 @ W3.T + b3, rtol=1e-12, atol=1e-12)
    # zero weights: uniform softmax over the 112 classes
    y = np.arange(37) % 112
    loss, g = oracle.mlp_loss_grad(np.zeros_like(w), x, y)
    assert loss == pytest.approx(37 * np.log(112.0), rel=1e-12)
    # cross-entropy against numpy's log-softmax
    z = oracle.mlp_forward(w, x)
    lse = np.log(np.exp(z - z.max(1, keepdims=True)).sum(1)) + z.max(1)
    loss, _ = oracle.mlp_loss_grad(w, x, y)
    assert loss == pytest.approx(float(np.sum(lse - z[np.arange(37), y])), rel=1e-12)


def test_network_gradient_matches_central_differences():
    w = _params(3)
    rng = np.random.default_rng(4)
    x = rng.normal(0, 1, (6, 48))
    y = rng.integers(0, 112, 6)
    _, g = oracle.mlp_loss_grad(w, x, y)
    idx = rng.choice(w.size, 300, replace=False)
    idx = np.concatenate([idx, [0, 64 * 48, 64 * 48 + 64, w.size - 1]])
    h = 1e-6
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        num = (oracle.mlp_loss_grad(wp, x, y)[0] - oracle.mlp_loss_grad(wm, x, y)[0]) / (2 * h)
        assert abs(num - g[i]) <= 1e-6 * max(1.0, abs(num)), i
