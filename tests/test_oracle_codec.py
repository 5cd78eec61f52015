"""Pins of the oracle encoder/decoder (Algorithms 1-2, Eq. 2-3) against
properties the paper fixes: lossless integer coding at threshold 0, the
closed-loop error bound of the recomputed tree, the degenerate all-dropped
stream, non-increasing PSNR as the threshold grows, the binomial filter's
impulse response (scipy), random access equal to full decoding, and rejection
of corrupt streams."""
import numpy as np
import pytest
from scipy.special import comb

import lf_synth
import oracle


def _small_lf(U, V, W, H, seed=0):
    rng = np.random.default_rng(seed)
    base = rng.integers(0, 256, size=(1, H, W, 3))
    noise = rng.integers(-12, 13, size=(U * V, H, W, 3))
    return np.clip(base + noise, 0, 255).astype(np.uint8)


def _padded(lf, B):
    V_U, H, W, _ = lf.shape
    Hp, Wp = -(-H // B) * B, -(-W // B) * B
    ys = np.minimum(np.arange(Hp), H - 1)
    xs = np.minimum(np.arange(Wp), W - 1)
    return lf[:, ys][:, :, xs]


# ---- Eq. 2 filter ------------------------------------------------------------

@pytest.mark.parametrize("Gu,Gv,c", [(5, 5, 5), (9, 9, 3), (17, 1, 5), (4, 4, 2), (6, 3, 4)])
def test_filter_impulse_response_is_binomial(Gu, Gv, c):
    ku, kv = oracle.tile_count(Gu, c), oracle.tile_count(Gv, c)
    for y in range(Gv):
        for x in range(Gu):
            child = np.zeros((Gu * Gv, 1), dtype=np.int32)
            child[y * Gu + x] = 1 << 20
            out = oracle.filter_level(child, Gu, Gv, c)
            a = next(a for a in range(ku) if (a * Gu) // ku <= x < ((a + 1) * Gu) // ku)
            b = next(b for b in range(kv) if (b * Gv) // kv <= y < ((b + 1) * Gv) // kv)
            x0, x1 = (a * Gu) // ku, ((a + 1) * Gu) // ku
            y0, y1 = (b * Gv) // kv, ((b + 1) * Gv) // kv
            mu, mv = x1 - x0, y1 - y0
            w = comb(mu - 1, x - x0, exact=True) * comb(mv - 1, y - y0, exact=True)
            expect = np.zeros(ku * kv, dtype=np.int64)
            expect[b * ku + a] = (w << 20) >> ((mu - 1) + (mv - 1))
            assert np.array_equal(out[:, 0], expect), (x, y)


def test_filter_of_four_views_is_the_rounded_mean():
    # Fig. 3: level 1 filters clusters of four images
    rng = np.random.default_rng(1)
    child = rng.integers(-255, 256, size=(4, 500)).astype(np.int32)
    out = oracle.filter_level(child, 2, 2, 2)
    assert np.array_equal(out[0], np.floor_divide(child.sum(axis=0) + 2, 4))


def test_filter_keeps_constants_and_is_mirror_symmetric():
    rng = np.random.default_rng(2)
    const = np.full((25, 10), -77, dtype=np.int32)
    assert np.all(oracle.filter_level(const, 5, 5, 5) == -77)
    child = rng.integers(-255, 256, size=(25, 64)).astype(np.int32)
    mirrored = child.reshape(5, 5, 64)[::-1, ::-1].reshape(25, 64)
    transposed = child.reshape(5, 5, 64).transpose(1, 0, 2).reshape(25, 64)
    out = oracle.filter_level(child, 5, 5, 5)
    assert np.array_equal(out, oracle.filter_level(mirrored, 5, 5, 5))
    assert np.array_equal(out, oracle.filter_level(transposed, 5, 5, 5))


# ---- lossless coding (Section 4: integer computations throughout) -------------

@pytest.mark.parametrize("U,V,W,H,B,L,c", [
    (5, 5, 16, 16, 4, 2, [0, 5]),
    (6, 6, 30, 21, 4, 2, [0, 3]),          # 4 top RKVs, padded views
    (9, 9, 16, 12, 4, 3, [0, 3, 3]),
    (6, 5, 13, 9, 2, 3, [0, 2, 3]),
    (4, 4, 24, 16, 8, 3, [0, 2, 2]),
    (8, 8, 8, 8, 4, 4, [0, 2, 2, 2]),
])
def test_threshold_zero_is_lossless(U, V, W, H, B, L, c):
    lf = _small_lf(U, V, W, H, seed=U * 100 + W)
    s = oracle.encode(lf, U, V, B=B, L=L, c=c, tau_p=0, tau_b=0, q=0)
    st = oracle.Stream(s)
    assert (st.W, st.H, st.B, st.L) == (W, H, B, L)
    assert np.array_equal(st.decode_all(), lf)


def test_tiny_preset_lossless_at_zero():
    p = lf_synth.PRESETS["tiny"]
    lf = lf_synth.preset_lightfield("tiny")
    s = oracle.encode(lf, p["U"], p["V"], B=4, L=p["L"], c=p["c"])
    assert np.array_equal(oracle.Stream(s).decode_all(), lf)


# ---- closed loop: errors do not propagate down the tree (Section 3.2) ---------

@pytest.mark.parametrize("L,c,tau_p,tau_b", [
    (2, [0, 3], 3, 40), (3, [0, 2, 3], 3, 40), (3, [0, 3, 2], 6, 10), (4, [0, 2, 2, 2], 2, 100),
])
def test_error_is_bounded_by_the_last_level_threshold(L, c, tau_p, tau_b):
    U, V, W, H, B = 6, 6, 20, 12, 4
    lf = _small_lf(U, V, W, H, seed=L * 7 + tau_p)
    s = oracle.encode(lf, U, V, B=B, L=L, c=c, tau_p=tau_p, tau_b=tau_b, q=0)
    st = oracle.Stream(s)
    ycc = oracle.ycocg_fwd(_padded(lf, B)).astype(np.int64)  # [views, Hp, Wp, 3]
    dropped_blocks = 0
    for view in range(U * V):
        for loc in range(st.nloc):
            bx, by = loc % st.nlx, loc // st.nlx
            dec = st.decode_block_ycc(view, loc).astype(np.int64)  # [3, B, B]
            orig = ycc[view, by * B:(by + 1) * B, bx * B:(bx + 1) * B].transpose(2, 0, 1)
            e = np.abs(orig - dec)
            for ch in range(3):
                big = e[ch][e[ch] >= tau_p]
                if big.size:
                    # only a dropped block can leave errors >= tau_p, and its
                    # thresholded energy was below tau_b
                    assert big.sum() < tau_b, (view, loc, ch)
                    dropped_blocks += 1
    assert dropped_blocks > 0


def test_all_blocks_dropped_decodes_the_top_rkv():
    U, V, W, H, B = 5, 5, 16, 16, 4
    lf = _small_lf(U, V, W, H, seed=3)
    s = oracle.encode(lf, U, V, B=B, L=2, c=[0, 5], tau_p=10 ** 6, tau_b=10 ** 6)
    st = oracle.Stream(s)
    child = oracle.ycocg_fwd(lf).reshape(U * V, -1)
    top = oracle.filter_level(child, U, V, 5).reshape(H, W, 3)
    expect = np.clip(oracle.ycocg_inv(top), 0, 255).astype(np.uint8)
    dec = st.decode_all()
    for view in range(U * V):
        assert np.array_equal(dec[view], expect)


def test_progressive_decode_stops_at_the_filtered_level():
    # threshold 0: level 1 is reconstructed exactly, so stopping there returns
    # the level-1 RKV, i.e. the filtered views (Section 3.6)
    U, V, W, H, B = 9, 9, 8, 8, 4
    lf = _small_lf(U, V, W, H, seed=4)
    st = oracle.Stream(oracle.encode(lf, U, V, B=B, L=3, c=[0, 3, 3]))
    child = oracle.ycocg_fwd(lf).reshape(U * V, -1)
    lvl1 = oracle.filter_level(child, U, V, 3).reshape(9, H, W, 3)
    lvl2 = oracle.filter_level(lvl1.reshape(9, -1), 3, 3, 3).reshape(1, H, W, 3)
    t = oracle.tree_from_clusters(U, V, 3, [0, 3, 3])
    for view in (0, 40, 80):
        for loc in range(st.nloc):
            bx, by = loc % st.nlx, loc // st.nlx
            sl = (slice(by * B, (by + 1) * B), slice(bx * B, (bx + 1) * B))
            p = t["parent"][0][view]
            got1 = st.decode_block_ycc(view, loc, stop_level=1)
            assert np.array_equal(got1, lvl1[p][sl].transpose(2, 0, 1))
            got2 = st.decode_block_ycc(view, loc, stop_level=2)
            assert np.array_equal(got2, lvl2[0][sl].transpose(2, 0, 1))


def test_psnr_does_not_rise_with_the_threshold():
    p = lf_synth.PRESETS["tiny"]
    lf = lf_synth.preset_lightfield("tiny")
    ycc = oracle.ycocg_fwd(lf).astype(np.int64)
    prev_mse, prev_psnr, sizes = None, None, []
    for tau in [0, 1, 2, 3, 4, 6, 8, 12, 16, 32, 64]:
        s = oracle.encode(lf, p["U"], p["V"], B=4, L=2, c=p["c"], tau_p=tau, tau_b=16 * tau)
        st = oracle.Stream(s)
        # pre-clamp YCoCg error, per channel (2-level tree: the zeroed and
        # dropped sets only grow with tau, so the error can only grow)
        dec_ycc = np.zeros_like(ycc)
        for view in range(25):
            for loc in range(st.nloc):
                bx, by = loc % st.nlx, loc // st.nlx
                dec_ycc[view, by * 4:(by + 1) * 4, bx * 4:(bx + 1) * 4] = \
                    st.decode_block_ycc(view, loc).transpose(1, 2, 0)
        mse = ((ycc - dec_ycc) ** 2).mean(axis=(0, 1, 2))
        psnr = oracle.psnr_ycocg(lf, st.decode_all())
        if prev_mse is not None:
            assert np.all(mse >= prev_mse)
            assert psnr <= prev_psnr + 1e-12
        prev_mse, prev_psnr = mse, psnr
        sizes.append(len(s))
    assert sizes[-1] < sizes[0]


# ---- random access (Section 3.5) ---------------------------------------------

def test_random_access_equals_full_decode():
    p = lf_synth.PRESETS["tiny"]
    lf = lf_synth.preset_lightfield("tiny")
    st = oracle.Stream(oracle.encode(lf, 5, 5, B=4, L=2, c=p["c"], tau_p=2, tau_b=32))
    full = st.decode_all()
    rng = np.random.default_rng(5)
    for _ in range(300):
        view, loc = int(rng.integers(25)), int(rng.integers(st.nloc))
        bx, by = loc % st.nlx, loc // st.nlx
        assert np.array_equal(st.decode_block(view, loc),
                              full[view, by * 4:(by + 1) * 4, bx * 4:(bx + 1) * 4])


# ---- corrupt streams -----------------------------------------------------------

def test_corrupt_streams_are_rejected():
    lf = _small_lf(5, 5, 16, 16, seed=9)
    s = bytearray(oracle.encode(lf, 5, 5, B=4, L=2, c=[0, 5], tau_p=2, tau_b=8))
    oracle.Stream(bytes(s))
    bad = bytearray(s); bad[0] ^= 1
    with pytest.raises(ValueError):
        oracle.Stream(bytes(bad))
    with pytest.raises(ValueError):
        oracle.Stream(bytes(s[:-4]))
    off_offsets = int.from_bytes(s[48:52], "little")
    bad = bytearray(s); bad[off_offsets + 4:off_offsets + 8] = (10 ** 7).to_bytes(4, "little")
    with pytest.raises(ValueError):
        oracle.Stream(bytes(bad))


# ---- quantisation and the per-block shift ---------------------------------------

@pytest.mark.parametrize("L,c,q", [(2, [0, 3], 1), (2, [0, 3], 2), (3, [0, 2, 3], 2), (3, [0, 3, 2], 3)])
def test_quantisation_error_is_at_most_half_a_step(L, c, q):
    # round half away from zero: |r - qv 2^q| <= 2^(q-1) for every kept value, and
    # a block whose values all quantise to zero has |r| < 2^(q-1); the closed
    # loop keeps this bound at every tree height
    U, V, W, H, B = 6, 6, 12, 8, 4
    lf = _small_lf(U, V, W, H, seed=20 + q)
    st = oracle.Stream(oracle.encode(lf, U, V, B=B, L=L, c=c, tau_p=0, tau_b=0, q=q))
    ycc = oracle.ycocg_fwd(_padded(lf, B)).astype(np.int64)
    worst = 0
    for view in range(U * V):
        for loc in range(st.nloc):
            bx, by = loc % st.nlx, loc // st.nlx
            dec = st.decode_block_ycc(view, loc).astype(np.int64)
            orig = ycc[view, by * B:(by + 1) * B, bx * B:(bx + 1) * B].transpose(2, 0, 1)
            worst = max(worst, int(np.abs(orig - dec).max()))
    assert worst <= 2 ** (q - 1)
    assert worst == 2 ** (q - 1)   # the bound is reached on this data


def _first_present_header(stream: bytes):
    """(byte offset of record (loc 0, channel 0), S) and the bit position of
    the first present block's header inside that record (format v1)."""
    S = int.from_bytes(stream[40:44], "little")
    off_offsets = int.from_bytes(stream[48:52], "little")
    off_records = int.from_bytes(stream[52:56], "little")
    w0 = int.from_bytes(stream[off_offsets:off_offsets + 4], "little")
    rec = off_records + 4 * w0
    mw = (S + 31) // 32
    mask = int.from_bytes(stream[rec:rec + 4 * mw], "little")
    pos = (mask & -mask).bit_length() - 1
    return rec, 32 * mw, pos


def test_block_shift_field_scales_the_block():
    # header bits 5..6 hold a per-block extra shift s: the block contributes
    # (min + u) * 2^(q + s).  Setting s = 1 on a stored block must add exactly
    # its contribution once more.
    U, V, W, H, B = 5, 5, 8, 8, 4
    lf = _small_lf(U, V, W, H, seed=31)
    s = bytearray(oracle.encode(lf, U, V, B=B, L=2, c=[0, 5], tau_p=0, tau_b=0))
    rec, hdr_bit, pos = _first_present_header(bytes(s))
    assert pos == 0   # view 0's level-0 block of location 0 is stored
    st = oracle.Stream(bytes(s))
    base = st.decode_block_ycc(0, 0)
    contrib = base - st.decode_block_ycc(0, 0, stop_level=1)
    bit = hdr_bit + 5
    s[rec + bit // 8] |= 1 << (bit % 8)
    shifted = oracle.Stream(bytes(s)).decode_block_ycc(0, 0)
    assert np.array_equal(shifted[0], base[0] + contrib[0])
    assert np.array_equal(shifted[1:], base[1:])
