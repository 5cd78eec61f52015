"""Batched random access and progressive decode through the C ABI
(rlfc_batch_*), against the CPU oracle.

Every configuration of the persistent binned kernel (warps per CTA, locations
per queue pop, staging, graph replay) must return the oracle's bytes for every
request, the same bytes as the per-request kernel, and the oracle's
progressive (filtered) value at every stop level.  Streams are written by the
oracle's encoder from the seeded synthetic light fields of lf_synth.
"""
import itertools

import numpy as np
import pytest
import torch

import lf_synth
import oracle

pytestmark = pytest.mark.gpu

E_INVALID_ARG, E_RANGE = 1, 6


@pytest.fixture(scope="module")
def rl():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1805_06019_gb300 import rlfc
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return rlfc


# (name, U, V, W, H, L, c, tau_p, tau_b, q)
CASES = [
    ("two_levels", 5, 5, 64, 64, 2, [0, 5], 2, 32, 0),
    ("odd_sizes_3lvl", 6, 5, 30, 21, 3, [0, 2, 3], 3, 40, 0),
    ("four_levels", 8, 8, 24, 24, 4, [0, 2, 2, 2], 2, 24, 0),
    ("four_tops", 6, 6, 32, 32, 2, [0, 3], 1, 8, 0),
    ("quantised", 5, 5, 20, 16, 3, [0, 2, 3], 0, 0, 2),
    ("lossless", 9, 9, 32, 32, 3, [0, 3, 3], 0, 0, 0),
    ("all_dropped", 4, 4, 16, 16, 2, [0, 4], 10 ** 5, 10 ** 5, 0),
]

_cache = {}


def _case(name):
    if name not in _cache:
        _, U, V, W, H, L, c, tp, tb, q = next(x for x in CASES if x[0] == name)
        lf = lf_synth.make_lightfield(U, V, W, H, [0.0, 0.7, 1.6], 1.0, preset_id=400 + len(_cache))
        _cache[name] = oracle.encode(lf, U, V, B=4, L=L, c=c, tau_p=tp, tau_b=tb, q=q)
    return _cache[name]


def _requests(n_views, nloc, n, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(0, n_views, n).astype(np.int32), rng.integers(0, nloc, n).astype(np.int32)


def _expected(ost, views, locs, level=0):
    out = np.empty((len(views), 4, 4, 3), dtype=np.uint8)
    for r, (v, l) in enumerate(zip(views.tolist(), locs.tolist())):
        if level == 0:
            out[r] = ost.decode_block(v, l)
        else:
            ycc = ost.decode_block_ycc(v, l, stop_level=level)          # [3, 4, 4]
            out[r] = np.clip(oracle.ycocg_inv(ycc.transpose(1, 2, 0)), 0, 255).astype(np.uint8)
    return out


CONFIGS = [dict(warps_per_cta=w, locs_per_pop=p, stage=s, graph=g)
           for w, p, s, g in itertools.product((4, 8, 16), (1, 4), (0, 1, 2), (0, 1))]


@pytest.mark.parametrize("name", [c[0] for c in CASES])
def test_every_configuration_matches_the_oracle(rl, name):
    data = _case(name)
    ost, st = oracle.Stream(data), rl.Stream(data)
    n = 3000
    pv, pl = _requests(st.n_views, st.nloc, n, seed=11)
    want = _expected(ost, pv, pl)
    views, locs = torch.from_numpy(pv).cuda(), torch.from_numpy(pl).cuda()
    per_request, _ = st.decode_blocks(views, locs)
    assert np.array_equal(per_request.cpu().numpy(), want)
    b = rl.Batch(st, n)
    out = torch.empty((n, 4, 4, 3), dtype=torch.uint8, device="cuda")
    status = torch.empty(n, dtype=torch.uint8, device="cuda")
    for cfg in CONFIGS:
        b.config = cfg
        out.fill_(123)
        status.fill_(9)
        b.decode(views, locs, out, status)
        assert np.array_equal(out.cpu().numpy(), want), cfg
        assert int(status.max()) == 0


@pytest.mark.parametrize("name", ["odd_sizes_3lvl", "four_levels", "quantised", "four_tops"])
def test_progressive_levels_match_the_oracle(rl, name):
    data = _case(name)
    ost, st = oracle.Stream(data), rl.Stream(data)
    n = 1500
    pv, pl = _requests(st.n_views, st.nloc, n, seed=12)
    views, locs = torch.from_numpy(pv).cuda(), torch.from_numpy(pl).cuda()
    b = rl.Batch(st, n)
    for graph in (0, 1):
        b.config = dict(graph=graph)
        for level in range(st.L):
            out, _ = b.decode(views, locs, level=level)
            assert np.array_equal(out.cpu().numpy(), _expected(ost, pv, pl, level)), (graph, level)


def test_crowded_locations_and_bad_requests(rl):
    data = _case("odd_sizes_3lvl")
    ost, st = oracle.Stream(data), rl.Stream(data)
    # 700 requests on two locations (bins far larger than one round of slots),
    # interleaved with out-of-range requests
    rng = np.random.default_rng(13)
    pv = rng.integers(0, st.n_views, 700).astype(np.int64)
    pl = np.where(rng.random(700) < 0.5, 0, st.nloc - 1).astype(np.int64)
    pv[::7] = st.n_views + np.arange(len(pv[::7]))
    pl[3::11] = st.nloc
    pl[5::13] = 2 ** 32 - 1
    views = torch.tensor(pv, dtype=torch.int64).to(torch.uint32).cuda()
    locs = torch.tensor(pl, dtype=torch.int64).to(torch.uint32).cuda()
    ref_out, ref_status = st.decode_blocks(views, locs)
    b = rl.Batch(st, 1000)
    for cfg in ({"graph": 0}, {"graph": 1, "warps_per_cta": 16, "locs_per_pop": 4, "stage": 1},
                {"graph": 1, "warps_per_cta": 8, "locs_per_pop": 1, "stage": 2}):
        b.config = cfg
        out = torch.full((700, 4, 4, 3), 77, dtype=torch.uint8, device="cuda")
        status = torch.full((700,), 9, dtype=torch.uint8, device="cuda")
        b.decode(views, locs, out, status)
        s = status.cpu().numpy()
        o = out.cpu().numpy()
        assert np.array_equal(s, ref_status.cpu().numpy())
        assert np.array_equal(o, ref_out.cpu().numpy())
        for r in range(700):
            if s[r] == 0:
                assert np.array_equal(o[r], ost.decode_block(int(pv[r]), int(pl[r])))
            else:
                assert s[r] == (1 if pv[r] >= st.n_views else 2) and not o[r].any()


def test_unaligned_output_graph_replay_and_limits(rl):
    data = _case("four_levels")
    ost, st = oracle.Stream(data), rl.Stream(data)
    n = 257
    pv, pl = _requests(st.n_views, st.nloc, n, seed=14)
    views, locs = torch.from_numpy(pv).cuda(), torch.from_numpy(pl).cuda()
    b = rl.Batch(st, n)
    buf = torch.zeros(n * 48 + 1, dtype=torch.uint8, device="cuda")
    out = buf[1:].view(n, 4, 4, 3)
    for graph in (0, 1):
        b.config = dict(graph=graph)
        out.zero_()
        b.decode(views, locs, out)
        assert np.array_equal(out.cpu().numpy(), _expected(ost, pv, pl)), graph
    # replaying the captured graph reads the arguments' current contents
    b.config = dict(graph=1)
    out2 = torch.empty((n, 4, 4, 3), dtype=torch.uint8, device="cuda")
    b.decode(views, locs, out2)
    pv2, pl2 = _requests(st.n_views, st.nloc, n, seed=15)
    views.copy_(torch.from_numpy(pv2))
    locs.copy_(torch.from_numpy(pl2))
    b.decode(views, locs, out2)
    assert np.array_equal(out2.cpu().numpy(), _expected(ost, pv2, pl2))
    # empty batch, too many requests, bad level
    e, _ = b.decode(views[:0], locs[:0])
    assert e.numel() == 0
    big = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    with pytest.raises(rl.RLFCError) as ei:
        b.decode(big, big)
    assert ei.value.code == E_RANGE
    with pytest.raises(rl.RLFCError) as ei:
        b.decode(views, locs, level=st.L)
    assert ei.value.code == E_INVALID_ARG
    with pytest.raises(rl.RLFCError) as ei:
        b.config = dict(warps_per_cta=5)
    assert ei.value.code == E_INVALID_ARG


def test_autotune_keeps_a_valid_configuration(rl):
    data = _case("lossless")
    ost, st = oracle.Stream(data), rl.Stream(data)
    n = 20000
    pv, pl = _requests(st.n_views, st.nloc, n, seed=16)
    views, locs = torch.from_numpy(pv).cuda(), torch.from_numpy(pl).cuda()
    b = rl.Batch(st, n)
    out = torch.empty((n, 4, 4, 3), dtype=torch.uint8, device="cuda")
    cfg = b.autotune(views, locs, out)
    assert cfg["warps_per_cta"] in (4, 8, 16) and cfg["locs_per_pop"] in (1, 4) and cfg["stage"] in (0, 1, 2)
    assert cfg == b.config
    want = _expected(ost, pv[:4000], pl[:4000])
    assert np.array_equal(out.cpu().numpy()[:4000], want)
    out.zero_()
    b.decode(views, locs, out)
    assert np.array_equal(out.cpu().numpy()[:4000], want)
