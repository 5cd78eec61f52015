"""Batched random access at full size: the 17 x 17 x 1024^2 light field
(8 planes, contrast-modulated so that blocks range from nearly empty to dense),
encoded by the oracle at threshold 4, and 10^6 uniform random requests in one
call, in the configuration the benchmark times (autotuned, replayed as a CUDA
graph).  Sampled requests are checked against the oracle one by one, the
whole output against the per-request kernel, and sampled blocks of a full
decode against the oracle.  Takes a few minutes (synthesis and the oracle's
encode dominate); set RLFC_SYNTH_CACHE to reuse the synthesised views."""
import numpy as np
import pytest
import torch

import lf_synth
import oracle

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def rl():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1805_06019_gb300 import rlfc
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return rlfc


def test_million_requests_on_the_batching_light_field(rl):
    p = lf_synth.PRESETS["batching"]
    U, V, tau = p["U"], p["V"], p["taus"][0]
    lf = lf_synth.preset_lightfield("batching")
    data = oracle.encode(lf, U, V, B=4, L=p["L"], c=p["c"], tau_p=tau, tau_b=16 * tau)
    ost, st = oracle.Stream(data), rl.Stream(data)
    n = p["n_requests"]
    pv, pl = lf_synth.random_requests(n, U * V, st.nloc, p["id"])
    views = torch.from_numpy(pv.view(np.int32)).cuda()
    locs = torch.from_numpy(pl.view(np.int32)).cuda()
    b = rl.Batch(st, n)
    out = torch.empty((n, 4, 4, 3), dtype=torch.uint8, device="cuda")
    b.config = dict(graph=0)
    b.autotune(views, locs, out)
    b.config = dict(graph=1)
    out.zero_()
    status = torch.full((n,), 9, dtype=torch.uint8, device="cuda")
    b.decode(views, locs, out, status)
    b.decode(views, locs, out, status)          # a replay of the captured graph
    assert int(status.max()) == 0
    ref, _ = st.decode_blocks(views, locs)
    assert torch.equal(out, ref)
    o = out.cpu().numpy()
    rng = np.random.default_rng(21)
    for r in rng.choice(n, 20000, replace=False).tolist():
        assert np.array_equal(o[r], ost.decode_block(int(pv[r]), int(pl[r]))), r
    # progressive: the level-1 reconstruction and the top RKV
    for level in (1, 2):
        lo, _ = b.decode(views, locs, level=level)
        lo = lo.cpu().numpy()
        for r in rng.choice(n, 3000, replace=False).tolist():
            ycc = ost.decode_block_ycc(int(pv[r]), int(pl[r]), stop_level=level)
            want = np.clip(oracle.ycocg_inv(ycc.transpose(1, 2, 0)), 0, 255).astype(np.uint8)
            assert np.array_equal(lo[r], want), (level, r)
    # full decode, sampled blocks
    full = st.decode_all().cpu().numpy()
    for _ in range(20000):
        v, l = int(rng.integers(0, U * V)), int(rng.integers(0, st.nloc))
        bx, by = l % st.nloc_x, l // st.nloc_x
        blk = full[v, 4 * by:4 * by + 4, 4 * bx:4 * bx + 4]
        assert np.array_equal(blk, ost.decode_block(v, l)), (v, l)
