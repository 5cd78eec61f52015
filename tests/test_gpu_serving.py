"""Serving runtime through the C ABI (rlfc_server_*): several resident light
fields, requests batched as they arrive over several CUDA streams under a
device-memory budget.  Each result must be bit-identical to the same request
served alone, and within the renderer's tolerance of the FP64 oracle."""
import time

import numpy as np
import pytest
import torch

import lf_synth
import oracle

pytestmark = pytest.mark.gpu

E_RANGE = 6

# (U, V, W, H, L, c, tau): streams written by the oracle's encoder
FLEET = [
    (5, 5, 64, 48, 3, [0, 2, 3], 2),
    (6, 5, 40, 40, 2, [0, 3], 4),
    (9, 9, 32, 32, 3, [0, 3, 3], 1),
]


@pytest.fixture(scope="module")
def fleet():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1805_06019_gb300 import rlfc
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    lfs = []
    for i, (U, V, W, H, L, c, tau) in enumerate(FLEET):
        lf = lf_synth.make_lightfield(U, V, W, H, [0.0, 0.6, 1.4], 1.0, preset_id=500 + i)
        data = oracle.encode(lf, U, V, B=4, L=L, c=c, tau_p=tau, tau_b=16 * tau)
        lfs.append((rlfc.Stream(data), oracle.Stream(data).decode_all(), (U, V, W, H)))
    return rlfc, lfs


def _requests(lfs, n, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for _ in range(n):
        k = int(rng.integers(0, len(lfs)))
        U, V, W, H = lfs[k][2]
        # native size mostly, some rescaled views (another kernel path)
        w, h = (W, H) if rng.random() < 0.7 else (W + 8, H - 4)
        reqs.append((k, float(rng.random() * (U - 1)), float(rng.random() * (V - 1)),
                     float(rng.choice([0.0, 0.6, 1.4])), w, h))
    return reqs


def _serve(rl, lfs, reqs, gaps=None, **cfg):
    srv = rl.Server(**cfg)
    ids = [srv.add(s) for s, _, _ in lfs]
    outs = [torch.empty((h, w, 3), dtype=torch.float32).pin_memory() for (_, _, _, _, w, h) in reqs]
    comps = []
    for i, (k, u, v, d, w, h) in enumerate(reqs):
        if gaps is None:
            srv.submit(ids[k], u, v, d, outs[i])
            comps += srv.poll(wait=True)          # alone: nothing else in flight
        else:
            srv.submit(ids[k], u, v, d, outs[i])
            time.sleep(gaps[i])
    comps += srv.poll(wait=True)
    srv.close()
    return outs, comps


def test_each_result_is_the_same_alone_and_in_the_mix(fleet):
    rl, lfs = fleet
    reqs = _requests(lfs, 96, seed=31)
    alone, comps_alone = _serve(rl, lfs, reqs, n_streams=1, max_batch=1, memory_budget=1 << 26)
    assert all(c["batch"] == 1 and c["status"] == 0 for c in comps_alone)
    # a burst of 48 requests, then Poisson arrivals at ~20k requests/s; a
    # budget of a few views and three streams: requests wait for memory and
    # for a free stream, share calls and overlap
    gaps = np.diff(np.concatenate([[0.0], lf_synth.poisson_arrivals(20000.0, len(reqs), preset_id=31)]))
    gaps[:48] = 0.0
    budget = 6 * (72 * 44 * 12 + 12)
    mixed, comps = _serve(rl, lfs, reqs, gaps=gaps, n_streams=3, max_batch=8, memory_budget=budget)
    assert len(comps) == len(reqs) and all(c["status"] == 0 for c in comps)
    assert sorted(c["ticket"] for c in comps) == list(range(1, len(reqs) + 1))
    for a, b in zip(alone, mixed):
        assert torch.equal(a, b)
    for c in comps:
        assert c["t_submit"] <= c["t_start"] <= c["t_done"]
    # against the FP64 oracle
    for i in range(0, len(reqs), 7):
        k, u, v, d, w, h = reqs[i]
        U, V, _, _ = lfs[k][2]
        want = oracle.render_view(lfs[k][1], U, V, u, v, d, w, h)
        assert np.abs(mixed[i].numpy() - want).max() <= 1e-3


def test_a_burst_shares_calls_that_overlap_on_two_streams(fleet):
    # 200 same-size requests for one light field at once: while both streams
    # hold a call, the rest queue in the server and leave together
    rl, _ = fleet
    U, V, W, H = 5, 5, 128, 128
    lf = lf_synth.make_lightfield(U, V, W, H, [0.0, 0.6, 1.4], 1.0, preset_id=510)
    data = oracle.encode(lf, U, V, B=4, L=3, c=[0, 2, 3], tau_p=2, tau_b=32)
    st = rl.Stream(data)
    rng = np.random.default_rng(33)
    cams = [(float(rng.random() * 4), float(rng.random() * 4), float(rng.choice([0.0, 0.6, 1.4])))
            for _ in range(200)]
    srv = rl.Server(n_streams=2, max_batch=64, memory_budget=1 << 28, max_inflight=1)
    lf_id = srv.add(st)
    outs = [torch.empty((H, W, 3), dtype=torch.float32).pin_memory() for _ in cams]
    for (u, v, d), o in zip(cams, outs):
        srv.submit(lf_id, u, v, d, o)
    comps = srv.poll(wait=True)
    srv.close()
    assert len(comps) == 200 and all(c["status"] == 0 for c in comps)
    assert max(c["batch"] for c in comps) > 1, "no request shared a call"
    calls = sorted({(c["t_start"], c["t_done"]) for c in comps})
    assert any(b[0] < a[1] for a, b in zip(calls, calls[1:])), "no two calls were in flight together"
    # each view equals the same request rendered on its own
    uv = torch.tensor([[u, v] for u, v, _ in cams], dtype=torch.float32, device="cuda")
    disp = torch.tensor([d for _, _, d in cams], dtype=torch.float32, device="cuda")
    for i in (0, 57, 199):
        alone = st.render(uv[i:i + 1], disp[i:i + 1], W, H).cpu()
        assert torch.equal(alone[0], outs[i])


def test_admission_limits(fleet):
    rl, lfs = fleet
    srv = rl.Server(n_streams=2, max_batch=4, memory_budget=64 * 48 * 12 + 12)
    lf = srv.add(lfs[0][0])
    big = torch.empty((48, 65, 3), dtype=torch.float32)
    with pytest.raises(rl.RLFCError) as ei:
        srv.submit(lf, 1.0, 1.0, 0.0, big)
    assert ei.value.code == E_RANGE
    with pytest.raises(rl.RLFCError):
        srv.submit(lf + 5, 1.0, 1.0, 0.0, torch.empty((48, 64, 3), dtype=torch.float32))
    # one view fits at a time: every request still completes, one per call
    outs = [torch.empty((48, 64, 3), dtype=torch.float32) for _ in range(10)]
    for i, o in enumerate(outs):
        srv.submit(lf, 0.3 * i, 0.4 * i, 0.6, o)
    comps = srv.poll(wait=True)
    assert len(comps) == 10 and all(c["batch"] == 1 for c in comps)
    srv.close()
    for i, o in enumerate(outs):
        want = oracle.render_view(lfs[0][1], 5, 5, 0.3 * i, 0.4 * i, 0.6, 64, 48)
        assert np.abs(o.numpy() - want).max() <= 1e-3


def test_8bit_and_float_requests_in_one_server(fleet):
    # interleaved 8-bit and float requests (same light field, same size, so
    # only the format keeps them apart); each 8-bit view equals the 8-bit
    # render of the same camera alone, each float view the float render
    rl, lfs = fleet
    st, _, (U, V, W, H) = lfs[0]
    rng = np.random.default_rng(35)
    cams = [(float(rng.random() * (U - 1)), float(rng.random() * (V - 1)), float(rng.choice([0.0, 0.6, 1.4])))
            for _ in range(64)]
    fmts = [torch.uint8 if i % 3 else torch.float32 for i in range(len(cams))]
    srv = rl.Server(n_streams=2, max_batch=16, memory_budget=1 << 26)
    lf_id = srv.add(st)
    outs = [torch.empty((H, W, 3), dtype=f).pin_memory() for f in fmts]
    for (u, v, d), o in zip(cams, outs):
        srv.submit(lf_id, u, v, d, o)
    comps = srv.poll(wait=True)
    srv.close()
    assert len(comps) == len(cams) and all(c["status"] == 0 for c in comps)
    uv = torch.tensor([[u, v] for u, v, _ in cams], dtype=torch.float32, device="cuda")
    disp = torch.tensor([d for _, _, d in cams], dtype=torch.float32, device="cuda")
    ref8 = st.render(uv, disp, W, H, u8=True).cpu()
    ref32 = st.render(uv, disp, W, H).cpu()
    for i, o in enumerate(outs):
        assert torch.equal(o, ref8[i] if fmts[i] == torch.uint8 else ref32[i]), i
