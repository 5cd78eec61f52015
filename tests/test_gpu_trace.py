"""Kernel tracing through the C ABI: while on, each library launch is timed
with CUDA events on its stream and counted per kernel; while off nothing is
recorded.  The traced calls must still produce the oracle's bytes."""
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
    from paper_1805_06019_gb300 import rlfc
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return rlfc


def test_trace_counts_launches_and_times(rl):
    U, V, W, H = 5, 5, 32, 24
    lf = lf_synth.make_lightfield(U, V, W, H, [0.0, 0.8], 1.0, preset_id=300)
    data = oracle.encode(lf, U, V, B=4, L=2, c=[0, 5], tau_p=2, tau_b=32)
    want = oracle.Stream(data).decode_all()
    st = rl.Stream(data)
    out = torch.empty((U * V, H, W, 3), dtype=torch.uint8, device="cuda")
    rl.trace_read(reset=True)
    st.decode_all(out)                       # untraced
    rl.trace_enable(True)
    try:
        for _ in range(3):
            st.decode_all(out)
        views = torch.empty((1, 24, 32, 3), dtype=torch.float32, device="cuda")
        uv = torch.tensor([[1.5, 2.25]], dtype=torch.float32, device="cuda")
        disp = torch.tensor([0.5], dtype=torch.float32, device="cuda")
        st.render(uv, disp, 32, 24, views)
        t = rl.trace_read(reset=True)
    finally:
        rl.trace_enable(False)
    assert t["decode_all_kernel"][0] == 3
    assert t["decode_all_kernel"][1] > 0.0
    assert sum(n for n, _ in t.values()) >= 4
    assert np.array_equal(out.cpu().numpy(), want)
    st.decode_all(out)                       # tracing off again
    torch.cuda.synchronize()
    assert rl.trace_read(reset=True) == {}
