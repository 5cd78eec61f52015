"""Debug builds: the device bounds checks (RLFC_DEBUG, rlfc_debug_flags).

The debug library checks every stored block before the full decode, the
per-request decode and the binned decode decode it: its mode, header and
payload must lie inside its record.  A failed check sets a flag and the block
is treated as absent, so a kernel never reads out of range.  A stream the
loader accepted raises no flag.  These tests run the debug build in a child
process, so that the rest of the run keeps binding the release library.
They check that every decode path gives the oracle's bytes with no flag
raised, and that the release build reports that it has no checks.
"""
import os
import subprocess
import sys

import pytest

import __graft_entry__

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
E_UNSUPPORTED = 3

CHILD = r'''
import os, sys
sys.path.insert(0, ROOT)
os.environ["RLFC_DEBUG_LIBRARY"] = "1"
import numpy as np
import torch
import lf_synth
import oracle
from paper_1805_06019_gb300 import rlfc

assert rlfc.library_path().endswith(os.path.join("_build_debug", "librlfc.so"))
torch.cuda.set_device(0)
# (U, V, W, H, L, cluster sides, tau_p, tau_b, q): a 2-level, a 3-level with
# odd sizes, a 4-level and a quantised tree
cases = [(5, 5, 64, 64, 2, [0, 5], 2, 32, 0), (6, 5, 30, 21, 3, [0, 2, 3], 3, 40, 0),
         (8, 8, 24, 24, 4, [0, 2, 2, 2], 2, 24, 0), (5, 5, 20, 16, 3, [0, 2, 3], 0, 0, 2)]
for k, (U, V, W, H, L, c, tp, tb, q) in enumerate(cases):
    lf = lf_synth.make_lightfield(U, V, W, H, [0.0, 0.7, 1.6], 1.0, preset_id=300 + k)
    data = oracle.encode(lf, U, V, B=4, L=L, c=c, tau_p=tp, tau_b=tb, q=q)
    ost = oracle.Stream(data)
    st = rlfc.Stream(data)
    ref = ost.decode_all()
    assert np.array_equal(st.decode_all().cpu().numpy(), ref), ("decode_all", k)
    rng = np.random.default_rng(k)
    n = 3000
    pv = rng.integers(0, st.n_views, n).astype(np.int32)
    pl = rng.integers(0, st.nloc, n).astype(np.int32)
    views, locs = torch.from_numpy(pv).cuda(), torch.from_numpy(pl).cuda()
    blocks, status = st.decode_blocks(views, locs)
    assert int(status.max()) == 0
    bl = blocks.cpu().numpy()
    for r in range(0, n, 97):
        assert np.array_equal(bl[r], ost.decode_block(int(pv[r]), int(pl[r]))), ("decode_blocks", k, r)
    b = rlfc.Batch(st, n)
    out = torch.empty((n, 4, 4, 3), dtype=torch.uint8, device="cuda")
    b.decode(views, locs, out)
    assert torch.equal(out, blocks), ("batch", k)
    b.close()
    # renders: four cameras (the packed full decode first) and one (decoded on demand)
    uv = torch.tensor([[0.3, 0.6], [1.5, 2.2], [U - 1.2, 0.4], [2.0, V - 1.5]], dtype=torch.float32, device="cuda")
    disp = torch.tensor([0.0, 0.7, -0.5, 1.2], dtype=torch.float32, device="cuda")
    for m in (4, 1):
        img = st.render(uv[:m], disp[:m], W, H).cpu().numpy()
        for r in range(m):
            want = oracle.render_view(ref, U, V, float(uv[r, 0]), float(uv[r, 1]), float(disp[r]), W, H)
            assert np.abs(img[r] - want).max() <= 1e-3, ("render", k, m, r)
    flags = st.debug_flags()
    assert flags == 0, ("flags", k, flags)
    st.close()
print("OK")
'''


def test_debug_build_decodes_the_oracle_bytes_without_flags():
    import paper_1805_06019_gb300 as pkg

    __graft_entry__.build()
    pkg.build(debug=True)
    r = subprocess.run([sys.executable, "-c", CHILD.replace("ROOT", repr(ROOT), 1)], capture_output=True,
                       text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert r.stdout.strip().endswith("OK")


def test_release_build_has_no_checks():
    import numpy as np

    import lf_synth
    import oracle
    from paper_1805_06019_gb300 import rlfc

    __graft_entry__.build()
    lf = lf_synth.make_lightfield(5, 5, 16, 16, [0.0, 1.0], 1.0, preset_id=310)
    data = oracle.encode(lf, 5, 5, B=4, L=2, c=[0, 5], tau_p=2, tau_b=32)
    st = rlfc.Stream(data)
    assert not rlfc.library_path().endswith(os.path.join("_build_debug", "librlfc.so"))
    with pytest.raises(rlfc.RLFCError) as ei:
        st.debug_flags()
    assert ei.value.code == E_UNSUPPORTED
    assert np.array_equal(st.decode_all().cpu().numpy(), oracle.Stream(data).decode_all())
    st.close()
