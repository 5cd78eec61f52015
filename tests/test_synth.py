"""The seeded input generator: the torch compositing path (used by the
benchmark to build large presets on the device) gives the numpy path's views
bit for bit.  Run here on torch's CPU backend; the same float32 operations run
on the device."""
import numpy as np
import pytest

import lf_synth


@pytest.mark.parametrize("args", [
    (5, 5, 64, 48, [0.0, 0.5, 1.5], 1.0, 0, False),
    (4, 3, 96, 80, [-2.0, -1.0, 0.0, 1.3, 2.0], 1.0, 2, True),
    (3, 3, 40, 36, [-0.7, 0.3], 2.0, 3, False),
    (2, 1, 33, 17, [0.25], 0.0, 5, False),
])
def test_torch_compositing_matches_numpy(args):
    torch = pytest.importorskip("torch")
    want = lf_synth.make_lightfield(*args)
    got = lf_synth.make_lightfield_torch(*args, device="cpu")
    assert got.dtype == torch.uint8
    assert np.array_equal(got.numpy(), want)
