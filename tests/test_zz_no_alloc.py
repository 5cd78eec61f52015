"""rlfc_encode_no_alloc, the encoder entry point for callers that cannot
allocate device memory (its scratch is the library's fixed 32 MiB array),
checked through the C ABI against the oracle's encoder and against
rlfc_encode: the streams must be byte-identical, as every encoder test
requires, over several calls in a row that reuse the shared array.  One case
sits just under the 32 MiB limit: the entry point carves the encoder's
buffers from no more than the scratch bound it computed, so an under-counted
bound fails that case.  This file runs last so that a failure here cannot
stop the rest of the GPU suite; it also passes on its own."""
import ctypes

import numpy as np
import pytest
import torch

import lf_synth
import oracle

pytestmark = pytest.mark.gpu

E_RANGE = 6


@pytest.fixture(scope="module")
def rl():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1805_06019_gb300 import rlfc
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return rlfc


def _params(rl, U, V, W, H, L, c, tau_p, tau_b, q=0):
    p = rl.EncParams()
    p.U, p.V, p.W, p.H, p.B, p.L = U, V, W, H, 4, L
    for l in range(1, L):
        p.c[l] = c[l]
    p.tau_p, p.tau_b, p.q = tau_p, tau_b, q
    return p


def _no_alloc(rl, p, d_rgb, capacity):
    buf = ctypes.create_string_buffer(max(capacity, 1))
    n = ctypes.c_size_t()
    rc = rl.lib().rlfc_encode_no_alloc(ctypes.byref(p), ctypes.c_void_p(d_rgb.data_ptr()),
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                       buf, capacity, ctypes.byref(n))
    return rc, buf.raw[: n.value], n.value


CASES = [
    # (U, V, W, H, L, c, tau_p, tau_b, q)
    (5, 5, 64, 64, 2, [0, 5], 2, 32, 0),
    (6, 5, 30, 21, 3, [0, 2, 3], 3, 40, 0),
    (5, 5, 20, 16, 3, [0, 2, 3], 0, 0, 2),
    # scratch bound 32 836 608 bytes, 97.9 % of the array (9 x 9 x 184^2
    # would need 34 312 192 and is rejected)
    (9, 9, 180, 180, 3, [0, 3, 3], 4, 64, 0),
]


def test_calls_in_a_row_match_the_oracle_and_the_allocating_encoder(rl):
    inputs = []
    for i, (U, V, W, H, L, c, tp, tb, q) in enumerate(CASES):
        lf = lf_synth.make_lightfield(U, V, W, H, [0.0, 0.5, 1.5], 1.0, preset_id=200 + i)
        d = torch.from_numpy(lf).cuda()
        want = oracle.encode(lf, U, V, B=4, L=L, c=c, tau_p=tp, tau_b=tb, q=q)
        assert rl.encode(d, U, V, L, c, tau_p=tp, tau_b=tb, q=q) == want
        inputs.append((d, _params(rl, U, V, W, H, L, c, tp, tb, q), want))
    # two passes over differently shaped light fields: the shared array must
    # carry nothing from one call into the next
    for _ in range(2):
        for d, p, want in inputs:
            rc, got, n = _no_alloc(rl, p, d, len(want) + 64)
            assert rc == 0, rl.lib().rlfc_last_error().decode()
            assert n == len(want)
            assert got == want


def test_light_fields_beyond_the_scratch_limit_are_rejected(rl):
    p = _params(rl, 9, 9, 512, 512, 3, [0, 3, 3], 4, 64)
    dummy = torch.zeros(16, dtype=torch.uint8, device="cuda")   # never read: rejected first
    rc, _, n = _no_alloc(rl, p, dummy, 1024)
    assert rc == E_RANGE and n == 0
    assert "33554432" in rl.lib().rlfc_last_error().decode()


def test_small_output_buffer_reports_the_size_needed(rl):
    U, V, W, H, L, c, tp, tb, q = CASES[0]
    lf = lf_synth.make_lightfield(U, V, W, H, [0.0, 0.5, 1.5], 1.0, preset_id=200)
    d = torch.from_numpy(lf).cuda()
    want = rl.encode(d, U, V, L, c, tau_p=tp, tau_b=tb, q=q)
    rc, _, n = _no_alloc(rl, _params(rl, U, V, W, H, L, c, tp, tb, q), d, 16)
    assert rc == E_RANGE and n == len(want)
    assert np.frombuffer(want[:4], dtype=np.uint8).tolist() == list(b"RLFC")


def test_binding_retries_with_the_size_the_call_reports(rl):
    U, V, W, H, L, c, tp, tb, q = CASES[1]
    lf = lf_synth.make_lightfield(U, V, W, H, [0.0, 0.5, 1.5], 1.0, preset_id=201)
    want = oracle.encode(lf, U, V, B=4, L=L, c=c, tau_p=tp, tau_b=tb, q=q)
    d = torch.from_numpy(lf).cuda()
    # a host buffer far too small: the first call reports the stream size,
    # the binding calls again with a buffer of that size
    assert rl.encode_no_alloc(d, U, V, L, c, tau_p=tp, tau_b=tb, q=q, capacity=8) == want
