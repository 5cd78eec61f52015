"""Host-side pieces of the serving workload: the seeded Poisson arrival
process and the request mix."""
import numpy as np

import lf_synth


def test_poisson_arrivals_have_the_requested_rate():
    t = lf_synth.poisson_arrivals(2000.0, 200000, preset_id=7)
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    # exponential gaps: mean 1 / rate, standard deviation 1 / rate
    assert abs(gaps.mean() * 2000.0 - 1.0) < 0.01
    assert abs(gaps.std() * 2000.0 - 1.0) < 0.02
    # counts in disjoint unit windows are Poisson: variance equals mean
    counts = np.bincount((t * 10).astype(int))[:-1]     # 0.1 s windows
    assert abs(counts.var() / counts.mean() - 1.0) < 0.15


def test_poisson_arrivals_are_seeded():
    a = lf_synth.poisson_arrivals(500.0, 100, preset_id=4)
    b = lf_synth.poisson_arrivals(500.0, 100, preset_id=4)
    c = lf_synth.poisson_arrivals(500.0, 100, preset_id=5)
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_serving_requests_cover_the_fleet_uniformly():
    lf, u, v, d = lf_synth.serving_requests(80000, len(lf_synth.SERVING_FLEET), preset_id=4)
    counts = np.bincount(lf, minlength=8)
    assert counts.min() > 0.9 * 10000 and counts.max() < 1.1 * 10000
    for x in (u, v, d):
        assert 0.0 <= x.min() and x.max() < 1.0
    sizes = {lf_synth.PRESETS[p]["W"] for p, _ in lf_synth.SERVING_FLEET}
    assert sizes == {256, 512, 1024}
