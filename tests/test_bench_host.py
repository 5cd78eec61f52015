"""Host-side helpers of bench.py that the roofline's algorithmic bytes rest
on: the neighbour views a set of cameras needs, the per-location record
words of a stream, and the whole-job throughput over replicas."""
import numpy as np

import bench
import lf_synth
import oracle


def test_needed_views_follow_the_grid_cells():
    U, V = 9, 9
    # one camera per corner cell needs that cell's 2 x 2 views
    assert bench._needed_views([(0.0, 0.0, 0.0)], U, V) == 4
    assert bench._needed_views([(U - 1.0, V - 1.0, 0.0)], U, V) == 4
    # two cameras in the same cell share its four views; cameras in
    # neighbouring cells share an edge of two
    assert bench._needed_views([(2.3, 4.1, 0.0), (2.9, 4.8, 1.0)], U, V) == 4
    assert bench._needed_views([(2.5, 4.5, 0.0), (3.5, 4.5, 0.0)], U, V) == 6
    # positions outside the grid clamp to it
    assert bench._needed_views([(-5.0, 40.0, 0.0)], U, V) == 4
    # enough random cameras touch every view; never more than four per camera
    cams = lf_synth.random_views(2000, U, V, 1)
    assert bench._needed_views(cams, U, V) == U * V
    few = lf_synth.random_views(3, U, V, 2)
    assert 4 <= bench._needed_views(few, U, V) <= 12
    # a single row or column of views
    assert bench._needed_views([(1.5, 0.0, 0.0)], 4, 1) == 2


def test_location_words_partition_the_records():
    rng = np.random.default_rng(3)
    lf = rng.integers(0, 256, size=(9, 12, 20, 3), dtype=np.uint8)
    data = oracle.encode(lf, 3, 3, B=4, L=2, c=[0, 3], tau_p=2, tau_b=16)
    words, nloc = bench._stream_location_words(data)
    assert nloc == 3 * 5
    record_words = int.from_bytes(data[56:60], "little")
    assert words.sum() == record_words and (words > 0).all()


def test_job_throughput_counts_every_replica():
    one = bench.job_mpix_per_s(1, 10_000_000, 2.0)
    assert abs(one - 5000.0) < 1e-9
    assert abs(bench.job_mpix_per_s(4, 10_000_000, 2.0) - 4 * one) < 1e-9


def test_kernel_bytes_of_the_plain_step():
    class Info:
        W = H = 512
    b = bench._kernel_bytes(Info, 14_000_000, 81, 81, 1000, 512, 512)
    assert b["decode_all_kernel"] == 14_000_000 + 3 * 512 * 512 * 81
    # only the method's bytes: the float views written (the packed views the
    # renderer decodes for itself are its intermediate)
    assert b["render_native_kernel"] == 12 * 1000 * 512 * 512
    assert b["decode_all_kernel<packed>"] == 14_000_000
