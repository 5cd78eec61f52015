"""Pins of the oracle's BISE (paper Section 3.3) against things other than itself:
the mode set's definition, the closed-form packed lengths, the entropy bound,
hand-derived bit layouts and an exhaustive round trip on small blocks."""
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_mode_set_is_the_ascending_union_of_power_of_two_ranges():
    table = oracle.mode_table()
    assert len(table) == 28
    expected = sorted({2 ** b for b in range(11)} | {3 * 2 ** b for b in range(9)}
                      | {5 * 2 ** b for b in range(8)})
    assert [N for N, _, _ in table] == expected
    for N, kind, b in table:
        assert N == (1, 3, 5)[kind] * 2 ** b


@pytest.mark.parametrize("n", list(range(0, 70)))
def test_packed_length_is_the_closed_form(n):
    # ASTC closed forms: n*b, n*b + ceil(8n/5) (trits), n*b + ceil(7n/3) (quints)
    for k, (N, kind, b) in enumerate(oracle.mode_table()):
        extra = (0, -(-8 * n // 5), -(-7 * n // 3))[kind]
        assert oracle.bise_bits(n, k) == n * b + extra


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 15, 16, 64])
def test_length_respects_the_entropy_bound(n):
    # no code for N^n equiprobable sequences can be shorter than n*log2(N)
    for k, (N, kind, b) in enumerate(oracle.mode_table()):
        bits = oracle.bise_bits(n, k)
        assert bits >= math.ceil(n * math.log2(N) - 1e-9)
        # BISE wastes at most 1.6 - log2(3) (trits) / 7/3 - log2(5) (quints)
        # bits per value plus one partial group
        assert bits <= n * math.log2(N) + 0.06 * n + 3


def _golden_bise():
    rows = []
    for line in open(os.path.join(GOLDEN, "bise_examples.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        head, hexs, nbits = [p.strip() for p in line.split("|")]
        f = [int(x) for x in head.split()]
        k, N, n, vals = f[0], f[1], f[2], f[3:]
        assert len(vals) == n
        rows.append((k, N, vals, bytes.fromhex(hexs), int(nbits)))
    return rows


@pytest.mark.parametrize("k,N,vals,expect,nbits", _golden_bise())
def test_hand_derived_bit_layouts(k, N, vals, expect, nbits):
    assert oracle.mode_table()[k][0] == N
    assert oracle.bise_bits(len(vals), k) == nbits
    packed = oracle.bise_pack(vals, k)
    assert packed == expect
    assert list(oracle.bise_unpack(packed, len(vals), k)) == vals


def test_exhaustive_round_trip_small_blocks():
    # every sequence with N^n <= 2e6, for every mode and n = 1..7
    checked = 0
    for k in range(28):
        for n in range(1, 8):
            r = oracle.bise_exhaustive(n, k, 2_000_000)
            if r < 0:
                break
            assert r == 0, (k, n)
            checked += 1
    assert checked > 60


@pytest.mark.parametrize("n", [16, 64])
def test_random_round_trip_full_blocks(n):
    rng = np.random.default_rng(7)
    for k, (N, _, _) in enumerate(oracle.mode_table()):
        for pos in (0, 5, 31):
            u = rng.integers(0, N, size=n)
            packed = oracle.bise_pack(u, k, pos)
            assert list(oracle.bise_unpack(packed, n, k, pos)) == list(u)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 16, 64])
def test_mode_search_is_the_smallest_feasible_range(n):
    # cost is non-decreasing in N, so the exhaustive min-cost search (ties to
    # the smaller index) must pick the smallest range that holds the span
    table = oracle.mode_table()
    costs = [oracle.bise_bits(n, k) for k in range(28)]
    assert all(a <= b for a, b in zip(costs, costs[1:]))
    for span in range(0, 1024):
        smallest = next(k for k, (N, _, _) in enumerate(table) if N >= span + 1)
        assert oracle.choose_mode(n, span) == smallest
    assert oracle.choose_mode(n, 1024) == -1


def test_sixteen_value_costs():
    # n = 16 (4x4 blocks): the cost ladder used by the stream
    expect = [0, 16, 26, 32, 38, 42, 48, 54, 58, 64, 70, 74, 80, 86, 90, 96, 102, 106,
              112, 118, 122, 128, 134, 138, 144, 150, 154, 160]
    assert [oracle.bise_bits(16, k) for k in range(28)] == expect
