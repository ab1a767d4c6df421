"""Pins for the stacked unknowns (Tile Low-rank MDD section) and the paper's printed sizes."""
import math
import os

import numpy as np
import pytest

import tlr_synth as synth
from oracle import layout

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if line:
            k, v = [t.strip() for t in line.split("=")]
            out[k] = [float(t) for t in v.split(",")]
    return out


@pytest.mark.parametrize("n", [1, 2, 3, 4, 7, 16, 24])
def test_pair_index_closed_form_matches_paper_order(n):
    # L-bar = (L_21, L_31, ..., L_N1, L_32, ..., L_N,N-1): column outer, row inner
    order = []
    for j in range(n):
        for i in range(j + 1, n):
            order.append((i, j))
    assert layout.pairs(n) == order
    for p, (i, j) in enumerate(order):
        assert layout.pair_index(i, j, n) == p


@pytest.mark.parametrize("nr,b,ranks,mode", [
    (256, 64, 8, "dense"), (4096, 256, 26, "rule"), (9216, 384, 64, "rule"),
    (64, 16, 2, "lowrank"), (48, 16, [1, 0, 16, 2, 0, 3], "rule"),
])
def test_sizes_and_offsets(nr, b, ranks, mode):
    lay = layout.make_layout(nr, b, ranks, mode)
    n = nr // b
    assert len(lay.pair_list) == n * (n - 1) // 2
    expect = sum(b * b if lay.dense[i] else b * lay.k_diag[i] for i in range(n))
    expect += 2 * sum(b * k for k in lay.k_pair)
    assert lay.size == expect
    # offsets are contiguous and increasing in stacking order
    offs = lay.off_diag + lay.off_l + lay.off_r
    assert offs == sorted(offs)
    tiles = synth.theta_tiles(nr, b, ranks, lay.dense)
    assert sum(t.rows * t.cols for t in tiles) == lay.size


def test_rule_dense_iff_rank_at_least_quarter_tile():
    lay = layout.make_layout(512, 128, [31, 32, 0, 128, 5, 6, 7, 8, 9, 10], "rule")
    assert lay.dense[:4] == [False, True, False, True]


def test_invalid_shapes_rejected():
    with pytest.raises(ValueError):
        layout.make_layout(100, 64, 4)
    with pytest.raises(ValueError):
        layout.make_layout(128, 64, 65)


def test_paper_printed_sizes():
    g = _golden()
    ns, nr = int(g["ns"][0]), int(g["nr"][0])
    assert ns == int(g["source_lines"][0]) * int(g["sources_per_line"][0])
    assert nr == int(g["receiver_lines"][0]) * int(g["receivers_per_line"][0])
    assert math.prod(int(x) for x in g["nr_prime_factors"]) == nr
    for t in g["tile_sizes_reported"]:
        assert nr % int(t) == 0
    # complex64 D, U (ns x nr) and X (nr x nr): "approximately 8 GB"
    gib = 8 * (2 * ns * nr + nr * nr) / 2**30
    assert abs(gib - g["gb_per_frequency"][0]) < 0.5
    # complex128 would be twice that: the reading "complex64" is the one that fits
    assert abs(2 * gib - g["gb_per_frequency"][0]) > 4
    lam = [10.0 * 0.1 ** s for s in range(3)]
    np.testing.assert_allclose(lam, g["lambda_schedule"])
