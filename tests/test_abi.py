"""The C-ABI library loads and exports every declared entry point; host-only
calls (layout, sizes, validation) agree with the oracle.  No GPU needed."""
import os
import re

import pytest

from oracle import layout

pt = pytest.importorskip("paper_2412_14973_gb300")
T = pt

HDR = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "tlr_mdd.h")


def _lib():
    try:
        return T.lib()
    except RuntimeError as e:  # not built in this checkout
        pytest.skip(str(e))


def test_exports_every_declared_symbol():
    L = _lib()
    src = open(HDR).read()
    declared = sorted(set(re.findall(r"\b(tlr_mdd_\w+)\s*\(", src)))
    assert declared, "no declarations parsed"
    for name in declared:
        assert hasattr(L, name), name
    assert set(declared) == set(T.EXPORTED)


@pytest.mark.parametrize("nr,b,ranks,mode,abimode", [
    (256, 64, 8, "dense", T.TLR_DIAG_DENSE),
    (4096, 256, 26, "rule", T.TLR_DIAG_RULE),
    (96, 16, [1, 0, 16, 2, 0, 3] + list(range(15)), "rule", T.TLR_DIAG_RULE),
    (64, 16, 2, "lowrank", T.TLR_DIAG_LOWRANK),
])
def test_theta_layout_bit_exact(nr, b, ranks, mode, abimode):
    _lib()
    lay = layout.make_layout(nr, b, ranks, mode)
    kw = dict(ranks=ranks) if isinstance(ranks, list) else dict(rank=ranks)
    d = T.desc(nr, nr, b, nx=nr, ny=1, diag_mode=abimode, **kw)
    od, ol, orr, dn = T.tlr_mdd_theta_layout(d)
    assert od == lay.off_diag
    assert ol == lay.off_l
    assert orr == lay.off_r
    assert dn == lay.dense
    assert T.tlr_mdd_theta_size(d) == lay.size
    assert T.tlr_mdd_workspace_bytes(d) > 8 * 5 * nr * nr


def test_per_tile_diag_mode():
    _lib()
    d = T.desc(48, 48, 16, rank=2, diag_mode=T.TLR_DIAG_PER_TILE, diag_dense=[True, False, True])
    lay = layout.make_layout(48, 16, 2, [True, False, True])
    assert T.tlr_mdd_theta_layout(d)[0] == lay.off_diag
    assert T.tlr_mdd_theta_size(d) == lay.size


@pytest.mark.parametrize("nr,b,ranks,dense", [
    (48, 16, 3, [False, True, False]),
    (64, 16, [1, 0, 4, 2] + [k % 5 for k in range(12)], [False, False, True, False]),
])
def test_general_theta_layout_bit_exact(nr, b, ranks, dense):
    # the general (non-reciprocal) stacking: diagonal blocks (Z, or L then R),
    # then L and R of the ordered pairs, column outer, row inner
    from oracle import general
    _lib()
    n = nr // b
    rl = ranks if isinstance(ranks, list) else [ranks] * (n + n * (n - 1))
    d = T.desc(nr, 10, b, ranks=rl, diag_mode=T.TLR_DIAG_PER_TILE, diag_dense=dense,
               reciprocity=T.TLR_RECIP_NONE)
    lay = general.make_general_layout(nr, b, rl, dense)
    od, ol, orr, dn = T.tlr_mdd_theta_layout(d)
    assert od == lay.off_diag and ol == lay.off_l and orr == lay.off_r
    assert dn == lay.dense
    assert T.tlr_mdd_theta_size(d) == lay.size


@pytest.mark.parametrize("tiles,ranks,dense,recip", [
    ([3, 5, 2], [1, 2, 2, 2, 1, 2], [False, True, False], False),
    ([48, 80, 16, 112], 9, [False, True, False, False], False),
    ([100, 28, 128], [5, 28, 7] + [3, 0, 28], [False, True, False], False),
    ([3, 5, 2], [1, 2, 2] + [2, 1, 3, 2, 2, 1], [False, True, False], True),
    ([40, 24, 64], 6, [True, False, False], True),
])
def test_nonuniform_theta_layout_bit_exact(tiles, ranks, dense, recip):
    # tile sizes d_i: L_ij is d_i x k, R_ij is d_j x k, diagonal blocks d_i x k or d_i x d_i
    from oracle import general
    _lib()
    nr, n = sum(tiles), len(tiles)
    npair = n * (n - 1) if recip else n * (n - 1) // 2
    rl = ranks if isinstance(ranks, list) else [ranks] * (n + npair)
    d = T.desc(nr, 10, 0, ranks=rl, diag_mode=T.TLR_DIAG_PER_TILE, diag_dense=dense, tiles=tiles,
               reciprocity=T.TLR_RECIP_NONE if recip else T.TLR_RECIP_SYMMETRIC)
    if recip:
        lay = general.make_general_layout(nr, None, rl, dense, tiles=tiles)
    else:
        lay = layout.make_layout(nr, None, rl, dense, tiles=tiles)
    od, ol, orr, dn = T.tlr_mdd_theta_layout(d)
    assert od == lay.off_diag and ol == lay.off_l and orr == lay.off_r
    assert dn == lay.dense
    assert T.tlr_mdd_theta_size(d) == lay.size
    assert T.tlr_mdd_workspace_bytes(d) > 0


def test_nonuniform_rule_uses_each_tile_size():
    # dense iff 4 k_ii >= d_i: with k = 8, tiles of 32 are dense, tiles of 33 are not
    _lib()
    tiles = [32, 33, 31, 40]
    d = T.desc(sum(tiles), 10, 0, rank=8, tiles=tiles)
    lay = layout.make_layout(sum(tiles), None, 8, "rule", tiles=tiles)
    assert T.tlr_mdd_theta_layout(d)[3] == lay.dense == [True, False, True, False]
    assert T.tlr_mdd_theta_size(d) == lay.size


@pytest.mark.parametrize("kw,code", [
    (dict(nr=10, ns=10, tile=0, rank=1, tiles=[3, 5, 1]), -2),      # sizes do not sum to nr
    (dict(nr=10, ns=10, tile=0, rank=1, tiles=[3, 0, 7]), -2),      # an empty tile
    (dict(nr=10, ns=10, tile=0, rank=3, tiles=[2, 8]), -2),         # rank above d_0
    (dict(nr=10, ns=10, tile=0, ranks=[1, 1, 4], tiles=[3, 7]), -2),  # pair rank above min(d_i, d_j)
    (dict(nr=10, ns=10, tile=0, rank=1, tiles=[]), -2),             # no tiles
])
def test_invalid_partitions_rejected(kw, code):
    _lib()
    d = T.desc(**kw)
    with pytest.raises(T.TLRError) as ei:
        T.tlr_mdd_theta_size(d)
    assert ei.value.code == code


@pytest.mark.parametrize("kw,code", [
    (dict(nr=100, ns=10, tile=64, rank=4), -2),          # tile does not divide nr
    (dict(nr=128, ns=10, tile=64, rank=65), -2),         # rank above tile
    (dict(nr=128, ns=10, tile=64, rank=-1), -2),
    (dict(nr=128, ns=0, tile=64, rank=4), -2),
    (dict(nr=128, ns=10, tile=64, rank=4, reciprocity=2), -1),  # unknown reciprocity mode
    (dict(nr=128, ns=10, tile=64, rank=4, precision=7), -1),
    (dict(nr=128, ns=10, tile=64, rank=4, diag_mode=9), -1),
])
def test_invalid_descriptions_rejected(kw, code):
    _lib()
    d = T.desc(**kw)
    with pytest.raises(T.TLRError) as ei:
        T.tlr_mdd_theta_size(d)
    assert ei.value.code == code
    assert T.tlr_mdd_workspace_bytes(d) == -1
    assert T.tlr_mdd_last_error()


@pytest.mark.parametrize("limit", [0, -5, 20_000_000_000])
def test_wait_selftest_rejects_bad_limits(limit):
    _lib()
    with pytest.raises(T.TLRError) as ei:
        T.tlr_mdd_wait_selftest(limit)
    assert ei.value.code == T.TLR_ERR_ARG


def test_random_partitions_match_the_oracle_layout():
    # random tile sizes, ranks within [0, min(d_i, d_j)], per-tile diagonal
    # modes, both forms: the library's stacking equals the oracle's
    from oracle import general
    import numpy as np
    _lib()
    g = np.random.default_rng(2412)
    for trial in range(60):
        n = int(g.integers(1, 7))
        tiles = [int(x) for x in g.integers(1, 40, n)]
        nr = sum(tiles)
        dense = [bool(x) for x in g.integers(0, 2, n)]
        recip = bool(trial % 2)
        pairs = general.ordered_pairs(n) if recip else layout.pairs(n)
        kd = [int(g.integers(0, tiles[i] + 1)) for i in range(n)]
        kp = [int(g.integers(0, min(tiles[i], tiles[j]) + 1)) for (i, j) in pairs]
        d = T.desc(nr, 7, 0, ranks=kd + kp, diag_mode=T.TLR_DIAG_PER_TILE, diag_dense=dense, tiles=tiles,
                   reciprocity=T.TLR_RECIP_NONE if recip else T.TLR_RECIP_SYMMETRIC)
        if recip:
            lay = general.make_general_layout(nr, None, kd + kp, dense, tiles=tiles)
        else:
            lay = layout.make_layout(nr, None, kd + kp, dense, tiles=tiles)
        od, ol, orr, dn = T.tlr_mdd_theta_layout(d)
        assert (od, ol, orr, dn) == (lay.off_diag, lay.off_l, lay.off_r, lay.dense), (tiles, kd, kp, dense)
        assert T.tlr_mdd_theta_size(d) == lay.size
        assert T.tlr_mdd_workspace_bytes(d) > 0


def test_noalloc_wrapper_rejects_bad_buffers_before_the_call():
    # the allocation-free adjoint has no handle that knows the buffer sizes,
    # so the binding checks dtype, contiguity, size and device before it calls
    # into the library (no device work, no GPU needed to reach these checks)
    torch = pytest.importorskip("torch")
    nr, ns = 8, 5
    ok_v = torch.zeros(nr * ns, dtype=torch.complex64)
    ok_g = torch.zeros(nr * nr, dtype=torch.complex64)
    short = torch.zeros(nr * ns - 1, dtype=torch.complex64)
    cases = [
        ((short, ok_v, ok_g), T.TLR_ERR_SHAPE),                        # V too short
        ((ok_v, short, ok_g), T.TLR_ERR_SHAPE),                        # Dt too short
        ((ok_v, ok_v, torch.zeros(nr * nr - 1, dtype=torch.complex64)), T.TLR_ERR_SHAPE),
        ((ok_v.to(torch.complex128), ok_v, ok_g), T.TLR_ERR_ARG),      # wrong dtype
        ((torch.zeros((ns, nr), dtype=torch.complex64).t(), ok_v, ok_g), T.TLR_ERR_ARG),  # not contiguous
        ((ok_v, ok_v, ok_g), T.TLR_ERR_ARG),                           # host tensors, not on the device
        ((None, ok_v, ok_g), T.TLR_ERR_ARG),
    ]
    for (V, Dt, G), code in cases:
        with pytest.raises(T.TLRError) as ei:
            T.tlr_mdd_adjoint_noalloc(V, Dt, nr, ns, G)
        assert ei.value.code == code
    with pytest.raises(T.TLRError) as ei:
        T.tlr_mdd_adjoint_noalloc(ok_v, ok_v, 0, ns, ok_g)
    assert ei.value.code == T.TLR_ERR_SHAPE


def test_pass_cta_cap_is_set_and_restored_without_a_gpu():
    # the cap is host state: setting it launches nothing
    _lib()
    prev = T.tlr_mdd_set_pass_ctas(37)
    assert prev >= 0
    assert T.tlr_mdd_set_pass_ctas(0) == 37
    with pytest.raises(T.TLRError):
        T.tlr_mdd_set_pass_ctas(-1)
    assert T.tlr_mdd_set_pass_ctas(prev) == 0
