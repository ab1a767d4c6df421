"""Pins for the Hilbert receiver reordering (eq. 10-14) in the oracle."""
import numpy as np
import pytest

from oracle import hilbert


@pytest.mark.parametrize("nx,ny", [(1, 1), (2, 2), (16, 16), (64, 32), (5, 3), (32, 32), (90, 7)])
def test_perm_is_bijection(nx, ny):
    p = hilbert.perm(nx, ny)
    assert sorted(p.tolist()) == list(range(nx * ny))


def test_base_cell_order():
    # the 2x2 base pattern of this variant: (0,0), (0,1), (1,1), (1,0)
    order = [hilbert.xy2d(2, x, y) for (x, y) in [(0, 0), (0, 1), (1, 1), (1, 0)]]
    assert order == [0, 1, 2, 3]


@pytest.mark.parametrize("n", [2, 4, 8, 16, 32, 64])
def test_unit_steps_on_square_grid(n):
    p = hilbert.perm(n, n)
    x, y = p % n, p // n
    steps = np.abs(np.diff(x)) + np.abs(np.diff(y))
    assert np.all(steps == 1)
    assert (x[0], y[0]) == (0, 0)
    assert (x[-1], y[-1]) == (n - 1, 0)


@pytest.mark.parametrize("n", [4, 8, 16, 32])
def test_recursive_construction(n):
    """The curve of side n is four copies of the curve of side n/2: the lower
    left one transposed, the two upper ones translated, the lower right one
    reflected and transposed -- the self-similar definition of the curve."""
    s = n // 2
    for x in range(n):
        for y in range(n):
            d = hilbert.xy2d(n, x, y)
            if x < s and y < s:
                ref = hilbert.xy2d(s, y, x)
            elif x < s:
                ref = s * s + hilbert.xy2d(s, x, y - s)
            elif y >= s:
                ref = 2 * s * s + hilbert.xy2d(s, x - s, y - s)
            else:
                ref = 3 * s * s + hilbert.xy2d(s, s - 1 - y, 2 * s - 1 - x)
            assert d == ref


def test_non_square_embedding_keys_unique():
    k = hilbert.keys(177, 10)
    assert len(set(k.tolist())) == k.size
    assert k.max() < 256 * 256


def test_reordering_keeps_symmetry_and_matches_column_selection():
    rng = np.random.default_rng(0)
    nx, ny = 8, 4
    n = nx * ny
    p = hilbert.perm(nx, ny)
    S = hilbert.hilbert_matrix(p)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    X = A + A.T
    Xh = S.T @ X @ S                                   # eq. (10)
    assert np.array_equal(Xh, Xh.T)
    np.testing.assert_array_equal(Xh, X[np.ix_(p, p)])
    D = rng.standard_normal((5, n)) + 0j
    np.testing.assert_array_equal(D @ S, D[:, p])      # D-hat = D S (eq. 14)
    np.testing.assert_allclose(S @ Xh @ S.T, X)        # eq. (11)
