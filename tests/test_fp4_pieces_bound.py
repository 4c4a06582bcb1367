"""The error bound of the FP4 form's panel pieces (no GPU): each column v, scaled by a power of
two 2^e that puts max |v| 2^e in (1.5, 3], is cut into six E2M1 pieces at scales 8^-k, each the
nearest E2M1 value to what the earlier pieces leave, times 8^k. The claims the form rests on:
the scaled remainder before every piece lies in [-4, 4] (no piece saturates at 6), and after
six pieces the remainder is at most 0.5 * 8^-5 of the scale. Checked on random unit-norm
columns and on values placed at the middle of every gap of the E2M1 grid (the worst case of
each rounding). This restates the decomposition in NumPy from its definition; the GPU's pieces
are checked through the statistics in tests/test_gpu_fp4.py."""
import numpy as np

# E2M1 magnitudes: 0, 0.5, 1, 1.5, 2, 3, 4, 6
GRID = np.array([0.0, 0.5, 1.0, 1.5, 2.0, 3.0, 4.0, 6.0])
PIECES = 6


def e2m1_nearest(x):
    """Nearest E2M1 value (ties to the even code, i.e. the grid point with an even index)."""
    a = np.abs(x)
    d = np.abs(a[..., None] - GRID)
    best = np.min(d, axis=-1, keepdims=True)
    idx = np.where(np.isclose(d, best, rtol=0.0, atol=1e-300), np.arange(GRID.size), 99)
    # among ties take the even index (an even mantissa bit)
    even = np.where(idx % 2 == 0, idx, 99).min(axis=-1)
    odd = idx.min(axis=-1)
    pick = np.where(even < 99, even, odd)
    return np.sign(x) * GRID[pick]


def pieces(v):
    """(scale exponent e, pieces q [PIECES][n], remainders before each piece, times 8^k)."""
    mx = np.max(np.abs(v))
    e = int(np.floor(np.log2(3.0 / mx)))
    z = v * 2.0 ** e
    res = z.copy()
    qs, before = [], []
    for k in range(PIECES):
        t = res * 8.0 ** k
        before.append(t)
        q = e2m1_nearest(t)
        qs.append(q)
        res = res - q * 8.0 ** -k
    return e, np.array(qs), np.array(before), res


def test_scale_puts_the_column_maximum_in_the_first_grid_range():
    rng = np.random.default_rng(5)
    for _ in range(50):
        v = rng.standard_normal(1000) * 10.0 ** rng.uniform(-6, 3)
        e = pieces(v)[0]
        m = np.max(np.abs(v)) * 2.0 ** e
        assert 1.5 < m <= 3.0


def test_no_piece_saturates_and_the_remainder_meets_the_bound():
    rng = np.random.default_rng(7)
    for n in (7, 1000, 23_000):
        v = rng.standard_normal(n)
        v /= np.linalg.norm(v)
        e, q, before, res = pieces(v)
        assert np.all(np.abs(before) <= 4.0 + 1e-12)    # never past the largest gap's end
        assert np.all(np.abs(q) <= 4.0)                 # 6 is never needed
        assert np.max(np.abs(res)) <= 0.5 * 8.0 ** -5 + 1e-15
        # the pieces reproduce the scaled column to that bound
        z = v * 2.0 ** e
        rebuilt = sum(q[k] * 8.0 ** -k for k in range(PIECES))
        assert np.max(np.abs(z - rebuilt)) <= 0.5 * 8.0 ** -5 + 1e-15


def test_worst_case_of_every_gap():
    """Values at the middle of each gap of the grid below the column maximum 3 (the gap [3, 4]
    only meets later pieces, whose inputs are remainders times 8): the remainder of each
    rounding is at most half a gap, 0.5 (gaps of 1 in [2, 4]), which times 8 is 4, the end of
    the range the next piece sees."""
    mids = np.array([0.25, 0.75, 1.25, 1.75, 2.5, 2.75])
    v = np.concatenate([[3.0], mids, -mids])
    e, q, before, res = pieces(v)
    assert e == 0
    assert np.all(np.abs(before) <= 4.0 + 1e-12)
    assert np.max(np.abs(res)) <= 0.5 * 8.0 ** -5 + 1e-15


def test_five_pieces_would_not_meet_the_bound():
    """With one piece fewer the remainder can reach 0.5 * 8^-4, eight times the six-piece bound
    (why the form takes six)."""
    v = np.array([3.0, 2.5 + 0.5 * 8.0 ** -1 * 0.999])
    e, q, before, res = pieces(v)
    rem5 = v * 2.0 ** e - sum(q[k] * 8.0 ** -k for k in range(PIECES - 1))
    assert np.max(np.abs(rem5)) > 0.5 * 8.0 ** -5
