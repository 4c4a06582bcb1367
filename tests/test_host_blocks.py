"""Host logic of tg_scan_host's blocking (no GPU): the block sizes it streams a genotype matrix
in, for the doubling of a context's first call and for the growth factors later calls take from
the measured scan / copy ratio."""
import pytest

import paper_2604_21095_gb300 as tg


def _round_up(x, m):
    return (x + m - 1) // m * m


@pytest.mark.parametrize("M,B", [(262144, 65536), (8_900_000, 65536), (3000, 2048), (3000, 1000),
                                 (1, 65536), (65536, 65536), (100_000, 2048)])
@pytest.mark.parametrize("f", [1.0, 1.17, 1.5, 2.0, 8.0])
def test_block_sizes_cover_the_matrix_and_grow_by_the_factor(M, B, f):
    sizes = tg.tg_host_block_sizes(M, B, f)
    assert sum(sizes) == M and all(0 < s <= B for s in sizes)
    first = _round_up(B // 8, 256) if B >= 2048 else B
    assert sizes[0] == min(first, M)
    for a, b in zip(sizes, sizes[1:-1]):  # every block but the last follows the rule
        assert b == min(B, _round_up(int(a * f), 256))
        assert b % 256 == 0 or b == B
    if len(sizes) > 1:  # the last block takes what is left, at most the rule's size
        assert sizes[-1] <= min(B, _round_up(int(sizes[-2] * f), 256))


def test_doubling_reaches_full_blocks_after_three_steps():
    assert tg.tg_host_block_sizes(262144, 65536, 2.0) == [8192, 16384, 32768, 65536, 65536,
                                                          65536, 8192]
    # a host link as slow as the scan: equal blocks of 1/8, so no copy outlasts a scan
    assert set(tg.tg_host_block_sizes(262144, 65536, 1.0)) == {8192}
    assert tg.tg_host_block_sizes(3000, 2048, 2.0) == [256, 512, 1024, 1208]


def test_degenerate_sizes_and_bad_arguments():
    assert tg.tg_host_block_sizes(0, 1000, 2.0) == []
    assert tg.tg_host_block_sizes(3000, 100_000, 1.3) == [3000]
    for args in ((100, 0, 2.0), (-1, 100, 2.0), (100, 100, 0.5), (100, 100, 9.0)):
        with pytest.raises(tg.TgError):
            tg.tg_host_block_sizes(*args)
    assert sum(tg.tg_host_block_sizes(10_007, 4096, 1.5)) == 10_007
    with pytest.raises(tg.TgError):  # a list it will not build
        tg.tg_host_block_sizes(1 << 40, 1, 1.0)
    with pytest.raises(tg.TgError):  # block sizes beyond 2^32 markers are refused
        tg.tg_host_block_sizes(1000, (1 << 32) + 1, 2.0)
    # the largest block size allowed, with f * size far inside int64
    assert tg.tg_host_block_sizes(1 << 34, 1 << 32, 8.0) == [1 << 29, 1 << 32, 1 << 32, 1 << 32,
                                                             (1 << 34) - (1 << 29) - 3 * (1 << 32)]


def test_count_only_call_builds_no_list():
    """The count comes back without a size buffer (capacity 0), and a short buffer receives
    the first sizes only."""
    import ctypes as C
    lib = tg.load()
    n = C.c_int64(-1)
    assert lib.tg_host_block_sizes(262144, 65536, 2.0, None, 0, C.byref(n)) == tg.TG_OK
    assert n.value == 7
    buf = (C.c_int64 * 2)(-7, -7)
    assert lib.tg_host_block_sizes(262144, 65536, 2.0, buf, 2, C.byref(n)) == tg.TG_OK
    assert n.value == 7 and list(buf) == [8192, 16384]
