"""Host checks of the tensor-core residual's bookkeeping (same formulas as the
kernel, no GPU): the work-item map covers every (row block, shift) exactly
once; the tile layout the split kernels write is the one the shared-memory
matrix descriptors describe (no swizzle, K-major core matrices of 8 rows x 16
bytes, 128 bytes apart along K and KG * 128 along rows); the issuing threads
own whole levels and split the 36 slice products evenly."""
import itertools

import pytest

KM, KN, KS, SL, GROUP = 128, 32, 32, 8, 16
KG = KS // 8


def task_coords(t, RB, cnt):
    full = (cnt // GROUP) * GROUP * RB
    if t < full:
        g, r = divmod(t, GROUP * RB)
        return r // GROUP, g * GROUP + r % GROUP
    gl = cnt - (cnt // GROUP) * GROUP
    r = t - full
    return r // gl, (cnt // GROUP) * GROUP + r % gl


def tile_off(row, k):
    return (((row >> 3) * KG + (k >> 3)) * 8 + (row & 7)) * 8 + (k & 7)


def level_owner(t, iss):
    if iss == 1:
        return 0
    o4 = t - 2 if t <= 5 else 9 - t
    return o4 if iss == 4 else (1 if o4 >= 2 else 0)


@pytest.mark.parametrize("RB,cnt", [(1, 1), (40, 2000), (3, 17), (8, 16), (5, 33), (79, 304), (2, 15)])
def test_work_items_cover_every_block_and_shift_once(RB, cnt):
    seen = [task_coords(t, RB, cnt) for t in range(RB * cnt)]
    assert len(set(seen)) == RB * cnt
    assert all(0 <= I < RB and 0 <= w < cnt for I, w in seen)
    # within a full group the 16 shifts of one row block are consecutive items
    if cnt >= GROUP:
        assert [task_coords(t, RB, cnt)[0] for t in range(GROUP)] == [0] * GROUP


@pytest.mark.parametrize("rows", [KM, KN])
def test_tile_layout_matches_descriptor_strides(rows):
    lbo, sbo = 128, KG * 128  # bytes: along K, along rows
    offs = set()
    for r, k in itertools.product(range(rows), range(KS)):
        b = 2 * tile_off(r, k)
        assert b == (r // 8) * sbo + (k // 8) * lbo + (r % 8) * 16 + (k % 8) * 2
        offs.add(b)
    assert offs == set(range(0, 2 * rows * KS, 2))  # dense, no overlap
    # the split kernels write 8 consecutive K elements of a row as one 16-byte vector
    for r in range(rows):
        for k8 in range(0, KS, 8):
            assert tile_off(r, k8) % 8 == 0
            assert [tile_off(r, k8 + e) for e in range(8)] == list(range(tile_off(r, k8), tile_off(r, k8) + 8))


@pytest.mark.parametrize("iss", [1, 2, 4])
def test_issuers_own_whole_levels_and_balance_the_products(iss):
    products = [0] * iss
    for t in range(2, SL + 2):
        ks = range(max(1, t - SL), min(SL, t - 1) + 1)
        products[level_owner(t, iss)] += len(ks)
    assert sum(products) == 36
    assert products == [36 // iss] * iss


def test_window_bound_and_stage_count():
    # 128 / KS stages per exact window; every level's window sum < 2^24
    assert 128 % KS == 0
    assert (SL) * 128 * 127 * 127 < 2 ** 24
    # one stage is 8 H tiles of 128 x KS and 8 Xhat tiles of 32 x KS BF16: 80 KB, two CTAs per SM
    stage = SL * (KM * KS + KN * KS) * 2
    assert stage == 81920 and 2 * (stage + 64) <= 227 * 1024


def test_two_32_row_tiles_side_by_side_form_one_64_row_tile():
    """The two-shift residual puts shift A's and shift B's Xhat slice tiles (32
    rows x 32 K each) next to each other and reads them as one 64-row B tile
    with the same strides: element (row, k) of the 64-row tile must be element
    (row mod 32, k) of tile row // 32."""
    KG = 32 // 8

    def off(row, k):
        return (((row >> 3) * KG + (k >> 3)) * 8 + (row & 7)) * 8 + (k & 7)

    tile = 32 * 32
    for row in range(64):
        for k in range(32):
            assert off(row, k) == (row // 32) * tile + off(row % 32, k)
