"""Host planning of the preconditioner kernels' work lists (no GPU): the CSR
row tiers and the V_e block-solve units cover every row and every block row
exactly once, with the sizes and orders the kernels rely on."""
import numpy as np
import pytest


def _group_for(avg):
    g = 1
    while g < 32 and g * 2 <= avg:
        g *= 2
    return g


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_csr_tiers_cover_every_row_once(built_lib, seed):
    rng = np.random.default_rng(seed)
    n = 3000
    lens = rng.integers(0, 12, size=n)                      # mostly short rows
    lens[rng.choice(n, 60, replace=False)] = rng.integers(65, 1024, size=60)
    lens[rng.choice(n, 9, replace=False)] = rng.integers(1025, 5000, size=9)
    lens[5] = 1024                                          # the CTA threshold itself stays a warp row
    ptr = np.concatenate([[0], np.cumsum(lens)])
    group, long_min, cta, warp = built_lib.plan_csr_tiers(ptr)
    short = lens[lens <= 64]
    assert group == max(1, _group_for(short.mean()) // 2)
    assert long_min == (1024 if group >= 32 else max(8 * group, 16))
    assert set(cta) == set(np.flatnonzero(lens > 1024))
    assert set(warp) == set(np.flatnonzero((lens > long_min) & (lens <= 1024)))
    assert len(set(cta)) == len(cta) and len(set(warp)) == len(warp)
    for lst in (cta, warp):   # longest first, ties in row order
        key = [(-lens[r], r) for r in lst]
        assert key == sorted(key)


def test_csr_tiers_of_empty_and_uniform_matrices(built_lib):
    g, lm, cta, warp = built_lib.plan_csr_tiers(np.zeros(1, dtype=np.int64))
    assert len(cta) == 0 and len(warp) == 0
    ptr = np.arange(0, 41 * 40, 40)                         # 40 rows of 40 entries
    g, lm, cta, warp = built_lib.plan_csr_tiers(ptr)
    assert g == 16 and lm == 128 and len(cta) == 0 and len(warp) == 0


def _check_units(dims, unit, ubase, brec, slot, inv_off):
    n = len(dims)
    seen_rows = np.zeros(n, dtype=np.int64)
    packed = np.zeros(n, dtype=np.int64)
    by_slot = {int(s): i for i, s in enumerate(slot)}
    work = []
    for u, (h, ub) in enumerate(zip(unit, ubase)):
        if h[3] == 0:                                        # 32-row panel of a large block
            b = by_slot[int(h[0])]
            assert h[1] == dims[b] > 16 and h[2] % 32 == 0 and 0 <= h[2] < dims[b]
            assert ub == inv_off[b] + h[2]
            seen_rows[b] += min(32, dims[b] - h[2])
            work.append(dims[b])
        else:                                                # small blocks packed side by side
            W, first, cnt = int(h[3]), int(h[0]), int(h[1])
            assert W in (4, 8, 16) and 1 <= cnt <= 32 // W and h[2] == 0 and ub == 0
            for j in range(first, first + cnt):
                s, d, lo, hi = (int(v) for v in brec[j])
                b = by_slot[s]
                assert d == dims[b] and d <= W and (W == 4 or d > W // 2)
                assert (lo & 0xffffffff) | (hi << 32) == inv_off[b]
                packed[b] += 1
                work.append(d)
    big = dims > 16
    assert np.array_equal(seen_rows[big], dims[big]) and not seen_rows[~big].any()
    assert np.all(packed[~big] == 1) and not packed[big].any()
    assert work == sorted(work, reverse=True)                # largest blocks first


@pytest.mark.parametrize("seed", [0, 1])
def test_block_units_cover_every_block_row_once(built_lib, seed):
    rng = np.random.default_rng(seed)
    dims = np.concatenate([rng.integers(1, 17, size=400), rng.integers(17, 300, size=40), [16, 17, 32, 33, 8, 4, 5]])
    rng.shuffle(dims)
    slot = np.concatenate([[0], np.cumsum(dims)[:-1]]).astype(np.int32)
    inv_off = np.concatenate([[0], np.cumsum(dims.astype(np.int64) ** 2)[:-1]]) + (5 << 32)   # above 2^32
    unit, ubase, brec = built_lib.plan_block_units(dims, slot, inv_off)
    _check_units(dims, unit, ubase, brec, slot, inv_off)


def test_block_units_reject_oversized_blocks(built_lib):
    with pytest.raises(built_lib.DGError):
        built_lib.plan_block_units([8193], [0], [0])
