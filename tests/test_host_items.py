"""Host planning of the operator's sub-face items (no GPU).  The kernels take a
tile's items (squares) or a chunk's items (cubes) in an order sorted by the
branches their threads take, and write every item's partials at the item's
position in sub-face order, which the per-node sums then read in order.  These
tests check that the sorted lists are permutations of that order within each
tile or chunk, that the position fields invert the permutation, that the keys
are sorted (ties in sub-face order), and that every sub-face record appears
exactly once."""
import numpy as np
import pytest

from paper_2009_01287_gb300 import inputs


def _key(dim, br2, interior, pn, full):
    if dim == 2:   # interior first by neighbour degree (descending), the boundary last
        return 16 - pn if interior else 32
    zv = 1 if (br2 and not (full & 1)) else 0
    yy = 1 if (br2 and interior and not (full & 2)) else 0
    return ((0 if interior else 1) << 12) | (zv << 11) | (yy << 10) | ((16 - pn) if interior else 0)


def _check(B, mesh, form):
    br2 = form == "br2"
    hs = B.HostSetup(mesh, B.make_options(form=B.DG_FORM_BR2 if br2 else B.DG_FORM_SIPG), amg=False)
    ptr, items, chunk, info = hs.face_items()
    dim = mesh.dim
    n = len(items)
    assert n > 0 and ptr[0] == 0 and ptr[-1] == n
    rec = items[:, 0]
    assert sorted(rec.tolist()) == list(range(n))          # every sub-face record once
    side = items[:, 1] & 0xFFFF
    pos = items[:, 1] >> 16
    n_sorted_chunks = 0
    for t in range(len(ptr) - 1):
        a, b, c = int(ptr[t]), int(ptr[t + 1]), int(chunk[t])
        assert c >= 1 or a == b
        prev_side = -1
        prev_rec = -1
        for c0 in range(a, b, max(c, 1)):
            c1 = min(c0 + c, b)
            m = c1 - c0
            p = pos[c0:c1]
            assert sorted(p.tolist()) == list(range(m))      # a permutation of the chunk
            keys = [_key(dim, br2, int(info[g, 0]), int(info[g, 1]), int(info[g, 2])) for g in range(c0, c1)]
            for g in range(m - 1):                          # sorted, ties in sub-face order
                assert (keys[g], p[g]) < (keys[g + 1], p[g + 1])
            # sub-face order restored from the positions: sides in element order,
            # a side's sub-faces as consecutive records
            orig = np.empty(m, dtype=np.int64)
            orig[p] = np.arange(c0, c1)
            for g in orig:
                s = int(side[g])
                assert s >= prev_side
                if s == prev_side:
                    assert rec[g] == prev_rec + 1
                prev_side, prev_rec = s, int(rec[g])
            n_sorted_chunks += int(any(p[g] != g for g in range(m)))
    return n_sorted_chunks


@pytest.mark.parametrize("form", ["sipg", "br2"])
@pytest.mark.parametrize("seed", [0, 3])
def test_square_items_sorted_within_tiles(built_lib, seed, form):
    mesh = inputs.small_hp_mesh(seed, base=4, depth=3, prob=0.4, pmax=6)
    # on an hp mesh with hanging sides some tile has items out of sub-face order
    assert _check(built_lib, mesh, form) > 0


@pytest.mark.parametrize("form", ["sipg", "br2"])
@pytest.mark.parametrize("seed", [1, 2])
def test_cube_items_sorted_within_chunks(built_lib, seed, form):
    mesh = inputs.small_hp_mesh(seed, base=3, depth=2, prob=0.3, pmax=4, dim=3)
    assert _check(built_lib, mesh, form) > 0


def test_uniform_mesh_items_keep_boundary_last(built_lib):
    # conforming, one degree: only interior / boundary differ, and the boundary items close each tile
    mesh = inputs.uniform_mesh(2, 4, 2)
    _check(built_lib, mesh, "sipg")
    hs = built_lib.HostSetup(mesh, built_lib.make_options(), amg=False)
    ptr, items, chunk, info = hs.face_items()
    for t in range(len(ptr) - 1):
        inter = info[ptr[t]:ptr[t + 1], 0]
        k = int(inter.sum())
        assert (inter[:k] == 1).all() and (inter[k:] == 0).all()
