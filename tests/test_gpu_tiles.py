"""Tile tuner (dg_options.tune_tiles): the operator kernel is timed over
candidate tile shapes at creation and the fastest is kept.  Whatever it
chooses, the apply stays within 1e-12 of the oracle (squares and cubes) and
the batched solve gives the same iterations as with the fixed tiles."""
import numpy as np
import pytest

from oracle import solver
from paper_2009_01287_gb300 import inputs

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("dim,form", [(2, "sipg"), (2, "br2"), (3, "br2")])
def test_tuned_tiles_keep_apply_parity(built_lib, cuda_device, dim, form):
    import torch
    B = built_lib
    if dim == 2:
        mesh = inputs.small_hp_mesh(2, base=6, depth=3, prob=0.5, pmin=1, pmax=8)
    else:
        mesh = inputs.small_hp_mesh(0, base=3, depth=2, prob=0.4, pmin=1, pmax=4, dim=3)
    fcode = B.DG_FORM_BR2 if form == "br2" else B.DG_FORM_SIPG
    _, _, A = solver.build_operator(mesh, form=form)
    M = B.Mesh(mesh, B.make_options(form=fcode, tune_tiles=1))
    st = M.stats
    assert st.tiles_tuned == 1 and st.apply_ms_tuned > 0 and st.apply_ms_tuned <= st.apply_ms_fixed
    if dim == 2:
        caps = [min(16, 256 // (p + 1) ** 2) for p in range(1, 9)]
        assert all(1 <= st.tile_elems[p] <= caps[p - 1] for p in range(1, 9))
    else:
        assert st.tile_smem_budget in (8 * 6656, 8 * 9216, 8 * 13312)
    x = inputs.random_vector(M.n_dofs, 41)
    xd = torch.tensor(x, dtype=torch.float64, device=cuda_device)
    yd = torch.empty_like(xd)
    B.dg_apply(M.h, xd, yd)
    torch.cuda.synchronize()
    assert rel(yd.cpu().numpy(), A @ x) <= 1e-12


def test_tuned_batch_matches_fixed(built_lib, cuda_device):
    import torch
    B = built_lib
    meshes = [inputs.config3_problem(k, dof_hi=20000)[0] for k in range(4)]
    out = []
    for tune in (0, 1):
        bat = B.Batch(meshes, n_rhs=2, opts=B.make_options(precision=B.DG_PREC_MIXED, tune_tiles=tune))
        b = torch.empty(bat.n_dofs, dtype=torch.float64, device=cuda_device)
        bat.rhs_sine([inputs.sine_rhs(2, 50 + i) for i in range(bat.n_inst)], b)
        x = torch.empty_like(b)
        res, _ = bat.solve(b, x, 1e-8, 3000)
        out.append(([r.iters for r in res], x.cpu().numpy(), bat.stats))
        bat.close()
    assert out[1][2].tiles_tuned == 1
    assert all(abs(a - b) <= 1 for a, b in zip(out[0][0], out[1][0]))
    assert np.abs(out[0][1] - out[1][1]).max() <= 1e-6 * np.abs(out[0][1]).max()
