"""Batched solver: every instance of the batch follows the iteration it would
follow alone (same iteration count, same solution within round-off), including
an instance with a piecewise-constant coefficient."""
import numpy as np
import pytest

from paper_2009_01287_gb300 import inputs

pytestmark = pytest.mark.gpu


def _problems():
    coef = inputs.small_hp_mesh(8, base=4, depth=2, prob=0.4, pmax=6)
    coef = inputs.with_coeff(coef, inputs.base_parity_coeff(coef, 4))   # a in {1, 20}
    return [inputs.small_hp_mesh(1, base=4, depth=3, prob=0.4, pmax=5),
            inputs.random_refined_mesh(2, 5, 3, 0.35, 1, 4, seed=9, base_y=3),
            inputs.uniform_mesh(2, 3, 2),
            inputs.small_hp_mesh(7, base=6, depth=2, prob=0.3, pmin=2, pmax=7),
            coef]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_matches_single_solves(built_lib, cuda_device, precision):
    import torch
    B = built_lib
    prec = B.DG_PREC_FP64 if precision == "fp64" else B.DG_PREC_MIXED
    opts = B.make_options(precision=prec)
    meshes = _problems()
    n_rhs = 2
    bat = B.Batch(meshes, n_rhs=n_rhs, opts=opts)
    b = torch.empty(bat.n_dofs, dtype=torch.float64, device=cuda_device)
    singles = []
    for k, m in enumerate(meshes):
        M = B.Mesh(m, opts)
        pc = B.Precond(M, opts)
        for r in range(n_rhs):
            i = k * n_rhs + r
            seg = b[bat.offsets[i]:bat.offsets[i + 1]]
            rh = inputs.sine_rhs(2, 10 * k + r)
            B.dg_rhs_sine(M.h, rh.amps, rh.waves, seg)
            x1 = torch.empty_like(seg)
            info = B.dg_pcg_solve(M.h, pc.h, seg.clone(), x1, 1e-8, 3000)
            singles.append((info, x1))
    x = torch.empty_like(b)
    res, ms = bat.solve(b, x, 1e-8, 3000)
    assert ms > 0
    for i, (info, x1) in enumerate(singles):
        xi = x[bat.offsets[i]:bat.offsets[i + 1]]
        assert res[i].status == B.DG_OK and res[i].rel_res <= 1e-8
        if precision == "fp64":
            assert res[i].iters == info.iters
            assert float((xi - x1).abs().max()) <= 1e-10 * float(x1.abs().max())
        else:
            assert abs(res[i].iters - info.iters) <= 2
            assert float((xi - x1).abs().max()) <= 1e-6 * float(x1.abs().max())


def test_batch_zero_rhs_instance(built_lib, cuda_device):
    import torch
    B = built_lib
    bat = B.Batch(_problems()[:2], n_rhs=1)
    b = torch.zeros(bat.n_dofs, dtype=torch.float64, device=cuda_device)
    b[bat.offsets[1]:bat.offsets[2]] = 1.0
    x = torch.full_like(b, 5.0)
    res, _ = bat.solve(b, x, 1e-8, 3000)
    assert res[0].iters == 0 and float(x[:bat.offsets[1]].abs().max()) == 0.0
    assert res[1].iters > 0 and res[1].rel_res <= 1e-8


def test_batch_br2_matches_single_solves(built_lib, cuda_device):
    """BR2 in the batched form (explicit eta): the union carries every mesh's
    multiplied-out liftings, so each instance again follows its own solve."""
    import torch
    B = built_lib
    opts = B.make_options(form=B.DG_FORM_BR2, eta=8.0, precision=B.DG_PREC_FP64)
    meshes = _problems()[:3] + _problems()[4:]   # hanging levels, ragged, uniform, a in {1, 20}
    bat = B.Batch(meshes, n_rhs=1, opts=opts)
    b = torch.empty(bat.n_dofs, dtype=torch.float64, device=cuda_device)
    singles = []
    for k, m in enumerate(meshes):
        M = B.Mesh(m, opts)
        pc = B.Precond(M, opts)
        seg = b[bat.offsets[k]:bat.offsets[k + 1]]
        rh = inputs.sine_rhs(2, 30 + k)
        B.dg_rhs_sine(M.h, rh.amps, rh.waves, seg)
        x1 = torch.empty_like(seg)
        info = B.dg_pcg_solve(M.h, pc.h, seg.clone(), x1, 1e-8, 3000)
        singles.append((info, x1))
    x = torch.empty_like(b)
    res, _ = bat.solve(b, x, 1e-8, 3000)
    for k, (info, x1) in enumerate(singles):
        xk = x[bat.offsets[k]:bat.offsets[k + 1]]
        assert res[k].status == B.DG_OK and res[k].rel_res <= 1e-8
        assert res[k].iters == info.iters
        assert float((xk - x1).abs().max()) <= 1e-10 * float(x1.abs().max())
