"""GPU parity on the full 2D hp-random workload (32x32 base squares refined at
random with probability 0.3 to depth 3, p ~ U{1..6}, seed 0: 98,127 DOFs), in
the launch configuration the benchmark times, SIPG (eta = 100) and BR2 (eta =
the largest number of sub-faces of one element), against the FP64 oracle
assembled at the same size.

Bars (Section 4.1: PCG to a relative residual of 1e-8):
- operator apply and FP64 preconditioner apply: 1e-12 relative (max-norm);
- FP64 PCG: iterations within +-1 of the oracle's, solution within 1e2 tol;
- mixed PCG (FP32 preconditioner, FP64 operator / residual / dots): at most
  10% more iterations than the oracle, its true FP64 residual below 1.5 tol,
  and its distance to the oracle's solution stated (recorded as a test
  property and printed) and within 1e2 tol.
"""
import numpy as np
import pytest

from oracle import dg, rhs, solver
from paper_2009_01287_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-8


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.fixture(scope="module", params=["sipg", "br2"])
def full(request, cuda_device, built_lib):
    import torch
    form = request.param
    mesh, rh = inputs.config1(0)
    prob = solver.build_problem(mesh, form=form)
    opc = solver.Preconditioner(prob, lor="amg")
    b = rhs.load_vector(prob.space, rh.amps, rh.waves)
    ref = solver.pcg(prob.A, b, opc.apply, TOL, 5000)
    assert ref.converged
    B = built_lib
    eta = dg.br2_eta(prob.topo) if form == "br2" else 100.0
    fcode = B.DG_FORM_BR2 if form == "br2" else B.DG_FORM_SIPG
    M = B.Mesh(mesh, B.make_options(form=fcode, eta=eta))
    pc64 = B.Precond(M, B.make_options(form=fcode, eta=eta, lor=B.DG_LOR_AMG))
    pc32 = B.Precond(M, B.make_options(form=fcode, eta=eta, lor=B.DG_LOR_AMG, precision=B.DG_PREC_MIXED))
    return dict(torch=torch, B=B, form=form, prob=prob, opc=opc, b=b, ref=ref, M=M, pc64=pc64, pc32=pc32)


def _dev(F, a):
    return F["torch"].tensor(np.asarray(a), dtype=F["torch"].float64, device="cuda")


def test_full_apply_whole_vector(full):
    F = full
    torch, B, M = F["torch"], F["B"], F["M"]
    assert M.n_dofs == F["prob"].space.n == 98127
    x = inputs.random_vector(M.n_dofs, 21)
    xd = _dev(F, x)
    yd = torch.empty_like(xd)
    B.dg_apply(M.h, xd, yd)
    torch.cuda.synchronize()
    assert rel(yd.cpu().numpy(), F["prob"].A @ x) <= 1e-12


def test_full_precond_fp64(full):
    F = full
    torch, B = F["torch"], F["B"]
    r = inputs.random_vector(F["M"].n_dofs, 22)
    rd = _dev(F, r)
    zd = torch.empty_like(rd)
    B.dg_precond_apply(F["pc64"].h, rd, zd)
    torch.cuda.synchronize()
    assert rel(zd.cpu().numpy(), F["opc"].apply(r)) <= 1e-12


def test_full_precond_mixed(full):
    F = full
    torch, B = F["torch"], F["B"]
    r = inputs.random_vector(F["M"].n_dofs, 23)
    rd = _dev(F, r)
    zd = torch.empty_like(rd)
    B.dg_precond_apply(F["pc32"].h, rd, zd)
    torch.cuda.synchronize()
    assert rel(zd.cpu().numpy(), F["opc"].apply(r)) <= 1e-4


def test_full_pcg_fp64(full, record_property):
    F = full
    torch, B, M, ref = F["torch"], F["B"], F["M"], F["ref"]
    bd = _dev(F, F["b"])
    xd = torch.empty_like(bd)
    info = B.dg_pcg_solve(M.h, F["pc64"].h, bd, xd, TOL, 5000)
    err = rel(xd.cpu().numpy(), ref.x)
    record_property("fp64_iters", info.iters)
    record_property("oracle_iters", ref.iters)
    record_property("fp64_oracle_rel_err", err)
    print(f"\n[{F['form']}] FP64 PCG {info.iters} iterations (oracle {ref.iters}), "
          f"solution vs oracle {err:.3e}")
    assert info.status == 0 and info.rel_res <= TOL
    assert abs(info.iters - ref.iters) <= 1
    assert err <= 1e2 * TOL


def test_full_pcg_mixed(full, record_property):
    F = full
    torch, B, M, ref = F["torch"], F["B"], F["M"], F["ref"]
    bd = _dev(F, F["b"])
    xd = torch.empty_like(bd)
    info = B.dg_pcg_solve(M.h, F["pc32"].h, bd, xd, TOL, 5000)
    # true residual of the mixed solution with the FP64 operator
    rd = torch.empty_like(bd)
    B.dg_apply(M.h, xd, rd)
    torch.cuda.synchronize()
    true_res = float(torch.linalg.norm(rd - bd) / torch.linalg.norm(bd))
    err = rel(xd.cpu().numpy(), ref.x)
    record_property("mixed_iters", info.iters)
    record_property("oracle_iters", ref.iters)
    record_property("mixed_oracle_rel_err", err)
    print(f"\n[{F['form']}] mixed PCG {info.iters} iterations (oracle {ref.iters}), "
          f"true residual {true_res:.3e}, solution vs oracle {err:.3e}")
    assert info.status == 0 and info.rel_res <= TOL
    assert info.iters <= int(1.1 * ref.iters)
    assert true_res <= 1.5 * TOL
    assert err <= 1e2 * TOL
