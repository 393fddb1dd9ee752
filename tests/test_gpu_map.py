"""GPU parity on mapped squares (Section 2: element maps T_kappa onto general
quadrilaterals, bilinear or curved; the mapped operator kernel) through the C
ABI, against the oracle's mapped space.

Tolerances as for boxes: operator and FP64 preconditioner applies to 1e-12
relative (max-norm), PCG iterations within +-1 of the oracle, the mixed
FP32-preconditioner path within +10% iterations of the FP64 path.
"""
import numpy as np
import pytest

from oracle import dg, rhs, solver
from paper_2009_01287_gb300 import inputs

pytestmark = pytest.mark.gpu


def _coef(mesh, base):
    return inputs.with_coeff(mesh, inputs.base_parity_coeff(mesh, base))


MESHES = {
    "par-hp": lambda: inputs.with_corners(inputs.small_hp_mesh(1, base=4, depth=3, prob=0.4, pmax=5),
                                          inputs.PARALLELOGRAM),
    "quad-hp": lambda: inputs.with_corners(inputs.small_hp_mesh(2, base=3, depth=3, prob=0.5, pmin=1, pmax=8),
                                           inputs.QUADRILATERAL),
    "quad-high": lambda: inputs.with_corners(inputs.small_hp_mesh(5, base=2, depth=2, prob=0.5, pmin=7, pmax=8),
                                             inputs.QUADRILATERAL),
    "quad-single": lambda: inputs.with_corners(inputs.uniform_mesh(2, 1, 8), inputs.QUADRILATERAL),
    "quad-ragged": lambda: inputs.with_corners(inputs.random_refined_mesh(2, 5, 3, 0.35, 1, 4, seed=9, base_y=3),
                                               ((0.0, 0.0), (1.1, 0.2), (-0.1, 0.6), (0.9, 0.75))),
    "quad-coef": lambda: inputs.with_corners(_coef(inputs.small_hp_mesh(6, base=4, depth=3, prob=0.4, pmax=6), 4),
                                             inputs.QUADRILATERAL),
    # curved elements: the caller's smooth map (inputs.WavyMap) evaluated at setup
    "wavy-hp": lambda: inputs.with_mapping(inputs.small_hp_mesh(1, base=4, depth=3, prob=0.4, pmax=5),
                                           inputs.WavyMap()),
    "wavy-coef-p8": lambda: inputs.with_mapping(
        _coef(inputs.small_hp_mesh(3, base=3, depth=2, prob=0.5, pmin=5, pmax=8), 3), inputs.WavyMap(ax=0.1)),
}


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.fixture(scope="module")
def torch_mod(cuda_device):
    import torch
    return torch


def dev(torch, a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda")


def _opts(B, form, **kw):
    return B.make_options(form=B.DG_FORM_BR2 if form == "br2" else B.DG_FORM_SIPG, **kw)


@pytest.mark.parametrize("form", ["sipg", "br2"])
@pytest.mark.parametrize("name", list(MESHES))
def test_apply_parity_mapped(built_lib, torch_mod, name, form):
    mesh = MESHES[name]()
    prob = solver.build_problem(mesh, form=form)
    B = built_lib
    M = B.Mesh(mesh, _opts(B, form))
    x = inputs.random_vector(M.n_dofs, 3)
    xd = dev(torch_mod, x)
    yd = torch_mod.empty_like(xd)
    B.dg_apply(M.h, xd, yd)
    torch_mod.cuda.synchronize()
    assert rel(yd.cpu().numpy(), prob.A @ x) <= 1e-12
    yd2 = torch_mod.empty_like(xd)
    B.dg_apply(M.h, xd, yd2)
    torch_mod.cuda.synchronize()
    assert torch_mod.equal(yd, yd2)


@pytest.mark.parametrize("lor", ["exact", "amg"])
@pytest.mark.parametrize("name", ["par-hp", "quad-ragged", "quad-coef", "wavy-hp"])
def test_precond_parity_fp64_mapped(built_lib, torch_mod, name, lor):
    mesh = MESHES[name]()
    prob = solver.build_problem(mesh)
    opc = solver.Preconditioner(prob, lor=lor)
    B = built_lib
    o = B.make_options(lor=B.DG_LOR_EXACT if lor == "exact" else B.DG_LOR_AMG)
    M = B.Mesh(mesh, o)
    pc = B.Precond(M, o)
    r = inputs.random_vector(M.n_dofs, 4)
    rd = dev(torch_mod, r)
    zd = torch_mod.empty_like(rd)
    B.dg_precond_apply(pc.h, rd, zd)
    torch_mod.cuda.synchronize()
    assert rel(zd.cpu().numpy(), opc.apply(r)) <= 1e-12


@pytest.mark.parametrize("name,form", [("par-hp", "sipg"), ("quad-hp", "sipg"), ("quad-ragged", "sipg"),
                                       ("quad-coef", "sipg"), ("wavy-hp", "sipg"), ("wavy-coef-p8", "sipg"),
                                       ("quad-hp", "br2"), ("quad-coef", "br2"), ("wavy-hp", "br2")])
def test_pcg_iterations_match_oracle_mapped(built_lib, torch_mod, name, form):
    mesh = MESHES[name]()
    prob = solver.build_problem(mesh, form=form)
    opc = solver.Preconditioner(prob, lor="amg")
    rh = inputs.sine_rhs(2, 0)
    b = rhs.load_vector(prob.space, rh.amps, rh.waves)
    tol = 1e-8
    ref = solver.pcg(prob.A, b, opc.apply, tol, 2000)
    B = built_lib
    M = B.Mesh(mesh, _opts(B, form))
    pc = B.Precond(M, _opts(B, form))
    bd = dev(torch_mod, b)
    # the library's own load vector of the same right-hand side
    bl = torch_mod.empty_like(bd)
    B.dg_rhs_sine(M.h, rh.amps, rh.waves, bl)
    assert rel(bl.cpu().numpy(), b) <= 1e-12
    xd = torch_mod.empty_like(bd)
    info = B.dg_pcg_solve(M.h, pc.h, bd, xd, tol, 2000)
    assert info.status == 0 and info.rel_res <= tol
    assert abs(info.iters - ref.iters) <= 1
    assert rel(xd.cpu().numpy(), ref.x) <= 1e2 * tol
    # mixed precision: within +10% iterations, true FP64 residual at tolerance
    pc32 = B.Precond(M, _opts(B, form, precision=B.DG_PREC_MIXED))
    x32 = torch_mod.empty_like(bd)
    i32 = B.dg_pcg_solve(M.h, pc32.h, bd, x32, tol, 2000)
    assert i32.iters <= int(1.1 * info.iters) + 1
    r = torch_mod.empty_like(bd)
    B.dg_apply(M.h, x32, r)
    torch_mod.cuda.synchronize()
    assert float(torch_mod.linalg.norm(r - bd) / torch_mod.linalg.norm(bd)) <= 1.5e-8


@pytest.mark.parametrize("which", ["quad", "wavy"])
def test_full_size_mapped_sampled(built_lib, torch_mod, which):
    """The 98,127-DOF 2D hp-random workload on the general quadrilateral and on
    the curved domain: the apply in the launch configuration the benchmark
    times, on sampled elements whose rows the oracle computes one by one, and
    a mixed solve checked by its true FP64 residual."""
    mesh, rh = inputs.config1_mapped(0) if which == "quad" else inputs.config1_curved(0)
    B = built_lib
    M = B.Mesh(mesh)
    x = inputs.random_vector(M.n_dofs, 10)
    xd = dev(torch_mod, x)
    yd = torch_mod.empty_like(xd)
    B.dg_apply(M.h, xd, yd)
    torch_mod.cuda.synchronize()
    y = yd.cpu().numpy()
    from oracle.geometry import MappedDGSpace
    from oracle.topology import Topology
    topo = Topology(mesh.lo, mesh.size, mesh.p, mesh.extent)
    space = MappedDGSpace(topo, mesh.lattice_h, mesh.corners, mapping=mesh.mapping)
    rng = np.random.default_rng(0)
    for k in rng.choice(topo.n, size=40, replace=False):
        ref = dg.element_rows(space, int(k), x, 100.0)
        assert rel(y[space.offset[k]:space.offset[k + 1]], ref) <= 1e-12, int(k)
    pc = B.Precond(M, B.make_options(precision=B.DG_PREC_MIXED))
    bd = torch_mod.empty_like(xd)
    B.dg_rhs_sine(M.h, rh.amps, rh.waves, bd)
    xs = torch_mod.empty_like(xd)
    info = B.dg_pcg_solve(M.h, pc.h, bd, xs, 1e-8, 3000)
    assert info.status == 0
    B.dg_apply(M.h, xs, yd)
    torch_mod.cuda.synchronize()
    assert float(torch_mod.linalg.norm(yd - bd) / torch_mod.linalg.norm(bd)) <= 1.5e-8


def test_mapped_unsupported_forms(built_lib, torch_mod):
    B = built_lib
    mesh = MESHES["par-hp"]()
    with pytest.raises(B.DGError) as e:
        B.Batch([mesh], n_rhs=1)
    assert e.value.code == B.DG_EUNSUPPORTED
