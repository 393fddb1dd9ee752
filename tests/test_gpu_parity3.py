"""GPU parity on cube meshes: the 3D operator (through the C ABI) against the
FP64 oracle, to 1e-12 relative (max-norm of the difference over the max-norm
of the oracle result), on hanging hp meshes, at degrees up to 8, and on the
full 3D hp-random workload (sampled elements); the load vector likewise."""
import numpy as np
import pytest

from oracle import dg, rhs, solver
from paper_2009_01287_gb300 import inputs

pytestmark = pytest.mark.gpu

MESHES3 = {
    "hp0": lambda: inputs.small_hp_mesh(0, base=2, depth=2, prob=0.5, pmin=1, pmax=4, dim=3),
    "hp1": lambda: inputs.small_hp_mesh(1, base=2, depth=2, prob=0.5, pmin=1, pmax=5, dim=3),
    "p8": lambda: inputs.small_hp_mesh(1, base=2, depth=1, prob=0.2, pmin=6, pmax=8, dim=3),
    "single": lambda: inputs.uniform_mesh(3, 1, 4),
    "ragged": lambda: inputs.random_refined_mesh(3, 3, 2, 0.3, 1, 3, seed=4),
}


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.fixture(scope="module")
def torch_mod(cuda_device):
    import torch
    return torch


def dev(torch, a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("form", ["sipg", "br2"])
@pytest.mark.parametrize("name", list(MESHES3))
def test_apply3_parity(built_lib, torch_mod, name, form):
    mesh = MESHES3[name]()
    _, space, A = solver.build_operator(mesh, form=form)
    B = built_lib
    M = B.Mesh(mesh, B.make_options(form=B.DG_FORM_BR2 if form == "br2" else B.DG_FORM_SIPG))
    assert M.n_dofs == space.n
    x = inputs.random_vector(M.n_dofs, 3)
    xd = dev(torch_mod, x)
    yd = torch_mod.empty_like(xd)
    B.dg_apply(M.h, xd, yd)
    torch_mod.cuda.synchronize()
    assert rel(yd.cpu().numpy(), A @ x) <= 1e-12
    yd2 = torch_mod.empty_like(xd)
    B.dg_apply(M.h, xd, yd2)
    torch_mod.cuda.synchronize()
    assert torch_mod.equal(yd, yd2)


def test_rhs3_parity(built_lib, torch_mod):
    mesh = MESHES3["hp1"]()
    _, space, _ = solver.build_operator(mesh)
    r = inputs.sine_rhs(3, 2)
    B = built_lib
    M = B.Mesh(mesh)
    bd = torch_mod.empty(M.n_dofs, dtype=torch_mod.float64, device="cuda")
    B.dg_rhs_sine(M.h, r.amps, r.waves, bd)
    torch_mod.cuda.synchronize()
    assert rel(bd.cpu().numpy(), rhs.load_vector(space, r.amps, r.waves)) <= 1e-12


def test_precond3_unsupported(built_lib, torch_mod):
    B = built_lib
    M = B.Mesh(MESHES3["hp0"]())
    with pytest.raises(B.DGError) as e:
        B.Precond(M)
    assert e.value.code == B.DG_EUNSUPPORTED


def test_full_size_config2_sampled(built_lib, torch_mod):
    """Full 3D hp-random workload (16^3 base, depth 2, p ~ U{1..5}, BR2): the
    apply checked on sampled elements whose rows the oracle computes one by one."""
    mesh, _ = inputs.config2(0)
    B = built_lib
    M = B.Mesh(mesh, B.make_options(form=B.DG_FORM_BR2))
    x = inputs.random_vector(M.n_dofs, 10)
    xd = dev(torch_mod, x)
    yd = torch_mod.empty_like(xd)
    B.dg_apply(M.h, xd, yd)
    torch_mod.cuda.synchronize()
    y = yd.cpu().numpy()
    from oracle.dg import DGSpace
    from oracle.topology3 import Topology3
    topo = Topology3(mesh.lo, mesh.size, mesh.p, mesh.extent)
    space = DGSpace(topo, mesh.lattice_h)
    eta = dg.br2_eta(topo)
    assert M.n_dofs == space.n
    rng = np.random.default_rng(0)
    for k in rng.choice(topo.n, size=30, replace=False):
        ref = dg.element_rows(space, int(k), x, eta, form="br2")
        got = y[space.offset[k]:space.offset[k + 1]]
        assert rel(got, ref) <= 1e-12, int(k)
