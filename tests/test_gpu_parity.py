"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances: operator and FP64 preconditioner applies to 1e-12 relative
(max-norm of the difference over the max-norm of the oracle result); PCG
iteration counts within +-1 of the oracle at the same tolerance; the mixed
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
    "cfg0": (lambda: inputs.config0()[0], 10.0, "p1sq"),
    "hp-a": (lambda: inputs.small_hp_mesh(1, base=4, depth=3, prob=0.4, pmax=5), None, "paper"),
    "hp-b": (lambda: inputs.small_hp_mesh(2, base=3, depth=3, prob=0.5, pmin=1, pmax=8), None, "paper"),
    "hp-high": (lambda: inputs.small_hp_mesh(5, base=2, depth=2, prob=0.5, pmin=7, pmax=8), None, "paper"),
    "single": (lambda: inputs.uniform_mesh(2, 1, 8), None, "paper"),
    "ragged": (lambda: inputs.random_refined_mesh(2, 5, 3, 0.35, 1, 4, seed=9, base_y=3), None, "paper"),
    # piecewise-constant coefficient a in {1, 20} by base-cell parity (Section 4.3)
    "coef-a": (lambda: _coef(inputs.small_hp_mesh(6, base=4, depth=3, prob=0.4, pmax=6), 4), None, "paper"),
    "coef-b": (lambda: _coef(inputs.small_hp_mesh(7, base=3, depth=2, prob=0.5, pmin=2, pmax=8), 3), None, "paper"),
}


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _opts(B, form, eta, pform, **kw):
    return B.make_options(form=B.DG_FORM_BR2 if form == "br2" else B.DG_FORM_SIPG, eta=eta or 0.0,
                          penalty_form=B.DG_PENALTY_P1SQ if pform == "p1sq" else B.DG_PENALTY_PAPER, **kw)


@pytest.fixture(scope="module")
def torch_mod(cuda_device):
    import torch
    return torch


def dev(torch, a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("form", ["sipg", "br2"])
@pytest.mark.parametrize("name", list(MESHES))
def test_apply_parity(built_lib, torch_mod, name, form):
    mk, eta, pform = MESHES[name]
    mesh = mk()
    prob = solver.build_problem(mesh, form=form, eta=eta, penalty_form=pform)
    B = built_lib
    M = B.Mesh(mesh, _opts(B, form, eta, pform))
    x = inputs.random_vector(M.n_dofs, 3)
    xd = dev(torch_mod, x)
    yd = torch_mod.empty_like(xd)
    B.dg_apply(M.h, xd, yd)
    torch_mod.cuda.synchronize()
    y = yd.cpu().numpy()
    assert rel(y, prob.A @ x) <= 1e-12
    # deterministic: a second apply is bit-identical
    yd2 = torch_mod.empty_like(xd)
    B.dg_apply(M.h, xd, yd2)
    torch_mod.cuda.synchronize()
    assert torch_mod.equal(yd, yd2)


@pytest.mark.parametrize("lor", ["exact", "amg"])
@pytest.mark.parametrize("name", ["cfg0", "hp-a", "hp-b", "ragged", "coef-a"])
def test_precond_parity_fp64(built_lib, torch_mod, name, lor):
    mk, eta, pform = MESHES[name]
    mesh = mk()
    prob = solver.build_problem(mesh, eta=eta, penalty_form=pform)
    opc = solver.Preconditioner(prob, lor=lor)
    B = built_lib
    o = _opts(B, "sipg", eta, pform, lor=B.DG_LOR_EXACT if lor == "exact" else B.DG_LOR_AMG)
    M = B.Mesh(mesh, o)
    pc = B.Precond(M, o)
    r = inputs.random_vector(M.n_dofs, 4)
    rd = dev(torch_mod, r)
    zd = torch_mod.empty_like(rd)
    B.dg_precond_apply(pc.h, rd, zd)
    torch_mod.cuda.synchronize()
    assert rel(zd.cpu().numpy(), opc.apply(r)) <= 1e-12


def test_precond_jacobi_only_fp64(built_lib, torch_mod):
    mk, eta, pform = MESHES["hp-a"]
    mesh = mk()
    prob = solver.build_problem(mesh)
    opc = solver.Preconditioner(prob, lor="amg", smoother="jacobi_only")
    B = built_lib
    o = _opts(B, "sipg", None, "paper", smoother=B.DG_SMOOTHER_JACOBI_ONLY)
    M = B.Mesh(mesh, o)
    pc = B.Precond(M, o)
    r = inputs.random_vector(M.n_dofs, 6)
    rd = dev(torch_mod, r)
    zd = torch_mod.empty_like(rd)
    B.dg_precond_apply(pc.h, rd, zd)
    torch_mod.cuda.synchronize()
    assert rel(zd.cpu().numpy(), opc.apply(r)) <= 1e-12


def test_precond_mixed_close(built_lib, torch_mod):
    """FP32 preconditioner: within FP32 round-off of the FP64 oracle."""
    mk, eta, pform = MESHES["hp-a"]
    mesh = mk()
    prob = solver.build_problem(mesh)
    opc = solver.Preconditioner(prob, lor="amg")
    B = built_lib
    o = _opts(B, "sipg", None, "paper", precision=B.DG_PREC_MIXED)
    M = B.Mesh(mesh, o)
    pc = B.Precond(M, o)
    r = inputs.random_vector(M.n_dofs, 7)
    rd = dev(torch_mod, r)
    zd = torch_mod.empty_like(rd)
    B.dg_precond_apply(pc.h, rd, zd)
    torch_mod.cuda.synchronize()
    assert rel(zd.cpu().numpy(), opc.apply(r)) <= 1e-4


@pytest.mark.parametrize("name,lor,form,tol", [("cfg0", "exact", "sipg", 1e-10), ("hp-a", "amg", "sipg", 1e-8),
                                               ("hp-b", "amg", "br2", 1e-8), ("ragged", "amg", "sipg", 1e-8),
                                               ("coef-a", "amg", "sipg", 1e-8), ("coef-b", "amg", "br2", 1e-8)])
def test_pcg_iterations_match_oracle(built_lib, torch_mod, name, lor, form, tol):
    mk, eta, pform = MESHES[name]
    mesh = mk()
    prob = solver.build_problem(mesh, form=form, eta=eta, penalty_form=pform)
    opc = solver.Preconditioner(prob, lor=lor)
    rh = inputs.sine_rhs(2, 0)
    b = rhs.load_vector(prob.space, rh.amps, rh.waves)
    ref = solver.pcg(prob.A, b, opc.apply, tol, 2000)
    B = built_lib
    o = _opts(B, form, eta, pform, lor=B.DG_LOR_EXACT if lor == "exact" else B.DG_LOR_AMG)
    M = B.Mesh(mesh, o)
    pc = B.Precond(M, o)
    bd = dev(torch_mod, b)
    xd = torch_mod.empty_like(bd)
    info = B.dg_pcg_solve(M.h, pc.h, bd, xd, tol, 2000)
    assert info.status == 0 and info.rel_res <= tol
    assert abs(info.iters - ref.iters) <= 1
    x = xd.cpu().numpy()
    assert rel(x, ref.x) <= 1e2 * tol


@pytest.mark.parametrize("name", ["hp-a", "ragged"])
def test_pcg_mixed_within_ten_percent(built_lib, torch_mod, name):
    mk, eta, pform = MESHES[name]
    mesh = mk()
    B = built_lib
    M = B.Mesh(mesh, _opts(B, "sipg", eta, pform))
    pc64 = B.Precond(M, _opts(B, "sipg", eta, pform))
    pc32 = B.Precond(M, _opts(B, "sipg", eta, pform, precision=B.DG_PREC_MIXED))
    bd = torch_mod.empty(M.n_dofs, dtype=torch_mod.float64, device="cuda")
    rh = inputs.sine_rhs(2, 1)
    B.dg_rhs_sine(M.h, rh.amps, rh.waves, bd)
    x64 = torch_mod.empty_like(bd)
    x32 = torch_mod.empty_like(bd)
    i64 = B.dg_pcg_solve(M.h, pc64.h, bd, x64, 1e-8, 2000)
    i32 = B.dg_pcg_solve(M.h, pc32.h, bd, x32, 1e-8, 2000)
    assert i32.rel_res <= 1e-8
    assert i32.iters <= int(1.1 * i64.iters) + 1
    # the true residual of the mixed solution, with the FP64 operator
    r = torch_mod.empty_like(bd)
    B.dg_apply(M.h, x32, r)
    torch_mod.cuda.synchronize()
    assert float(torch_mod.linalg.norm(r - bd) / torch_mod.linalg.norm(bd)) <= 1.5e-8


def test_rhs_matches_oracle(built_lib, torch_mod):
    mesh = MESHES["hp-b"][0]()
    prob = solver.build_problem(mesh)
    rh = inputs.sine_rhs(2, 3)
    B = built_lib
    M = B.Mesh(mesh)
    bd = torch_mod.empty(M.n_dofs, dtype=torch_mod.float64, device="cuda")
    B.dg_rhs_sine(M.h, rh.amps, rh.waves, bd)
    assert rel(bd.cpu().numpy(), rhs.load_vector(prob.space, rh.amps, rh.waves)) <= 1e-12


def test_pcg_host_entry_identical(built_lib, torch_mod):
    mesh = MESHES["hp-a"][0]()
    B = built_lib
    M = B.Mesh(mesh)
    pc = B.Precond(M)
    b = inputs.random_vector(M.n_dofs, 8)
    xd = torch_mod.empty(M.n_dofs, dtype=torch_mod.float64, device="cuda")
    i1 = B.dg_pcg_solve(M.h, pc.h, dev(torch_mod, b), xd, 1e-8, 1000)
    xh = np.zeros(M.n_dofs)
    i2 = B.dg_pcg_solve_host(M.h, pc.h, b, xh, 1e-8, 1000)
    assert i1.iters == i2.iters
    assert np.array_equal(xd.cpu().numpy(), xh)


def test_zero_rhs_and_maxit(built_lib, torch_mod):
    mesh = MESHES["hp-a"][0]()
    B = built_lib
    M = B.Mesh(mesh)
    pc = B.Precond(M)
    b = torch_mod.zeros(M.n_dofs, dtype=torch_mod.float64, device="cuda")
    x = torch_mod.full_like(b, 7.0)
    info = B.dg_pcg_solve(M.h, pc.h, b, x, 1e-8, 100)
    assert info.iters == 0 and float(x.abs().max()) == 0.0
    b = dev(torch_mod, inputs.random_vector(M.n_dofs, 9))
    info = B.dg_pcg_solve(M.h, pc.h, b, x, 1e-14, 3, raise_on_notconv=False)
    assert info.status == B.DG_ENOTCONV and info.iters == 3


def test_full_size_config1_sampled(built_lib, torch_mod):
    """Full 2D hp-random workload (32x32 base, depth 3): the apply in the
    launch configuration the benchmark times, checked on sampled elements
    whose rows the oracle computes one by one."""
    mesh, _ = inputs.config1(0)
    B = built_lib
    M = B.Mesh(mesh)
    x = inputs.random_vector(M.n_dofs, 10)
    xd = dev(torch_mod, x)
    yd = torch_mod.empty_like(xd)
    B.dg_apply(M.h, xd, yd)
    torch_mod.cuda.synchronize()
    y = yd.cpu().numpy()
    from oracle.dg import DGSpace
    from oracle.topology import Topology
    topo = Topology(mesh.lo, mesh.size, mesh.p, mesh.extent)
    space = DGSpace(topo, mesh.lattice_h)
    rng = np.random.default_rng(0)
    ks = rng.choice(topo.n, size=40, replace=False)
    for k in ks:
        ref = dg.element_rows(space, int(k), x, 100.0)
        got = y[space.offset[k]:space.offset[k + 1]]
        assert rel(got, ref) <= 1e-12, int(k)


def test_pcg_host_loop_matches_graph(built_lib, torch_mod, monkeypatch):
    """The host-driven PCG loop (graphs disabled) stops at the same iteration
    and returns the same iterate as the graph-launched loop."""
    mesh = MESHES["hp-a"][0]()
    B = built_lib
    M = B.Mesh(mesh)
    b = dev(torch_mod, inputs.random_vector(M.n_dofs, 12))
    pc_g = B.Precond(M)
    xg = torch_mod.empty_like(b)
    ig = B.dg_pcg_solve(M.h, pc_g.h, b, xg, 1e-10, 2000)
    monkeypatch.setenv("DG_PCG_GRAPH", "0")
    pc_h = B.Precond(M)
    xh = torch_mod.empty_like(b)
    ih = B.dg_pcg_solve(M.h, pc_h.h, b, xh, 1e-10, 2000)
    assert ih.iters == ig.iters
    assert torch_mod.equal(xg, xh)


def test_one_graph_serves_any_buffers_and_tolerance(built_lib, torch_mod):
    """The solve graph is captured once per preconditioner (at setup) on the
    handle's own copies of b and x, with the limits in device memory: solves
    with other buffers, tolerances and limits on the same handle match solves
    on fresh handles."""
    mesh = MESHES["hp-a"][0]()
    B = built_lib
    M = B.Mesh(mesh)
    pc = B.Precond(M)
    runs = [(12, 1e-6, 2000), (13, 1e-10, 2000), (12, 1e-10, 5)]
    got = []
    for seed, tol, maxit in runs:
        b = dev(torch_mod, inputs.random_vector(M.n_dofs, seed))
        x = torch_mod.full_like(b, 5.0)
        info = B.dg_pcg_solve(M.h, pc.h, b, x, tol, maxit, raise_on_notconv=False)
        got.append((info.iters, info.status, x.clone()))
    for (seed, tol, maxit), (it, st, x) in zip(runs, got):
        M2 = B.Mesh(mesh)
        pc2 = B.Precond(M2)
        b = dev(torch_mod, inputs.random_vector(M2.n_dofs, seed))
        x2 = torch_mod.empty_like(b)
        info = B.dg_pcg_solve(M2.h, pc2.h, b, x2, tol, maxit, raise_on_notconv=False)
        assert (info.iters, info.status) == (it, st)
        assert torch_mod.equal(x, x2)
    assert got[2][1] == B.DG_ENOTCONV and got[2][0] == 5


def test_dof_layout_and_device_bytes(built_lib, torch_mod):
    mesh = MESHES["ragged"][0]()
    B = built_lib
    M = B.Mesh(mesh)
    off = B.dg_dof_layout(M.h, mesh.n_elems)
    want = np.concatenate([[0], np.cumsum((mesh.p.astype(np.int64) + 1) ** 2)])
    assert np.array_equal(off, want)
    pc = B.Precond(M)
    # the handles' own counts of their device bytes: at least the vectors
    # (x / traces for the mesh; six PCG work vectors for the preconditioner)
    assert M.stats.device_bytes > 8 * M.n_dofs
    assert pc.stats.device_bytes > 6 * 8 * M.n_dofs


@pytest.mark.parametrize("name,lor", [("hp-a", "amg"), ("cfg0", "exact")])
def test_profile_entries_compute_the_same(built_lib, torch_mod, name, lor):
    """dg_precond_profile (parts run one after another) and dg_apply_profile
    (trace and operator kernels timed apart) give bit-identical results to
    dg_precond_apply and dg_apply, and positive part times."""
    mk, eta, pform = MESHES[name]
    B = built_lib
    o = _opts(B, "sipg", eta, pform, lor=B.DG_LOR_EXACT if lor == "exact" else B.DG_LOR_AMG,
              precision=B.DG_PREC_MIXED)
    M = B.Mesh(mk(), o)
    pc = B.Precond(M, o)
    r = dev(torch_mod, inputs.random_vector(M.n_dofs, 31))
    z1, z2 = torch_mod.empty_like(r), torch_mod.empty_like(r)
    B.dg_precond_apply(pc.h, r, z1)
    t = B.dg_precond_profile(pc.h, r, z2)
    torch_mod.cuda.synchronize()
    assert torch_mod.equal(z1, z2)
    assert t.total_ms > 0 and t.final_ms > 0 and t.lor_ms > 0
    assert pc.stats.apply_bytes > pc.stats.block_bytes >= 0
    y1, y2 = torch_mod.empty_like(r), torch_mod.empty_like(r)
    B.dg_apply(M.h, r, y1)
    ta = B.dg_apply_profile(M.h, r, y2)
    torch_mod.cuda.synchronize()
    assert torch_mod.equal(y1, y2)
    assert ta.trace_ms > 0 and ta.apply_ms > 0


def test_fp64_probe_is_plausible(built_lib, torch_mod):
    tf, ms = built_lib.dg_fp64_fma_probe(20000)
    # GB300: about 1.2-1.3 TFLOP/s of FP64 FMA at full clock
    assert 0.3 < tf < 3.0 and ms > 0
