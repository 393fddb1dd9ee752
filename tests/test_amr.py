"""The hp-adaptive refinement driver (Section 4.2, the internal-layer
problem) on the CPU: its problem data, marking, hp decision and refinement,
and a few AMR steps with the oracle as the solver (the meshes stay valid, the
error falls, the preconditioned iteration counts stay bounded)."""
import numpy as np
import pytest

from oracle import rhs, solver
from oracle.topology import Topology
from paper_2009_01287_gb300 import amr, inputs


def test_layer_f_is_minus_laplacian_of_u():
    rng = np.random.default_rng(0)
    x = rng.uniform(0.0, 1.0, size=(50, 2))
    e = 1e-4
    lap = np.zeros(len(x))
    for d in range(2):
        dd = np.zeros(2)
        dd[d] = e
        lap += (amr.layer_u(x + dd) - 2 * amr.layer_u(x) + amr.layer_u(x - dd)) / e ** 2
    scale = np.abs(amr.layer_f(x)).max()
    assert np.abs(amr.layer_f(x) + lap).max() <= 1e-4 * scale


def test_bulk_marking():
    eta = np.array([1.0, 3.0, 2.0, 3.0, 0.5])
    m = amr.bulk_mark(eta, 0.5)
    # 3, 3 (by index: 1 then 3): 18 of 23.25 >= half; one of them alone (9) is not
    assert m.tolist() == [False, True, False, True, False]
    assert not amr.bulk_mark(np.zeros(3)).any()


def _area_ok(mesh):
    topo = Topology(mesh.lo, mesh.size, mesh.p, mesh.extent)   # validates the tiling
    assert topo.n == mesh.n_elems
    assert (mesh.size.astype(np.int64) ** 2).sum() == int(mesh.extent[0]) * int(mesh.extent[1])


def test_refine_splits_and_enriches():
    mesh = inputs.uniform_mesh(2, 2, 2)
    h = np.array([True, False, False, False])
    p = np.array([False, True, False, False])
    m2 = amr.refine(mesh, h, p)
    _area_ok(m2)
    assert m2.n_elems == 7 and m2.extent == (4, 4) and m2.lattice_h == 0.25
    assert m2.p.tolist() == [2, 2, 2, 2, 3, 2, 2]
    m3 = amr.refine(m2, np.array([True] + [False] * 6), np.zeros(7, bool))
    _area_ok(m3)
    assert m3.extent == (8, 8)


def test_smoothness_ratio():
    """A polynomial of degree below p per direction has an empty last shell;
    a rough vector does not."""
    mesh = inputs.uniform_mesh(2, 1, 5)
    g = amr._gll(5)
    X, Y = np.meshgrid(g, g)
    smooth = (1 + X + X ** 2 * Y ** 3).ravel()
    _, r = amr.element_indicators(mesh, smooth, exact=lambda x: np.zeros(len(x)))
    assert r[0] < 1e-3          # round-off only, far below the threshold
    rough = np.random.default_rng(1).standard_normal(36)
    _, r = amr.element_indicators(mesh, rough, exact=lambda x: np.zeros(len(x)))
    assert r[0] > amr.SMOOTH


def oracle_solver(mesh, problem=amr.LAYER):
    prob = solver.build_problem(mesh)
    pc = solver.Preconditioner(prob, lor="amg")
    b = rhs.dirichlet_load(prob.space, problem.f, problem.u, 100.0)
    res = solver.pcg(prob.A, b, pc.apply, 1e-8, 5000)
    pcj = solver.Preconditioner(prob, lor="amg", smoother="jacobi_only")
    resj = solver.pcg(prob.A, b, pcj.apply, 1e-8, 5000)
    sizes = [len(bk) for bk in prob.cs.blocks]
    return res.x, {"iters": res.iters, "iters_jacobi": resj.iters, "n_blocks": len(sizes),
                   "max_block": max(sizes) if sizes else 0}


def test_amr_steps_with_the_oracle():
    meshes = []
    recs = amr.run(oracle_solver, steps=8, callback=lambda m, x, r: meshes.append(m))
    for m in meshes:
        _area_ok(m)
    assert [r.step for r in recs] == list(range(9))
    assert all(r.n_dofs > 0 for r in recs)
    assert recs[-1].err_l2 < recs[0].err_l2
    assert recs[-1].n_dofs > recs[0].n_dofs
    assert max(r.iters for r in recs) < 200
    assert any(r.n_h for r in recs[:-1]) and any(r.n_p for r in recs[:-1])


def test_lshape_solution_is_harmonic_and_vanishes_on_the_corner_edges():
    rng = np.random.default_rng(2)
    x = rng.uniform(1.05, 1.95, size=(40, 2))      # away from the corner, inside the domain
    e = 1e-4
    lap = np.zeros(len(x))
    for d in range(2):
        dd = np.zeros(2)
        dd[d] = e
        lap += (amr.lshape_u(x + dd) - 2 * amr.lshape_u(x) + amr.lshape_u(x - dd)) / e ** 2
    assert np.abs(lap).max() <= 1e-5
    t = np.linspace(0.0, 1.0, 7)
    edges = np.concatenate([np.stack([1.0 + 0 * t, t], 1), np.stack([t, 1.0 + 0 * t], 1)])
    assert np.abs(amr.lshape_u(edges)).max() <= 1e-15
    m = amr.lshape_initial()
    _area_ok_l(m)


def _area_ok_l(mesh):
    Topology(mesh.lo, mesh.size, mesh.p, mesh.extent)
    assert mesh.n_elems == 12 and (mesh.size.astype(np.int64) ** 2).sum() == 12


def test_amr_lshape_steps_with_the_oracle():
    recs = amr.run(lambda m: oracle_solver(m, amr.LSHAPE), steps=6, problem=amr.LSHAPE)
    assert recs[0].n_dofs == 48 and recs[-1].n_dofs > 48
    assert recs[-1].err_l2 < recs[0].err_l2
    assert max(r.iters for r in recs) < 100


def test_refine_keeps_coefficient_and_geometry():
    mesh = inputs.with_coeff(inputs.uniform_mesh(2, 2, 1), [1.0, 2.0, 3.0, 4.0])
    mesh = inputs.with_corners(mesh, inputs.QUADRILATERAL)
    m2 = amr.refine(mesh, np.array([False, True, False, False]), np.array([True, False, False, False]))
    assert m2.coeff.tolist() == [1.0, 2.0, 2.0, 2.0, 2.0, 3.0, 4.0]
    assert np.array_equal(m2.corners, mesh.corners)
    # the physical domain is the same: the lattice doubled, its spacing halved
    assert m2.extent[0] * m2.lattice_h == mesh.extent[0] * mesh.lattice_h


def test_l2_indicator_is_exact_on_polynomials():
    """eta_k = ||u - u_h||_L2(k): zero when u_h interpolates a polynomial of
    degree <= p exactly, and the element's area^(1/2) * |c| for u - u_h = c."""
    mesh = inputs.small_hp_mesh(3, base=3, depth=2, prob=0.5, pmin=2, pmax=4)
    off = np.concatenate([[0], np.cumsum((mesh.p.astype(np.int64) + 1) ** 2)])
    u = lambda x: 1.0 + x[:, 0] * x[:, 1] - 0.5 * x[:, 1] ** 2
    x = np.zeros(off[-1])
    h = mesh.size * mesh.lattice_h
    for k in range(mesh.n_elems):
        g = amr._gll(int(mesh.p[k]))
        X, Y = np.meshgrid(g, g)
        pts = np.stack([mesh.lo[k, 0] * mesh.lattice_h + h[k] * X.ravel(),
                        mesh.lo[k, 1] * mesh.lattice_h + h[k] * Y.ravel()], axis=1)
        x[off[k]:off[k + 1]] = u(pts)
    eta, _ = amr.element_indicators(mesh, x, exact=u)
    assert eta.max() <= 1e-13
    eta, _ = amr.element_indicators(mesh, x, exact=lambda p: u(p) + 0.25)
    assert np.abs(eta - 0.25 * h).max() <= 1e-13


def test_indicators_refuse_mapped_meshes():
    mesh = inputs.uniform_mesh(2, 2, 2)
    x = np.zeros(mesh.n_dofs())
    for m in (inputs.with_corners(mesh, inputs.QUADRILATERAL), inputs.with_mapping(mesh, inputs.WavyMap())):
        with pytest.raises(ValueError):
            amr.element_indicators(m, x)
