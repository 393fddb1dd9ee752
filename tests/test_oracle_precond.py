"""Pins of the oracle's preconditioner, AMG and PCG (Thm. 2, Section 4.1)."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import amg, solver
from paper_2009_01287_gb300 import inputs


def kappa(B, A):
    ev = np.sort(np.linalg.eigvals(B @ A).real)
    assert ev[0] > 0
    return ev[-1] / ev[0]


def fig1_mesh(n, pc=2, pf=1):
    """A coarse degree-pc square beside a column of n fine degree-pf squares
    (Fig. 1 with square fine elements)."""
    lo = [(0, 0)] + [(n, j) for j in range(n)]
    return inputs.MeshDesc(2, np.asarray(lo, dtype=np.int32),
                           np.asarray([n] + [1] * n, dtype=np.int32),
                           np.asarray([pc] + [pf] * n, dtype=np.int32), (n + 1, n), 1.0 / n)


def test_fig1_full_B_vs_jacobi_only():
    """Section 4.1: B~ = J_B + B_C degrades on the hp-interface of Fig. 1
    while B = B_B + B_C does not."""
    kb, kt = [], []
    for n in [2, 4, 8]:
        prob = solver.build_problem(fig1_mesh(n))
        A = prob.A.toarray()
        kb.append(kappa(solver.Preconditioner(prob, lor="exact").matrix(), A))
        kt.append(kappa(solver.Preconditioner(prob, lor="exact", smoother="jacobi_only").matrix(), A))
    assert kt[0] > 10 * kb[0] and kt[-1] > 20 * kb[-1]
    assert max(kb) < 40


@pytest.mark.parametrize("eta", [10.0, 100.0, 1000.0, 10000.0])
def test_kappa_bounded_in_eta(eta):
    """Thm. 2: the condition number does not grow with the penalty."""
    mesh = inputs.small_hp_mesh(4, base=2, depth=2, prob=0.5, pmin=2, pmax=4)
    prob = solver.build_problem(mesh, eta=eta)
    k = kappa(solver.Preconditioner(prob, lor="exact").matrix(), prob.A.toarray())
    assert k < 60


def test_kappa_bounded_in_h_and_p():
    ks = []
    for n, p in [(2, 2), (4, 2), (8, 2), (2, 4), (2, 6), (4, 4)]:
        prob = solver.build_problem(inputs.uniform_mesh(2, n, p))
        ks.append(kappa(solver.Preconditioner(prob, lor="exact").matrix(), prob.A.toarray()))
    assert max(ks) < 15


def test_br2_kappa_bounded_in_eta():
    ks = []
    mesh = inputs.small_hp_mesh(4, base=2, depth=2, prob=0.5, pmin=2, pmax=4)
    for eta in [4.0, 40.0, 400.0]:
        prob = solver.build_problem(mesh, form="br2", eta=eta)
        ks.append(kappa(solver.Preconditioner(prob, lor="exact").matrix(), prob.A.toarray()))
    assert max(ks) < 60


def _poisson5(n):
    T = sp.diags([-1, 2, -1], [-1, 0, 1], shape=(n, n))
    return (sp.kron(sp.identity(n), T) + sp.kron(T, sp.identity(n))).tocsr()


def test_amg_vcycle_properties():
    A = _poisson5(40)                      # 1600 unknowns -> several levels below 64 rows
    levels = amg.setup(A, coarse_max=64)
    assert len(levels) >= 3
    n = A.shape[0]
    rng = np.random.default_rng(0)
    x, y = rng.standard_normal(n), rng.standard_normal(n)
    # symmetric: <M x, y> = <x, M y>
    assert abs(amg.vcycle(levels, x) @ y - x @ amg.vcycle(levels, y)) < 1e-10 * abs(x @ amg.vcycle(levels, x))
    # Galerkin coarse operators
    for L, Lc in zip(levels[:-1], levels[1:]):
        assert abs(L.P.T @ L.A @ L.P - Lc.A).max() < 1e-12 * abs(L.A).max()
    # aggregates partition the fine level: every row of T has exactly one 1
    agg = amg.aggregate(levels[0].A)
    assert agg.min() == 0 and len(np.unique(agg)) == agg.max() + 1
    # the two-grid error propagation I - M A contracts
    M = np.stack([amg.vcycle(levels, e) for e in np.eye(n)[:: n // 200]], axis=1)
    E = np.eye(n) - np.stack([amg.vcycle(levels, c) for c in A.toarray().T], axis=1)
    ev = np.abs(np.linalg.eigvals(E))
    assert ev.max() < 0.95


def test_amg_single_level_is_exact():
    A = _poisson5(10)
    levels = amg.setup(A)
    assert len(levels) == 1
    b = np.arange(100.0)
    np.testing.assert_allclose(A @ amg.vcycle(levels, b), b, atol=1e-10)


def test_pcg_direct_solution():
    rng = np.random.default_rng(1)
    Q = rng.standard_normal((30, 30))
    A = Q @ Q.T + 30 * np.eye(30)
    b = rng.standard_normal(30)
    res = solver.pcg(A, b, lambda r: r / np.diag(A), 1e-13, 30)
    assert res.converged and res.iters <= 30
    np.testing.assert_allclose(res.x, np.linalg.solve(A, b), rtol=1e-10)


def test_config0_pcg_converges():
    mesh, rhs_ = inputs.config0()
    prob = solver.build_problem(mesh, eta=10.0, penalty_form="p1sq")
    from oracle import rhs
    b = rhs.load_vector(prob.space, rhs_.amps, rhs_.waves)
    pc = solver.Preconditioner(prob, lor="exact")
    res = solver.pcg(prob.A, b, pc.apply, 1e-10, 200)
    assert res.converged and res.iters < 40
    x = sp.linalg.spsolve(prob.A.tocsc(), b)
    assert np.abs(res.x - x).max() < 1e-8 * np.abs(x).max()
