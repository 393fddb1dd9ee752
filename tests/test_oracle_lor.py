"""Pins of the oracle's low-order-refined matrices (Section 3.4, Prop. 1)."""
import numpy as np
import pytest

from oracle import basis, dg, lor, solver
from paper_2009_01287_gb300 import inputs


def test_q1_cell_closed_form():
    # unit square bilinear stiffness: diagonal 2/3, edge neighbours -1/6,
    # opposite corner -1/3 (textbook)
    K = lor.q1_cell_stiffness(1.0, 1.0)
    expect = np.array([[4, -1, -1, -2], [-1, 4, -2, -1], [-1, -2, 4, -1], [-2, -1, -1, 4]]) / 6.0
    np.testing.assert_allclose(K, expect, atol=1e-15)
    # rectangle a x b: K = (b/a) Kx(x)My + (a/b) Mx(x)Ky
    a, b = 0.3, 1.7
    K = lor.q1_cell_stiffness(a, b)
    k1 = np.array([[1, -1], [-1, 1]])
    m1 = np.array([[2, 1], [1, 2]]) / 6.0
    expect = (b / a) * np.kron(m1, k1) + (a / b) * np.kron(k1, m1)
    np.testing.assert_allclose(K, expect, atol=1e-13)


def test_p1_lor_equals_high_order():
    """For p = 1 the LOR sub-mesh is the element itself: A-tilde = A-hat."""
    mesh = inputs.small_hp_mesh(0, base=2, depth=2, prob=0.5, pmin=1, pmax=1)
    prob = solver.build_problem(mesh)
    At = lor.assemble_lor(prob.space)
    Ah = dg.assemble(prob.space, 1.0, broken_only=True)
    assert abs(At - Ah).max() < 1e-13


def test_lor_spectral_equivalence_bounded_in_p():
    """Prop. 1: generalized eigenvalues of (A_C, A-tilde_C) stay in a fixed
    interval as p grows (uniform mesh, p = 1..8)."""
    lo, hi = [], []
    for p in range(1, 9):
        mesh = inputs.uniform_mesh(2, 2, p)
        prob = solver.build_problem(mesh)
        P = prob.cs.P.toarray()
        Ac = P.T @ dg.assemble(prob.space, 1.0, broken_only=True).toarray() @ P
        At = P.T @ lor.assemble_lor(prob.space).toarray() @ P
        ev = np.linalg.eigvals(np.linalg.solve(At, Ac)).real
        lo.append(ev.min())
        hi.append(ev.max())
    # measured: [0.85, 1.0] and [1.0, 4.09] for p = 1..8; growth levels off
    assert min(lo) > 0.8 and max(hi) < 5.0
    assert hi[7] / hi[3] < 1.35
