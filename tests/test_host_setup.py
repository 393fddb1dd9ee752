"""The library's host setup (run through the inspection library, no GPU)
against the oracle: topology-derived operator rows, conforming prolongation,
V_J / V_e split, LOR matrix, block inverses and AMG hierarchy."""
import numpy as np
import pytest

from oracle import solver
from paper_2009_01287_gb300 import inputs

def _coef(mesh, base):
    return inputs.with_coeff(mesh, inputs.base_parity_coeff(mesh, base))


CASES = [
    ("cfg0", lambda: inputs.config0()[0], "sipg", 10.0, "p1sq"),
    ("hp1", lambda: inputs.small_hp_mesh(1, base=4, depth=3, prob=0.4, pmax=5), "sipg", None, "paper"),
    ("hp2-br2", lambda: inputs.small_hp_mesh(2, base=4, depth=3, prob=0.4, pmax=6), "br2", None, "paper"),
    ("hp3-p8", lambda: inputs.small_hp_mesh(3, base=3, depth=2, prob=0.5, pmin=6, pmax=8), "sipg", None, "paper"),
    ("single", lambda: inputs.uniform_mesh(2, 1, 3), "sipg", None, "paper"),
    # piecewise-constant coefficient a in {1, 20} by base-cell parity (Section 4.3)
    ("coef-sipg", lambda: _coef(inputs.small_hp_mesh(4, base=4, depth=3, prob=0.4, pmax=5), 4), "sipg", None,
     "paper"),
    ("coef-br2", lambda: _coef(inputs.small_hp_mesh(5, base=4, depth=2, prob=0.4, pmax=6), 4), "br2", None,
     "paper"),
    # a domain with a hole: the L-shape of the adaptive-refinement problems (Section 4.2)
    ("lshape", lambda: inputs.lshape(inputs.small_hp_mesh(6, base=4, depth=3, prob=0.4, pmax=5)), "sipg", None,
     "paper"),
    ("lshape-br2", lambda: inputs.lshape(inputs.small_hp_mesh(7, base=4, depth=2, prob=0.5, pmax=4)), "br2", None,
     "paper"),
]


def _pair(built_lib, mk, form, eta, pform):
    mesh = mk()
    prob = solver.build_problem(mesh, form=form, eta=eta, penalty_form=pform)
    B = built_lib
    opts = B.make_options(form=B.DG_FORM_BR2 if form == "br2" else B.DG_FORM_SIPG, eta=eta or 0.0,
                          penalty_form=B.DG_PENALTY_P1SQ if pform == "p1sq" else B.DG_PENALTY_PAPER)
    return prob, B.HostSetup(mesh, opts)


@pytest.mark.parametrize("name,mk,form,eta,pform", CASES, ids=[c[0] for c in CASES])
def test_host_setup_matches_oracle(built_lib, name, mk, form, eta, pform):
    prob, hs = _pair(built_lib, mk, form, eta, pform)
    x = inputs.random_vector(prob.space.n, 11)
    ya, yb = prob.A @ x, hs.apply(x)
    assert np.abs(ya - yb).max() <= 1e-12 * np.abs(ya).max()
    assert hs.nC == prob.cs.n
    assert abs(prob.cs.P - hs.P).max() < 1e-13
    assert np.array_equal(prob.cs.kind, hs.kind)
    assert len(hs.blocks) == len(prob.cs.blocks)
    for a, b in zip(prob.cs.blocks, hs.blocks):
        assert np.array_equal(a, b)
    pc = solver.Preconditioner(prob, lor="amg")
    assert abs(pc.Ac - hs.Ac).max() <= 1e-13 * abs(pc.Ac).max()
    d = np.where(pc.jmask, pc.dinv, 0.0)
    assert np.abs(d - hs.dinv).max() <= 1e-12 * np.abs(d).max()
    for a, b in zip(pc.block_inv, hs.block_inv):
        assert np.abs(a - b).max() <= 1e-10 * np.abs(a).max()
    assert [L.n for L in pc.levels] == [l.shape[0] for l in hs.levels]
    for L, l in zip(pc.levels, hs.levels):
        assert abs(L.A - l).max() <= 1e-11 * abs(L.A).max()


def test_default_br2_penalty_matches(built_lib):
    prob, hs = _pair(built_lib, CASES[2][1], "br2", None, "paper")
    from oracle.dg import br2_eta
    assert hs.eta == br2_eta(prob.topo)


def test_lshape_load_with_boundary_data(built_lib):
    """The library's load vector with weak Dirichlet data on an L-shaped hp
    mesh (boundary sub-faces along the hole) against the oracle's."""
    from oracle import rhs as R
    mesh = inputs.lshape(inputs.small_hp_mesh(8, base=4, depth=3, prob=0.4, pmax=6))
    prob = solver.build_problem(mesh)
    B = built_lib
    hs = B.HostSetup(mesh, B.make_options(), amg=False)
    f = lambda x: np.cos(2 * x[:, 0]) + x[:, 1]
    g = lambda x: np.hypot(x[:, 0] - 0.5, x[:, 1] - 0.5) ** (2.0 / 3.0)
    ref = R.dirichlet_load(prob.space, f, g, 100.0)
    assert np.abs(hs.rhs_eval(f, g) - ref).max() <= 1e-12 * np.abs(ref).max()
