"""The library's host mirror of the operator on cube meshes (run through the
inspection library, no GPU) against the oracle: topology, sub-face records,
face tables, penalties and the BR2 default eta."""
import numpy as np
import pytest

from oracle import dg, solver
from paper_2009_01287_gb300 import inputs

def _coef(mesh, base):
    return inputs.with_coeff(mesh, inputs.base_parity_coeff(mesh, base))


CASES = [
    ("hp0", lambda: inputs.small_hp_mesh(0, base=2, depth=2, prob=0.5, pmin=1, pmax=4, dim=3)),
    ("hp1", lambda: inputs.small_hp_mesh(1, base=2, depth=2, prob=0.5, pmin=1, pmax=4, dim=3)),
    ("hp1-p8", lambda: inputs.small_hp_mesh(1, base=2, depth=1, prob=0.2, pmin=6, pmax=8, dim=3)),
    ("single", lambda: inputs.uniform_mesh(3, 1, 3)),
    ("coef", lambda: _coef(inputs.small_hp_mesh(2, base=2, depth=2, prob=0.5, pmin=1, pmax=4, dim=3), 2)),
]


@pytest.mark.parametrize("form", ["sipg", "br2"])
@pytest.mark.parametrize("name,mk", CASES, ids=[c[0] for c in CASES])
def test_host_apply3_matches_oracle(built_lib, name, mk, form):
    B = built_lib
    mesh = mk()
    hs = B.HostSetup(mesh, B.make_options(form=B.DG_FORM_BR2 if form == "br2" else B.DG_FORM_SIPG), amg=False)
    topo, space, A = solver.build_operator(mesh, form=form)
    if form == "br2":
        assert hs.eta == dg.br2_eta(topo)
    assert hs.n == space.n
    x = inputs.random_vector(space.n, 5)
    ya, yb = A @ x, hs.apply(x)
    assert np.abs(ya - yb).max() <= 1e-12 * np.abs(ya).max()


PC_CASES = [
    ("hp0-sipg", lambda: inputs.small_hp_mesh(0, base=2, depth=2, prob=0.3, pmin=1, pmax=3, dim=3), "sipg"),
    ("hp1-br2", lambda: inputs.small_hp_mesh(1, base=2, depth=2, prob=0.3, pmin=1, pmax=4, dim=3), "br2"),
    ("hp3-sipg", lambda: inputs.small_hp_mesh(3, base=2, depth=2, prob=0.4, pmin=1, pmax=2, dim=3), "sipg"),
    ("uniform", lambda: inputs.uniform_mesh(3, 2, 3), "sipg"),
    ("coef-sipg", lambda: _coef(inputs.small_hp_mesh(4, base=2, depth=2, prob=0.3, pmin=1, pmax=3, dim=3), 2),
     "sipg"),
    ("coef-br2", lambda: _coef(inputs.small_hp_mesh(5, base=2, depth=2, prob=0.3, pmin=1, pmax=3, dim=3), 2),
     "br2"),
]


@pytest.mark.parametrize("name,mk,form", PC_CASES, ids=[c[0] for c in PC_CASES])
def test_host_precond3_matches_oracle(built_lib, name, mk, form):
    """Conforming numbering and P, node classes, V_e blocks, the V_J diagonal
    (closed form), block inverses, LOR matrix and AMG levels on cube meshes."""
    B = built_lib
    mesh = mk()
    prob = solver.build_problem(mesh, form=form)
    hs = B.HostSetup(mesh, B.make_options(form=B.DG_FORM_BR2 if form == "br2" else B.DG_FORM_SIPG))
    cs = prob.cs
    assert hs.nC == cs.n
    assert abs(cs.P - hs.P).max() < 1e-13
    assert np.array_equal(cs.kind, hs.kind)
    assert len(hs.blocks) == len(cs.blocks)
    assert all(np.array_equal(a, b) for a, b in zip(cs.blocks, hs.blocks))
    pc = solver.Preconditioner(prob, lor="amg")
    assert abs(pc.Ac - hs.Ac).max() <= 1e-13 * abs(pc.Ac).max()
    d = np.where(pc.jmask, pc.dinv, 0.0)
    assert np.abs(d - hs.dinv).max() <= 1e-12 * np.abs(d).max()
    for a, b in zip(pc.block_inv, hs.block_inv):
        assert np.abs(a - b).max() <= 1e-10 * np.abs(a).max()
    assert [L.n for L in pc.levels] == [l.shape[0] for l in hs.levels]
    for L, l in zip(pc.levels, hs.levels):
        assert abs(L.A - l).max() <= 1e-11 * abs(L.A).max()
