"""The library's host mirror of the operator on cube meshes (run through the
inspection library, no GPU) against the oracle: topology, sub-face records,
face tables, penalties and the BR2 default eta."""
import numpy as np
import pytest

from oracle import dg, solver
from paper_2009_01287_gb300 import inputs

CASES = [
    ("hp0", lambda: inputs.small_hp_mesh(0, base=2, depth=2, prob=0.5, pmin=1, pmax=4, dim=3)),
    ("hp1", lambda: inputs.small_hp_mesh(1, base=2, depth=2, prob=0.5, pmin=1, pmax=4, dim=3)),
    ("hp1-p8", lambda: inputs.small_hp_mesh(1, base=2, depth=1, prob=0.2, pmin=6, pmax=8, dim=3)),
    ("single", lambda: inputs.uniform_mesh(3, 1, 3)),
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
