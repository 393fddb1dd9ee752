"""hp-adaptive refinement on the GPU (Section 4.2, the internal-layer and the
L-shaped domain problems):
the AMR driver runs its solves through the C ABI (weak Dirichlet data by
dg_rhs_eval, PCG with B = B_B + B_C and with B~ = J_B + B_C), and on every
mesh it produces the oracle solves the same system: B's iteration count within
+-1 of the oracle's, B~'s within 5% (its conditioning makes CG's path depend on
the summation order of the dot products), the solution within 1e2 tol, and the
V_e count and largest block equal."""
import numpy as np
import pytest

from oracle import rhs, solver
from paper_2009_01287_gb300 import amr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_mod(cuda_device):
    import torch
    return torch


@pytest.mark.parametrize("which", ["layer", "lshape"])
def test_amr_steps_match_oracle(built_lib, torch_mod, which):
    problem = amr.LAYER if which == "layer" else amr.LSHAPE
    checked = []

    def check(mesh, x, rec):
        prob = solver.build_problem(mesh)
        b = rhs.dirichlet_load(prob.space, problem.f, problem.u, 100.0)
        ref = solver.pcg(prob.A, b, solver.Preconditioner(prob, lor="amg").apply, 1e-8, 20000)
        refj = solver.pcg(prob.A, b, solver.Preconditioner(prob, lor="amg", smoother="jacobi_only").apply,
                          1e-8, 20000)
        assert abs(rec.iters - ref.iters) <= 1, (rec.step, rec.iters, ref.iters)
        assert abs(rec.iters_jacobi - refj.iters) <= 0.05 * refj.iters + 1, (rec.step, rec.iters_jacobi, refj.iters)
        assert np.abs(x - ref.x).max() <= 1e2 * 1e-8 * np.abs(ref.x).max()
        sizes = [len(bk) for bk in prob.cs.blocks]
        assert rec.n_blocks == len(sizes) and rec.max_block == (max(sizes) if sizes else 0)
        checked.append(rec.step)

    recs = amr.run(amr.library_solver(built_lib, torch_mod, problem=problem), steps=8, callback=check,
                   problem=problem)
    assert checked == list(range(9))
    assert recs[-1].n_dofs > recs[0].n_dofs and recs[-1].err_l2 < recs[0].err_l2
