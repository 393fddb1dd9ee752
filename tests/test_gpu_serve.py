"""Serving loop: requests admitted while others are in flight give the same
result as the same request solved alone (same calls on its own handles)."""
import numpy as np
import pytest

from paper_2009_01287_gb300 import inputs

pytestmark = pytest.mark.gpu


def _meshes():
    return [inputs.small_hp_mesh(1, base=4, depth=3, prob=0.4, pmax=5),
            inputs.random_refined_mesh(2, 5, 3, 0.35, 1, 4, seed=9, base_y=3),
            inputs.small_hp_mesh(7, base=6, depth=2, prob=0.3, pmin=2, pmax=7)]


def test_results_same_alone_and_in_the_mix(built_lib, cuda_device):
    import torch
    from paper_2009_01287_gb300 import serve
    B = built_lib
    reqs = serve.poisson_stream(12, rate=1e6, meshes=_meshes(), seed=3)
    srv = serve.Server(slots=4, keep_solutions=True)
    res = srv.run(reqs, realtime=False)
    srv.close()
    assert all(r.ok for r in res) and srv.max_inflight >= 2
    for rq, r in zip(reqs, res):
        M = B.Mesh(rq.mesh, srv.opts)
        pc = B.Precond(M, srv.opts)
        b = torch.empty(M.n_dofs, dtype=torch.float64, device=cuda_device)
        B.dg_rhs_sine(M.h, rq.rhs.amps, rq.rhs.waves, b)
        x = torch.empty_like(b)
        info = B.dg_pcg_solve(M.h, pc.h, b, x, rq.tol, rq.maxit)
        assert info.iters == r.iters
        xa = x.cpu().numpy()
        assert np.abs(xa - r.x).max() <= 1e-12 * np.abs(xa).max()


def test_small_memory_budget_serialises(built_lib, cuda_device):
    from paper_2009_01287_gb300 import serve
    reqs = serve.poisson_stream(6, rate=1e6, meshes=_meshes(), seed=4)
    srv = serve.Server(slots=4, memory_budget=1)
    res = srv.run(reqs, realtime=False)
    srv.close()
    assert all(r.ok for r in res)
    assert srv.max_inflight == 1


def test_bad_request_does_not_stop_the_server(built_lib, cuda_device):
    from paper_2009_01287_gb300 import serve
    reqs = serve.poisson_stream(4, rate=1e6, meshes=_meshes()[:2], seed=5)
    bad = inputs.uniform_mesh(2, 2, 3)
    bad.p[0] = 12   # degree out of range
    reqs.append(serve.Request(rid=99, arrival=0.0, mesh=bad, rhs=reqs[0].rhs))
    srv = serve.Server(slots=2)
    res = srv.run(reqs, realtime=False)
    srv.close()
    by = {r.rid: r for r in res}
    assert not by[99].ok and "degree" in by[99].error
    assert all(by[r.rid].ok for r in reqs if r.rid != 99)
