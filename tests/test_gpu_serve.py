"""Serving loop: requests admitted while others are in flight give the same
result as the same request solved alone (same calls on its own handles)."""
import numpy as np
import pytest

from paper_2009_01287_gb300 import inputs

pytestmark = pytest.mark.gpu


def _meshes():
    return [inputs.small_hp_mesh(1, base=4, depth=3, prob=0.4, pmax=5),
            inputs.random_refined_mesh(2, 5, 3, 0.35, 1, 4, seed=9, base_y=3),
            inputs.small_hp_mesh(7, base=6, depth=2, prob=0.3, pmin=2, pmax=7),
            inputs.small_hp_mesh(0, base=2, depth=2, prob=0.4, pmin=1, pmax=3, dim=3)]


def _alone(B, srv, rq, device):
    """The same request solved alone, on fresh handles."""
    import torch
    opts = srv.opts[rq.mesh.dim]
    M = B.Mesh(rq.mesh, opts)
    pc = B.Precond(M, opts)
    b = torch.empty(M.n_dofs, dtype=torch.float64, device=device)
    B.dg_rhs_sine(M.h, rq.rhs.amps, rq.rhs.waves, b)
    x = torch.empty_like(b)
    info = B.dg_pcg_solve(M.h, pc.h, b, x, rq.tol, rq.maxit)
    return info, x.cpu().numpy()


def test_results_same_alone_and_in_the_mix(built_lib, cuda_device):
    import torch
    from paper_2009_01287_gb300 import serve
    B = built_lib
    reqs = serve.poisson_stream(12, rate=1e6, meshes=_meshes(), seed=3)
    srv = serve.Server(slots=4, keep_solutions=True)
    res = srv.run(reqs, realtime=False)
    srv.close()
    assert all(r.ok for r in res) and srv.max_inflight >= 2
    assert any(r.dim == 3 for r in res)
    for rq, r in zip(reqs, res):
        info, xa = _alone(B, srv, rq, cuda_device)
        assert info.iters == r.iters
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


def test_tight_budget_evicts_and_every_request_succeeds(built_lib, cuda_device):
    """A budget that holds about one resident mesh at a time, four slots and
    repeated meshes: entries in use are never evicted, idle ones are, requests
    that do not fit wait, and every request succeeds with the result it has
    alone."""
    from paper_2009_01287_gb300 import serve
    B = built_lib
    meshes = _meshes()
    srv = serve.Server(slots=4, keep_solutions=True)
    # measured bytes of every mesh's handles; the estimates use the largest
    # bytes per DOF of each dimension, so they are never below the real bytes
    sizes = []
    for m in meshes:
        r = serve._Resident(m, srv.opts[m.dim])
        sizes.append(r.bytes)
        srv.bytes_per_dof[m.dim] = max(srv.bytes_per_dof.get(m.dim, 0.0), r.bytes / r.n_dofs)
        r.close()
    big = sorted(sizes)
    srv.budget = big[-1] + big[-2] // 2   # the largest fits; the two largest never fit together
    reqs = serve.poisson_stream(24, rate=1e6, meshes=meshes, seed=6)
    res = srv.run(reqs, realtime=False)
    srv.close()
    assert all(r.ok for r in res), [r.error for r in res if not r.ok]
    assert srv.evictions > 0
    assert srv.peak_bytes <= srv.budget
    for rq, r in list(zip(reqs, res))[:6]:
        info, xa = _alone(B, srv, rq, cuda_device)
        assert info.iters == r.iters
        assert np.abs(xa - r.x).max() <= 1e-12 * np.abs(xa).max()


def test_same_mesh_from_many_slots_is_built_once(built_lib, cuda_device):
    from paper_2009_01287_gb300 import serve
    mesh = _meshes()[0]
    reqs = serve.poisson_stream(8, rate=1e6, meshes=[mesh], seed=7)
    srv = serve.Server(slots=4)
    res = srv.run(reqs, realtime=False)
    assert all(r.ok for r in res)
    assert sum(1 for r in res if r.setup_s > 0) == 1 and len(srv.cache) == 1
    srv.close()
