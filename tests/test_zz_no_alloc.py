"""dg_pcg_solve_noalloc: the PCG solve for callers that must not have the
library allocate memory (device, pinned host, or graphs) while they solve -
for example a service that reserves all device memory up front, since
cudaMalloc/cudaFree can synchronise the whole device.  Its work vectors live
in one fixed library-wide device array; it must give the same answer as
dg_pcg_solve, call after call, and leave the device's free memory unchanged.
Kept in a file that runs last."""
import numpy as np
import pytest

from paper_2009_01287_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dim", [2, 3])
def test_noalloc_matches_pcg_solve_twice(built_lib, cuda_device, dim):
    import torch
    B = built_lib
    if dim == 2:
        mesh, opts = inputs.small_hp_mesh(1, base=4, depth=3, prob=0.4, pmax=5), B.make_options()
    else:
        mesh = inputs.small_hp_mesh(0, base=2, depth=2, prob=0.4, pmin=1, pmax=3, dim=3)
        opts = B.make_options(form=B.DG_FORM_BR2)
    b = torch.tensor(inputs.random_vector(mesh.n_dofs(), 21), dtype=torch.float64, device=cuda_device)
    # the no-alloc solves run first on their own fresh handles
    M = B.Mesh(mesh, opts)
    pc = B.Precond(M, opts)
    x = torch.full_like(b, 3.0)
    B.dg_pcg_solve_noalloc(M.h, pc.h, b, x, 1e-10, 2000)   # looks up the scratch address
    torch.cuda.synchronize()
    outs = []
    for _ in range(2):
        free0, _ = torch.cuda.mem_get_info()
        x = torch.full_like(b, 3.0)          # allocated (by torch) before the measured window
        free1, _ = torch.cuda.mem_get_info()
        info = B.dg_pcg_solve_noalloc(M.h, pc.h, b, x, 1e-10, 2000)
        torch.cuda.synchronize()
        free2, _ = torch.cuda.mem_get_info()
        assert free2 == free1, (free0, free1, free2)
        outs.append((info, x))
    # the reference solve on separate handles
    M2 = B.Mesh(mesh, opts)
    pc2 = B.Precond(M2, opts)
    x_ref = torch.empty_like(b)
    ref = B.dg_pcg_solve(M2.h, pc2.h, b, x_ref, 1e-10, 2000)
    scale = float(x_ref.abs().max())
    for info, x in outs:
        assert info.status == B.DG_OK and info.iters == ref.iters
        assert abs(info.rel_res - ref.rel_res) <= 1e-12
        assert float((x - x_ref).abs().max()) <= 1e-12 * scale


def test_noalloc_rejects_oversized_mesh(built_lib, cuda_device):
    B = built_lib
    mesh = inputs.uniform_mesh(2, 64, 8)          # 331,776 unknowns > 262,144
    M = B.Mesh(mesh)
    with pytest.raises(B.DGError) as e:
        B.dg_pcg_solve_noalloc(M.h, 0, 0, 0, 1e-8, 10)
    assert e.value.code == B.DG_EINVAL and "exceeds the static scratch limit" in str(e.value)
