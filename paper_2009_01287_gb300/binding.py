"""ctypes binding of the C ABI in include/dg.h (argument marshalling only).

Functions keep the C names.  Vector arguments are CUDA tensors (torch) or raw
device pointers (int); the library does all the work.  If the shared library
has not been built, `lib()` raises: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

from .inputs import MeshDesc

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libdgsc.so")
INSPECT_PATH = os.path.join(HERE, "_lib", "libdgsc_inspect.so")

DG_OK, DG_EINVAL, DG_ENOMEM, DG_ECUDA, DG_ENOTCONV, DG_ETIMEOUT, DG_EUNSUPPORTED = range(7)
DG_FORM_SIPG, DG_FORM_BR2 = 0, 1
DG_PENALTY_PAPER, DG_PENALTY_P1SQ = 0, 1
DG_PREC_FP64, DG_PREC_MIXED = 0, 1
DG_LOR_EXACT, DG_LOR_AMG = 0, 1
DG_SMOOTHER_FULL, DG_SMOOTHER_JACOBI_ONLY = 0, 1

# every entry point declared in include/dg.h
ABI_SYMBOLS = (
    "dg_mesh_create", "dg_mesh_destroy", "dg_num_dofs", "dg_mesh_stats_get", "dg_dof_layout", "dg_apply",
    "dg_precond_setup",
    "dg_precond_destroy", "dg_precond_stats_get", "dg_precond_apply", "dg_pcg_solve",
    "dg_pcg_solve_host", "dg_pcg_solve_noalloc", "dg_rhs_sine", "dg_rhs_eval", "dg_last_error",
    "dg_batch_create", "dg_batch_destroy", "dg_batch_num_dofs", "dg_batch_offsets", "dg_batch_rhs_sine",
    "dg_batch_solve", "dg_batch_stats_get", "dg_precond_profile", "dg_apply_profile", "dg_fp64_fma_probe",
)


# dg_map_fn: (n, X, x, J, ctx) - images and Jacobians of n pre-image points
DgMapFn = C.CFUNCTYPE(None, C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double),
                      C.c_void_p)


class DgMeshDesc(C.Structure):
    _fields_ = [("dim", C.c_int), ("n_elems", C.c_int64), ("lo", C.POINTER(C.c_int32)),
                ("size", C.POINTER(C.c_int32)), ("p", C.POINTER(C.c_int32)),
                ("extent", C.POINTER(C.c_int32)), ("lattice_h", C.c_double),
                ("coeff", C.POINTER(C.c_double)), ("corners", C.POINTER(C.c_double)),
                ("map", DgMapFn), ("map_ctx", C.c_void_p)]


# dg_field_fn: (n, x, out, ctx) - values of a field at n physical points
DgFieldFn = C.CFUNCTYPE(None, C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_void_p)


def _field_callback(fn):
    """A dg_field_fn evaluating fn(x) (x: (n, 2)) -> (n,); None -> NULL.  On an
    exception the outputs are set to NaN, which the library reports."""
    if fn is None:
        return DgFieldFn()

    def cb(n, x, out, ctx):
        o = np.ctypeslib.as_array(out, shape=(n,))
        try:
            o[:] = fn(np.ctypeslib.as_array(x, shape=(n, 2)))
        except Exception:   # noqa: BLE001 - reported through the NaN outputs
            o[:] = np.nan
    return DgFieldFn(cb)


def _map_callback(mapping):
    """A dg_map_fn that evaluates a Python map object (__call__(X) -> x,
    jacobian(X) -> J of shape (n, 2, 2)).  An exception inside leaves the
    outputs as the library pre-filled them (NaN), which it reports as
    DG_EINVAL."""
    def cb(n, X, x, J, ctx):
        try:
            Xa = np.ctypeslib.as_array(X, shape=(n, 2))
            np.ctypeslib.as_array(x, shape=(n, 2))[:] = mapping(Xa)
            np.ctypeslib.as_array(J, shape=(n, 4))[:] = np.asarray(mapping.jacobian(Xa)).reshape(n, 4)
        except Exception:   # noqa: BLE001 - reported through the NaN outputs
            pass
    return DgMapFn(cb)


class DgOptions(C.Structure):
    _fields_ = [("form", C.c_int), ("eta", C.c_double), ("penalty_form", C.c_int),
                ("precision", C.c_int), ("lor", C.c_int), ("smoother", C.c_int),
                ("remark_cases", C.c_int), ("tune_tiles", C.c_int)]


class DgSolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int), ("rel_res", C.c_double), ("status", C.c_int),
                ("solve_ms", C.c_double)]


class DgMeshStats(C.Structure):
    _fields_ = [("n_elems", C.c_int64), ("n_dofs", C.c_int64), ("n_subfaces", C.c_int64),
                ("max_level_gap", C.c_int64), ("apply_flops", C.c_double), ("apply_bytes", C.c_double),
                ("device_bytes", C.c_int64), ("tile_elems", C.c_int32 * 9), ("tile_smem_budget", C.c_int64),
                ("tiles_tuned", C.c_int32), ("apply_ms_fixed", C.c_double), ("apply_ms_tuned", C.c_double)]


class DgPrecondStats(C.Structure):
    _fields_ = [("n_dofs", C.c_int64), ("n_conforming", C.c_int64), ("n_j", C.c_int64),
                ("n_e", C.c_int64), ("n_blocks", C.c_int64), ("max_block", C.c_int64),
                ("lor_nnz", C.c_int64), ("p_nnz", C.c_int64), ("n_levels", C.c_int),
                ("level_rows", C.c_int64 * 16), ("level_nnz", C.c_int64 * 16),
                ("level_plain", C.c_int * 16), ("kernels_per_apply", C.c_int), ("device_bytes", C.c_int64),
                ("apply_bytes", C.c_double), ("block_bytes", C.c_double)]


class DgPrecondTimes(C.Structure):
    _fields_ = [("blocks_ms", C.c_double), ("restrict_ms", C.c_double), ("lor_ms", C.c_double),
                ("final_ms", C.c_double), ("total_ms", C.c_double)]


class DgApplyTimes(C.Structure):
    _fields_ = [("trace_ms", C.c_double), ("apply_ms", C.c_double)]


_lib = None
_inspect = None


def _load(path: str):
    if not os.path.exists(path):
        raise RuntimeError(f"{os.path.basename(path)} is not built: run __graft_entry__.build()")
    return C.CDLL(path)


def lib():
    global _lib
    if _lib is None:
        L = _load(LIB_PATH)
        vp, i64, dp, st = C.c_void_p, C.c_int64, C.c_void_p, C.c_int
        L.dg_mesh_create.argtypes = [C.POINTER(DgMeshDesc), C.POINTER(DgOptions), vp, C.POINTER(vp)]
        L.dg_mesh_destroy.argtypes = [vp]
        L.dg_num_dofs.argtypes = [vp]
        L.dg_num_dofs.restype = i64
        L.dg_mesh_stats_get.argtypes = [vp, C.POINTER(DgMeshStats)]
        L.dg_dof_layout.argtypes = [vp, vp]
        L.dg_precond_profile.argtypes = [vp, dp, dp, C.POINTER(DgPrecondTimes), vp]
        L.dg_apply_profile.argtypes = [vp, dp, dp, C.POINTER(DgApplyTimes), vp]
        L.dg_fp64_fma_probe.argtypes = [C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_double), vp]
        L.dg_apply.argtypes = [vp, dp, dp, vp]
        L.dg_precond_setup.argtypes = [vp, C.POINTER(DgOptions), C.POINTER(vp)]
        L.dg_precond_destroy.argtypes = [vp]
        L.dg_precond_stats_get.argtypes = [vp, C.POINTER(DgPrecondStats)]
        L.dg_precond_apply.argtypes = [vp, dp, dp, vp]
        L.dg_pcg_solve.argtypes = [vp, vp, dp, dp, C.c_double, C.c_int, C.POINTER(DgSolveInfo), vp]
        L.dg_pcg_solve_host.argtypes = [vp, vp, dp, dp, C.c_double, C.c_int, C.POINTER(DgSolveInfo), vp]
        L.dg_pcg_solve_noalloc.argtypes = [vp, vp, dp, dp, C.c_double, C.c_int, C.POINTER(DgSolveInfo), vp]
        L.dg_rhs_sine.argtypes = [vp, C.c_int, dp, dp, dp, vp]
        L.dg_rhs_eval.argtypes = [vp, DgFieldFn, DgFieldFn, vp, dp, vp]
        L.dg_last_error.restype = C.c_char_p
        L.dg_batch_create.argtypes = [C.POINTER(DgMeshDesc), C.c_int, C.c_int, C.POINTER(DgOptions), vp,
                                      C.POINTER(vp)]
        L.dg_batch_destroy.argtypes = [vp]
        L.dg_batch_destroy.restype = None
        L.dg_batch_num_dofs.argtypes = [vp]
        L.dg_batch_num_dofs.restype = i64
        L.dg_batch_offsets.argtypes = [vp, vp]
        L.dg_batch_stats_get.argtypes = [vp, C.POINTER(DgMeshStats)]
        L.dg_batch_rhs_sine.argtypes = [vp, C.c_int, dp, dp, dp, vp]
        L.dg_batch_solve.argtypes = [vp, dp, dp, C.c_double, C.c_int, C.POINTER(DgSolveInfo),
                                     C.POINTER(C.c_double), vp]
        for name in ABI_SYMBOLS:
            if name not in ("dg_mesh_destroy", "dg_precond_destroy", "dg_num_dofs", "dg_last_error",
                            "dg_batch_destroy", "dg_batch_num_dofs"):
                getattr(L, name).restype = st
        L.dg_mesh_destroy.restype = None
        L.dg_precond_destroy.restype = None
        _lib = L
    return _lib


class DGError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"dg status {code}: {msg}")
        self.code = code


def _check(code: int) -> None:
    if code != DG_OK:
        raise DGError(code, lib().dg_last_error().decode())


def _ptr(t) -> int:
    if t is None:
        return 0
    if isinstance(t, int):
        return t
    return int(t.data_ptr())


def _stream(s) -> int:
    if s is None:
        return 0
    if isinstance(s, int):
        return s
    return int(s.cuda_stream)


def make_desc(mesh: MeshDesc):
    lo = np.ascontiguousarray(mesh.lo, dtype=np.int32)
    size = np.ascontiguousarray(mesh.size, dtype=np.int32)
    p = np.ascontiguousarray(mesh.p, dtype=np.int32)
    ext = np.ascontiguousarray(mesh.extent, dtype=np.int32)
    coeff = getattr(mesh, "coeff", None)
    if coeff is not None:
        coeff = np.ascontiguousarray(coeff, dtype=np.float64)
    corners = getattr(mesh, "corners", None)
    if corners is not None:
        corners = np.ascontiguousarray(corners, dtype=np.float64).reshape(8)
    mapping = getattr(mesh, "mapping", None)
    fn = _map_callback(mapping) if mapping is not None else DgMapFn()
    keep = (lo, size, p, ext, coeff, corners, fn)
    d = DgMeshDesc(mesh.dim, mesh.n_elems, lo.ctypes.data_as(C.POINTER(C.c_int32)),
                   size.ctypes.data_as(C.POINTER(C.c_int32)), p.ctypes.data_as(C.POINTER(C.c_int32)),
                   ext.ctypes.data_as(C.POINTER(C.c_int32)), float(mesh.lattice_h),
                   None if coeff is None else coeff.ctypes.data_as(C.POINTER(C.c_double)),
                   None if corners is None else corners.ctypes.data_as(C.POINTER(C.c_double)),
                   fn, None)
    return d, keep


def make_options(form=DG_FORM_SIPG, eta=0.0, penalty_form=DG_PENALTY_PAPER, precision=DG_PREC_FP64,
                 lor=DG_LOR_AMG, smoother=DG_SMOOTHER_FULL, remark_cases=0, tune_tiles=0) -> DgOptions:
    return DgOptions(form, eta, penalty_form, precision, lor, smoother, remark_cases, tune_tiles)


# ------------------------------------------------------------ C-named calls
def dg_mesh_create(mesh: MeshDesc, opts: Optional[DgOptions] = None, stream=None) -> int:
    d, keep = make_desc(mesh)
    h = C.c_void_p()
    _check(lib().dg_mesh_create(C.byref(d), C.byref(opts) if opts else None, _stream(stream), C.byref(h)))
    return h.value


def dg_mesh_destroy(h: int) -> None:
    lib().dg_mesh_destroy(h)


def dg_num_dofs(h: int) -> int:
    return int(lib().dg_num_dofs(h))


def dg_mesh_stats_get(h: int) -> DgMeshStats:
    s = DgMeshStats()
    _check(lib().dg_mesh_stats_get(h, C.byref(s)))
    return s


def dg_dof_layout(h: int, n_elems: int) -> np.ndarray:
    """Offsets of each element's first DG entry (n_elems + 1 values)."""
    out = np.zeros(n_elems + 1, dtype=np.int64)
    _check(lib().dg_dof_layout(h, out.ctypes.data))
    return out


def dg_apply(h: int, x, y, stream=None) -> None:
    _check(lib().dg_apply(h, _ptr(x), _ptr(y), _stream(stream)))


def dg_precond_setup(mesh_h: int, opts: Optional[DgOptions] = None) -> int:
    h = C.c_void_p()
    _check(lib().dg_precond_setup(mesh_h, C.byref(opts) if opts else None, C.byref(h)))
    return h.value


def dg_precond_destroy(h: int) -> None:
    lib().dg_precond_destroy(h)


def dg_precond_stats_get(h: int) -> DgPrecondStats:
    s = DgPrecondStats()
    _check(lib().dg_precond_stats_get(h, C.byref(s)))
    return s


def dg_precond_apply(h: int, r, z, stream=None) -> None:
    _check(lib().dg_precond_apply(h, _ptr(r), _ptr(z), _stream(stream)))


def dg_precond_profile(h: int, r, z, stream=None) -> DgPrecondTimes:
    t = DgPrecondTimes()
    _check(lib().dg_precond_profile(h, _ptr(r), _ptr(z), C.byref(t), _stream(stream)))
    return t


def dg_apply_profile(h: int, x, y, stream=None) -> DgApplyTimes:
    t = DgApplyTimes()
    _check(lib().dg_apply_profile(h, _ptr(x), _ptr(y), C.byref(t), _stream(stream)))
    return t


def dg_fp64_fma_probe(iters: int = 20000, stream=None):
    """(TFLOP/s, ms) of the FP64 FMA-chain probe."""
    tf, ms = C.c_double(), C.c_double()
    _check(lib().dg_fp64_fma_probe(iters, C.byref(tf), C.byref(ms), _stream(stream)))
    return tf.value, ms.value


def dg_pcg_solve(mesh_h: int, pc_h: int, b, x, rtol: float, maxit: int, stream=None,
                 raise_on_notconv: bool = True) -> DgSolveInfo:
    info = DgSolveInfo()
    code = lib().dg_pcg_solve(mesh_h, pc_h, _ptr(b), _ptr(x), rtol, maxit, C.byref(info), _stream(stream))
    if code != DG_ENOTCONV or raise_on_notconv:
        _check(code)
    return info


def _host_ptr(a) -> int:
    if isinstance(a, np.ndarray):
        assert a.dtype == np.float64 and a.flags.c_contiguous
        return a.ctypes.data
    return _ptr(a)   # a CPU torch tensor (e.g. pinned) or a raw address


def dg_pcg_solve_host(mesh_h: int, pc_h: int, b, x, rtol: float, maxit: int, stream=None) -> DgSolveInfo:
    """b, x: host float64 buffers (numpy arrays, CPU tensors or addresses)."""
    info = DgSolveInfo()
    _check(lib().dg_pcg_solve_host(mesh_h, pc_h, _host_ptr(b), _host_ptr(x), rtol, maxit,
                                   C.byref(info), _stream(stream)))
    return info


def dg_pcg_solve_noalloc(mesh_h: int, pc_h: int, b, x, rtol: float, maxit: int, stream=None) -> DgSolveInfo:
    """PCG that allocates nothing at call time (fixed library-wide device
    scratch, at most 262144 unknowns; see include/dg.h)."""
    info = DgSolveInfo()
    _check(lib().dg_pcg_solve_noalloc(mesh_h, pc_h or 0, _ptr(b), _ptr(x), rtol, maxit, C.byref(info),
                                      _stream(stream)))
    return info


def dg_rhs_eval(mesh_h: int, f, g, b, stream=None) -> None:
    """b = load vector of f (volume) and weakly imposed boundary data g (SIPG);
    f, g: Python functions of the (n, 2) physical points, or None."""
    cf, cg = _field_callback(f), _field_callback(g)
    _check(lib().dg_rhs_eval(mesh_h, cf, cg, None, _ptr(b), _stream(stream)))


def dg_rhs_sine(mesh_h: int, amps, waves, b, stream=None) -> None:
    a = np.ascontiguousarray(amps, dtype=np.float64)
    w = np.ascontiguousarray(waves, dtype=np.int32)
    _check(lib().dg_rhs_sine(mesh_h, len(a), a.ctypes.data, w.ctypes.data, _ptr(b), _stream(stream)))


# ------------------------------------------------------------ handles with lifetime
class Mesh:
    def __init__(self, mesh: MeshDesc, opts: Optional[DgOptions] = None, stream=None):
        self.desc = mesh
        self.opts = opts or make_options()
        self.h = dg_mesh_create(mesh, self.opts, stream)
        self.n_dofs = dg_num_dofs(self.h)
        self.stats = dg_mesh_stats_get(self.h)

    def close(self):
        if self.h:
            dg_mesh_destroy(self.h)
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Precond:
    def __init__(self, mesh: Mesh, opts: Optional[DgOptions] = None):
        self.mesh = mesh
        self.h = dg_precond_setup(mesh.h, opts or mesh.opts)
        self.stats = dg_precond_stats_get(self.h)

    def close(self):
        if self.h:
            dg_precond_destroy(self.h)
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many problems x n_rhs right-hand sides solved by one graph launch."""

    def __init__(self, meshes, n_rhs: int = 1, opts: Optional[DgOptions] = None, stream=None):
        descs = (DgMeshDesc * len(meshes))()
        self._keep = []
        for i, m in enumerate(meshes):
            d, keep = make_desc(m)
            descs[i] = d
            self._keep.append(keep)
        self.n_problems = len(meshes)
        self.n_rhs = n_rhs
        self.n_inst = len(meshes) * n_rhs
        o = opts or make_options(precision=DG_PREC_MIXED)
        h = C.c_void_p()
        _check(lib().dg_batch_create(descs, len(meshes), n_rhs, C.byref(o), _stream(stream), C.byref(h)))
        self.h = h.value
        self.n_dofs = int(lib().dg_batch_num_dofs(self.h))
        off = np.zeros(self.n_inst + 1, dtype=np.int64)
        _check(lib().dg_batch_offsets(self.h, off.ctypes.data))
        self.offsets = off
        self.stats = DgMeshStats()
        _check(lib().dg_batch_stats_get(self.h, C.byref(self.stats)))

    def rhs_sine(self, rhs_list, b, stream=None):
        """rhs_list: one SineRHS per instance (same number of modes)."""
        amps = np.ascontiguousarray(np.concatenate([r.amps for r in rhs_list]), dtype=np.float64)
        waves = np.ascontiguousarray(np.concatenate([np.asarray(r.waves).ravel() for r in rhs_list]),
                                     dtype=np.int32)
        _check(lib().dg_batch_rhs_sine(self.h, len(rhs_list[0].amps), amps.ctypes.data, waves.ctypes.data,
                                       _ptr(b), _stream(stream)))

    def solve(self, b, x, rtol: float, maxit: int, stream=None, raise_on_notconv: bool = True):
        res = (DgSolveInfo * self.n_inst)()
        ms = C.c_double()
        code = lib().dg_batch_solve(self.h, _ptr(b), _ptr(x), rtol, maxit, res, C.byref(ms), _stream(stream))
        if code != DG_ENOTCONV or raise_on_notconv:
            _check(code)
        return list(res), ms.value

    def close(self):
        if self.h:
            lib().dg_batch_destroy(self.h)
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------ host inspection
def inspect_lib():
    global _inspect
    if _inspect is None:
        L = _load(INSPECT_PATH)
        vp = C.c_void_p
        L.dginspect_create.argtypes = [C.POINTER(DgMeshDesc), C.POINTER(DgOptions), C.c_int]
        L.dginspect_create.restype = vp
        L.dginspect_last_status.restype = C.c_int
        L.dginspect_rhs_eval.argtypes = [vp, DgFieldFn, DgFieldFn, vp, C.c_void_p]
        L.dginspect_rhs_eval.restype = C.c_int
        L.dginspect_destroy.argtypes = [vp]
        L.dginspect_last_error.restype = C.c_char_p
        for n in ("dginspect_sizes", "dginspect_kind", "dginspect_dinv"):
            getattr(L, n).argtypes = [vp, vp]
        for n in ("dginspect_P", "dginspect_lor"):
            getattr(L, n).argtypes = [vp, vp, vp, vp]
        L.dginspect_blocks.argtypes = [vp, vp, vp, vp]
        L.dginspect_level_rows.argtypes = [vp, C.c_int]
        L.dginspect_level_rows.restype = C.c_int64
        L.dginspect_level_nnz.argtypes = [vp, C.c_int]
        L.dginspect_level_nnz.restype = C.c_int64
        L.dginspect_level_A.argtypes = [vp, C.c_int, vp, vp, vp]
        L.dginspect_apply.argtypes = [vp, vp, vp]
        L.dginspect_item_sizes.argtypes = [vp, vp]
        L.dginspect_items.argtypes = [vp, vp, vp, vp, vp]
        L.dginspect_block_units.argtypes = [C.c_int64, vp, vp, vp, vp, vp, vp, C.c_int64]
        L.dginspect_block_units.restype = C.c_int64
        L.dginspect_csr_tiers.argtypes = [C.c_int64, vp, vp, vp, vp, vp]
        L.dginspect_csr_tiers.restype = C.c_int
        _inspect = L
    return _inspect


def plan_block_units(dims, slot, inv_off):
    """The library's block-solve work units for blocks of the given sizes
    (host planning only): (unit int32 (n, 4), ubase int64 (n,), brec int32 (m, 4))."""
    L = inspect_lib()
    dims = np.ascontiguousarray(dims, dtype=np.int32)
    slot = np.ascontiguousarray(slot, dtype=np.int32)
    inv_off = np.ascontiguousarray(inv_off, dtype=np.int64)
    nb = len(dims)
    cap = int(np.sum((dims.astype(np.int64) + 31) // 32)) + nb + 1
    unit = np.zeros((cap, 4), dtype=np.int32)
    ubase = np.zeros(cap, dtype=np.int64)
    brec = np.zeros((max(nb, 1), 4), dtype=np.int32)
    n = L.dginspect_block_units(nb, dims.ctypes.data, slot.ctypes.data, inv_off.ctypes.data,
                                unit.ctypes.data, ubase.ctypes.data, brec.ctypes.data, cap)
    if n < 0:
        raise DGError(DG_EINVAL, L.dginspect_last_error().decode())
    m = int(np.sum(unit[:n, 1][unit[:n, 3] != 0]))
    return unit[:n].copy(), ubase[:n].copy(), brec[:m].copy()


def plan_csr_tiers(ptr):
    """The library's row tiers of the CSR row kernel for row pointers `ptr`
    (host planning only): (group, long_min, cta rows, warp rows)."""
    L = inspect_lib()
    ptr = np.ascontiguousarray(ptr, dtype=np.int64)
    rows = len(ptr) - 1
    out2 = np.zeros(2, dtype=np.int32)
    counts = np.zeros(2, dtype=np.int64)
    cta = np.zeros(max(rows, 1), dtype=np.int32)
    warp = np.zeros(max(rows, 1), dtype=np.int32)
    if L.dginspect_csr_tiers(rows, ptr.ctypes.data, out2.ctypes.data, counts.ctypes.data, cta.ctypes.data,
                             warp.ctypes.data) != 0:
        raise DGError(DG_EINVAL, L.dginspect_last_error().decode())
    return int(out2[0]), int(out2[1]), cta[:counts[0]].copy(), warp[:counts[1]].copy()


class HostSetup:
    """The library's host-side setup, run without a GPU (inspection only)."""

    def __init__(self, mesh: MeshDesc, opts: Optional[DgOptions] = None, amg: bool = True):
        import scipy.sparse as sp
        self._sp = sp
        L = inspect_lib()
        d, keep = make_desc(mesh)
        o = opts or make_options()
        self.h = L.dginspect_create(C.byref(d), C.byref(o), 1 if amg else 0)
        if not self.h:
            raise DGError(int(L.dginspect_last_status()), L.dginspect_last_error().decode())
        s = np.zeros(9, dtype=np.int64)
        L.dginspect_sizes(self.h, s.ctypes.data)
        self.n, self.nC, nnzP, nnzA, nb, nbd, self.n_levels, eta, nsq = (int(v) for v in s)
        self.eta = eta / 1e6
        self.P = self._csr(L.dginspect_P, self.n, self.nC, nnzP)
        self.Ac = self._csr(L.dginspect_lor, self.nC, self.nC, nnzA)
        self.kind = np.zeros(self.n, dtype=np.int8)
        L.dginspect_kind(self.h, self.kind.ctypes.data)
        self.dinv = np.zeros(self.n)
        L.dginspect_dinv(self.h, self.dinv.ctypes.data)
        off = np.zeros(nb + 1, dtype=np.int64)
        nodes = np.zeros(max(nbd, 1), dtype=np.int64)
        inv = np.zeros(max(nsq, 1))
        L.dginspect_blocks(self.h, off.ctypes.data, nodes.ctypes.data, inv.ctypes.data)
        self.blocks = [nodes[off[i]:off[i + 1]].copy() for i in range(nb)]
        self.block_inv = []
        q = 0
        for b in self.blocks:
            d2 = len(b) * len(b)
            self.block_inv.append(inv[q:q + d2].reshape(len(b), len(b)).copy())
            q += d2
        self.levels = []
        for l in range(self.n_levels):
            r = int(L.dginspect_level_rows(self.h, l))
            nz = int(L.dginspect_level_nnz(self.h, l))
            self.levels.append(self._csr(lambda h, a, b, c, l=l: L.dginspect_level_A(h, l, a, b, c), r, r, nz))

    def _csr(self, fn, rows, cols, nnz):
        ptr = np.zeros(rows + 1, dtype=np.int64)
        idx = np.zeros(max(nnz, 1), dtype=np.int32)
        val = np.zeros(max(nnz, 1))
        fn(self.h, ptr.ctypes.data, idx.ctypes.data, val.ctypes.data)
        return self._sp.csr_matrix((val[:nnz], idx[:nnz], ptr), shape=(rows, cols))

    def apply(self, x: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.zeros(self.n)
        inspect_lib().dginspect_apply(self.h, x.ctypes.data, y.ctypes.data)
        return y

    def rhs_eval(self, f, g) -> np.ndarray:
        """The library's load vector of f and boundary data g (host_load)."""
        L = inspect_lib()
        b = np.zeros(self.n)
        if L.dginspect_rhs_eval(self.h, _field_callback(f), _field_callback(g), None, b.ctypes.data) != 0:
            raise DGError(DG_EINVAL, L.dginspect_last_error().decode())
        return b

    def face_items(self):
        """The operator's tiles and sub-face items as the kernels read them:
        (item_ptr, items (n, 2), chunk per tile, info (n, 3): interior,
        neighbour degree, whole-side flags)."""
        L = inspect_lib()
        s = np.zeros(3, dtype=np.int64)
        L.dginspect_item_sizes(self.h, s.ctypes.data)
        nt, ni = int(s[0]), int(s[1])
        ptr = np.zeros(nt + 1, dtype=np.int32)
        items = np.zeros(2 * max(ni, 1), dtype=np.int32)
        chunk = np.zeros(max(nt, 1), dtype=np.int32)
        info = np.zeros(3 * max(ni, 1), dtype=np.int32)
        L.dginspect_items(self.h, ptr.ctypes.data, items.ctypes.data, chunk.ctypes.data, info.ctypes.data)
        return ptr, items[:2 * ni].reshape(ni, 2), chunk[:nt], info[:3 * ni].reshape(ni, 3)

    def __del__(self):
        try:
            inspect_lib().dginspect_destroy(self.h)
        except Exception:
            pass

