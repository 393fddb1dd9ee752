"""The library's host setup on mapped squares (Section 2 element maps onto
general quadrilaterals), run through the inspection library without a GPU,
against the oracle's mapped space: the host mirror of the mapped operator
kernel, the conforming prolongation, the V_J / V_e split, the Q1 LOR matrix on
the mapped cells, the block inverses, the Jacobi diagonal and the AMG
hierarchy, for SIPG and BR2; and the input checks of mapped meshes."""
import numpy as np
import pytest

from oracle import solver
from paper_2009_01287_gb300 import inputs


def _coef(mesh, base):
    return inputs.with_coeff(mesh, inputs.base_parity_coeff(mesh, base))


CASES = [
    ("par-hp", lambda: inputs.with_corners(inputs.small_hp_mesh(1, base=4, depth=3, prob=0.4, pmax=5),
                                           inputs.PARALLELOGRAM)),
    ("quad-hp", lambda: inputs.with_corners(inputs.small_hp_mesh(2, base=4, depth=3, prob=0.4, pmax=6),
                                            inputs.QUADRILATERAL)),
    ("quad-p8", lambda: inputs.with_corners(inputs.small_hp_mesh(3, base=3, depth=2, prob=0.5, pmin=6, pmax=8),
                                            inputs.QUADRILATERAL)),
    ("quad-coef", lambda: inputs.with_corners(_coef(inputs.small_hp_mesh(4, base=4, depth=3, prob=0.4, pmax=5), 4),
                                              inputs.QUADRILATERAL)),
    ("quad-ragged", lambda: inputs.with_corners(inputs.random_refined_mesh(2, 5, 3, 0.35, 1, 4, seed=9, base_y=3),
                                                ((0.0, 0.0), (1.1, 0.2), (-0.1, 0.6), (0.9, 0.75)))),
]


@pytest.mark.parametrize("name,mk", CASES, ids=[c[0] for c in CASES])
def test_host_setup_matches_oracle_mapped(built_lib, name, mk, form="sipg"):
    mesh = mk()
    prob = solver.build_problem(mesh, form=form)
    B = built_lib
    hs = B.HostSetup(mesh, B.make_options(form=B.DG_FORM_BR2 if form == "br2" else B.DG_FORM_SIPG))
    assert abs(hs.eta - (dg_br2_eta(prob) if form == "br2" else 100.0)) < 1e-6
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


def dg_br2_eta(prob):
    from oracle import dg
    return dg.br2_eta(prob.topo)


@pytest.mark.parametrize("name,mk", CASES[:3] + [
    ("wavy-br2", lambda: inputs.with_mapping(inputs.small_hp_mesh(6, base=4, depth=3, prob=0.4, pmax=5),
                                             inputs.WavyMap()))], ids=["par-hp", "quad-hp", "quad-p8", "wavy-br2"])
def test_host_setup_matches_oracle_mapped_br2(built_lib, name, mk):
    test_host_setup_matches_oracle_mapped(built_lib, name, mk, form="br2")


def test_similarity_corners_give_the_box_operator(built_lib):
    """A rotated, scaled, shifted square gives the operator of the boxes."""
    mesh = inputs.small_hp_mesh(5, base=3, depth=2, prob=0.5, pmax=6)
    th, s, sh = -0.4, 0.8, np.array([2.0, 1.0])
    R = s * np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    L = mesh.extent[0] * mesh.lattice_h
    corners = [sh, sh + R @ [L, 0], sh + R @ [0, L], sh + R @ [L, L]]
    B = built_lib
    a = B.HostSetup(mesh, B.make_options(), amg=False)
    b = B.HostSetup(inputs.with_corners(mesh, corners), B.make_options(), amg=False)
    x = inputs.random_vector(a.n, 2)
    ya, yb = a.apply(x), b.apply(x)
    assert np.abs(ya - yb).max() <= 1e-12 * np.abs(ya).max()
    assert abs(a.Ac - b.Ac).max() <= 1e-12 * abs(a.Ac).max()


def test_mapped_input_checks(built_lib):
    B = built_lib
    mesh = inputs.small_hp_mesh(1)
    with pytest.raises(B.DGError) as e:
        B.HostSetup(inputs.with_corners(mesh, ((0, 0), (1, 0), (0, 1), (0.2, 0.2))), B.make_options())
    assert e.value.code == B.DG_EINVAL
    # clockwise corners (a reflection) are rejected too
    with pytest.raises(B.DGError):
        B.HostSetup(inputs.with_corners(mesh, ((0, 0), (0, 1), (1, 0), (1, 1))), B.make_options())
    with pytest.raises(B.DGError):
        B.HostSetup(inputs.with_corners(mesh, ((0, 0), (1, 0), (0, 1), (np.nan, 1))), B.make_options())


# ---------------------------------------------------------------- curved maps
CURVED = [
    ("wavy-hp", lambda: inputs.with_mapping(inputs.small_hp_mesh(1, base=4, depth=3, prob=0.4, pmax=5),
                                            inputs.WavyMap())),
    ("wavy-coef-p8", lambda: inputs.with_mapping(
        _coef(inputs.small_hp_mesh(3, base=3, depth=2, prob=0.5, pmin=5, pmax=8), 3), inputs.WavyMap(ax=0.1))),
]


@pytest.mark.parametrize("name,mk", CURVED, ids=[c[0] for c in CURVED])
def test_host_setup_matches_oracle_curved(built_lib, name, mk):
    test_host_setup_matches_oracle_mapped(built_lib, name, mk)


def test_bilinear_callback_matches_corners(built_lib):
    """The corners' bilinear map given through the map callback builds the
    same operator and LOR matrix as the corners themselves."""
    from oracle.geometry import BilinearMap
    mesh = inputs.small_hp_mesh(2, base=4, depth=3, prob=0.4, pmax=6)
    L = mesh.extent[0] * mesh.lattice_h
    B = built_lib
    a = B.HostSetup(inputs.with_corners(mesh, inputs.QUADRILATERAL), B.make_options(), amg=False)
    b = B.HostSetup(inputs.with_mapping(mesh, BilinearMap(inputs.QUADRILATERAL, L, L)), B.make_options(),
                    amg=False)
    x = inputs.random_vector(a.n, 5)
    ya, yb = a.apply(x), b.apply(x)
    assert np.abs(ya - yb).max() <= 1e-13 * np.abs(ya).max()
    assert abs(a.Ac - b.Ac).max() <= 1e-13 * abs(a.Ac).max()


class _Folded(inputs.WavyMap):
    """A map that folds the domain over (det J < 0 inside)."""
    def jacobian(self, X):
        J = super().jacobian(X)
        J[:, 1, 1] = -0.5
        return J


class _Broken(inputs.WavyMap):
    def __call__(self, X):
        raise RuntimeError("no geometry here")


def test_curved_input_checks(built_lib):
    B = built_lib
    mesh = inputs.small_hp_mesh(1)
    for bad in (_Folded(), _Broken()):
        with pytest.raises(B.DGError) as e:
            B.HostSetup(inputs.with_mapping(mesh, bad), B.make_options())
        assert e.value.code == B.DG_EINVAL
    both = inputs.with_mapping(inputs.with_corners(mesh, inputs.QUADRILATERAL), inputs.WavyMap())
    with pytest.raises(B.DGError):
        B.HostSetup(both, B.make_options())


# ---------------------------------------------------------------- load vectors from callbacks
def test_host_load_matches_oracle(built_lib):
    """The library's load vector of caller-supplied f and weakly imposed
    Dirichlet data g (host_load) against the oracle's dirichlet_load, on a
    hanging hp mesh with a coefficient, on a mapped quadrilateral and on
    curved elements (f alone and with g)."""
    from oracle import rhs as R
    B = built_lib
    f = lambda x: np.sin(3 * x[:, 0]) * np.exp(x[:, 1])
    g = lambda x: np.arctan(20.0 * (np.hypot(x[:, 0] + 0.05, x[:, 1] + 0.05) - 0.7))
    mesh = _coef(inputs.small_hp_mesh(4, base=4, depth=3, prob=0.4, pmax=6), 4)
    prob = solver.build_problem(mesh)
    hs = B.HostSetup(mesh, B.make_options(), amg=False)
    ref = R.dirichlet_load(prob.space, f, g, 100.0)
    assert np.abs(hs.rhs_eval(f, g) - ref).max() <= 1e-12 * np.abs(ref).max()
    base = inputs.small_hp_mesh(5, base=3, depth=2, prob=0.5, pmax=5)
    for md in (inputs.with_mapping(base, inputs.WavyMap()),
               inputs.with_corners(_coef(base, 3), inputs.QUADRILATERAL)):
        prob = solver.build_problem(md)
        hs = B.HostSetup(md, B.make_options(), amg=False)
        ref = R.load_vector_fn(prob.space, f)
        assert np.abs(hs.rhs_eval(f, None) - ref).max() <= 1e-12 * np.abs(ref).max()
        ref = R.dirichlet_load(prob.space, f, g, 100.0)
        assert np.abs(hs.rhs_eval(f, g) - ref).max() <= 1e-12 * np.abs(ref).max()
    with pytest.raises(B.DGError):
        hs.rhs_eval(lambda x: x[:, 5], None)   # a failing callback
    hb = B.HostSetup(md, B.make_options(form=B.DG_FORM_BR2), amg=False)
    with pytest.raises(B.DGError):
        hb.rhs_eval(f, g)   # boundary data: SIPG only


def test_mapped_cubes_refused(built_lib):
    B = built_lib
    mesh = inputs.small_hp_mesh(0, base=2, depth=1, prob=0.4, pmin=1, pmax=2, dim=3)
    with pytest.raises(B.DGError) as e:
        B.HostSetup(inputs.with_mapping(mesh, inputs.WavyMap()), B.make_options())
    assert e.value.code == B.DG_EUNSUPPORTED
    bad = inputs.MeshDesc(dim=3, lo=mesh.lo, size=mesh.size, p=mesh.p, extent=mesh.extent,
                          lattice_h=mesh.lattice_h, corners=np.zeros((4, 2)))
    with pytest.raises(B.DGError) as e:
        B.HostSetup(bad, B.make_options())
    assert e.value.code == B.DG_EUNSUPPORTED


def test_load_callback_that_writes_nothing_is_reported(built_lib):
    """A C callback that leaves its outputs unwritten: the library pre-fills
    them with NaN and reports DG_EINVAL instead of using stale values."""
    B = built_lib
    L = B.inspect_lib()
    silent = B.DgFieldFn(lambda n, x, out, ctx: None)
    for mesh in (inputs.uniform_mesh(2, 2, 2), inputs.with_mapping(inputs.uniform_mesh(2, 2, 2), inputs.WavyMap())):
        hs = B.HostSetup(mesh, B.make_options(), amg=False)
        b = np.zeros(hs.n)
        assert L.dginspect_rhs_eval(hs.h, silent, B.DgFieldFn(), None, b.ctypes.data) != 0
        assert L.dginspect_rhs_eval(hs.h, B.DgFieldFn(), silent, None, b.ctypes.data) != 0
        assert L.dginspect_rhs_eval(hs.h, B.DgFieldFn(), B.DgFieldFn(), None, b.ctypes.data) == 0
        assert not b.any()


# ---------------------------------------------------------------- mapped domains with holes
HOLED = [
    ("lshape-quad", lambda: inputs.with_corners(
        inputs.lshape(inputs.small_hp_mesh(8, base=4, depth=3, prob=0.4, pmax=6)), inputs.QUADRILATERAL)),
    ("lshape-wavy", lambda: inputs.with_mapping(
        inputs.lshape(inputs.small_hp_mesh(7, base=4, depth=2, prob=0.5, pmax=5)), inputs.WavyMap())),
]


@pytest.mark.parametrize("form", ["sipg", "br2"])
@pytest.mark.parametrize("name,mk", HOLED, ids=[c[0] for c in HOLED])
def test_host_setup_matches_oracle_mapped_holes(built_lib, name, mk, form):
    """L-shaped lattices (a hole) carried by the bilinear and the curved map:
    the boundary sub-faces along the hole take the mapped face factors."""
    test_host_setup_matches_oracle_mapped(built_lib, name, mk, form=form)


@pytest.mark.parametrize("name,mk", HOLED, ids=[c[0] for c in HOLED])
def test_host_load_mapped_holes(built_lib, name, mk):
    from oracle import rhs as R
    mesh = mk()
    prob = solver.build_problem(mesh)
    hs = built_lib.HostSetup(mesh, built_lib.make_options(), amg=False)
    f = lambda x: np.cos(2 * x[:, 0]) + x[:, 1]
    g = lambda x: np.hypot(x[:, 0] - 0.5, x[:, 1] - 0.5) ** (2.0 / 3.0)
    ref = R.dirichlet_load(prob.space, f, g, 100.0)
    assert np.abs(hs.rhs_eval(f, g) - ref).max() <= 1e-12 * np.abs(ref).max()
