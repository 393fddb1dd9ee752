"""Pins of the oracle's mapped elements (Section 2: element maps T_kappa onto
general quadrilaterals), each against something the mathematics fixes:
  - a similarity map (rotation, scaling, shift) leaves the 2D SIPG matrix and
    the LOR matrix unchanged;
  - on an affine (sheared) map, a manufactured solution in the DG space is
    reproduced exactly, with -Laplace(u) formed in closed form;
  - on a bilinear map, harmonic polynomials that lie in the space give zero
    residual on every element away from the boundary (element-wise
    integration by parts, exact under the quadrature rule), and linear
    functions do the same for the Q1 LOR blocks at the sub-grid's interior
    nodes;
  - element areas sum to the shoelace area of the domain, the load vector of
    f = 1 sums to it, and the matrix is SPD;
  - curved maps (a caller's smooth map): the map's Jacobian against finite
    differences, areas against a global high-order rule, a bilinear map given
    as a generic map gives the corner form's matrix, and the nodal error of a
    manufactured solution on the curved domain (f by symbolic differentiation
    of the pulled-back Laplacian) falls like h^(p+1) under refinement."""
import numpy as np
import pytest

from oracle import geometry, rhs, solver
from paper_2009_01287_gb300 import inputs


def _mesh(seed=1, pmin=1, pmax=4, base=3, depth=2):
    return inputs.small_hp_mesh(seed, base=base, depth=depth, prob=0.5, pmin=pmin, pmax=pmax)


def _shoelace(c):
    q = np.asarray(c)[[0, 1, 3, 2]]      # corners in boundary order
    x, y = q[:, 0], q[:, 1]
    return 0.5 * abs(np.dot(x, np.roll(y, -1)) - np.dot(y, np.roll(x, -1)))


def _interior_elements(topo):
    bnd = set()
    for f in topo.subfaces:
        if f.kp < 0:
            bnd.add(f.km)
    return [k for k in range(topo.n) if k not in bnd]


def test_bilinear_map_corners_and_jacobian():
    c = np.array(inputs.QUADRILATERAL)
    F = geometry.BilinearMap(c, 2.0, 3.0)
    X = np.array([[0, 0], [2, 0], [0, 3], [2, 3]], dtype=float)
    assert np.allclose(F(X), c, atol=1e-15)
    # the Jacobian against central differences of the map
    rng = np.random.default_rng(0)
    P = rng.uniform([0, 0], [2, 3], size=(5, 2))
    e = 1e-6
    for j in range(2):
        d = np.zeros(2)
        d[j] = e
        fd = (F(P + d) - F(P - d)) / (2 * e)
        assert np.allclose(F.jacobian(P)[:, :, j], fd, atol=1e-8)


def test_similarity_map_leaves_matrices_unchanged():
    mesh = _mesh(2, pmax=5)
    th, s, sh = 0.7, 1.3, np.array([0.4, -0.2])
    R = s * np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    L = mesh.extent[0] * mesh.lattice_h
    corners = [sh, sh + R @ [L, 0], sh + R @ [0, L], sh + R @ [L, L]]
    pa = solver.build_problem(mesh)
    pb = solver.build_problem(inputs.with_corners(mesh, corners))
    assert abs(pa.A - pb.A).max() <= 1e-12 * abs(pa.A).max()
    pca = solver.Preconditioner(pa, lor="exact")
    pcb = solver.Preconditioner(pb, lor="exact")
    assert abs(pca.Ac - pcb.Ac).max() <= 1e-12 * abs(pca.Ac).max()
    for k in range(pa.topo.n):
        assert abs(pb.space.hpen(k) - s * pa.space.hpen(k)) <= 1e-14


def test_affine_map_reproduces_manufactured_solution():
    # u = U(Phi^{-1}(x)), U(X, Y) = X (L - X) Y (L - Y): zero on the boundary
    # of the parallelogram, in Q_2 of every element, so the discrete solution
    # is u itself
    mesh = _mesh(3, pmin=2, pmax=4)
    c = np.array(inputs.PARALLELOGRAM)
    md = inputs.with_corners(mesh, c)
    L = mesh.extent[0] * mesh.lattice_h
    A = np.stack([(c[1] - c[0]) / L, (c[2] - c[0]) / L], axis=1)      # x = c0 + A X
    Ai = np.linalg.inv(A)
    Gm = Ai @ Ai.T                                                   # d^2 / dx^2 = Ai^T H_X Ai

    def pre(x):
        return (x - c[0]) @ Ai.T

    def u(x):
        X = pre(x)
        return X[:, 0] * (L - X[:, 0]) * X[:, 1] * (L - X[:, 1])

    def f(x):   # -Laplace(u) = -tr(Gm H_X U)
        X, Y = pre(x).T
        hxx = -2.0 * Y * (L - Y)
        hyy = -2.0 * X * (L - X)
        hxy = (L - 2 * X) * (L - 2 * Y)
        return -(Gm[0, 0] * hxx + 2 * Gm[0, 1] * hxy + Gm[1, 1] * hyy)

    prob = solver.build_problem(md)
    b = rhs.load_vector_fn(prob.space, f, extra=3)
    x = np.linalg.solve(prob.A.toarray(), b)
    ui = rhs.interpolate(prob.space, u)
    assert np.abs(x - ui).max() <= 1e-10 * np.abs(ui).max()


@pytest.mark.parametrize("fn", ["x2-y2", "xy", "linear"])
def test_bilinear_map_harmonic_patch(fn):
    pmin = 1 if fn == "linear" else 2
    mesh = _mesh(4, pmin=pmin, pmax=5, base=4)
    md = inputs.with_corners(mesh, inputs.QUADRILATERAL)
    prob = solver.build_problem(md)
    u = {"x2-y2": lambda x: x[:, 0] ** 2 - x[:, 1] ** 2,
         "xy": lambda x: x[:, 0] * x[:, 1],
         "linear": lambda x: 0.3 * x[:, 0] - 1.7 * x[:, 1] + 0.2}[fn]
    ui = rhs.interpolate(prob.space, u)
    r = prob.A @ ui
    inner = _interior_elements(prob.topo)
    assert inner
    scale = np.abs(prob.A).max() * np.abs(ui).max()
    for k in inner:
        assert np.abs(r[prob.space.dofs(k)]).max() <= 1e-12 * scale
    # the boundary rows do carry the boundary terms
    assert np.abs(r).max() > 1e-6 * scale


def test_bilinear_map_lor_patch():
    mesh = _mesh(5, pmin=2, pmax=6)
    md = inputs.with_corners(mesh, inputs.QUADRILATERAL)
    prob = solver.build_problem(md)
    u = lambda x: 0.8 * x[:, 0] + 0.5 * x[:, 1] - 0.1
    for k in range(prob.topo.n):
        p = int(prob.topo.p[k])
        Ak = geometry.lor_element_mapped(prob.space, k)
        assert np.abs(Ak - Ak.T).max() <= 1e-13 * np.abs(Ak).max()
        r = Ak @ u(prob.space.node_coords(k))
        n = p + 1
        for j in range(1, p):
            for i in range(1, p):
                assert abs(r[j * n + i]) <= 1e-13 * np.abs(Ak).max()


def test_mapped_lor_of_rectangle_is_q1_box():
    g = np.array([[0.0, 0.0], [0.3, 0.0], [0.0, 0.7], [0.3, 0.7]])
    from oracle import lor
    assert np.abs(geometry.q1_quad_stiffness(g) - lor.q1_cell_stiffness(0.3, 0.7)).max() <= 1e-15


@pytest.mark.parametrize("corners", [inputs.PARALLELOGRAM, inputs.QUADRILATERAL])
def test_areas_and_load_vector_of_one(corners):
    mesh = _mesh(6, pmax=3)
    md = inputs.with_corners(mesh, corners)
    prob = solver.build_problem(md)
    tot = sum(prob.space.area(k) for k in range(prob.topo.n))
    assert abs(tot - _shoelace(corners)) <= 1e-14
    b = rhs.load_vector_fn(prob.space, lambda x: np.ones(len(x)))
    assert abs(b.sum() - _shoelace(corners)) <= 1e-13


def test_bilinear_map_spd():
    mesh = _mesh(7, pmax=3)
    md = inputs.with_corners(mesh, inputs.QUADRILATERAL)
    A = solver.build_problem(md).A.toarray()
    assert np.abs(A - A.T).max() <= 1e-12 * np.abs(A).max()
    assert np.linalg.eigvalsh(A).min() > 0.0


def test_non_convex_corners_rejected():
    mesh = _mesh(1)
    bad = ((0.0, 0.0), (1.0, 0.0), (0.0, 1.0), (0.2, 0.2))
    with pytest.raises(ValueError):
        solver.build_problem(inputs.with_corners(mesh, bad))


# ---------------------------------------------------------------- curved maps
def test_wavy_map_jacobian_and_area():
    F = inputs.WavyMap()
    rng = np.random.default_rng(1)
    P = rng.uniform(0, 1, size=(6, 2))
    e = 1e-6
    for j in range(2):
        d = np.zeros(2)
        d[j] = e
        assert np.allclose(F.jacobian(P)[:, :, j], (F(P + d) - F(P - d)) / (2 * e), atol=1e-8)
    # element areas (each by its own p+2 rule) sum to the domain's area, here
    # by a 40-point tensor rule over the whole domain
    mesh = _mesh(6, pmax=3)
    prob = solver.build_problem(inputs.with_mapping(mesh, F))
    from oracle import basis
    x, w = basis.gauss(40)
    X = np.stack(np.meshgrid(x, x), axis=-1).reshape(-1, 2)
    ref = np.outer(w, w).ravel() @ np.linalg.det(F.jacobian(X))
    assert abs(sum(prob.space.area(k) for k in range(prob.topo.n)) - ref) <= 1e-8


def test_bilinear_map_as_a_generic_map_matches_corners():
    mesh = _mesh(3, pmax=5)
    c = np.array(inputs.QUADRILATERAL)
    L = mesh.extent[0] * mesh.lattice_h
    pa = solver.build_problem(inputs.with_corners(mesh, c))
    pb = solver.build_problem(inputs.with_mapping(mesh, geometry.BilinearMap(c, L, L)))
    assert abs(pa.A - pb.A).max() <= 1e-13 * abs(pa.A).max()


def _wavy_manufactured():
    """U(X, Y) = sin(pi X) sin(pi Y) in the pre-image, zero on the boundary of
    the curved domain; f = -Laplace_x(u) pulled back to X by the chain rule,
    -(1/det J) div_X(det J J^-1 J^-T grad_X U), differentiated symbolically."""
    sympy = pytest.importorskip("sympy")
    F = inputs.WavyMap()
    X, Y = sympy.symbols("X Y")
    L, ax, ay = F.L, F.ax, F.ay
    J = sympy.Matrix([[1, ax * sympy.pi * sympy.cos(sympy.pi * Y / L)],
                      [ay * sympy.pi * sympy.cos(sympy.pi * X / L), 1]])
    det = J.det()
    Ji = J.inv()
    K = sympy.simplify(det * Ji * Ji.T)
    U = sympy.sin(sympy.pi * X) * sympy.sin(sympy.pi * Y)
    g = sympy.Matrix([sympy.diff(U, X), sympy.diff(U, Y)])
    flux = K * g
    lap = (sympy.diff(flux[0], X) + sympy.diff(flux[1], Y)) / det
    f = sympy.lambdify((X, Y), -lap, "numpy")
    u = sympy.lambdify((X, Y), U, "numpy")
    return F, (lambda P: f(P[:, 0], P[:, 1])), (lambda P: u(P[:, 0], P[:, 1]))


@pytest.mark.parametrize("p", [2, 3])
def test_curved_map_converges_at_the_optimal_rate(p):
    """Nodal error of the SIPG solution on the curved domain under uniform
    refinement falls like h^(p+1) (a wrong metric term, normal or weight
    breaks this)."""
    F, fX, uX = _wavy_manufactured()
    errs = []
    for base in (2, 4, 8):
        mesh = inputs.with_mapping(inputs.uniform_mesh(2, base, p), F)
        prob = solver.build_problem(mesh)
        sp_ = prob.space
        b = np.zeros(sp_.n)
        for k in range(prob.topo.n):
            pts, W = sp_.volume_quadrature(k, p + 3)
            v, _ = sp_.eval(k, pts)
            b[sp_.dofs(k)] = v.T @ (W * fX(pts))
        x = np.linalg.solve(prob.A.toarray(), b)
        from oracle.dg import DGSpace
        Xn = np.concatenate([DGSpace.node_coords(sp_, k) for k in range(prob.topo.n)])
        errs.append(np.abs(x - uX(Xn)).max())
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert errs[-1] < 1e-3
    assert rates[-1] > p + 1 - 0.6, (errs, rates)


# ---------------------------------------------------------------- BR2 on mapped elements
def test_br2_similarity_map_leaves_matrix_unchanged():
    mesh = _mesh(2, pmax=5)
    th, s, sh = -1.1, 0.7, np.array([0.3, 0.9])
    R = s * np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    L = mesh.extent[0] * mesh.lattice_h
    corners = [sh, sh + R @ [L, 0], sh + R @ [0, L], sh + R @ [L, L]]
    pa = solver.build_problem(mesh, form="br2")
    pb = solver.build_problem(inputs.with_corners(mesh, corners), form="br2")
    assert abs(pa.A - pb.A).max() <= 1e-12 * abs(pa.A).max()


def test_br2_affine_map_reproduces_manufactured_solution():
    mesh = _mesh(3, pmin=2, pmax=4)
    c = np.array(inputs.PARALLELOGRAM)
    L = mesh.extent[0] * mesh.lattice_h
    A = np.stack([(c[1] - c[0]) / L, (c[2] - c[0]) / L], axis=1)
    Ai = np.linalg.inv(A)
    Gm = Ai @ Ai.T

    def pre(x):
        return (x - c[0]) @ Ai.T

    def u(x):
        X = pre(x)
        return X[:, 0] * (L - X[:, 0]) * X[:, 1] * (L - X[:, 1])

    def f(x):
        X, Y = pre(x).T
        return -(Gm[0, 0] * -2.0 * Y * (L - Y) + 2 * Gm[0, 1] * (L - 2 * X) * (L - 2 * Y)
                 + Gm[1, 1] * -2.0 * X * (L - X))

    prob = solver.build_problem(inputs.with_corners(mesh, c), form="br2")
    b = rhs.load_vector_fn(prob.space, f, extra=3)
    x = np.linalg.solve(prob.A.toarray(), b)
    ui = rhs.interpolate(prob.space, u)
    assert np.abs(x - ui).max() <= 1e-10 * np.abs(ui).max()


def test_br2_bilinear_harmonic_patch_and_spd():
    mesh = _mesh(4, pmin=2, pmax=5, base=4)
    prob = solver.build_problem(inputs.with_corners(mesh, inputs.QUADRILATERAL), form="br2")
    ui = rhs.interpolate(prob.space, lambda x: x[:, 0] * x[:, 1])
    r = prob.A @ ui
    scale = np.abs(prob.A).max() * np.abs(ui).max()
    for k in _interior_elements(prob.topo):
        assert np.abs(r[prob.space.dofs(k)]).max() <= 1e-12 * scale
    A = prob.A.toarray()
    assert np.abs(A - A.T).max() <= 1e-12 * np.abs(A).max()
    assert np.linalg.eigvalsh(A).min() > 0.0


@pytest.mark.parametrize("p", [2])
def test_br2_curved_map_converges(p):
    F, fX, uX = _wavy_manufactured()
    errs = []
    for base in (2, 4, 8):
        prob = solver.build_problem(inputs.with_mapping(inputs.uniform_mesh(2, base, p), F), form="br2")
        sp_ = prob.space
        b = np.zeros(sp_.n)
        for k in range(prob.topo.n):
            pts, W = sp_.volume_quadrature(k, p + 3)
            v, _ = sp_.eval(k, pts)
            b[sp_.dofs(k)] = v.T @ (W * fX(pts))
        x = np.linalg.solve(prob.A.toarray(), b)
        from oracle.dg import DGSpace
        Xn = np.concatenate([DGSpace.node_coords(sp_, k) for k in range(prob.topo.n)])
        errs.append(np.abs(x - uX(Xn)).max())
    rate = np.log2(errs[1] / errs[2])
    assert rate > p + 1 - 0.6, (errs, rate)


def test_br2_lifting_energy_uses_the_mapped_mass():
    """On one mapped element, the BR2 lifting energy of the boundary jump of u
    is eta * b^T M^-1 b with M the element's physical mass matrix: checked
    against the same quantity from an independently assembled mass matrix
    (a 12-point rule; exact for the bilinear map)."""
    mesh = inputs.uniform_mesh(2, 1, 3)
    md = inputs.with_corners(mesh, inputs.QUADRILATERAL)
    prob = solver.build_problem(md, form="br2", eta=1.0)
    sp_ = prob.space
    from oracle import basis
    from oracle.dg import DGSpace
    pts, W = DGSpace.volume_quadrature(sp_, 0, 12)
    W = W * np.linalg.det(sp_.map.jacobian(pts))
    v, _ = sp_.eval(0, pts)
    M = v.T @ (W[:, None] * v)
    Minv = np.linalg.inv(M)
    # A with eta = 1 minus A with eta = 0 is the lifting energy alone
    A0 = solver.build_problem(md, form="br2", eta=0.0).A.toarray()
    E = prob.A.toarray() - A0
    Bf = np.zeros((sp_.n, sp_.n))
    for f in prob.topo.subfaces:
        q = int(prob.topo.p[0]) + 2
        fp, fw, _ = sp_.face_quadrature(f, q)
        vf, _ = sp_.eval(0, fp)
        bb = (vf.T * fw) @ vf
        Bf += bb.T @ Minv @ bb
    assert np.abs(E - Bf).max() <= 1e-10 * np.abs(Bf).max()


def _phys_manufactured():
    """u = sin(2x) e^y + x^2 - y in physical coordinates, -Laplace(u) =
    3 sin(2x) e^y - 2: nonzero on the boundary of any of the domains."""
    u = lambda P: np.sin(2 * P[:, 0]) * np.exp(P[:, 1]) + P[:, 0] ** 2 - P[:, 1]
    f = lambda P: 3 * np.sin(2 * P[:, 0]) * np.exp(P[:, 1]) - 2.0
    return u, f


@pytest.mark.parametrize("p", [2, 3])
@pytest.mark.parametrize("geom", ["wavy", "quad"])
def test_weak_dirichlet_data_on_mapped_domains_converges(p, geom):
    """Weak Dirichlet data on a curved and on a bilinear domain (the oracle's
    dirichlet_load on mapped elements: boundary points, arc length and the
    physical normal in both boundary terms): the nodal error of a
    manufactured solution with nonzero boundary values falls like h^(p+1).
    Dropping either boundary term or flipping the normal breaks it."""
    u, f = _phys_manufactured()
    errs = []
    for base in (2, 4, 8):
        mesh = inputs.uniform_mesh(2, base, p)
        mesh = (inputs.with_mapping(mesh, inputs.WavyMap()) if geom == "wavy"
                else inputs.with_corners(mesh, inputs.QUADRILATERAL))
        prob = solver.build_problem(mesh)
        sp_ = prob.space
        b = rhs.dirichlet_load(sp_, f, u, 100.0)
        x = np.linalg.solve(prob.A.toarray(), b)
        Xn = np.concatenate([sp_.node_coords(k) for k in range(prob.topo.n)])   # physical
        errs.append(np.abs(x - u(Xn)).max())
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert errs[-1] < 1e-3 * np.abs(u(Xn)).max()
    assert rates[-1] > p + 1 - 0.6, (errs, rates)
