"""Pins of the oracle's piecewise-constant coefficient a (the random-refinement
problem -div(a grad u) = f of Section 4.3) against linearity, an interface
solution with continuous flux, closed-form penalty energies and the LOR
spectral bounds (Section 3.4)."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import rhs, solver
from oracle.lor import lor_conforming
from paper_2009_01287_gb300 import inputs


def _mesh(lo, size, p, extent, lh, coeff=None):
    return inputs.MeshDesc(len(extent), np.asarray(lo, dtype=np.int32), np.asarray(size, dtype=np.int32),
                           np.asarray(p, dtype=np.int32), tuple(extent), lh,
                           None if coeff is None else np.asarray(coeff, dtype=np.float64))


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("form", ["sipg", "br2"])
def test_constant_coefficient_scales_the_operator(dim, form):
    """a = c everywhere: every term of the form is linear in a, so A(c) = c A(1)."""
    mesh = inputs.small_hp_mesh(1, base=2, depth=2, prob=0.4, pmin=1, pmax=3, dim=dim)
    _, _, A1 = solver.build_operator(mesh, form=form)
    _, _, Ac = solver.build_operator(inputs.with_coeff(mesh, np.full(mesh.n_elems, 7.5)), form=form)
    assert abs(Ac - 7.5 * A1).max() <= 1e-13 * abs(Ac).max()


# Interface solution: a = 1 for x < 1/2 and 20 for x > 1/2 (base-cell parity on a
# 2-wide base grid).  u = g(x) w(y[, z]) with w = y(1-y)[z(1-z)], g continuous at
# 1/2 with a g' continuous there (both equal 1) and g(0) = g(1) = 0:
#   g = x (2 - x) on the left, (1 - x)(3.05 - 3.1 (1 - x)) on the right.
A_L, A_R = 1.0, 20.0


def _g(x):
    return np.where(x < 0.5, x * (2 - x), (1 - x) * (3.05 - 3.1 * (1 - x)))


def _g2(x):   # g''
    return np.where(x < 0.5, -2.0, -6.2)


def _interface_u(X):
    return _g(X[:, 0]) * np.prod(X[:, 1:] * (1 - X[:, 1:]), axis=1)


def _interface_f(X):
    a = np.where(X[:, 0] < 0.5, A_L, A_R)
    x, t = X[:, 0], X[:, 1:]
    w = np.prod(t * (1 - t), axis=1)
    lap = _g2(x) * w
    for d in range(t.shape[1]):   # -2 times the product of the other factors
        lap = lap + _g(x) * (-2.0) * np.prod(np.delete(t * (1 - t), d, axis=1), axis=1)
    return -a * lap


def test_interface_solution_has_continuous_flux():
    # the construction itself: both branches and their derivatives at x = 1/2
    gl = lambda x: x * (2 - x)
    gr = lambda x: (1 - x) * (3.05 - 3.1 * (1 - x))
    dgl = lambda x: 2 - 2 * x
    dgr = lambda x: -3.05 + 6.2 * (1 - x)
    assert abs(gl(0.5) - gr(0.5)) < 1e-15
    assert abs(A_L * dgl(0.5) - 1.0) < 1e-14 and abs(A_R * dgr(0.5) - 1.0) < 1e-13
    assert gl(0.0) == 0.0 and gr(1.0) == 0.0
    x = np.array([0.2, 0.7])
    assert np.allclose(_g(x), [gl(0.2), gr(0.7)])


@pytest.mark.parametrize("dim,pmin,pmax", [(2, 2, 5), (3, 2, 3)])
@pytest.mark.parametrize("form", ["sipg", "br2"])
@pytest.mark.parametrize("seed", [0, 1])
def test_interface_solution_reproduced(dim, pmin, pmax, form, seed):
    """u is piecewise Q2 on every element (the interface x = 1/2 is a base-cell
    boundary) with a grad u . n continuous, so the weighted averages make both
    forms consistent: A u_I = (f, phi) exactly on hanging, variable-p meshes.
    Unweighted averages {grad u} would leave a residual on the interface."""
    mesh = inputs.small_hp_mesh(seed, base=2, depth=2, prob=0.5, pmin=pmin, pmax=pmax, dim=dim)
    mesh = inputs.with_coeff(mesh, inputs.base_parity_coeff(mesh, 2, (A_L, A_R)))
    prob = solver.build_problem(mesh, form=form)
    u = rhs.interpolate(prob.space, _interface_u)
    b = rhs.load_vector_fn(prob.space, _interface_f)
    assert np.abs(prob.A @ u - b).max() < 1e-9 * np.abs(b).max()


def test_interface_solution_needs_the_weighted_average():
    """Planted mistake: the same solution with the coefficient left out of the
    face averages (a = 1 in the form, a in f only) is not reproduced."""
    mesh = inputs.small_hp_mesh(0, base=2, depth=2, prob=0.5, pmin=2, pmax=4)
    prob = solver.build_problem(mesh)
    u = rhs.interpolate(prob.space, _interface_u)
    b = rhs.load_vector_fn(prob.space, _interface_f)
    assert np.abs(prob.A @ u - b).max() > 1e-2 * np.abs(b).max()


def test_sipg_penalty_closed_form_with_coefficient():
    """u = 1 on the left square of a 2x1 mesh: a(u,u) = sum over faces of
    sigma |[[u]]|^2 |e|, sigma carrying the larger a of the two sides."""
    h = 0.5
    for (pl, pr), (al, ar) in [((1, 1), (1.0, 20.0)), ((2, 3), (20.0, 1.0)), ((4, 2), (3.0, 0.5))]:
        mesh = _mesh([(0, 0), (1, 0)], [1, 1], [pl, pr], (2, 1), h, [al, ar])
        prob = solver.build_problem(mesh, form="sipg", eta=7.0)
        u = np.zeros(prob.space.n)
        u[:(pl + 1) ** 2] = 1.0
        expect = max(al, ar) * 7.0 * max(pl, pr) ** 2 + 3 * al * 7.0 * pl ** 2
        assert abs(u @ prob.A @ u - expect) < 1e-12 * expect


def test_br2_penalty_closed_form_with_coefficient():
    """Same jump with BR2: each side's lifting energy (p+1)^2 (1/4 on the
    interior face, 1 on the boundary) carries the larger a of the sub-face's
    two sides (the boundary faces: the element's own a)."""
    for (pl, pr), (al, ar) in [((1, 1), (1.0, 20.0)), ((2, 3), (20.0, 1.0)), ((5, 2), (3.0, 0.5))]:
        mesh = _mesh([(0, 0), (1, 0)], [1, 1], [pl, pr], (2, 1), 0.25, [al, ar])
        prob = solver.build_problem(mesh, form="br2", eta=3.0)
        u = np.zeros(prob.space.n)
        u[:(pl + 1) ** 2] = 1.0
        expect = 3.0 * (0.25 * max(al, ar) * ((pl + 1) ** 2 + (pr + 1) ** 2) + 3 * al * (pl + 1) ** 2)
        assert abs(u @ prob.A @ u - expect) < 1e-11 * expect


@pytest.mark.parametrize("form", ["sipg", "br2"])
def test_spd_with_coefficient(form):
    mesh = inputs.small_hp_mesh(3, base=2, depth=2, prob=0.5, pmin=1, pmax=4)
    mesh = inputs.with_coeff(mesh, inputs.base_parity_coeff(mesh, 2))
    A = solver.build_problem(mesh, form=form).A.toarray()
    assert np.abs(A - A.T).max() < 1e-12 * np.abs(A).max()
    assert np.linalg.eigvalsh(A).min() > 0


def _lor_extremes(mesh):
    prob = solver.build_problem(mesh, form="sipg")
    P = prob.cs.P
    Kc = (P.T @ prob.A @ P).toarray()
    Ac = lor_conforming(prob.space, P).toarray()
    ev = sla.eigh(Kc, Ac, eigvals_only=True)
    return ev.min(), ev.max()


def test_lor_equivalence_is_independent_of_the_contrast():
    """Section 3.4: with a_k on each LOR element block, the conforming
    operator and its LOR matrix stay spectrally equivalent with the bounds of
    a = 1, whatever the contrast (both scale by a_k element by element).  An
    unweighted LOR matrix would move the upper bound by the contrast, 20."""
    mesh = inputs.small_hp_mesh(2, base=2, depth=1, prob=0.5, pmin=2, pmax=4)
    lo1, hi1 = _lor_extremes(mesh)
    lo20, hi20 = _lor_extremes(inputs.with_coeff(mesh, inputs.base_parity_coeff(mesh, 2)))
    assert lo20 > 0.5 * lo1 and hi20 < 2.0 * hi1


@pytest.mark.parametrize("form", ["sipg", "br2"])
def test_condition_number_robust_in_the_contrast(form):
    """kappa(BA) with the exact LOR solve on a small hp mesh stays within a
    factor 1.5 of its a = 1 value for contrasts 20 and 1000 (SIPG penalty and
    BR2 lifting energies both with the larger a of the two sides; BR2 with
    each side's own a grows from 25 to about 1560 at contrast 1000)."""
    mesh = inputs.small_hp_mesh(2, base=4, depth=2, prob=0.4, pmin=1, pmax=4)
    kap = []
    for c in (1.0, 20.0, 1000.0):
        m = inputs.with_coeff(mesh, inputs.base_parity_coeff(mesh, 4, (1.0, c)))
        prob = solver.build_problem(m, form=form)
        B = solver.Preconditioner(prob, lor="exact").matrix()
        ev = np.real(np.linalg.eigvals(B @ prob.A.toarray()))
        kap.append(ev.max() / ev.min())
    assert max(kap) < 1.5 * kap[0] and min(kap) > kap[0] / 1.5


def test_sipg_penalty_closed_form_hanging_cubes_with_coefficient():
    """One coarse cube next to four fine ones, piecewise-constant u and a: a(u,u)
    = sum over sub-faces of sigma |F| [[u]]^2, sigma carrying the larger a."""
    lh, eta = 0.25, 3.0
    lo = [(0, 0, 0)] + [(2, j, k) for k in (0, 1) for j in (0, 1)]
    size = [2, 1, 1, 1, 1]
    p = [2, 1, 3, 2, 1]
    a = [20.0, 1.0, 3.0, 1.0, 50.0]
    mesh = _mesh(lo, size, p, (3, 2, 2), lh, a)
    topo, space, A = solver.build_operator(mesh, form="sipg", eta=eta)
    c = np.array([1.0, -2.0, 0.5, 3.0, 0.0])
    u = np.concatenate([np.full((pk + 1) ** 3, ck) for pk, ck in zip(p, c)])
    expect = 0.0
    for f in topo.subfaces:
        area = (f.hi[0] - f.lo[0]) * (f.hi[1] - f.lo[1]) * lh * lh
        if f.kp >= 0:
            s = max(a[f.km], a[f.kp]) * eta * max(p[f.km], p[f.kp]) ** 2 / (lh * min(size[f.km], size[f.kp]))
            expect += s * area * (c[f.km] - c[f.kp]) ** 2
        else:
            s = a[f.km] * eta * p[f.km] ** 2 / (lh * size[f.km])
            expect += s * area * c[f.km] ** 2
    assert abs(u @ A @ u - expect) < 1e-12 * expect


def test_br2_penalty_closed_form_cubes_with_coefficient():
    """Conforming 2x1x1 cubes, u = 1 on the left one: each side's lifting energy
    (p+1)^2 h (1/4 per side on the interior face, all of it on the five
    boundary faces) carries the larger a of the sub-face."""
    h, eta = 0.5, 2.0
    for (pl, pr), (al, ar) in [((1, 1), (1.0, 20.0)), ((2, 3), (20.0, 1.0)), ((3, 1), (0.5, 4.0))]:
        mesh = _mesh([(0, 0, 0), (1, 0, 0)], [1, 1], [pl, pr], (2, 1, 1), h, [al, ar])
        _, space, A = solver.build_operator(mesh, form="br2", eta=eta)
        u = np.zeros(space.n)
        u[:(pl + 1) ** 3] = 1.0
        expect = eta * (0.25 * max(al, ar) * ((pl + 1) ** 2 * h + (pr + 1) ** 2 * h) + 5 * al * (pl + 1) ** 2 * h)
        assert abs(u @ A @ u - expect) < 1e-11 * expect
