"""Pins of two oracle helpers that the GPU parity tests lean on:

- dg.element_rows (A x restricted to one element, used to check sampled
  outputs of meshes too large to assemble) against the rows of the assembled
  matrix dg.assemble, for every element of hanging hp meshes, 2D and 3D, SIPG
  and BR2, with and without a coefficient (Section 2, Eq. fe-problem; BR2 of
  Section 4.4; coefficient of Section 4.3);
- rhs.load_vector (b_i = int f phi_i for the sine right-hand side) against
  closed-form integrals of a polynomial times a sine.
"""
import math

import numpy as np
import pytest

from oracle import dg, rhs, solver
from paper_2009_01287_gb300 import inputs


@pytest.mark.parametrize("dim,form,coef", [(2, "sipg", False), (2, "br2", False), (2, "sipg", True),
                                           (2, "br2", True), (3, "sipg", False), (3, "br2", True)])
def test_element_rows_equal_assembled_rows(dim, form, coef):
    if dim == 2:
        mesh = inputs.small_hp_mesh(5, base=3, depth=3, prob=0.45, pmin=1, pmax=5)
    else:
        mesh = inputs.small_hp_mesh(2, base=2, depth=2, prob=0.4, pmin=1, pmax=3, dim=3)
    if coef:
        mesh = inputs.with_coeff(mesh, inputs.base_parity_coeff(mesh, 3 if dim == 2 else 2))
    topo, space, A = solver.build_operator(mesh, form=form)
    eta = dg.br2_eta(topo) if form == "br2" else 100.0
    x = inputs.random_vector(space.n, 11)
    y = A @ x
    scale = np.abs(y).max()
    for k in range(topo.n):
        yk = dg.element_rows(space, k, x, eta, form=form)
        assert np.abs(yk - y[space.dofs(k)]).max() <= 1e-12 * scale, k


@pytest.mark.parametrize("geom", ["quad", "wavy", "lshape"])
@pytest.mark.parametrize("form", ["sipg", "br2"])
def test_element_rows_equal_assembled_rows_mapped(geom, form):
    """The same on mapped, curved and L-shaped meshes (the full-size GPU tests
    of those check sampled elements against element_rows)."""
    mesh = inputs.small_hp_mesh(6, base=4, depth=2, prob=0.45, pmin=1, pmax=5)
    mesh = {"quad": lambda: inputs.with_corners(mesh, inputs.QUADRILATERAL),
            "wavy": lambda: inputs.with_mapping(mesh, inputs.WavyMap()),
            "lshape": lambda: inputs.lshape(mesh)}[geom]()
    topo, space, A = solver.build_operator(mesh, form=form)
    eta = dg.br2_eta(topo) if form == "br2" else 100.0
    x = inputs.random_vector(space.n, 12)
    y = A @ x
    scale = np.abs(y).max()
    for k in range(topo.n):
        yk = dg.element_rows(space, k, x, eta, form=form)
        assert np.abs(yk - y[space.dofs(k)]).max() <= 1e-12 * scale, k


# ---------------------------------------------------------------- load vector

# Gauss-Lobatto points on [0,1] in closed form (the golden file
# tests/golden/gll_closed_forms.txt lists the same values)
GLL = {1: [0.0, 1.0], 2: [0.0, 0.5, 1.0],
       3: [0.0, 0.5 - math.sqrt(5.0) / 10.0, 0.5 + math.sqrt(5.0) / 10.0, 1.0]}


def _lagrange_coeffs(nodes):
    """Monomial coefficients (ascending) of the Lagrange polynomials."""
    out = []
    for i, ti in enumerate(nodes):
        c = np.array([1.0])
        for j, tj in enumerate(nodes):
            if j != i:
                c = np.convolve(c, np.array([-tj, 1.0])) / (ti - tj)
        out.append(c)
    return out


def _moments(beta, mmax, terms=40):
    """J_m = int_0^1 t^m exp(i beta t) dt, m = 0..mmax, from the termwise
    integrated exponential series sum_k (i beta)^k / (k! (m + k + 1))."""
    J = np.zeros(mmax + 1, dtype=complex)
    for m in range(mmax + 1):
        s, term = 0.0 + 0.0j, 1.0 + 0.0j
        for k in range(terms):
            s += term / (m + k + 1)
            term *= 1j * beta / (k + 1)
        J[m] = s
    return J


def _int_1d(p, lo, h, omega):
    """int_lo^{lo+h} l_i((x - lo)/h) sin(omega x) dx for every node i."""
    J = _moments(omega * h, p)
    ph = complex(math.cos(omega * lo), math.sin(omega * lo))
    return np.array([h * (ph * np.dot(c, J[:len(c)])).imag for c in _lagrange_coeffs(GLL[p])])


def _gauss_error_1d(p, h, omega):
    """Bound on the error of the n = p+3 point Gauss rule for
    int_0^1 h l_i(t) sin(omega h t + c) dt:  h K_n max|g^(2n)| with
    K_n = (n!)^4 / ((2n+1) ((2n)!)^3) and, by Leibniz' rule,
    |g^(2n)| <= sum_j C(2n, j) max|l_i^(j)| beta^(2n-j), beta = omega h."""
    n = p + 3
    K = math.factorial(n) ** 4 / ((2 * n + 1) * math.factorial(2 * n) ** 3)
    beta = omega * h
    bound = 0.0
    for j in range(p + 1):
        # max over [0,1] of |l_i^(j)| <= sum of |coefficients| of the derivative
        Lj = max(np.abs(np.polynomial.polynomial.polyder(c, j)).sum() if j else np.abs(c).sum()
                 for c in _lagrange_coeffs(GLL[p]))
        bound += math.comb(2 * n, j) * Lj * beta ** (2 * n - j)
    return h * K * bound


def _closed_form_load(mesh, amps, waves):
    """Closed-form b and, per entry, the bound on the Gauss rule's error: for
    each separable mode the tensor rule returns the product of the 1D rules,
    so |Q - I| <= prod(|I_d| + E_d) - prod |I_d|."""
    lh = mesh.lattice_h
    b, tol = [], []
    for k in range(mesh.n_elems):
        p = int(mesh.p[k])
        h = float(mesh.size[k]) * lh
        bk = np.zeros((p + 1) ** mesh.dim)
        tk = np.zeros_like(bk)
        for a, wv in zip(amps, waves):
            om = [math.pi * float(wv[d]) for d in range(mesh.dim)]
            f1 = [_int_1d(p, float(mesh.lo[k, d]) * lh, h, om[d]) for d in range(mesh.dim)]
            e1 = [_gauss_error_1d(p, h, om[d]) for d in range(mesh.dim)]
            if mesh.dim == 2:   # local index iy (p+1) + ix
                prod = np.outer(f1[1], f1[0]).ravel()
                up = np.outer(np.abs(f1[1]) + e1[1], np.abs(f1[0]) + e1[0]).ravel()
            else:               # iz (p+1)^2 + iy (p+1) + ix
                prod = np.einsum("z,y,x->zyx", f1[2], f1[1], f1[0]).ravel()
                up = np.einsum("z,y,x->zyx", np.abs(f1[2]) + e1[2], np.abs(f1[1]) + e1[1],
                               np.abs(f1[0]) + e1[0]).ravel()
            bk += a * prod
            tk += abs(a) * (up - np.abs(prod))
        b.append(bk)
        tol.append(tk)
    return np.concatenate(b), np.concatenate(tol)


def _check(got, want, tol):
    # the quadrature's bound plus rounding of the summed products
    assert np.all(np.abs(got - want) <= tol + 1e-14 * np.abs(want).max())


@pytest.mark.parametrize("p", [1, 2, 3])
def test_load_vector_closed_form_2d(p):
    mesh = inputs.random_refined_mesh(2, 16, 1, 0.4, p, p, seed=3)
    amps = np.array([0.7, -1.3])
    waves = np.array([[1, 2], [2, 1]], dtype=np.int32)
    _, space, _ = solver.build_operator(mesh)
    got = rhs.load_vector(space, amps, waves)
    want, tol = _closed_form_load(mesh, amps, waves)
    assert tol.max() < 1e-9 * np.abs(want).max()     # the bound is tight enough to pin
    _check(got, want, tol)


def test_load_vector_closed_form_p1_single_element():
    # one p = 1 square [1/4, 1/2] x [1/2, 3/4] inside a 4x4 grid, f = sin(pi x) sin(2 pi y):
    # the four entries are products of 1D integrals of (1 - t) and t against a sine
    mesh = inputs.uniform_mesh(2, 4, 1)
    _, space, _ = solver.build_operator(mesh)
    b = rhs.load_vector(space, np.array([1.0]), np.array([[1, 2]], dtype=np.int32))
    k = 2 * 4 + 1
    x0, y0, h = 0.25, 0.5, 0.25

    def ints(w, c):
        # int_c^{c+h} (c + h - x)/h sin(w x) dx and int_c^{c+h} (x - c)/h sin(w x) dx
        e = c + h
        left = (h * math.cos(w * c) / w + (math.sin(w * c) - math.sin(w * e)) / w ** 2) / h
        right = (-h * math.cos(w * e) / w + (math.sin(w * e) - math.sin(w * c)) / w ** 2) / h
        return np.array([left, right])

    ix, iy = ints(math.pi, x0), ints(2 * math.pi, y0)
    want = np.outer(iy, ix).ravel()
    ex, ey = _gauss_error_1d(1, h, math.pi), _gauss_error_1d(1, h, 2 * math.pi)
    tol = np.outer(np.abs(iy) + ey, np.abs(ix) + ex).ravel() - np.abs(want)
    _check(b[space.dofs(k)], want, tol)


@pytest.mark.parametrize("p", [1, 2])
def test_load_vector_closed_form_3d(p):
    mesh = inputs.random_refined_mesh(3, 8, 1, 0.3, p, p, seed=4)
    amps = np.array([1.1])
    waves = np.array([[1, 2, 1]], dtype=np.int32)
    _, space, _ = solver.build_operator(mesh)
    got = rhs.load_vector(space, amps, waves)
    want, tol = _closed_form_load(mesh, amps, waves)
    assert tol.max() < 1e-7 * np.abs(want).max()
    _check(got, want, tol)


def test_dirichlet_load_reproduces_polynomial_with_boundary_data():
    """Weakly imposed inhomogeneous Dirichlet data (SIPG): a polynomial in the
    DG space with nonzero boundary values, f = -Laplace(u), g = u on the
    boundary, is reproduced exactly (consistency), on a hanging hp mesh, with
    and without a map of the domain."""
    from oracle import rhs as R
    mesh = inputs.small_hp_mesh(3, base=3, depth=2, prob=0.5, pmin=2, pmax=4)
    # total degree 2: in Q_2 of every element, boxes or affine images of boxes
    u = lambda x: 1.0 + x[:, 0] - 0.5 * x[:, 1] + x[:, 0] * x[:, 1] + 0.3 * x[:, 0] ** 2
    f = lambda x: np.full(len(x), -0.6)
    for md in (mesh, inputs.with_corners(mesh, inputs.PARALLELOGRAM)):
        prob = solver.build_problem(md)
        b = R.dirichlet_load(prob.space, f, u, 100.0)
        x = np.linalg.solve(prob.A.toarray(), b)
        ui = R.interpolate(prob.space, u)
        assert np.abs(x - ui).max() <= 1e-10 * np.abs(ui).max()
    # with g = 0 the boundary terms vanish
    prob = solver.build_problem(mesh)
    b0 = R.dirichlet_load(prob.space, f, lambda x: np.zeros(len(x)), 100.0)
    assert np.abs(b0 - R.load_vector_fn(prob.space, f)).max() == 0.0
