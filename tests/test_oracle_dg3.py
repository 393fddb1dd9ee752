"""Pins of the oracle's DG matrix on cubes (Section 2 read for hexahedra;
BR2 of Section 4.4): sub-face cover, consistency, closed-form penalty
energies and a textbook continuous assembly."""
import itertools

import numpy as np
import pytest

from oracle import basis, rhs, solver
from oracle.topology3 import Topology3
from paper_2009_01287_gb300 import inputs


def _mesh(lo, size, p, extent, lh):
    return inputs.MeshDesc(3, np.asarray(lo, dtype=np.int32).reshape(-1, 3),
                           np.asarray(size, dtype=np.int32), np.asarray(p, dtype=np.int32),
                           tuple(extent), lh)


U = lambda X: np.prod(X * (1 - X), axis=1)


def F(X):   # -Laplace(U)
    q = X * (1 - X)
    return 2 * (q[:, 1] * q[:, 2] + q[:, 0] * q[:, 2] + q[:, 0] * q[:, 1])


def _brute_subfaces(mesh):
    """Pairwise rectangle intersections, O(n^2): an independent count."""
    lo, h, ext = mesh.lo.astype(int), mesh.size.astype(int), mesh.extent
    out = set()
    for a in range(mesh.n_elems):
        for ax in range(3):
            t = [d for d in range(3) if d != ax]
            up = lo[a, ax] + h[a]
            if up == ext[ax]:
                out.add((a, -1, ax, up, tuple(lo[a, t]), tuple(lo[a, t] + h[a])))
            if lo[a, ax] == 0:
                out.add((a, -1, ax, 0, tuple(lo[a, t]), tuple(lo[a, t] + h[a])))
            for b in range(mesh.n_elems):
                if lo[b, ax] != up:
                    continue
                l0 = np.maximum(lo[a, t], lo[b, t])
                h0 = np.minimum(lo[a, t] + h[a], lo[b, t] + h[b])
                if np.all(h0 > l0):
                    out.add((a, b, ax, up, tuple(l0), tuple(h0)))
    return out


@pytest.mark.parametrize("seed", [0, 1])
def test_subfaces_match_brute_force_and_cover_faces(seed):
    mesh = inputs.small_hp_mesh(seed, base=2, depth=2, prob=0.5, pmin=1, pmax=3, dim=3)
    topo = Topology3(mesh.lo, mesh.size, mesh.p, mesh.extent)
    got = {(f.km, f.kp, f.axis, f.c, f.lo, f.hi) for f in topo.subfaces}
    assert len(got) == len(topo.subfaces)
    assert got == _brute_subfaces(mesh)
    area = np.zeros(topo.n)
    for f in topo.subfaces:
        a = (f.hi[0] - f.lo[0]) * (f.hi[1] - f.lo[1])
        area[f.km] += a
        if f.kp >= 0:
            area[f.kp] += a
    assert np.array_equal(area, 6 * topo.size.astype(float) ** 2)


@pytest.mark.parametrize("form", ["sipg", "br2"])
@pytest.mark.parametrize("seed", [0, 1])
def test_manufactured_q2_reproduced(form, seed):
    """A Q2 solution vanishing on the boundary lies in V_h (p >= 2); both forms
    are consistent, so A u_I = (f, phi) on hanging, variable-p cube meshes."""
    mesh = inputs.small_hp_mesh(seed, base=2, depth=2, prob=0.5, pmin=2, pmax=3, dim=3)
    _, space, A = solver.build_operator(mesh, form=form)
    u = rhs.interpolate(space, U)
    b = rhs.load_vector_fn(space, F)
    assert np.abs(A @ u - b).max() < 1e-10 * np.abs(b).max()


def test_planted_sign_mistake_fails_consistency():
    """The consistency terms entered with the wrong sign break the pin above
    (A = K + C + S with K the volume, C the consistency, S the penalty part)."""
    from oracle import dg
    mesh = inputs.small_hp_mesh(0, base=2, depth=1, prob=0.5, pmin=2, pmax=2, dim=3)
    _, space, A = solver.build_operator(mesh, form="sipg")
    _, _, A0 = solver.build_operator(mesh, form="sipg", eta=0.0)      # K + C
    K = dg.assemble(space, 0.0, form="sipg", broken_only=True)
    bad = A - 2 * (A0 - K)                                            # K - C + S
    u = rhs.interpolate(space, U)
    b = rhs.load_vector_fn(space, F)
    assert np.abs(A @ u - b).max() < 1e-10 * np.abs(b).max()
    assert np.abs(bad @ u - b).max() > 1e-3 * np.abs(b).max()


@pytest.mark.parametrize("form", ["sipg", "br2"])
def test_symmetric_positive_definite(form):
    mesh = inputs.small_hp_mesh(2, base=2, depth=2, prob=0.4, pmin=1, pmax=2, dim=3)
    _, _, A = solver.build_operator(mesh, form=form)
    A = A.toarray()
    assert np.abs(A - A.T).max() < 1e-12 * np.abs(A).max()
    assert np.linalg.eigvalsh(A).min() > 0


def test_sipg_penalty_closed_form_hanging():
    """Piecewise constant u: gradients vanish, so a(u,u) = sum over sub-faces
    of sigma |F| [[u]]^2.  One coarse cube next to four fine ones."""
    lh, eta = 0.25, 3.0
    lo = [(0, 0, 0)] + [(2, j, k) for k in (0, 1) for j in (0, 1)]
    size = [2, 1, 1, 1, 1]
    p = [2, 1, 3, 2, 1]
    mesh = _mesh(lo, size, p, (3, 2, 2), lh)
    topo, space, A = solver.build_operator(mesh, form="sipg", eta=eta)
    c = np.array([1.0, -2.0, 0.5, 3.0, 0.0])
    u = np.concatenate([np.full((pk + 1) ** 3, ck) for pk, ck in zip(p, c)])
    expect = 0.0
    for f in topo.subfaces:
        area = (f.hi[0] - f.lo[0]) * (f.hi[1] - f.lo[1]) * lh * lh
        if f.kp >= 0:
            s = eta * max(p[f.km], p[f.kp]) ** 2 / (lh * min(size[f.km], size[f.kp]))
            expect += s * area * (c[f.km] - c[f.kp]) ** 2
        else:
            s = eta * p[f.km] ** 2 / (lh * size[f.km])
            expect += s * area * c[f.km] ** 2
    assert len(topo.subfaces) == 4 + 4 + 5 + 4 * 3   # coarse|fine, fine|fine, boundary
    assert abs(u @ A @ u - expect) < 1e-12 * expect


def test_br2_penalty_closed_form_conforming():
    """Piecewise constant u on a conforming 2x1x1 mesh: the lifting of a unit
    jump on a full face of a cube of side h and degree p has energy
    (p+1)^2 h (the 1D inverse-trace constant (p+1)^2/h times the face area);
    interior faces carry 1/4 of it per side, boundary faces all of it."""
    h, eta = 0.5, 2.0
    for pl, pr in [(1, 1), (2, 3), (3, 1)]:
        mesh = _mesh([(0, 0, 0), (1, 0, 0)], [1, 1], [pl, pr], (2, 1, 1), h)
        _, space, A = solver.build_operator(mesh, form="br2", eta=eta)
        u = np.zeros(space.n)
        u[:(pl + 1) ** 3] = 1.0
        expect = eta * (0.25 * ((pl + 1) ** 2 * h + (pr + 1) ** 2 * h) + 5 * (pl + 1) ** 2 * h)
        assert abs(u @ A @ u - expect) < 1e-11 * expect


@pytest.mark.parametrize("p", [1, 2, 3])
def test_continuous_restriction_is_textbook_fem(p):
    """On a conforming uniform cube mesh, G^T A G (G: continuous nodal gather
    built from node coordinates) is the textbook continuous Q_p stiffness
    assembled from 1D GLL matrices, h^(d-2) (K x M x M + M x K x M + M x M x K)."""
    n = 2
    mesh = inputs.uniform_mesh(3, n, p)
    _, space, A = solver.build_operator(mesh, form="sipg")
    g = basis.gll_nodes(p)
    xg, wg = basis.gauss(p + 1)
    l, dl = basis.lagrange(g, xg), basis.lagrange_deriv(g, xg)
    M1 = (l.T * wg) @ l
    K1 = (dl.T * wg) @ dl
    h = 1.0 / n
    Kel = h * (np.kron(M1, np.kron(M1, K1)) + np.kron(M1, np.kron(K1, M1)) + np.kron(K1, np.kron(M1, M1)))
    # global continuous nodes on the (n p + 1)^3 lattice of GLL points, interior only
    m = n * p + 1
    gid = -np.ones((m, m, m), dtype=np.int64)
    cnt = 0
    for iz, iy, ix in itertools.product(range(1, m - 1), repeat=3):
        gid[iz, iy, ix] = cnt
        cnt += 1
    Kt = np.zeros((cnt, cnt))
    G = np.zeros((space.n, cnt))
    for e in range(mesh.n_elems):
        ex, ey, ez = mesh.lo[e]
        loc = []
        for iz, iy, ix in itertools.product(range(p + 1), repeat=3):
            loc.append(gid[ez * p + iz, ey * p + iy, ex * p + ix])
        loc = np.array(loc)
        for a, ga in enumerate(loc):
            if ga >= 0:
                G[space.offset[e] + a, ga] = 1.0
                for b_, gb in enumerate(loc):
                    if gb >= 0:
                        Kt[ga, gb] += Kel[a, b_]
    GAG = G.T @ (A @ G)
    assert np.abs(GAG - Kt).max() < 1e-11 * np.abs(Kt).max()
