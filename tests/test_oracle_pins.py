"""Pins of the FP64 oracle to things other than itself (CPU only).

Each pin comes from the mathematics of the paper's method, not from the oracle's code:
  * the 1D operator of every sweep is assembled here in finite-volume flux form,
    A = (1 + lambda dt/3) I + (D dt/dx^2) G^T G with G the first difference (zero flux at the
    ends), and solved with LAPACK (numpy) or exactly in rational arithmetic (sympy);
  * closed forms: uniform-field decay (1 + lambda dt/3)^-3 per step, the decay of separable
    cosine modes, D = 0 reducing a step to pointwise division, the source update at D = 0;
  * invariants: mass, discrete maximum principle, sweep-order independence (Kronecker
    operators commute), Dirichlet steady state;
  * the adjoint: dot-product identity and central finite differences.
A plausible slip anywhere in the oracle (sign of a_i, end-row b, an index or stride, the
stage order, the decay split, the source formula) breaks at least one of these.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2602_05017_gb300 import inputs

RNG = np.random.default_rng(12345)


# ---------------------------------------------------------------------------------------------
# Independent dense construction of the operators.
# ---------------------------------------------------------------------------------------------

def fvm_matrix(n, D, dt, dx, lam):
    """(1 + lam dt/3) I + r G^T G: flux form of the zero-flux 1D implicit diffusion-decay step."""
    G = np.zeros((max(n - 1, 0), n))
    for i in range(n - 1):
        G[i, i], G[i, i + 1] = -1.0, 1.0
    return (1.0 + lam * dt / 3.0) * np.eye(n) + (D * dt / dx ** 2) * (G.T @ G)


def dense_sweep(axis, field, D, lam, dt, dx):
    """Apply the inverse of the Kronecker-assembled 3D operator of one sweep, per substrate."""
    nz, ny, nx, ns = field.shape
    out = np.empty_like(field)
    for s in range(ns):
        if axis == 0:
            M = np.kron(np.eye(nz), np.kron(np.eye(ny), fvm_matrix(nx, D[s], dt, dx, lam[s])))
        elif axis == 1:
            M = np.kron(np.eye(nz), np.kron(fvm_matrix(ny, D[s], dt, dx, lam[s]), np.eye(nx)))
        else:
            M = np.kron(fvm_matrix(nz, D[s], dt, dx, lam[s]), np.kron(np.eye(ny), np.eye(nx)))
        out[..., s] = np.linalg.solve(M, field[..., s].reshape(-1)).reshape(nz, ny, nx)
    return out


def face_mask(nz, ny, nx):
    m = np.zeros((nz, ny, nx), dtype=bool)
    m[0], m[-1], m[:, 0], m[:, -1], m[:, :, 0], m[:, :, -1] = (True,) * 6
    return m


def dense_step(w, rho):
    """Src, B, X^-1, B, Y^-1, B, Z^-1, B built from dense pieces."""
    nz, ny, nx, ns = w.shape
    rho = rho.copy()
    if w.n_agents:
        alpha = np.zeros(nz * ny * nx * ns)
        beta = np.zeros_like(alpha)
        wt = np.ones(w.n_agents) if w.weight is None else w.weight
        for k in range(w.n_agents):
            for s in range(ns):
                e = w.voxel[k] * ns + s
                alpha[e] += w.dt * wt[k] * w.secretion[k, s] * w.target[k, s]
                beta[e] += w.dt * wt[k] * (w.secretion[k, s] + w.uptake[k, s])
        rho = ((rho.reshape(-1) + alpha) / (1.0 + beta)).reshape(rho.shape)
    fm = face_mask(nz, ny, nx)

    def B(u):
        u = u.copy()
        if w.dirichlet_on is not None:
            for s in range(ns):
                if w.dirichlet_on[s]:
                    u[..., s][fm] = w.dirichlet_value[s]
        if w.dirichlet_nodes is not None:  # after the faces, in list order
            flat = u.reshape(-1)
            for v, s, val in zip(*w.dirichlet_nodes):
                flat[int(v) * ns + int(s)] = val
        return u

    rho = B(rho)
    h3 = (w.dx,) * 3 if w.spacing is None else w.spacing
    for axis in range(3):
        rho = B(dense_sweep(axis, rho, w.D, w.lam, w.dt, h3[axis]))
    return rho


def P(w):
    return oracle.Problem(**w.oracle_kwargs())


# ---------------------------------------------------------------------------------------------
# Thomas and Appendix A.
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 7, 64])
def test_thomas_matches_lapack_on_diagonally_dominant_systems(n):
    a = RNG.uniform(-1, 1, n)
    c = RNG.uniform(-1, 1, n)
    b = np.abs(a) + np.abs(c) + RNG.uniform(0.1, 2, n)
    d = RNG.normal(size=n)
    M = np.diag(b) + np.diag(a[1:], -1) + np.diag(c[:-1], 1)
    x = oracle.thomas(a, b, c, d)
    np.testing.assert_allclose(x, np.linalg.solve(M, d), rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("n", [1, 2, 3, 10])
def test_appendix_a_matrix_equals_fvm_flux_form(n):
    """a, b, c of App. A (with a_i = c_i = -r) assemble to (1+lam dt/3) I + r G^T G."""
    D, dt, dx, lam = 1e5, 0.01, 20.0, 0.1
    r = D * dt / dx ** 2
    a, b, c, den, cp = oracle.axis_coefficients(n, r, lam * dt / 3)
    M = np.diag(b) + np.diag(a[1:], -1) + np.diag(c[:-1], 1)
    np.testing.assert_allclose(M, fvm_matrix(n, D, dt, dx, lam), rtol=1e-15, atol=1e-15)
    # constant_c and denom are the LU factors of M: M = L U, L = lower(den, a), U = unit upper(c')
    L = np.diag(den) + np.diag(a[1:], -1)
    U = np.eye(n) + np.diag(cp[:-1], 1)
    np.testing.assert_allclose(L @ U, M, rtol=1e-14, atol=1e-14)


# ---------------------------------------------------------------------------------------------
# Sweeps and the full step against dense solves.
# ---------------------------------------------------------------------------------------------

SHAPES = [(1, 1, 1), (1, 2, 3), (3, 1, 2), (2, 3, 1), (6, 5, 4), (3, 3, 3), (5, 2, 6)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_sweep_matches_dense_kronecker_solve(shape, axis):
    nx, ny, nz = shape
    w = inputs.random_problem(RNG, nx, ny, nz, 2)
    got = P(w).sweep(axis, w.rho0)
    ref = dense_sweep(axis, w.rho0, w.D, w.lam, w.dt, w.dx)
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("shape", [(6, 5, 4), (3, 2, 5), (1, 4, 3), (4, 4, 1)])
@pytest.mark.parametrize("dirichlet", [False, True])
@pytest.mark.parametrize("nodes", [0, 9])
def test_step_matches_dense_composition(shape, dirichlet, nodes):
    nx, ny, nz = shape
    w = inputs.random_problem(RNG, nx, ny, nz, 3, n_agents=7, dirichlet=dirichlet, n_nodes=nodes)
    got = P(w).step(w.rho0, 1)
    ref = dense_step(w, w.rho0)
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-12)


def test_step_exact_rational_brute_force():
    """A 3x2x2 grid, 1 substrate, solved exactly in rationals; the oracle is within FP64 rounding."""
    sympy = pytest.importorskip("sympy")
    nx, ny, nz = 3, 2, 2
    D, lam, dt, dx = Fraction(7, 2), Fraction(1, 5), Fraction(1, 10), Fraction(1, 2)
    rho = [Fraction(int(v), 7) for v in RNG.integers(0, 200, nx * ny * nz)]

    def mat(n):
        r = D * dt / dx ** 2
        M = sympy.zeros(n, n)
        for i in range(n):
            M[i, i] = 1 + lam * dt / 3
            if i > 0:
                M[i, i] += r
                M[i, i - 1] = -r
            if i < n - 1:
                M[i, i] += r
                M[i, i + 1] = -r
        return M

    def kron(A, B):
        return sympy.Matrix(sympy.kronecker_product(A, B))

    Ax, Ay, Az = mat(nx), mat(ny), mat(nz)
    X = kron(sympy.eye(nz), kron(sympy.eye(ny), Ax))
    Y = kron(sympy.eye(nz), kron(Ay, sympy.eye(nx)))
    Z = kron(Az, kron(sympy.eye(ny), sympy.eye(nx)))
    v = sympy.Matrix(rho)
    v = Z.LUsolve(Y.LUsolve(X.LUsolve(v)))
    exact = np.array([float(t) for t in v]).reshape(nz, ny, nx, 1)
    w = inputs.Workload("exact", nx, ny, nz, 1, float(dx), float(dt), np.array([float(D)]),
                        np.array([float(lam)]), 1)
    got = P(w).step(np.array([float(t) for t in rho]).reshape(nz, ny, nx, 1), 1)
    np.testing.assert_allclose(got, exact, rtol=4e-16 * 20, atol=0)


# ---------------------------------------------------------------------------------------------
# Closed forms.
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("shape", [(1, 1, 1), (7, 5, 3), (16, 16, 16)])
def test_uniform_field_decays_by_exact_factor(shape):
    nx, ny, nz = shape
    w = inputs.random_problem(RNG, nx, ny, nz, 4)
    c = RNG.uniform(1, 38, 4)
    rho = np.broadcast_to(c, w.shape).copy()
    out = P(w).step(rho, 5)
    factor = (1.0 + w.lam * w.dt / 3.0) ** (-15)
    np.testing.assert_allclose(out, np.broadcast_to(c * factor, w.shape), rtol=2e-14)


def cosine_mode(nx, ny, nz, k):
    ix, iy, iz = np.arange(nx), np.arange(ny), np.arange(nz)
    fx = np.cos(k[0] * np.pi * (ix + 0.5) / nx)
    fy = np.cos(k[1] * np.pi * (iy + 0.5) / ny)
    fz = np.cos(k[2] * np.pi * (iz + 0.5) / nz)
    return fz[:, None, None] * fy[None, :, None] * fx[None, None, :]


def mode_factor(n, k, D, lam, dt, dx):
    r = D * dt / dx ** 2
    out = 1.0
    for nd, kd in zip(n, k):
        out /= 1.0 + lam * dt / 3.0 + 2.0 * r * (1.0 - math.cos(kd * math.pi / nd))
    return out


@pytest.mark.parametrize("k", list(itertools.product([0, 1, 4], [0, 1, 5], [0, 3, 11])))
def test_cosine_modes_decay_by_closed_form(k):
    nx, ny, nz = 8, 10, 12
    D = np.array([1e5, 3e2])
    lam = np.array([0.1, 0.7])
    w = inputs.Workload("cos", nx, ny, nz, 2, 20.0, 0.01, D, lam, 1)
    base = cosine_mode(nx, ny, nz, k)
    rho = np.stack([base, base], axis=-1)
    out = P(w).step(rho, 3)
    for s in range(2):
        f = mode_factor((nx, ny, nz), k, D[s], lam[s], w.dt, w.dx) ** 3
        # rounding scales with the amplitude before the steps (1), not with the decayed one
        np.testing.assert_allclose(out[..., s], f * base, rtol=1e-12, atol=1e-14)


# ---------------------------------------------------------------------------------------------
# Anisotropic spacing (dx, dy, dz): each axis's App. A system takes r = D dt / h^2 with its own h.
# ---------------------------------------------------------------------------------------------

def test_isotropic_spacing_triple_equals_scalar():
    w = inputs.random_problem(RNG, 7, 6, 5, 2, n_agents=8, dirichlet=True)
    a = P(w).step(w.rho0, 2)
    w.spacing = (w.dx, w.dx, w.dx)
    assert np.array_equal(P(w).step(w.rho0, 2), a)


@pytest.mark.parametrize("dirichlet", [False, True])
def test_anisotropic_step_matches_dense_composition(dirichlet):
    w = inputs.random_problem(RNG, 5, 4, 6, 2, n_agents=7, dirichlet=dirichlet)
    w.spacing = (10.0, 25.0, 40.0)
    np.testing.assert_allclose(P(w).step(w.rho0, 1), dense_step(w, w.rho0), rtol=1e-12,
                               atol=1e-12)


@pytest.mark.parametrize("k", [(1, 0, 0), (0, 2, 0), (0, 0, 3), (2, 1, 4)])
def test_anisotropic_cosine_modes_decay_by_closed_form(k):
    """prod_d 1 / (1 + lambda dt/3 + 2 (D dt / h_d^2) (1 - cos(k_d pi / n_d)))."""
    nx, ny, nz = 9, 8, 10
    h3 = (12.0, 20.0, 31.0)
    D, lam, dt = 2e4, 0.3, 0.01
    w = inputs.Workload("cos", nx, ny, nz, 1, h3[0], dt, np.array([D]), np.array([lam]), 1)
    w.spacing = h3
    base = cosine_mode(nx, ny, nz, k)
    out = P(w).step(base[..., None], 2)[..., 0]
    f = 1.0
    for nd, kd, hd in zip((nx, ny, nz), k, h3):
        f /= 1.0 + lam * dt / 3.0 + 2.0 * (D * dt / hd ** 2) * (1.0 - math.cos(kd * math.pi / nd))
    np.testing.assert_allclose(out, f ** 2 * base, rtol=1e-12, atol=1e-14)


def test_anisotropic_adjoint_D_matches_finite_differences():
    w = inputs.random_problem(RNG, 6, 5, 4, 2, n_agents=5, dirichlet=True)
    w.spacing = (15.0, 22.0, 30.0)
    probes = RNG.choice(w.rho0.size, 20, replace=False)
    targets = RNG.uniform(0, 38, 20)
    L0, _, dD, dl, _, _ = _loss_and_grads(w, 2, probes, targets)
    import copy
    for s in range(2):
        h = 1e-6 * max(1.0, abs(w.D[s]))
        up, dn = copy.deepcopy(w), copy.deepcopy(w)
        up.D = w.D.copy()
        dn.D = w.D.copy()
        up.D[s] += h
        dn.D[s] -= h
        fd = (_loss_and_grads(up, 2, probes, targets)[0] -
              _loss_and_grads(dn, 2, probes, targets)[0]) / (2 * h)
        noise = 8 * np.finfo(float).eps * abs(L0) / h
        assert dD[s] == pytest.approx(fd, rel=1e-6, abs=noise), s


def test_zero_diffusion_is_pointwise_division():
    w = inputs.random_problem(RNG, 5, 4, 3, 3)
    w.D = np.zeros(3)
    out = P(w).step(w.rho0, 2)
    np.testing.assert_allclose(out, w.rho0 * (1 + w.lam * w.dt / 3) ** (-6), rtol=1e-15)


def test_zero_diffusion_zero_decay_is_the_source_update():
    w = inputs.random_problem(RNG, 6, 5, 4, 2, n_agents=30)
    w.D = np.zeros(2)
    w.lam = np.zeros(2)
    out = P(w).step(w.rho0, 1)
    # aggregate exactly as stated: alpha = sum dt w S rho*, beta = sum dt w (S + U)
    alpha = np.zeros(w.rho0.size)
    beta = np.zeros(w.rho0.size)
    for k in range(w.n_agents):
        for s in range(2):
            e = w.voxel[k] * 2 + s
            alpha[e] += w.dt * w.weight[k] * w.secretion[k, s] * w.target[k, s]
            beta[e] += w.dt * w.weight[k] * (w.secretion[k, s] + w.uptake[k, s])
    ref = (w.rho0.reshape(-1) + alpha) / (1 + beta)
    np.testing.assert_allclose(out.reshape(-1), ref, rtol=1e-15)


def test_source_fixed_point_and_pure_uptake():
    w = inputs.Workload("src", 4, 3, 2, 1, 20.0, 0.1, np.zeros(1), np.zeros(1), 1)
    w.voxel = np.array([0, 5], dtype=np.int64)
    w.secretion = np.array([[7.0], [0.0]])
    w.target = np.array([[38.0], [38.0]])
    w.uptake = np.array([[0.0], [2.5]])
    rho = np.full(w.shape, 38.0)
    rho.reshape(-1)[5] = 10.0
    out = P(w).step(rho, 1).reshape(-1)
    assert out[0] == pytest.approx(38.0, rel=1e-15)  # a secreting voxel at its target stays there
    assert out[5] == pytest.approx(10.0 / (1 + 0.1 * 2.5), rel=1e-15)


def test_agent_order_does_not_matter():
    w = inputs.random_problem(RNG, 5, 5, 5, 2, n_agents=60)
    w.voxel[:30] = w.voxel[30:]  # many shared voxels
    a = P(w).step(w.rho0, 2)
    perm = RNG.permutation(w.n_agents)
    w.voxel, w.secretion, w.target, w.uptake, w.weight = (
        w.voxel[perm], w.secretion[perm], w.target[perm], w.uptake[perm], w.weight[perm])
    b = P(w).step(w.rho0, 2)
    np.testing.assert_allclose(a, b, rtol=1e-14)


# ---------------------------------------------------------------------------------------------
# Invariants.
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("shape", [(9, 7, 5), (1, 6, 6), (13, 1, 2)])
def test_mass_scales_by_decay_factor_for_any_field(shape):
    nx, ny, nz = shape
    w = inputs.random_problem(RNG, nx, ny, nz, 3)
    out = P(w).step(w.rho0, 1)
    m0 = w.rho0.sum(axis=(0, 1, 2))
    m1 = out.sum(axis=(0, 1, 2))
    np.testing.assert_allclose(m1, m0 * (1 + w.lam * w.dt / 3) ** (-3), rtol=1e-13)


def test_mass_conserved_without_decay():
    w = inputs.random_problem(RNG, 11, 8, 6, 2)
    w.lam = np.zeros(2)
    out = P(w).step(w.rho0, 10)
    np.testing.assert_allclose(out.sum(axis=(0, 1, 2)), w.rho0.sum(axis=(0, 1, 2)), rtol=1e-13)


def test_mass_change_equals_source_change_when_D_only():
    """With lambda = 0, diffusion moves mass around; the source update alone changes it."""
    w = inputs.random_problem(RNG, 7, 6, 5, 2, n_agents=25)
    w.lam = np.zeros(2)
    out = P(w).step(w.rho0, 1)
    w0 = inputs.Workload("s", 7, 6, 5, 2, w.dx, w.dt, np.zeros(2), np.zeros(2), 1)
    w0.voxel, w0.secretion, w0.target, w0.uptake, w0.weight = (
        w.voxel, w.secretion, w.target, w.uptake, w.weight)
    src_only = P(w0).step(w.rho0, 1)
    np.testing.assert_allclose(out.sum(axis=(0, 1, 2)), src_only.sum(axis=(0, 1, 2)), rtol=1e-13)


def test_sweep_order_does_not_matter_without_dirichlet():
    w = inputs.random_problem(RNG, 9, 6, 7, 2)
    p = P(w)
    xyz = p.sweep(2, p.sweep(1, p.sweep(0, w.rho0)))
    zyx = p.sweep(0, p.sweep(1, p.sweep(2, w.rho0)))
    np.testing.assert_allclose(xyz, zyx, rtol=1e-13)


def test_discrete_maximum_principle():
    w = inputs.random_problem(RNG, 10, 9, 8, 3)
    out = P(w).step(w.rho0, 4)
    assert out.min() >= 0.0
    assert (out.max(axis=(0, 1, 2)) <= w.rho0.max(axis=(0, 1, 2)) * (1 + 1e-14)).all()


def test_dirichlet_steady_state_and_faces():
    w = inputs.random_problem(RNG, 7, 6, 5, 2, dirichlet=True)
    w.dirichlet_on = np.array([1, 1], dtype=np.uint8)
    w.lam = np.zeros(2)
    c = w.dirichlet_value
    rho = np.broadcast_to(c, w.shape).copy()
    out = P(w).step(rho, 3)
    np.testing.assert_allclose(out, rho, rtol=1e-14)
    # from a random start, faces equal the value after every step
    out = P(w).step(w.rho0, 2)
    fm = face_mask(5, 6, 7)
    for s in range(2):
        assert np.all(out[..., s][fm] == c[s])


def test_dirichlet_nodes_steady_state_and_values():
    """Nodes holding the value of a uniform field keep it exactly without decay (the field is
    then a fixed point of every stage); from a random start each listed element holds its last
    listed value after every step, and an element listed twice takes the later value."""
    w = inputs.random_problem(RNG, 6, 5, 7, 2, n_nodes=12)
    w.lam = np.zeros(2)
    c = 11.0
    voxel, sub, _ = w.dirichlet_nodes
    w.dirichlet_nodes = (voxel, sub, np.full(voxel.size, c))
    rho = np.full(w.shape, c)
    np.testing.assert_allclose(P(w).step(rho, 3), rho, rtol=1e-14)
    w = inputs.random_problem(RNG, 6, 5, 7, 2, n_agents=10, n_nodes=12)
    voxel, sub, val = w.dirichlet_nodes
    assert (voxel[0], sub[0]) == (voxel[-1], sub[-1]) and val[0] != val[-1]
    out = P(w).step(w.rho0, 2).reshape(-1)
    last = {}
    for v, s_, x in zip(voxel, sub, val):
        last[int(v) * 2 + int(s_)] = x
    for e, x in last.items():
        assert out[e] == x


def test_face_value_nodes_equal_face_dirichlet():
    """The same value on all six faces, given as per-face nodes, is the face Dirichlet
    condition: identical steps."""
    w = inputs.random_problem(RNG, 5, 6, 4, 3, n_agents=9, dirichlet=True)
    faces = np.full((6, 3), np.nan)
    for s in range(3):
        if w.dirichlet_on[s]:
            faces[:, s] = w.dirichlet_value[s]
    ref = P(w).step(w.rho0, 2)
    w.dirichlet_nodes = inputs.face_value_nodes(5, 6, 4, faces)
    w.dirichlet_on, w.dirichlet_value = None, None
    np.testing.assert_array_equal(P(w).step(w.rho0, 2), ref)


# ---------------------------------------------------------------------------------------------
# Adjoint.
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("nodes", [0, 10])
def test_adjoint_dot_product_identity(nodes):
    w = inputs.random_problem(RNG, 6, 5, 4, 2, n_agents=9, dirichlet=True, n_nodes=nodes)
    p = P(w)
    u = RNG.normal(size=w.shape)
    v = RNG.normal(size=w.shape)
    zero = np.zeros(w.shape)
    Ju = p.step(u, 1) - p.step(zero, 1)  # the step is affine in rho
    JTv = p.adjoint_step(u, v)[0]
    lhs, rhs = float((Ju * v).sum()), float((u * JTv).sum())
    assert abs(lhs - rhs) <= 1e-13 * (abs(lhs) + abs(rhs))


def _loss_and_grads(w, n_steps, probes, targets):
    p = P(w)
    states = [w.rho0.copy()]
    for _ in range(n_steps):
        states.append(p.step(states[-1], 1))
    fin = states[-1].reshape(-1)
    loss = float(((fin[probes] - targets) ** 2).sum())
    g = np.zeros(fin.size)
    g[probes] = 2.0 * (fin[probes] - targets)
    g = g.reshape(w.shape)
    dD = np.zeros(w.ns)
    dl = np.zeros(w.ns)
    ds = np.zeros((w.n_agents, w.ns))
    du = np.zeros((w.n_agents, w.ns))
    for k in range(n_steps - 1, -1, -1):
        g, a, b, c, u = p.adjoint_step(states[k], g)
        dD += a
        dl += b
        ds += c
        du += u
    return loss, g, dD, dl, ds, du


@pytest.mark.parametrize("nodes", [0, 8])
def test_adjoint_matches_central_finite_differences(nodes):
    """Central differences with step h carry a rounding error of about eps*|L|/h on top of the
    O(h^2) truncation; the tolerance is 1e-6 relative plus that bound.  With Dirichlet nodes,
    some of them sit on agents' voxels (their secretion then has no effect)."""
    w = inputs.random_problem(RNG, 6, 5, 4, 2, n_agents=6, dirichlet=True, n_nodes=nodes)
    w.dirichlet_on = np.array([1, 0], dtype=np.uint8)
    if nodes:
        voxel, sub, val = w.dirichlet_nodes
        voxel[:2], sub[:2] = w.voxel[:2], 1
        w.dirichlet_nodes = (voxel, sub, val)
    nsteps = 3
    probes = RNG.choice(w.rho0.size, 25, replace=False)
    targets = RNG.uniform(0, 38, 25)
    L0, g0, dD, dl, ds, du = _loss_and_grads(w, nsteps, probes, targets)

    def loss_with(**kw):
        import copy
        ww = copy.deepcopy(w)
        for k, v in kw.items():
            setattr(ww, k, v)
        return _loss_and_grads(ww, nsteps, probes, targets)[0]

    def check(grad, fd, h, what):
        noise = 8 * np.finfo(float).eps * abs(L0) / h
        assert grad == pytest.approx(fd, rel=1e-6, abs=noise), what

    for s in range(2):
        for name, grad in (("D", dD), ("lam", dl)):
            base = getattr(w, name)
            h = 1e-6 * max(1.0, abs(base[s]))
            up, dn = base.copy(), base.copy()
            up[s] += h
            dn[s] -= h
            check(grad[s], (loss_with(**{name: up}) - loss_with(**{name: dn})) / (2 * h), h,
                  (name, s))
    for k in range(w.n_agents):
        for s in range(2):
            h = 1e-5 * max(1.0, abs(w.secretion[k, s]))
            up, dn = w.secretion.copy(), w.secretion.copy()
            up[k, s] += h
            dn[k, s] -= h
            check(ds[k, s], (loss_with(secretion=up) - loss_with(secretion=dn)) / (2 * h), h,
                  ("sec", k, s))
            # uptake rate: the sinks' rates and the sources' zero uptake alike
            h = 1e-5 * max(1.0, abs(w.uptake[k, s]))
            up, dn = w.uptake.copy(), w.uptake.copy()
            up[k, s] += h
            dn[k, s] -= h
            check(du[k, s], (loss_with(uptake=up) - loss_with(uptake=dn)) / (2 * h), h,
                  ("upt", k, s))
    flat = w.rho0.reshape(-1)
    for e in RNG.choice(flat.size, 12, replace=False):
        h = 1e-5 * max(1.0, abs(flat[e]))
        up, dn = w.rho0.copy(), w.rho0.copy()
        up.reshape(-1)[e] += h
        dn.reshape(-1)[e] -= h
        check(g0.reshape(-1)[e], (loss_with(rho0=up) - loss_with(rho0=dn)) / (2 * h), h,
              ("rho0", e))


# ---------------------------------------------------------------------------------------------
# Argument checking.
# ---------------------------------------------------------------------------------------------

def test_bad_arguments_are_rejected():
    w = inputs.random_problem(RNG, 3, 3, 3, 1, n_agents=2)
    w.voxel[0] = 27  # out of range
    with pytest.raises(ValueError):
        P(w).step(w.rho0, 1)
    with pytest.raises(ValueError):
        oracle.axis_coefficients(0, 1.0, 0.0)


# ---------------------------------------------------------------------------------------------
# The OpenMP copy (paper-style CPU rate) computes every line with the same statements.
# ---------------------------------------------------------------------------------------------

def test_openmp_copy_gives_the_same_bits_as_the_plain_oracle():
    rng = np.random.default_rng(404)
    w = inputs.random_problem(rng, 23, 19, 17, 3, n_agents=60, dirichlet=True, n_nodes=25)
    w.spacing = (20.0, 17.0, 26.0)
    a = P(w).step(w.rho0, 3)
    b = oracle.Problem(**w.oracle_kwargs(), parallel=True).step(w.rho0, 3)
    np.testing.assert_array_equal(a, b)
