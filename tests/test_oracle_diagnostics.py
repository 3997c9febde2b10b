"""Pins of the lambda_2 vortex criterion (Section 3.2.3; Jeong and Hussain,
1995): the middle eigenvalue of S^2 + Omega^2 from the cell gradients of
Algorithm 4.  The central cell gradient is exact on linear velocity fields
away from the boundary, so interior cells must give the closed forms of
solid-body rotation, pure strain, simple shear and a stretched vortex, and,
for a general gradient G, the middle root of the characteristic polynomial
of (G G + G^T G^T) / 2 (the same matrix written without S and Omega)."""
import numpy as np
import pytest

from oracle.diagnostics import lambda2
from oracle.geometry import Geometry
from paper_2603_21869_gb300 import cases


def _box(nx=8, ny=7, nz=6, L=(1.0, 0.875, 0.75)):
    faces = [cases.Patch(cases.OUTLET) for _ in range(6)]
    spec = cases.CaseSpec(nx=nx, ny=ny, nz=nz, Lx=L[0], Ly=L[1], Lz=L[2], nu=1e-5, faces=faces,
                          dt=0.01, dt_adapt=0, mg_levels=2)
    return Geometry(spec)


def _centres(geo):
    axes = [(np.arange(n) + 0.5) * h for n, h in zip(geo.shape, geo.h)]
    return np.meshgrid(*axes, indexing="ij")


def _linear(geo, G, c=(0.3, -0.2, 0.1)):
    """u_i = c_i + G_ij (x_j - 0.4)."""
    X = _centres(geo)
    return [c[i] + sum(G[i][j] * (X[j] - 0.4) for j in range(3)) for i in range(3)]


def _interior(a):
    return a[1:-1, 1:-1, 1:-1]


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_solid_body_rotation_gives_minus_omega_squared(axis):
    """Rigid rotation at rate W about any axis: S = 0, Omega^2 has
    eigenvalues -W^2, -W^2, 0, so lambda_2 = -W^2."""
    geo = _box()
    W = 1.7
    a, b = [d for d in range(3) if d != axis]
    G = np.zeros((3, 3))
    G[a, b] = -W
    G[b, a] = W
    lam = lambda2(geo, *_linear(geo, G))
    assert np.allclose(_interior(lam), -W * W, rtol=1e-12, atol=0)


def test_pure_strain_gives_plus_a_squared():
    """u = a x, v = -a y: S = diag(a, -a, 0), Omega = 0, eigenvalues a^2, a^2, 0."""
    geo = _box()
    a = 0.9
    lam = lambda2(geo, *_linear(geo, np.diag([a, -a, 0.0])))
    assert np.allclose(_interior(lam), a * a, rtol=1e-12, atol=0)


@pytest.mark.parametrize("i,j", [(0, 1), (2, 0), (1, 2)])
def test_simple_shear_is_not_a_vortex(i, j):
    """u_i = g x_j: S^2 and Omega^2 cancel exactly, lambda_2 = 0."""
    geo = _box()
    g = 2.3
    G = np.zeros((3, 3))
    G[i, j] = g
    lam = lambda2(geo, *_linear(geo, G))
    assert np.max(np.abs(_interior(lam))) <= 1e-12 * g * g


@pytest.mark.parametrize("a,W", [(0.6, 1.1), (2.0, 0.5)])
def test_stretched_vortex(a, W):
    """Rotation W about z with axial strain a (u = -a x/2 - W y, v = W x - a y/2,
    w = a z): eigenvalues a^2/4 - W^2 (twice) and a^2, so lambda_2 = a^2/4 - W^2,
    negative exactly when the rotation beats the in-plane strain."""
    geo = _box()
    G = np.array([[-a / 2, -W, 0.0], [W, -a / 2, 0.0], [0.0, 0.0, a]])
    lam = lambda2(geo, *_linear(geo, G))
    assert np.allclose(_interior(lam), a * a / 4 - W * W, rtol=1e-12, atol=1e-14)
    assert (np.all(_interior(lam) < 0)) == (W > a / 2)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_general_gradient_matches_characteristic_polynomial(seed):
    G = np.random.default_rng(seed).normal(size=(3, 3))
    geo = _box()
    lam = lambda2(geo, *_linear(geo, G))
    M = 0.5 * (G @ G + G.T @ G.T)
    roots = np.sort(np.real(np.roots(np.poly(M))))
    assert np.allclose(_interior(lam), roots[1], rtol=1e-9, atol=1e-12)


def test_two_dimensional_gradient():
    """nz = 1: only the 2x2 block of G acts; M has a zero row and column, and
    lambda_2 is the middle of its two block eigenvalues and 0."""
    faces = [cases.Patch(cases.OUTLET) for _ in range(6)]
    spec = cases.CaseSpec(nx=10, ny=8, nz=1, Lx=1.0, Ly=0.8, Lz=0.1, nu=1e-5, faces=faces, dt=0.01,
                          dt_adapt=0, mg_levels=2)
    geo = Geometry(spec)
    G2 = np.array([[0.4, -1.3], [0.7, -0.4]])
    G = np.zeros((3, 3))
    G[:2, :2] = G2
    X = _centres(geo)
    u = [0.2 + sum(G[i][j] * X[j] for j in range(2)) for i in range(3)]
    lam = lambda2(geo, *u)
    M2 = 0.5 * (G2 @ G2 + G2.T @ G2.T)
    expect = np.sort(np.concatenate([np.linalg.eigvals(M2).real, [0.0]]))[1]
    assert np.allclose(lam[1:-1, 1:-1, 0], expect, rtol=1e-12, atol=1e-14)


def test_solid_cells_zero_and_fluid_finite():
    spec = cases.heated_channel_3d(32, 16, 16, mg_levels=2, init_perturb=0.2,
                                   boxes=[cases.Box(8, 14, 4, 10, 0, 6, thermal=cases.HEAT_FLUX, T_value=100.0)])
    geo = Geometry(spec)
    rng = np.random.default_rng(4)
    u = [rng.normal(size=geo.shape) for _ in range(3)]
    lam = lambda2(geo, *u)
    assert np.all(lam[~geo.fluid] == 0.0)
    assert np.all(np.isfinite(lam))
    # lambda_2 is quadratic in the gradient, and wall, obstacle and outlet ghosts
    # are odd in u: away from the inlet plane (i = 0) reversing u changes nothing
    flipped = lambda2(geo, *[-x for x in u])
    assert np.allclose(flipped[1:], lam[1:], rtol=0, atol=1e-12 * np.max(np.abs(lam)))
    assert not np.allclose(flipped[0], lam[0])


def test_taylor_green_vortex_converges_at_second_order():
    """For a planar divergence-free flow S^2 + Omega^2 = -det(G) on the plane
    (Cayley-Hamilton for a traceless 2x2 G) and 0 across it, so lambda_2 =
    u_y v_x - u_x v_y.  The Taylor-Green vortex u = sin x cos y, v = -cos x sin y
    gives cos^2 x cos^2 y - sin^2 x sin^2 y; the central cell gradient makes the
    discrete value converge to it at second order."""
    errs = []
    for n in (16, 32, 64):
        faces = [cases.Patch(cases.OUTLET) for _ in range(6)]
        L = 2 * np.pi
        spec = cases.CaseSpec(nx=n, ny=n, nz=1, Lx=L, Ly=L, Lz=L / n, nu=1e-5, faces=faces, dt=0.01,
                              dt_adapt=0, mg_levels=2)
        geo = Geometry(spec)
        x = (np.arange(n) + 0.5) * L / n
        X, Y = np.meshgrid(x, x, indexing="ij")
        u = (np.sin(X) * np.cos(Y))[:, :, None]
        v = (-np.cos(X) * np.sin(Y))[:, :, None]
        lam = lambda2(geo, u, v, np.zeros_like(u))[:, :, 0]
        exact = np.cos(X) ** 2 * np.cos(Y) ** 2 - np.sin(X) ** 2 * np.sin(Y) ** 2
        errs.append(float(np.max(np.abs(lam - exact)[1:-1, 1:-1])))
    assert 3.6 < errs[0] / errs[1] < 4.4 and 3.6 < errs[1] / errs[2] < 4.4, errs
