"""Pins of the oracle's Poisson operator, multigrid and projection
(Section 2.4, Algorithm 1) against the printed kernel, polynomial
exactness, brute-force dense solves and a manufactured solution."""
import os

import numpy as np
import pytest

from oracle import poisson
from oracle.geometry import Geometry
from oracle.poisson import Multigrid, apply_A, direct_solve, prolong, restrict
from oracle.step import OracleCase
from paper_2603_21869_gb300 import cases

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _spec(nx, ny, nz, L=(1.0, 1.0, 1.0), outlet_faces=(1,), boxes=(), levels=2, **kw):
    faces = [cases.Patch(cases.WALL) for _ in range(6)]
    for f in outlet_faces:
        faces[f] = cases.Patch(cases.OUTLET)
    if nz == 1:
        faces[4] = cases.Patch(cases.EMPTY)
        faces[5] = cases.Patch(cases.EMPTY)
    return cases.CaseSpec(nx=nx, ny=ny, nz=nz, Lx=L[0], Ly=L[1], Lz=L[2], faces=faces,
                          boxes=list(boxes), mg_levels=levels, **kw)


def test_printed_laplacian_kernel():
    """A applied to a unit impulse reproduces the printed 3x3x3 kernel (x -1/dx^2)."""
    rows = [list(map(float, l.split())) for l in open(os.path.join(GOLDEN, "laplacian_kernel.txt"))
            if l.strip() and not l.startswith("#")]
    K = np.array(rows).reshape(3, 3, 3)          # [k][j][i]
    h = 0.125
    geo = Geometry(_spec(8, 8, 8))
    lev = geo.level0
    e = np.zeros(lev.shape)
    e[4, 4, 4] = 1.0
    Ae = apply_A(lev, e)
    # A = -(1/h^2) K * BC(p): the response at cell c to an impulse at (4,4,4) is
    # -(1/h^2) K[offset], and K is symmetric so orientation does not matter
    got = Ae[3:6, 3:6, 3:6].transpose(2, 1, 0)
    assert np.allclose(got, -K / h ** 2, rtol=1e-14, atol=0)
    assert np.count_nonzero(Ae) == 7


def test_jacobi_diagonal_is_six_over_dx2():
    """Eq. jacobi_pc: D replaced by the scalar 6/dx^2 (isotropic 3D)."""
    geo = Geometry(_spec(8, 8, 8))
    assert geo.level0.diag() == pytest.approx(6.0 / 0.125 ** 2, rel=1e-15)
    geo2 = Geometry(_spec(8, 4, 1, L=(1.0, 0.5, 0.125)))
    assert geo2.level0.diag() == pytest.approx(4.0 / 0.125 ** 2, rel=1e-15)


def test_A_exact_on_quadratic():
    """-Laplacian_h of x^2 + 3 y^2 - z^2 is exactly -(2 + 6 - 2) = -6 in the interior."""
    geo = Geometry(_spec(8, 8, 8))
    x = (np.arange(8) + 0.5) / 8
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    Ap = apply_A(geo.level0, X ** 2 + 3 * Y ** 2 - Z ** 2)
    assert np.allclose(Ap[1:-1, 1:-1, 1:-1], -6.0, rtol=0, atol=1e-10)


def test_neumann_and_dirichlet_ghosts():
    """Zero-gradient faces: A(const) = 0 next to walls; an outlet face adds
    2/h^2 (ghost = -p puts p = 0 on the face)."""
    geo = Geometry(_spec(8, 8, 8, outlet_faces=(1,)))
    Ap = apply_A(geo.level0, np.ones((8, 8, 8)))
    assert np.allclose(Ap[:-1], 0.0, atol=1e-10)
    assert np.allclose(Ap[-1], 2.0 / 0.125 ** 2, rtol=1e-14)


def test_restrict_prolong_properties():
    lev = Geometry(_spec(8, 8, 8, outlet_faces=())).level0
    clev = lev.coarsen()                     # all faces zero-gradient
    c = np.random.default_rng(0).normal(size=(4, 4, 4))
    # RES is the mean of children: constant in, constant out; sums scale by 1/8
    r = np.random.default_rng(1).normal(size=(8, 8, 8))
    assert np.allclose(restrict(lev, np.full((8, 8, 8), 3.5)), 3.5)
    assert restrict(lev, r).sum() == pytest.approx(r.sum() / 8, rel=1e-13)
    # PROL reproduces constants everywhere (zero-gradient ghosts) and linear functions away
    # from the domain faces
    assert np.allclose(prolong(clev, np.full((4, 4, 4), 2.0), (8, 8, 8)), 2.0)
    xc = (np.arange(4) + 0.5) * 2.0
    xf = np.arange(8) + 0.5
    lin_c = xc[:, None, None] + 0 * c
    lin_f = prolong(clev, lin_c, (8, 8, 8))
    assert np.allclose(lin_f[1:-1, :, :], xf[1:-1, None, None], atol=1e-13)
    # weights (27, 9, 9, 3, 9, 3, 3, 1)/64 around an interior fine cell
    imp = np.zeros((4, 4, 4))
    imp[1, 1, 1] = 64.0
    pf = prolong(clev, imp, (8, 8, 8))
    assert pf[2, 2, 2] == pytest.approx(27) and pf[3, 3, 3] == pytest.approx(27)
    assert pf[1, 2, 2] == pytest.approx(9) and pf[1, 1, 2] == pytest.approx(3)
    assert pf[1, 1, 1] == pytest.approx(1) and pf[4, 4, 4] == pytest.approx(1)


def test_prolong_takes_the_coarse_ghost_beyond_a_domain_face():
    """Across a zero-value (outlet) face the neighbour is the negated cell: a
    function linear in x that vanishes on that face is interpolated exactly up
    to the face, and a constant falls to half its value in the fine cells
    touching the face (the linear profile through 0 on the face).  Across a
    zero-gradient face the neighbour is the cell itself."""
    lev = Geometry(_spec(8, 8, 8, outlet_faces=(0,))).level0   # x- face zero-value
    clev = lev.coarsen()
    xc = (np.arange(4) + 0.5) * 2.0          # coarse centres (h = 1 on the fine grid), face at x = 0
    xf = np.arange(8) + 0.5
    lin_f = prolong(clev, xc[:, None, None] * np.ones((4, 4, 4)), (8, 8, 8))
    assert np.allclose(lin_f[:-1], np.broadcast_to(xf[:-1, None, None], (7, 8, 8)), rtol=0, atol=1e-13)
    # the x+ face is zero-gradient: the last fine cell takes 3/4 + 1/4 of the last coarse cell
    assert np.allclose(lin_f[-1], xc[-1], rtol=0, atol=1e-13)
    const = prolong(clev, np.full((4, 4, 4), 4.0), (8, 8, 8))
    assert np.allclose(const[0], 2.0, rtol=0, atol=1e-14) and np.allclose(const[1:], 4.0, rtol=0, atol=1e-14)


def test_prolong_corner_ghost_carries_both_face_signs():
    """A fine cell in the corner of two zero-value faces: of its 8 (2D: 4)
    interpolation points, the ghost across both faces is the cell with two
    sign flips (+), the two single-face ghosts are negated."""
    lev = Geometry(_spec(8, 8, 1, L=(1.0, 1.0, 0.125), outlet_faces=(0, 2))).level0   # x- and y- zero-value
    clev = lev.coarsen()
    c = np.zeros((4, 4, 1))
    c[0, 0, 0] = 16.0
    pf = prolong(clev, c, (8, 8, 1))
    # fine (0, 0): 9/16 c + 3/16 (-c) [x ghost] + 3/16 (-c) [y ghost] + 1/16 (+c) [corner] = 4/16 c
    assert pf[0, 0, 0] == pytest.approx(4.0, rel=1e-14)
    # fine (1, 0): parent (0,0), x neighbour (1,0) = 0; y ghost row: -c and the ghost of (1, 0), 0
    assert pf[1, 0, 0] == pytest.approx(16.0 * (9 - 3) / 16, rel=1e-14)
    # fine (1, 1): no ghost involved
    assert pf[1, 1, 0] == pytest.approx(9.0, rel=1e-14)


@pytest.mark.parametrize("shape,boxes,levels", [
    ((16, 8, 8), (), 3),
    ((16, 8, 8), (cases.Box(4, 8, 2, 6, 0, 4),), 3),
    ((16, 8, 1), (), 3),
    ((32, 16, 1), (cases.Box(12, 16, 0, 8, 0, 1),), 4),
])
def test_vcycles_converge_to_dense_solution(shape, boxes, levels):
    """Brute force: the V-cycle iterates converge to the dense LU solution
    (isotropic cells; point Jacobi with full coarsening is not a smoother
    for stretched cells)."""
    nx, ny, nz = shape
    spec = _spec(nx, ny, nz, L=(2.0, 1.0, 1.0 if nz > 1 else 1.0 / ny), boxes=boxes,
                 levels=levels, outlet_faces=(1,), pre_sweeps=3, post_sweeps=3)
    geo = Geometry(spec)
    lev = geo.level0
    b = np.random.default_rng(7).normal(size=lev.shape)
    b[lev.solid] = 0.0
    p_direct = direct_solve(lev, b)
    mg = Multigrid(geo, levels)
    p = np.zeros(lev.shape)
    rels = []
    for _ in range(40):
        p = mg.vcycle(p, b)
        rels.append(mg.rel_residual(p, b))
        if rels[-1] < 1e-13:
            break
    assert np.max(np.abs(p - p_direct)) <= 1e-10 * np.max(np.abs(p_direct))
    assert np.all(p[lev.solid] == 0.0)


@pytest.mark.parametrize("levels,sweeps,bound", [(2, 2, 0.3), (4, 3, 0.3)])
def test_vcycle_contraction_factor(levels, sweeps, bound):
    """Sanity bound on the asymptotic residual contraction per cycle: the
    two-grid V(2,2) and the 4-level V(3,3) with weighted Jacobi, child-mean
    restriction and trilinear prolongation contract by better than 0.3."""
    spec = _spec(32, 32, 32, levels=levels, outlet_faces=(1,), pre_sweeps=sweeps, post_sweeps=sweeps)
    geo = Geometry(spec)
    mg = Multigrid(geo, levels)
    b = np.random.default_rng(2).normal(size=geo.shape)
    p = np.zeros(geo.shape)
    rs = [mg.rel_residual(p, b)]
    for _ in range(8):
        p = mg.vcycle(p, b)
        rs.append(mg.rel_residual(p, b))
    rho = (rs[-1] / rs[4]) ** (1 / 4)
    assert rho < bound


def _manufactured_error(n):
    Lx, Ly, Lz = 2.0, 1.0, 1.0
    spec = _spec(2 * n, n, n, L=(Lx, Ly, Lz), outlet_faces=(1,), levels=3)
    geo = Geometry(spec)
    hx, hy, hz = geo.h
    x = (np.arange(2 * n) + 0.5) * hx
    y = (np.arange(n) + 0.5) * hy
    z = (np.arange(n) + 0.5) * hz
    X, Y, Z = np.meshgrid(x, y, z, indexing="ij")
    # dp/dn = 0 on x = 0 and on the y, z walls; p = 0 on the outlet face x = Lx
    p_ex = np.cos(np.pi * X / (2 * Lx)) * np.cos(np.pi * Y / Ly) * np.cos(np.pi * Z / Lz)
    lam = np.pi ** 2 * (1 / (4 * Lx ** 2) + 1 / Ly ** 2 + 1 / Lz ** 2)
    b = lam * p_ex
    mg = Multigrid(geo, 3)
    p = np.zeros(geo.shape)
    for _ in range(60):
        p = mg.vcycle(p, b)
        if mg.rel_residual(p, b) < 1e-12:
            break
    return np.max(np.abs(p - p_ex))


def test_manufactured_solution_second_order():
    e1 = _manufactured_error(8)
    e2 = _manufactured_error(16)
    assert 3.3 < e1 / e2 < 4.7
    assert e2 < 5e-3


def test_projection_with_direct_solve_is_divergence_free():
    """With the exact discrete pressure the corrected face fluxes have zero
    divergence: div = dt (A p - b)."""
    spec = cases.heated_channel_3d(16, 8, 8, mg_levels=2, init_perturb=0.05,
                                   boxes=[cases.Box(5, 8, 2, 5, 0, 3)])
    c = OracleCase(spec)
    c.destruction_half()
    c.explicit()
    c.destruction_half()
    c.rhs()
    lev = c.mg.levels[0]
    p = direct_solve(lev, c.b)
    u, v, w = c.state[:3]
    div = poisson.face_divergence(c.geo, lev, u, v, w, p, c.dt)
    scale = np.max(np.abs(c.b)) * c.dt
    assert scale > 1e-6
    assert np.max(np.abs(div)) < 1e-11 * scale
    # and for an arbitrary p the identity div = dt (A p - b) holds exactly
    q = np.random.default_rng(4).normal(size=lev.shape)
    q[lev.solid] = 0.0
    div_q = poisson.face_divergence(c.geo, lev, u, v, w, q, c.dt)
    ident = c.dt * (apply_A(lev, q) - c.b)
    assert np.allclose(div_q[lev.fluid], ident[lev.fluid], rtol=0, atol=1e-12 * scale * 1e3)


def test_rhs_zero_for_uniform_through_flow():
    """Uniform u with matching inlet speed and zero-gradient outlet is
    discretely divergence free: b = 0."""
    spec = cases.heated_channel_3d(16, 8, 8, mg_levels=2)
    faces = list(spec.faces)
    faces[2] = faces[3] = faces[4] = faces[5] = cases.Patch(cases.OUTLET)
    spec = spec.replace(faces=faces, init_perturb=0.0)
    c = OracleCase(spec)
    c.rhs()
    assert np.max(np.abs(c.b)) == 0.0


# ------------------------------------------------------------------ the paper's scheme (Algorithm 1)
def test_nearest_upsampling_is_a_kronecker_product_with_ones():
    from oracle.poisson import prolong_nearest
    rng = np.random.default_rng(3)
    c3 = rng.normal(size=(3, 2, 4))
    assert np.array_equal(prolong_nearest(c3, (6, 4, 8)), np.kron(c3, np.ones((2, 2, 2))))
    c2 = rng.normal(size=(5, 3, 1))
    assert np.array_equal(prolong_nearest(c2, (10, 6, 1)), np.kron(c2, np.ones((2, 2, 1))))


def test_paper_scheme_keeps_the_exact_solution_and_reduces_the_residual():
    """The discrete solution of A p = b is a fixed point of an Algorithm-1
    iteration (every correction it forms is zero there), and from zero the
    iteration lowers the residual every step on this case, more slowly than
    a V(3,3) cycle."""
    from paper_2603_21869_gb300 import cases
    from oracle.step import OracleCase
    from oracle.poisson import direct_solve
    spec = cases.heated_channel_3d(32, 16, 16, mg_levels=3)
    mg = OracleCase(spec).mg
    lev = mg.levels[0]
    rng = np.random.default_rng(1)
    b = np.where(lev.fluid, rng.normal(size=lev.shape), 0.0)
    pstar = direct_solve(lev, b)
    assert np.max(np.abs(mg.paper_cycle(pstar, b) - pstar)) <= 1e-13 * np.max(np.abs(pstar))
    p = np.zeros(lev.shape)
    q = np.zeros(lev.shape)
    rel = [1.0]
    for _ in range(6):
        p = mg.paper_cycle(p, b)
        q = mg.vcycle(q, b)
        rel.append(mg.rel_residual(p, b))
    assert all(a > c for a, c in zip(rel, rel[1:]))
    assert mg.rel_residual(q, b) < rel[-1]


def test_paper_scheme_converges_at_any_depth():
    """With the fine grid's A and D on every level (one shared kernel), the
    scheme's contraction does not degrade with the number of levels (with
    coarse operators rescaled to each level's spacing it diverges from four
    levels on: each level's single Jacobi step then overshoots)."""
    from paper_2603_21869_gb300 import cases
    from oracle.step import OracleCase
    rates = []
    for nx, ny, nz, L in ((32, 16, 16, 3), (128, 32, 32, 5)):
        mg = OracleCase(cases.heated_channel_3d(nx, ny, nz, mg_levels=L)).mg
        lev = mg.levels[0]
        b = np.where(lev.fluid, np.random.default_rng(1).normal(size=lev.shape), 0.0)
        p = np.zeros(lev.shape)
        for _ in range(10):
            p = mg.paper_cycle(p, b)
        rates.append(mg.rel_residual(p, b))
    assert rates[1] < 0.1 and rates[1] < 1.5 * rates[0]


# ------------------------------------------------------------------ flexible CG acceleration (krylov = 1)
def _room_problem():
    from paper_2603_21869_gb300 import cases
    from oracle.step import OracleCase
    spec = cases.room_3d(64, 32, 32, seed=3, mg_levels=4, h=0.08)
    mg = OracleCase(spec).mg
    lev = mg.levels[0]
    b = np.where(lev.fluid, np.random.default_rng(11).normal(size=lev.shape), 0.0)
    return spec, mg, lev, b


def _fluid_operator(lev):
    """A restricted to the fluid cells as a scipy LinearOperator (zero on solid cells)."""
    from scipy.sparse.linalg import LinearOperator
    n = int(np.prod(lev.shape))
    return LinearOperator((n, n), matvec=lambda x: apply_A(lev, x.reshape(lev.shape)).ravel(), dtype=np.float64)


def test_fcg_with_an_exact_preconditioner_solves_in_one_step():
    """With the exact inverse as the preconditioner, d = A^-1 r is the error
    and alpha = (r, d) / (d, A d) = 1: one step lands on the discrete solution."""
    from paper_2603_21869_gb300 import cases
    from oracle.step import OracleCase
    from oracle.poisson import direct_solve
    mg = OracleCase(cases.heated_channel_3d(16, 8, 8, mg_levels=3)).mg   # 1024 cells: a dense solve is cheap
    lev = mg.levels[0]
    b = np.where(lev.fluid, np.random.default_rng(11).normal(size=lev.shape), 0.0)
    mg.vcycle = lambda p, r, l=0: direct_solve(lev, r)
    p, n, rel = mg.fcg_solve(np.zeros(lev.shape), b, 5, 1e-12, 1)
    assert n == 1 and rel <= 1e-11
    assert np.max(np.abs(p - direct_solve(lev, b))) <= 1e-10 * np.max(np.abs(p))


def test_fcg_with_a_fixed_jacobi_preconditioner_is_textbook_pcg():
    """With a fixed symmetric positive definite preconditioner (r / D on
    fluid cells) one kept direction already makes every direction
    A-orthogonal: the iterates are those of preconditioned CG (scipy's cg
    with the same preconditioner, from zero)."""
    from scipy.sparse.linalg import LinearOperator, cg
    spec, mg, lev, b = _room_problem()
    D = lev.diag()
    n = int(np.prod(lev.shape))
    M = LinearOperator((n, n), matvec=lambda x: np.where(lev.fluid, x.reshape(lev.shape) / D, 0.0).ravel(),
                       dtype=np.float64)
    ref = []
    cg(_fluid_operator(lev), b.ravel(), x0=np.zeros(n), M=M, rtol=1e-30, maxiter=12,
       callback=lambda xk: ref.append(xk.reshape(lev.shape).copy()))
    mg.vcycle = lambda p, r, l=0: np.where(lev.fluid, r / D, 0.0)
    for k in (1, 2, 5, 12):
        p, _, _ = mg.fcg_solve(np.zeros(lev.shape), b, 0, 0.0, k)
        assert np.max(np.abs(p - ref[k - 1])) <= 1e-9 * np.max(np.abs(ref[k - 1])), k


def test_fcg_error_energy_never_grows_and_beats_plain_cycles():
    """Each step minimises the A-norm of the error along its direction, so
    that norm is non-increasing (against the solution from scipy's cg to
    1e-13); on the room (a small outlet) it also needs fewer cycles than
    plain V-cycles to the same tolerance."""
    from scipy.sparse.linalg import cg
    spec, mg, lev, b = _room_problem()
    ps, info = cg(_fluid_operator(lev), b.ravel(), x0=np.zeros(b.size), rtol=1e-13, maxiter=5000)
    assert info == 0
    ps = ps.reshape(lev.shape)

    def energy(p):
        e = np.where(lev.fluid, p - ps, 0.0)
        return float(np.sum(e * apply_A(lev, e)))

    last = energy(np.zeros(lev.shape))
    _, n_fcg, rel_fcg = mg.fcg_solve(np.zeros(lev.shape), b, 60, 1e-8, 0)
    for k in range(1, 8):
        p, _, _ = mg.fcg_solve(np.zeros(lev.shape), b, 60, 0.0, k)
        E = energy(p)
        assert E <= last * (1 + 1e-9), k
        last = E
    q = np.zeros(lev.shape)
    n_plain = 0
    while mg.rel_residual(q, b) > 1e-8 and n_plain < 60:
        q = mg.vcycle(q, b)
        n_plain += 1
    assert rel_fcg <= 1e-8 and n_fcg < n_plain


# ------------------------------------------------------------------ per-level sweep counts
def test_coarse_sweeps_change_only_the_coarser_levels_and_keep_the_fixed_point():
    """coarse_sweeps = the finest level's counts is the plain V-cycle exactly; with one sweep
    on the coarser levels the V-cycle still contracts to the discrete solution (a dense
    solve) on a box channel."""
    from paper_2603_21869_gb300 import cases
    from oracle.step import OracleCase
    spec = cases.heated_channel_3d(16, 8, 8, mg_levels=3, boxes=[cases.Box(4, 8, 2, 5, 0, 4)])
    mg = OracleCase(spec).mg
    lev = mg.levels[0]
    b = np.where(lev.fluid, np.random.default_rng(4).normal(size=lev.shape), 0.0)
    p0 = np.zeros(lev.shape)
    same = OracleCase(spec.replace(coarse_sweeps=spec.pre_sweeps)).mg
    assert np.array_equal(mg.vcycle(p0, b), same.vcycle(p0, b))
    one = OracleCase(spec.replace(coarse_sweeps=1)).mg
    assert one.sweeps(0) == (spec.pre_sweeps, spec.post_sweeps) and one.sweeps(1) == (1, 1)
    assert not np.array_equal(mg.vcycle(p0, b), one.vcycle(p0, b))
    p = p0
    for _ in range(30):
        p = one.vcycle(p, b)
    pd = direct_solve(lev, b)
    assert np.max(np.abs(p - pd)) <= 1e-9 * np.max(np.abs(pd))



@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_chebyshev_weights_give_the_scaled_chebyshev_polynomial(n):
    """prod_i (1 - w_i x) equals T_n((hi + lo - 2x)/(hi - lo)) / T_n((hi + lo)/(hi - lo)) (the
    Chebyshev polynomial of [lo, hi] = [1/4, 2] scaled to 1 at 0, its own closed form
    cos(n arccos t) inside the interval) at points spanning the interval; n = 1 is the single
    weight 1 / 1.125."""
    lo, hi = 0.25, 2.0
    w = poisson.chebyshev_weights(n)
    assert len(w) == n and all(np.diff(w) > 0)          # largest root first
    x = np.linspace(lo, hi, 41)
    prod = np.prod([1.0 - wi * x for wi in w], axis=0)
    t = (hi + lo - 2 * x) / (hi - lo)
    tn = np.cos(n * np.arccos(t))
    t0 = (hi + lo) / (hi - lo)
    tn0 = np.cosh(n * np.arccosh(t0))
    assert np.allclose(prod, tn / tn0, rtol=0, atol=1e-14)
    assert np.max(np.abs(prod)) <= 1.0 / tn0 + 1e-14
    if n == 1:
        assert w[0] == pytest.approx(1.0 / 1.125, rel=1e-15)


@pytest.mark.parametrize("smoother", [0, 1])
def test_sweeps_scale_a_neumann_eigenmode_by_the_weight_polynomial(smoother):
    """In a closed box (every face zero-gradient, no solid) the cosine modes are eigenvectors of
    A with eigenvalue sum_d (2 - 2 cos(pi m_d / n_d)) / h_d^2; n sweeps with b = 0 scale such a mode
    by prod_i (1 - w_i lambda / D) with the weights the V-cycle uses (pre order, then post order)."""
    spec = _spec(8, 8, 4, L=(1.0, 1.0, 0.5), outlet_faces=(), smoother=smoother)
    lev = Geometry(spec).levels(1)[0]
    h = np.array(lev.h, dtype=float)
    n = np.array(lev.shape)
    D = float(np.sum(2.0 / h ** 2))
    for m in [(1, 0, 0), (3, 2, 1), (7, 7, 3), (4, 1, 2)]:
        g = np.meshgrid(*[np.cos(np.pi * m[d] * (np.arange(n[d]) + 0.5) / n[d]) for d in range(3)], indexing="ij")
        e = g[0] * g[1] * g[2]
        lam = float(np.sum((2.0 - 2.0 * np.cos(np.pi * np.array(m) / n)) / h ** 2))
        assert np.allclose(apply_A(lev, e), lam * e, atol=1e-9 * lam)
        for post in (False, True):
            w = poisson.sweep_weights(lev, spec, 3, post)
            got = poisson.smooth(lev, e, np.zeros(lev.shape), 3, w)
            want = e * np.prod([1.0 - wi * lam / D for wi in w])
            assert np.max(np.abs(got - want)) <= 1e-12 * max(1.0, np.max(np.abs(want)))
    w0 = poisson.sweep_weights(lev, spec, 2, False)
    if smoother == 0:
        assert w0 == [6.0 / 7.0] * 2
    else:
        assert w0 == poisson.chebyshev_weights(2) and poisson.sweep_weights(lev, spec, 2, True) == w0[::-1]


def test_chebyshev_sweeps_damp_the_high_band_and_never_amplify():
    """On a small room level (solids, an outlet) the eigenvalues x of D^-1 A lie in [0, 2]; the
    Chebyshev sweeps' polynomial is at most 1 in magnitude on all of them and at most
    1 / T_n(9/7) on those at or above 1/4, the band the weights target."""
    spec = _spec(8, 8, 4, L=(1.0, 1.0, 0.5), outlet_faces=(1,), boxes=[cases.Box(2, 4, 2, 5, 0, 2)])
    lev = Geometry(spec).levels(1)[0]
    M = poisson.dense_operator(lev)
    fl = lev.fluid.ravel()
    D = float(np.sum(2.0 / np.array(lev.h, dtype=float) ** 2))
    x = np.linalg.eigvals(M[np.ix_(fl, fl)] / D).real
    assert x.min() > 0.0 and x.max() <= 2.0 + 1e-12
    for n in (2, 3, 4):
        w = poisson.chebyshev_weights(n)
        pol = np.prod([1.0 - wi * x for wi in w], axis=0)
        assert np.max(np.abs(pol)) <= 1.0
        bound = 1.0 / np.cosh(n * np.arccosh(2.25 / 1.75))
        assert np.max(np.abs(pol[x >= 0.25])) <= bound + 1e-12


def test_chebyshev_smoother_keeps_the_fixed_point_and_needs_fewer_cycles():
    """The discrete solution is a fixed point of the V-cycle with either smoother, and on a room
    the flexible-CG solve to 1e-8 needs fewer V(2,2) cycles with the Chebyshev weights."""
    spec = cases.room_3d(32, 16, 16, seed=2, mg_levels=3, h=0.1, precision=cases.FP64, pre_sweeps=2,
                         post_sweeps=2, krylov=1)
    counts = {}
    for sm in (0, 1):
        mg = OracleCase(spec.replace(smoother=sm)).mg
        lev = mg.levels[0]
        b = np.where(lev.fluid, np.random.default_rng(9).normal(size=lev.shape), 0.0)
        pd = direct_solve(lev, b)
        assert np.max(np.abs(mg.vcycle(pd, b) - pd)) <= 1e-10 * np.max(np.abs(pd))
        _, counts[sm], rel = mg.fcg_solve(np.zeros(lev.shape), b, 60, 1e-8, 0)
        assert rel <= 1e-8
    assert counts[1] < counts[0], counts


def test_fcg_restarts_when_the_kept_direction_cancels_the_new_one():
    """With a preconditioner whose directions carry no descent ((r, B r) = 0 for a skew-symmetric
    B) the step length is zero, so the next direction equals the kept one: orthogonalising leaves
    d = 0 and (d, A d) = 0, and the step restarts along z alone (the rule the GPU's flexible-CG
    pass applies) instead of dividing by zero; p stays where it was."""
    spec = _spec(8, 8, 4, L=(1.0, 1.0, 0.5), outlet_faces=(1,))
    mg = Multigrid(Geometry(spec), 2)
    lev = mg.levels[0]
    fl = lev.fluid
    n = int(fl.sum())
    rng = np.random.default_rng(5)
    K = rng.standard_normal((n, n))
    S = 0.01 * (K - K.T)                      # skew-symmetric: (r, S r) = 0

    def skew(p, r):
        out = np.zeros(lev.shape)
        out[fl] = S @ r[fl]
        return out

    mg.vcycle = skew
    b = np.where(fl, rng.standard_normal(lev.shape), 0.0)
    p0 = np.zeros(lev.shape)
    for m in range(1, 5):
        p, cycles, rel = mg.fcg_solve(p0, b, 0, 0.0, m)
        assert cycles == m and np.isfinite(rel)
        assert np.allclose(p, p0, atol=1e-14), m
