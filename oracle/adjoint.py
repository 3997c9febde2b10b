"""Adjoint of the pressure projection: the vector-Jacobian product of
u* -> (u^{n+1}, p) for a differentiable step.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The map (Section 2.4, Algorithm 1, with the projection reading of the step):
    b = -div(u*) / dt          (face velocities L * BC(u*), Eq. pc_residual)
    A p = b                    (solved exactly here, not to a tolerance)
    u^{n+1} = u* - dt G p      (G the cell gradient L * D * BC(p))
is affine in u*: inlet ghosts add constants, everything else is linear.  Its
Jacobian J is therefore one fixed matrix, and the vector-Jacobian product of
a cotangent (ubar, vbar, wbar, pbar) is J^T applied to it.

J is built from the forward oracle functions by the definition.  The three
local pieces (b(u*), the gradient term of the projection, A) reach only the
cells within one index of a cell along each axis, so evaluating each piece
on 27 probe fields -- all cells with (i mod 3, j mod 3, k mod 3) equal to one
colour set to 1 -- recovers every matrix entry exactly: an output cell sees
exactly one probed cell within its reach (Curtis, Powell and Reid, 1974).
A^{-1} is a sparse direct solve on the fluid cells (solid cells hold p = 0).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .poisson import apply_A, poisson_rhs, project


def local_jacobian(apply, n_in, shape):
    """Matrix of the affine map `apply` (a list of n_in arrays of `shape` -> a
    list of arrays of `shape`) whose outputs depend only on inputs within one
    index along each axis.  Rows and columns are field-major, each field in
    numpy C order.  The matrix is checked against the map on a random input."""
    N = int(np.prod(shape))
    zero = [np.zeros(shape) for _ in range(n_in)]
    y0 = apply(zero)
    n_out = len(y0)
    idx = np.indices(shape)
    rows, cols, vals = [], [], []
    for fi in range(n_in):
        for colour in np.ndindex(3, 3, 3):
            mask = np.ones(shape, dtype=bool)
            for a in range(3):
                mask &= (idx[a] % 3) == colour[a]
            if not mask.any():
                continue
            x = [np.zeros(shape) for _ in range(n_in)]
            x[fi][mask] = 1.0
            y = apply(x)
            # for every output cell, the probed cell within its reach: along each
            # axis the index among (q - 1, q, q + 1) with the colour's residue
            src = []
            ok = np.ones(shape, dtype=bool)
            for a in range(3):
                q = idx[a]
                s = q - 1 + ((colour[a] - (q - 1)) % 3)
                ok &= (s >= 0) & (s < shape[a])
                src.append(np.clip(s, 0, shape[a] - 1))
            src_flat = np.ravel_multi_index(src, shape)
            for fo in range(n_out):
                d = y[fo] - y0[fo]
                nz = (d != 0.0)
                assert not (nz & ~ok).any(), "output outside the reach of its probe"
                r = np.flatnonzero(nz)
                rows.append(fo * N + r)
                cols.append(fi * N + src_flat.ravel()[r])
                vals.append(d.ravel()[r])
    J = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n_out * N, n_in * N))
    rng = np.random.default_rng(12345)
    x = [rng.standard_normal(shape) for _ in range(n_in)]
    want = np.concatenate([(a - b).ravel() for a, b in zip(apply(x), y0)])
    got = J @ np.concatenate([a.ravel() for a in x])
    assert np.allclose(got, want, rtol=1e-12, atol=1e-12 * np.max(np.abs(want))), "Jacobian check"
    return J


class ProjectionAdjoint:
    """J^T of u* -> (u^{n+1}, v^{n+1}, w^{n+1}, p) on one case's level-0 grid."""

    def __init__(self, geo, lev0, dt):
        shape = geo.shape
        self.shape = shape
        self.N = N = int(np.prod(shape))
        self.JB = local_jacobian(lambda x: [poisson_rhs(geo, x[0], x[1], x[2], dt)], 3, shape)
        z = np.zeros(shape)
        self.JPp = local_jacobian(lambda x: project(geo, lev0, z, z, z, x[0], dt), 1, shape)
        self.JPu = local_jacobian(lambda x: project(geo, lev0, x[0], x[1], x[2], z, dt), 3, shape)
        A = local_jacobian(lambda x: [apply_A(lev0, x[0])], 1, shape)
        self.fluid = np.flatnonzero(lev0.fluid.ravel())
        self.AFF = A[self.fluid][:, self.fluid].tocsc()
        self._luT = spla.splu(self.AFF.T.tocsc())
        self._lu = spla.splu(self.AFF)

    def _solve(self, b, transpose=False):
        out = np.zeros(self.N)
        lu = self._luT if transpose else self._lu
        out[self.fluid] = lu.solve(b[self.fluid])
        return out

    def forward_linear(self, du, dv, dw):
        """J applied to a velocity perturbation: (du', dv', dw', dp)."""
        x = np.concatenate([a.ravel() for a in (du, dv, dw)])
        dp = self._solve(self.JB @ x)
        y = self.JPu @ x + self.JPp @ dp
        N = self.N
        return [y[i * N:(i + 1) * N].reshape(self.shape) for i in range(3)] + [dp.reshape(self.shape)]

    def vjp(self, ubar, vbar, wbar, pbar=None):
        """J^T (ubar, vbar, wbar, pbar): the cotangent of u*, v*, w*."""
        ybar = np.concatenate([a.ravel() for a in (ubar, vbar, wbar)])
        q = self.JPp.T @ ybar
        if pbar is not None:
            q = q + pbar.ravel()
        xbar = self.JPu.T @ ybar + self.JB.T @ self._solve(q, transpose=True)
        N = self.N
        return [xbar[i * N:(i + 1) * N].reshape(self.shape) for i in range(3)]
