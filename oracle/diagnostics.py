"""The lambda_2 vortex criterion of the transient results (Section 3.2.3).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper marks vortex structures by iso-surfaces of lambda_2, the second
largest eigenvalue of the symmetric matrix S^2 + Omega^2 built from the strain
and rotation tensors of the velocity gradient (the criterion of Jeong and
Hussain, 1995); negative values mark vortex cores.  The paper does not say
how the gradient is discretised for it.  The reading used here: the same cell
gradient L_j * D_j * BC_j(u_i) that Algorithm 4 uses for the destruction
terms, so boundary and obstacle cells take their ghost values from
Section 2.7.  Solid cells get 0.
"""
import numpy as np

from . import model
from .geometry import U, V, W, cell_gradient


def s2_plus_omega2(S, O):
    """The matrix M = S S + Omega Omega as nested lists of arrays: M_ij =
    sum_k (S_ik S_kj + Omega_ik Omega_kj)."""
    return [[sum(S[i][k] * S[k][j] + O[i][k] * O[k][j] for k in range(3)) for j in range(3)] for i in range(3)]


def lambda2(geo, u, v, w):
    """lambda_2 at every cell: the middle one of the three (real) eigenvalues
    of S^2 + Omega^2, from the cell velocity gradients of Algorithm 4."""
    grads = [cell_gradient(geo, phi, f) for phi, f in ((u, U), (v, V), (w, W))]
    S, O = model.strain_rotation(grads)
    M = s2_plus_omega2(S, O)
    stacked = np.stack([np.stack(row, axis=-1) for row in M], axis=-2)   # (..., 3, 3)
    ev = np.linalg.eigvalsh(stacked)                                       # ascending
    return np.where(geo.fluid, ev[..., 1], 0.0)
