"""Semi-implicit destruction of k and omega (Section 2.5, Algorithm 4).

The destruction terms Y_k = beta* f_beta* k omega and Y_omega = beta f_beta
omega^2 (Eqs. k_des, o_des) are advanced by the semi-implicit Euler step of
Eqs. k_des_step / o_des_step:

    k1 = k / (1 + dt beta* f_beta* omega),   omega1 = omega / (1 + dt beta f_beta omega)

Both updates use the omega from before the update.  Cell gradients follow
Algorithm 4: D_j * BC_j(phi) on faces, then L_j back to cells.
"""
import numpy as np

from . import model
from .geometry import U, V, W, K, OM, cell_gradient


def destruction_step(geo, u, v, w, k, om, dt):
    """Advance k and omega by the destruction terms over `dt`.

    Returns new (k, omega); solid cells keep their values."""
    nu = geo.spec.nu
    grads = [cell_gradient(geo, phi, f) for phi, f in ((u, U), (v, V), (w, W))]
    gk = cell_gradient(geo, k, K)
    gw = cell_gradient(geo, om, OM)
    S, O = model.strain_rotation(grads)
    chik = model.chi_k(gk, gw, om)
    fbs = model.f_beta_star(chik)
    bs = model.beta_star(k, om, nu)
    k_new = k / (1.0 + dt * bs * fbs * om)
    chiw = model.chi_omega(S, O, om)
    fb = model.f_beta(chiw)
    om_new = om / (1.0 + dt * model.BETA * fb * om)
    fluid = geo.fluid
    return np.where(fluid, k_new, k), np.where(fluid, om_new, om)
