"""k-omega closure: constants and pointwise formulas (Section 2.1).

Every function works elementwise on float64 numpy arrays.
"""
import numpy as np

# Section 2.1, after Eq. Re_t: alpha*_inf = 1, alpha*_0 = beta_i / 3, R_k = 6
ALPHA_STAR_INF = 1.0
BETA_I = 0.072
ALPHA_STAR_0 = BETA_I / 3.0
R_K = 6.0
# after Eq. a: alpha_inf = 0.52, alpha_0 = 1/9, R_omega = 2.95
ALPHA_INF = 0.52
ALPHA_0 = 1.0 / 9.0
R_OMEGA = 2.95
# after Eq. o_des: beta*_inf = 0.09, beta = beta_i = 0.072
BETA_STAR_INF = 0.09
BETA = BETA_I
# R_beta appears in Eq. beta_star without a value: standard Wilcox value 8
R_BETA = 8.0
# Section 3.2.4: C_mu = 0.09
C_MU = 0.09
# epsilon of max(omega, eps) in Algorithm 4 (no value printed)
EPS_OMEGA = 1e-12
# positivity clamps of the explicit stage (Section A.4; no value printed)
K_MIN = 1e-14
OMEGA_MIN = 1e-8


def omega_safe(om):
    """max(omega, eps) of Algorithm 4."""
    return np.where(np.real(om) > EPS_OMEGA, om, EPS_OMEGA)


def re_t(k, om, nu):
    """Turbulent Reynolds number, Eq. Re_t, with max(omega, eps)."""
    return k / (nu * omega_safe(om))


def alpha_star(k, om, nu):
    """Low-Reynolds damping alpha*, Eq. a_star."""
    r = re_t(k, om, nu) / R_K
    return ALPHA_STAR_INF * (ALPHA_STAR_0 + r) / (1.0 + r)


def nu_t(k, om, nu):
    """Eddy viscosity nu_t = alpha* k / omega, Eq. ko_turb_diff."""
    return alpha_star(k, om, nu) * k / omega_safe(om)


def alpha_coef(k, om, nu):
    """alpha of the omega production, Eq. a."""
    r = re_t(k, om, nu) / R_OMEGA
    return ALPHA_INF / alpha_star(k, om, nu) * (ALPHA_0 + r) / (1.0 + r)


def strain_rotation(grad):
    """S_ij (Eq. strain_rate) and Omega_ij (Eq. rotation_rate) from the
    velocity gradient grad[i][j] = d u_i / d x_j (nested lists of arrays)."""
    S = [[0.5 * (grad[i][j] + grad[j][i]) for j in range(3)] for i in range(3)]
    O = [[0.5 * (grad[i][j] - grad[j][i]) for j in range(3)] for i in range(3)]
    return S, O


def strain_magnitude_sq(S):
    """S^2 with S = sqrt(2 S_ij S_ij), Eq. strain_rate_magnitude."""
    acc = 0.0
    for i in range(3):
        for j in range(3):
            acc = acc + S[i][j] * S[i][j]
    return 2.0 * acc


def production_k(k, om, nu, S2):
    """G_k = nu_t S^2, Eq. k_gen."""
    return nu_t(k, om, nu) * S2


def production_omega(k, om, nu, S2):
    """G_omega = alpha (omega / k) G_k, Eq. o_gen."""
    return alpha_coef(k, om, nu) * om / k * production_k(k, om, nu, S2)


def beta_star(k, om, nu):
    """beta* of Eq. beta_star."""
    x4 = (re_t(k, om, nu) / R_BETA) ** 4
    return BETA_STAR_INF * (4.0 / 15.0 + x4) / (1.0 + x4)


def f_beta_star(chi_k):
    """f_beta* of Eq. k_des: 1 for chi_k <= 0, (1 + 680 chi^2)/(1 + 400 chi^2) otherwise."""
    return np.where(chi_k <= 0.0, 1.0, (1.0 + 680.0 * chi_k ** 2) / (1.0 + 400.0 * chi_k ** 2))


def chi_k(grad_k, grad_om, om):
    """chi_k = (dk/dx_j domega/dx_j) / omega^3 (Eq. k_des, Algorithm 4 with max(omega, eps))."""
    dot = grad_k[0] * grad_om[0] + grad_k[1] * grad_om[1] + grad_k[2] * grad_om[2]
    return dot / omega_safe(om) ** 3


def chi_omega(S, O, om):
    """chi_omega = |Omega_ij Omega_jk S_ki / (beta*_inf omega)^3| (Eq. o_des)."""
    acc = 0.0
    for i in range(3):
        for j in range(3):
            for kk in range(3):
                acc = acc + O[i][j] * O[j][kk] * S[kk][i]
    return np.abs(acc / (BETA_STAR_INF * omega_safe(om)) ** 3)


def f_beta(chi_w):
    """f_beta = (1 + 70 chi_omega)/(1 + 80 chi_omega), Eq. o_des."""
    return (1.0 + 70.0 * chi_w) / (1.0 + 80.0 * chi_w)


def inlet_turbulence(U, intensity, length_scale):
    """Inlet k0 and omega0 (Section 3.2.4): k0 = 1.5 (I0 u0)^2,
    eps0 = k0^1.5 / l0, omega0 = eps0 / (C_mu k0)."""
    k0 = 1.5 * (intensity * U) ** 2
    eps0 = k0 ** 1.5 / length_scale
    om0 = eps0 / (C_MU * k0)
    return k0, om0


def omega_wall(nu, d):
    """Near-wall omega = 6 nu / (beta_i d^2), d = centroid-to-wall distance (Section 2.7)."""
    return 6.0 * nu / (BETA_I * d * d)
