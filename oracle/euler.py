"""2-D Euler physics (oracle). Test infrastructure only.

Sec. 2.1: e = (rho, rho u, rho v, E) (eq. flow_flux), perfect gas
E = p/(gamma-1) + rho |u|^2 / 2 (eq. perfect_gas), p = rho theta (eq. p_T),
fluxes f_x = (rho u, rho u^2 + p, rho u v, u (E + p)),
       f_y = (rho v, rho u v, rho v^2 + p, v (E + p))   (eq. euler 2d equation),
sound speed a = sqrt(gamma p / rho) (eq. snd_sp).
Sec. 5.1: MWSB S = |u| + |v| + a (eq. Flux_der_Euler_2) and proxy
Phi = |u| sqrt(rho / (gamma p)) (local Mach number).
"""
import numpy as np


def primitives(e, gamma):
    rho = e[0]
    u = e[1] / rho
    v = e[2] / rho
    p = (gamma - 1.0) * (e[3] - 0.5 * rho * (u * u + v * v))
    return rho, u, v, p


def cons_from_prim(rho, u, v, p, gamma):
    return np.stack([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)])


def flux_x(e, gamma):
    rho, u, v, p = primitives(e, gamma)
    return np.stack([e[1], e[1] * u + p, e[1] * v, u * (e[3] + p)])


def flux_y(e, gamma):
    rho, u, v, p = primitives(e, gamma)
    return np.stack([e[2], e[2] * u, e[2] * v + p, v * (e[3] + p)])


def sound_speed(e, gamma):
    rho, u, v, p = primitives(e, gamma)
    return np.sqrt(gamma * p / rho)


def mwsb(e, gamma):
    """S = |u| + |v| + a (Sec. 5.1 item 3, eq. Flux_der_Euler_2)."""
    rho, u, v, p = primitives(e, gamma)
    return np.abs(u) + np.abs(v) + np.sqrt(gamma * p / rho)


def proxy_mach(e, gamma):
    """Phi = |u| sqrt(rho / (gamma p)) (Sec. 5.1)."""
    rho, u, v, p = primitives(e, gamma)
    return np.sqrt(u * u + v * v) * np.sqrt(rho / (gamma * p))


def temperature(e, gamma):
    """theta = p / rho (eq. p_T)."""
    rho, u, v, p = primitives(e, gamma)
    return p / rho


def energy_from_theta(rho, mu_, mv_, theta, gamma):
    """E = rho theta/(gamma-1) + |rho u|^2/(2 rho) (eq. perfect_gas_T)."""
    return rho * theta / (gamma - 1.0) + 0.5 * (mu_ * mu_ + mv_ * mv_) / rho
