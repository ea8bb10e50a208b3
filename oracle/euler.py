"""2-D Euler physics (oracle). Test infrastructure only.

Sec. 2.1: e = (rho, rho u, rho v, E) (eq. flow_flux), perfect gas
E = p/(gamma-1) + rho |u|^2 / 2 (eq. perfect_gas), p = rho theta (eq. p_T),
fluxes f_x = (rho u, rho u^2 + p, rho u v, u (E + p)),
       f_y = (rho v, rho u v, rho v^2 + p, v (E + p))   (eq. euler 2d equation),
sound speed a = sqrt(gamma p / rho) (eq. snd_sp).
Sec. 5.1: MWSB S = |u| + |v| + a (eq. Flux_der_Euler_2) and proxy
Phi = |u| sqrt(rho / (gamma p)) (local Mach number).
Remark adiabatic: derivatives of E and p by the sum and product rules from those of
rho, rho u, rho v and theta, and the flux divergence formed from them.
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


def product_rule_derivatives(Q, DQ, gamma):
    """Derivatives of e = (rho, rho u, rho v, E) and of p along one direction from those of
    Q = (rho, rho u, rho v, theta), by the sum and product rules applied to p = rho theta
    (eq. p_T) and E = rho theta/(gamma-1) + |rho u|^2/(2 rho) (eq. perfect_gas_T), as the
    no-slip adiabatic wall treatment prescribes (Remark adiabatic):
        dp = theta drho + rho dtheta,
        dE = dp/(gamma-1) + (rho u d(rho u) + rho v d(rho v))/rho - |rho u|^2/(2 rho^2) drho.
    Returns (De, Dp) with De = (drho, d(rho u), d(rho v), dE)."""
    rho, mx, my, th = Q
    drho, dmx, dmy, dth = DQ
    dp = th * drho + rho * dth
    dE = dp / (gamma - 1.0) + (mx * dmx + my * dmy) / rho - 0.5 * (mx * mx + my * my) / (rho * rho) * drho
    return np.stack([drho, dmx, dmy, dE]), dp


def flux_divergence_product(e, theta, ex, px, ey, py):
    """d/dx f_x(e) + d/dy f_y(e) (eq. euler 2d equation) by the sum and product rules from
    the x and y derivatives of rho, rho u, rho v, E (ex, ey) and p (px, py), with u = rho u/rho,
    v = rho v/rho, p = rho theta and du = (d(rho u) - u drho)/rho (Remark adiabatic)."""
    rho, mx, my, E = e
    u, v = mx / rho, my / rho
    p = rho * theta
    ux = (ex[1] - u * ex[0]) / rho  # d/dx u
    vy = (ey[2] - v * ey[0]) / rho  # d/dy v
    return np.stack([
        ex[1] + ey[2],
        (u * ex[1] + mx * ux + px) + (v * ey[1] + mx * vy),
        (u * ex[2] + my * ux) + (v * ey[2] + my * vy + py),
        (E + p) * (ux + vy) + u * (ex[3] + px) + v * (ey[3] + py),
    ])
