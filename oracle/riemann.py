"""Exact Riemann solver for the 1-D Euler equations (perfect gas).

Test infrastructure only. Not part of the paper's method: it is the textbook
closed-form solution (pressure function with Newton iteration for the star
pressure, then sampling of rarefaction / shock / contact waves) used to pin the
shock-tube workload. Written from the Rankine-Hugoniot and isentropic
rarefaction relations.
"""
import numpy as np


def _fk(p, rho, pk, ak, g):
    if p > pk:  # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        s = np.sqrt(A / (p + B))
        return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (p + B))
    pr = p / pk  # rarefaction
    f = 2.0 * ak / (g - 1.0) * (pr ** ((g - 1.0) / (2.0 * g)) - 1.0)
    return f, 1.0 / (rho * ak) * pr ** (-(g + 1.0) / (2.0 * g))


def star_state(L, R, g=1.4):
    rl, ul, pl = L
    rr, ur, pr = R
    al, ar = np.sqrt(g * pl / rl), np.sqrt(g * pr / rr)
    p = 0.5 * (pl + pr)
    for _ in range(100):
        fl, dl = _fk(p, rl, pl, al, g)
        fr, dr = _fk(p, rr, pr, ar, g)
        dp = (fl + fr + ur - ul) / (dl + dr)
        p = max(p - dp, 1e-14)
        if abs(dp) < 1e-15 * p:
            break
    fl, _ = _fk(p, rl, pl, al, g)
    fr, _ = _fk(p, rr, pr, ar, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sample(L, R, xi, g=1.4):
    """Primitive (rho, u, p) at similarity coordinates xi = (x - x0) / t."""
    rl, ul, pl = L
    rr, ur, pr = R
    al, ar = np.sqrt(g * pl / rl), np.sqrt(g * pr / rr)
    ps, us = star_state(L, R, g)
    xi = np.asarray(xi, float)
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    gm = (g - 1.0) / (g + 1.0)
    for n, s in enumerate(xi.flat):
        if s <= us:  # left of contact
            if ps > pl:
                SL = ul - al * np.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
                if s <= SL:
                    r_, u_, p_ = rl, ul, pl
                else:
                    r_, u_, p_ = rl * (ps / pl + gm) / (gm * ps / pl + 1), us, ps
            else:
                ash = al * (ps / pl) ** ((g - 1) / (2 * g))
                if s <= ul - al:
                    r_, u_, p_ = rl, ul, pl
                elif s >= us - ash:
                    r_, u_, p_ = rl * (ps / pl) ** (1 / g), us, ps
                else:
                    c = 2 / (g + 1) + gm / al * (ul - s)
                    r_ = rl * c ** (2 / (g - 1))
                    u_ = 2 / (g + 1) * (al + (g - 1) / 2 * ul + s)
                    p_ = pl * c ** (2 * g / (g - 1))
        else:
            if ps > pr:
                SR = ur + ar * np.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
                if s >= SR:
                    r_, u_, p_ = rr, ur, pr
                else:
                    r_, u_, p_ = rr * (ps / pr + gm) / (gm * ps / pr + 1), us, ps
            else:
                ash = ar * (ps / pr) ** ((g - 1) / (2 * g))
                if s >= ur + ar:
                    r_, u_, p_ = rr, ur, pr
                elif s <= us + ash:
                    r_, u_, p_ = rr * (ps / pr) ** (1 / g), us, ps
                else:
                    c = 2 / (g + 1) - gm / ar * (ur - s)
                    r_ = rr * c ** (2 / (g - 1))
                    u_ = 2 / (g + 1) * (-ar + (g - 1) / 2 * ur + s)
                    p_ = pr * c ** (2 * g / (g - 1))
        rho.flat[n], u.flat[n], p.flat[n] = r_, u_, p_
    return rho, u, p
