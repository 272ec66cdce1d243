"""Exact solution of the Riemann problem of the 1-D Euler equations for an
ideal gas (the textbook two-rarefaction / two-shock construction with a
Newton iteration for the star pressure, as in Toro, "Riemann Solvers and
Numerical Methods for Fluid Dynamics", ch. 4).  Used only by the tests, as
the Kn -> 0 limit of the particle solution of the Sod problem."""
import math

import numpy as np


def _f(p, rho, pk, g):
    a = math.sqrt(g * pk / rho)
    if p > pk:  # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        s = math.sqrt(A / (p + B))
        return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (p + B))
    # rarefaction
    r = (p / pk) ** ((g - 1.0) / (2.0 * g))
    return 2.0 * a / (g - 1.0) * (r - 1.0), 1.0 / (rho * a) * (p / pk) ** (-(g + 1.0) / (2.0 * g))


def star(L, R, g):
    rl, ul, pl = L
    rr, ur, pr = R
    p = 0.5 * (pl + pr)
    for _ in range(100):
        fl, dl = _f(p, rl, pl, g)
        fr, dr = _f(p, rr, pr, g)
        dp = (fl + fr + ur - ul) / (dl + dr)
        p = max(1e-12, p - dp)
        if abs(dp) < 1e-15 * p:
            break
    fl, _ = _f(p, rl, pl, g)
    fr, _ = _f(p, rr, pr, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sample(L, R, g, xi):
    """Primitive state (rho, u, p) at similarity coordinate xi = x/t."""
    rl, ul, pl = L
    rr, ur, pr = R
    ps, us = star(L, R, g)
    al, ar = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    out = np.zeros((3, len(xi)))
    for i, s in enumerate(xi):
        if s <= us:  # left of contact
            if ps > pl:
                rs = rl * ((ps / pl + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pl + 1))
                S = ul - al * math.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
                out[:, i] = (rl, ul, pl) if s < S else (rs, us, ps)
            else:
                rs = rl * (ps / pl) ** (1 / g)
                ast = al * (ps / pl) ** ((g - 1) / (2 * g))
                if s < ul - al:
                    out[:, i] = (rl, ul, pl)
                elif s > us - ast:
                    out[:, i] = (rs, us, ps)
                else:
                    u = 2 / (g + 1) * (al + (g - 1) / 2 * ul + s)
                    c = 2 / (g + 1) * (al + (g - 1) / 2 * (ul - s))
                    rho = rl * (c / al) ** (2 / (g - 1))
                    out[:, i] = (rho, u, pl * (c / al) ** (2 * g / (g - 1)))
        else:  # right of contact
            if ps > pr:
                rs = rr * ((ps / pr + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pr + 1))
                S = ur + ar * math.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
                out[:, i] = (rr, ur, pr) if s > S else (rs, us, ps)
            else:
                rs = rr * (ps / pr) ** (1 / g)
                ast = ar * (ps / pr) ** ((g - 1) / (2 * g))
                if s > ur + ar:
                    out[:, i] = (rr, ur, pr)
                elif s < us + ast:
                    out[:, i] = (rs, us, ps)
                else:
                    u = 2 / (g + 1) * (-ar + (g - 1) / 2 * ur + s)
                    c = 2 / (g + 1) * (ar - (g - 1) / 2 * (ur - s))
                    rho = rr * (c / ar) ** (2 / (g - 1))
                    out[:, i] = (rho, u, pr * (c / ar) ** (2 * g / (g - 1)))
    return out
