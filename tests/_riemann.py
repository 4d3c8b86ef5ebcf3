"""Exact solution of the 1D Riemann problem of the Euler equations for an
ideal gas (the textbook construction: the star-region pressure is the root of
f_L(p) + f_R(p) + u_R - u_L = 0, where f_K is the velocity change across a
shock (Rankine-Hugoniot) or a rarefaction (Riemann invariant), solved by
Newton's method; the solution is then sampled along x/t).  Test
infrastructure: the reference for the Sod problem of Sec. 4."""
import math

import numpy as np


class Riemann:
    def __init__(self, left, right, gamma=1.4):
        self.g = gamma
        self.rl, self.ul, self.pl = left
        self.rr, self.ur, self.pr = right
        self.cl = math.sqrt(gamma * self.pl / self.rl)
        self.cr = math.sqrt(gamma * self.pr / self.rr)
        self.p_star, self.u_star = self._star()

    def _f(self, p, rk, pk, ck):
        g = self.g
        if p > pk:  # shock
            a = 2.0 / ((g + 1.0) * rk)
            b = (g - 1.0) / (g + 1.0) * pk
            q = math.sqrt(a / (p + b))
            return (p - pk) * q, q * (1.0 - 0.5 * (p - pk) / (p + b))
        # rarefaction
        e = (g - 1.0) / (2.0 * g)
        return 2.0 * ck / (g - 1.0) * ((p / pk) ** e - 1.0), (p / pk) ** (-(g + 1.0) / (2.0 * g)) / (rk * ck)

    def _star(self):
        p = max(1e-12, 0.5 * (self.pl + self.pr))
        for _ in range(100):
            fl, dl = self._f(p, self.rl, self.pl, self.cl)
            fr, dr = self._f(p, self.rr, self.pr, self.cr)
            step = (fl + fr + self.ur - self.ul) / (dl + dr)
            p_new = max(1e-12, p - step)
            if abs(p_new - p) <= 1e-15 * (p_new + p):
                p = p_new
                break
            p = p_new
        fl, _ = self._f(p, self.rl, self.pl, self.cl)
        fr, _ = self._f(p, self.rr, self.pr, self.cr)
        return p, 0.5 * (self.ul + self.ur) + 0.5 * (fr - fl)

    def star_densities(self):
        """densities left and right of the contact"""
        return self._rho_star(self.rl, self.pl), self._rho_star(self.rr, self.pr)

    def _rho_star(self, rk, pk):
        g, ps = self.g, self.p_star
        if ps > pk:
            r = ps / pk
            gm = (g - 1.0) / (g + 1.0)
            return rk * (r + gm) / (gm * r + 1.0)
        return rk * (ps / pk) ** (1.0 / g)

    def shock_speed(self, side):
        """speed of the shock on the given side (+1 right, -1 left)"""
        g = self.g
        if side > 0:
            return self.ur + self.cr * math.sqrt((g + 1.0) / (2.0 * g) * self.p_star / self.pr + (g - 1.0) / (2.0 * g))
        return self.ul - self.cl * math.sqrt((g + 1.0) / (2.0 * g) * self.p_star / self.pl + (g - 1.0) / (2.0 * g))

    def sample(self, s):
        """(rho, u, p) at x/t = s"""
        g = self.g
        ps, us = self.p_star, self.u_star
        if s <= us:  # left of the contact
            rk, uk, pk, ck, sign = self.rl, self.ul, self.pl, self.cl, -1.0
        else:
            rk, uk, pk, ck, sign = self.rr, self.ur, self.pr, self.cr, 1.0
        if ps > pk:  # shock on this side
            sk = self.shock_speed(sign)
            if (sign < 0 and s <= sk) or (sign > 0 and s >= sk):
                return rk, uk, pk
            return self._rho_star(rk, pk), us, ps
        # rarefaction on this side
        c_star = ck * (ps / pk) ** ((g - 1.0) / (2.0 * g))
        head = uk + sign * ck
        tail = us + sign * c_star
        if (sign < 0 and s <= head) or (sign > 0 and s >= head):
            return rk, uk, pk
        if (sign < 0 and s >= tail) or (sign > 0 and s <= tail):
            return self._rho_star(rk, pk), us, ps
        # inside the fan
        c = 2.0 / (g + 1.0) * (ck - sign * (g - 1.0) / 2.0 * (uk - s))
        u = 2.0 / (g + 1.0) * (-sign * ck + (g - 1.0) / 2.0 * uk + s)
        rho = rk * (c / ck) ** (2.0 / (g - 1.0))
        p = pk * (c / ck) ** (2.0 * g / (g - 1.0))
        return rho, u, p

    def cell_averages(self, edges, t, x0, sub=400):
        """averages of rho, rho u and E over the cells [edges[i], edges[i+1]]
        at time t for a discontinuity initially at x0 (midpoint rule with
        `sub` points per cell)"""
        g = self.g
        out = np.zeros((3, len(edges) - 1))
        for i in range(len(edges) - 1):
            xs = edges[i] + (np.arange(sub) + 0.5) * (edges[i + 1] - edges[i]) / sub
            acc = np.zeros(3)
            for x in xs:
                r, u, p = self.sample((x - x0) / t)
                acc += (r, r * u, p / (g - 1.0) + 0.5 * r * u * u)
            out[:, i] = acc / sub
        return out
