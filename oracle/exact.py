"""TEST INFRASTRUCTURE — exact-arithmetic mini-oracle (tiny systems only).

Runs Algorithms 3 (ssBiCGSafe2), 4 (p-BiCGSafe) and 5 (p-BiCGSafe-rr) of
Huynh & Suito (arXiv 2108.10591) over Python ``fractions.Fraction``, with the
same readings as the FP64 oracle (s_0 = A r_0 for the pipelined variants,
zero auxiliaries, the i = 0 branch, r0* = r_0, l_i = A t_i in the
replacement step).  In exact arithmetic the stop test sqrt(r_i) <= eps*||r_0||
with eps = 0 is "(r_i, r_i) == 0", so the runs end at exact termination.

What this pins, independently of any floating-point code: BiCG-type finite
termination (the BiCG factor R_n(A) r_0 vanishes, so r_i = 0 at some i <= n)
with x equal to the exact solution, and the Section 3 claim that Alg. 4 is
an equivalent rewrite of Alg. 3 (identical scalars and residuals in exact
arithmetic; Alg. 5 likewise, since its replacements are exact there).
"""
from fractions import Fraction


def _mv(A, v):
    return [sum((a * x for a, x in zip(row, v)), Fraction(0)) for row in A]


def _dot(u, v):
    return sum((a * b for a, b in zip(u, v)), Fraction(0))


def _lin(*terms):
    """sum of coefficient * vector."""
    n = len(terms[0][1])
    out = [Fraction(0)] * n
    for c, v in terms:
        for j in range(n):
            out[j] += c * v[j]
    return out


def solve(A, b, kind="p-BiCGSafe", maxit=50, rr_m=2, rr_M=10**9):
    """A: dense list of lists of Fractions; b: list of Fractions; x_0 = 0.
    Returns dict(x, rr (list of (r_i, r_i)), scalars (alpha, beta, zeta, eta),
    iterations, terminated)."""
    n = len(b)
    Z = [Fraction(0)] * n
    x = list(Z)
    Ax0 = _mv(A, x)
    r = [bi - ai for bi, ai in zip(b, Ax0)]
    rs = list(r)
    y, t, p, u, z, w, l, g = (list(Z) for _ in range(8))
    pipelined = kind != "ssBiCGSafe2"
    rr = kind == "p-BiCGSafe-rr"
    s = _mv(A, r) if pipelined else list(Z)
    hist, scal = [], []
    alpha_p = zeta_p = f_p = None
    for i in range(maxit + 1):
        if pipelined:
            As = _mv(A, s)
        else:
            s = _mv(A, r)
        a, d, f, gg, rrr = _dot(s, s), _dot(s, r), _dot(rs, r), _dot(rs, s), _dot(r, r)
        hist.append(rrr)
        if rrr == 0:
            return dict(x=x, rr=hist, scalars=scal, iterations=i, terminated=True)
        if i == 0:
            beta, alpha, zeta, eta = Fraction(0), f / gg, d / a, Fraction(0)
        else:
            bb, c, e, h = _dot(y, y), _dot(s, y), _dot(y, r), _dot(rs, t)
            beta = (alpha_p * f) / (zeta_p * f_p)
            alpha = f / (gg + beta * h)
            den = a * bb - c * c
            if den == 0:
                zeta, eta = d / a, Fraction(0)
            else:
                zeta = (bb * d - c * e) / den
                eta = (a * e - c * d) / den
        scal.append((alpha, beta, zeta, eta))
        if i == maxit:
            break
        rr_step = rr and i > 0 and i % rr_m == 0 and i < rr_M
        p = _lin((1, r), (beta, p), (-beta, u))
        o = _lin((1, s), (beta, t))
        u = _lin((zeta, o), (eta, y), (eta * beta, u))
        if not pipelined:
            w = _mv(A, u)
        elif rr_step:
            q = _mv(A, o)
            w = _mv(A, u)
        else:
            q = _lin((1, As), (beta, l))
            w = _lin((zeta, q), (eta, g), (eta * beta, w))
        t = _lin((1, o), (-1, w))
        z = _lin((zeta, r), (eta, z), (-alpha, u))
        y_new = _lin((zeta, s), (eta, y), (-alpha, w))
        x = _lin((1, x), (alpha, p), (1, z))
        if rr_step:
            Ax = _mv(A, x)
            r = [bi - ai for bi, ai in zip(b, Ax)]
            l = _mv(A, t)
            y = y_new
            g = _mv(A, y)
            s = _mv(A, r)
        else:
            r = _lin((1, r), (-alpha, o), (-1, y_new))
            y = y_new
            if pipelined:
                Aw = _mv(A, w)
                l = _lin((1, q), (-1, Aw))
                g = _lin((zeta, As), (eta, g), (-alpha, Aw))
                s = _lin((1, s), (-alpha, q), (-1, g))
        alpha_p, zeta_p, f_p = alpha, zeta, f
    return dict(x=x, rr=hist, scalars=scal, iterations=maxit, terminated=False)
