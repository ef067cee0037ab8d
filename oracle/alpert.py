"""Hybrid Gauss-trapezoidal correction for log-singular integrands -- oracle side.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The single-layer matrix corrects the trapezoidal rule near each target with
Alpert's hybrid Gauss-trapezoidal quadrature for a logarithmic singularity
(Sec. 3.1; Sec. 3.2, Eq. Mreal-decompose; Sec. 4.1 uses orders 4 and 8).  The
paper gives neither nodes nor weights, so they are derived here from the
defining exactness conditions.

Reading (the paper is silent on the rule's construction): on each side of the
singular point the trapezoidal nodes at offsets 1 .. a-1 are dropped and
replaced by ``j`` auxiliary nodes at offsets v_1..v_j (units of the node
spacing h) with weights w_1..w_j.  With the generalised Euler-Maclaurin
expansion of h * sum_{i>=1} f(ih) for f(x) = x^p and f(x) = x^p log x, the
corrected end rule integrates both families exactly (p = 0..j-1) when

    sum_k w_k v_k^p          = sum_{i=1}^{a-1} i^p - zeta(-p)
    sum_k w_k v_k^p log v_k  = sum_{i=1}^{a-1} i^p log i + zeta'(-p)

so that the first neglected term is O(h^{j+1} log h): order = j + 1.  Order 4
uses (j, a) = (3, 3), order 8 uses (j, a) = (7, 5).

The system is solved by Newton iteration, first in float64 and then polished
in 60-digit decimal arithmetic.  zeta(-p) comes from Bernoulli numbers and
zeta'(-p) from the differentiated Euler-Maclaurin continuation of zeta.

Parity: pinned by closed-form log-singular integrals (tests check the rule's
convergence order and the values -pi/n of the Fourier cosine integrals of
log|2 sin(t/2)|) and by textbook values of zeta'(0), zeta'(-1), zeta'(-2).
"""
from __future__ import annotations

import decimal
from decimal import Decimal
from fractions import Fraction
from functools import lru_cache

import numpy as np

ORDER_TABLE = {4: (3, 3), 8: (7, 5)}
_PREC = 60


def bernoulli(n: int) -> Fraction:
    """B_n with the convention B_1 = -1/2 (explicit double-sum formula)."""
    total = Fraction(0)
    for k in range(n + 1):
        inner = Fraction(0)
        for v in range(k + 1):
            c = 1
            # binomial(k, v)
            for t in range(v):
                c = c * (k - t) // (t + 1)
            inner += Fraction((-1) ** v * c * (v + 1) ** n)
        total += inner / (k + 1)
    # the formula above yields B_1 = +1/2; switch to the B_1 = -1/2 convention
    if n == 1:
        total = -total
    return total


def zeta_neg(p: int) -> Fraction:
    """zeta(-p) for integer p >= 0: (-1)^p B_{p+1} / (p+1)."""
    return Fraction((-1) ** p) * bernoulli(p + 1) / (p + 1)


def _dln(x: Decimal) -> Decimal:
    return x.ln()


@lru_cache(maxsize=None)
def zeta_prime_neg(p: int, n_cut: int = 40, k_terms: int = 24) -> Decimal:
    """zeta'(-p) from the s-derivative of the Euler-Maclaurin form of zeta(s)."""
    with decimal.localcontext() as ctx:
        ctx.prec = _PREC
        s = Decimal(-p)
        N = Decimal(n_cut)
        lnN = _dln(N)
        acc = Decimal(0)
        for n in range(2, n_cut):
            dn = Decimal(n)
            acc -= _dln(dn) * (dn ** p)  # d/ds n^{-s} at s = -p
        Ns = N ** p  # N^{-s}
        acc += N * Ns * (-lnN / (s - 1) - 1 / ((s - 1) ** 2))
        acc += -lnN * Ns / 2
        fact = Decimal(1)
        for k in range(1, k_terms + 1):
            fact *= (2 * k - 1) * (2 * k)
            b = bernoulli(2 * k)
            ck = Decimal(b.numerator) / Decimal(b.denominator) / fact
            factors = [s + i for i in range(2 * k - 1)]
            P = Decimal(1)
            for f in factors:
                P *= f
            dP = Decimal(0)
            for i in range(len(factors)):
                t = Decimal(1)
                for l, f in enumerate(factors):
                    if l != i:
                        t *= f
                dP += t
            pw = Ns / (N ** (2 * k - 1))
            acc += ck * pw * (dP - lnN * P)
        return +acc


def _targets(j: int, a: int):
    m = []
    n = []
    with decimal.localcontext() as ctx:
        ctx.prec = _PREC
        for p in range(j):
            z = zeta_neg(p)
            mp_ = sum(Decimal(i) ** p for i in range(1, a)) - Decimal(z.numerator) / Decimal(z.denominator)
            np_ = sum((Decimal(i) ** p) * Decimal(i).ln() for i in range(2, a)) + zeta_prime_neg(p)
            m.append(+mp_)
            n.append(+np_)
    return m, n


def _residual_f64(z, j, m, n):
    v, w = z[:j], z[j:]
    lv = np.log(v)
    r = np.empty(2 * j)
    J = np.empty((2 * j, 2 * j))
    for p in range(j):
        vp = v ** p
        r[p] = np.sum(w * vp) - m[p]
        r[j + p] = np.sum(w * vp * lv) - n[p]
        dvp = p * v ** (p - 1) if p > 0 else np.zeros_like(v)
        J[p, :j] = w * dvp
        J[p, j:] = vp
        J[j + p, :j] = w * (dvp * lv + vp / v)
        J[j + p, j:] = vp * lv
    return r, J


def _solve_dec(A, b):
    """Gaussian elimination with partial pivoting on lists of Decimals."""
    n = len(b)
    A = [row[:] for row in A]
    b = b[:]
    for c in range(n):
        piv = max(range(c, n), key=lambda r: abs(A[r][c]))
        A[c], A[piv] = A[piv], A[c]
        b[c], b[piv] = b[piv], b[c]
        for r in range(c + 1, n):
            f = A[r][c] / A[c][c]
            for k in range(c, n):
                A[r][k] -= f * A[c][k]
            b[r] -= f * b[c]
    x = [Decimal(0)] * n
    for r in range(n - 1, -1, -1):
        acc = b[r]
        for k in range(r + 1, n):
            acc -= A[r][k] * x[k]
        x[r] = acc / A[r][r]
    return x


@lru_cache(maxsize=None)
def alpert_rule(order: int = 4):
    """Return (v, w, a): auxiliary offsets, weights (float64 arrays) and a."""
    j, a = ORDER_TABLE[order]
    m_dec, n_dec = _targets(j, a)
    m = np.array([float(x) for x in m_dec])
    n = np.array([float(x) for x in n_dec])
    best = None
    # deterministic starting guesses: nodes clustered towards the singularity
    for shape in (2.0, 1.5, 2.5, 3.0, 1.2, 4.0):
        for scale in (1.0, 0.8, 1.2, 0.6):
            v = scale * a * ((np.arange(j) + 0.5) / j) ** shape
            z = np.concatenate([v, np.full(j, (a - 0.5) / j)])
            for _ in range(200):
                r, J = _residual_f64(z, j, m, n)
                try:
                    dz = np.linalg.solve(J, -r)
                except np.linalg.LinAlgError:
                    break
                lam = 1.0
                while lam > 1e-6:
                    zn = z + lam * dz
                    if np.all(zn[:j] > 0):
                        rn, _ = _residual_f64(zn, j, m, n)
                        if np.linalg.norm(rn) < np.linalg.norm(r) or lam < 1e-3:
                            break
                    lam *= 0.5
                z = zn
                if np.linalg.norm(r) < 1e-13:
                    break
            r, _ = _residual_f64(z, j, m, n)
            vv, ww = z[:j], z[j:]
            if (np.linalg.norm(r) < 1e-11 and np.all(vv > 0) and np.all(vv < a + 1)
                    and np.all(ww > 0)):
                best = z
                break
        if best is not None:
            break
    if best is None:
        raise RuntimeError(f"no Alpert rule found for order {order}")
    order_idx = np.argsort(best[:j])
    best = np.concatenate([best[:j][order_idx], best[j:][order_idx]])
    # polish in decimal arithmetic
    with decimal.localcontext() as ctx:
        ctx.prec = _PREC
        zd = [Decimal(repr(float(x))) for x in best]
        for _ in range(8):
            v, w = zd[:j], zd[j:]
            lv = [x.ln() for x in v]
            r = []
            J = []
            for p in range(j):
                r.append(sum(w[k] * v[k] ** p for k in range(j)) - m_dec[p])
                J.append([w[k] * (p * v[k] ** (p - 1) if p > 0 else Decimal(0)) for k in range(j)]
                         + [v[k] ** p for k in range(j)])
            for p in range(j):
                r.append(sum(w[k] * v[k] ** p * lv[k] for k in range(j)) - n_dec[p])
                J.append([w[k] * ((p * v[k] ** (p - 1) if p > 0 else Decimal(0)) * lv[k] + v[k] ** p / v[k])
                          for k in range(j)] + [v[k] ** p * lv[k] for k in range(j)])
            dz = _solve_dec(J, [-x for x in r])
            zd = [zd[i] + dz[i] for i in range(2 * j)]
        res = max(abs(x) for x in r)
        if res > Decimal("1e-40"):
            raise RuntimeError("Alpert rule polish did not converge")
    v = np.array([float(x) for x in zd[:j]])
    w = np.array([float(x) for x in zd[j:]])
    return v, w, a


def lagrange_stencil(t: float, q: int):
    """Offsets and Lagrange weights interpolating at offset t from q nodes.

    The q integer offsets are the ones nearest to t: floor(t) - q/2 + 1 ..
    floor(t) + q/2 (q even), which keeps the stencil mirror-symmetric in t.
    """
    base = int(np.floor(t))
    offs = np.arange(base - q // 2 + 1, base + q // 2 + 1)
    wts = np.ones(q)
    for i in range(q):
        for k in range(q):
            if k != i:
                wts[i] *= (t - offs[k]) / (offs[i] - offs[k])
    return offs, wts


def interp_points(order: int = 4) -> int:
    """Lagrange stencil size used to carry nodal densities to auxiliary nodes."""
    return order + 2


def corrected_periodic_integral(f_smooth_nodes, f_at, n_nodes: int, order: int = 4):
    """Integral over [0, 2 pi) of a kernel with a log singularity at s = 0.

    ``f_at(s)`` evaluates the full integrand at any s != 0 (mod 2 pi) and
    ``f_smooth_nodes`` is unused unless None -- a helper for the rule's own
    tests, where the integrand is known everywhere.
    """
    v, w, a = alpert_rule(order)
    h = 2.0 * np.pi / n_nodes
    idx = np.arange(a, n_nodes - a + 1)
    total = h * np.sum(f_at(idx * h))
    for k in range(len(v)):
        total += h * w[k] * (f_at(v[k] * h) + f_at(-v[k] * h))
    return total
