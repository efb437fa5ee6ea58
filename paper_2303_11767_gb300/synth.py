"""Seeded synthetic initial fields on the sphere.

This module is the one input generator that both the CUDA path's tests and
benchmark and the CPU oracle's tests use.  It holds none of the DG method's
arithmetic: it only evaluates a smooth analytic field at points the caller
supplies.  The paper's own workloads are Williamson test cases whose formulas
are not part of this project; these seeded fields stand in for them with the
same character (a deep layer of about 6 km with a smooth 200 m perturbation
and a smooth flow of at most 20 m/s):

* depth  h = 5960 m + 200 m * Y, with Y a random combination of real
  orthonormal spherical harmonics Y_lm of degree 1 <= l <= 4 (coefficients
  N(0, 1) from splitmix64 + Box-Muller), scaled so that max |Y| = 1 on a
  0.25 degree sample grid (l = 0 is left out so that the mean depth stays);
* velocity from a random stream function psi of the same family,
  u = -(1/R) dpsi/dtheta,  v = 1/(R cos theta) dpsi/dlambda, scaled so that
  max sqrt(u^2 + v^2) = 20 m/s on the sample grid (finite at the poles since
  Y_lm carries cos^|m| theta);
* momenta hu = h u and hv = h v pointwise.

theta is latitude in [-pi/2, pi/2], lambda longitude in [0, 2 pi].
"""
from __future__ import annotations

import math

import numpy as np

H0 = 5960.0
H_AMP = 200.0
U_MAX = 20.0
LMAX = 4
EARTH_RADIUS = 6.37122e6

_MASK64 = (1 << 64) - 1


def splitmix64(seed: int):
    """splitmix64 (Steele, Lea & Flood 2014) as an infinite generator of
    64-bit integers."""
    state = seed & _MASK64
    while True:
        state = (state + 0x9E3779B97F4A7C15) & _MASK64
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        yield z ^ (z >> 31)


def normals(seed: int, count: int) -> np.ndarray:
    """count N(0, 1) draws by Box-Muller from splitmix64 uniforms in (0, 1)."""
    gen = splitmix64(seed)
    out = []
    while len(out) < count:
        u1 = ((next(gen) >> 11) + 0.5) * 2.0 ** -53
        u2 = ((next(gen) >> 11) + 0.5) * 2.0 ** -53
        r = math.sqrt(-2.0 * math.log(u1))
        out.append(r * math.cos(2.0 * math.pi * u2))
        out.append(r * math.sin(2.0 * math.pi * u2))
    return np.array(out[:count])


def _modes():
    return [(l, m) for l in range(1, LMAX + 1) for m in range(-l, l + 1)]


def _assoc(l: int, m: int):
    """Q(x) = d^m P_l / dx^m and Q'(x) as numpy polynomials; the associated
    Legendre function is P_l^m(sin th) = cos^m th * Q(sin th)."""
    q = np.polynomial.legendre.Legendre.basis(l).deriv(m) if m > 0 else np.polynomial.legendre.Legendre.basis(l)
    return q, q.deriv(1)


def _norm(l: int, m: int) -> float:
    n = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - m) / math.factorial(l + m))
    return n if m == 0 else math.sqrt(2.0) * n


class _Harmonic:
    """sum_lm c_lm Y_lm(lambda, theta) with its derivatives in theta and
    (1/cos theta) d/dlambda, all finite at the poles."""

    def __init__(self, coeffs: np.ndarray):
        self.terms = []
        for c, (l, m) in zip(coeffs, _modes()):
            am = abs(m)
            q, dq = _assoc(l, am)
            self.terms.append((c * _norm(l, am), m, am, q, dq))

    def eval_grid(self, lam1, th1):
        """Values and derivatives on the tensor grid th1 x lam1 (rows: theta),
        evaluated as a sum of separable theta-part x lambda-part products."""
        s, c = np.sin(th1), np.cos(th1)
        A = []   # theta parts: value, d/dth, (for d/dlam)/cos
        B = []   # lambda parts: trig, dtrig
        for coef, m, am, q, dq in self.terms:
            qs, dqs = q(s), dq(s)
            d = c ** (am + 1) * dqs
            if am > 0:
                d = d - am * c ** (am - 1) * s * qs
            o = c ** (am - 1) * qs if am > 0 else np.zeros_like(s)
            A.append((coef * c ** am * qs, coef * d, coef * o))
            trig = np.cos(am * lam1) if m >= 0 else np.sin(am * lam1)
            dtrig = -am * np.sin(am * lam1) if m >= 0 else am * np.cos(am * lam1)
            B.append((trig, dtrig))
        val = sum(np.outer(a[0], b[0]) for a, b in zip(A, B))
        dth = sum(np.outer(a[1], b[0]) for a, b in zip(A, B))
        dl = sum(np.outer(a[2], b[1]) for a, b in zip(A, B))
        return val, dth, dl

    def eval(self, lam, th):
        lam = np.asarray(lam, dtype=np.float64)
        th = np.asarray(th, dtype=np.float64)
        s, c = np.sin(th), np.cos(th)
        val = np.zeros(np.broadcast(lam, th).shape)
        dth = np.zeros_like(val)
        dlam_over_cos = np.zeros_like(val)
        for coef, m, am, q, dq in self.terms:
            trig = np.cos(am * lam) if m >= 0 else np.sin(am * lam)
            dtrig = -am * np.sin(am * lam) if m >= 0 else am * np.cos(am * lam)
            qs, dqs = q(s), dq(s)
            cm = c ** am
            val += coef * cm * qs * trig
            # d/dth [cos^m th Q(sin th)] = -m cos^(m-1) sin Q + cos^(m+1) Q'
            d = c ** (am + 1) * dqs
            if am > 0:
                d = d - am * c ** (am - 1) * s * qs
            dth += coef * d * trig
            if am > 0:
                dlam_over_cos += coef * c ** (am - 1) * qs * dtrig
        return val, dth, dlam_over_cos


def _sample_grid():
    """The 0.25 degree sample grid (1-D axes: lambda, theta)."""
    lam = np.arange(1440) * (2.0 * math.pi / 1440)
    th = np.linspace(-0.5 * math.pi, 0.5 * math.pi, 721)
    return lam, th


class SmoothField:
    """The seeded smooth field of one member (seed) on a sphere of radius R."""

    def __init__(self, seed: int, radius: float = EARTH_RADIUS):
        self.seed = int(seed)
        self.radius = float(radius)
        nm = len(_modes())
        draws = normals(self.seed, 2 * nm)
        self._h = _Harmonic(draws[:nm])
        self._psi = _Harmonic(draws[nm:])
        lam, th = _sample_grid()
        y, _, _ = self._h.eval_grid(lam, th)
        self._hscale = H_AMP / np.max(np.abs(y))
        _, dth, dl = self._psi.eval_grid(lam, th)
        speed = np.sqrt(dth ** 2 + dl ** 2) / self.radius
        self._uscale = U_MAX / np.max(speed)

    def depth(self, lam, th):
        y, _, _ = self._h.eval(lam, th)
        return H0 + self._hscale * y

    def velocity(self, lam, th):
        _, dth, dl = self._psi.eval(lam, th)
        u = -self._uscale * dth / self.radius
        v = self._uscale * dl / self.radius
        return u, v

    def fields_grid(self, lam1, th1):
        """(h, hu, hv) on the tensor grid th1 x lam1, each shaped
        [len(th1), len(lam1)]."""
        y, _, _ = self._h.eval_grid(lam1, th1)
        h = H0 + self._hscale * y
        _, dth, dl = self._psi.eval_grid(lam1, th1)
        u = -self._uscale * dth / self.radius
        v = self._uscale * dl / self.radius
        return h, h * u, h * v

    def fields(self, lam, th):
        """(h, hu, hv) at the given points."""
        h = self.depth(lam, th)
        u, v = self.velocity(lam, th)
        return h, h * u, h * v


def geostrophic_adjustment_grid(L=1.0e7, h0=1000.0, h1=5.0, sigma_frac=1.0 / 20.0):
    """Initial fields of the planar geostrophic adjustment set-up of the paper
    (Sec. 4.3): a Gaussian hump h0 + h1 exp(-r^2 / (2 sigma^2)) centred in
    [0, L]^2 with sigma = L sigma_frac, fluid at rest.  Returns fn(x1, y1) ->
    (h, hu, hv) on the tensor grid y1 x x1."""
    sigma = sigma_frac * L

    def fn(x1, y1):
        x, y = np.meshgrid(np.asarray(x1), np.asarray(y1))
        h = h0 + h1 * np.exp(-((x - L / 2) ** 2 + (y - L / 2) ** 2) / (2 * sigma * sigma))
        return h, np.zeros_like(h), np.zeros_like(h)

    return fn


CONFIG_SEEDS = {"c1": 1, "c2": 2, "c3": 3}


def ensemble_member_seed(k: int) -> int:
    return 1000 + int(k)


def ensemble_members(count: int = 256, seed: int = 4, nlat_range=(20, 180), degrees=(1, 2, 3, 4)):
    """Mesh sizes of a batched ensemble: nlat uniform on the integers of
    nlat_range, nlon = 2 nlat, degree uniform on `degrees` (splitmix64 draws).
    Returns lists (nlon, nlat, degree)."""
    gen = splitmix64(seed)
    lo, hi = nlat_range
    nlon, nlat, deg = [], [], []
    for _ in range(count):
        la = lo + next(gen) % (hi - lo + 1)
        d = degrees[next(gen) % len(degrees)]
        nlat.append(int(la))
        nlon.append(int(2 * la))
        deg.append(int(d))
    return nlon, nlat, deg
