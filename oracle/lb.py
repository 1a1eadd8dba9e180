"""Plain CPU oracle of the multi-relaxation-time lattice Boltzmann equation (Sec. IV).

TEST INFRASTRUCTURE ONLY (same rules as the rest of ``oracle/``).

The Boltzmann average of the over-relaxed lattice gas (Sec. IV) is a linear MRT
lattice Boltzmann scheme: with the moments M^a = sum_i m_i^a f_i of a transform
matrix orthonormal under the weights (sum_i m_i^a w_i m_i^b = delta^ab), the
equilibrium f_i^0 = w_i rho carries only the density, and one time step is

    f_i(x + v_i, t + 1) = f_i^0 + sum_a w_i m_i^a (1 - omega^a) sum_j m_j^a (f_j - f_j^0)

(Sec. IV, Eq. MRTLB, read with f^0 added and the sign of the non-equilibrium part as
in the moment-space collision of Eq. momentspaceOm).  The relaxation rates are
omega^rho (arbitrary: the density is conserved, here 1), omega^j for the current
moments and omega for the remaining (even) moments.  The lattice gas with collision
fraction omega* and the flip has omega^j = 2 - omega*, omega = omega* (Eq. omegaj);
without the flip both equal omega*.

D1Q3 uses the transform matrix the paper prints (Sec. IV, Eq. transform), rows
(rho, j, Pi) over velocities (-1, 0, +1), reordered here to the storage order
(0, +1, -1).  D2Q5 (not in the paper) uses the analogous Hermite basis: 1,
v_x / sqrt(theta), v_y / sqrt(theta), (v^2 - 2 theta) / sqrt(2 theta (1 - 2 theta)),
(v_x^2 - v_y^2) / sqrt(2 theta), the last two relaxing with omega.  D2Q9 (weights the
products of the D1Q3 weights in x and y) uses the products e_a(v_x) e_b(v_y) of the
paper's D1Q3 rows e_0 = 1, e_1 = v / sqrt(theta), e_2 = (v^2 - theta) / sqrt(theta (1 -
theta)); a product is odd in the velocity when a + b is odd.

Everything is plain numpy in double precision, one full matrix product per node,
no fusion.  Pins: ``tests/test_oracle_lb.py``.
"""
from __future__ import annotations

import math

import numpy as np

from . import D1Q3, D2Q5, D2Q9, Lattice, weights

# velocities in storage order (rest first); D2Q5 rows are (v_x, v_y)
_VEL = {D1Q3: np.array([[0], [1], [-1]]), D2Q5: np.array([[0, 0], [1, 0], [-1, 0], [0, 1], [0, -1]]),
        D2Q9: np.array([[0, 0], [1, 0], [-1, 0], [0, 1], [0, -1], [1, 1], [-1, -1], [1, -1], [-1, 1]])}


def velocities(lattice: int) -> np.ndarray:
    return _VEL[lattice].copy()


def basis(lattice: int, theta: float):
    """(m, odd): transform matrix m[a, i] in storage order and, per moment, whether
    it is odd in the velocity (a current) -- odd moments relax with omega^j."""
    if lattice == D1Q3:
        # the paper's matrix over v = (-1, 0, +1)
        r = math.sqrt(1.0 / theta)
        p, q = math.sqrt((1.0 - theta) / theta), math.sqrt(theta / (1.0 - theta))
        paper = np.array([[1.0, 1.0, 1.0],
                          [-r, 0.0, r],
                          [p, -q, p]])
        # storage order (0, +1, -1) = paper columns (1, 2, 0)
        return paper[:, [1, 2, 0]], np.array([False, True, False])
    if lattice == D2Q9:
        v = _VEL[D2Q9].astype(float)
        def e(a, u):
            return [np.ones_like(u), u / math.sqrt(theta), (u * u - theta) / math.sqrt(theta * (1.0 - theta))][a]
        rows, odd = [], []
        for a in range(3):
            for b in range(3):
                rows.append(e(a, v[:, 0]) * e(b, v[:, 1]))
                odd.append((a + b) % 2 == 1)
        return np.array(rows), np.array(odd)
    v = _VEL[D2Q5].astype(float)
    vx, vy = v[:, 0], v[:, 1]
    v2 = vx * vx + vy * vy
    m = np.array([np.ones(5),
                  vx / math.sqrt(theta),
                  vy / math.sqrt(theta),
                  (v2 - 2.0 * theta) / math.sqrt(2.0 * theta * (1.0 - 2.0 * theta)),
                  (vx * vx - vy * vy) / math.sqrt(2.0 * theta)])
    return m, np.array([False, True, True, False, False])


def rates_from_omega_eff(omega_eff: float):
    """(omega^j, omega) of the lattice gas with parameter omega_eff (Sec. III/IV):
    above 1 the flip is on, omega^j = omega_eff and omega = 2 - omega_eff."""
    if omega_eff > 1.0:
        return omega_eff, 2.0 - omega_eff
    return omega_eff, omega_eff


class LB:
    """One periodic lattice of the MRT scheme; state f[i, y, x] (float64)."""

    def __init__(self, lattice, Lx, Ly=1, theta=1.0 / 3.0, omega_j=1.0, omega=1.0):
        self.lattice, self.Lx, self.Ly = lattice, int(Lx), int(Ly if lattice != D1Q3 else 1)
        self.theta, self.omega_j, self.omega = float(theta), float(omega_j), float(omega)
        self.Q = {D1Q3: 3, D2Q5: 5, D2Q9: 9}[lattice]
        self.w = np.array(weights(lattice, self.theta))
        self.m, self.odd = basis(lattice, self.theta)
        # relaxation factor (1 - omega^a) per moment; omega^rho = 1
        lam = np.where(self.odd, 1.0 - self.omega_j, 1.0 - self.omega)
        lam[0] = 0.0
        self.lam = lam
        self.v = velocities(lattice)

    @property
    def shape(self):
        return (self.Q, self.Ly, self.Lx)

    def init_mean(self, **ilg) -> np.ndarray:
        """f_i(x, 0) = lambda_i(x), the mean of the lattice gas's Poisson initial state
        (Sec. V), taken from the integer oracle's own lambda."""
        lat = Lattice(self.lattice, self.Lx, self.Ly, theta=self.theta, **ilg)
        f = np.zeros(self.shape)
        for i in range(self.Q):
            for y in range(self.Ly):
                for x in range(self.Lx):
                    f[i, y, x] = lat.init_lambda(x, y, i)
        return f

    def collide(self, f: np.ndarray) -> np.ndarray:
        """Post-collision distributions of every node (no streaming)."""
        rho = f.sum(axis=0)
        f0 = self.w[:, None, None] * rho[None]
        M = np.einsum("ai,iyx->ayx", self.m, f - f0)                 # non-equilibrium moments
        back = np.einsum("i,ai,a,ayx->iyx", self.w, self.m, self.lam, M)
        return f0 + back

    def stream(self, post: np.ndarray) -> np.ndarray:
        out = np.empty_like(post)
        for i in range(self.Q):
            vx = int(self.v[i, 0])
            vy = int(self.v[i, 1]) if self.lattice != D1Q3 else 0
            out[i] = np.roll(np.roll(post[i], vx, axis=1), vy, axis=0)
        return out

    def step(self, f: np.ndarray) -> np.ndarray:
        return self.stream(self.collide(f))

    def run(self, f: np.ndarray, steps: int) -> np.ndarray:
        for _ in range(steps):
            f = self.step(f)
        return f

    def observables(self, f: np.ndarray, modes):
        """(mass, [(re, im, amp)]) for axis modes (mx, my) (one of them zero): with
        D = C - M / L the column (row) sums less their mean, re = sum cos(2 pi r / L) D,
        im = sum sin(2 pi r / L) D over r = (m x) mod L, and amp = im / (Lx Ly / 2)
        (the measured amplitude of Sec. V).  Sums rounded once (math.fsum)."""
        N = f.sum(axis=0)
        M = math.fsum(N.ravel())
        out = []
        for mx, my in modes:
            if my == 0:
                C, L, m = N.sum(axis=0), self.Lx, mx
            else:
                C, L, m = N.sum(axis=1), self.Ly, my
            re, im = [], []
            for x in range(L):
                r = (m * x) % L
                a = 2.0 * math.pi * r / L
                d = C[x] - M / L
                re.append(math.cos(a) * d)
                im.append(math.sin(a) * d)
            re_s, im_s = math.fsum(re), math.fsum(im)
            out.append((re_s, im_s, im_s / (self.Lx * self.Ly / 2.0)))
        return M, out


def ensemble_prediction(lb: LB, f0: np.ndarray, mode: int, T: int) -> dict:
    """Exact ensemble statistics of the lattice gas's mode amplitude a(t) = re + i im,
    re = sum_x cos(2 pi r / L) N(x), im = sum_x sin(2 pi r / L) N(x) (r = (mode x) mod L,
    D1Q3 ring, mode not a multiple of L), for replicas started from independent
    Poisson occupations with means f0, at t = 0..T.

    Binomial thinning, multinomial redistribution, the flip and streaming map
    independent Poisson occupations to independent Poisson occupations, and the
    conditional mean of one step is the lattice Boltzmann step (Sec. IV).  So at
    every t the occupations are independent Poisson with means f(t) = LB^t f0, and
    Cov(n(t), n(0)) = LB^t diag(f0).  Hence
      <re>, <im>     = projections of rho(t) = sum_i f_i(t)
      Var re, Var im = sum_x cos^2 rho(t), sum_x sin^2 rho(t)
      <da(t) conj(da(0))> = sum_x e(x) [rho_c(x, t) - i rho_s(x, t)],
    with e = cos + i sin and rho_c, rho_s the densities of LB^t (f0 cos), LB^t (f0 sin)."""
    L = lb.Lx
    x = np.arange(L)
    r = (mode * x) % L
    c = np.array([math.cos(2.0 * math.pi * v / L) for v in r])
    s = np.array([math.sin(2.0 * math.pi * v / L) for v in r])
    f, fc, fs = f0.copy(), f0 * c[None, None, :], f0 * s[None, None, :]
    out = {k: np.zeros(T + 1) for k in ("mean_re", "mean_im", "var_re", "var_im", "cov_re", "cov_im")}
    for t in range(T + 1):
        rho, rc, rs = f.sum(axis=0)[0], fc.sum(axis=0)[0], fs.sum(axis=0)[0]
        out["mean_re"][t] = math.fsum(c * rho)
        out["mean_im"][t] = math.fsum(s * rho)
        out["var_re"][t] = math.fsum(c * c * rho)
        out["var_im"][t] = math.fsum(s * s * rho)
        out["cov_re"][t] = math.fsum(np.concatenate([c * rc, s * rs]))
        out["cov_im"][t] = math.fsum(np.concatenate([s * rc, -c * rs]))
        if t < T:
            f, fc, fs = lb.step(f), lb.step(fc), lb.step(fs)
    return out
