"""Seeded problem definitions (coefficients, sources, boundary data, exact
solutions) for the HPS workloads.

The operator is L u = a(x) Lap u + b(x) . grad u + c(x) u on a box (Section 1
of the paper, the elliptic boundary value problem).  Boundary data is either
Dirichlet values (DtN variant) or incoming impedance data u_n + i eta u
(ItI variant, Section 2, definition of the impedance maps).

Each factory returns a :class:`Problem` whose callables take an ``(m, d)``
array of points.  Derivatives of the manufactured solutions are written out
in closed form.
"""

from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np


def box_normals(xb: np.ndarray, lo, hi, tol: float = 1e-12) -> np.ndarray:
    """Outward unit normals at points lying on the faces of the box [lo, hi].

    Boundary Gauss points never sit on an edge or corner, so exactly one
    coordinate matches a face."""
    xb = np.atleast_2d(xb)
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    n = np.zeros_like(xb)
    scale = np.maximum(hi - lo, 1.0)
    for k in range(xb.shape[1]):
        n[np.abs(xb[:, k] - lo[k]) <= tol * scale[k], k] = -1.0
        n[np.abs(xb[:, k] - hi[k]) <= tol * scale[k], k] = 1.0
    if not np.all(np.abs(n).sum(axis=1) == 1):
        raise ValueError("a point is not on exactly one face of the box")
    return n


@dataclass
class Problem:
    name: str
    dim: int
    lo: tuple
    hi: tuple
    kind: str  # "dtn" or "iti"
    seed: Optional[int]
    coeffs: Callable[[np.ndarray], dict]
    source: Callable[[np.ndarray], np.ndarray]
    boundary: Callable[[np.ndarray], np.ndarray]
    u_exact: Optional[Callable[[np.ndarray], np.ndarray]] = None
    eta: Optional[float] = None
    info: dict = field(default_factory=dict)

    @property
    def complex(self) -> bool:
        return self.kind == "iti"

    def coefficient_arrays(self, x: np.ndarray, n_leaves: int, npl: int):
        """Coefficients sampled at leaf nodes, each shaped (n_leaves, npl)."""
        c = self.coeffs(x)
        out = {"a": c["a"].reshape(n_leaves, npl),
               "b": [bk.reshape(n_leaves, npl) for bk in c["b"]],
               "c": c["c"].reshape(n_leaves, npl)}
        return out


# ---------------------------------------------------------------------------
# polynomial fields with derivatives
# ---------------------------------------------------------------------------

class PolyField:
    """u(x) = sum_k c_k prod_j x_j^{e_kj} with its gradient and Laplacian."""

    def __init__(self, exps: np.ndarray, coef: np.ndarray):
        self.exps = np.asarray(exps, int)
        self.coef = np.asarray(coef, float)

    @staticmethod
    def _mono(x, e):
        out = np.ones(x.shape[0])
        for j, ej in enumerate(e):
            if ej:
                out = out * x[:, j] ** ej
        return out

    def value(self, x):
        x = np.atleast_2d(x)
        return sum(c * self._mono(x, e) for c, e in zip(self.coef, self.exps))

    def grad(self, x):
        x = np.atleast_2d(x)
        d = x.shape[1]
        g = [np.zeros(x.shape[0]) for _ in range(d)]
        for c, e in zip(self.coef, self.exps):
            for j in range(d):
                if e[j] == 0:
                    continue
                e2 = e.copy()
                e2[j] -= 1
                g[j] = g[j] + c * e[j] * self._mono(x, e2)
        return g

    def lap(self, x):
        x = np.atleast_2d(x)
        d = x.shape[1]
        out = np.zeros(x.shape[0])
        for c, e in zip(self.coef, self.exps):
            for j in range(d):
                if e[j] < 2:
                    continue
                e2 = e.copy()
                e2[j] -= 2
                out = out + c * e[j] * (e[j] - 1) * self._mono(x, e2)
        return out


def polynomial_field(dim: int, degree: int, seed: int, tensor: bool = False) -> PolyField:
    """Random polynomial with coefficients U[-1, 1].

    tensor=False: total degree <= degree.  tensor=True: degree <= degree in
    each variable separately (the space Q_degree)."""
    rng = np.random.default_rng(seed)
    rngs = [range(degree + 1)] * dim
    exps = np.array(np.meshgrid(*rngs, indexing="ij")).reshape(dim, -1).T
    if not tensor:
        exps = exps[exps.sum(axis=1) <= degree]
    coef = rng.uniform(-1.0, 1.0, size=len(exps))
    return PolyField(exps, coef)


def _const_coeffs(dim, a=1.0, c=0.0):
    def f(x):
        x = np.atleast_2d(x)
        m = x.shape[0]
        return {"a": np.full(m, a), "b": [np.zeros(m) for _ in range(dim)], "c": np.full(m, c)}
    return f



def poly_varcoef(dim: int, degree: int, seed: int, kind: str = "dtn", eta: float = 2.0) -> Problem:
    """A tensor polynomial u in Q_degree with smooth, seeded, non-constant
    coefficients: a = 1 + 0.3 sin(k_a . x + phi_a) in [0.7, 1.3],
    b_j = 0.5 cos(k_b . x + phi_b + j), c = 0.7 + 0.5 sin(k_c . x + phi_c),
    wave vectors U[-2, 2]^dim and phases U[0, 2 pi) from ``seed + 100``.
    f = a Lap u + b . grad u + c u is formed from the closed-form derivatives
    of u, so a collocation that reproduces u exactly also reproduces f
    exactly at every node, whatever a, b and c are.  Boundary data:
    Dirichlet values (dtn) or incoming impedance u_n + i eta u (iti)."""
    P = polynomial_field(dim, degree, seed, tensor=True)
    rng = np.random.default_rng(seed + 100)
    kv = rng.uniform(-2.0, 2.0, (3, dim))
    ph = rng.uniform(0.0, 2.0 * np.pi, 3)
    lo, hi = (-1.0,) * dim, (1.0,) * dim

    def coeffs(x):
        x = np.atleast_2d(x)
        return {"a": 1.0 + 0.3 * np.sin(x @ kv[0] + ph[0]),
                "b": [0.5 * np.cos(x @ kv[1] + ph[1] + j) for j in range(dim)],
                "c": 0.7 + 0.5 * np.sin(x @ kv[2] + ph[2])}

    def f(x):
        x = np.atleast_2d(x)
        co = coeffs(x)
        gr = P.grad(x)
        out = co["a"] * P.lap(x) + co["c"] * P.value(x)
        for j in range(dim):
            out = out + co["b"][j] * gr[j]
        return out if kind == "dtn" else out.astype(complex)

    if kind == "dtn":
        return Problem(f"poly_varcoef{dim}d_deg{degree}_seed{seed}", dim, lo, hi, "dtn", seed,
                       coeffs, f, P.value, P.value, info={"poly": P})

    def g(xb):
        nn = box_normals(xb, lo, hi)
        gr = P.grad(xb)
        return sum(nn[:, k] * gr[k] for k in range(dim)) + 1j * eta * P.value(xb)

    return Problem(f"poly_varcoef{dim}d_deg{degree}_seed{seed}", dim, lo, hi, "iti", seed,
                   coeffs, f, g, P.value, eta=eta, info={"poly": P})

# ---------------------------------------------------------------------------
# workload 1: 2D Poisson, Dirichlet, u = sin(pi x) sin(pi y) + P5
# ---------------------------------------------------------------------------

def poisson_poly_2d(seed: int = 0, degree: int = 5, with_sine: bool = True,
                    tensor: bool = False, lo=(-1.0, -1.0), hi=(1.0, 1.0)) -> Problem:
    """Lap u = f on [-1,1]^2 with Dirichlet data; u = sin(pi x) sin(pi y) + P(x,y)
    where P has total degree <= ``degree`` and coefficients U[-1,1] from ``seed``."""
    P = polynomial_field(2, degree, seed, tensor=tensor)
    s = 1.0 if with_sine else 0.0

    def u(x):
        x = np.atleast_2d(x)
        return s * np.sin(np.pi * x[:, 0]) * np.sin(np.pi * x[:, 1]) + P.value(x)

    def f(x):
        x = np.atleast_2d(x)
        return (-2 * np.pi ** 2 * s * np.sin(np.pi * x[:, 0]) * np.sin(np.pi * x[:, 1])
                + P.lap(x))

    return Problem(name=f"poisson2d_poly{degree}_seed{seed}", dim=2, lo=tuple(lo), hi=tuple(hi),
                   kind="dtn", seed=seed, coeffs=_const_coeffs(2), source=f,
                   boundary=u, u_exact=u, info={"degree": degree, "sine": with_sine})


# ---------------------------------------------------------------------------
# workload 2: 2D variable-coefficient Helmholtz, ItI, complex128
# ---------------------------------------------------------------------------

def helmholtz_bumps_2d(seed: int = 1, k: float = 20.0, eta: Optional[float] = None,
                       n_bumps: int = 4, amp: float = 0.5, width: float = 0.1) -> Problem:
    """Lap u + k^2 (1 - n(x)) u = f on [-1,1]^2 with incoming impedance data.

    n(x) = sum_i amp exp(-|x - z_i|^2 / (2 width^2)), z_i ~ U[-0.8, 0.8]^2.
    f is one Gaussian of the same width (amplitude 1) at a seeded centre.
    g is the incoming impedance u_n + i eta u of the plane wave exp(i k d.x)
    with a seeded unit direction d.  eta defaults to k."""
    rng = np.random.default_rng(seed)
    z = rng.uniform(-0.8, 0.8, size=(n_bumps, 2))
    zf = rng.uniform(-0.8, 0.8, size=2)
    theta = rng.uniform(0.0, 2 * np.pi)
    d = np.array([np.cos(theta), np.sin(theta)])
    eta = float(k if eta is None else eta)
    lo, hi = (-1.0, -1.0), (1.0, 1.0)

    def nfield(x):
        x = np.atleast_2d(x)
        out = np.zeros(x.shape[0])
        for zi in z:
            out += amp * np.exp(-((x - zi) ** 2).sum(axis=1) / (2 * width ** 2))
        return out

    def coeffs(x):
        x = np.atleast_2d(x)
        m = x.shape[0]
        return {"a": np.ones(m), "b": [np.zeros(m), np.zeros(m)],
                "c": k ** 2 * (1.0 - nfield(x))}

    def f(x):
        x = np.atleast_2d(x)
        return np.exp(-((x - zf) ** 2).sum(axis=1) / (2 * width ** 2)).astype(complex)

    def g(xb):
        xb = np.atleast_2d(xb)
        nrm = box_normals(xb, lo, hi)
        w = np.exp(1j * k * (xb @ d))
        return 1j * k * (nrm @ d) * w + 1j * eta * w

    return Problem(name=f"helmholtz2d_k{k:g}_seed{seed}", dim=2, lo=lo, hi=hi, kind="iti",
                   seed=seed, coeffs=coeffs, source=f, boundary=g, eta=eta,
                   info={"k": k, "bump_centres": z.tolist(), "source_centre": zf.tolist(),
                         "direction": d.tolist()})


def grid_interp_matrix(x: np.ndarray, n: int = 64, lo=(-1.0, -1.0), hi=(1.0, 1.0)):
    """Sparse (len(x) x n^2) matrix of tensor cubic Lagrange interpolation from
    an n x n grid of values on [lo, hi] (grid point (i, j) at lo + (i, j) h,
    h = (hi - lo) / (n - 1); flattened index i + n j) to the points x.  Each
    point uses the 4 x 4 grid points around it (shifted inward at the edges).
    Linear in the grid values, so its transpose is the exact adjoint."""
    import scipy.sparse as sps
    x = np.atleast_2d(x)
    m = x.shape[0]
    rows, cols, vals = [], [], []
    w_axes, i_axes = [], []
    for a in range(2):
        h = (hi[a] - lo[a]) / (n - 1)
        t = (x[:, a] - lo[a]) / h
        i0 = np.clip(np.floor(t).astype(int) - 1, 0, n - 4)
        loc = t - i0                       # position within the 4 stencil points 0..3
        w = np.ones((m, 4))
        for k in range(4):
            for j in range(4):
                if j != k:
                    w[:, k] *= (loc - j) / (k - j)
        w_axes.append(w)
        i_axes.append(i0)
    for kx in range(4):
        for ky in range(4):
            rows.append(np.arange(m))
            cols.append((i_axes[0] + kx) + n * (i_axes[1] + ky))
            vals.append(w_axes[0][:, kx] * w_axes[1][:, ky])
    return sps.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(m, n * n))


def helmholtz_theta_2d(seed: int = 5, k: float = 20.0, n: int = 64):
    """Differentiation workload: the operator of helmholtz_bumps_2d(seed=1)
    with its refractive field n(x) replaced by theta, an n x n grid of values
    carried to the nodes by grid_interp_matrix; c = k^2 (1 - I theta).
    Returns the base problem (source, boundary data, eta), theta_true (a
    smooth seeded field: the sum of 6 Gaussian bumps of width 0.15 and
    amplitude U[0.2, 0.5] sampled on the grid), theta_0 (zero field) and the
    16 seeded grid entries and the seeded unit direction used for the
    finite-difference check."""
    base = helmholtz_bumps_2d(seed=1, k=k)
    rng = np.random.default_rng(seed)
    zc = rng.uniform(-0.7, 0.7, size=(6, 2))
    am = rng.uniform(0.2, 0.5, size=6)
    g1 = np.linspace(-1.0, 1.0, n)
    X, Y = np.meshgrid(g1, g1, indexing="ij")
    th = np.zeros((n, n))
    for zi, ai in zip(zc, am):
        th += ai * np.exp(-((X - zi[0]) ** 2 + (Y - zi[1]) ** 2) / (2 * 0.15 ** 2))
    theta_true = th.reshape(-1, order="F")          # index i + n j
    theta_0 = np.zeros(n * n)
    probe = rng.choice(n * n, 16, replace=False)
    direction = rng.standard_normal(n * n)
    direction /= np.linalg.norm(direction)
    return {"problem": base, "k": k, "n": n, "theta_true": theta_true, "theta_0": theta_0,
            "probe": probe, "direction": direction}


# ---------------------------------------------------------------------------
# workload 3: 3D divergence-form elliptic problem
# ---------------------------------------------------------------------------

def _elliptic(dim: int, seed: int, n_modes: int, lo, hi) -> Problem:
    rng = np.random.default_rng(seed)
    km = rng.uniform(-3.0, 3.0, size=(n_modes, dim))
    phim = rng.uniform(0, 2 * np.pi, size=n_modes)
    alpha = rng.uniform(-1.0, 1.0, size=n_modes)
    S = np.abs(alpha).sum()
    kc = rng.uniform(-2.0, 2.0, size=dim)
    phic = rng.uniform(0, 2 * np.pi)
    w1 = rng.uniform(-2.0, 2.0, size=dim)
    w2 = rng.uniform(-2.0, 2.0, size=dim)
    p1, p2 = rng.uniform(0, 2 * np.pi, size=2)

    def a_and_grad(x):
        arg = x @ km.T + phim
        s = (alpha * np.sin(arg)).sum(axis=1)
        ds = (alpha * np.cos(arg)) @ km
        return 1.0 + 0.5 * s / S, 0.5 * ds / S

    def cfun(x):
        return 0.5 + 0.5 * np.sin(x @ kc + phic)

    def coeffs(x):
        x = np.atleast_2d(x)
        a, ga = a_and_grad(x)
        return {"a": a, "b": [ga[:, k] for k in range(dim)], "c": cfun(x)}

    def u(x):
        x = np.atleast_2d(x)
        return np.sin(x @ w1 + p1) + 0.5 * np.cos(x @ w2 + p2)

    def grad_u(x):
        return (np.cos(x @ w1 + p1)[:, None] * w1
                - 0.5 * np.sin(x @ w2 + p2)[:, None] * w2)

    def lap_u(x):
        return (-(w1 @ w1) * np.sin(x @ w1 + p1) - 0.5 * (w2 @ w2) * np.cos(x @ w2 + p2))

    def f(x):
        x = np.atleast_2d(x)
        a, ga = a_and_grad(x)
        return a * lap_u(x) + (ga * grad_u(x)).sum(axis=1) + cfun(x) * u(x)

    return Problem(name=f"elliptic{dim}d_seed{seed}", dim=dim, lo=tuple(lo), hi=tuple(hi), kind="dtn",
                   seed=seed, coeffs=coeffs, source=f, boundary=u, u_exact=u,
                   info={"n_modes": n_modes})


def elliptic_3d(seed: int = 2, n_modes: int = 8, lo=(-1.0, -1.0, -1.0),
                hi=(1.0, 1.0, 1.0)) -> Problem:
    """div(a grad u) + c u = f on [-1,1]^3, Dirichlet data.

    Expanded as a Lap u + grad(a) . grad u + c u, so the first-order
    coefficients are b = grad a.  a = 1 + 0.5 s(x)/S with s a sum of
    ``n_modes`` seeded modes alpha_m sin(k_m . x + phi_m) and S = sum|alpha_m|,
    so a lies in [0.5, 1.5].  c = 0.5 + 0.5 sin(kc . x + phic) lies in [0, 1].
    The manufactured solution is u = sin(w1 . x + p1) + 0.5 cos(w2 . x + p2)."""
    return _elliptic(3, seed, n_modes, lo, hi)


def elliptic_2d(seed: int = 4, n_modes: int = 8, lo=(-1.0, -1.0), hi=(1.0, 1.0)) -> Problem:
    """The 2D counterpart of elliptic_3d (same construction on [-1,1]^2): a
    variable-coefficient DtN problem whose coefficient field is drawn from
    ``seed``, used for the rebuild requests of the serving workload."""
    return _elliptic(2, seed, n_modes, lo, hi)


def sharp_source_3d(seed: int = 3, width: float = 0.05) -> Problem:
    """Poisson problem on [-1,1]^3 driven by a seeded sharp Gaussian source
    exp(-|x - z|^2 / (2 width^2)), z ~ U[-0.5, 0.5]^3, zero Dirichlet data.
    Used to build an adaptively refined octree (leaf depths 2-5)."""
    rng = np.random.default_rng(seed)
    z = rng.uniform(-0.5, 0.5, size=3)

    def f(x):
        x = np.atleast_2d(x)
        return np.exp(-((x - z) ** 2).sum(axis=1) / (2 * width ** 2))

    def g(xb):
        return np.zeros(np.atleast_2d(xb).shape[0])

    return Problem(name=f"sharp3d_seed{seed}", dim=3, lo=(-1.0,) * 3, hi=(1.0,) * 3, kind="dtn",
                   seed=seed, coeffs=_const_coeffs(3), source=f, boundary=g,
                   info={"centre": z.tolist(), "width": width})


def adaptive_3d(seed_coeffs: int = 2, seed_source: int = 3, width: float = 0.05) -> Problem:
    """Workload 3b: the variable-coefficient operator of elliptic_3d (seed 2)
    driven by the sharp seeded Gaussian source of sharp_source_3d (seed 3,
    width 0.05) with zero Dirichlet data.  The adaptive tree is refined on f,
    a and c (eps = 1e-4, leaf depths 2..5)."""
    pe = elliptic_3d(seed=seed_coeffs)
    ps = sharp_source_3d(seed=seed_source, width=width)
    return Problem(name=f"adaptive3d_seed{seed_coeffs}_{seed_source}", dim=3, lo=pe.lo, hi=pe.hi, kind="dtn",
                   seed=seed_source, coeffs=pe.coeffs, source=ps.source, boundary=ps.boundary,
                   info={"centre": ps.info["centre"], "width": width, "eps": 1e-4, "min_depth": 2,
                         "max_depth": 5, "refine_on": ["f", "a", "c"]})


# ---------------------------------------------------------------------------
# the paper's closed-form test problems (Sections 5.1 and 6.1)
# ---------------------------------------------------------------------------

def e1_dtn_2d() -> Problem:
    """Lap u - cos(5 y) u_x + sin(5 y) u_y = f on [-1,1]^2, Dirichlet data,
    u = exp(5x) sin(5y) + sin(10 pi x) sin(pi y)  (Section 5.1)."""
    lo, hi = (-1.0, -1.0), (1.0, 1.0)
    pi = np.pi

    def u(x):
        x = np.atleast_2d(x)
        X, Y = x[:, 0], x[:, 1]
        return np.exp(5 * X) * np.sin(5 * Y) + np.sin(10 * pi * X) * np.sin(pi * Y)

    def coeffs(x):
        x = np.atleast_2d(x)
        m = x.shape[0]
        return {"a": np.ones(m), "b": [-np.cos(5 * x[:, 1]), np.sin(5 * x[:, 1])],
                "c": np.zeros(m)}

    def f(x):
        x = np.atleast_2d(x)
        X, Y = x[:, 0], x[:, 1]
        ux = 5 * np.exp(5 * X) * np.sin(5 * Y) + 10 * pi * np.cos(10 * pi * X) * np.sin(pi * Y)
        uy = 5 * np.exp(5 * X) * np.cos(5 * Y) + pi * np.sin(10 * pi * X) * np.cos(pi * Y)
        lap = (25 - 25) * np.exp(5 * X) * np.sin(5 * Y) \
            - (100 * pi ** 2 + pi ** 2) * np.sin(10 * pi * X) * np.sin(pi * Y)
        return lap - np.cos(5 * Y) * ux + np.sin(5 * Y) * uy

    return Problem(name="E1_dtn2d", dim=2, lo=lo, hi=hi, kind="dtn", seed=None,
                   coeffs=coeffs, source=f, boundary=u, u_exact=u)


def e2_iti_2d() -> Problem:
    """Lap u + (1 + exp(-50|x|^2)) u = f on [-1,1]^2 with u_n + i u = g,
    u = exp(20 i x) + exp(30 i y)  (Section 5.1, eta = 1)."""
    lo, hi = (-1.0, -1.0), (1.0, 1.0)

    def u(x):
        x = np.atleast_2d(x)
        return np.exp(20j * x[:, 0]) + np.exp(30j * x[:, 1])

    def cfun(x):
        return 1.0 + np.exp(-50 * (x ** 2).sum(axis=1))

    def coeffs(x):
        x = np.atleast_2d(x)
        m = x.shape[0]
        return {"a": np.ones(m), "b": [np.zeros(m), np.zeros(m)], "c": cfun(x)}

    def f(x):
        x = np.atleast_2d(x)
        lap = -400 * np.exp(20j * x[:, 0]) - 900 * np.exp(30j * x[:, 1])
        return lap + cfun(x) * u(x)

    def g(xb):
        xb = np.atleast_2d(xb)
        nrm = box_normals(xb, lo, hi)
        gx = 20j * np.exp(20j * xb[:, 0])
        gy = 30j * np.exp(30j * xb[:, 1])
        return nrm[:, 0] * gx + nrm[:, 1] * gy + 1j * u(xb)

    return Problem(name="E2_iti2d", dim=2, lo=lo, hi=hi, kind="iti", seed=None,
                   coeffs=coeffs, source=f, boundary=g, u_exact=u, eta=1.0)


def e7_wavefront_3d() -> Problem:
    """Lap u = f on [0,1]^3, Dirichlet data, u = arctan(10 r - 0.7) with
    r = |x - (0.5, 0.5, 0.5)|  (Section 6.1)."""
    lo, hi = (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)

    def u(x):
        x = np.atleast_2d(x)
        r = np.sqrt(((x - 0.5) ** 2).sum(axis=1))
        return np.arctan(10 * r - 0.7)

    def f(x):
        # radial Laplacian: u'' + (2/r) u'
        x = np.atleast_2d(x)
        r = np.sqrt(((x - 0.5) ** 2).sum(axis=1))
        s = 10 * r - 0.7
        up = 10.0 / (1 + s ** 2)
        upp = -200.0 * s / (1 + s ** 2) ** 2
        with np.errstate(divide="ignore", invalid="ignore"):
            out = upp + 2.0 * up / r
        return out

    return Problem(name="E7_wavefront3d", dim=3, lo=lo, hi=hi, kind="dtn", seed=None,
                   coeffs=_const_coeffs(3), source=f, boundary=u, u_exact=u)
