"""Seeded synthetic catalogues shaped like the paper's workloads.

This module only draws input positions. It holds none of the estimator's
arithmetic (no quantisation, no pair counting, no normalisation), so both
the CPU oracle tests and the GPU path may take their inputs from it.

Workload shapes follow Sect. 4.1-4.2 of the paper (halo catalogues in a
periodic box or a slab, uniform random catalogues with M times the data
density) and the synthetic stand-ins used for measurement:

* ``neyman_scott``: a Poisson cluster process.  Parents are uniform with
  number density ``n_parent``; a fixed number of children is assigned to
  parents uniformly at random and offset by an isotropic Gaussian of width
  ``sigma``; positions wrap periodically.  Its correlation function has the
  closed form ``xi(r) = exp(-r^2 / 4 sigma^2) / (n_parent (4 pi sigma^2)^1.5)``
  (up to a factor (N_d-1)/N_d * N_p/(n_p V) from fixing N_d and N_p).
* ``uniform_box``: uniform random catalogue in a periodic cube.
* ``shell_octant_*``: an open cut-sky geometry, the x, y, z >= 0 octant of a
  spherical shell around an observer at the origin.

Every generator is driven by ``numpy.random.Generator(Philox)`` keyed by a
``SeedSequence`` built from (config id, mock index, catalogue role), so a
given (config, mock, role) always yields the same catalogue on one machine.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# catalogue roles used in seed derivation
ROLE_DATA = 0
ROLE_RANDOM = 1  # random subset i uses ROLE_RANDOM + i


def rng_for(config_id: int, mock: int, role: int) -> np.random.Generator:
    """Counter-based generator (Philox) keyed by (config, mock, role)."""
    ss = np.random.SeedSequence([int(config_id), int(mock), int(role), 220511852])
    return np.random.Generator(np.random.Philox(ss))


def uniform_box(rng: np.random.Generator, n: int, L: float) -> np.ndarray:
    """n points uniform in [0, L)^3, float64 [n][3]."""
    x = rng.random((n, 3)) * L
    # rng.random is in [0,1); the product can round up to L exactly
    x[x >= L] = 0.0
    return x


def uniform_slab(rng: np.random.Generator, n: int, dims=(1500.0, 1500.0, 300.0)) -> np.ndarray:
    """n points uniform in the slab [0, dims[0]) x [0, dims[1]) x [0, dims[2]) (the paper's simulation
    slab is 1500 x 1500 x 300 (Mpc/h)^3), float64 [n][3]."""
    d = np.asarray(dims, dtype=np.float64)
    x = rng.random((n, 3)) * d
    x[x >= d] = 0.0
    return x


def neyman_scott(rng: np.random.Generator, n: int, L: float, n_parent: float,
                 sigma: float) -> np.ndarray:
    """n children of a Neyman-Scott process in a periodic cube of side L.

    Parents: Poisson(n_parent * L^3) uniform points (at least one).
    Children: each picks a parent uniformly at random and is displaced by
    N(0, sigma^2) per axis; positions wrap into [0, L).
    """
    n_p = max(1, int(rng.poisson(n_parent * L ** 3)))
    parents = rng.random((n_p, 3)) * L
    which = rng.integers(0, n_p, size=n)
    x = parents[which] + rng.normal(0.0, sigma, size=(n, 3))
    x = np.mod(x, L)
    x[x >= L] = 0.0
    return x


def neyman_scott_xi(r, n_parent: float, sigma: float):
    """Closed-form correlation function of the Neyman-Scott generator (large-N limit)."""
    r = np.asarray(r, dtype=np.float64)
    return np.exp(-r * r / (4.0 * sigma * sigma)) / (n_parent * (4.0 * math.pi * sigma * sigma) ** 1.5)


def _octant_shell_mask(x: np.ndarray, r_min: float, r_max: float) -> np.ndarray:
    r2 = np.einsum("ij,ij->i", x, x)
    return (x[:, 0] >= 0) & (x[:, 1] >= 0) & (x[:, 2] >= 0) & (r2 >= r_min * r_min) & (r2 < r_max * r_max)


def shell_octant_uniform(rng: np.random.Generator, n: int, r_min: float, r_max: float) -> np.ndarray:
    """n points uniform in volume inside the x,y,z>=0 octant of the shell r_min <= r < r_max."""
    u = rng.random(n)
    r = np.cbrt(u * (r_max ** 3 - r_min ** 3) + r_min ** 3)
    d = np.abs(rng.normal(size=(n, 3)))
    d /= np.linalg.norm(d, axis=1)[:, None]
    x = d * r[:, None]
    # rounding can push a point onto r_max; pull it back inside
    bad = ~_octant_shell_mask(x, r_min, r_max)
    if bad.any():
        x[bad] *= (1.0 - 1e-12)
        x[~_octant_shell_mask(x, r_min, r_max)] = d[~_octant_shell_mask(x, r_min, r_max)] * (0.5 * (r_min + r_max))
    return x


def shell_octant_neyman_scott(rng: np.random.Generator, n: int, r_min: float, r_max: float,
                              n_parent: float, sigma: float) -> np.ndarray:
    """n Neyman-Scott points drawn in the enclosing cube [0, r_max)^3 and masked to the octant shell."""
    out = []
    have = 0
    frac = (math.pi / 6.0) * (r_max ** 3 - r_min ** 3) / r_max ** 3
    while have < n:
        m = int((n - have) / frac * 1.15) + 1024
        x = neyman_scott(rng, m, r_max, n_parent, sigma)
        x = x[_octant_shell_mask(x, r_min, r_max)]
        out.append(x)
        have += len(x)
    return np.concatenate(out)[:n]


@dataclass
class Mock:
    """One mock: a data catalogue and M random subsets (float64 [n][3] each)."""
    data: np.ndarray
    randoms: list = field(default_factory=list)


@dataclass
class Workload:
    """A named workload: geometry, binning and the recipe for its catalogues."""
    name: str
    config_id: int
    n_mock: int
    geometry: str            # "periodic" | "open"
    L: float                 # periodic box side, or bounding-cube side for open
    origin: tuple            # lower corner of the bounding cube (open)
    n_d: int                 # data points per mock (mean for uneven)
    M: int                   # random subsets per mock
    s_max: float
    n_s: int
    n_mu: int
    los: str                 # "x" | "midpoint"
    observer: tuple = (0.0, 0.0, 0.0)
    n_parent: float = 1e-5
    sigma: float = 2.0
    shell: tuple | None = None       # (r_min, r_max) for the cut-sky octant
    n_d_range: tuple | None = None   # uneven sizes: (lo, hi)

    @property
    def s_edges(self) -> np.ndarray:
        return np.linspace(0.0, self.s_max, self.n_s + 1)

    def n_d_of(self, mock: int) -> int:
        if self.n_d_range is None:
            return self.n_d
        rng = rng_for(self.config_id, mock, 999)
        lo, hi = self.n_d_range
        lam = rng.uniform(lo, hi)
        return int(min(max(rng.poisson(lam), lo), hi))

    def make_mock(self, mock: int, n_d: int | None = None, M: int | None = None) -> Mock:
        """Draw mock ``mock``; ``n_d``/``M`` override sizes for scaled-down cases."""
        nd = self.n_d_of(mock) if n_d is None else n_d
        m_sub = self.M if M is None else M
        rng = rng_for(self.config_id, mock, ROLE_DATA)
        if self.shell is None:
            d = neyman_scott(rng, nd, self.L, self.n_parent, self.sigma)
            rs = [uniform_box(rng_for(self.config_id, mock, ROLE_RANDOM + i), nd, self.L)
                  for i in range(m_sub)]
        else:
            r0, r1 = self.shell
            d = shell_octant_neyman_scott(rng, nd, r0, r1, self.n_parent, self.sigma)
            rs = [shell_octant_uniform(rng_for(self.config_id, mock, ROLE_RANDOM + i), nd, r0, r1)
                  for i in range(m_sub)]
        return Mock(d, rs)


# The five workloads of the measurement plan: periodic small / mid / scale
# boxes of Neyman-Scott data with uniform randoms, the uneven cut-sky
# batching workload, and the covariance-only precision workload.
SMALL = Workload("small", 0, 16, "periodic", 500.0, (0.0, 0.0, 0.0), 4000, 2, 100.0, 20, 1, "x",
                 n_parent=1e-5, sigma=2.0)
MID = Workload("mid", 1, 100, "periodic", 1000.0, (0.0, 0.0, 0.0), 100_000, 2, 200.0, 40, 10, "x",
               n_parent=1e-5, sigma=3.0)
BATCHING = Workload("batching", 2, 1000, "open", 2400.0, (0.0, 0.0, 0.0), 225_000, 2, 200.0, 40, 5,
                    "midpoint", observer=(0.0, 0.0, 0.0), n_parent=1e-5, sigma=3.0,
                    shell=(1200.0, 2400.0), n_d_range=(50_000, 400_000))
SCALE = Workload("scale", 4, 200, "periodic", 2000.0, (0.0, 0.0, 0.0), 1_000_000, 2, 200.0, 40, 10, "x",
                 n_parent=2e-6, sigma=3.0)
WORKLOADS = {w.name: w for w in (SMALL, MID, BATCHING, SCALE)}


def synthetic_xi_variants(config_id: int, n_mock: int, nbin: int, n_d: int = 100_000,
                          seed_role: int = 7) -> tuple:
    """Per-mock correlation-function rows with realistic covariance structure.

    Used as input for covariance-only measurements (no pair counting): three
    variants (R1, R2, R1 u R2) of a 2PCF-like vector per mock, built from a
    shared per-mock clustering fluctuation plus independent random-catalogue
    noise whose amplitude follows the 1/M scaling of Eq. (randomtheory).
    Returns float64 arrays xi_a1, xi_a2, xi_b of shape [n_mock][nbin].
    """
    rng = rng_for(config_id, 0, seed_role)
    k = np.arange(nbin)
    base = 0.5 * np.exp(-k / (0.2 * nbin))
    # correlated data fluctuation: smooth modes shared by all variants
    n_modes = 8
    modes = np.stack([np.cos(np.pi * (j + 0.5) * k / nbin) for j in range(n_modes)])
    amp = rng.normal(size=(n_mock, n_modes)) * (0.02 / (1 + np.arange(n_modes)))
    data = base + amp @ modes + 0.003 * rng.normal(size=(n_mock, nbin))
    noise_scale = 0.004
    e1 = noise_scale * rng.normal(size=(n_mock, nbin))
    e2 = noise_scale * rng.normal(size=(n_mock, nbin))
    xi_a1 = data + e1
    xi_a2 = data + e2
    xi_b = data + 0.5 * (e1 + e2)
    return xi_a1, xi_a2, xi_b
