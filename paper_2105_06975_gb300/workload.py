"""Seeded synthetic inputs for the weak-constraint 4D-Var saddle-point workloads.

This module holds the workload definitions (sizes, covariance parameters,
model coefficients) and the seeded random draws both the CUDA library and
the FP64 oracle consume.  It contains none of the method's arithmetic: no
covariance matrix, no model operator, no preconditioner.  Everything that
turns these draws into a saddle-point problem is done separately by each side.

Workloads (all synthetic; the paper's own datasets and Lorenz-96 code are not
available, so these stand in for its experiments with the shapes below):

* ``tiny``  -- 1D periodic advection-diffusion, s=100, N=10, p=50 (every 2nd
  point), SOAR B/Q/R, block-diagonal preconditioner with exact D, R and Schur
  complement, MINRES.  n = (2s+p)(N+1) = 2750.
* ``scale`` -- the same covariances at s=2048, N=64, p=1024 observed points
  drawn without replacement and sorted.  n = 332,800.
* ``l96``   -- Lorenz-96, s=1000, F=8, RK4 dt=0.025 with 5 steps per
  observation time, N=50, every 2nd variable observed, 3 Gauss-Newton loops.
* ``batch`` -- ``batch_windows``: independent windows of uneven size,
  s = 4 U{32..512}, N = U{8..96}, p = s/2 or s/4, advection-diffusion (the
  scale workload's covariances) or Lorenz-96 (its covariances, lengths in grid
  points, and the paper's time step 1e-4 of Sec. 7.1) by a fair coin each.
* ``heat``  -- the heat equation with homogeneous Dirichlet boundaries
  (Sec. 7.2, forward Euler, r = 0.4), s=50,000, N=5, p=12,500 random sorted
  observed points (p/s = 0.25), the banded "modified SOAR" B and Q of
  Sec. 6.1 (amplitude, length, maxval = 0.4, 0.6, 100 and 0.2, 0.5, 120) and
  the channel-block R_i of Sec. 6.1.  n = 750,000.

Seeds: master seed m in {0, 1, 2}; window w of a batch uses m*1000 + w.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import Optional

import numpy as np

MODEL_STENCIL3 = 0
MODEL_BANDED = 1


@dataclass(frozen=True)
class Workload:
    name: str
    s: int
    N: int
    p: int
    # observation pattern: "even" (every 2nd grid point) or "random" (sorted
    # draw without replacement, shared by all times, Sec. 6.1)
    obs: str
    # model: "advdiff" (periodic 3-point stencil), "l96" or "heat" (Dirichlet)
    model: str
    # SOAR (variance, length as a fraction of the periodic unit domain)
    soar_b: tuple = ()
    soar_q: tuple = ()
    soar_r: tuple = ()
    # advection-diffusion: upwind Courant number c and diffusion number d give
    # x'_j = (c+d) x_{j-1} + (1-c-2d) x_j + d x_{j+1}
    courant: float = 0.5
    diffusion: float = 0.2
    # Lorenz-96
    forcing: float = 8.0
    dt: float = 0.025
    steps_per_obs: int = 5
    spinup_steps: int = 2000
    outer_loops: int = 1
    # synthetic truth for the linear model: Gaussian bump of this width
    bump_width: float = 0.05
    # heat equation: r = alpha dt / dx^2
    heat_r: float = 0.4
    # B and Q: "soar" (chordal SOAR above) or "msoar" (the banded circulant
    # modified SOAR of Sec. 6.1: amplitude, length, maxval)
    cov: str = "soar"
    msoar_b: tuple = (0.4, 0.6, 100)
    msoar_q: tuple = (0.2, 0.5, 120)
    # R_i: "soar" (chordal SOAR over the observed points) or "block" (the
    # channel-block matrix of Sec. 6.1): r_blocks equal channel blocks, sparse
    # random factors of density r_density, off-diagonal factors pcorr drawn in
    # (0, r_pcorr_max) with probability 1 - r_uncorrelated (else 0), diagonal
    # blocks weighted by a modified SOAR (amplitude, length, maxval), and the
    # smallest eigenvalue set to r_lmin
    r_kind: str = "soar"
    r_blocks: int = 8
    r_density: float = 0.2
    r_pcorr_max: float = 0.5
    r_uncorrelated: float = 0.5
    r_msoar: tuple = (1.0, 0.5, 10)
    r_lmin: float = 0.41
    # per-time observation sets: time i observes its own p sorted points drawn
    # without replacement (H_i and R_i differ between times)
    obs_per_time: bool = False

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)

    @property
    def n(self) -> int:
        return (2 * self.s + self.p) * (self.N + 1)

    def stencil(self) -> tuple:
        c, d = self.courant, self.diffusion
        return (c + d, 1.0 - c - 2.0 * d, d)

    def heat_bands(self) -> np.ndarray:
        """The heat model's M_t as bands [N][s][3] (offsets -1, 0, +1): forward
        Euler with r = heat_r on interior points, homogeneous Dirichlet rows and
        columns (the boundary points 0 and s-1 carry nothing)."""
        r, s = self.heat_r, self.s
        b = np.zeros((self.N, s, 3))
        j = np.arange(1, s - 1)
        b[:, j, 0] = np.where(j - 1 >= 1, r, 0.0)
        b[:, j, 1] = 1.0 - 2.0 * r
        b[:, j, 2] = np.where(j + 1 <= s - 2, r, 0.0)
        return b


TINY = Workload(name="tiny", s=100, N=10, p=50, obs="even", model="advdiff",
                soar_b=(1.0, 0.1), soar_q=(0.05, 0.05), soar_r=(0.1, 0.05))

SCALE = Workload(name="scale", s=2048, N=64, p=1024, obs="random", model="advdiff",
                 soar_b=(1.0, 0.1), soar_q=(0.05, 0.05), soar_r=(0.1, 0.05))

L96 = Workload(name="l96", s=1000, N=50, p=500, obs="even", model="l96",
               soar_b=(1.0, 5.0 / 1000), soar_q=(0.1, 5.0 / 1000),
               soar_r=(0.5, 4.0 / 1000), outer_loops=3)

HEAT = Workload(name="heat", s=50000, N=5, p=12500, obs="random", model="heat", cov="msoar", r_kind="block")

# the heat window at full size with R the chordal SOAR over the observed points
# (4-point length; the channel-block R of HEAT needs a p x p generator draw)
HEAT_SOAR_R = HEAT.with_(name="heat-soar-r", r_kind="soar", soar_r=(0.5, 4.0 / 50000))

WORKLOADS = {w.name: w for w in (TINY, SCALE, L96, HEAT, HEAT_SOAR_R)}


def block_sizes(p: int, blocks: int) -> np.ndarray:
    """pvec of the channel-block R_i: ``blocks`` sizes summing to p, as equal
    as possible (the first p mod blocks one larger)."""
    blocks = max(1, min(int(blocks), int(p)))
    q, r = divmod(int(p), blocks)
    return np.array([q + 1] * r + [q] * (blocks - r), dtype=np.int64)


def batch_windows(count: int = 256, seed: int = 0) -> list:
    """The windows of the batched workload with their draw seeds: a list of
    (Workload, seed) with seed = 1000 * seed + window index."""
    g = rng(1000 * int(seed) + 999)
    out = []
    for i in range(int(count)):
        s = 4 * int(g.integers(32, 513))
        N = int(g.integers(8, 97))
        p = s // 2 if g.random() < 0.5 else s // 4
        if g.random() < 0.5:
            w = SCALE.with_(name=f"batch{i}-advdiff", s=s, N=N, p=p)
        else:
            w = small(L96, s=s, N=N, p=p).with_(name=f"batch{i}-l96", dt=1e-4, outer_loops=1)
        out.append((w, 1000 * int(seed) + i))
    return out


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


@dataclass
class Draws:
    """Raw seeded draws for one assimilation window (no method arithmetic)."""
    obs_idx: np.ndarray            # int32 [p], sorted, distinct, in [0, s)
    bump_center: float             # truth bump centre in [0, 1)
    z_b: np.ndarray                # [s]        standard normal (background error)
    z_q: np.ndarray                # [N, s]     standard normal (model error)
    z_r: np.ndarray                # [N+1, p]   standard normal (observation error)
    x0_pert: np.ndarray            # [s]        standard normal (Lorenz-96 initial state)
    rhs_probe: np.ndarray          # [n]        standard normal (generic right-hand side)
    extra: dict = field(default_factory=dict)


def observed_indices(w: Workload, g: np.random.Generator) -> np.ndarray:
    if w.obs == "even":
        step = w.s // w.p
        idx = np.arange(w.p, dtype=np.int64) * step
    elif w.obs == "random":
        idx = np.sort(g.choice(w.s, size=w.p, replace=False))
    else:
        raise ValueError(w.obs)
    return idx.astype(np.int32)


def draws(w: Workload, seed: int = 0) -> Draws:
    g = rng(seed)
    obs_idx = observed_indices(w, g)
    center = float(g.random())
    z_b = g.standard_normal(w.s)
    z_q = g.standard_normal((w.N, w.s))
    z_r = g.standard_normal((w.N + 1, w.p))
    x0_pert = g.standard_normal(w.s)
    rhs_probe = g.standard_normal(w.n)
    extra = {}
    # drawn after the draws every workload takes, so those do not change
    if w.cov == "msoar":
        extra["psi"] = g.uniform(0.0, 0.5, size=2)          # shifts psi of B, Q (Sec. 6.1)
    if w.r_kind == "block":
        nb = len(block_sizes(w.p, w.r_blocks))
        npairs = nb * (nb - 1) // 2
        extra["pcorr_on"] = g.random(npairs)                 # < 1 - r_uncorrelated: correlated pair
        extra["pcorr_u"] = g.random(npairs)                  # pcorr = r_pcorr_max * u
        extra["r_u"] = g.random((w.p, w.p))                  # sparse random factors (mask and value)
    if w.obs_per_time:
        extra["obs_list"] = [np.sort(g.choice(w.s, size=w.p, replace=False)).astype(np.int32)
                             for _ in range(w.N + 1)]
    return Draws(obs_idx=obs_idx, bump_center=center, z_b=z_b, z_q=z_q, z_r=z_r,
                 x0_pert=x0_pert, rhs_probe=rhs_probe, extra=extra)


def bump(w: Workload, center: float) -> np.ndarray:
    """Synthetic truth initial state for the linear workloads: a unit Gaussian
    bump of width ``w.bump_width`` centred at ``center`` on the periodic unit
    domain, sampled at x_j = j/s."""
    x = np.arange(w.s) / w.s
    d = np.abs(x - center)
    d = np.minimum(d, 1.0 - d)
    return np.exp(-0.5 * (d / w.bump_width) ** 2)


def random_vector(n: int, seed: int) -> np.ndarray:
    return rng(seed).standard_normal(n)


def small(w: Workload, s: int, N: int, p: Optional[int] = None, **kw) -> Workload:
    """A reduced copy of a workload (same covariance lengths as fractions of
    the domain) for tests the oracle finishes in seconds."""
    p = p if p is not None else max(1, (s * w.p) // w.s)
    if w.model == "l96":
        # Lorenz-96 lengths are fixed in grid points, not domain fractions
        f = w.s / s
        kw.setdefault("soar_b", (w.soar_b[0], w.soar_b[1] * f))
        kw.setdefault("soar_q", (w.soar_q[0], w.soar_q[1] * f))
        kw.setdefault("soar_r", (w.soar_r[0], w.soar_r[1] * f))
    return w.with_(s=s, N=N, p=p, **kw)
