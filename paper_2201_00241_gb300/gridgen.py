"""Seeded synthetic power-grid inputs.

This module draws random numbers only: topology, branch parameters, bus types,
a planted voltage profile, generator costs, load-scenario factors and Hessian
directions.  It evaluates none of the power-flow arithmetic (no admittances, no
injections, no derivatives); each consumer (the CUDA library and the CPU
oracle) derives the loads that make the planted voltages an exact solution with
its own code.

The case shapes follow the paper's Table 1 (bus, branch and generator counts of
IEEE118, PEGASE1354, PEGASE2869 and PEGASE9241).  The PGLIB instances the paper
uses are not available, so these seeded grids stand in for them:

* buses are uniform random points in the unit square;
* a spanning tree attaches each bus (random order) to its nearest already
  placed bus;
* extra branches are drawn uniformly from the not-yet-connected pairs among each
  bus's 8 nearest neighbours until the branch count is reached (a near-planar,
  power-grid-like topology with bounded LU fill);
* r ~ U[0.001, 0.05], x ~ U[0.01, 0.3], b ~ U[0, 0.05] (p.u., pi model);
* generator buses are drawn uniformly; the first one drawn is the slack;
* planted |V| ~ U[0.95, 1.05] and theta ~ N(0, 0.1) rad per bus, drawn as
  spatially smooth random fields over the bus positions (stationary Gaussian
  fields with squared-exponential correlation of length 0.1, by random Fourier
  features; |V| through the normal CDF so that its marginal is uniform), and
  theta shifted so that theta_slack = 0.  Independent draws per bus would put
  neighbouring buses of a low-impedance branch at unrelated angles and
  voltages, an operating point next to voltage collapse on which a +-10 %
  load change has no power-flow solution; smooth fields keep the marginals and
  give operating points like those of real grids;
* quadratic cost c2 ~ U[0.01, 0.1], c1 ~ U[10, 40] per generator.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

REF, PV, PQ = 0, 1, 2

# Weight of one forward level when the symbolic phase compares its two
# fill-reducing orders: an order costs (factor entries off the bus blocks) x n_p
# + ORDER_LEVEL_COST x (forward levels).  The paper leaves the pivot order to a
# host LU; this build's order rule takes the weight as a parameter of the grid
# record.  1.7e6: one level of the four direction sweeps costs GB300 about as
# much time as 1.7 M entry-direction FMAs (measured).
ORDER_LEVEL_COST = 1_700_000

# Table 1 shapes (n_v, n_e, generators) and the seed of each synthetic case.
CASES = {
    "case118": dict(n_bus=118, n_branch=186, n_gen=54, seed=20220100),
    "case1354": dict(n_bus=1354, n_branch=1991, n_gen=260, seed=20220101),
    "case9241": dict(n_bus=9241, n_branch=16049, n_gen=1445, seed=20220102),
    "case2869": dict(n_bus=2869, n_branch=4582, n_gen=510, seed=20220104),
}


@dataclass
class Grid:
    n_bus: int
    n_branch: int
    fr: np.ndarray          # int32 [n_branch], fr < to
    to: np.ndarray          # int32 [n_branch]
    r: np.ndarray           # float64 [n_branch] series resistance
    x: np.ndarray           # float64 [n_branch] series reactance
    b: np.ndarray           # float64 [n_branch] total line charging
    bus_type: np.ndarray    # int8 [n_bus]: 0 slack, 1 PV, 2 PQ
    v_star: np.ndarray      # float64 [n_bus] planted voltage magnitude
    theta_star: np.ndarray  # float64 [n_bus] planted angle, 0 at the slack
    c2: np.ndarray          # float64 [n_bus] quadratic cost ($/MW^2 h), 0 off generators
    c1: np.ndarray          # float64 [n_bus] linear cost ($/MWh), 0 off generators
    base_mva: float
    seed: int
    order_level_cost: int = ORDER_LEVEL_COST

    @property
    def n_gen(self) -> int:
        return int(np.count_nonzero(self.bus_type != PQ))

    @property
    def n_pv(self) -> int:
        return int(np.count_nonzero(self.bus_type == PV))

    @property
    def n_pq(self) -> int:
        return int(np.count_nonzero(self.bus_type == PQ))

    @property
    def n_x(self) -> int:
        return self.n_pv + 2 * self.n_pq

    @property
    def n_p(self) -> int:
        return 2 * self.n_gen - 1


def _nearest_tree(pts: np.ndarray, order: np.ndarray) -> list[tuple[int, int]]:
    edges = []
    placed = np.empty((0, 2))
    placed_ids: list[int] = []
    for k, bus in enumerate(order):
        if k > 0:
            d = ((placed - pts[bus]) ** 2).sum(axis=1)
            j = placed_ids[int(np.argmin(d))]
            edges.append((min(bus, j), max(bus, j)))
        placed = np.vstack([placed, pts[bus]])
        placed_ids.append(int(bus))
    return edges


def _knn(pts: np.ndarray, k: int) -> np.ndarray:
    n = pts.shape[0]
    out = np.empty((n, k), dtype=np.int64)
    for s in range(0, n, 1024):
        blk = pts[s:s + 1024]
        d = ((blk[:, None, :] - pts[None, :, :]) ** 2).sum(axis=2)
        d[np.arange(blk.shape[0]), np.arange(s, s + blk.shape[0])] = np.inf
        kk = min(k, n - 1)
        part = np.argpartition(d, kk - 1, axis=1)[:, :kk]
        rows = np.arange(blk.shape[0])[:, None]
        srt = np.argsort(d[rows, part], axis=1, kind="stable")
        out[s:s + blk.shape[0], :kk] = part[rows, srt]
        if kk < k:
            out[s:s + blk.shape[0], kk:] = -1
    return out


def _smooth_field(rng: np.random.Generator, pts: np.ndarray, ell: float, m: int = 64) -> np.ndarray:
    """Unit-variance stationary Gaussian field with correlation exp(-|d|^2 / (2 ell^2)),
    approximated by m random Fourier features, evaluated at pts."""
    w = rng.normal(0.0, 1.0 / ell, (m, 2))
    ph = rng.uniform(0.0, 2.0 * np.pi, m)
    return math.sqrt(2.0 / m) * np.cos(pts @ w.T + ph).sum(axis=1)


def _normal_cdf(z: np.ndarray) -> np.ndarray:
    return np.array([0.5 * (1.0 + math.erf(float(t) / math.sqrt(2.0))) for t in z])


def make_grid(n_bus: int, n_branch: int, n_gen: int, seed: int,
              base_mva: float = 100.0, lossless: bool = False) -> Grid:
    """Draw one synthetic grid.  ``lossless`` sets every r to 0."""
    if n_bus < 2 or n_gen < 1 or n_gen > n_bus or n_branch < n_bus - 1:
        raise ValueError("inconsistent grid shape")
    rng = np.random.Generator(np.random.PCG64(seed))
    pts = rng.random((n_bus, 2))
    order = rng.permutation(n_bus)
    tree = _nearest_tree(pts, order)
    have = set(tree)
    knn = _knn(pts, 8)
    cand = set()
    for i in range(n_bus):
        for j in knn[i]:
            if j < 0:
                continue
            e = (min(i, int(j)), max(i, int(j)))
            if e not in have:
                cand.add(e)
    cand = sorted(cand)
    extra = n_branch - len(tree)
    if extra > len(cand):
        raise ValueError("not enough local candidate branches")
    pick = rng.permutation(len(cand))[:extra]
    edges = sorted(tree + [cand[i] for i in pick])
    fr = np.array([e[0] for e in edges], dtype=np.int32)
    to = np.array([e[1] for e in edges], dtype=np.int32)

    r = rng.uniform(0.001, 0.05, n_branch)
    x = rng.uniform(0.01, 0.3, n_branch)
    b = rng.uniform(0.0, 0.05, n_branch)
    if lossless:
        r[:] = 0.0

    gens = rng.choice(n_bus, size=n_gen, replace=False)
    bus_type = np.full(n_bus, PQ, dtype=np.int8)
    bus_type[gens] = PV
    bus_type[gens[0]] = REF

    z_theta = _smooth_field(rng, pts, 0.1)
    z_v = _smooth_field(rng, pts, 0.1)
    theta_star = 0.1 * (z_theta - z_theta[gens[0]])
    v_star = 0.95 + 0.1 * _normal_cdf(z_v)

    c2 = np.zeros(n_bus)
    c1 = np.zeros(n_bus)
    c2[gens] = rng.uniform(0.01, 0.1, n_gen)
    c1[gens] = rng.uniform(10.0, 40.0, n_gen)
    return Grid(n_bus, n_branch, fr, to, r, x, b, bus_type, v_star, theta_star,
                c2, c1, float(base_mva), int(seed))


def make_case(name: str, lossless: bool = False) -> Grid:
    c = CASES[name]
    return make_grid(c["n_bus"], c["n_branch"], c["n_gen"], c["seed"], lossless=lossless)


def random_directions(n_p: int, n_dir: int, seed: int) -> np.ndarray:
    """Gaussian directions with unit 2-norm, column-major (n_p, n_dir) float64."""
    rng = np.random.Generator(np.random.PCG64(seed + 1000))
    w = rng.normal(size=(n_p, n_dir))
    w /= np.linalg.norm(w, axis=0, keepdims=True)
    return np.asfortranarray(w)


def load_scales(n_bus: int, n_scen: int, seed: int) -> np.ndarray:
    """Per-bus load factors s ~ U[0.9, 1.1] for each scenario, shape (n_scen, n_bus)."""
    rng = np.random.Generator(np.random.PCG64(seed + 2000))
    return rng.uniform(0.9, 1.1, (n_scen, n_bus))
