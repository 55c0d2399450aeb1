"""Seeded synthetic power grids and load scenarios.

This module only draws inputs: topology, branch parameters, generator data,
costs and loads.  It holds none of the solver's arithmetic (no admittances, no
flows, no QP data) and is imported both by the test oracle's callers and by
the GPU path's callers.

The recipes follow the shapes of the paper's test networks (MATPOWER cases of
9 to 6,468 buses, Section IV) with the parameter distributions below; every
array is float64 (int32 for indices) in per-unit on ``base_mva``:

* branches: r ~ U(0.01, 0.08), x = r * U(2, 6), charging b ~ U(0, 0.05),
  rating ~ U(0.5, 2.0), angle-difference limit +-30 degrees, tap 1, shift 0;
* generators at distinct buses (the first one sits at the reference bus):
  Pmin = 0, Pmax ~ U(0.5, 3), Q in [-1, 1], cost c2 ~ U(0.01, 0.1),
  c1 ~ U(10, 40) (per MW), c0 = 0; on meshed grids the weakest load leaves
  get one and the rest are spread so that every bus has a generator within
  two hops (see ``_spread_generators``); the 30-bus tree-plus-edges grid places them
  uniformly at random;
* loads: pd ~ U(0.1, 0.5), qd = pd * U(0.2, 0.4), scaled so that the total
  load is at most 60% of the total Pmax;
* voltage limits [0.94, 1.06] on the 30-bus grid and [0.9, 1.1] on the
  meshed grids of hundreds to tens of thousands of buses, shunts 0, base
  100 MVA.  (With the narrow band, the synthetic meshed grids of 300 buses
  and more leave load pockets whose reactive supply cannot stay within it;
  the wider band is the one large test systems commonly use.)

Feasibility guard (input recipe, not solver arithmetic): a DC power-flow
estimate of the branch flows under a dispatch proportional to Pmax is taken
with a plain Laplacian solve, and every rating is raised to at least
1.5 * |estimate| + 0.25 so that no load pocket is cut off by a rating drawn
below its demand.  Ratings drawn above that floor are kept, so limits still
bind in the optimum when cheap generation is far away.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

REF = 3  # bus_type of the reference (slack) bus
PQ = 1


@dataclass
class Grid:
    nbus: int
    bus_type: np.ndarray
    pd: np.ndarray
    qd: np.ndarray
    gs: np.ndarray
    bs: np.ndarray
    vmin: np.ndarray
    vmax: np.ndarray
    f: np.ndarray
    t: np.ndarray
    r: np.ndarray
    x: np.ndarray
    b: np.ndarray
    rate: np.ndarray
    angmin: np.ndarray
    angmax: np.ndarray
    tap: np.ndarray
    shift: np.ndarray
    gbus: np.ndarray
    pmin: np.ndarray
    pmax: np.ndarray
    qmin: np.ndarray
    qmax: np.ndarray
    c2: np.ndarray
    c1: np.ndarray
    c0: np.ndarray
    base_mva: float = 100.0
    xy: np.ndarray | None = field(default=None, repr=False)
    name: str = ""

    @property
    def nbranch(self) -> int:
        return int(self.f.shape[0])

    @property
    def ngen(self) -> int:
        return int(self.gbus.shape[0])

    def with_loads(self, pd: np.ndarray, qd: np.ndarray, name: str | None = None) -> "Grid":
        return replace(self, pd=np.ascontiguousarray(pd, dtype=np.float64),
                       qd=np.ascontiguousarray(qd, dtype=np.float64),
                       name=self.name if name is None else name)


# --------------------------------------------------------------------------
# topology
# --------------------------------------------------------------------------
def _prufer_tree(n: int, rng: np.random.Generator) -> list[tuple[int, int]]:
    """Edges of the labelled tree encoded by a uniformly random Pruefer sequence."""
    if n == 1:
        return []
    if n == 2:
        return [(0, 1)]
    seq = rng.integers(0, n, size=n - 2)
    degree = np.ones(n, dtype=np.int64)
    for s in seq:
        degree[s] += 1
    edges = []
    for s in seq:
        leaf = int(np.flatnonzero(degree == 1)[0])
        edges.append((leaf, int(s)))
        degree[leaf] -= 1
        degree[s] -= 1
    u, v = np.flatnonzero(degree == 1)
    edges.append((int(u), int(v)))
    return edges


class _DSU:
    def __init__(self, n):
        self.p = np.arange(n)

    def find(self, a):
        p = self.p
        root = a
        while p[root] != root:
            root = p[root]
        while p[a] != root:
            p[a], a = root, p[a]
        return root

    def union(self, a, b):
        ra, rb = self.find(a), self.find(b)
        if ra == rb:
            return False
        self.p[ra] = rb
        return True


def _geometric_edges(xy: np.ndarray, m: int, rng: np.random.Generator, scale: float = 0.15) -> list[tuple[int, int]]:
    """Connected random geometric graph with exactly ``m`` edges.

    A shortest-edge spanning tree over the k-nearest-neighbour pairs joins
    every bus (components of the candidate graph are joined by their closest
    pair of points).  The remaining ``m - (n-1)`` edges are long-range links
    of a Waxman-type model: from a random bus, a link of exponentially
    distributed length (mean ``scale``) in a random direction ends at the bus
    nearest to that point.  Without such links a nearest-neighbour graph of
    thousands of buses has a diameter of dozens of hops and cannot carry its
    load within the angle and voltage limits.
    """
    from scipy.spatial import cKDTree

    n = xy.shape[0]
    k = min(n - 1, 8)
    tree = cKDTree(xy)
    dist, idx = tree.query(xy, k=k + 1)
    cand = {}
    for i in range(n):
        for d, j in zip(dist[i, 1:], idx[i, 1:]):
            a, b = (i, int(j)) if i < j else (int(j), i)
            cand[(a, b)] = float(d)
    items = sorted(cand.items(), key=lambda kv: (kv[1], kv[0]))
    dsu = _DSU(n)
    chosen = []
    for (a, b), d in items:
        if dsu.union(a, b):
            chosen.append((a, b))
    # join leftover components, each to its nearest point of the others
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import connected_components

    while True:
        ee = np.array(chosen, dtype=np.int64).reshape(-1, 2)
        adj = csr_matrix((np.ones(len(ee)), (ee[:, 0], ee[:, 1])), shape=(n, n))
        ncomp, lab = connected_components(adj, directed=False)
        if ncomp <= 1:
            break
        sizes = np.bincount(lab, minlength=ncomp)
        for c in np.argsort(sizes, kind="stable")[: ncomp - 1]:
            ins = np.flatnonzero(lab == c)
            outs = np.flatnonzero(lab != c)
            sub = cKDTree(xy[outs])
            d, j = sub.query(xy[ins], k=1)
            a = int(ins[int(np.argmin(d))])
            b = int(outs[int(j[int(np.argmin(d))])])
            if dsu.union(a, b):
                chosen.append((min(a, b), max(a, b)))
            lab[lab == c] = lab[b]
    have = set(chosen)
    tries = 0
    while len(chosen) < m:
        tries += 1
        if tries > 100 * m:
            raise ValueError("could not draw the requested number of distinct branches")
        u = int(rng.integers(n))
        length = rng.exponential(scale)
        ang = rng.uniform(0.0, 2.0 * np.pi)
        target = xy[u] + length * np.array([np.cos(ang), np.sin(ang)])
        _, v = tree.query(target, k=1)
        v = int(v)
        if v == u:
            continue
        key = (min(u, v), max(u, v))
        if key in have:
            continue
        have.add(key)
        chosen.append(key)
    return chosen[:m]


# --------------------------------------------------------------------------
# parameters
# --------------------------------------------------------------------------
def _dc_flow_estimate(n, f, t, x, pinj, ref):
    """Branch flows of a DC power flow (B theta = P, theta_ref = 0)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla

    bser = 1.0 / x
    rows = np.concatenate([f, t, f, t])
    cols = np.concatenate([f, t, t, f])
    vals = np.concatenate([bser, bser, -bser, -bser])
    B = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    keep = np.ones(n, dtype=bool)
    keep[ref] = False
    th = np.zeros(n)
    A = B[keep][:, keep]
    if n <= 20000:
        th[keep] = spla.spsolve(A.tocsc(), pinj[keep])
    else:  # direct factorisation fills in badly on large meshed graphs
        d = A.diagonal()
        M = spla.LinearOperator(A.shape, matvec=lambda v: v / d)
        th[keep], _ = spla.cg(A.tocsr(), pinj[keep], rtol=1e-10, maxiter=20000, M=M)
    return bser * (th[f] - th[t])


def _spread_generators(n, f, t, r, x, pd, qd, ngen, rng):
    """Distinct generator buses spread over the network.

    1. Load leaves (degree-1 buses with load) whose voltage-drop estimate
       r*pd + x*(qd + pd^2) over their only branch exceeds 0.06 receive a
       generator, weakest first (at most ngen/3 of them): random
       voltage-limited grids are otherwise infeasible at heavily loaded leaves
       behind a high reactance.
    2. Buses are visited in random order; one with no generator within two hops
       receives one.
    3. Any generators left go to random buses.
    The first generator placed is the reference bus.
    """
    adj = [[] for _ in range(n)]
    for a, b in zip(f.tolist(), t.tolist()):
        adj[a].append(b)
        adj[b].append(a)
    has = np.zeros(n, dtype=bool)
    covered = np.zeros(n, dtype=bool)
    chosen = []

    def take(u):
        chosen.append(int(u))
        has[u] = True
        covered[u] = True
        for v in adj[u]:
            covered[v] = True
            for w in adj[v]:
                covered[w] = True

    order = rng.permutation(n)
    take(order[0])
    deg = np.bincount(np.concatenate([f, t]), minlength=n)
    br = np.full(n, -1)
    br[f] = np.arange(f.shape[0])
    br[t] = np.arange(t.shape[0])
    weak = np.zeros(n)
    leaf = (deg == 1) & (pd > 0)
    lb = br[leaf]
    weak[leaf] = r[lb] * pd[leaf] + x[lb] * (qd[leaf] + pd[leaf] ** 2)
    weak[has] = 0.0
    cand = np.flatnonzero(weak > 0.06)
    cand = cand[np.argsort(-weak[cand], kind="stable")][: max(0, min(ngen - 1, ngen // 3))]
    for u in cand.tolist():
        take(u)
    for u in order[1:]:
        if len(chosen) >= ngen:
            break
        if not covered[u]:
            take(u)
    if len(chosen) < ngen:
        rest = np.flatnonzero(~has)
        chosen.extend(rng.choice(rest, size=ngen - len(chosen), replace=False).tolist())
    return np.asarray(chosen[:ngen], dtype=np.int32)


def _assemble(n, edges, ngen, nload, rng, xy=None, name="", spread=True, vband=(0.94, 1.06)):
    edges = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    m = edges.shape[0]
    # random orientation of every branch
    flip = rng.random(m) < 0.5
    f = np.where(flip, edges[:, 1], edges[:, 0]).astype(np.int32)
    t = np.where(flip, edges[:, 0], edges[:, 1]).astype(np.int32)
    r = rng.uniform(0.01, 0.08, m)
    x = r * rng.uniform(2.0, 6.0, m)
    b = rng.uniform(0.0, 0.05, m)
    rate = rng.uniform(0.5, 2.0, m)
    ang = math.radians(30.0)
    angmin = np.full(m, -ang)
    angmax = np.full(m, ang)

    pmax = rng.uniform(0.5, 3.0, ngen)
    pmin = np.zeros(ngen)
    qmin = -np.ones(ngen)
    qmax = np.ones(ngen)
    c2 = rng.uniform(0.01, 0.1, ngen)
    c1 = rng.uniform(10.0, 40.0, ngen)
    c0 = np.zeros(ngen)

    lb = rng.choice(n, size=nload, replace=False)
    pd = np.zeros(n)
    qd = np.zeros(n)
    pd[lb] = rng.uniform(0.1, 0.5, nload)
    qd[lb] = pd[lb] * rng.uniform(0.2, 0.4, nload)
    cap = 0.6 * pmax.sum()
    if pd.sum() > cap:
        s = cap / pd.sum()
        pd *= s
        qd *= s
    if spread:
        gb = _spread_generators(n, f, t, r, x, pd, qd, ngen, rng)
    else:
        gb = rng.choice(n, size=ngen, replace=False).astype(np.int32)

    bus_type = np.full(n, PQ, dtype=np.int32)
    bus_type[gb[0]] = REF

    # feasibility guard on ratings (see module docstring)
    pinj = -pd.copy()
    np.add.at(pinj, gb, pmax * (pd.sum() / pmax.sum()))
    est = np.abs(_dc_flow_estimate(n, f, t, x, pinj, int(gb[0])))
    rate = np.maximum(rate, 1.5 * est + 0.25)

    return Grid(
        nbus=n, bus_type=bus_type, pd=pd, qd=qd, gs=np.zeros(n), bs=np.zeros(n),
        vmin=np.full(n, vband[0]), vmax=np.full(n, vband[1]),
        f=f, t=t, r=r, x=x, b=b, rate=rate, angmin=angmin, angmax=angmax,
        tap=np.ones(m), shift=np.zeros(m),
        gbus=gb, pmin=pmin, pmax=pmax, qmin=qmin, qmax=qmax, c2=c2, c1=c1, c0=c0,
        base_mva=100.0, xy=xy, name=name)


def tree_plus_grid(nbus: int, nextra: int, ngen: int, nload: int, seed: int, name: str = "") -> Grid:
    """Random spanning tree (Pruefer sequence) plus ``nextra`` distinct extra edges."""
    rng = np.random.default_rng(seed)
    edges = _prufer_tree(nbus, rng)
    have = {(min(a, b), max(a, b)) for a, b in edges}
    while len(edges) < nbus - 1 + nextra:
        a, b = rng.integers(0, nbus, size=2)
        if a == b:
            continue
        key = (int(min(a, b)), int(max(a, b)))
        if key in have:
            continue
        have.add(key)
        edges.append(key)
    xy = rng.random((nbus, 2))
    return _assemble(nbus, edges, ngen, nload, rng, xy=xy, name=name or f"tree{nbus}-s{seed}", spread=False)


def _morton(xy: np.ndarray) -> np.ndarray:
    """Z-order (Morton) keys of points in [0,1]^2: 16-bit coordinates with
    their bits interleaved."""
    q = np.clip((xy * 65535.0).astype(np.uint64), 0, 65535)

    def spread(v):
        v = (v | (v << 8)) & np.uint64(0x00FF00FF)
        v = (v | (v << 4)) & np.uint64(0x0F0F0F0F)
        v = (v | (v << 2)) & np.uint64(0x33333333)
        v = (v | (v << 1)) & np.uint64(0x55555555)
        return v

    return spread(q[:, 0]) | (spread(q[:, 1]) << np.uint64(1))


def relabel_regional(g: Grid) -> Grid:
    """The same grid with buses numbered along a Z-order curve of their
    coordinates and branches sorted by (lower, higher) end bus, so that buses
    close in the plane, and the branches between them, are close in every
    array (regional numbering, as in published grid cases).  Generators keep
    their order; only labels change."""
    if g.xy is None:
        return g
    perm = np.argsort(_morton(g.xy), kind="stable")      # new bus -> old bus
    inv = np.empty_like(perm)
    inv[perm] = np.arange(g.nbus)
    f = inv[g.f].astype(np.int32)
    t = inv[g.t].astype(np.int32)
    border = np.lexsort((np.maximum(f, t), np.minimum(f, t)))
    bus = {k: getattr(g, k)[perm] for k in ("bus_type", "pd", "qd", "gs", "bs", "vmin", "vmax")}
    br = {k: getattr(g, k)[border] for k in ("r", "x", "b", "rate", "angmin", "angmax", "tap", "shift")}
    return replace(g, **bus, **br, f=f[border], t=t[border], gbus=inv[g.gbus].astype(np.int32), xy=g.xy[perm])


def geometric_grid(nbus: int, seed: int, nbranch: int | None = None, ngen: int | None = None,
                   nload: int | None = None, name: str = "", regional: bool = True) -> Grid:
    """Random geometric graph on U[0,1]^2 with mean degree 2*nbranch/nbus.
    With regional=True (default) the grid is relabelled by relabel_regional;
    regional=False keeps the labels of the construction (random in the plane)."""
    rng = np.random.default_rng(seed)
    nbranch = int(round(1.35 * nbus)) if nbranch is None else nbranch
    ngen = max(2, int(round(0.2 * nbus))) if ngen is None else ngen
    nload = int(round(0.6 * nbus)) if nload is None else nload
    xy = rng.random((nbus, 2))
    edges = _geometric_edges(xy, nbranch, rng)
    g = _assemble(nbus, edges, ngen, nload, rng, xy=xy, name=name or f"geo{nbus}-s{seed}", vband=(0.9, 1.1))
    return relabel_regional(g) if regional else g


# --------------------------------------------------------------------------
# load scenarios
# --------------------------------------------------------------------------
def scenarios_cholesky(grid: Grid, n: int, seed: int, sigma: float = 0.05, ell: float = 0.1):
    """``n`` load scenarios pd*(1+e), qd*(1+e); e ~ N(0, sigma^2 K), K squared-exponential
    over bus coordinates with length scale ``ell``; sampled through a Cholesky factor."""
    rng = np.random.default_rng(seed)
    xy = grid.xy
    d2 = ((xy[:, None, :] - xy[None, :, :]) ** 2).sum(-1)
    K = np.exp(-0.5 * d2 / ell ** 2) + 1e-8 * np.eye(grid.nbus)
    Lc = np.linalg.cholesky(K)
    out = []
    for s in range(n):
        e = sigma * (Lc @ rng.standard_normal(grid.nbus))
        out.append(grid.with_loads(grid.pd * (1 + e), grid.qd * (1 + e), name=f"{grid.name}/sc{s}"))
    return out


def scenarios_rff(grid: Grid, n: int, seed: int, sigma: float = 0.05, ell: float = 0.1, nfeat: int = 512):
    """Same field as :func:`scenarios_cholesky`, approximated by random Fourier features
    (for grids where a dense Cholesky factor does not fit)."""
    rng = np.random.default_rng(seed)
    xy = grid.xy
    out = []
    for s in range(n):
        W = rng.standard_normal((nfeat, 2)) / ell
        phase = rng.uniform(0, 2 * np.pi, nfeat)
        a = rng.standard_normal(nfeat)
        e = sigma * math.sqrt(2.0 / nfeat) * (np.cos(xy @ W.T + phase) @ a)
        out.append(grid.with_loads(grid.pd * (1 + e), grid.qd * (1 + e), name=f"{grid.name}/rff{s}"))
    return out


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------
def hub_grid(nspokes: int = 40, seed: int = 21) -> Grid:
    """One hub bus joined to nspokes spoke buses, the spokes joined in a ring:
    the hub has nspokes incident branches (a bus of unusually high degree)."""
    rng = np.random.default_rng(seed)
    n = nspokes + 1
    edges = [(0, k) for k in range(1, n)] + [(k, k % nspokes + 1) for k in range(1, n)]
    return _assemble(n, edges, max(2, n // 5), int(0.6 * n), rng, xy=rng.random((n, 2)), name=f"hub{n}-s{seed}",
                     spread=False)


def grid_30bus(seed: int = 3) -> Grid:
    """30 buses, 41 branches (a 29-edge spanning tree plus 12 extra edges),
    6 generators, 20 loads."""
    return tree_plus_grid(30, 12, 6, 20, seed, name=f"syn30-s{seed}")


def grid_2000bus(seed: int = 2, regional: bool = True) -> Grid:
    """2,000 buses, about 2,700 branches (mean degree 2.7), 400 generators, 1,200 loads."""
    return geometric_grid(2000, seed, name=f"syn2000-s{seed}", regional=regional)


def grid_70k(seed: int = 5) -> Grid:
    """70,000 buses, 90,000 branches, 10,000 generators, 40,000 loads."""
    return geometric_grid(70000, seed, nbranch=90000, ngen=10000, nload=40000, name=f"syn70k-s{seed}")


def batched_uneven(seed: int = 3, nscen: int = 256, ngrids: int = 64, base: Grid | None = None,
                   regional: bool = True):
    """256 correlated load scenarios of the 2,000-bus grid plus 64 grids whose bus
    counts are log-uniform in [118, 10000]."""
    base = grid_2000bus(regional=regional) if base is None else base
    out = scenarios_cholesky(base, nscen, seed=1000 + seed)
    rng = np.random.default_rng(seed)
    sizes = np.round(np.exp(rng.uniform(math.log(118), math.log(10000), ngrids))).astype(int)
    for k, nb in enumerate(sizes):
        out.append(geometric_grid(int(nb), seed=10_000 + 97 * seed + k, regional=regional))
    return out


def two_bus(lossless: bool = True, rate: float = 5.0, pd2: float = 0.8, qd2: float = 0.2,
            c2=(0.02, 0.05), c1=(20.0, 30.0), pmax=(2.0, 2.0), angle_limits: bool = False) -> Grid:
    """Two buses, one branch, a generator at each bus, load at bus 2."""
    ang = math.radians(30.0) if angle_limits else 2 * math.pi
    return Grid(
        nbus=2, bus_type=np.array([REF, PQ], dtype=np.int32),
        pd=np.array([0.0, pd2]), qd=np.array([0.0, qd2]), gs=np.zeros(2), bs=np.zeros(2),
        vmin=np.array([0.94, 0.94]), vmax=np.array([1.06, 1.06]),
        f=np.array([0], dtype=np.int32), t=np.array([1], dtype=np.int32),
        r=np.array([0.0 if lossless else 0.02]), x=np.array([0.1]),
        b=np.array([0.0 if lossless else 0.02]), rate=np.array([rate]),
        angmin=np.array([-ang]), angmax=np.array([ang]), tap=np.ones(1), shift=np.zeros(1),
        gbus=np.array([0, 1], dtype=np.int32), pmin=np.zeros(2), pmax=np.array(pmax, float),
        qmin=-np.ones(2), qmax=np.ones(2), c2=np.array(c2, float), c1=np.array(c1, float),
        c0=np.zeros(2), base_mva=100.0, xy=np.array([[0.0, 0.0], [1.0, 0.0]]), name="two-bus")


# --------------------------------------------------------------------------
# warm-start network: initial weights
# --------------------------------------------------------------------------
def mlp_init(dims, seed: int) -> np.ndarray:
    """Initial parameters of a network with layer widths dims, as one FP32
    array (per layer W [out x in] row-major, then b): W ~ N(0, 1/in) (LeCun
    normal), b = 0."""
    rng = np.random.default_rng(seed)
    parts = []
    for i in range(len(dims) - 1):
        parts.append((rng.standard_normal((dims[i + 1], dims[i])) / math.sqrt(dims[i])).ravel())
        parts.append(np.zeros(dims[i + 1]))
    return np.concatenate(parts).astype(np.float32)
