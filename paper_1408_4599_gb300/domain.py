"""Spatial domain decomposition across ranks (§4: subvolumes with halo
cells, one exchange per step, load balanced by the per-cell cost of Eq. 6).

One process per GPU.  The periodic box is cut along cell planes into one
subvolume per rank, balanced by the load-cost estimate

    n_d = sum over cells c of the subvolume:  N_c / 2 (N_c + sum over the 26 neighbours of c of N_c')

(§4 Eq. 6: the pair work of a cell grows with its own occupation times the
occupation around it).  Two partitions:

  * ``kd`` (§4.3, tree-based decomposition): the box is bisected
    recursively by planes perpendicular to alternating axes, each plane the
    one of least load imbalance between the two halves (per rank of each
    half), until every rank has a brick; every brick covers at least
    ``min_cells`` cells along each axis;
  * ``slab``: cuts along the longest axis only.

Each step a rank

  1. receives from every other rank the molecules that lie within r_c of
     its subvolume (the halo: every partner of an owned molecule inside the
     centre-of-mass cut-off is then present locally),
  2. evaluates forces and torques of its owned + halo set on its own GPU with
     the global periodic box (the minimum image is unchanged, so the force on
     an owned molecule is exactly the single-domain force), keeps the owned
     rows, and advances the owned molecules,
  3. hands molecules that left its subvolume to the rank that now owns them.

``rebalance()`` (dynamic load balancing, §4: every 100 to 1000 steps) sums
the ranks' cell histograms, recomputes the partition from the current
occupation and migrates the molecules to their new owners.

Energies, virials and pair counts are pair sums: with A the owned and H the
halo molecules of a rank, pairs inside A count once and pairs between A and
H are seen by two ranks, so the rank contributes

    X_rank = 1/2 [X(A u H) + X(A) - X(H)]    (X = U, W, W_aa, pair counts)

and the all-reduced sum over ranks is the single-domain value, with no
change to the kernels.  Observables are formed on demand (three local
evaluations); forces need one.

The local evaluation is a backend object with

    forces(r, q) -> (F, tau, obs)       obs: U, W, Wxx, Wyy, Wzz, n_mol_pairs
    step(state, dt, T_target) -> state  one leapfrog step of the given state

``GpuBackend`` runs the CUDA library (md.System); the collectives go
through ``torch.distributed`` (NCCL between GPUs, gloo on the host).
"""
from __future__ import annotations

import math

import numpy as np

OBS_KEYS = ("U", "W", "Wxx", "Wyy", "Wzz", "n_mol_pairs")


def cell_grid(box, rc):
    """Cells per axis, floor(L / rc) as the library forms them."""
    return [max(1, int(math.floor(L / (rc * (1.0 + 1e-9))))) for L in box]


def cell_index(r, box, rc):
    """Cell coordinates (x, y, z) of each position on the linked-cell grid,
    periodic wrap included; returns (idx[n, 3], nc)."""
    nc = cell_grid(box, rc)
    L = np.asarray(box, float)
    idx = np.floor(np.mod(r, L) / (L / nc)).astype(np.int64)
    return np.clip(idx, 0, np.asarray(nc) - 1), nc


def cell_counts(r, box, rc):
    """Molecules per cell, N[nz, ny, nx]."""
    idx, nc = cell_index(r, box, rc)
    N = np.zeros((nc[2], nc[1], nc[0]))
    np.add.at(N, (idx[:, 2], idx[:, 1], idx[:, 0]), 1.0)
    return N


def cell_costs(r, box, rc):
    """Per-cell load estimate n_d = N_c / 2 (N_c + sum of the 26 neighbours'
    N) on the linked-cell grid (§4 Eq. 6); returns (costs[nz, ny, nx], nc)."""
    return costs_from_counts(cell_counts(r, box, rc)), cell_grid(box, rc)


def costs_from_counts(N):
    """Eq. 6 from the cell occupation N[nz, ny, nx] (periodic neighbours)."""
    around = np.zeros_like(N)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if dx or dy or dz:
                    around += np.roll(N, shift=(dz, dy, dx), axis=(0, 1, 2))
    return 0.5 * N * (N + around)


def partition(r, box, rc, world):
    """Slab decomposition along the longest axis: (axis, boundaries, shares)
    with boundaries[k] .. boundaries[k + 1] the coordinate interval of rank
    k, cut on cell planes so that the ranks' shares of the Eq. 6 load
    estimate are as equal as the planes allow, each slab at least one cell
    (>= r_c) thick."""
    costs, _ = cell_costs(r, box, rc)
    return partition_slab(costs, box, rc, world)


def partition_slab(costs, box, rc, world):
    """The slab decomposition of `partition` from per-cell costs."""
    nc = cell_grid(box, rc)
    axis = int(np.argmax(box))
    if world > nc[axis]:
        raise ValueError(f"{world} slabs need at least {world} cells along axis {axis} (have {nc[axis]})")
    layer = costs.sum(axis=tuple(k for k in range(3) if k != 2 - axis))  # cost per cell plane along `axis`
    cum = np.concatenate([[0.0], np.cumsum(layer)])
    cuts = [0]
    for k in range(1, world):
        target = cum[-1] * k / world
        c = int(np.argmin(np.abs(cum - target)))
        c = max(c, cuts[-1] + 1)                    # at least one plane per slab
        c = min(c, nc[axis] - (world - k))          # leave a plane for every later slab
        cuts.append(c)
    cuts.append(nc[axis])
    ell = box[axis] / nc[axis]
    return axis, [c * ell for c in cuts], [float(cum[cuts[k + 1]] - cum[cuts[k]]) for k in range(world)]


def partition_kd(costs, world, min_cells=2, coarse_cells=None):
    """Tree-based decomposition (§4.3) of the cell grid with per-cell costs
    costs[nz, ny, nx] into `world` bricks.  A region holding p ranks is cut
    by a cell plane perpendicular to the axis of its depth in the tree
    (x, y, z, x, ...; the next axis when that one admits no plane) into a
    lower part for p // 2 ranks and an upper part for the rest; of the
    admissible planes the one with the least load imbalance, the larger of
    cost / ranks of the two sides, is taken.  A plane is admissible if both
    parts can in turn be cut the same way into bricks of at least min_cells
    cells along every axis.

    coarse_cells (the simplified first levels of §4.3 for very large
    volumes): while a region holds more cells than this, it is halved by
    volume instead (the middle plane of the axis), and its ranks are divided
    between the halves in proportion to their costs (the nearest division
    for which both halves can still be decomposed).

    Returns (bricks, shares): bricks[k] = ((x0, y0, z0), (x1, y1, z1)) in
    cells, half-open, and shares[k] its summed cost.  Raises ValueError if
    no such decomposition exists."""
    from functools import lru_cache

    nc = (costs.shape[2], costs.shape[1], costs.shape[0])

    def child_dims(dims, axis, length):
        d = list(dims)
        d[axis] = length
        return tuple(d)

    @lru_cache(maxsize=None)
    def feasible(dims, p, depth):
        if p == 1:
            return all(d >= min_cells for d in dims)
        p_lo = p // 2
        for t in range(3):
            axis = (depth + t) % 3
            for c in range(1, dims[axis]):
                if feasible(child_dims(dims, axis, c), p_lo, (depth + 1) % 3) and \
                        feasible(child_dims(dims, axis, dims[axis] - c), p - p_lo, (depth + 1) % 3):
                    return True
        return False

    if world < 1 or not feasible(nc, world, 0):
        raise ValueError(f"cannot give {world} ranks bricks of at least {min_cells} cells per axis "
                         f"on a {nc[0]} x {nc[1]} x {nc[2]} cell grid")
    bricks = [None] * world

    def region_cost(lo, hi):
        return float(costs[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]].sum())

    def coarse_split(lo, hi, p, depth, dims):
        """Equal-volume halving with ranks in proportion to the halves'
        costs: (axis, plane, p_lo) or None."""
        for t in range(3):
            axis = (depth + t) % 3
            h = dims[axis] // 2
            if h < 1:
                continue
            d_lo, d_hi = child_dims(dims, axis, h), child_dims(dims, axis, dims[axis] - h)
            hi_lo = list(hi)
            hi_lo[axis] = lo[axis] + h
            total = region_cost(lo, hi)
            ideal = p * region_cost(lo, hi_lo) / total if total > 0 else p / 2
            for q in sorted(range(1, p), key=lambda q: (abs(q - ideal), q)):
                if feasible(d_lo, q, (depth + 1) % 3) and feasible(d_hi, p - q, (depth + 1) % 3):
                    return axis, lo[axis] + h, q
        return None

    def split(lo, hi, r0, p, depth):
        if p == 1:
            bricks[r0] = (tuple(lo), tuple(hi))
            return
        dims = tuple(hi[a] - lo[a] for a in range(3))
        if coarse_cells is not None and dims[0] * dims[1] * dims[2] > coarse_cells:
            cs = coarse_split(lo, hi, p, depth, dims)
            if cs is not None:
                axis, c, q = cs
                hi_lo, lo_hi = list(hi), list(lo)
                hi_lo[axis] = c
                lo_hi[axis] = c
                split(lo, hi_lo, r0, q, depth + 1)
                split(lo_hi, hi, r0 + q, p - q, depth + 1)
                return
        p_lo, p_hi = p // 2, p - p // 2
        for t in range(3):
            axis = (depth + t) % 3
            cuts = [c for c in range(1, dims[axis])
                    if feasible(child_dims(dims, axis, c), p_lo, (depth + 1) % 3)
                    and feasible(child_dims(dims, axis, dims[axis] - c), p_hi, (depth + 1) % 3)]
            if cuts:
                break
        sub = costs[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
        planes = sub.sum(axis=tuple(k for k in range(3) if k != 2 - axis))  # cost per plane along `axis`
        cum = np.concatenate([[0.0], np.cumsum(planes)])
        cuts = np.asarray(cuts)
        worst = np.maximum(cum[cuts] / p_lo, (cum[-1] - cum[cuts]) / p_hi)
        c = lo[axis] + int(cuts[int(np.argmin(worst))])
        hi_lo, lo_hi = list(hi), list(lo)
        hi_lo[axis] = c
        lo_hi[axis] = c
        split(lo, hi_lo, r0, p_lo, depth + 1)
        split(lo_hi, hi, r0 + p_lo, p_hi, depth + 1)

    split([0, 0, 0], list(nc), 0, world, 0)
    shares = [float(costs[b[0][2]:b[1][2], b[0][1]:b[1][1], b[0][0]:b[1][0]].sum()) for b in bricks]
    return bricks, shares


def _periodic_gap(x, lo, hi, L):
    """Distance along one periodic axis from coordinates x to the interval
    [lo, hi) (0 inside it)."""
    if hi - lo >= L:
        return np.zeros_like(x)
    inside = (x >= lo) & (x < hi)
    return np.where(inside, 0.0, np.minimum(np.mod(lo - x, L), np.mod(x - hi, L)))


class Domain:
    """One rank's slab [lo, hi) along `axis` of the periodic box."""

    def __init__(self, rank, world, box, rc, axis, bounds):
        self.rank, self.world = rank, world
        self.box = np.asarray(box, float)
        self.rc, self.axis = float(rc), axis
        self.lo, self.hi = float(bounds[rank]), float(bounds[rank + 1])
        self.bounds = list(bounds)
        self.left, self.right = (rank - 1) % world, (rank + 1) % world

    def owner(self, r, bounds):
        """Rank owning each position (periodic coordinate along the axis)."""
        x = np.mod(r[:, self.axis], self.box[self.axis])
        return np.clip(np.searchsorted(np.asarray(bounds[1:-1]), x, side="right"), 0, self.world - 1)

    def halo_out(self, r):
        """Owned molecules within r_c of the lower face (for the left
        neighbour) and of the upper face (for the right neighbour)."""
        L = self.box[self.axis]
        x = np.mod(r[:, self.axis], L)
        d_lo = np.mod(x - self.lo, L)       # distance above the lower face
        d_hi = np.mod(self.hi - x, L)       # distance below the upper face
        return np.nonzero(d_lo < self.rc)[0], np.nonzero(d_hi <= self.rc)[0]

    def halo_routes(self, r):
        """Indices of the owned molecules each rank needs as its halo."""
        to_l, to_r = self.halo_out(r)
        routes = [np.zeros(0, np.int64) for _ in range(self.world)]
        routes[self.left] = to_l
        routes[self.right] = np.union1d(routes[self.right], to_r)  # one rank on both sides: once
        return routes

    def owner_of(self, r):
        return self.owner(r, self.bounds)


class BrickDomain:
    """One rank's brick of a tree-based decomposition (§4.3): bricks[k] =
    ((x0, y0, z0), (x1, y1, z1)) in cells of the linked-cell grid."""

    def __init__(self, rank, world, box, rc, bricks):
        self.rank, self.world = rank, world
        self.box = np.asarray(box, float)
        self.rc = float(rc)
        self.bricks = [tuple(map(tuple, b)) for b in bricks]
        self.nc = cell_grid(box, rc)
        self.ell = self.box / np.asarray(self.nc, float)
        self.grid = np.full((self.nc[2], self.nc[1], self.nc[0]), -1, np.int64)  # owner of each cell
        for k, (lo, hi) in enumerate(self.bricks):
            self.grid[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] = k
        if (self.grid < 0).any():
            raise ValueError("the bricks do not cover the cell grid")

    def owner_of(self, r):
        """Rank owning each position: the brick of its cell."""
        idx, _ = cell_index(r, self.box, self.rc)
        return self.grid[idx[:, 2], idx[:, 1], idx[:, 0]]

    def gap(self, r, k):
        """Periodic distance of each position from brick k (0 inside)."""
        lo, hi = self.bricks[k]
        x = np.mod(r, self.box)
        g2 = np.zeros(r.shape[0])
        for a in range(3):
            g = _periodic_gap(x[:, a], lo[a] * self.ell[a], hi[a] * self.ell[a], self.box[a])
            g2 += g * g
        return np.sqrt(g2)

    def halo_routes(self, r):
        """Indices of the owned molecules within r_c of each other rank's
        brick: every centre-of-mass partner of a molecule of that brick
        (minimum image, |X| < r_c) is within r_c of the brick."""
        routes = [np.zeros(0, np.int64) for _ in range(self.world)]
        for k in range(self.world):
            if k != self.rank and r.shape[0]:
                routes[k] = np.nonzero(self.gap(r, k) <= self.rc * (1.0 + 1e-9))[0]
        return routes


def _exchange(sends, keys, widths, rank, world, dist, group=None):
    """Sends sends[k] (a dict of arrays with the given keys and row widths,
    one row per molecule) to rank k and receives what every rank sent here:
    the counts of all ranks by one all-gather, then the float64 payloads by
    non-blocking point-to-point pairs (no ordering deadlock).  Host tensors:
    under NCCL pass a gloo group.  Returns the received rows of all ranks,
    concatenated in rank order, as one dict."""
    import torch
    width = sum(widths[k] for k in keys)

    def pack(d):
        n = d[keys[0]].shape[0]
        return torch.from_numpy(np.concatenate([np.asarray(d[k], float).reshape(n, widths[k]) for k in keys], axis=1)
                                .reshape(-1).copy()), n

    packed = [pack(sends[k]) if k != rank else (None, 0) for k in range(world)]
    mine = torch.tensor([n for _, n in packed], dtype=torch.int64)
    counts = [torch.zeros(world, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(counts, mine, group=group)
    incoming = [int(counts[k][rank].item()) for k in range(world)]  # rows rank k sends here
    bufs = [torch.zeros(incoming[k] * width, dtype=torch.float64) for k in range(world)]
    reqs = []
    for k in range(world):
        if k != rank and packed[k][1]:
            reqs.append(dist.isend(packed[k][0], k, group=group, tag=7))
        if k != rank and incoming[k]:
            reqs.append(dist.irecv(bufs[k], k, group=group, tag=7))
    for q in reqs:
        q.wait()
    rows = np.concatenate([b.numpy().reshape(-1, width) for b in bufs], axis=0) if sum(incoming) else \
        np.zeros((0, width))
    out, c = {}, 0
    for k in keys:
        w = widths[k]
        out[k] = rows[:, c:c + w] if w > 1 else rows[:, c]
        c += w
    return out


class DecomposedSystem:
    """The owned molecules of one rank (global ids kept with them) and the
    per-step halo exchange, local evaluation and migration."""

    STATE = ("r", "v", "q", "j")
    KEYS = ("r", "v", "q", "j", "ids")
    WIDTHS = {"r": 3, "v": 3, "q": 4, "j": 3, "ids": 1}

    def __init__(self, domain, bounds, backend, state, ids, dist, group=None, method="slab", min_cells=2,
                 rebalance_every=0):
        """rebalance_every: repartition every that many steps (§4: every 100
        to 1000 steps; 0 = only when rebalance() is called)."""
        self.dom, self.bounds, self.be, self.dist, self.group = domain, bounds, backend, dist, group
        self.st = {k: np.ascontiguousarray(state[k], float) for k in self.STATE}
        self.ids = np.asarray(ids, np.int64)
        self.method, self.min_cells = method, min_cells
        self.rebalance_every, self.n_steps = int(rebalance_every), 0

    @staticmethod
    def make_domain(rank, world, box, rc, counts, method="slab", min_cells=2):
        """The partition of the cell occupation counts[nz, ny, nx] among
        `world` ranks by its Eq. 6 costs: (domain, bounds) with bounds the
        slab boundaries ("slab") or the bricks ("kd")."""
        costs = costs_from_counts(counts)
        if method == "kd":
            bricks, _ = partition_kd(costs, world, min_cells)
            return BrickDomain(rank, world, box, rc, bricks), bricks
        if method != "slab":
            raise ValueError(f"unknown partition {method!r} (slab or kd)")
        axis, bounds, _ = partition_slab(costs, box, rc, world)
        return Domain(rank, world, box, rc, axis, bounds), bounds

    @classmethod
    def scatter_from(cls, rank, world, cfg, backend, dist, group=None, method="slab", min_cells=2,
                     rebalance_every=0):
        """Every rank holds the same full configuration (seeded input) and
        keeps the molecules of its subvolume (method: "slab" or "kd")."""
        counts = cell_counts(cfg["r"], cfg["box"], cfg["rc"])
        dom, bounds = cls.make_domain(rank, world, cfg["box"], cfg["rc"], counts, method, min_cells)
        mine = np.nonzero(dom.owner_of(cfg["r"]) == rank)[0]
        return cls(dom, bounds, backend, {k: cfg[k][mine] for k in cls.STATE}, mine, dist, group, method, min_cells,
                   rebalance_every)

    def _rows(self, ix):
        return {**{k: self.st[k][ix] for k in self.STATE}, "ids": self.ids[ix].astype(float)}

    def _send(self, routes):
        return _exchange([self._rows(ix) for ix in routes], self.KEYS, self.WIDTHS, self.dom.rank, self.dom.world,
                         self.dist, self.group)

    def _halo(self):
        if self.dom.world == 1:  # the periodic box itself: no halo
            return {**{k: self.st[k][:0] for k in self.STATE}, "ids": np.zeros(0)}
        return self._send(self.dom.halo_routes(self.st["r"]))

    def forces(self):
        """Forces and torques on the owned molecules (rows in self.ids order)."""
        halo = self._halo()
        r = np.concatenate([self.st["r"], halo["r"]])
        q = np.concatenate([self.st["q"], halo["q"]])
        F, tau, _ = self.be.forces(r, q)
        n = self.ids.shape[0]
        return F[:n], tau[:n]

    def observables(self):
        """All-reduced U, W, W_aa and interacting pair counts of the whole
        system (the owned/halo identity of the module docstring)."""
        import torch
        halo = self._halo()
        rA, qA = self.st["r"], self.st["q"]
        parts = []
        for r, q in ((np.concatenate([rA, halo["r"]]), np.concatenate([qA, halo["q"]])), (rA, qA),
                     (halo["r"], halo["q"])):
            if r.shape[0] == 0:
                parts.append(np.zeros(len(OBS_KEYS)))
                continue
            _, _, o = self.be.forces(r, q)
            parts.append(np.array([o[k] for k in OBS_KEYS], float))
        mine = 0.5 * (parts[0] + parts[1] - parts[2])
        t = torch.from_numpy(mine.copy())
        self.dist.all_reduce(t, group=self.group)
        return dict(zip(OBS_KEYS, t.numpy().tolist()))

    def step(self, dt, T_target=0.0):
        """One leapfrog step: halo exchange, local step of owned + halo
        (the halo's own update is discarded), migration of the molecules
        that left the subvolume.  NVE only when T_target <= 0 (the velocity-
        rescaling factor needs a global kinetic energy: not offered)."""
        if T_target > 0:
            raise NotImplementedError("velocity rescaling is not offered across domains")
        if self.rebalance_every > 0 and self.n_steps > 0 and self.n_steps % self.rebalance_every == 0:
            self.rebalance()
        self.n_steps += 1
        halo = self._halo()
        n = self.ids.shape[0]
        full = {k: np.concatenate([self.st[k], halo[k]]) for k in self.STATE}
        new = self.be.step(full, dt)
        self.st = {k: np.ascontiguousarray(new[k][:n]) for k in self.STATE}
        self._migrate()

    def _migrate(self):
        """Molecules whose owner (by the current partition) is another rank
        move there, wherever it is."""
        if self.dom.world == 1:
            return
        own = self.dom.owner_of(self.st["r"])
        stay = np.nonzero(own == self.dom.rank)[0]
        got = self._send([np.nonzero(own == k)[0] if k != self.dom.rank else np.zeros(0, np.int64)
                          for k in range(self.dom.world)])
        self.st = {k: np.concatenate([self.st[k][stay], got[k]]) for k in self.STATE}
        self.ids = np.concatenate([self.ids[stay], got["ids"].astype(np.int64)])

    def rebalance(self):
        """Dynamic load balancing (§4: every 100 to 1000 steps): the ranks'
        cell histograms are summed by one all-reduce, every rank forms the
        same partition of the current occupation (the method chosen at
        set-up) and the molecules migrate to their new owners."""
        import torch
        box, rc = self.dom.box, self.dom.rc
        N = torch.from_numpy(cell_counts(self.st["r"], box, rc))
        self.dist.all_reduce(N, group=self.group)
        self.dom, self.bounds = self.make_domain(self.dom.rank, self.dom.world, box, rc, N.numpy(), self.method,
                                                 self.min_cells)
        self._migrate()


class GpuBackend:
    """Local evaluation on this rank's GPU through the C ABI (md.System with
    the global periodic box; owned + halo molecules are set each call)."""

    def __init__(self, cfg, half_shell=1):
        from . import md
        self.md, self.cfg, self.half = md, cfg, half_shell

    def _system(self, r, q, v=None, j=None):
        s = self.md.System(self.cfg, deterministic=0 if self.half else 1, half_shell=self.half)
        z = np.zeros_like(r)
        s.set(r, q, z if v is None else v, z if j is None else j)
        return s

    def forces(self, r, q):
        s = self._system(r, q)
        s.compute_forces()
        F, tau = s.forces()
        o = s.observables()
        s.close()
        obs = {"U": o["U_pot"], "W": o["W"], "Wxx": o["W_xx"], "Wyy": o["W_yy"], "Wzz": o["W_zz"],
               "n_mol_pairs": float(o["n_mol_pairs"])}
        return F, tau, obs

    def step(self, st, dt):
        s = self._system(st["r"], st["q"], st["v"], st["j"])
        s.step(1, dt)
        r, v, q, j = s.molecules()
        s.close()
        return {"r": r, "v": v, "q": q, "j": j}
