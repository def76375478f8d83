"""Spatial domain decomposition across ranks (§4: subvolumes with halo
cells, one exchange per step, load balanced by the per-cell cost of Eq. 6).

One process per GPU.  The periodic box is cut into slabs along its longest
axis; slab boundaries fall on cell planes and are placed so that every rank
gets an equal share of the load-cost estimate

    n_d = sum over cells c of the slab:  N_c / 2 (N_c + sum over the 26 neighbours of c of N_c')

(§4 Eq. 6: the pair work of a cell grows with its own occupation times the
occupation around it).  Each step a rank

  1. receives from each neighbouring slab the molecules that lie within r_c
     of its faces (the halo: every partner of an owned molecule inside the
     centre-of-mass cut-off is then present locally),
  2. evaluates forces and torques of its owned + halo set on its own GPU with
     the global periodic box (the minimum image is unchanged, so the force on
     an owned molecule is exactly the single-domain force), keeps the owned
     rows, and advances the owned molecules,
  3. hands molecules that left its slab to the neighbour that now owns them.

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


def cell_costs(r, box, rc):
    """Per-cell load estimate n_d = N_c / 2 (N_c + sum of the 26 neighbours'
    N) on the linked-cell grid (§4 Eq. 6); returns (costs[nz, ny, nx], nc)."""
    nc = cell_grid(box, rc)
    L = np.asarray(box, float)
    idx = np.floor(np.mod(r, L) / (L / nc)).astype(np.int64)
    idx = np.minimum(idx, np.asarray(nc) - 1)
    N = np.zeros((nc[2], nc[1], nc[0]))
    np.add.at(N, (idx[:, 2], idx[:, 1], idx[:, 0]), 1.0)
    around = np.zeros_like(N)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if dx or dy or dz:
                    around += np.roll(N, shift=(dz, dy, dx), axis=(0, 1, 2))
    return 0.5 * N * (N + around), nc


def partition(r, box, rc, world):
    """Slab decomposition along the longest axis: (axis, boundaries) with
    boundaries[k] .. boundaries[k + 1] the coordinate interval of rank k,
    cut on cell planes so that the ranks' shares of the Eq. 6 load estimate
    are as equal as the planes allow, each slab at least one cell (>= r_c)
    thick."""
    costs, nc = cell_costs(r, box, rc)
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


class Domain:
    """One rank's slab [lo, hi) along `axis` of the periodic box."""

    def __init__(self, rank, world, box, rc, axis, bounds):
        self.rank, self.world = rank, world
        self.box = np.asarray(box, float)
        self.rc, self.axis = float(rc), axis
        self.lo, self.hi = float(bounds[rank]), float(bounds[rank + 1])
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


def _exchange(arrays_to_left, arrays_to_right, domain, dist, group=None):
    """Sends one dict of arrays to each neighbour and receives theirs
    (counts first, then float64 payloads; non-blocking pairs, no ordering
    deadlock).  Host tensors: under NCCL pass a gloo group.  Returns
    (from_left, from_right)."""
    import torch
    keys = sorted(arrays_to_left)
    widths = {k: (arrays_to_left[k].shape[1] if arrays_to_left[k].ndim == 2 else 1) for k in keys}

    def pack(d):
        n = next(iter(d.values())).shape[0]
        return torch.from_numpy(np.concatenate([np.asarray(d[k], float).reshape(n, widths[k]) for k in keys], axis=1)
                                .reshape(-1).copy()), n

    def unpack(t, n):
        a = t.numpy().reshape(n, -1) if n else np.zeros((0, sum(widths.values())))
        out, c = {}, 0
        for k in keys:
            w = widths[k]
            out[k] = a[:, c:c + w] if w > 1 or arrays_to_left[k].ndim == 2 else a[:, c]
            c += w
        return out

    pl, nl = pack(arrays_to_left)
    pr, nr = pack(arrays_to_right)
    cnt_in_l, cnt_in_r = torch.zeros(1, dtype=torch.int64), torch.zeros(1, dtype=torch.int64)
    reqs = [dist.isend(torch.tensor([nl], dtype=torch.int64), domain.left, group=group, tag=1),
            dist.isend(torch.tensor([nr], dtype=torch.int64), domain.right, group=group, tag=2),
            dist.irecv(cnt_in_r, domain.right, group=group, tag=1), dist.irecv(cnt_in_l, domain.left, group=group, tag=2)]
    for q in reqs:
        q.wait()
    width = sum(widths.values())
    buf_l = torch.zeros(int(cnt_in_l.item()) * width, dtype=torch.float64)
    buf_r = torch.zeros(int(cnt_in_r.item()) * width, dtype=torch.float64)
    reqs = []
    if nl:
        reqs.append(dist.isend(pl, domain.left, group=group, tag=3))
    if nr:
        reqs.append(dist.isend(pr, domain.right, group=group, tag=4))
    if buf_r.numel():
        reqs.append(dist.irecv(buf_r, domain.right, group=group, tag=3))
    if buf_l.numel():
        reqs.append(dist.irecv(buf_l, domain.left, group=group, tag=4))
    for q in reqs:
        q.wait()
    return unpack(buf_l, int(cnt_in_l.item())), unpack(buf_r, int(cnt_in_r.item()))


class DecomposedSystem:
    """The owned molecules of one rank (global ids kept with them) and the
    per-step halo exchange, local evaluation and migration."""

    STATE = ("r", "v", "q", "j")

    def __init__(self, domain, bounds, backend, state, ids, dist, group=None):
        self.dom, self.bounds, self.be, self.dist, self.group = domain, bounds, backend, dist, group
        self.st = {k: np.ascontiguousarray(state[k], float) for k in self.STATE}
        self.ids = np.asarray(ids, np.int64)

    @classmethod
    def scatter_from(cls, rank, world, cfg, backend, dist, group=None):
        """Every rank holds the same full configuration (seeded input) and
        keeps the molecules of its slab."""
        axis, bounds, _ = partition(cfg["r"], cfg["box"], cfg["rc"], world)
        dom = Domain(rank, world, cfg["box"], cfg["rc"], axis, bounds)
        mine = np.nonzero(dom.owner(cfg["r"], bounds) == rank)[0]
        return cls(dom, bounds, backend, {k: cfg[k][mine] for k in cls.STATE}, mine, dist, group)

    def _halo(self):
        if self.dom.world == 1:  # the periodic box itself: no halo
            return {**{k: self.st[k][:0] for k in self.STATE}, "ids": np.zeros(0)}
        to_l, to_r = self.dom.halo_out(self.st["r"])
        pick = lambda ix: {**{k: self.st[k][ix] for k in self.STATE}, "ids": self.ids[ix].astype(float)}
        from_l, from_r = _exchange(pick(to_l), pick(to_r), self.dom, self.dist, self.group)
        halo = {k: np.concatenate([from_l[k], from_r[k]]) for k in (*self.STATE, "ids")}
        if self.dom.world == 2:  # both neighbours are the same rank: a molecule near both faces came twice
            _, keep = np.unique(halo["ids"], return_index=True)
            halo = {k: v[np.sort(keep)] for k, v in halo.items()}
        return halo

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
        that left the slab.  NVE only when T_target <= 0 (the velocity-
        rescaling factor needs a global kinetic energy: not offered)."""
        if T_target > 0:
            raise NotImplementedError("velocity rescaling is not offered across domains")
        halo = self._halo()
        n = self.ids.shape[0]
        full = {k: np.concatenate([self.st[k], halo[k]]) for k in self.STATE}
        new = self.be.step(full, dt)
        self.st = {k: np.ascontiguousarray(new[k][:n]) for k in self.STATE}
        self._migrate()

    def _migrate(self):
        if self.dom.world == 1:
            return
        own = self.dom.owner(self.st["r"], self.bounds)
        # after one step a molecule moves far less than a slab: only to a neighbour
        go_l = np.nonzero(own == self.dom.left)[0]
        go_r = np.nonzero((own == self.dom.right) & (own != self.dom.left))[0]
        stay = np.nonzero(own == self.dom.rank)[0]
        if own.size and np.setdiff1d(np.nonzero(own != self.dom.rank)[0], np.concatenate([go_l, go_r])).size:
            raise RuntimeError("a molecule moved past a neighbouring slab in one step")
        pick = lambda ix: {**{k: self.st[k][ix] for k in self.STATE}, "ids": self.ids[ix].astype(float)}
        from_l, from_r = _exchange(pick(go_l), pick(go_r), self.dom, self.dist, self.group)
        self.st = {k: np.concatenate([self.st[k][stay], from_l[k], from_r[k]]) for k in self.STATE}
        self.ids = np.concatenate([self.ids[stay], from_l["ids"].astype(np.int64), from_r["ids"].astype(np.int64)])


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
