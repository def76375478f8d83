"""Spatial domain decomposition (§4: slabs or the tree-based bricks of
§4.3, balanced by the load cost of Eq. 6, one halo exchange per step,
migration, dynamic rebalancing) with 2-4 gloo ranks on the host.  The local
evaluation on each rank is the FP64 oracle (the GPU library takes its
place on GPUs): the decomposed forces, energies, virials, pair counts and
short trajectories must equal the single-domain oracle's."""
import os
import socket

import numpy as np
import pytest

import mdgen

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1408_4599_gb300 import domain  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleBackend:
    """Local evaluation by the FP64 oracle (linked cells, one thread)."""

    def __init__(self, cfg):
        import oracle
        self.oracle, self.cfg = oracle, cfg
        self.setup = oracle.setup_from_config(cfg)

    def forces(self, r, q):
        F, tau, o = self.oracle.forces(self.cfg["model"], self.setup, r, q, use_cells=True, n_threads=1)
        return F, tau, {"U": o["U"], "W": o["W"], "Wxx": o["Wxx"], "Wyy": o["Wyy"], "Wzz": o["Wzz"],
                        "n_mol_pairs": o["n_mol_pairs"]}

    def step(self, st, dt):
        return self.oracle.step(self.cfg["model"], self.setup, st, dt, 1, use_cells=True, n_threads=1)


def _slab_fast():
    """The slab moving as a whole along z at speed 25 (a Galilean boost: the
    forces are unchanged), so that the molecules within 0.3 sigma of a slab
    face cross it in six steps of 0.002."""
    cfg = mdgen.config_slab(n=24000)
    cfg["v"] = cfg["v"].copy()
    cfg["v"][:, 2] += 25.0
    return cfg


def _2cljq_fast():
    """The 2CLJQ fluid moving as a whole along (1, 1, 1) at speed 30 per
    axis (Galilean boost), so that molecules cross brick faces of every
    orientation within a few steps of 0.001."""
    cfg = mdgen.config_2cljq(n=2500)
    cfg["v"] = cfg["v"] + 30.0
    return cfg


CASES = {
    "2cljq": lambda: mdgen.config_2cljq(n=2500),
    "2cljq-fast": _2cljq_fast,
    "slab": lambda: mdgen.config_slab(n=24000),
    "slab-fast": _slab_fast,
    "4site": lambda: mdgen.config_4site(n=1500),
}


def _rank_main(rank, world, port, case, n_steps, out, method="slab", rebalance_at=-1, rebalance_every=0):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cfg = CASES[case]()
    ds = domain.DecomposedSystem.scatter_from(rank, world, cfg, OracleBackend(cfg), dist, method=method,
                                              rebalance_every=rebalance_every)
    F, tau = ds.forces()
    obs = ds.observables()
    res = {"ids0": ds.ids.copy(), "F": F, "tau": tau, "obs": obs, "bounds": ds.bounds}
    for k in range(n_steps):
        if k == rebalance_at:
            before = ds.bounds
            ds.rebalance()
            res["rebalanced"] = {"before": before, "after": ds.bounds,
                                 "owned_here": bool(np.all(ds.dom.owner_of(ds.st["r"]) == rank))}
        ds.step(cfg["dt"])
    res.update({"ids": ds.ids.copy(), **{k: ds.st[k].copy() for k in ("r", "v", "q", "j")}})
    res["owned_here"] = bool(np.all(ds.dom.owner_of(ds.st["r"]) == rank))
    out[rank] = res
    dist.destroy_process_group()


def _run(case, world, n_steps=0, method="slab", rebalance_at=-1, rebalance_every=0):
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), case, n_steps, out, method, rebalance_at, rebalance_every),
                 nprocs=world, join=True)
        return [out[k] for k in range(world)]


def _single(case, n_steps=0):
    import oracle
    cfg = CASES[case]()
    s = oracle.setup_from_config(cfg)
    F, tau, o = oracle.forces(cfg["model"], s, cfg["r"], cfg["q"], use_cells=True)
    st = {k: cfg[k] for k in ("r", "v", "q", "j")}
    for _ in range(n_steps):
        st = oracle.step(cfg["model"], s, st, cfg["dt"], 1, use_cells=True)
    return cfg, F, tau, o, st


@pytest.mark.parametrize("case,world,method", [("2cljq", 2, "slab"), ("2cljq", 3, "slab"), ("slab", 4, "slab"),
                                               ("4site", 2, "slab"), ("2cljq", 3, "kd"), ("2cljq", 4, "kd"),
                                               ("slab", 4, "kd"), ("4site", 2, "kd")])
def test_decomposed_forces_and_observables_equal_single_domain(case, world, method):
    res = _run(case, world, method=method)
    cfg, F, tau, o, _ = _single(case)
    ids = np.concatenate([r["ids0"] for r in res])
    assert np.array_equal(np.sort(ids), np.arange(cfg["r"].shape[0]))  # every molecule owned once
    Fd, td = np.concatenate([r["F"] for r in res]), np.concatenate([r["tau"] for r in res])
    sc = np.abs(F).max()
    assert np.allclose(Fd, F[ids], rtol=0, atol=1e-11 * sc)
    if np.abs(tau).max() > 0:
        assert np.allclose(td, tau[ids], rtol=0, atol=1e-11 * np.abs(tau).max())
    obs = res[0]["obs"]
    for r in res[1:]:
        assert r["obs"] == obs  # all-reduced: the same on every rank
    assert obs["n_mol_pairs"] == pytest.approx(o["n_mol_pairs"], abs=1e-9)
    for k in ("U", "W", "Wxx", "Wyy", "Wzz"):
        assert obs[k] == pytest.approx(o[k], rel=1e-11, abs=1e-9 * o["abs_W"]), k


def test_slab_trajectory_with_periodic_rebalancing():
    """Six NVE steps of the boosted slab on three slabs repartitioned every
    two steps (rebalance_every): the state gathered by global id equals the
    single-domain trajectory and every molecule ends on the rank whose slab
    holds it."""
    n_steps = 6
    res = _run("slab-fast", 3, n_steps, method="slab", rebalance_every=2)
    cfg, _, _, _, st = _single("slab-fast", n_steps)
    ids = np.concatenate([r["ids"] for r in res])
    assert np.array_equal(np.sort(ids), np.arange(cfg["r"].shape[0]))
    assert all(r["owned_here"] for r in res)
    L = np.asarray(cfg["box"])
    for k in ("r", "v", "q", "j"):
        d = np.concatenate([r[k] for r in res]) - st[k][ids]
        if k == "r":
            d -= L * np.rint(d / L)
        assert np.abs(d).max() <= 1e-9 * max(1.0, np.abs(st[k]).max()), k


def test_decomposed_trajectory_with_migration():
    """Six NVE steps of the slab with fast vapour molecules: some migrate to
    a neighbouring slab, every molecule is still owned exactly once, and the
    decomposed state, gathered by global id, equals the single-domain
    trajectory."""
    n_steps = 6
    res = _run("slab-fast", 3, n_steps)
    cfg, _, _, _, st = _single("slab-fast", n_steps)
    ids = np.concatenate([r["ids"] for r in res])
    assert np.array_equal(np.sort(ids), np.arange(cfg["r"].shape[0]))
    moved = sum(int(np.setdiff1d(r["ids"], r["ids0"]).size) for r in res)
    L = np.asarray(cfg["box"])
    for k in ("r", "v", "q", "j"):
        a = np.concatenate([r[k] for r in res])
        b = st[k][ids]
        d = a - b
        if k == "r":
            d -= L * np.rint(d / L)
        assert np.abs(d).max() <= 1e-9 * max(1.0, np.abs(b).max()), k
    assert moved > 0


def test_kd_trajectory_with_migration_and_rebalance():
    """Six NVE steps of the boosted 2CLJQ fluid on four bricks of the
    tree-based decomposition, rebalanced after the third step from the
    summed cell histograms: molecules migrate across brick faces, every
    molecule is owned exactly once by the rank whose brick holds it, and the
    state gathered by global id equals the single-domain trajectory."""
    n_steps = 6
    res = _run("2cljq-fast", 4, n_steps, method="kd", rebalance_at=3)
    cfg, _, _, _, st = _single("2cljq-fast", n_steps)
    ids = np.concatenate([r["ids"] for r in res])
    assert np.array_equal(np.sort(ids), np.arange(cfg["r"].shape[0]))
    assert all(r["owned_here"] and r["rebalanced"]["owned_here"] for r in res)
    assert all(r["rebalanced"]["after"] == res[0]["rebalanced"]["after"] for r in res)  # one partition
    moved = sum(int(np.setdiff1d(r["ids"], r["ids0"]).size) for r in res)
    assert moved > 0
    L = np.asarray(cfg["box"])
    for k in ("r", "v", "q", "j"):
        a = np.concatenate([r[k] for r in res])
        b = st[k][ids]
        d = a - b
        if k == "r":
            d -= L * np.rint(d / L)
        assert np.abs(d).max() <= 1e-9 * max(1.0, np.abs(b).max()), k


def _brute_best_cut(costs, axis, lo, hi, p_lo, p_hi, min_cells):
    """The least-imbalance plane along `axis` of the region lo..hi, by trying
    every admissible plane one by one."""
    best, best_c = None, None
    for c in range(lo[axis] + min_cells * p_lo, hi[axis] - min_cells * p_hi + 1):
        sl_lo = [slice(lo[a], hi[a]) for a in range(3)]
        sl_hi = [slice(lo[a], hi[a]) for a in range(3)]
        sl_lo[axis] = slice(lo[axis], c)
        sl_hi[axis] = slice(c, hi[axis])
        a_ = costs[sl_lo[2], sl_lo[1], sl_lo[0]].sum() / p_lo
        b_ = costs[sl_hi[2], sl_hi[1], sl_hi[0]].sum() / p_hi
        if best is None or max(a_, b_) < best - 1e-12:
            best, best_c = max(a_, b_), c
    return best_c


def test_kd_partition_tiles_the_grid_and_balances():
    """Tree-based decomposition (§4.3): the bricks tile the cell grid, each
    at least two cells along every axis; the first cut is perpendicular to
    x at the least-imbalance plane (checked by trying every plane), the
    second ones perpendicular to y; and on the vapour-liquid slab the
    bricks' shares of the Eq. 6 cost are far more even than an equal-volume
    split along the long axis."""
    for cfg in (mdgen.config_slab(n=24000), mdgen.config_2cljq(n=2500)):
        costs, nc = domain.cell_costs(cfg["r"], cfg["box"], cfg["rc"])
        for world in (2, 3, 4, 5, 8):
            bricks, shares = domain.partition_kd(costs, world)
            cover = np.zeros_like(costs, dtype=int)
            for lo, hi in bricks:
                assert all(hi[a] - lo[a] >= 2 for a in range(3))
                cover[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] += 1
            assert (cover == 1).all()
            assert sum(shares) == pytest.approx(costs.sum())
        full = ((0, 0, 0), tuple(nc))
        bricks, _ = domain.partition_kd(costs, 2)
        c = _brute_best_cut(costs, 0, full[0], full[1], 1, 1, 2)
        assert bricks[0] == ((0, 0, 0), (c, nc[1], nc[2])) and bricks[1] == ((c, 0, 0), tuple(nc))
        bricks, _ = domain.partition_kd(costs, 4)
        assert bricks[0][1][0] == bricks[1][1][0] and bricks[0][1][1] < nc[1]  # x first, then y
    cfg = mdgen.config_slab(n=24000)
    costs, nc = domain.cell_costs(cfg["r"], cfg["box"], cfg["rc"])
    _, shares = domain.partition_kd(costs, 4)
    mean = costs.sum() / 4
    assert max(shares) <= 1.2 * mean
    layer = costs.sum(axis=(1, 2))  # equal-volume split along z
    eq = [layer[k * nc[2] // 4:(k + 1) * nc[2] // 4].sum() for k in range(4)]
    assert max(eq) > 1.5 * mean


def test_kd_partition_rejects_too_many_ranks():
    cfg = mdgen.config_lj_fluid(n=500)
    costs, nc = domain.cell_costs(cfg["r"], cfg["box"], cfg["rc"])
    with pytest.raises(ValueError):
        domain.partition_kd(costs, (nc[0] // 2) * (nc[1] // 2) * (nc[2] // 2) + 1)


def test_partition_balances_the_eq6_cost():
    """Slab boundaries on cell planes, every slab at least one plane thick,
    and each rank's share of the load estimate within one cell plane's cost
    of the mean (the vapour-liquid slab: a uniform split by volume would put
    most of the liquid on the middle ranks)."""
    cfg = mdgen.config_slab(n=24000)
    costs, nc = domain.cell_costs(cfg["r"], cfg["box"], cfg["rc"])
    for world in (2, 3, 4, 7):
        axis, bounds, share = domain.partition(cfg["r"], cfg["box"], cfg["rc"], world)
        assert axis == 2
        ell = cfg["box"][2] / nc[2]
        planes = [b / ell for b in bounds]
        assert all(abs(p - round(p)) < 1e-9 for p in planes)
        assert all(round(planes[k + 1]) > round(planes[k]) for k in range(world))
        layer = costs.sum(axis=(1, 2))
        assert sum(share) == pytest.approx(costs.sum())
        assert max(abs(s - costs.sum() / world) for s in share) <= layer.max() + 1e-9
    # the Eq. 6 estimate follows the occupation: liquid planes dominate
    layer = costs.sum(axis=(1, 2))
    assert layer.max() > 50 * layer[layer > 0].min()


def test_partition_rejects_more_slabs_than_cell_planes():
    cfg = mdgen.config_lj_fluid(n=500)
    nc = domain.cell_grid(cfg["box"], cfg["rc"])
    with pytest.raises(ValueError):
        domain.partition(cfg["r"], cfg["box"], cfg["rc"], max(nc) + 1)


def test_kd_partition_properties_on_random_grids():
    """On random cell grids and random, partly empty Eq. 6 costs: whenever
    bricks of at least two cells per axis exist for `world` ranks, they tile
    the grid, their shares add up to the total, and the brick count fits
    the grid's volume; otherwise the partition refuses with ValueError."""
    rng = np.random.default_rng(14080)
    for _ in range(60):
        nc = rng.integers(2, 13, size=3)
        costs = rng.exponential(1.0, size=(nc[2], nc[1], nc[0])) * (rng.random((nc[2], nc[1], nc[0])) < 0.7)
        world = int(rng.integers(1, 10))
        try:
            bricks, shares = domain.partition_kd(costs, world)
        except ValueError:
            assert world > 1
            continue
        assert len(bricks) == world
        assert world <= (nc[0] // 2) * (nc[1] // 2) * (nc[2] // 2)
        cover = np.zeros(costs.shape, dtype=int)
        for lo, hi in bricks:
            assert all(hi[a] - lo[a] >= 2 for a in range(3))
            cover[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] += 1
        assert (cover == 1).all()
        assert sum(shares) == pytest.approx(costs.sum())


def test_kd_coarse_levels_halve_by_volume_and_share_ranks_by_cost():
    """The simplified first levels of §4.3 for very large volumes: a region
    larger than `coarse_cells` is halved at its middle plane, and its ranks
    go to the halves in proportion to their costs; smaller regions are cut
    by the least-imbalance plane as before."""
    nc = (16, 8, 8)
    costs = np.ones((nc[2], nc[1], nc[0]))
    costs[:, :, :4] += 5.0  # the lower x half carries 3/4 of the load
    bricks, shares = domain.partition_kd(costs, 8, coarse_cells=16 * 8 * 8 - 1)
    lower = [b for b in bricks if b[1][0] <= 8]
    assert all(b[0][0] >= 8 or b[1][0] <= 8 for b in bricks)  # nothing straddles the middle plane
    assert len(lower) == 6  # 8 ranks x 3/4 of the cost
    cover = np.zeros(costs.shape, dtype=int)
    for lo, hi in bricks:
        cover[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] += 1
    assert (cover == 1).all()
    # without coarse levels the first cut is the least-imbalance plane for
    # 4 + 4 ranks instead: x = 3, where the cost is halved
    exact, _ = domain.partition_kd(costs, 8)
    assert sum(1 for b in exact if b[1][0] <= 3) == 4
    assert all(b[0][0] >= 3 or b[1][0] <= 3 for b in exact)
