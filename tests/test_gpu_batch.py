"""Batched replicas (md_batch_*): one launch per kernel over many uneven
systems must give every replica the same result as evaluating it alone,
and the FP64 oracle's result within the force-parity tolerances."""
import math

import numpy as np
import pytest

import mdgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1408_4599_gb300 import md  # noqa: E402
from test_gpu_parity import check_parity, rel_err  # noqa: E402


def _replicas(n_rep=9, n_min=300, n_max=3000, seed_k=3):
    specs = mdgen.replica_specs(n_rep, n_min, n_max, seed_k=seed_k)
    cfgs = []
    for k, (n, rho, T) in enumerate(specs):
        rho = max(rho, 0.1)
        if (n / rho) ** (1 / 3) < 6.0:  # box >= 2 rc
            rho = n / 6.0 ** 3
        cfgs.append(mdgen.config_replica(k, n, rho, T))
    return cfgs


def _split(a, cfgs):
    out, s = [], 0
    for c in cfgs:
        n = c["r"].shape[0]
        out.append(a[s:s + n])
        s += n
    return out


@pytest.mark.parametrize("half", [1, 0])
def test_batch_forces_match_oracle_per_replica(half):
    cfgs = _replicas()
    assert any(min(int(L // 3.0) for L in c["box"]) < 3 for c in cfgs)  # includes small boxes
    b = md.Batch(cfgs, half_shell=half).set()
    b.compute_forces()
    F, tau = b.forces()
    obs = b.observables()
    b.close()
    for c, Fk, tk, ok in zip(cfgs, _split(F, cfgs), _split(tau, cfgs), obs):
        s = oracle.setup_from_config(c)
        Fo, to, oo = oracle.forces(c["model"], s, c["r"], c["q"], use_cells=True)
        ncs = [int(math.floor(L / (c["rc"] * (1 + 1e-9)))) for L in c["box"]]
        check_parity(f"batch/{c['name']}/half{half}", c, Fk, tk, ok, Fo, to, oo, exact_examined=min(ncs) >= 3)
        assert ok["n_molecules"] == c["r"].shape[0]


def test_batch_equals_single_systems():
    """Full stencil everywhere: the batched kernels and the single-system
    kernels do the same arithmetic in the same order per molecule, except
    that the batch keeps each molecule's FP64 force and torque totals in its
    FP32 records (read by the batched integrator of mixed-shell replicas),
    where the single system keeps them in FP64.  That rounding (2^-24 of a
    molecule's total; forces reach ~1e4 in these overlapping lattice starts)
    bounds the velocity difference after six steps by ~6 dt 2^-24 F_max / m
    (a few roundings: 1e-6 relative is allowed), the positions by dt times
    that; any difference in the arithmetic itself would show at the level of
    the forces."""
    cfgs = _replicas(n_rep=6, seed_k=5)
    b = md.Batch(cfgs, half_shell=0).set()
    b.step(6, 0.001, use_graph=False)
    rb, vb, qb, jb = b.molecules()
    obs_b = b.observables()
    b.close()
    for c, r, v, q, o_b in zip(cfgs, _split(rb, cfgs), _split(vb, cfgs), _split(qb, cfgs), obs_b):
        s = md.System(c, deterministic=1)
        s.set(c["r"], c["q"], c["v"], c["j"])
        s.step(6, 0.001)
        r1, v1, q1, j1 = s.molecules()
        o1 = s.observables()
        F1, _ = s.forces()
        s.close()
        L = np.array(c["box"])
        dr = r - r1
        dr -= L * np.rint(dr / L)
        dv_tol = 1e-6 * 6 * 0.001 * np.abs(F1).max() / mdgen.model_mass(c["model"])
        assert np.abs(v - v1).max() < dv_tol and np.abs(dr).max() < 6 * 0.001 * dv_tol
        assert np.abs(q - q1).max() < 1e-7
        assert o_b["n_mol_pairs"] == o1["n_mol_pairs"]
        assert o_b["U_pot"] == pytest.approx(o1["U_pot"], rel=1e-6, abs=1e-9)
        assert o_b["K_trans"] == pytest.approx(o1["K_trans"], rel=1e-6)
        assert o_b["K_rot"] == pytest.approx(o1["K_rot"], rel=1e-6)
        assert o_b["U_lrc"] == pytest.approx(o1["U_lrc"], rel=1e-12)


def test_graph_replay_equals_eager_steps():
    cfgs = _replicas(n_rep=5, seed_k=7)
    res, obs = [], []
    for use_graph in (False, True):
        b = md.Batch(cfgs, half_shell=0).set()
        b.step(5, 0.001, use_graph=use_graph)   # 2 graph replays + 1 eager step
        o5 = b.observables()
        b.step(4, 0.001, use_graph=use_graph)   # other buffer parity; replays graphs captured above
        res.append(b.molecules())
        o = b.observables()
        assert all(x["step"] == 9 for x in o)
        obs.append(o5 + o)
        b.close()
    for a, c in zip(res[0], res[1]):
        assert np.array_equal(a, c)
    # the observables after a replay come from that replay's forces (no stale FP64 copy)
    for a, c in zip(obs[0], obs[1]):
        for k in ("U_pot", "W", "K_trans", "K_rot", "n_mol_pairs"):
            assert a[k] == c[k], k


def test_tuner_and_nve_energy():
    cfgs = _replicas(n_rep=6, seed_k=9)
    for c in cfgs:
        c["v"] *= 0.3
        c["j"] *= 0.3
    b = md.Batch(cfgs, half_shell=1).set()
    t = b.tune()
    assert t["chunk"] in (1, 2, 4, 8, 16) and t["grid_pct"] in (50, 100) and t["force_ms"] > 0
    b.step(2, 0.0005)
    e0 = [o["U_pot"] + o["K_trans"] + o["K_rot"] for o in b.observables()]
    b.step(20, 0.0005)
    e1 = [o["U_pot"] + o["K_trans"] + o["K_rot"] for o in b.observables()]
    b.close()
    for a, c, cfg in zip(e0, e1, cfgs):
        assert np.isfinite(c)
        # no blow-up: lattice starts with overlapping sites carry large energies;
        # the centre-of-mass cut-off also lets E jump when pairs cross r_c
        assert abs(c - a) < 0.01 * max(abs(a), cfg["r"].shape[0])


def test_batch_argument_errors():
    cfgs = _replicas(n_rep=2)
    boxes = np.array([c["box"] for c in cfgs], dtype=np.float64)
    boxes[1, 2] = 5.0  # < 2 rc
    L = md.lib()
    M = md.Model(cfgs[0]["model"])
    h = md.C.c_void_p()
    o = md.md_options(math.inf, 0, 1, 0, 1)
    assert L.md_batch_create(2, boxes.ctypes.data_as(md.dp), 3.0, md.C.byref(M.types), md.C.byref(o),
                             md.C.byref(h)) == -2
    b = md.Batch(cfgs)
    with pytest.raises(md.MDError) as e:
        b.compute_forces()
    assert e.value.code == -3
    b.close()


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_nvt_matches_single_systems(use_graph):
    """Per-replica velocity rescaling (§2 NVT): the batched step with a
    target per replica (one replica left NVE) equals each replica's own
    md_step with that target (to the rounding of the batch's FP32 force
    records), and each thermostatted replica's half-step temperature equals
    its target."""
    from test_oracle_pins import _half_step_temperature
    cfgs = _replicas(n_rep=5, seed_k=11)
    targets = [0.8, 1.5, 0.0, 1.1, 2.0]
    b = md.Batch(cfgs, half_shell=0).set()
    b.set_thermostat(targets)
    b.step(6, 0.001, use_graph=use_graph)
    rb, vb, qb, jb = b.molecules()
    b.close()
    for c, T, r, v, q, j in zip(cfgs, targets, _split(rb, cfgs), _split(vb, cfgs), _split(qb, cfgs), _split(jb, cfgs)):
        s = md.System(c, deterministic=1)
        s.set(c["r"], c["q"], c["v"], c["j"])
        s.step(6, 0.001, T_target=T)
        r1, v1, q1, j1 = s.molecules()
        F1, t1 = s.forces()
        s.close()
        L = np.array(c["box"])
        dr = r - r1
        dr -= L * np.rint(dr / L)
        # FP32 records in the batch, FP64 totals in the single system (the
        # bound of test_batch_equals_single_systems)
        dv_tol = 1e-6 * 6 * 0.001 * np.abs(F1).max() / mdgen.model_mass(c["model"])
        assert np.abs(v - v1).max() < dv_tol and np.abs(dr).max() < 6 * 0.001 * dv_tol
        assert np.abs(j - j1).max() < 1e-6 * 6 * 0.001 * np.abs(t1).max()
        if T > 0:
            assert _half_step_temperature(c["model"], v, q, j) == pytest.approx(T, rel=1e-6)


def test_batch_thermostat_argument_errors():
    cfgs = _replicas(n_rep=2)
    b = md.Batch(cfgs)
    with pytest.raises(ValueError):
        b.set_thermostat([1.0])
    with pytest.raises(md.MDError) as e:
        b.set_thermostat([1.0, math.nan])
    assert e.value.code == -1
    b.set_thermostat(None)
    b.close()


def test_full_size_batch_sampled_parity():
    """The batched workload at full size (512 replicas, 2.61 M molecules,
    half shell where a replica has >= 3 cells per axis): forces of every
    replica in one launch, eight seeded replicas checked in full against
    the oracle."""
    specs = mdgen.replica_specs(512)
    cfgs = [mdgen.config_replica(k, n, min(rho, n / 216.0), T) for k, (n, rho, T) in enumerate(specs)]
    b = md.Batch(cfgs, half_shell=1).set()
    b.tune()
    b.compute_forces()
    F, tau = b.forces()
    obs = b.observables()
    b.close()
    Fs, ts = _split(F, cfgs), _split(tau, cfgs)
    for k in sorted(np.random.default_rng(1408_0499).choice(len(cfgs), 8, replace=False)):
        c = cfgs[k]
        s = oracle.setup_from_config(c)
        Fo, to, oo = oracle.forces(c["model"], s, c["r"], c["q"], use_cells=True)
        ncs = [int(math.floor(L / (c["rc"] * (1 + 1e-9)))) for L in c["box"]]
        check_parity(f"batch512/{c['name']}", c, Fs[k], ts[k], obs[k], Fo, to, oo, exact_examined=min(ncs) >= 3)


def test_tile_tuner_choices_cache_and_results(tmp_path):
    """md_batch_tune_tiles on a dilute and a dense replica set: the chosen
    tiles are among the candidates and no slower than the defaults (which
    are candidates), the forces with the chosen tiles agree with the
    defaults' within the parity tolerance (the tiles change only the
    summation order and the stencil form), the two sets fall in different
    occupancy buckets of the cache key, and a second call takes the cached
    choice without timing."""
    cache = str(tmp_path / "tune.txt")
    keys = set()
    for name, rho in (("dilute", 0.06), ("dense", 0.7)):
        cfgs = [mdgen.config_replica(k, 1500 + 400 * k, rho, 1.0) for k in range(6)]
        b = md.Batch(cfgs, half_shell=1).set()
        b.compute_forces()
        F0, t0 = b.forces()
        t = b.tune_tiles(cache)
        assert t["from_cache"] == 0
        assert t["chunk"] in (1, 2, 4, 8) and t["grid_pct"] in (100, 50) and t["test_width"] in (4, 8)
        assert t["half_min_occ"] in (0.0, 2.0, 6.0)
        assert t["ms"] <= 1.15 * t["default_ms"], t
        b.compute_forces()
        F1, t1 = b.forces()
        ef, et = rel_err(F1, F0), rel_err(t1, t0)
        assert np.median(ef) <= 1e-5 and ef.max() <= 1e-3
        assert np.median(et) <= 1e-5 and et.max() <= 1e-3
        t2 = b.tune_tiles(cache)
        assert t2["from_cache"] == 1 and t2["key"] == t["key"]
        assert (t2["chunk"], t2["grid_pct"], t2["test_width"], t2["half_min_occ"]) == \
            (t["chunk"], t["grid_pct"], t["test_width"], t["half_min_occ"])
        keys.add(t["key"])
        b.close()
    assert len(keys) == 2
