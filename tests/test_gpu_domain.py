"""The domain decomposition's GPU path: two ranks (processes sharing cuda:0,
exchanging halos and migrants over gloo on the host; no kernel waits on
another rank) evaluate their owned + halo molecules with the CUDA library.
Forces, torques and the all-reduced energy, virial and pair counts meet the
parity tolerances against the single-domain FP64 oracle, and a short
trajectory keeps every molecule owned exactly once."""
import os
import socket

import numpy as np
import pytest

import mdgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from test_gpu_parity import rel_err  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    from paper_1408_4599_gb300 import domain
    cfg = mdgen.config_2cljq(n=6000)
    ds = domain.DecomposedSystem.scatter_from(rank, world, cfg, domain.GpuBackend(cfg), dist)
    F, tau = ds.forces()
    obs = ds.observables()
    ids0 = ds.ids.copy()
    for _ in range(3):
        ds.step(cfg["dt"])
    out[rank] = {"ids0": ids0, "F": F, "tau": tau, "obs": obs, "ids": ds.ids.copy()}
    dist.destroy_process_group()


def test_two_rank_decomposition_on_the_gpu():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = [out[k] for k in range(world)]
    cfg = mdgen.config_2cljq(n=6000)
    s = oracle.setup_from_config(cfg)
    Fo, to, oo = oracle.forces(cfg["model"], s, cfg["r"], cfg["q"], use_cells=True)
    ids = np.concatenate([r["ids0"] for r in res])
    assert np.array_equal(np.sort(ids), np.arange(cfg["r"].shape[0]))
    ef = rel_err(np.concatenate([r["F"] for r in res]), Fo[ids])
    et = rel_err(np.concatenate([r["tau"] for r in res]), to[ids])
    assert np.median(ef) <= 1e-5 and ef.max() <= 1e-3
    assert np.median(et) <= 1e-5 and et.max() <= 1e-3
    obs = res[0]["obs"]
    assert obs == res[1]["obs"]
    assert obs["n_mol_pairs"] == pytest.approx(oo["n_mol_pairs"], abs=1e-6)
    assert abs(obs["U"] - oo["U"]) <= 1e-5 * oo["abs_U"]
    assert abs(obs["W"] - oo["W"]) <= 1e-5 * oo["abs_W"]
    after = np.concatenate([r["ids"] for r in res])
    assert np.array_equal(np.sort(after), np.arange(cfg["r"].shape[0]))
