"""The 200M-molecule single-evaluation point of the slab workload (a
homogeneous LJTS fluid at rho = 0.73, L = 649.5 sigma, 259^3 cells): one
force evaluation in the bench's launch configuration (half shell), checked
against the FP64 oracle's exact forces on a seeded sample of 100,000
molecules (the oracle evaluates those one by one over the full cell list).

Needs ~70 GB of device memory and ~60 GB of host memory; skipped when the
machine has less free (checked before anything is allocated)."""
import os

import numpy as np
import pytest

import mdgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1408_4599_gb300 import md  # noqa: E402
from test_gpu_parity import _log  # noqa: E402

N_BIG = 200_000_000
N_SAMPLE = 100_000


def _host_available_gb():
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) / 1024 ** 2
    except OSError:
        pass
    return 0.0


def test_zz_200m_homogeneous_sampled_parity():
    free_dev = torch.cuda.mem_get_info()[0] / 1024 ** 3
    free_host = _host_available_gb()
    if free_dev < 120 or free_host < 150:
        pytest.skip(f"needs >= 120 GB free device and >= 150 GB available host memory "
                    f"(have {free_dev:.0f} / {free_host:.0f} GB)")
    cfg = mdgen.config_lj_homogeneous(N_BIG)
    n = cfg["r"].shape[0]
    s = md.System(cfg, deterministic=0, half_shell=1)
    s.set(cfg["r"], cfg["q"], cfg["v"], cfg["j"])
    s.compute_forces()
    dev = torch.device("cuda:0")
    F = torch.empty((n, 3), dtype=torch.float64, device=dev)
    tau = torch.empty((n, 3), dtype=torch.float64, device=dev)
    s.forces(F=F, tau=tau)
    obs = s.observables()
    s.close()
    del tau
    sel = np.sort(np.random.default_rng(1408_0399).choice(n, N_SAMPLE, replace=False))
    Fg = F[torch.from_numpy(sel).to(dev)].cpu().numpy()
    del F
    torch.cuda.empty_cache()
    Fo, _ = oracle.forces_subset(cfg["model"], oracle.setup_from_config(cfg), cfg["r"], cfg["q"], sel)
    frms = np.sqrt((Fo ** 2).sum(axis=1).mean())
    rel = np.linalg.norm(Fg - Fo, axis=1) / np.maximum(np.linalg.norm(Fo, axis=1), 0.01 * frms)
    # interacting pairs per molecule near rho (4 pi / 3) rc^3 / 2 for a homogeneous fluid
    expect = 0.5 * n * cfg["box"][0] ** -3 * n * (4.0 / 3.0) * np.pi * cfg["rc"] ** 3
    _log(case="lj-homog-200M/half1/sampled", n=n, sample=N_SAMPLE, med=float(np.median(rel)), max=float(rel.max()),
         mol_pairs=int(obs["n_mol_pairs"]), mol_pairs_expected=float(expect), U_per_mol=obs["U_pot"] / n)
    assert np.median(rel) <= 1e-5 and rel.max() <= 1e-3
    assert abs(obs["n_mol_pairs"] / expect - 1.0) < 0.08  # a jittered fcc lattice sits ~3% above
    assert np.isfinite(obs["U_pot"]) and obs["n_molecules"] == n
