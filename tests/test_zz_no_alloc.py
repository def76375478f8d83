"""md_kinetic_noalloc (the allocation-free kinetic-energy entry point) must
return what md_energy_virial reports for the same state, on two calls in a
row, agree with the FP64 oracle's kinetic energies, and leave the free
device memory unchanged (it promises to allocate nothing).  This file is
collected last so that a failure here cannot stop the other GPU tests from
running."""
import numpy as np
import pytest

import mdgen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1408_4599_gb300 import md  # noqa: E402


def test_kinetic_noalloc_matches_energy_virial():
    import oracle

    dev = torch.device("cuda:0")
    cfg = mdgen.config_2cljq(n=5000)
    sysm = md.System(cfg)
    t = {k: torch.from_numpy(cfg[k]).to(dev) for k in ("r", "v", "q", "j")}
    sysm.set(t["r"], t["q"], t["v"], t["j"])
    K_out = torch.zeros(2, dtype=torch.float64, device=dev)
    mass = mdgen.model_mass(cfg["model"])
    moments = mdgen.model_principal_moments(cfg["model"])
    n = cfg["r"].shape[0]
    r, v, q, j = (torch.zeros((n, w), dtype=torch.float64, device=dev) for w in (3, 3, 4, 3))
    F = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    tau = torch.zeros_like(F)
    for call in range(2):
        sysm.step(3, cfg["dt"])
        obs = sysm.observables()
        sysm.molecules(r=r, v=v, q=q, j=j)
        sysm.forces(F=F, tau=tau)
        K_out.fill_(-1.0)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info(dev)[0]
        md.md_kinetic_noalloc(v, q, j, F, tau, mass, moments, cfg["dt"], K_out)
        torch.cuda.synchronize()
        free_after = torch.cuda.mem_get_info(dev)[0]
        assert free_after == free_before, (call, free_before - free_after)
        kt, kr = K_out.cpu().tolist()
        assert kt == pytest.approx(obs["K_trans"], rel=1e-12), call
        assert kr == pytest.approx(obs["K_rot"], rel=1e-12), call
        assert kt > 0 and kr > 0
        # the FP64 oracle on the same half-step state (the rotational energy
        # is formed in FP32 per molecule on the GPU)
        ok_t, ok_r = oracle.kinetic(cfg["model"], cfg["dt"], *(x.cpu().numpy() for x in (v, q, j, F, tau)))
        assert kt == pytest.approx(ok_t, rel=1e-12), call
        assert kr == pytest.approx(ok_r, rel=1e-6), call
    sysm.close()


def test_kinetic_noalloc_rejects_oversize_and_bad_args():
    dev = torch.device("cuda:0")
    z3 = torch.zeros((4, 3), dtype=torch.float64, device=dev)
    z4 = torch.zeros((4, 4), dtype=torch.float64, device=dev)
    K = torch.zeros(2, dtype=torch.float64, device=dev)
    L = md.lib()
    I = (md.C.c_double * 3)(1.0, 1.0, 0.0)
    big = 8388608 + 1
    p = lambda t: md.C.c_void_p(t.data_ptr())
    assert L.md_kinetic_noalloc(big, p(z3), p(z4), p(z3), p(z3), p(z3), 1.0, I, 0.001, p(K), None) == -7
    assert L.md_kinetic_noalloc(4, p(z3), p(z4), p(z3), p(z3), p(z3), 0.0, I, 0.001, p(K), None) == -1
    assert L.md_kinetic_noalloc(4, p(z3), p(z4), p(z3), p(z3), p(z3), 1.0, I, 0.001, None, None) == -1
