"""GPU parameter sensitivities (md_param_grad, the adjoint kernel) against
the FP64 oracle's analytic gradient, whose own pins are central finite
differences (tests/test_oracle_grad.py).

Tolerance: each component within 1e-5 of the sum over pairs of the
magnitudes of its per-pair terms (reported by the oracle): the FP32 pair
terms are summed in FP32 per lane and in FP64 per block, so the error of a
component is bounded by a few ulp of that sum, not of the (possibly
cancelling) component itself.  Mean U: 1e-5 of sum |u_ij|.
"""
import json
import math
import os

import numpy as np
import pytest

import mdgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1408_4599_gb300 import md  # noqa: E402
from paper_1408_4599_gb300.autograd import ensemble_uw  # noqa: E402

LOG = os.environ.get("MD_PARITY_LOG")


def _ensemble(name):
    if name == "4site-50000":  # the full-size configuration, four of its configurations
        cfgs = mdgen.configs_4site(4)
    elif name == "4site":
        cfgs = [mdgen.config_4site(n=3000, cfg=c) for c in range(3)]
    elif name == "2cljdq-rf":
        cfgs = [mdgen.config_replica(c, 2000, 0.6, 1.0) for c in range(3)]
    elif name == "2cljq":
        cfgs = [mdgen.config_2cljq(n=3000, seed_k=c) for c in range(2)]
    else:  # shifted single-site LJ
        cfgs = [mdgen.config_lj_fluid(n=2000, seed_k=c) for c in range(2)]
    box = cfgs[0]["box"]
    for c in cfgs:
        assert c["box"] == box
    return cfgs[0], np.stack([c["r"] for c in cfgs]), np.stack([c["q"] for c in cfgs])


def _close(d, d_ref, d_abs, rel=1e-5):
    return np.abs(d - d_ref) <= rel * d_abs + 1e-12 * np.abs(d_ref)


@pytest.mark.parametrize("name", ["4site", "2cljdq-rf", "2cljq", "ljts", "4site-50000"])
def test_param_grad_matches_oracle(name):
    cfg, r_all, q_all = _ensemble(name)
    s = oracle.setup_from_config(cfg)
    dUo, dWo, Uo, Wo, aU, aW = oracle.param_grad(cfg["model"], s, r_all, q_all, use_cells=True, with_abs=True)
    absU = np.mean([oracle.forces(cfg["model"], s, r, q, use_cells=True)[2]["abs_U"] for r, q in zip(r_all, q_all)])
    sysm = md.System(cfg)
    assert md.md_n_params(sysm.h) == len(dUo)
    dU, dW, U, W = sysm.param_grad(r_all, q_all)
    sysm.close()
    if LOG:
        with open(LOG, "a") as f:
            f.write(json.dumps({"case": "adjoint/" + name,
                                "dU_rel": (np.abs(dU - dUo) / np.maximum(np.abs(dUo), 1e-300)).tolist(),
                                "dW_rel": (np.abs(dW - dWo) / np.maximum(np.abs(dWo), 1e-300)).tolist(),
                                "U": [U, Uo], "W": [W, Wo]}) + "\n")
    assert abs(U - Uo) <= 1e-5 * absU
    assert np.all(_close(dU, dUo, aU)), (dU, dUo, aU)
    assert np.all(_close(dW, dWo, aW)), (dW, dWo, aW)
    # components that do not cancel heavily (|component| >= 1% of the sum of
    # its terms' magnitudes) also meet a plain relative bound
    for d, do, a in ((dU, dUo, aU), (dW, dWo, aW)):
        big = np.abs(do) >= 1e-2 * a
        rel = np.abs(d - do) / np.maximum(np.abs(do), 1e-300)
        assert np.all(rel[big] <= 1e-4), (rel, big)


def test_device_configurations_and_parameter_round_trip():
    cfg, r_all, q_all = _ensemble("4site")
    sysm = md.System(cfg)
    th0 = sysm.params()
    assert np.allclose(th0, oracle.model_param_vector(cfg["model"]))
    dev = torch.device("cuda:0")
    dU1, dW1, U1, W1 = sysm.param_grad(r_all, q_all)
    dU2, dW2, U2, W2 = sysm.param_grad(torch.from_numpy(r_all).to(dev), torch.from_numpy(q_all).to(dev))
    assert np.allclose(dU1, dU2, rtol=1e-12, atol=0) and U1 == pytest.approx(U2, rel=1e-12)
    th = th0.copy()
    th[0] *= 1.1
    th[4] = 0.3
    sysm.set_params(th)
    assert np.array_equal(sysm.params(), th)
    dU3, _, U3, _ = sysm.param_grad(r_all, q_all)
    so = oracle.setup_from_config(cfg)
    dUo, _, Uo, _, aU, _ = oracle.param_grad(oracle.model_with_params(cfg["model"], th), so, r_all, q_all,
                                             use_cells=True, with_abs=True)
    assert np.all(_close(dU3, dUo, aU))
    with pytest.raises(md.MDError):
        sysm.set_params(th[:-1])
    bad = th.copy()
    bad[2] = -1.0  # sigma must stay positive
    with pytest.raises(md.MDError):
        sysm.set_params(bad)
    assert np.array_equal(sysm.params(), th)
    sysm.close()


def test_autograd_function_backward():
    """EnsembleUW: forward = the ensemble means of one adjoint pass (equal to
    the force kernel's observables), backward = that pass's derivatives
    contracted with the incoming gradient."""
    cfg, r_all, q_all = _ensemble("2cljdq-rf")
    sysm = md.System(cfg)
    theta = torch.tensor(sysm.params(), dtype=torch.float64, requires_grad=True)
    out = ensemble_uw(theta, sysm, r_all, q_all)
    loss = 2.0 * out[0] - 0.5 * out[1]
    loss.backward()
    dU, dW, U, W = sysm.param_grad(r_all, q_all)
    assert out[0].item() == pytest.approx(U, rel=1e-12)
    assert out[1].item() == pytest.approx(W, rel=1e-12, abs=1e-12)
    assert np.allclose(theta.grad.numpy(), 2.0 * dU - 0.5 * dW, rtol=1e-12, atol=1e-12)
    # the means agree with the force kernel's observables
    Uf = Wf = 0.0
    for c in range(r_all.shape[0]):
        sysm.set(r_all[c], q_all[c])
        sysm.compute_forces()
        o = sysm.observables()
        Uf += o["U_pot"] + o["U_lrc"]
        Wf += o["W"] + o["W_lrc"]
    assert out[0].item() == pytest.approx(Uf / r_all.shape[0], rel=1e-6)
    assert out[1].item() == pytest.approx(Wf / r_all.shape[0], rel=1e-5, abs=1e-3)
    sysm.close()
