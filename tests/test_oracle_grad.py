"""Pins of the oracle's force-field parameter derivatives (CPU only).

The derivatives of the mean total energy and virial (pair sum inside the
cut-off + the §3 long-range correction) with respect to the per-type LJ
parameters (Eq. 1 with the §2 combination rules), charges, dipole and
quadrupole moments are checked against central finite differences of the
oracle's own energy (h = 1e-4, FP64) and against exact scaling laws.
"""
import math

import numpy as np
import pytest

import mdgen
import oracle


def _configs(n_cfg=3, n=300):
    cfgs = [mdgen.config_4site(n=n, rho=0.5, cfg=c) for c in range(n_cfg)]
    r = np.stack([c["r"] for c in cfgs])
    q = np.stack([c["q"] for c in cfgs])
    return cfgs[0], r, q


def _UW(model, s, r_all, q_all):
    U = W = 0.0
    for r, q in zip(r_all, q_all):
        _, _, o = oracle.forces(model, s, r, q)
        U += o["U"] + o["U_lrc"]
        W += o["W"] + o["W_lrc"]
    return U / len(r_all), W / len(r_all)


@pytest.mark.parametrize("shift", [0, 1])
def test_param_grad_matches_central_differences(shift):
    cfg, r_all, q_all = _configs()
    model = cfg["model"]
    s = oracle.make_setup(cfg["box"], cfg["rc"], eps_rf=math.inf, lj_shift=shift, lj_lrc=1 - shift)
    dU, dW, Um, Wm = oracle.param_grad(model, s, r_all, q_all)
    U0, W0 = _UW(model, s, r_all, q_all)
    assert Um == pytest.approx(U0, rel=1e-12)
    assert Wm == pytest.approx(W0, rel=1e-12)
    th = oracle.model_param_vector(model)
    assert len(th) == oracle.n_params(model) == 8
    h = 1e-4
    for p in range(len(th)):
        tp = th.copy(); tp[p] += h
        tm = th.copy(); tm[p] -= h
        Up, Wp = _UW(oracle.model_with_params(model, tp), s, r_all, q_all)
        Umn, Wmn = _UW(oracle.model_with_params(model, tm), s, r_all, q_all)
        gU = (Up - Umn) / (2 * h)
        gW = (Wp - Wmn) / (2 * h)
        assert dU[p] == pytest.approx(gU, rel=1e-6, abs=1e-6 * max(1.0, abs(U0))), p
        assert dW[p] == pytest.approx(gW, rel=1e-6, abs=1e-6 * max(1.0, abs(W0))), p


def test_energy_is_homogeneous_in_strengths_and_eps():
    """U_LJ is linear in every eps (Euler: sum eps dU/deps = U_LJ); the
    electrostatic energy is bilinear in the strengths (sum s dU/ds = 2 U_el)."""
    cfg, r_all, q_all = _configs(n_cfg=2)
    model = cfg["model"]
    s = oracle.make_setup(cfg["box"], cfg["rc"], eps_rf=math.inf, lj_shift=0, lj_lrc=1)
    dU, dW, Um, Wm = oracle.param_grad(model, s, r_all, q_all)
    th = oracle.model_param_vector(model)
    lj_only = oracle.model_with_params(model, np.concatenate([th[:4], np.zeros(4)]))
    el_only = oracle.model_with_params(model, np.concatenate([[0.0, 0.0], th[2:4], th[4:]]))
    U_lj, W_lj = _UW(lj_only, s, r_all, q_all)
    U_el, W_el = _UW(el_only, s, r_all, q_all)
    assert U_lj + U_el == pytest.approx(Um, rel=1e-11)
    assert float(th[:2] @ dU[:2]) == pytest.approx(U_lj, rel=1e-11)
    assert float(th[:2] @ dW[:2]) == pytest.approx(W_lj, rel=1e-11)
    assert float(th[4:] @ dU[4:]) == pytest.approx(2 * U_el, rel=1e-11)
    assert float(th[4:] @ dW[4:]) == pytest.approx(2 * W_el, rel=1e-11)
    # doubling every eps doubles the LJ part exactly
    U2, _ = _UW(oracle.model_with_params(model, np.concatenate([2 * th[:2], th[2:4], np.zeros(4)])), s, r_all, q_all)
    assert U2 == pytest.approx(2 * U_lj, rel=1e-12)
