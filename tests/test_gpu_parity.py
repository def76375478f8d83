"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle,
element by element on the same seeded inputs.

Tolerances (FP32 site math, FP64 accumulation):
  * forces and torques: floored relative error
    |F - F_ref| / max(|F_ref|, 0.01 F_rms) with median <= 1e-5, max <= 1e-3;
  * energy and virial: |dU| <= 1e-5 * sum_ij |u_ij| and |dW| <= 1e-5 *
    sum_ij |w_ij| (an FP32 sum's error is bounded by a few ulp of the sum of
    magnitudes of its terms);
  * interacting / examined pair counts: exact (the pair set is decided in
    FP64 near the cut-off);
  * positions and quaternions after a short trajectory: 1e-5 absolute.
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
from test_oracle_pins import _half_step_temperature  # noqa: E402

LOG = os.environ.get("MD_PARITY_LOG")


def _log(**kw):
    if LOG:
        with open(LOG, "a") as f:
            f.write(json.dumps(kw) + "\n")


def gpu_eval(cfg, deterministic=1, half=0, device=True, cell_div=1):
    s = md.System(cfg, deterministic=deterministic, half_shell=half, cell_div=cell_div)
    if device:
        d = torch.device("cuda:0")
        t = {k: torch.from_numpy(np.ascontiguousarray(cfg[k])).to(d) for k in ("r", "v", "q", "j")}
        s.set(t["r"], t["q"], t["v"], t["j"])
    else:
        s.set(cfg["r"], cfg["q"], cfg["v"], cfg["j"])
    s.compute_forces()
    F, tau = s.forces()
    obs = s.observables()
    s.close()
    return F, tau, obs


def oracle_eval(cfg, cells=True):
    s = oracle.setup_from_config(cfg)
    return oracle.forces(cfg["model"], s, cfg["r"], cfg["q"], use_cells=cells)


def rel_err(A, B):
    rms = math.sqrt(float((B ** 2).sum(axis=1).mean())) if len(B) else 1.0
    floor = max(0.01 * rms, 1e-300)
    return np.linalg.norm(A - B, axis=1) / np.maximum(np.linalg.norm(B, axis=1), floor)


def check_parity(name, cfg, F, tau, obs, Fo, to, oo, exact_examined=True):
    assert obs["n_mol_pairs"] == int(oo["n_mol_pairs"])
    assert obs["n_site_pairs"] == int(oo["n_site_pairs"])
    if exact_examined:
        assert obs["n_examined"] == int(oo["n_examined"])
    ef = rel_err(F, Fo)
    et = rel_err(tau, to) if np.abs(to).max() > 0 else np.zeros(1)
    dU = abs(obs["U_pot"] - oo["U"]) / max(oo["abs_U"], 1e-300)
    dW = abs(obs["W"] - oo["W"]) / max(oo["abs_W"], 1e-300)
    _log(case=name, n=len(F), f_med=float(np.median(ef)), f_max=float(ef.max()), t_med=float(np.median(et)),
         t_max=float(et.max()), dU=dU, dW=dW, pairs=obs["n_mol_pairs"])
    assert np.median(ef) <= 1e-5 and ef.max() <= 1e-3, (np.median(ef), ef.max())
    assert np.median(et) <= 1e-5 and et.max() <= 1e-3, (np.median(et), et.max())
    assert dU <= 1e-5, dU
    assert dW <= 1e-5, dW
    for k in ("Wxx", "Wyy", "Wzz"):
        assert abs(obs["W_" + k[1:]] - oo[k]) <= 1e-5 * oo["abs_W"]
    assert obs["U_lrc"] == pytest.approx(oo["U_lrc"], rel=1e-12, abs=1e-300)
    assert obs["W_lrc"] == pytest.approx(oo["W_lrc"], rel=1e-12, abs=1e-300)
    # reaction-field self energy (reading R4), reported apart from U_pot
    assert obs["U_rf_self"] == pytest.approx(oo["U_rf_self"], rel=1e-12, abs=1e-300)
    if any(d["mu"] != 0 for d in cfg["model"]["dipoles"]) and cfg.get("eps_rf", math.inf) != 1.0:
        assert obs["U_rf_self"] < 0.0


CASES = {
    "lj-4096": lambda: mdgen.config_lj_fluid(n=4096),
    "lj-ragged-1999": lambda: mdgen.config_lj_fluid(n=1999, rho=0.45),
    "2cljq-20000": lambda: mdgen.config_2cljq(n=20000),
    "2cljdq-3000": lambda: mdgen.config_replica(7, 3000, 0.6, 1.0),
    "2cljdq-smallbox-500": lambda: mdgen.config_replica(3, 500, 0.75, 1.1),
    "2cljdq-dilute-700": lambda: mdgen.config_replica(5, 700, 0.05, 0.9),
    "4site-6000": lambda: mdgen.config_4site(n=6000),
    "slab-60000": lambda: mdgen.config_slab(n=60000),
    # dense cells: > 32 molecules per cell (several i passes per cell) and
    # > 256 stencil candidates (several staged windows per pass)
    "lj-dense-cells-12000": lambda: mdgen.config_lj_fluid(n=12000, rho=0.9, rc=4.0),
    "2cljq-dense-cells-8000": lambda: mdgen.config_2cljq(n=8000, rho=0.6, rc=5.0),
}


@pytest.mark.parametrize("half", [0, 1])
@pytest.mark.parametrize("name", list(CASES))
def test_force_parity(name, half):
    cfg = CASES[name]()
    Fo, to, oo = oracle_eval(cfg)
    F, tau, obs = gpu_eval(cfg, deterministic=1 - half, half=half)
    ncs = [int(math.floor(L / (cfg["rc"] * (1 + 1e-9)))) for L in cfg["box"]]
    check_parity(f"{name}/half{half}", cfg, F, tau, obs, Fo, to, oo, exact_examined=min(ncs) >= 3)


@pytest.mark.parametrize("name", ["2cljq-20000", "4site-6000", "lj-dense-cells-12000"])
def test_full_shell_cells_from_counter(name):
    """Full shell with `deterministic` off: the force kernel takes cells from
    a counter instead of a fixed grid stride, and in these small systems
    (fewer cells than half the resident warps) splits each cell's i
    molecules into several units of work.  Forces and torques meet the
    oracle tolerance and agree with the deterministic run (one unit per
    cell) up to FP32 summation order; the pair counts are identical."""
    cfg = CASES[name]()
    Fo, to, oo = oracle_eval(cfg)
    F, tau, obs = gpu_eval(cfg, deterministic=0, half=0)
    check_parity(f"{name}/counter", cfg, F, tau, obs, Fo, to, oo, exact_examined=True)
    Fd, taud, obsd = gpu_eval(cfg, deterministic=1, half=0)
    assert np.median(rel_err(F, Fd)) <= 1e-6 and rel_err(F, Fd).max() <= 1e-4
    if np.abs(taud).max() > 0:
        assert np.median(rel_err(tau, taud)) <= 1e-6 and rel_err(tau, taud).max() <= 1e-4
    assert obs["n_mol_pairs"] == obsd["n_mol_pairs"] and obs["n_examined"] == obsd["n_examined"]


# ------------------------------------------- cells of edge r_c / 2 (§3)
def _examined_pairs(r, box, rc, m):
    """Unordered molecule pairs whose cells (floor(m L / r_c) per axis, the
    cell of x is floor(x / edge)) are at most m cells apart along every axis,
    periodically: the pairs a stencil of radius m examines when every axis
    has at least 2m + 1 cells."""
    L = np.asarray(box, dtype=float)
    nc = np.floor(L * m / (rc * (1.0 + 1e-9))).astype(np.int64)
    iell = 1.0 / (L / nc)
    c = np.clip(np.floor(r * iell).astype(np.int64), 0, nc - 1)
    n, tot = len(r), 0
    for i0 in range(0, n, 128):
        d = np.abs(c[i0:i0 + 128, None, :] - c[None, :, :])
        d = np.minimum(d, nc - d)
        ok = (d <= m).all(axis=2) & (np.arange(n)[None, :] > np.arange(i0, min(i0 + 128, n))[:, None])
        tot += int(ok.sum())
    return tot


HALF_CELL_CASES = ["lj-4096", "lj-ragged-1999", "2cljq-20000", "2cljdq-3000", "2cljdq-smallbox-500",
                   "2cljdq-dilute-700", "4site-6000", "slab-60000", "2cljq-dense-cells-8000"]


@pytest.mark.parametrize("half", [0, 1])
@pytest.mark.parametrize("name", HALF_CELL_CASES)
def test_force_parity_half_cutoff_cells(name, half):
    """cell_div = 2 (§3 smaller cells: edge >= r_c / 2, the 125-cell
    stencil): the same interacting pairs and results as the oracle, and the
    examined pairs are exactly those of the smaller stencil."""
    cfg = CASES[name]()
    Fo, to, oo = oracle_eval(cfg)
    F, tau, obs = gpu_eval(cfg, deterministic=1 - half, half=half, cell_div=2)
    check_parity(f"{name}/div2/half{half}", cfg, F, tau, obs, Fo, to, oo, exact_examined=False)
    ncs = [int(math.floor(2 * L / (cfg["rc"] * (1 + 1e-9)))) for L in cfg["box"]]
    if min(ncs) >= 5 and len(F) <= 20000:
        assert obs["n_examined"] == _examined_pairs(cfg["r"], cfg["box"], cfg["rc"], 2)
    assert obs["n_examined"] <= oo["n_examined"]  # equal when one stencil already covers the box


def test_half_cutoff_cells_hit_fraction_matches_paper():
    """§3: cells of edge r_c examine 27 r_c^3 around a molecule and ~16% of
    the computed distances of a homogeneous configuration are inside r_c;
    cells of edge r_c / 2 examine 15.6 r_c^3 and ~27% are.  Homogeneous here:
    seeded uniform positions (a lattice commensurate with the cells would
    bias the examined count) in a box of 15 cut-off lengths, so both cell
    sizes divide it exactly."""
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))
    L = 15 * 2.5 * (1 + 1e-8)
    n = int(0.6 * L ** 3)
    cfg = mdgen.config_lj_fluid(n=n)
    assert cfg["rc"] == 2.5
    cfg["box"] = (L, L, L)
    cfg["r"] = np.random.default_rng(1408_0007).uniform(0.0, L, size=(n, 3))
    frac = {}
    for div in (1, 2):
        _, _, obs = gpu_eval(cfg, deterministic=0, half=1, cell_div=div)
        frac[div] = obs["n_mol_pairs"] / obs["n_examined"]
    assert frac[1] == pytest.approx(g["hit_fraction_rc_cells"]["value"], abs=0.01)
    assert frac[2] == pytest.approx(g["hit_fraction_half_rc_cells"]["value"], abs=0.01)
    assert frac[2] == pytest.approx((4 * math.pi / 3) / g["half_cell_volume_rc3"]["value"], rel=0.03)


@pytest.mark.parametrize("half", [0, 1])
def test_trajectory_half_cutoff_cells(half):
    _traj_compare(mdgen.config_2cljq(n=4000), 20, 1e-5, half=half, cell_div=2)
    _traj_compare(mdgen.config_lj_fluid(n=4096), 50, 1e-5, T_target=0.8, half=half, cell_div=2)


def test_param_grad_refuses_half_cutoff_cells():
    cfg = mdgen.config_4site(n=2000)
    s = md.System(cfg, cell_div=2)
    with pytest.raises(md.MDError) as e:
        s.param_grad(cfg["r"][None], cfg["q"][None])
    assert e.value.code == -9
    s.close()


def test_full_shell_is_deterministic():
    cfg = mdgen.config_2cljq(n=8000)
    F1, t1, o1 = gpu_eval(cfg)
    F2, t2, o2 = gpu_eval(cfg)
    assert np.array_equal(F1, F2) and np.array_equal(t1, t2)
    assert o1["U_pot"] == o2["U_pot"] and o1["W"] == o2["W"]


def test_host_and_device_inputs_agree():
    cfg = mdgen.config_4site(n=3000)
    F1, t1, o1 = gpu_eval(cfg, device=True)
    F2, t2, o2 = gpu_eval(cfg, device=False)
    assert np.array_equal(F1, F2) and np.array_equal(t1, t2)


def _pair_cfg(X, model=None, L=12.0, rc=3.0, shift=0):
    model = model or mdgen.model_lj()
    c = np.array([L / 2, L / 2, L / 2])
    r = np.array([c + np.asarray(X, float), c])
    q = np.tile([1.0, 0, 0, 0], (2, 1))
    return {"name": "pair", "model": model, "box": (L, L, L), "rc": rc, "lj_shift": shift, "lj_lrc": 0,
            "eps_rf": math.inf, "dt": 0.001, "T": 1.0, "r": r, "q": q, "v": np.zeros((2, 3)), "j": np.zeros((2, 3))}


def test_cutoff_decided_in_fp64():
    """Pairs within 1e-9 of rc (beyond FP32 resolution) are decided exactly
    as the FP64 definition decides them; exactly rc is outside (strict)."""
    for frac, expect in ((1 - 1e-9, 1), (1 + 1e-9, 0), (1.0, 0), (1 - 1e-6, 1)):
        cfg = _pair_cfg((3.0 * frac, 0, 0))
        F, tau, obs = gpu_eval(cfg)
        assert obs["n_mol_pairs"] == expect, frac
    # across the periodic boundary
    cfg = _pair_cfg((0, 0, 0), L=12.0)
    cfg["r"] = np.array([[0.2, 6.0, 6.0], [12.0 - 2.8 * (1 + 1e-9), 6.0, 6.0]])
    assert gpu_eval(cfg)[2]["n_mol_pairs"] == 0
    cfg["r"] = np.array([[0.2, 6.0, 6.0], [12.0 - 2.8 * (1 - 1e-9), 6.0, 6.0]])
    assert gpu_eval(cfg)[2]["n_mol_pairs"] == 1


def test_two_molecule_closed_form():
    """Eq. 1 at r = 1.5: U = 4 (1.5^-12 - 1.5^-6); F = -dU/dr along x."""
    cfg = _pair_cfg((1.5, 0, 0))
    F, tau, obs = gpu_eval(cfg)
    r = 1.5
    assert obs["U_pot"] == pytest.approx(4 * (r ** -12 - r ** -6), rel=2e-6)
    assert F[0, 0] == pytest.approx(-4 * (-12 * r ** -13 + 6 * r ** -7), rel=2e-6)
    assert F[1, 0] == pytest.approx(-F[0, 0], rel=1e-6)


def test_empty_and_single_molecule():
    cfg = mdgen.config_lj_fluid(n=64, rho=0.05)
    for n in (0, 1):
        c = dict(cfg)
        for k in ("r", "v", "q", "j"):
            c[k] = cfg[k][:n]
        F, tau, obs = gpu_eval(c, device=False)
        assert obs["n_mol_pairs"] == 0 and obs["U_pot"] == 0.0 and obs["W"] == 0.0
        assert F.shape == (n, 3) and (n == 0 or np.all(F == 0.0))


def test_positions_outside_box_are_wrapped():
    cfg = mdgen.config_2cljq(n=2000)
    shifted = dict(cfg)
    shifted["r"] = cfg["r"] + np.array(cfg["box"]) * np.array([3.0, -2.0, 1.0])
    F1, t1, o1 = gpu_eval(cfg, device=False)
    F2, t2, o2 = gpu_eval(shifted, device=False)
    assert o1["n_mol_pairs"] == o2["n_mol_pairs"]
    assert np.abs(F1 - F2).max() <= 1e-5 * np.abs(F1).max()


def test_state_round_trip():
    cfg = mdgen.config_4site(n=1500)
    s = md.System(cfg)
    s.set(cfg["r"], cfg["q"], cfg["v"], cfg["j"])
    r, v, q, j = s.molecules()
    s.close()
    assert np.array_equal(v, cfg["v"]) and np.array_equal(j, cfg["j"])
    assert np.allclose(r, np.mod(cfg["r"], np.array(cfg["box"])), atol=1e-12)
    assert np.allclose(q, cfg["q"] / np.linalg.norm(cfg["q"], axis=1, keepdims=True), atol=1e-15)


def test_call_order_errors():
    cfg = mdgen.config_lj_fluid(n=100)
    s = md.System(cfg)
    with pytest.raises(md.MDError) as e:
        s.compute_forces()
    assert e.value.code == -3
    with pytest.raises(md.MDError) as e:
        s.step(1, 0.001)
    assert e.value.code == -3
    with pytest.raises(md.MDError) as e:
        s.observables()
    assert e.value.code == -3
    s.close()


def test_nonfinite_input_rejected_on_host():
    cfg = mdgen.config_lj_fluid(n=100)
    bad = cfg["r"].copy()
    bad[7, 1] = np.nan
    s = md.System(cfg)
    with pytest.raises(md.MDError) as e:
        s.set(bad, cfg["q"])
    assert e.value.code == -1
    s.close()


# ----------------------------------------------------------- trajectories
def _traj_compare(cfg, n_steps, tol, T_target=0.0, half=0, cell_div=1):
    s = md.System(cfg, deterministic=1 - half, half_shell=half, cell_div=cell_div)
    s.set(cfg["r"], cfg["q"], cfg["v"], cfg["j"])
    s.step(n_steps, cfg["dt"], T_target=T_target)
    r, v, q, j = s.molecules()
    F, tau = s.forces()
    obs = s.observables()
    s.close()
    st = oracle.step(cfg["model"], oracle.setup_from_config(cfg), {k: cfg[k] for k in ("r", "v", "q", "j")},
                     cfg["dt"], n_steps, use_cells=True, T_target=T_target)
    if T_target > 0:
        # the half-step temperature the thermostat set, from the GPU state
        T_half = _half_step_temperature(cfg["model"], v, q, j)
        assert T_half == pytest.approx(T_target, rel=1e-6)
    L = np.array(cfg["box"])
    dr = r - st["r"]
    dr -= L * np.rint(dr / L)
    dq = np.minimum(np.abs(q - st["q"]).max(axis=1), np.abs(q + st["q"]).max(axis=1))
    _log(case="traj/" + cfg["name"], steps=n_steps, dr=float(np.abs(dr).max()), dq=float(dq.max()),
         dv=float(np.abs(v - st["v"]).max()), dj=float(np.abs(j - st["j"]).max()))
    assert np.abs(dr).max() < tol
    assert dq.max() < tol
    assert obs["step"] == n_steps
    kt, kr = oracle.kinetic(cfg["model"], cfg["dt"], st["v"], st["q"], st["j"], st["F"], st["tau"])
    assert obs["K_trans"] == pytest.approx(kt, rel=1e-5)
    assert obs["K_rot"] == pytest.approx(kr, rel=1e-5, abs=1e-12)


def test_trajectory_lj_100_steps():
    _traj_compare(mdgen.config_lj_fluid(n=4096), 100, 1e-5)


def test_trajectory_2cljq_20_steps():
    _traj_compare(mdgen.config_2cljq(n=4000), 20, 1e-5)


def test_trajectory_4site_10_steps():
    cfg = mdgen.config_4site(n=2000)
    cfg["v"] *= 0.1
    cfg["j"] *= 0.1
    _traj_compare(cfg, 10, 1e-5)


@pytest.mark.parametrize("half", [0, 1])
def test_trajectory_2cljq_nvt(half):
    """Velocity rescaling (§2 NVT) to a temperature well away from the start."""
    _traj_compare(mdgen.config_2cljq(n=4000), 20, 1e-5, T_target=1.4, half=half)


def test_trajectory_4site_nvt():
    cfg = mdgen.config_4site(n=2000)
    cfg["v"] *= 0.1
    cfg["j"] *= 0.1
    _traj_compare(cfg, 10, 1e-5, T_target=0.05)


def test_trajectory_lj_nvt():
    _traj_compare(mdgen.config_lj_fluid(n=4096), 50, 1e-5, T_target=0.8)


# -------------------------------------------------- full benchmark sizes
@pytest.mark.parametrize("half", [0, 1])
def test_full_size_2cljq_parity(half):
    """The bench workload (N = 262144 2CLJQ, rc = 3), every molecule."""
    cfg = mdgen.config_2cljq()
    Fo, to, oo = oracle_eval(cfg)
    F, tau, obs = gpu_eval(cfg, deterministic=1 - half, half=half)
    check_parity(f"2cljq-262144/half{half}", cfg, F, tau, obs, Fo, to, oo)


def test_full_size_slab_parity():
    """Vapour-liquid slab, N = 4,194,304 single-site LJTS (uneven cells)."""
    cfg = mdgen.config_slab()
    Fo, to, oo = oracle_eval(cfg)
    F, tau, obs = gpu_eval(cfg, deterministic=0, half=1)
    check_parity("slab-4194304/half1", cfg, F, tau, obs, Fo, to, oo)


# ------------------------------------------------- NVE drift over 1000 steps
def _energy_series(run_chunk, n_chunks):
    E = []
    for _ in range(n_chunks):
        E.append(run_chunk())
    return np.array(E)


def equilibrated_2cljq(n=4000, seed_k=0):
    """The 2CLJQ fluid (rho = 0.55, T = 1, rc = 3) after the untimed warm-up
    of the measurement recipe, run by the FP64 oracle: 200 velocity-rescaled
    steps at dt / 10, then 100 at dt (dt = 0.001)."""
    cfg = mdgen.config_2cljq(n=n, seed_k=seed_k)
    setup = oracle.setup_from_config(cfg)
    st = {k: cfg[k] for k in ("r", "v", "q", "j")}
    st = oracle.step(cfg["model"], setup, st, cfg["dt"] / 10, 200, use_cells=True, T_target=cfg["T"])
    st = oracle.step(cfg["model"], setup, st, cfg["dt"], 100, use_cells=True, T_target=cfg["T"])
    out = dict(cfg)
    out.update({k: st[k] for k in ("r", "v", "q", "j")})
    return out


def nve_drift(cfg, n_steps=1000, every=10):
    """Total energy U + K_trans + K_rot every `every` steps over n_steps NVE
    leapfrog steps, GPU (deterministic full shell) and FP64 oracle from the
    same start; returns (drift_gpu, drift_oracle, rms_fluct_oracle) over the
    run (linear fits) and the per-step-per-molecule drifts."""
    dt, n_chunks = cfg["dt"], n_steps // every
    s = md.System(cfg, deterministic=1)
    s.set(cfg["r"], cfg["q"], cfg["v"], cfg["j"])

    def gpu_chunk():
        s.step(every, dt)
        o = s.observables()
        return o["U_pot"] + o["K_trans"] + o["K_rot"]

    Eg = _energy_series(gpu_chunk, n_chunks)
    s.close()
    setup = oracle.setup_from_config(cfg)
    st = {k: cfg[k] for k in ("r", "v", "q", "j")}
    Eo = []
    for _ in range(n_chunks):
        st = oracle.step(cfg["model"], setup, st, dt, every, use_cells=True)
        kt, kr = oracle.kinetic(cfg["model"], dt, st["v"], st["q"], st["j"], st["F"], st["tau"])
        Eo.append(st["obs"]["U"] + kt + kr)
    Eo = np.array(Eo)
    t = np.arange(1, n_chunks + 1) * every * dt
    fit_g, fit_o = np.polyfit(t, Eg, 1), np.polyfit(t, Eo, 1)
    span = t[-1] - t[0]
    n = cfg["r"].shape[0]
    return {"drift_gpu": float(fit_g[0] * span), "drift_oracle": float(fit_o[0] * span),
            "rms_fluct_oracle": float(np.std(Eo - np.polyval(fit_o, t))), "E_scale": float(np.abs(Eo).max()),
            "drift_gpu_per_step_per_mol": float(fit_g[0] * dt / n),
            "drift_oracle_per_step_per_mol": float(fit_o[0] * dt / n), "steps": n_steps}


@pytest.mark.parametrize("which", ["lj-4096", "2cljq-4000"])
def test_nve_energy_drift_1000_steps(which):
    """1000 NVE leapfrog steps: the total energy of the GPU path drifts no
    more than the FP64 oracle's own drift plus three times the oracle's
    energy fluctuation (linear fits over the run; the trajectories
    themselves diverge, as chaotic trajectories do, once rounding differs).
    LJTS fluid (N = 4096, T = 0.95, dt = 0.002, no rotation) and the rigid
    2CLJQ fluid (N = 4000, dt = 0.001, the rotational leapfrog of Eqs. 4-5
    in play) started from its oracle-equilibrated state."""
    cfg = mdgen.config_lj_fluid(n=4096) if which == "lj-4096" else equilibrated_2cljq(4000)
    d = nve_drift(cfg)
    _log(case=f"nve-drift/{which}", **d)
    assert abs(d["drift_gpu"]) <= abs(d["drift_oracle"]) + 3.0 * d["rms_fluct_oracle"] + 1e-9 * d["E_scale"], d


# ------------------------------------- models outside the compiled signatures
def _triangle_model():
    """Three LJ centres (two types) on an equilateral triangle about the
    centre of mass, each carrying a charge (net zero), plus a point dipole
    at the centre of mass along z: merged roles LJ|q, LJ|q, LJ|q, mu -- no
    compiled signature, so the run-time-signature kernels run."""
    r = 0.45
    pts = [(r, 0.0, 0.0), (-0.5 * r, 0.5 * math.sqrt(3.0) * r, 0.0), (-0.5 * r, -0.5 * math.sqrt(3.0) * r, 0.0)]
    return {"lj_types": {"eps": [1.0, 0.7], "sigma": [1.0, 0.85]}, "xi": None, "eta": None,
            "lj": [{"pos": pts[0], "type": 0, "mass": 1.0 / 3.0},
                   {"pos": pts[1], "type": 1, "mass": 1.0 / 3.0},
                   {"pos": pts[2], "type": 1, "mass": 1.0 / 3.0}],
            "charges": [{"pos": pts[0], "q": 0.5}, {"pos": pts[1], "q": -0.25}, {"pos": pts[2], "q": -0.25}],
            "dipoles": [{"pos": (0.0, 0.0, 0.0), "axis": (0.0, 0.0, 1.0), "mu": 0.8}],
            "quads": []}


def _triangle_config(n=3000, rho=0.45, T=1.1, seed=77):
    rng = np.random.default_rng(seed)
    model = _triangle_model()
    L = (n / rho) ** (1.0 / 3.0)
    box = (L, L, L)
    pos = mdgen.fcc_subset(n, box, rng, jitter=0.05)
    q = mdgen.random_quaternions(n, rng)
    q = mdgen.resolve_site_overlaps(model, pos, q, box, rng, d_min=0.6)
    v = mdgen.mb_velocities(n, T, mdgen.model_mass(model), rng)
    j = mdgen.angular_momenta(q, mdgen.model_principal_moments(model), T, rng)
    return {"name": f"triangle-qmu-N{n}", "model": model, "box": box, "rc": 3.0, "lj_shift": 0, "lj_lrc": 1,
            "eps_rf": 8.0, "dt": 0.001, "T": T, "r": np.ascontiguousarray(np.mod(pos, box)), "v": v, "q": q, "j": j}


@pytest.mark.parametrize("half", [0, 1])
def test_runtime_signature_model_parity(half):
    cfg = _triangle_config()
    Fo, to, oo = oracle_eval(cfg)
    F, tau, obs = gpu_eval(cfg, deterministic=1 - half, half=half)
    check_parity(f"{cfg['name']}/half{half}", cfg, F, tau, obs, Fo, to, oo)


def test_runtime_signature_model_trajectory():
    cfg = _triangle_config(n=2000, rho=0.3)
    cfg["v"] *= 0.3
    cfg["j"] *= 0.3
    _traj_compare(cfg, 10, 1e-5)


@pytest.mark.parametrize("T_target", [0.0, 1.3])
def test_step_graph_replay_equals_single_steps(T_target):
    """md_step(n >= 2) replays captured pairs of steps (per buffer parity);
    in the deterministic full shell the result is bitwise that of n calls of
    md_step(1), across parities, a change of dt and the observables."""
    cfg = mdgen.config_2cljq(n=6000)
    res = []
    for graphs in (False, True):
        s = md.System(cfg, deterministic=1)
        s.set(cfg["r"], cfg["q"], cfg["v"], cfg["j"])
        plan = [(5, 0.001), (4, 0.001), (3, 0.0005)]
        for n, dt in plan:
            if graphs:
                s.step(n, dt, T_target=T_target)
            else:
                for _ in range(n):
                    s.step(1, dt, T_target=T_target)
        o = s.observables()
        res.append((s.molecules(), s.forces(), o))
        s.close()
    (m0, f0, o0), (m1, f1, o1) = res
    for a, b in zip(m0 + f0, m1 + f1):
        assert np.array_equal(a, b)
    assert o0["step"] == o1["step"] == 12
    for k in ("U_pot", "W", "K_trans", "K_rot", "n_mol_pairs", "time"):
        assert o0[k] == o1[k], k
