"""FP64 CPU oracle for the rigid multi-site MD hot path (arXiv 1408.4599).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the CUDA library never does.

The arithmetic lives in ``md_oracle.c`` (plain C99, FP64, optional OpenMP);
this module compiles it with gcc on first use and marshals numpy arrays and
the model dictionaries of :mod:`mdgen` through ctypes.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "md_oracle.c")
_HDR = os.path.join(_HERE, "md_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
# a prebuilt library to load instead (the pins' mutation test points this at
# copies of the oracle with planted mistakes); never rebuilt here
_LIB_OVERRIDE = os.environ.get("MD_ORACLE_LIB") or None
_lock = threading.Lock()
_lib = None

MAXT = 8
MAXE = 16
NOBS = 16
OBS = {"U": 0, "W": 1, "Wxx": 2, "Wyy": 3, "Wzz": 4, "n_mol_pairs": 5, "n_site_pairs": 6,
       "n_examined": 7, "U_lrc": 8, "W_lrc": 9, "U_rf_self": 10, "abs_U": 11, "abs_W": 12}


def build(force: bool = False) -> str:
    """Compile liboracle.so (gcc, -O2, OpenMP) if missing or stale."""
    if _LIB_OVERRIDE:
        return _LIB_OVERRIDE
    with _lock:
        stale = (not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
        if force or stale:
            tmp = _LIB + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True, cwd=_HERE)
            os.replace(tmp, _LIB)
    return _LIB


class Model(C.Structure):
    _fields_ = [("n_types", C.c_int32), ("eps", C.c_double * MAXT), ("sigma", C.c_double * MAXT),
                ("xi", C.c_double * (MAXT * MAXT)), ("eta", C.c_double * (MAXT * MAXT)),
                ("n_lj", C.c_int32), ("lj_pos", C.c_double * (MAXE * 3)), ("lj_type", C.c_int32 * MAXE),
                ("lj_mass", C.c_double * MAXE),
                ("n_chg", C.c_int32), ("chg_pos", C.c_double * (MAXE * 3)), ("chg_q", C.c_double * MAXE),
                ("n_dip", C.c_int32), ("dip_pos", C.c_double * (MAXE * 3)), ("dip_axis", C.c_double * (MAXE * 3)),
                ("dip_mu", C.c_double * MAXE),
                ("n_quad", C.c_int32), ("quad_pos", C.c_double * (MAXE * 3)), ("quad_axis", C.c_double * (MAXE * 3)),
                ("quad_Q", C.c_double * MAXE)]


class Setup(C.Structure):
    _fields_ = [("box", C.c_double * 3), ("rc", C.c_double), ("eps_rf", C.c_double),
                ("lj_shift", C.c_int32), ("lj_lrc", C.c_int32)]


def _lib_handle():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        P = C.POINTER
        d, i64, i32 = C.c_double, C.c_int64, C.c_int
        dp = P(d)
        lib.orc_forces.argtypes = [P(Model), P(Setup), i64, dp, dp, i32, i32, dp, dp, dp]
        lib.orc_forces_subset.argtypes = [P(Model), P(Setup), i64, dp, dp, i64, P(i64), i32, dp, dp]
        lib.orc_step.argtypes = [P(Model), P(Setup), i64, d, i32, i32, i32, dp, dp, dp, dp, dp, dp, dp]
        lib.orc_step_T.argtypes = [P(Model), P(Setup), i64, d, i32, d, i32, i32, dp, dp, dp, dp, dp, dp, dp]
        lib.orc_kinetic.argtypes = [P(Model), i64, d, dp, dp, dp, dp, dp, dp]
        lib.orc_lrc.argtypes = [P(Model), P(Setup), i64, dp]
        lib.orc_n_params.argtypes = [P(Model)]
        lib.orc_param_grad.argtypes = [P(Model), P(Setup), i32, i64, dp, dp, i32, i32, dp, dp, dp, dp, dp]
        lib.orc_rotmat.argtypes = [dp, dp]
        _lib = lib
    return _lib


def make_model(md: dict) -> Model:
    """Marshal an :mod:`mdgen` model dictionary into the oracle's struct."""
    m = Model()
    eps = md["lj_types"]["eps"]
    sig = md["lj_types"]["sigma"]
    T = len(eps)
    assert T <= MAXT
    m.n_types = T
    for t in range(T):
        m.eps[t] = eps[t]
        m.sigma[t] = sig[t]
    xi = md.get("xi")
    eta = md.get("eta")
    for a in range(T):
        for b in range(T):
            m.xi[a * T + b] = 1.0 if xi is None else xi[a][b]
            m.eta[a * T + b] = 1.0 if eta is None else eta[a][b]
    lj = md["lj"]
    m.n_lj = len(lj)
    for k, s in enumerate(lj):
        for c in range(3):
            m.lj_pos[3 * k + c] = s["pos"][c]
        m.lj_type[k] = s["type"]
        m.lj_mass[k] = s["mass"]
    ch = md["charges"]
    m.n_chg = len(ch)
    for k, s in enumerate(ch):
        for c in range(3):
            m.chg_pos[3 * k + c] = s["pos"][c]
        m.chg_q[k] = s["q"]
    dp = md["dipoles"]
    m.n_dip = len(dp)
    for k, s in enumerate(dp):
        for c in range(3):
            m.dip_pos[3 * k + c] = s["pos"][c]
            m.dip_axis[3 * k + c] = s["axis"][c]
        m.dip_mu[k] = s["mu"]
    qd = md["quads"]
    m.n_quad = len(qd)
    for k, s in enumerate(qd):
        for c in range(3):
            m.quad_pos[3 * k + c] = s["pos"][c]
            m.quad_axis[3 * k + c] = s["axis"][c]
        m.quad_Q[k] = s["Q"]
    return m


def make_setup(box, rc, eps_rf=math.inf, lj_shift=0, lj_lrc=0) -> Setup:
    s = Setup()
    for c in range(3):
        s.box[c] = box[c]
    s.rc = rc
    s.eps_rf = eps_rf
    s.lj_shift = int(lj_shift)
    s.lj_lrc = int(lj_lrc)
    return s


def setup_from_config(cfg: dict) -> Setup:
    return make_setup(cfg["box"], cfg["rc"], cfg.get("eps_rf", math.inf), cfg.get("lj_shift", 0),
                      cfg.get("lj_lrc", 0))


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _c(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def forces(model: dict, setup: Setup, r, q, use_cells: bool = False, n_threads: int = 0):
    """F, tau (n x 3 each) and observables dict for one configuration."""
    lib = _lib_handle()
    r = _c(r)
    q = _c(q)
    n = r.shape[0]
    F = np.zeros((n, 3))
    tau = np.zeros((n, 3))
    obs = np.zeros(NOBS)
    M = make_model(model)
    rc = lib.orc_forces(C.byref(M), C.byref(setup), n, _dp(r), _dp(q), int(use_cells), int(n_threads),
                        _dp(F), _dp(tau), _dp(obs))
    if rc != 0:
        raise ValueError(f"orc_forces failed with code {rc}")
    return F, tau, {k: float(obs[v]) for k, v in OBS.items()}


def forces_subset(model: dict, setup: Setup, r, q, sel, n_threads: int = 0):
    lib = _lib_handle()
    r = _c(r)
    q = _c(q)
    sel = np.ascontiguousarray(sel, dtype=np.int64)
    F = np.zeros((sel.shape[0], 3))
    tau = np.zeros((sel.shape[0], 3))
    M = make_model(model)
    rc = lib.orc_forces_subset(C.byref(M), C.byref(setup), r.shape[0], _dp(r), _dp(q), sel.shape[0],
                               sel.ctypes.data_as(C.POINTER(C.c_int64)), int(n_threads), _dp(F), _dp(tau))
    if rc != 0:
        raise ValueError(f"orc_forces_subset failed with code {rc}")
    return F, tau


def step(model: dict, setup: Setup, state: dict, dt: float, n_steps: int, use_cells: bool = False,
         n_threads: int = 0, T_target: float = 0.0):
    """Advance a copy of ``state`` (r, v, q, j and optionally F, tau) by
    n_steps leapfrog steps; returns the new state dict with F, tau, obs.
    T_target > 0: velocity rescaling to T_target after every step (orc_step_T)."""
    lib = _lib_handle()
    r = _c(state["r"]).copy()
    v = _c(state["v"]).copy()
    q = _c(state["q"]).copy()
    j = _c(state["j"]).copy()
    if "F" in state:
        F = _c(state["F"]).copy()
        tau = _c(state["tau"]).copy()
    else:
        F, tau, _ = forces(model, setup, r, q, use_cells, n_threads)
    obs = np.zeros(NOBS)
    M = make_model(model)
    rc = lib.orc_step_T(C.byref(M), C.byref(setup), r.shape[0], float(dt), int(n_steps), float(T_target),
                        int(use_cells), int(n_threads), _dp(r), _dp(v), _dp(q), _dp(j), _dp(F), _dp(tau), _dp(obs))
    if rc != 0:
        raise ValueError(f"orc_step failed with code {rc}")
    out = {"r": r, "v": v, "q": q, "j": j, "F": F, "tau": tau}
    if n_steps > 0:
        out["obs"] = {k: float(obs[vv]) for k, vv in OBS.items()}
    return out


def kinetic(model: dict, dt: float, v, q, j, F, tau):
    """(K_trans, K_rot) at the integer time step from half-step v, j."""
    lib = _lib_handle()
    v, q, j, F, tau = (_c(a) for a in (v, q, j, F, tau))
    K = np.zeros(2)
    M = make_model(model)
    lib.orc_kinetic(C.byref(M), v.shape[0], float(dt), _dp(v), _dp(q), _dp(j), _dp(F), _dp(tau), _dp(K))
    return float(K[0]), float(K[1])


def lrc(model: dict, setup: Setup, n: int):
    lib = _lib_handle()
    out = np.zeros(3)
    M = make_model(model)
    lib.orc_lrc(C.byref(M), C.byref(setup), int(n), _dp(out))
    return float(out[0]), float(out[1]), float(out[2])


def n_params(model: dict) -> int:
    lib = _lib_handle()
    M = make_model(model)
    return int(lib.orc_n_params(C.byref(M)))


def param_grad(model: dict, setup: Setup, r_all, q_all, use_cells: bool = False, n_threads: int = 0,
               with_abs: bool = False):
    """(dU/dtheta, dW/dtheta, <U>, <W>) averaged over the configurations in
    r_all (n_cfg x n x 3) and q_all (n_cfg x n x 4); with_abs also returns
    the sums of |per-pair derivative| (the error scales of the sums)."""
    lib = _lib_handle()
    r_all = _c(r_all)
    q_all = _c(q_all)
    n_cfg, n = r_all.shape[0], r_all.shape[1]
    M = make_model(model)
    P = int(lib.orc_n_params(C.byref(M)))
    dU = np.zeros(P)
    dW = np.zeros(P)
    means = np.zeros(2)
    aU = np.zeros(P)
    aW = np.zeros(P)
    rc = lib.orc_param_grad(C.byref(M), C.byref(setup), n_cfg, n, _dp(r_all), _dp(q_all), int(use_cells),
                            int(n_threads), _dp(dU), _dp(dW), _dp(means), _dp(aU), _dp(aW))
    if rc != 0:
        raise ValueError(f"orc_param_grad failed with code {rc}")
    if with_abs:
        return dU, dW, float(means[0]), float(means[1]), aU, aW
    return dU, dW, float(means[0]), float(means[1])


def rotmat(q) -> np.ndarray:
    lib = _lib_handle()
    q = _c(q)
    R = np.zeros(9)
    lib.orc_rotmat(_dp(q), _dp(R))
    return R.reshape(3, 3)


def model_param_vector(model: dict) -> np.ndarray:
    """theta in the oracle's order: eps_t, sigma_t, charges, dipoles, quads."""
    th = list(model["lj_types"]["eps"]) + list(model["lj_types"]["sigma"])
    th += [c["q"] for c in model["charges"]]
    th += [d["mu"] for d in model["dipoles"]]
    th += [qq["Q"] for qq in model["quads"]]
    return np.array(th, dtype=np.float64)


def model_with_params(model: dict, theta) -> dict:
    """Copy of ``model`` with parameters replaced by theta (oracle order)."""
    import copy
    m = copy.deepcopy(model)
    T = len(m["lj_types"]["eps"])
    th = list(theta)
    m["lj_types"]["eps"] = th[:T]
    m["lj_types"]["sigma"] = th[T:2 * T]
    k = 2 * T
    for c in m["charges"]:
        c["q"] = th[k]
        k += 1
    for d in m["dipoles"]:
        d["mu"] = th[k]
        k += 1
    for qq in m["quads"]:
        qq["Q"] = th[k]
        k += 1
    return m
