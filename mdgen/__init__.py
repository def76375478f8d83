"""Seeded synthetic inputs for the rigid-molecule MD hot path.

This module only *builds inputs*: molecular models (site geometry and
parameters), lattices, orientations, velocities and angular momenta.  It holds
none of the method's arithmetic (no pair potentials, no forces, no
integrator).  Both the FP64 CPU oracle (``oracle/``) and the CUDA library
(``paper_1408_4599_gb300``) consume what it returns; neither imports the other.

Units are reduced Lennard-Jones units of the first LJ type
(epsilon = sigma = m = k_B = k_C = 1), cf. the paper's units paragraph in §2
(k_B = 1, k_C = 1).

Model dictionaries (consumed by both sides, each marshals its own C struct)::

    {"lj_types": {"eps": [...], "sigma": [...]},   # per LJ type (Lorentz-Berthelot inputs, §2)
     "xi": None | TxT, "eta": None | TxT,          # binary interaction parameters (1 if None)
     "lj":      [{"pos": (x,y,z), "type": t, "mass": m}, ...],
     "charges": [{"pos": ..., "q": ...}, ...],
     "dipoles": [{"pos": ..., "axis": ..., "mu": ...}, ...],
     "quads":   [{"pos": ..., "axis": ..., "Q": ...}, ...]}

Body-frame positions are relative to the centre of mass and expressed in the
principal-axes frame (the generator guarantees it).  Quaternions are
(w, x, y, z) and rotate body-frame vectors into the space frame.
"""
from __future__ import annotations

import math
import os

import numpy as np

SEED_BASE = 1408_0000


def seed_for(config: int, k: int = 0) -> int:
    """Seed recipe: 1408_0000 + 100*config + k."""
    return SEED_BASE + 100 * config + k


# --------------------------------------------------------------------------
# Molecular models (§2: rigid multi-centre molecules of LJ sites, point
# charges, dipoles, quadrupoles).
# --------------------------------------------------------------------------

def model_lj() -> dict:
    """Single-site Lennard-Jones molecule (epsilon = sigma = m = 1)."""
    return {"lj_types": {"eps": [1.0], "sigma": [1.0]}, "xi": None, "eta": None,
            "lj": [{"pos": (0.0, 0.0, 0.0), "type": 0, "mass": 1.0}],
            "charges": [], "dipoles": [], "quads": []}


def model_2cljq(elong: float = 0.5, Q2: float = 2.0) -> dict:
    """Two-centre LJ + point quadrupole (2CLJQ).

    Two LJ sites (eps = sigma = 1, mass 1/2) at +-elong/2 on the body z axis
    and a linear point quadrupole of reduced strength Q*^2 = Q2 at the centre
    of mass, along the axis.
    """
    h = 0.5 * elong
    return {"lj_types": {"eps": [1.0], "sigma": [1.0]}, "xi": None, "eta": None,
            "lj": [{"pos": (0.0, 0.0, -h), "type": 0, "mass": 0.5},
                   {"pos": (0.0, 0.0, +h), "type": 0, "mass": 0.5}],
            "charges": [], "dipoles": [],
            "quads": [{"pos": (0.0, 0.0, 0.0), "axis": (0.0, 0.0, 1.0), "Q": math.sqrt(Q2)}]}


def model_2cljdq(elong: float = 0.5, mu2: float = 1.5, Q2: float = 2.0) -> dict:
    """2CLJQ plus a point dipole (mu*^2 = mu2) at the centre of mass, both
    multipoles along the molecular axis."""
    m = model_2cljq(elong, Q2)
    m["dipoles"] = [{"pos": (0.0, 0.0, 0.0), "axis": (0.0, 0.0, 1.0), "mu": math.sqrt(mu2)}]
    return m


def model_4site(mu2: float = 1.5, Q2: float = 2.0, charge: float = 0.4) -> dict:
    """Four-site polar rigid model used for force-field-gradient work.

    Sites (before the centre-of-mass shift): LJ type A (eps 1, sigma 1) at the
    apex; two LJ type B sites (eps 0.8, sigma 0.9) at 0.55 sigma from A with a
    105 degree B-A-B angle, carrying charges +charge / -charge; a massless
    point P on the bisector 0.2 sigma from A carrying a dipole along the
    bisector and a linear quadrupole normal to the molecular plane.  Masses
    1/3 per LJ site.  The result is shifted to the centre of mass; the
    molecule lies in the xy plane with the bisector along y, which are
    principal axes by symmetry (checked below).
    """
    half = math.radians(105.0) / 2.0
    A = np.array([0.0, 0.0, 0.0])
    B1 = 0.55 * np.array([math.sin(half), math.cos(half), 0.0])
    B2 = 0.55 * np.array([-math.sin(half), math.cos(half), 0.0])
    P = np.array([0.0, 0.2, 0.0])
    masses = np.array([1.0 / 3.0] * 3)
    com = (masses[0] * A + masses[1] * B1 + masses[2] * B2) / masses.sum()
    A, B1, B2, P = A - com, B1 - com, B2 - com, P - com
    pts = np.stack([A, B1, B2])
    inertia = np.zeros((3, 3))
    for mi, p in zip(masses, pts):
        inertia += mi * (np.dot(p, p) * np.eye(3) - np.outer(p, p))
    off = inertia - np.diag(np.diag(inertia))
    assert np.abs(off).max() < 1e-14, "4-site model must already be in principal axes"
    t = lambda v: tuple(float(x) for x in v)
    return {"lj_types": {"eps": [1.0, 0.8], "sigma": [1.0, 0.9]}, "xi": None, "eta": None,
            "lj": [{"pos": t(A), "type": 0, "mass": 1.0 / 3.0},
                   {"pos": t(B1), "type": 1, "mass": 1.0 / 3.0},
                   {"pos": t(B2), "type": 1, "mass": 1.0 / 3.0}],
            "charges": [{"pos": t(B1), "q": +charge}, {"pos": t(B2), "q": -charge}],
            "dipoles": [{"pos": t(P), "axis": (0.0, 1.0, 0.0), "mu": math.sqrt(mu2)}],
            "quads": [{"pos": t(P), "axis": (0.0, 0.0, 1.0), "Q": math.sqrt(Q2)}]}


def model_mass(model: dict) -> float:
    return float(sum(s["mass"] for s in model["lj"]))


def model_principal_moments(model: dict) -> np.ndarray:
    """Principal moments of the (already principal-frame) model, used only to
    draw initial angular momenta."""
    I = np.zeros(3)
    for s in model["lj"]:
        x, y, z = s["pos"]
        I += s["mass"] * np.array([y * y + z * z, x * x + z * z, x * x + y * y])
    return I


# --------------------------------------------------------------------------
# Elementary seeded generators
# --------------------------------------------------------------------------

def fcc_subset(n: int, box, rng: np.random.Generator, jitter: float = 0.05,
               cells=None, origin=(0.0, 0.0, 0.0)) -> np.ndarray:
    """n positions drawn from an fcc lattice filling ``box``.

    ``cells`` = fcc unit cells per axis (default: ceil((n/4)^(1/3)) cubic);
    a seeded random subset of n lattice sites is kept (no void region), then
    each coordinate is jittered by U(-jitter, +jitter).
    """
    box = np.asarray(box, dtype=np.float64)
    if cells is None:
        k = int(math.ceil((n / 4.0) ** (1.0 / 3.0) - 1e-9))
        cells = (k, k, k)
    cells = np.asarray(cells, dtype=np.int64)
    a = box / cells
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]], dtype=np.float64)
    total = 4 * int(np.prod(cells))
    assert total >= n, "lattice too small"
    pick = np.sort(rng.choice(total, size=n, replace=False))
    b = pick % 4
    c = pick // 4
    cx = c % cells[0]
    cy = (c // cells[0]) % cells[1]
    cz = c // (cells[0] * cells[1])
    frac = np.stack([cx, cy, cz], axis=1).astype(np.float64) + 0.25 + basis[b]
    pos = frac * a + np.asarray(origin, dtype=np.float64)
    pos += rng.uniform(-jitter, jitter, size=pos.shape)
    return pos


def random_quaternions(n: int, rng: np.random.Generator) -> np.ndarray:
    """Uniform random unit quaternions (w, x, y, z) by Shoemake's method."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    a, b = np.sqrt(1.0 - u1), np.sqrt(u1)
    q = np.stack([a * np.sin(2 * np.pi * u2), a * np.cos(2 * np.pi * u2),
                  b * np.sin(2 * np.pi * u3), b * np.cos(2 * np.pi * u3)], axis=1)
    return q


def _rotate_body_to_space(q: np.ndarray, v: np.ndarray) -> np.ndarray:
    """v' = q v q* for unit quaternions (w, x, y, z); input preparation only."""
    w = q[:, :1]
    u = q[:, 1:]
    t = 2.0 * np.cross(u, v)
    return v + w * t + np.cross(u, t)


def site_positions(model: dict, r: np.ndarray, q: np.ndarray):
    """Space-frame positions of every LJ centre, charge, dipole and
    quadrupole (input preparation only) and the owning molecule index."""
    pts = [e["pos"] for key in ("lj", "charges", "dipoles", "quads") for e in model[key]]
    n = r.shape[0]
    out = np.empty((n * len(pts), 3))
    own = np.repeat(np.arange(n), len(pts))
    for k, p in enumerate(pts):
        out[k::len(pts)] = r + _rotate_body_to_space(q, np.tile(np.asarray(p, float), (n, 1)))
    return out, own


def resolve_site_overlaps(model: dict, r: np.ndarray, q: np.ndarray, box, rng: np.random.Generator,
                          d_min: float = 0.6, max_passes: int = 100) -> np.ndarray:
    """Re-draw the orientation of molecules whose interaction sites come
    closer than d_min to a site of another molecule (periodic box), until
    none do or max_passes is reached.  Returns the new quaternions."""
    from scipy.spatial import cKDTree
    box = np.asarray(box, float)
    q = q.copy()
    for _ in range(max_passes):
        sp, own = site_positions(model, r, q)
        tree = cKDTree(np.mod(sp, box), boxsize=box)
        pairs = tree.query_pairs(d_min, output_type="ndarray")
        if len(pairs):
            pairs = pairs[own[pairs[:, 0]] != own[pairs[:, 1]]]
        if len(pairs) == 0:
            break
        bad = np.unique(np.maximum(own[pairs[:, 0]], own[pairs[:, 1]]))
        q[bad] = random_quaternions(len(bad), rng)
    return q


def relieve_site_overlaps(model: dict, r: np.ndarray, q: np.ndarray, box, rng: np.random.Generator,
                          d_min: float = 0.85, tries: int = 24, max_passes: int = 40) -> np.ndarray:
    """Geometric relief of close contacts between molecules of a lattice
    start with random orientations (positions stay).  Each pass finds the
    molecules with an interaction site closer than d_min to a site of
    another molecule, takes a random half of them, and gives each the
    orientation, among its current one and `tries` random ones, whose
    sites lie farthest from every other molecule's sites; until no contact
    is left or max_passes is reached.  Purely geometric: no interaction
    law is evaluated.  Returns the new quaternions."""
    from scipy.spatial import cKDTree
    box = np.asarray(box, float)
    pts = np.unique(np.array([e["pos"] for key in ("lj", "charges", "dipoles", "quads") for e in model[key]], float),
                    axis=0)
    S, n = len(pts), r.shape[0]
    q = q.copy()

    def sites(rr, qq):
        m = rr.shape[0]
        off = _rotate_body_to_space(np.repeat(qq, S, axis=0), np.tile(pts, (m, 1))).reshape(m, S, 3)
        return np.mod(rr[:, None, :] + off, box).reshape(-1, 3)

    own = np.repeat(np.arange(n), S)

    def nearest_other(tree, pos, mine):
        # distance from each point to the nearest site of another molecule
        # (among its S + 1 nearest sites: at most S are the molecule's own)
        d, idx = tree.query(pos, k=S + 1, workers=-1)
        return np.where(own[np.minimum(idx, n * S - 1)] == mine[:, None], np.inf, d).min(axis=1)

    for _ in range(max_passes):
        sp = sites(r, q)
        tree = cKDTree(sp, boxsize=box)
        close = nearest_other(tree, sp, own) < d_min
        if not close.any():
            break
        bad = np.unique(own[close])
        rng.shuffle(bad)
        bad = bad[: max(1, len(bad) // 2)]
        nb, K = len(bad), tries + 1
        cand = np.concatenate([q[bad][:, None, :], random_quaternions(nb * tries, rng).reshape(nb, tries, 4)], axis=1)
        d = nearest_other(tree, sites(np.repeat(r[bad], K, axis=0), cand.reshape(-1, 4)),
                          np.repeat(np.repeat(bad, K), S))
        best = d.reshape(nb, K, S).min(axis=2).argmax(axis=1)
        q[bad] = cand[np.arange(nb), best]
    return q


def mb_velocities(n: int, T: float, mass: float, rng: np.random.Generator) -> np.ndarray:
    """Maxwell-Boltzmann velocities at temperature T, zero total momentum,
    rescaled so that sum(m v^2) = (3n - 3) T exactly."""
    v = rng.normal(0.0, math.sqrt(T / mass), size=(n, 3))
    if n > 1:
        v -= v.mean(axis=0)
        k2 = mass * float((v * v).sum())
        v *= math.sqrt((3 * n - 3) * T / k2)
    return v


def angular_momenta(q: np.ndarray, moments: np.ndarray, T: float, rng: np.random.Generator) -> np.ndarray:
    """Space-frame angular momenta j = R(q) I omega_body with
    omega_k ~ N(0, sqrt(T / I_k)) for each nonzero principal moment."""
    n = q.shape[0]
    jb = np.zeros((n, 3))
    for k in range(3):
        if moments[k] > 1e-12:
            jb[:, k] = moments[k] * rng.normal(0.0, math.sqrt(T / moments[k]), size=n)
    return _rotate_body_to_space(q, jb)


def _state(model, box, rng, T, pos, oriented=True):
    n = pos.shape[0]
    m = model_mass(model)
    mom = model_principal_moments(model)
    if oriented and np.any(mom > 1e-12):
        q = random_quaternions(n, rng)
    else:
        q = np.tile(np.array([1.0, 0.0, 0.0, 0.0]), (n, 1))
    v = mb_velocities(n, T, m, rng)
    j = angular_momenta(q, mom, T, rng)
    box = np.asarray(box, dtype=np.float64)
    pos = np.mod(pos, box)
    return {"r": np.ascontiguousarray(pos), "v": np.ascontiguousarray(v),
            "q": np.ascontiguousarray(q), "j": np.ascontiguousarray(j)}


# --------------------------------------------------------------------------
# The five workloads (reduced units).  Each returns a dict with the model,
# box, cutoff, options, integration settings and the FP64 state.
# --------------------------------------------------------------------------

def config_lj_fluid(n: int = 4096, rho: float = 0.6, T: float = 0.95, rc: float = 2.5, seed_k: int = 0) -> dict:
    """Single-site LJTS fluid: jittered fcc subset, MB velocities at T."""
    rng = np.random.default_rng(seed_for(1, seed_k))
    L = (n / rho) ** (1.0 / 3.0)
    box = (L, L, L)
    model = model_lj()
    pos = fcc_subset(n, box, rng, jitter=0.05)
    st = _state(model, box, rng, T, pos, oriented=False)
    return {"name": f"lj-fluid-N{n}", "model": model, "box": box, "rc": rc,
            "lj_shift": 1, "lj_lrc": 0, "eps_rf": math.inf, "dt": 0.002, "T": T, **st}


def config_2cljq(n: int = 262144, rho: float = 0.55, T: float = 1.0, rc: float = 3.0, seed_k: int = 0,
                 relieve: bool = True) -> dict:
    """2CLJQ fluid (elongation 0.5, Q*^2 = 2): fcc subset, random
    orientations; with `relieve`, orientations giving intermolecular site
    contacts closer than 0.85 sigma are replaced (relieve_site_overlaps), so
    that the start is a fluid-like configuration (negative energy) rather
    than one dominated by a few overlapping pairs."""
    rng = np.random.default_rng(seed_for(2, seed_k))
    L = (n / rho) ** (1.0 / 3.0)
    box = (L, L, L)
    model = model_2cljq()
    pos = fcc_subset(n, box, rng, jitter=0.05)
    st = _state(model, box, rng, T, pos)
    if relieve:
        st["q"] = relieve_site_overlaps(model, st["r"], st["q"], box, rng, d_min=0.85)
        st["j"] = angular_momenta(st["q"], model_principal_moments(model), T, rng)
    return {"name": f"2cljq-N{n}", "model": model, "box": box, "rc": rc,
            "lj_shift": 0, "lj_lrc": 1, "eps_rf": math.inf, "dt": 0.001, "T": T, **st}


def config_slab(n: int = 4194304, rho_l: float = 0.73, rho_v: float = 0.02, frac_l: float = 0.4,
                T: float = 0.85, rc: float = 2.5, seed_k: int = 0) -> dict:
    """Vapour-liquid slab of single-site LJTS in a 1:1:4 periodic box.

    The liquid slab (density rho_l) is centred along z and fills frac_l of
    L_z: an fcc lattice over the slab, trimmed to count by a seeded random
    subset.  The vapour (density rho_v) fills the rest: a seeded random subset
    of a coarse simple-cubic grid with +-0.5 sigma jitter, which keeps every
    vapour molecule at least ~2.6 sigma from the others and ~1.4 sigma from
    the liquid faces.
    """
    rng = np.random.default_rng(seed_for(3, seed_k))
    V = n / (frac_l * rho_l + (1.0 - frac_l) * rho_v)
    Lx = (V / 4.0) ** (1.0 / 3.0)
    box = (Lx, Lx, 4.0 * Lx)
    Lz = box[2]
    n_l = int(round(rho_l * frac_l * V))
    n_v = n - n_l
    t = frac_l * Lz
    a_l = (4.0 / rho_l) ** (1.0 / 3.0)
    cxy = int(math.ceil(Lx / a_l))
    cz = int(math.ceil(t / a_l))
    while 4 * cxy * cxy * cz < n_l:
        cz += 1
    z0 = 0.5 * (Lz - t)
    liq = fcc_subset(n_l, (Lx, Lx, t), rng, jitter=0.05, cells=(cxy, cxy, cz), origin=(0.0, 0.0, z0))
    # vapour: the periodic interval [z0 + t, z0 + Lz) of length Lz - t; grid
    # layers sit half a spacing inside both ends, so no vapour molecule
    # approaches either liquid face closer than dz/2 - 0.5
    s = (1.0 / rho_v) ** (1.0 / 3.0)
    gxy = max(1, int(math.floor(Lx / s)))
    while True:
        gz = int(math.ceil(n_v / (gxy * gxy)))
        if (Lz - t) / gz >= 2.0:
            break
        gxy += 1
    total = gxy * gxy * gz
    pick = np.sort(rng.choice(total, size=n_v, replace=False)) if n_v > 0 else np.zeros(0, dtype=np.int64)
    ix = pick % gxy
    iy = (pick // gxy) % gxy
    iz = pick // (gxy * gxy)
    dz = (Lz - t) / gz
    zz = np.mod(z0 + t + (iz + 0.5) * dz, Lz)
    vap = np.stack([(ix + 0.5) * (Lx / gxy), (iy + 0.5) * (Lx / gxy), zz], axis=1)
    vap += rng.uniform(-0.5, 0.5, size=vap.shape)
    vap = np.mod(vap, np.asarray(box))
    pos = np.concatenate([liq, vap], axis=0)
    model = model_lj()
    st = _state(model, box, rng, T, pos, oriented=False)
    return {"name": f"lj-slab-N{n}", "model": model, "box": box, "rc": rc,
            "lj_shift": 1, "lj_lrc": 0, "eps_rf": math.inf, "dt": 0.002, "T": T,
            "n_liquid": n_l, "n_vapour": n_v, **st}


def config_lj_homogeneous(n: int, rho: float = 0.73, T: float = 0.85, rc: float = 2.5, seed_k: int = 1) -> dict:
    """Homogeneous LJTS fluid of n molecules (the single-evaluation size point)."""
    rng = np.random.default_rng(seed_for(3, seed_k))
    L = (n / rho) ** (1.0 / 3.0)
    box = (L, L, L)
    model = model_lj()
    pos = fcc_subset(n, box, rng, jitter=0.05)
    st = _state(model, box, rng, T, pos, oriented=False)
    return {"name": f"lj-homog-N{n}", "model": model, "box": box, "rc": rc,
            "lj_shift": 1, "lj_lrc": 0, "eps_rf": math.inf, "dt": 0.002, "T": T, **st}


def replica_specs(n_rep: int = 512, n_min: int = 500, n_max: int = 20000, seed_k: int = 0):
    """(N_k, rho_k, T_k) for the batched-replica workload: N log-uniform in
    [n_min, n_max], rho ~ U(0.05, 0.75), T ~ U(0.7, 1.3)."""
    rng = np.random.default_rng(seed_for(4, seed_k))
    ns = np.rint(np.exp(rng.uniform(math.log(n_min), math.log(n_max), size=n_rep))).astype(np.int64)
    rhos = rng.uniform(0.05, 0.75, size=n_rep)
    Ts = rng.uniform(0.7, 1.3, size=n_rep)
    return [(int(a), float(b), float(c)) for a, b, c in zip(ns, rhos, Ts)]


def config_replica(k: int, n: int, rho: float, T: float, rc: float = 3.0) -> dict:
    """One replica of the batched workload: 2CLJQ + dipole (mu*^2 = 1.5,
    Q*^2 = 2), reaction field with eps_RF = infinity, LRC on."""
    rng = np.random.default_rng(seed_for(4, 1000 + k))
    L = (n / rho) ** (1.0 / 3.0)
    box = (L, L, L)
    model = model_2cljdq()
    pos = fcc_subset(n, box, rng, jitter=0.05)
    st = _state(model, box, rng, T, pos)
    return {"name": f"replica{k}-N{n}", "model": model, "box": box, "rc": rc,
            "lj_shift": 0, "lj_lrc": 1, "eps_rf": math.inf, "dt": 0.001, "T": T, **st}


def config_4site(n: int = 50000, rho: float = 0.5, T: float = 1.0, rc: float = 3.0, cfg: int = 0) -> dict:
    """One configuration of the 4-site polar model (force-field gradient
    workload): fcc subset, random orientations (close intermolecular site
    contacts relieved, relieve_site_overlaps), seeded per configuration."""
    rng = np.random.default_rng(seed_for(5, cfg))
    L = (n / rho) ** (1.0 / 3.0)
    box = (L, L, L)
    model = model_4site()
    pos = fcc_subset(n, box, rng, jitter=0.05)
    st = _state(model, box, rng, T, pos)
    # lattice start with random orientations: relieve the close site
    # contacts between molecules (0.8 sigma)
    st["q"] = relieve_site_overlaps(model, st["r"], st["q"], box, rng, d_min=0.8)
    st["j"] = angular_momenta(st["q"], model_principal_moments(model), T, rng)
    return {"name": f"4site-N{n}-cfg{cfg}", "model": model, "box": box, "rc": rc,
            "lj_shift": 0, "lj_lrc": 1, "eps_rf": math.inf, "dt": 0.001, "T": T, **st}


def random_cluster(model: dict, n: int, box, rng: np.random.Generator, min_sep: float = 1.1,
                   region=None) -> dict:
    """n molecules at random positions (COM separation >= min_sep, by
    rejection), random orientations, random velocities/angular momenta.  Used
    for small hand-checkable test systems."""
    box = np.asarray(box, dtype=np.float64)
    lo, hi = (np.zeros(3), box) if region is None else (np.asarray(region[0]), np.asarray(region[1]))
    pts = []
    tries = 0
    while len(pts) < n:
        tries += 1
        assert tries < 200000, "cannot place molecules"
        p = rng.uniform(lo, hi)
        ok = True
        for o in pts:
            d = p - o
            d -= box * np.rint(d / box)
            if np.dot(d, d) < min_sep * min_sep:
                ok = False
                break
        if ok:
            pts.append(p)
    pos = np.array(pts)
    return _state(model, box, rng, 1.0, pos)


# --------------------------------------------------------------------------
# Cached ensembles (the overlap relief of the 4-site lattice starts takes
# seconds per configuration; generated configurations are kept on disk)
# --------------------------------------------------------------------------

_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_cache")


def _source_tag() -> str:
    import hashlib
    with open(os.path.abspath(__file__), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:12]


def _config_4site_cached(args):
    n, rho, T, rc, c = args
    path = os.path.join(_CACHE, f"4site_n{n}_rho{rho}_T{T}_rc{rc}_cfg{c}_{_source_tag()}.npz")
    if os.path.exists(path):
        z = np.load(path)
        st = {k: z[k] for k in ("r", "v", "q", "j")}
    else:
        cfg = config_4site(n=n, rho=rho, T=T, rc=rc, cfg=c)
        st = {k: cfg[k] for k in ("r", "v", "q", "j")}
        os.makedirs(_CACHE, exist_ok=True)
        tmp = path + f".{os.getpid()}.tmp.npz"
        np.savez(tmp, **st)
        os.replace(tmp, path)
    return st


def configs_4site(n_cfg: int, n: int = 50000, rho: float = 0.5, T: float = 1.0, rc: float = 3.0,
                  workers: int = 0) -> list:
    """Configurations 0 .. n_cfg-1 of config_4site, generated in parallel
    (a 'spawn' process pool: safe after the caller has initialised CUDA) and
    kept in mdgen/_cache/ keyed by the arguments and this file's contents."""
    import multiprocessing as mp
    jobs = [(n, rho, T, rc, c) for c in range(n_cfg)]
    workers = workers or min(len(jobs), os.cpu_count() or 1)
    if workers > 1 and len(jobs) > 1:
        with mp.get_context("spawn").Pool(workers) as pool:
            states = pool.map(_config_4site_cached, jobs)
    else:
        states = [_config_4site_cached(j) for j in jobs]
    base = config_4site(n=8, rho=rho, T=T, rc=rc)  # model and settings only
    out = []
    for c, st in enumerate(states):
        cfg = {k: v for k, v in base.items() if k not in ("r", "v", "q", "j")}
        L = (n / rho) ** (1.0 / 3.0)
        cfg.update(st, box=(L, L, L), name=f"4site-N{n}-cfg{c}")
        out.append(cfg)
    return out
