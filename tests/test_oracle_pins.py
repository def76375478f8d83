"""Pins of the FP64 oracle against facts other than itself (CPU only).

Each test states what fixes the expected value: a closed form of the paper's
Eq. 1, textbook electrostatics (plain Coulomb sums over explicit point-charge
clusters, the method of images), finite differences, invariants, numerical
quadrature, or brute force.  A plausible mistake in the oracle (a dropped
term, a wrong sign, an index or transposed operand) fails at least one.
"""
import copy
import json
import math
import os

import numpy as np
import pytest

import mdgen
import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
BIG = 60.0  # box edge for "isolated" systems
RC_BIG = 25.0


def two_mol(model, X, qa=(1, 0, 0, 0), qb=(1, 0, 0, 0), rc=RC_BIG, box=BIG, eps_rf=1.0, shift=0):
    """Molecule 0 at the box centre + X, molecule 1 at the centre."""
    c = np.full(3, box / 2.0)
    r = np.array([c + np.asarray(X, float), c])
    q = np.array([qa, qb], dtype=float)
    s = oracle.make_setup((box, box, box), rc, eps_rf=eps_rf, lj_shift=shift)
    return oracle.forces(model, s, r, q)


def lj_only(eps=(1.0,), sig=(1.0,), types=(0,), pos=((0, 0, 0),), xi=None, eta=None):
    return {"lj_types": {"eps": list(eps), "sigma": list(sig)}, "xi": xi, "eta": eta,
            "lj": [{"pos": p, "type": t, "mass": 1.0} for p, t in zip(pos, types)],
            "charges": [], "dipoles": [], "quads": []}


# ------------------------------------------------------------------ Eq. 1
@pytest.mark.parametrize("r", [1.0, 2.0 ** (1.0 / 6.0), 1.5, 2.5, 3.7])
def test_lj_closed_form(r):
    """Eq. 1: U = 4 eps [(sigma/r)^12 - (sigma/r)^6]; F = -dU/dr."""
    F, tau, o = two_mol(lj_only(), (r, 0, 0))
    U = 4.0 * (r ** -12 - r ** -6)
    dUdr = 4.0 * (-12 * r ** -13 + 6 * r ** -7)
    assert o["U"] == pytest.approx(U, rel=1e-14, abs=1e-15)
    assert F[0, 0] == pytest.approx(-dUdr, rel=1e-13, abs=1e-14)
    assert np.allclose(F[0], -F[1], rtol=0, atol=1e-15)
    assert o["W"] == pytest.approx(-r * dUdr, rel=1e-13, abs=1e-14)


def test_lj_special_points():
    """U(sigma) = 0; minimum -eps at r = 2^(1/6) sigma with zero force."""
    _, _, o = two_mol(lj_only(), (1.0, 0, 0))
    assert abs(o["U"]) < 1e-15
    F, _, o = two_mol(lj_only(), (2.0 ** (1 / 6), 0, 0))
    assert o["U"] == pytest.approx(-1.0, rel=1e-14)
    assert abs(F[0, 0]) < 1e-13
    _, _, o = two_mol(lj_only(), (1.5, 0, 0))
    assert o["U"] == pytest.approx(-0.32033659, abs=1e-8)  # 4 (1.5^-12 - 1.5^-6)


def test_ljts_shift_and_cutoff():
    """LJTS: energy shifted to vanish at rc, force unchanged; pairs at or
    beyond rc (centre-of-mass distance) do not interact."""
    rc = 2.5
    F0, _, o0 = two_mol(lj_only(), (2.0, 0, 0), rc=rc, shift=0)
    F1, _, o1 = two_mol(lj_only(), (2.0, 0, 0), rc=rc, shift=1)
    assert o1["U"] == pytest.approx(o0["U"] - 4.0 * (rc ** -12 - rc ** -6), rel=1e-14)
    assert np.array_equal(F0, F1)
    _, _, o = two_mol(lj_only(), (rc * (1 - 1e-12), 0, 0), rc=rc, shift=1)
    assert abs(o["U"]) < 1e-12 and o["n_mol_pairs"] == 1
    _, _, o = two_mol(lj_only(), (rc, 0, 0), rc=rc, shift=1)
    assert o["n_mol_pairs"] == 0 and o["U"] == 0.0


def test_lorentz_berthelot():
    """§2 combination rules: eps_ab = xi sqrt(eps_a eps_b), sigma_ab = eta (sigma_a + sigma_b)/2."""
    m = lj_only(eps=(1.0, 0.25), sig=(1.0, 2.0))
    # unlike pair: molecule with type-0 site and molecule with type-1 site is
    # not expressible with one component, so use a two-site model and compare
    # the sum of the four site pairs at large separation along x.
    m = lj_only(eps=(1.0, 0.25), sig=(1.0, 2.0), types=(0, 1), pos=((0, 0, -5.0), (0, 0, 5.0)))
    X = (3.0, 0, 0)
    _, _, o = two_mol(m, X)
    def u(e, s, r):
        return 4 * e * ((s / r) ** 12 - (s / r) ** 6)
    r_cross = math.sqrt(9.0 + 100.0)
    ref = u(1.0, 1.0, 3.0) + u(0.25, 2.0, 3.0) + 2 * u(0.5, 1.5, r_cross)
    assert o["U"] == pytest.approx(ref, rel=1e-13)
    xi = [[1.0, 0.9], [0.9, 1.0]]
    eta = [[1.0, 1.1], [1.1, 1.0]]
    m2 = copy.deepcopy(m)
    m2["xi"], m2["eta"] = xi, eta
    _, _, o = two_mol(m2, X)
    ref = u(1.0, 1.0, 3.0) + u(0.25, 2.0, 3.0) + 2 * u(0.45, 1.65, r_cross)
    assert o["U"] == pytest.approx(ref, rel=1e-13)


# ---------------------------------------------- §2 multipoles: textbook values
def test_textbook_dipole_quadrupole_values():
    """Classic fixed-orientation energies (Gray & Gubbins conventions):
    dipoles head-to-tail -2 mu^2/r^3, side-by-side antiparallel -mu^2/r^3;
    linear quadrupoles end-to-end +6 Q^2/r^5, T-shape -3 Q^2/r^5 ... with
    the parallel side-by-side arrangement +3 Q^2/(4 r^5)."""
    mu, Q, r = 1.3, 0.9, 2.0
    dip = {"lj_types": {"eps": [], "sigma": []}, "xi": None, "eta": None, "lj": [], "charges": [],
           "dipoles": [{"pos": (0, 0, 0), "axis": (1, 0, 0), "mu": mu}], "quads": []}
    _, _, o = two_mol(dip, (r, 0, 0))
    assert o["U"] == pytest.approx(-2 * mu * mu / r ** 3, rel=1e-13)
    flip = (0.0, 0.0, 0.0, 1.0)  # 180 degrees about z: x -> -x
    _, _, o = two_mol(dip, (0, r, 0), qa=(1, 0, 0, 0), qb=flip)
    assert o["U"] == pytest.approx(-mu * mu / r ** 3, rel=1e-13)
    quad = {"lj_types": {"eps": [], "sigma": []}, "xi": None, "eta": None, "lj": [], "charges": [],
            "dipoles": [], "quads": [{"pos": (0, 0, 0), "axis": (1, 0, 0), "Q": Q}]}
    _, _, o = two_mol(quad, (r, 0, 0))
    assert o["U"] == pytest.approx(6 * Q * Q / r ** 5, rel=1e-13)
    rot90 = (math.cos(math.pi / 4), 0.0, 0.0, math.sin(math.pi / 4))  # x -> y
    _, _, o = two_mol(quad, (r, 0, 0), qa=(1, 0, 0, 0), qb=rot90)
    assert o["U"] == pytest.approx(-3 * Q * Q / r ** 5, rel=1e-13)
    _, _, o = two_mol(quad, (0, r, 0))
    assert o["U"] == pytest.approx(2.25 * Q * Q / r ** 5, rel=1e-13)


# --------------------------- §2 multipoles vs explicit point-charge clusters
def _cluster_model(model, h):
    """Replace every dipole by charges +-mu/h at +-h/2 along its axis and
    every linear quadrupole by (q, -2q, q) at (-h, 0, +h) with 2 q h^2 = Q."""
    m = copy.deepcopy(model)
    ch = list(m["charges"])
    for d in m["dipoles"]:
        p, e, mu = np.array(d["pos"]), np.array(d["axis"]), d["mu"]
        ch.append({"pos": tuple(p + 0.5 * h * e), "q": mu / h})
        ch.append({"pos": tuple(p - 0.5 * h * e), "q": -mu / h})
    for qd in m["quads"]:
        p, e, Q = np.array(qd["pos"]), np.array(qd["axis"]), qd["Q"]
        qq = Q / (2 * h * h)
        ch.append({"pos": tuple(p + h * e), "q": qq})
        ch.append({"pos": tuple(p), "q": -2 * qq})
        ch.append({"pos": tuple(p - h * e), "q": qq})
    m["charges"] = ch
    m["dipoles"] = []
    m["quads"] = []
    return m


def _richardson(f, h):
    """Three-level Richardson extrapolation to h -> 0 of an even function."""
    a, b, c = f(h), f(h / 2), f(h / 4)
    r1 = (4 * b - a) / 3
    r2 = (4 * c - b) / 3
    return (16 * r2 - r1) / 15


MIXES = {
    "q": dict(charges=[{"pos": (0.1, -0.2, 0.05), "q": 0.7}]),
    "mu": dict(dipoles=[{"pos": (0.1, 0.2, -0.1), "axis": (0.6, 0.0, 0.8), "mu": 1.1}]),
    "Q": dict(quads=[{"pos": (-0.15, 0.1, 0.2), "axis": (0.0, 0.6, 0.8), "Q": 0.9}]),
    "q+mu": dict(charges=[{"pos": (0.3, 0.0, 0.0), "q": -0.5}],
                 dipoles=[{"pos": (-0.2, 0.1, 0.0), "axis": (0.0, 0.0, 1.0), "mu": 1.2}]),
    "q+Q": dict(charges=[{"pos": (0.0, 0.3, 0.0), "q": 0.6}],
                quads=[{"pos": (0.1, -0.2, 0.1), "axis": (0.8, 0.6, 0.0), "Q": 1.1}]),
    "mu+Q": dict(dipoles=[{"pos": (0.0, 0.0, 0.25), "axis": (0.0, 1.0, 0.0), "mu": 0.9}],
                 quads=[{"pos": (0.2, 0.0, -0.1), "axis": (0.6, 0.0, 0.8), "Q": 1.3}]),
    "all": dict(charges=[{"pos": (0.3, 0.0, 0.0), "q": 0.4}, {"pos": (-0.3, 0.0, 0.0), "q": -0.4}],
                dipoles=[{"pos": (0.0, 0.2, 0.0), "axis": (0.0, 1.0, 0.0), "mu": 1.2}],
                quads=[{"pos": (0.0, 0.2, 0.0), "axis": (0.0, 0.0, 1.0), "Q": 1.4}]),
}


def _mix_model(name):
    m = {"lj_types": {"eps": [], "sigma": []}, "xi": None, "eta": None, "lj": [],
         "charges": [], "dipoles": [], "quads": []}
    m.update(copy.deepcopy(MIXES[name]))
    return m


@pytest.mark.parametrize("name", list(MIXES))
@pytest.mark.parametrize("seed", [0, 1])
def test_multipoles_match_point_charge_clusters(name, seed):
    """Energy, force and torque of every multipole law (charge, dipole,
    quadrupole and all cross terms) equal the h -> 0 limit of plain Coulomb
    sums over explicit point-charge clusters."""
    rng = np.random.default_rng(100 + seed)
    model = _mix_model(name)
    X = rng.normal(size=3)
    X *= (1.8 + rng.random()) / np.linalg.norm(X)
    qa, qb = mdgen.random_quaternions(2, rng)
    F, tau, o = two_mol(model, X, qa, qb)

    def cl(h, what):
        Fc, tc, oc = two_mol(_cluster_model(model, h), X, qa, qb)
        return {"U": oc["U"], "F": Fc[0], "t0": tc[0], "t1": tc[1], "W": oc["W"]}[what]

    h = 0.08  # balances the O(h^6) remainder against cancellation in the cluster sums
    U_lim = _richardson(lambda hh: cl(hh, "U"), h)
    assert o["U"] == pytest.approx(U_lim, rel=1e-7, abs=1e-9)
    W_lim = _richardson(lambda hh: cl(hh, "W"), h)
    assert o["W"] == pytest.approx(W_lim, rel=1e-7, abs=1e-9)
    for what, ref in (("F", F[0]), ("t0", tau[0]), ("t1", tau[1])):
        lim = _richardson(lambda hh: cl(hh, what), h)
        assert np.allclose(ref, lim, rtol=1e-6, atol=1e-7 * np.abs(ref).max()), (what, ref, lim)


# -------------------------------------------------- reaction field (§1, §3)
def test_reaction_field_conducting_limit_is_method_of_images():
    """eps_RF = infinity: the cavity of radius rc around dipole j is a
    grounded conductor.  The field of j's image charges at dipole i,
    computed by the method of images for an explicit +-q pair, gives the
    reaction-field pair energy in the limit h -> 0."""
    rc, mu_i, mu_j = 3.0, 1.1, 0.8
    rng = np.random.default_rng(7)
    X = rng.normal(size=3)
    X *= 1.7 / np.linalg.norm(X)
    ea = rng.normal(size=3); ea /= np.linalg.norm(ea)
    eb = rng.normal(size=3); eb /= np.linalg.norm(eb)

    def images_energy(h):
        # j's dipole as charges at +-h/2 eb about the origin; each charge qk
        # at s_k has an image -qk rc/|s_k| at s_k rc^2/|s_k|^2.  Dipole i is
        # the pair +-mu_i/h at X +- h/2 ea.
        qj = [(mu_j / h, 0.5 * h * eb), (-mu_j / h, -0.5 * h * eb)]
        qi = [(mu_i / h, X + 0.5 * h * ea), (-mu_i / h, X - 0.5 * h * ea)]
        U = 0.0
        for qk, sk in qj:
            ns = np.linalg.norm(sk)
            qim, sim = -qk * rc / ns, sk * rc * rc / ns ** 2
            for ql, pl in qi:
                U += ql * qim / np.linalg.norm(pl - sim)
        return U

    U_img = _richardson(images_energy, 0.02)
    m = {"lj_types": {"eps": [], "sigma": []}, "xi": None, "eta": None, "lj": [], "charges": [],
         "dipoles": [{"pos": (0, 0, 0), "axis": (0, 0, 1), "mu": 1.0}], "quads": []}
    qa = _quat_from_z(ea)
    qb = _quat_from_z(eb)
    s_inf = oracle.make_setup((BIG,) * 3, rc, eps_rf=math.inf)
    s_vac = oracle.make_setup((BIG,) * 3, rc, eps_rf=1.0)
    c = np.full(3, BIG / 2)
    r = np.array([c + X, c])
    _, _, oi = oracle.forces(m, s_inf, r, np.array([qa, qb]))
    _, _, ov = oracle.forces(m, s_vac, r, np.array([qa, qb]))
    # the pair energy scales with mu_i mu_j; the oracle model has mu = 1
    assert (oi["U"] - ov["U"]) * mu_i * mu_j == pytest.approx(U_img, rel=1e-7)


def test_reaction_field_self_energy_is_method_of_images():
    """§3 reaction field, self term (reading R4): a molecule's own dipoles at
    the centre of a grounded conducting cavity of radius rc (eps_RF = inf)
    meet the field of their own images.  Two dipoles of one molecule as
    explicit +-q pairs at the centre, Kelvin images of every charge, half
    the charge-image energy, h -> 0: -|sum_a mu_a e_a|^2 / (2 rc^3) per
    molecule.  Pins the sign, the 1/2, the rc^-3 and the cross term of two
    dipoles of one molecule."""
    rc = 3.0
    dips = [(1.1, np.array([0.6, 0.0, 0.8])), (0.7, np.array([0.0, 1.0, 0.0]))]

    def images_self_energy(h):
        ch = []
        for mu, e in dips:
            ch += [(mu / h, 0.5 * h * e), (-mu / h, -0.5 * h * e)]
        U = 0.0
        for qk, sk in ch:
            ns = np.linalg.norm(sk)
            qim, sim = -qk * rc / ns, sk * rc * rc / ns ** 2
            for ql, pl in ch:
                U += 0.5 * ql * qim / np.linalg.norm(pl - sim)
        return U

    U_img = _richardson(images_self_energy, 0.02)
    m = {"lj_types": {"eps": [], "sigma": []}, "xi": None, "eta": None, "lj": [], "charges": [],
         "dipoles": [{"pos": (0, 0, 0), "axis": tuple(e), "mu": mu} for mu, e in dips], "quads": []}
    n = 7
    s = oracle.make_setup((BIG,) * 3, rc, eps_rf=math.inf)
    assert oracle.lrc(m, s, n)[2] == pytest.approx(n * U_img, rel=1e-8)


def test_reaction_field_self_energy_hand_values():
    """The self term for one point dipole mu per molecule: -N mu^2 / (2 rc^3)
    at eps_RF = inf, nothing at eps_RF = 1 (no continuum), and the Onsager
    factor 2 (eps - 1) / (2 eps + 1) of the cavity field in between; two
    dipoles of one molecule enter through their vector sum (antiparallel
    equal dipoles cancel)."""
    rc, n, mu = 2.5, 10, 1.3
    one = {"lj_types": {"eps": [], "sigma": []}, "xi": None, "eta": None, "lj": [], "charges": [],
           "dipoles": [{"pos": (0.2, 0, 0), "axis": (0, 0, 1), "mu": mu}], "quads": []}
    box = (BIG,) * 3
    assert oracle.lrc(one, oracle.make_setup(box, rc, eps_rf=math.inf), n)[2] == pytest.approx(
        -n * mu * mu / (2 * rc ** 3), rel=1e-14)
    assert oracle.lrc(one, oracle.make_setup(box, rc, eps_rf=1.0), n)[2] == 0.0
    for eps in (2.0, 8.0, 80.0):
        f = 2 * (eps - 1) / (2 * eps + 1)
        assert oracle.lrc(one, oracle.make_setup(box, rc, eps_rf=eps), n)[2] == pytest.approx(
            -f * n * mu * mu / (2 * rc ** 3), rel=1e-14)
    anti = copy.deepcopy(one)
    anti["dipoles"].append({"pos": (-0.2, 0, 0), "axis": (0, 0, -1), "mu": mu})
    assert oracle.lrc(anti, oracle.make_setup(box, rc, eps_rf=math.inf), n)[2] == 0.0
    perp = copy.deepcopy(one)
    perp["dipoles"].append({"pos": (-0.2, 0, 0), "axis": (1, 0, 0), "mu": 0.5})
    assert oracle.lrc(perp, oracle.make_setup(box, rc, eps_rf=math.inf), n)[2] == pytest.approx(
        -n * (mu * mu + 0.25) / (2 * rc ** 3), rel=1e-14)


def test_reaction_field_vacuum_vanishes_and_no_force():
    """eps_RF = 1 (no dielectric continuum) gives no reaction field; the RF
    term never changes forces, only energy and torques."""
    m = _mix_model("mu")
    rng = np.random.default_rng(3)
    X = np.array([1.2, -0.7, 0.9])
    qa, qb = mdgen.random_quaternions(2, rng)
    F1, t1, o1 = two_mol(m, X, qa, qb, rc=3.0, eps_rf=1.0)
    F2, t2, o2 = two_mol(m, X, qa, qb, rc=3.0, eps_rf=math.inf)
    Fc, tc, oc = two_mol(_cluster_model(m, 1e-3), X, qa, qb, rc=3.0, eps_rf=1.0)
    assert o1["U"] == pytest.approx(oc["U"], rel=1e-5)
    assert np.allclose(F1, F2, rtol=1e-13, atol=1e-14)
    assert not np.allclose(t1, t2)


def _quat_from_z(e):
    """Unit quaternion rotating +z onto e."""
    z = np.array([0.0, 0.0, 1.0])
    e = np.asarray(e, float) / np.linalg.norm(e)
    c = float(np.dot(z, e))
    if c < -1 + 1e-12:
        return np.array([0.0, 1.0, 0.0, 0.0])
    axis = np.cross(z, e)
    w = math.sqrt((1 + c) / 2)
    v = axis / (2 * w)
    return np.array([w, *v])


def test_rotmat_is_rotation():
    rng = np.random.default_rng(0)
    for q in mdgen.random_quaternions(20, rng):
        R = oracle.rotmat(q)
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-14)
        assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-14)
        # quaternion rotation of a vector, written with the Hamilton product
        v = rng.normal(size=3)
        w, u = q[0], q[1:]
        ref = v + 2 * w * np.cross(u, v) + 2 * np.cross(u, np.cross(u, v))
        assert np.allclose(R @ v, ref, atol=1e-14)


# ---------------------------------------------------- finite differences
MODELS_FD = {
    "lj": mdgen.model_lj(),
    "2cljq": mdgen.model_2cljq(),
    "2cljdq": mdgen.model_2cljdq(),
    "4site": mdgen.model_4site(),
}


def _small_system(model, n=12, L=9.0, seed=0):
    rng = np.random.default_rng(seed)
    st = mdgen.random_cluster(model, n, (L, L, L), rng, min_sep=1.6)
    return st, oracle.make_setup((L, L, L), 3.0, eps_rf=math.inf, lj_shift=0)


def _energy(model, s, r, q):
    return oracle.forces(model, s, r, q)[2]["U"]


@pytest.mark.parametrize("name", list(MODELS_FD))
def test_forces_are_minus_gradient(name):
    """F_i = -dU/dR_i by central differences (PBC, brute force)."""
    model = MODELS_FD[name]
    st, s = _small_system(model)
    F, _, _ = oracle.forces(model, s, st["r"], st["q"])
    h = 1e-6
    for i in (0, 5, 11):
        for k in range(3):
            rp = st["r"].copy(); rp[i, k] += h
            rm = st["r"].copy(); rm[i, k] -= h
            g = (_energy(model, s, rp, st["q"]) - _energy(model, s, rm, st["q"])) / (2 * h)
            assert -g == pytest.approx(F[i, k], rel=1e-6, abs=1e-6 * max(1.0, abs(F[i]).max()))


def _rotate_quat(q, axis, ang):
    a = np.asarray(axis, float) / np.linalg.norm(axis)
    p = np.array([math.cos(ang / 2), *(math.sin(ang / 2) * a)])
    w1, v1 = p[0], p[1:]
    w2, v2 = q[0], q[1:]
    return np.array([w1 * w2 - v1 @ v2, *(w1 * v2 + w2 * v1 + np.cross(v1, v2))])


@pytest.mark.parametrize("name", ["2cljq", "2cljdq", "4site"])
def test_torques_are_minus_angular_gradient(name):
    """tau_i . n = -dU/dphi for a rotation of molecule i by phi about the
    space-frame axis n through its centre of mass."""
    model = MODELS_FD[name]
    st, s = _small_system(model, seed=1)
    _, tau, _ = oracle.forces(model, s, st["r"], st["q"])
    h = 1e-6
    for i in (0, 7):
        for k in range(3):
            n = np.eye(3)[k]
            qp = st["q"].copy(); qp[i] = _rotate_quat(qp[i], n, h)
            qm = st["q"].copy(); qm[i] = _rotate_quat(qm[i], n, -h)
            g = (_energy(model, s, st["r"], qp) - _energy(model, s, st["r"], qm)) / (2 * h)
            assert -g == pytest.approx(tau[i, k], rel=1e-6, abs=1e-6 * max(1.0, abs(tau[i]).max()))


@pytest.mark.parametrize("name", list(MODELS_FD))
def test_virial_is_minus_scaling_derivative(name):
    """Molecular virial: W_aa = -dU/dlambda_a when centre-of-mass positions
    and the box are scaled by (1 + lambda_a) along axis a (orientations fixed)."""
    model = MODELS_FD[name]
    st, s = _small_system(model, seed=2)
    _, _, o = oracle.forces(model, s, st["r"], st["q"])
    L = np.array(list(s.box))
    h = 1e-7
    tot = 0.0
    for k, key in enumerate(("Wxx", "Wyy", "Wzz")):
        vals = []
        for sgn in (1, -1):
            fac = np.ones(3); fac[k] += sgn * h
            s2 = oracle.make_setup(tuple(L * fac), 3.0, eps_rf=math.inf)
            vals.append(_energy(model, s2, st["r"] * fac, st["q"]))
        d = (vals[0] - vals[1]) / (2 * h)
        assert -d == pytest.approx(o[key], rel=1e-6, abs=1e-6)
        tot += o[key]
    assert tot == pytest.approx(o["W"], rel=1e-12)


# ------------------------------------------------------------- invariants
@pytest.mark.parametrize("name", list(MODELS_FD))
def test_invariants(name):
    """Zero net force (PBC); zero net torque about the origin and rotational
    invariance of U for an isolated cluster; translation and relabelling
    invariance."""
    model = MODELS_FD[name]
    st, s = _small_system(model, n=20, L=10.0, seed=4)
    F, tau, o = oracle.forces(model, s, st["r"], st["q"])
    scale = np.abs(F).max()
    assert np.abs(F.sum(axis=0)).max() < 1e-12 * max(1.0, scale) * 20
    # translation with wrap
    r2 = np.mod(st["r"] + np.array([3.3, -1.7, 8.1]), 10.0)
    _, _, o2 = oracle.forces(model, s, r2, st["q"])
    assert o2["U"] == pytest.approx(o["U"], rel=1e-12)
    # relabelling
    p = np.random.default_rng(1).permutation(20)
    Fp, tp, op = oracle.forces(model, s, st["r"][p], st["q"][p])
    assert op["U"] == pytest.approx(o["U"], rel=1e-12)
    assert np.allclose(Fp, F[p], atol=1e-12 * max(1, scale))
    # isolated cluster: no periodic images within the cut-off
    rng = np.random.default_rng(5)
    stc = mdgen.random_cluster(model, 10, (BIG,) * 3, rng, min_sep=1.15,
                               region=((27, 27, 27), (33, 33, 33)))
    sc = oracle.make_setup((BIG,) * 3, RC_BIG, eps_rf=1.0)
    Fc, tc, oc = oracle.forces(model, sc, stc["r"], stc["q"])
    net_t = np.cross(stc["r"], Fc).sum(axis=0) + tc.sum(axis=0)
    assert np.abs(net_t).max() < 1e-10 * max(1.0, np.abs(Fc).max() * BIG)
    qrot = np.array([0.3, -0.5, 0.7, 0.4]); qrot /= np.linalg.norm(qrot)
    Rm = oracle.rotmat(qrot)
    cen = np.full(3, BIG / 2)
    rr = (stc["r"] - cen) @ Rm.T + cen
    w1, v1 = qrot[0], qrot[1:]
    qq = np.array([[w1 * q[0] - v1 @ q[1:], *(w1 * q[1:] + q[0] * v1 + np.cross(v1, q[1:]))] for q in stc["q"]])
    _, _, orr = oracle.forces(model, sc, rr, qq)
    assert orr["U"] == pytest.approx(oc["U"], rel=1e-11)


# -------------------------------------------------- brute force vs cells
@pytest.mark.parametrize("which", ["lj", "2cljq", "4site", "2cljdq-smallbox"])
def test_brute_force_equals_linked_cells(which):
    """§3 linked cells change only the order of summation."""
    if which == "lj":
        cfg = mdgen.config_lj_fluid(n=864)
    elif which == "2cljq":
        cfg = mdgen.config_2cljq(n=1000)
    elif which == "4site":
        cfg = mdgen.config_4site(n=800)
    else:
        cfg = mdgen.config_replica(0, 500, 0.7, 1.0)  # 2 cells per axis
    s = oracle.setup_from_config(cfg)
    Fb, tb, ob = oracle.forces(cfg["model"], s, cfg["r"], cfg["q"])
    Fc, tc, oc = oracle.forces(cfg["model"], s, cfg["r"], cfg["q"], use_cells=True)
    sc = np.abs(Fb).max()
    assert np.allclose(Fb, Fc, rtol=0, atol=1e-11 * sc)
    assert np.allclose(tb, tc, rtol=0, atol=1e-11 * max(1, np.abs(tb).max()))
    assert oc["U"] == pytest.approx(ob["U"], rel=1e-12)
    assert oc["W"] == pytest.approx(ob["W"], rel=1e-12)
    assert oc["n_mol_pairs"] == ob["n_mol_pairs"]


@pytest.mark.parametrize("which", ["2cljq", "4site"])
def test_forces_subset_equals_full_evaluation(which):
    """orc_forces_subset (the checker of sampled parity on systems too large
    for a full evaluation) returns, for each selected molecule in selection
    order, exactly the row of the full linked-cell evaluation; selections
    include molecules in the first and last cells (periodic neighbours),
    repeats and an unsorted order."""
    cfg = mdgen.config_2cljq(n=1500) if which == "2cljq" else mdgen.config_4site(n=900)
    s = oracle.setup_from_config(cfg)
    F, tau, _ = oracle.forces(cfg["model"], s, cfg["r"], cfg["q"], use_cells=True)
    r = cfg["r"]
    L = np.asarray(cfg["box"])
    edge = np.where(((r % L) < 0.5).any(axis=1) | ((r % L) > L - 0.5).any(axis=1))[0]
    rng = np.random.default_rng(5)
    sel = np.concatenate([edge[:20], rng.choice(r.shape[0], 40, replace=False), edge[:3], [0, r.shape[0] - 1, 0]])
    rng.shuffle(sel)
    Fs, ts = oracle.forces_subset(cfg["model"], s, cfg["r"], cfg["q"], sel)
    assert Fs.shape == (sel.shape[0], 3) and ts.shape == (sel.shape[0], 3)
    scF, sct = np.abs(F).max(), np.abs(tau).max()
    assert np.allclose(Fs, F[sel], rtol=0, atol=1e-14 * scF)
    assert np.allclose(ts, tau[sel], rtol=0, atol=1e-14 * sct)


# ------------------------------------------------------- hit ratio (§3)
def test_hit_fraction_matches_paper():
    """§3: with cells of edge rc a homogeneous configuration has ~16% of the
    examined distances inside rc (sphere 4.2 rc^3 vs 27 rc^3 examined)."""
    g = json.load(open(os.path.join(HERE, "golden", "paper_numbers.json")))
    assert g["sphere_volume_rc3"]["value"] == pytest.approx(4 * math.pi / 3, abs=0.02)
    rc, nc, n = 2.0, 6, 4000
    L = rc * nc  # cell edge exactly rc (oracle: floor(L/rc) cells)
    rng = np.random.default_rng(11)
    r = rng.uniform(0, L, size=(n, 3))
    q = np.tile([1.0, 0, 0, 0], (n, 1))
    s = oracle.make_setup((L, L, L), rc * (1 - 1e-9))
    _, _, o = oracle.forces(mdgen.model_lj(), s, r, q, use_cells=True)
    frac = o["n_mol_pairs"] / o["n_examined"]
    assert frac == pytest.approx(g["hit_fraction_rc_cells"]["value"], abs=0.01)
    assert frac == pytest.approx((4 * math.pi / 3) / 27, rel=0.03)


# ----------------------------------------------- long-range correction (§3)
def test_lrc_equals_quadrature_of_eq1():
    """U_LRC and W_LRC are the mean-field tail integrals of Eq. 1 with g = 1
    beyond rc, summed over LJ centre pairs (numerical quadrature here)."""
    from scipy.integrate import quad
    model = mdgen.model_4site()
    n, L, rc = 1234, 13.0, 3.0
    s = oracle.make_setup((L, L, L), rc, lj_lrc=1)
    U, W, _ = oracle.lrc(model, s, n)
    T = model["lj_types"]
    Uq = Wq = 0.0
    for a in model["lj"]:
        for b in model["lj"]:
            e = math.sqrt(T["eps"][a["type"]] * T["eps"][b["type"]])
            sg = 0.5 * (T["sigma"][a["type"]] + T["sigma"][b["type"]])
            u = lambda r: 4 * e * ((sg / r) ** 12 - (sg / r) ** 6)
            du = lambda r: 4 * e * (-12 * sg ** 12 / r ** 13 + 6 * sg ** 6 / r ** 7)
            Uq += quad(lambda r: r * r * u(r), rc, np.inf, epsabs=1e-14, epsrel=1e-12)[0]
            Wq += quad(lambda r: r * r * (-r * du(r)), rc, np.inf, epsabs=1e-14, epsrel=1e-12)[0]
    pre = 2 * math.pi * n * n / L ** 3
    assert U == pytest.approx(pre * Uq, rel=1e-9)
    assert W == pytest.approx(pre * Wq, rel=1e-9)
    s0 = oracle.make_setup((L, L, L), rc, lj_lrc=0)
    assert oracle.lrc(model, s0, n)[:2] == (0.0, 0.0)


# ---------------------------------------------------------- leapfrog (§3)
def test_free_linear_rotor_matches_exact_rotation():
    """Eqs. 4-5 with no torque: a linear rotor with j perpendicular to its
    axis spins about j at omega = |j|/I; the numerical axis converges to the
    exact one at second order in dt."""
    model = mdgen.model_2cljq()
    I = 0.0625
    L = 40.0
    s = oracle.make_setup((L, L, L), 3.0)
    q0 = _quat_from_z(np.array([1.0, 0.2, -0.3]))
    e0 = oracle.rotmat(q0)[:, 2]
    jdir = np.cross(e0, [0.0, 0.0, 1.0]); jdir /= np.linalg.norm(jdir)
    omega = 1.3
    j0 = I * omega * jdir
    errs = []
    tfin = 1.0
    for dt in (0.01, 0.005):
        st = {"r": np.array([[20.0, 20.0, 20.0]]), "v": np.zeros((1, 3)), "q": q0[None, :].copy(),
              "j": j0[None, :].copy(), "F": np.zeros((1, 3)), "tau": np.zeros((1, 3))}
        out = oracle.step(model, s, st, dt, int(round(tfin / dt)))
        e = oracle.rotmat(out["q"][0])[:, 2]
        ang = omega * tfin
        ex = e0 * math.cos(ang) + np.cross(jdir, e0) * math.sin(ang)  # Rodrigues, e0 . jdir = 0
        errs.append(np.linalg.norm(e - ex))
        assert np.allclose(out["j"], j0, atol=1e-15)
    assert errs[0] < 1e-4
    assert 3.0 < errs[0] / errs[1] < 5.0


def test_translational_time_reversal():
    """Eqs. 2-3 are time-reversible: after n steps, reversing the
    half-step velocity (advanced by a full kick) retraces the trajectory."""
    cfg = mdgen.config_lj_fluid(n=256)
    s = oracle.setup_from_config(cfg)
    st = {k: cfg[k] for k in ("r", "v", "q", "j")}
    out = oracle.step(cfg["model"], s, st, 0.002, 50)
    back = dict(out)
    back["v"] = -(out["v"] + 0.002 * out["F"])
    ret = oracle.step(cfg["model"], s, back, 0.002, 50)
    d = ret["r"] - cfg["r"]
    d -= np.array(cfg["box"]) * np.rint(d / np.array(cfg["box"]))
    assert np.abs(d).max() < 1e-9


def test_energy_fluctuation_scales_as_dt_squared():
    """Leapfrog (Eqs. 2-5): for an isolated cluster of asymmetric rigid
    molecules (every pair inside the cut-off, so no energy jumps at rc) the
    RMS fluctuation of the total energy over a fixed time span shrinks ~4x
    when dt is halved, and the total angular momentum is conserved."""
    model = mdgen.model_4site()
    rng = np.random.default_rng(21)
    st0 = mdgen.random_cluster(model, 8, (BIG,) * 3, rng, min_sep=1.7, region=((27, 27, 27), (33, 33, 33)))
    s = oracle.make_setup((BIG,) * 3, RC_BIG, eps_rf=math.inf)
    res = []
    for dt in (0.002, 0.001):
        st = {k: st0[k].copy() for k in ("r", "v", "q", "j")}
        st["v"] -= st["v"].mean(axis=0)
        F, tau, _ = oracle.forces(model, s, st["r"], st["q"])
        st["F"], st["tau"] = F, tau
        E = []
        Lang = []
        n = int(round(0.4 / dt))
        for k in range(n):
            st = oracle.step(model, s, st, dt, 1)
            kt, kr = oracle.kinetic(model, dt, st["v"], st["q"], st["j"], st["F"], st["tau"])
            E.append(st["obs"]["U"] + kt + kr)
            vt = st["v"] + 0.5 * dt * st["F"]
            jt = st["j"] + 0.5 * dt * st["tau"]
            Lang.append(np.cross(st["r"], vt).sum(axis=0) + jt.sum(axis=0))
        res.append(np.std(np.array(E)))
        Lang = np.array(Lang)
        assert np.abs(Lang - Lang[0]).max() < 1e-9 * max(1.0, np.abs(Lang).max())
    ratio = res[0] / res[1]
    assert 3.0 < ratio < 5.0, ratio


# ------------------------------------------- NVT velocity rescaling (§2)
def _rot_axis_angle_form(q):
    """R(q) as (w^2 - |u|^2) 1 + 2 u u^T + 2 w [u]x, built independently of
    the oracle's element-wise matrix."""
    w, u = q[0], np.asarray(q[1:], dtype=np.float64)
    ux = np.array([[0.0, -u[2], u[1]], [u[2], 0.0, -u[0]], [-u[1], u[0], 0.0]])
    return (w * w - u @ u) * np.eye(3) + 2.0 * np.outer(u, u) + 2.0 * w * ux


def _half_step_temperature(model, v, q, j):
    """2 (K_trans + K_rot) / dof of the stored half-step state, with
    K_rot = sum_k b_k^2 / (2 I_k) over the non-zero principal moments
    (b = body-frame angular momentum)."""
    m = sum(s["mass"] for s in model["lj"])
    In = np.zeros((3, 3))
    for s in model["lj"]:
        p = np.asarray(s["pos"], dtype=np.float64)
        In += s["mass"] * ((p @ p) * np.eye(3) - np.outer(p, p))
    assert np.abs(In - np.diag(np.diag(In))).max() < 1e-12  # body frame = principal frame
    I = np.diag(In)
    live = I > 1e-12
    kt = 0.5 * m * (v * v).sum()
    kr = 0.0
    for qi, ji in zip(q, j):
        b = _rot_axis_angle_form(qi).T @ ji
        kr += 0.5 * (b[live] ** 2 / I[live]).sum()
    n = v.shape[0]
    dof = 3 * n - 3 + int(live.sum()) * n
    return 2.0 * (kt + kr) / dof


@pytest.mark.parametrize("which", ["2cljq", "4site"])
def test_velocity_rescaling_reaches_target(which):
    """After every thermostatted step the half-step kinetic temperature
    (translation + rotation, dof = 3N - 3 + N rot. dof) equals T_target."""
    if which == "2cljq":
        cfg = mdgen.config_2cljq(n=400, rho=0.3)
    else:
        cfg = mdgen.config_4site(n=300, rho=0.3)
    s = oracle.setup_from_config(cfg)
    st = {k: cfg[k] for k in ("r", "v", "q", "j")}
    T0 = _half_step_temperature(cfg["model"], st["v"], st["q"], st["j"])
    for T_target in (0.7, 1.6):
        cur = st
        for _ in range(3):
            cur = oracle.step(cfg["model"], s, cur, cfg["dt"], 1, T_target=T_target)
            T = _half_step_temperature(cfg["model"], cur["v"], cur["q"], cur["j"])
            assert T == pytest.approx(T_target, rel=1e-12), (T, T_target, T0)


def test_velocity_rescaling_is_one_common_factor_after_the_update():
    """One thermostatted step = the NVE step (same positions, orientations
    and new forces) with v and j of every molecule scaled by one factor."""
    cfg = mdgen.config_4site(n=300, rho=0.3)
    s = oracle.setup_from_config(cfg)
    st = {k: cfg[k] for k in ("r", "v", "q", "j")}
    a = oracle.step(cfg["model"], s, st, cfg["dt"], 1)
    b = oracle.step(cfg["model"], s, st, cfg["dt"], 1, T_target=2.5)
    assert np.array_equal(a["r"], b["r"]) and np.array_equal(a["q"], b["q"])
    assert np.array_equal(a["F"], b["F"]) and np.array_equal(a["tau"], b["tau"])
    ratio_v = b["v"] / a["v"]
    ratio_j = b["j"] / a["j"]
    beta = ratio_v.flat[0]
    assert beta > 1.0
    assert np.allclose(ratio_v, beta, rtol=1e-14, atol=0) and np.allclose(ratio_j, beta, rtol=1e-14, atol=0)
    T_nve = _half_step_temperature(cfg["model"], a["v"], a["q"], a["j"])
    assert beta == pytest.approx(math.sqrt(2.5 / T_nve), rel=1e-12)
