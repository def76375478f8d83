"""The oracle's pins catch plausible mistakes.  Each case below plants one
mistake in a copy of oracle/md_oracle.c (a dropped factor, a flipped sign,
a wrong index, a transposed operand, a wrong mixing rule, a missing half
step), compiles that copy, and runs every oracle pin (test_oracle_pins.py,
test_oracle_grad.py) against it in a child process: the pins must fail.
The unchanged source, compiled the same way, must pass them.  Mistakes are
planted on the CPU, in the oracle only."""
import os
import shutil
import subprocess
import sys
import tempfile
import concurrent.futures as cf

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")
PINS = [os.path.join(ROOT, "tests", "test_oracle_pins.py"), os.path.join(ROOT, "tests", "test_oracle_grad.py")]

# (name, exact text in md_oracle.c, planted replacement)
#
# One plausible mistake is left out because no pin catches it: forming the
# on-step angular momentum of the half-step orientation with the full step
# (j + dt tau instead of j + dt/2 tau).  It changes the midpoint estimate
# of the orientation at O(dt^2), so the scheme stays second order and keeps
# the exact free rotation (tau = 0); the pins bound the order of the
# rotational leapfrog, not its error constant.
MUTANTS = [
    ("lj_force_drops_factor_2",
     "double fr = 24.0 * eps * (2.0 * sr12 - sr6) / r2;",
     "double fr = 24.0 * eps * (sr12 - sr6) / r2;"),
    ("lj_shift_wrong_sign",
     "u -= 4.0 * eps * (sc12 - sc6);",
     "u += 4.0 * eps * (sc12 - sc6);"),
    ("lb_geometric_sigma",
     "*sig = m->eta[ta * T + tb] * 0.5 * (m->sigma[ta] + m->sigma[tb]);",
     "*sig = m->eta[ta * T + tb] * sqrt(m->sigma[ta] * m->sigma[tb]);"),
    ("lb_xi_dropped",
     "*eps = m->xi[ta * T + tb] * sqrt(m->eps[ta] * m->eps[tb]);",
     "*eps = sqrt(m->eps[ta] * m->eps[tb]);"),
    ("charge_dipole_sign",
     "*U = pb * u2;",
     "*U = -pb * u2;"),
    ("dipole_dipole_sign",
     "*U = (cab - 3.0 * pa * pb) * u3;",
     "*U = (cab + 3.0 * pa * pb) * u3;"),
    ("dipole_quadrupole_term",
     "*U = c * (-pa * (5.0 * pb * pb - 1.0) + 2.0 * pb * cab);",
     "*U = c * (-pa * (5.0 * pb * pb - 1.0) + 2.0 * pa * cab);"),
    ("quadrupole_quadrupole_coefficient",
     "double c = 0.75 * u5;",
     "double c = 1.5 * u5;"),
    ("quadrupole_quadrupole_cross_term",
     "double t = cab - 5.0 * pa * pb;",
     "double t = cab - 3.0 * pa * pb;"),
    ("reaction_field_factor",
     "return 2.0 * (eps_rf - 1.0) / (2.0 * eps_rf + 1.0);",
     "return (eps_rf - 1.0) / (2.0 * eps_rf + 1.0);"),
    ("reaction_field_sign",
     "U1 += -frf * cab;",
     "U1 += frf * cab;"),
    ("rf_self_energy_half_dropped",
     "out[2] = -0.5 * rf_factor(s->eps_rf) * (double)n * dot3(M, M) / rc3;",
     "out[2] = -rf_factor(s->eps_rf) * (double)n * dot3(M, M) / rc3;"),
    ("electrostatic_lever_torque_transposed",
     "cross3(gi->el[a], Fa, c);",
     "cross3(Fa, gi->el[a], c);"),
    ("orientation_torque_dropped",
     "cross3(ea, ga1, c);\n            for (int k = 0; k < 3; k++) o->ti[k] += sab * c[k];",
     "cross3(ea, ga1, c);\n            for (int k = 0; k < 3; k++) o->ti[k] += 0.0 * c[k];"),
    ("virial_with_site_separation",
     "double w = dot3(X, Fa);",
     "double w = dot3(x, Fa);"),
    ("min_image_floor",
     "X[k] = d - box[k] * rint(d / box[k]);",
     "X[k] = d - box[k] * floor(d / box[k]);"),
    ("stencil_missing_layer",
     "for (int dz = -1; dz <= 1; dz++)",
     "for (int dz = -1; dz <= 0; dz++)"),
    ("lrc_energy_coefficient",
     "U += 4.0 * eps * (s12 / (9.0 * rc9) - s6 / (3.0 * rc3));",
     "U += 4.0 * eps * (s12 / (9.0 * rc9) - s6 / (6.0 * rc3));"),
    ("rotation_matrix_sign",
     "R[1] = 2 * (x * y - w * z);",
     "R[1] = 2 * (x * y + w * z);"),
    ("quaternion_rate_sign",
     "qd[1] = 0.5 * (q[0] * w[0] + q[2] * w[2] - q[3] * w[1]);",
     "qd[1] = 0.5 * (q[0] * w[0] - q[2] * w[2] + q[3] * w[1]);"),
    ("kinetic_energy_without_half_step",
     "vt[k] = v[3 * i + k] + 0.5 * dt * F[3 * i + k] / mass;",
     "vt[k] = v[3 * i + k];"),
    ("velocity_rescaling_without_root",
     "const double beta = sqrt(T_target / T);",
     "const double beta = T_target / T;"),
    ("forces_subset_wrong_index",
     "forces_for_i(m, s, n, r, q, &C, sel[t], &F[3 * t], &tau[3 * t], &Sl, NULL, NULL, NULL, NULL);",
     "forces_for_i(m, s, n, r, q, &C, t, &F[3 * t], &tau[3 * t], &Sl, NULL, NULL, NULL, NULL);"),
    ("grad_eps_chain_rule",
     "double deps_t = eps * nt / (2.0 * m->eps[t]);\n                    double dsig_t = m->eta[ta * T + tb] * nt * 0.5;\n                    gU[t]",
     "double deps_t = eps * nt / m->eps[t];\n                    double dsig_t = m->eta[ta * T + tb] * nt * 0.5;\n                    gU[t]"),
    ("grad_strength_uses_own_strength",
     "gU[gi->pidx[a]] += gj->str[b] * U1;",
     "gU[gi->pidx[a]] += gi->str[a] * U1;"),
]


def build_mutant(before, after, workdir):
    """Compile md_oracle.c with `before` replaced by `after` (None: unchanged)
    into workdir/liboracle.so, the oracle package's own compiler flags."""
    src = open(os.path.join(ORACLE, "md_oracle.c")).read()
    if before is not None:
        assert src.count(before) == 1, f"planting site not unique or gone: {before!r}"
        src = src.replace(before, after)
    with open(os.path.join(workdir, "md_oracle.c"), "w") as f:
        f.write(src)
    shutil.copy(os.path.join(ORACLE, "md_oracle.h"), workdir)
    so = os.path.join(workdir, "liboracle.so")
    subprocess.run(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-o", so,
                    os.path.join(workdir, "md_oracle.c"), "-lm"], check=True, cwd=workdir)
    return so


def run_pins(so):
    """Every oracle pin against the library `so`, in a child process that
    stops at the first failure; (return code, output)."""
    env = dict(os.environ, MD_ORACLE_LIB=so, OMP_NUM_THREADS="2")
    p = subprocess.run([sys.executable, "-m", "pytest", *PINS, "-x", "-q", "-p", "no:cacheprovider"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return p.returncode, p.stdout + p.stderr


def _outcome(before, after):
    with tempfile.TemporaryDirectory(prefix="oracle_mutant_") as d:
        return run_pins(build_mutant(before, after, d))


@pytest.fixture(scope="module")
def outcomes():
    jobs = [("unchanged", None, None)] + MUTANTS
    workers = max(1, min(8, (os.cpu_count() or 2) // 2))
    with cf.ThreadPoolExecutor(workers) as ex:
        res = list(ex.map(lambda m: _outcome(m[1], m[2]), jobs))
    return {m[0]: r for m, r in zip(jobs, res)}


def test_unchanged_oracle_passes_its_pins(outcomes):
    rc, out = outcomes["unchanged"]
    assert rc == 0, out[-3000:]


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(outcomes, name):
    rc, out = outcomes[name]
    # return code 1: tests ran and at least one failed (not a collection or
    # usage error, which would be 2 or more)
    assert rc == 1, f"the pins did not catch '{name}' (rc {rc}):\n{out[-3000:]}"
