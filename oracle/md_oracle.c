/*
 * md_oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY; see
 * md_oracle.h).  Everything is double precision and written for a reader
 * who checks it against the paper by eye: no blocking, no fusion, no
 * reordering beyond the definitions cited per function.
 *
 * Conventions
 *   - quaternion q = (w, x, y, z), unit, rotates body-frame vectors into the
 *     space frame; R(q) is that rotation matrix.
 *   - For a molecule pair (i, j): X = R_i - R_j under the minimum image.
 *     The pair interacts iff |X|^2 < rc^2 (centre-of-mass cut-off).
 *   - For entities a (on i) and b (on j): x = r_a - r_b = X + d_a - d_b with
 *     d the space-frame offset of the entity from its molecule's centre.
 *   - Force on entity a:  F_a = -dU/dx; on b: -F_a.
 *   - Molecular virial W = sum_{i<j} X . F_ij with F_ij the force on i from j.
 */
#include "md_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- vectors */
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double *a, const double *b, double *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* Rotation matrix of a unit quaternion (w, x, y, z), body -> space. */
int orc_rotmat(const double *q, double *R)
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
    return 0;
}

static void matvec(const double *R, const double *v, double *o)
{
    o[0] = R[0] * v[0] + R[1] * v[1] + R[2] * v[2];
    o[1] = R[3] * v[0] + R[4] * v[1] + R[5] * v[2];
    o[2] = R[6] * v[0] + R[7] * v[1] + R[8] * v[2];
}

static void matTvec(const double *R, const double *v, double *o)
{
    o[0] = R[0] * v[0] + R[3] * v[1] + R[6] * v[2];
    o[1] = R[1] * v[0] + R[4] * v[1] + R[7] * v[2];
    o[2] = R[2] * v[0] + R[5] * v[1] + R[8] * v[2];
}

/* ----------------------------------------------------- molecule geometry */
/* Electrostatic entity kinds (§2: point charges, dipoles, quadrupoles). */
enum { K_CHG = 0, K_DIP = 1, K_QUAD = 2 };

typedef struct {
    int n_lj, n_el;
    double lj[ORC_MAXE][3];     /* space-frame offsets of LJ centres */
    int lj_type[ORC_MAXE];
    double el[3 * ORC_MAXE][3]; /* space-frame offsets of electrostatic entities */
    double ax[3 * ORC_MAXE][3]; /* space-frame axes (zero vector for charges) */
    double str[3 * ORC_MAXE];   /* strength q, mu or Q */
    int kind[3 * ORC_MAXE];
    int pidx[3 * ORC_MAXE];     /* parameter index of the strength */
} geom;

static void mol_geom(const orc_model *m, const double *q, geom *g)
{
    double R[9];
    orc_rotmat(q, R);
    g->n_lj = m->n_lj;
    for (int a = 0; a < m->n_lj; a++) {
        matvec(R, &m->lj_pos[3 * a], g->lj[a]);
        g->lj_type[a] = m->lj_type[a];
    }
    int k = 0, base = 2 * m->n_types;
    for (int a = 0; a < m->n_chg; a++, k++) {
        matvec(R, &m->chg_pos[3 * a], g->el[k]);
        g->ax[k][0] = g->ax[k][1] = g->ax[k][2] = 0.0;
        g->str[k] = m->chg_q[a];
        g->kind[k] = K_CHG;
        g->pidx[k] = base + a;
    }
    base += m->n_chg;
    for (int a = 0; a < m->n_dip; a++, k++) {
        matvec(R, &m->dip_pos[3 * a], g->el[k]);
        matvec(R, &m->dip_axis[3 * a], g->ax[k]);
        g->str[k] = m->dip_mu[a];
        g->kind[k] = K_DIP;
        g->pidx[k] = base + a;
    }
    base += m->n_dip;
    for (int a = 0; a < m->n_quad; a++, k++) {
        matvec(R, &m->quad_pos[3 * a], g->el[k]);
        matvec(R, &m->quad_axis[3 * a], g->ax[k]);
        g->str[k] = m->quad_Q[a];
        g->kind[k] = K_QUAD;
        g->pidx[k] = base + a;
    }
    g->n_el = k;
}

int orc_n_params(const orc_model *m) { return 2 * m->n_types + m->n_chg + m->n_dip + m->n_quad; }

/* ------------------------------------------------ LJ mixing (§2, Eq. 1) */
/* Lorentz-Berthelot: sigma_ab = eta_ab (sigma_a + sigma_b)/2,
 * eps_ab = xi_ab sqrt(eps_a eps_b). */
static void lj_mix(const orc_model *m, int ta, int tb, double *eps, double *sig)
{
    int T = m->n_types;
    *eps = m->xi[ta * T + tb] * sqrt(m->eps[ta] * m->eps[tb]);
    *sig = m->eta[ta * T + tb] * 0.5 * (m->sigma[ta] + m->sigma[tb]);
}

/* ------------------------------------------- multipole energies (§2) ---
 * Unit-strength interaction energy of entity kinds ka (at r_a) and kb (at
 * r_b) and its partial derivatives with respect to r = |x|,
 * pa = e_a . x/r, pb = e_b . x/r and cab = e_a . e_b, with x = r_a - r_b.
 * Each law is the energy of one point multipole in the electrostatic
 * potential of the other (k_C = 1); linear quadrupoles in the Buckingham
 * convention (Q = Theta_zz).  In terms of n = -x/r (from a to b) the laws
 * are the textbook forms:
 *   q-q   : 1/r
 *   q-mu  : -c_b / r^2           mu-q : +c_a / r^2
 *   mu-mu : (cab - 3 c_a c_b) / r^3
 *   q-Q   : (3 c_b^2 - 1) / (2 r^3)     Q-q : (3 c_a^2 - 1) / (2 r^3)
 *   mu-Q  : 3/(2 r^4) [c_a (5 c_b^2 - 1) - 2 c_b cab]
 *   Q-mu  : 3/(2 r^4) [-c_b (5 c_a^2 - 1) + 2 c_a cab]
 *   Q-Q   : 3/(4 r^5) [1 - 5c_a^2 - 5c_b^2 - 15 c_a^2 c_b^2 + 2 (cab - 5 c_a c_b)^2]
 * with c = -p.  The tests pin every law and sign against plain Coulomb sums
 * over explicit point-charge clusters. */
static void elec_law(int ka, int kb, double r, double pa, double pb, double cab, double *U, double *Ur,
                     double *Upa, double *Upb, double *Ucab)
{
    double u = 1.0 / r, u2 = u * u, u3 = u2 * u, u4 = u3 * u, u5 = u4 * u;
    *U = *Ur = *Upa = *Upb = *Ucab = 0.0;
    if (ka == K_CHG && kb == K_CHG) {
        *U = u;
        *Ur = -u2;
    } else if (ka == K_CHG && kb == K_DIP) {
        *U = pb * u2;
        *Ur = -2.0 * pb * u3;
        *Upb = u2;
    } else if (ka == K_DIP && kb == K_CHG) {
        *U = -pa * u2;
        *Ur = 2.0 * pa * u3;
        *Upa = -u2;
    } else if (ka == K_DIP && kb == K_DIP) {
        *U = (cab - 3.0 * pa * pb) * u3;
        *Ur = -3.0 * (*U) * u;
        *Upa = -3.0 * pb * u3;
        *Upb = -3.0 * pa * u3;
        *Ucab = u3;
    } else if (ka == K_CHG && kb == K_QUAD) {
        *U = 0.5 * (3.0 * pb * pb - 1.0) * u3;
        *Ur = -3.0 * (*U) * u;
        *Upb = 3.0 * pb * u3;
    } else if (ka == K_QUAD && kb == K_CHG) {
        *U = 0.5 * (3.0 * pa * pa - 1.0) * u3;
        *Ur = -3.0 * (*U) * u;
        *Upa = 3.0 * pa * u3;
    } else if (ka == K_DIP && kb == K_QUAD) {
        double c = 1.5 * u4;
        *U = c * (-pa * (5.0 * pb * pb - 1.0) + 2.0 * pb * cab);
        *Ur = -4.0 * (*U) * u;
        *Upa = c * (-(5.0 * pb * pb - 1.0));
        *Upb = c * (-10.0 * pa * pb + 2.0 * cab);
        *Ucab = c * 2.0 * pb;
    } else if (ka == K_QUAD && kb == K_DIP) {
        double c = 1.5 * u4;
        *U = c * (pb * (5.0 * pa * pa - 1.0) - 2.0 * pa * cab);
        *Ur = -4.0 * (*U) * u;
        *Upb = c * (5.0 * pa * pa - 1.0);
        *Upa = c * (10.0 * pa * pb - 2.0 * cab);
        *Ucab = -c * 2.0 * pa;
    } else { /* Q-Q */
        double c = 0.75 * u5;
        double t = cab - 5.0 * pa * pb;
        double B = 1.0 - 5.0 * pa * pa - 5.0 * pb * pb - 15.0 * pa * pa * pb * pb + 2.0 * t * t;
        *U = c * B;
        *Ur = -5.0 * (*U) * u;
        *Upa = c * (-10.0 * pa - 30.0 * pa * pb * pb - 20.0 * pb * t);
        *Upb = c * (-10.0 * pb - 30.0 * pa * pa * pb - 20.0 * pa * t);
        *Ucab = c * 4.0 * t;
    }
}

/* Reaction-field factor 2(eps_RF - 1)/(2 eps_RF + 1) (§1, §3: reaction field
 * for dipolar molecules); 1 in the conducting limit eps_RF -> infinity. */
static double rf_factor(double eps_rf)
{
    if (isinf(eps_rf)) return 1.0;
    return 2.0 * (eps_rf - 1.0) / (2.0 * eps_rf + 1.0);
}

/* ------------------------------------------------ one molecule pair -----
 * Adds the interaction of molecule i (geometry gi) with molecule j (gj) at
 * centre-of-mass separation X = R_i - R_j (already known to be inside the
 * cut-off).  Outputs: force on i (Fi; force on j is -Fi), torques on i and
 * j, energy, virial X.F_ij and its diagonal.  If gU/gW are non-NULL the
 * derivatives of energy and virial with respect to the parameters are
 * added to them. */
typedef struct {
    double U, W, Wd[3];
    double Fi[3], ti[3], tj[3];
    long nsite;
} pair_acc;

static void pair_mol(const orc_model *m, const orc_setup *s, const double *X, const geom *gi, const geom *gj,
                     pair_acc *o, double *gU, double *gW)
{
    const int T = m->n_types;
    double rc = s->rc;
    /* --- Lennard-Jones centres (Eq. 1, LJTS, Lorentz-Berthelot) --- */
    for (int a = 0; a < gi->n_lj; a++) {
        for (int b = 0; b < gj->n_lj; b++) {
            int ta = gi->lj_type[a], tb = gj->lj_type[b];
            double eps, sig;
            lj_mix(m, ta, tb, &eps, &sig);
            double x[3];
            for (int k = 0; k < 3; k++) x[k] = X[k] + gi->lj[a][k] - gj->lj[b][k];
            double r2 = dot3(x, x);
            double sr2 = sig * sig / r2, sr6 = sr2 * sr2 * sr2, sr12 = sr6 * sr6;
            double u = 4.0 * eps * (sr12 - sr6);
            double dsig_u = 4.0 * eps / sig * (12.0 * sr12 - 6.0 * sr6);
            if (s->lj_shift) {
                double sc2 = sig * sig / (rc * rc), sc6 = sc2 * sc2 * sc2, sc12 = sc6 * sc6;
                u -= 4.0 * eps * (sc12 - sc6);
                dsig_u -= 4.0 * eps / sig * (12.0 * sc12 - 6.0 * sc6);
            }
            double fr = 24.0 * eps * (2.0 * sr12 - sr6) / r2; /* F_a = fr * x */
            double Fa[3] = {fr * x[0], fr * x[1], fr * x[2]};
            double w = dot3(X, Fa);
            o->U += u;
            o->W += w;
            for (int k = 0; k < 3; k++) {
                o->Wd[k] += X[k] * Fa[k];
                o->Fi[k] += Fa[k];
            }
            double c[3], mFa[3] = {-Fa[0], -Fa[1], -Fa[2]};
            cross3(gi->lj[a], Fa, c);
            for (int k = 0; k < 3; k++) o->ti[k] += c[k];
            cross3(gj->lj[b], mFa, c);
            for (int k = 0; k < 3; k++) o->tj[k] += c[k];
            o->nsite++;
            if (gU) {
                /* d/d eps_ab and d/d sigma_ab of u and w, then chain rule to
                 * the per-type parameters through the mixing rules. */
                double du_deps = u / eps, dw_deps = w / eps;
                double dfr_dsig = 24.0 * eps * (24.0 * sr12 - 6.0 * sr6) / (sig * r2);
                double dw_dsig = dfr_dsig * dot3(X, x);
                for (int t = 0; t < T; t++) {
                    double nt = (double)((ta == t) + (tb == t));
                    if (nt == 0.0) continue;
                    double deps_t = eps * nt / (2.0 * m->eps[t]);
                    double dsig_t = m->eta[ta * T + tb] * nt * 0.5;
                    gU[t] += du_deps * deps_t;
                    gW[t] += dw_deps * deps_t;
                    gU[T + t] += dsig_u * dsig_t;
                    gW[T + t] += dw_dsig * dsig_t;
                }
            }
        }
    }
    /* --- electrostatic entities (§2 multipole expansion) + reaction field --- */
    double frf = rf_factor(s->eps_rf) / (rc * rc * rc);
    for (int a = 0; a < gi->n_el; a++) {
        for (int b = 0; b < gj->n_el; b++) {
            double x[3];
            for (int k = 0; k < 3; k++) x[k] = X[k] + gi->el[a][k] - gj->el[b][k];
            double r = sqrt(dot3(x, x));
            double xh[3] = {x[0] / r, x[1] / r, x[2] / r};
            const double *ea = gi->ax[a], *eb = gj->ax[b];
            double pa = dot3(ea, xh), pb = dot3(eb, xh), cab = dot3(ea, eb);
            double U1, Ur, Upa, Upb, Ucab;
            elec_law(gi->kind[a], gj->kind[b], r, pa, pb, cab, &U1, &Ur, &Upa, &Upb, &Ucab);
            if (gi->kind[a] == K_DIP && gj->kind[b] == K_DIP) {
                /* reaction field (Barker-Watts): -f mu_a mu_b (e_a.e_b) / rc^3 */
                U1 += -frf * cab;
                Ucab += -frf;
            }
            double sab = gi->str[a] * gj->str[b];
            double dUdx1[3], Fa1[3];
            for (int k = 0; k < 3; k++) {
                dUdx1[k] = Ur * xh[k] + Upa * (ea[k] - pa * xh[k]) / r + Upb * (eb[k] - pb * xh[k]) / r;
                Fa1[k] = -dUdx1[k];
            }
            double ga1[3], gb1[3];
            for (int k = 0; k < 3; k++) {
                ga1[k] = -(Upa * xh[k] + Ucab * eb[k]);
                gb1[k] = -(Upb * xh[k] + Ucab * ea[k]);
            }
            double w1 = dot3(X, Fa1);
            o->U += sab * U1;
            o->W += sab * w1;
            double Fa[3], mFa[3], c[3];
            for (int k = 0; k < 3; k++) {
                Fa[k] = sab * Fa1[k];
                mFa[k] = -Fa[k];
                o->Wd[k] += X[k] * Fa[k];
                o->Fi[k] += Fa[k];
            }
            cross3(gi->el[a], Fa, c);
            for (int k = 0; k < 3; k++) o->ti[k] += c[k];
            cross3(ea, ga1, c);
            for (int k = 0; k < 3; k++) o->ti[k] += sab * c[k];
            cross3(gj->el[b], mFa, c);
            for (int k = 0; k < 3; k++) o->tj[k] += c[k];
            cross3(eb, gb1, c);
            for (int k = 0; k < 3; k++) o->tj[k] += sab * c[k];
            o->nsite++;
            if (gU) {
                /* energy and virial are bilinear in the two strengths */
                gU[gi->pidx[a]] += gj->str[b] * U1;
                gW[gi->pidx[a]] += gj->str[b] * w1;
                gU[gj->pidx[b]] += gi->str[a] * U1;
                gW[gj->pidx[b]] += gi->str[a] * w1;
            }
        }
    }
}

/* Minimum image (§3, periodic boundary conditions). */
static void min_image(const double *box, const double *ri, const double *rj, double *X)
{
    for (int k = 0; k < 3; k++) {
        double d = ri[k] - rj[k];
        X[k] = d - box[k] * rint(d / box[k]);
    }
}

static int check_setup(const orc_model *m, const orc_setup *s)
{
    if (!(s->rc > 0.0)) return -1;
    for (int k = 0; k < 3; k++)
        if (!(s->box[k] >= 2.0 * s->rc)) return -2;
    if (m->n_types < 0 || m->n_types > ORC_MAXT) return -1;
    if (m->n_lj > ORC_MAXE || m->n_chg > ORC_MAXE || m->n_dip > ORC_MAXE || m->n_quad > ORC_MAXE) return -1;
    return 0;
}

/* ---------------------------------------------------- linked cells (§3) ---
 * Cells of edge >= rc: n_c = floor(L / rc) per axis.  For molecule i the
 * candidate partners are the molecules of the distinct cells among the 27
 * cells around its own (fewer when an axis has < 3 cells); each pair is
 * then tested with the minimum image.  A CSR list (cell_start, order) is
 * built by counting sort. */
typedef struct {
    int nc[3];
    int64_t ncell;
    int64_t *start, *order;
    int *cell;
} cells_t;

static int64_t cell_of(const double *box, const int *nc, const double *r)
{
    int c[3];
    for (int k = 0; k < 3; k++) {
        double x = r[k] - box[k] * floor(r[k] / box[k]);
        int ck = (int)floor(x / (box[k] / nc[k]));
        if (ck < 0) ck = 0;
        if (ck >= nc[k]) ck = nc[k] - 1;
        c[k] = ck;
    }
    return ((int64_t)c[2] * nc[1] + c[1]) * nc[0] + c[0];
}

static int cells_build(const orc_setup *s, int64_t n, const double *r, cells_t *C)
{
    for (int k = 0; k < 3; k++) {
        C->nc[k] = (int)floor(s->box[k] / s->rc);
        if (C->nc[k] < 1) C->nc[k] = 1;
    }
    C->ncell = (int64_t)C->nc[0] * C->nc[1] * C->nc[2];
    C->start = (int64_t *)calloc((size_t)C->ncell + 1, sizeof(int64_t));
    C->order = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    C->cell = (int *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int));
    if (!C->start || !C->order || !C->cell) return -5;
    int64_t *cnt = (int64_t *)calloc((size_t)C->ncell, sizeof(int64_t));
    if (!cnt) return -5;
    for (int64_t i = 0; i < n; i++) {
        int64_t c = cell_of(s->box, C->nc, &r[3 * i]);
        C->cell[i] = (int)c;
        cnt[c]++;
    }
    for (int64_t c = 0; c < C->ncell; c++) C->start[c + 1] = C->start[c] + cnt[c];
    memset(cnt, 0, (size_t)C->ncell * sizeof(int64_t));
    for (int64_t i = 0; i < n; i++) {
        int64_t c = C->cell[i];
        C->order[C->start[c] + cnt[c]++] = i;
    }
    free(cnt);
    return 0;
}

static void cells_free(cells_t *C)
{
    free(C->start);
    free(C->order);
    free(C->cell);
}

/* distinct neighbour cells of cell c (including c itself) */
static int neighbour_cells(const cells_t *C, int64_t c, int64_t *out)
{
    int cx = (int)(c % C->nc[0]), cy = (int)((c / C->nc[0]) % C->nc[1]), cz = (int)(c / ((int64_t)C->nc[0] * C->nc[1]));
    int cnt = 0;
    for (int dz = -1; dz <= 1; dz++)
        for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
                int x = ((cx + dx) % C->nc[0] + C->nc[0]) % C->nc[0];
                int y = ((cy + dy) % C->nc[1] + C->nc[1]) % C->nc[1];
                int z = ((cz + dz) % C->nc[2] + C->nc[2]) % C->nc[2];
                int64_t nb = ((int64_t)z * C->nc[1] + y) * C->nc[0] + x;
                int dup = 0;
                for (int t = 0; t < cnt; t++)
                    if (out[t] == nb) dup = 1;
                if (!dup) out[cnt++] = nb;
            }
    return cnt;
}

/* ------------------------------------------------ forces (§3 "summation") */
typedef struct {
    double U, W, Wd[3];
    double nmol, nsite, nexam;
    double absU, absW; /* sums of |u_ij| and |w_ij| over molecule pairs (error scales) */
} sums_t;

/* Full pass over molecule i's partners (each ordered pair visited from both
 * sides); i-side force and torque, half the pair energy and virial. */
static void forces_for_i(const orc_model *m, const orc_setup *s, int64_t n, const double *r, const double *q,
                         const cells_t *C, int64_t i, double *Fi, double *ti, sums_t *S, double *gU, double *gW,
                         double *aU, double *aW)
{
    geom gi, gj;
    mol_geom(m, &q[4 * i], &gi);
    double rc2 = s->rc * s->rc;
    Fi[0] = Fi[1] = Fi[2] = ti[0] = ti[1] = ti[2] = 0.0;
    int64_t nb[27];
    int nnb = 0;
    if (C) nnb = neighbour_cells(C, C->cell[i], nb);
    int64_t cursor_cell = 0;
    int64_t jbeg = 0, jend = C ? 0 : n, jj = 0;
    for (;;) {
        if (C) {
            if (jj >= jend) {
                if (cursor_cell >= nnb) break;
                jbeg = C->start[nb[cursor_cell]];
                jend = C->start[nb[cursor_cell] + 1];
                cursor_cell++;
                jj = jbeg;
                continue;
            }
        } else if (jj >= jend) {
            break;
        }
        int64_t j = C ? C->order[jj] : jj;
        jj++;
        if (j == i) continue;
        double X[3];
        min_image(s->box, &r[3 * i], &r[3 * j], X);
        S->nexam += 0.5;
        if (dot3(X, X) >= rc2) continue;
        mol_geom(m, &q[4 * j], &gj);
        pair_acc o;
        memset(&o, 0, sizeof o);
        double lgU[64], lgW[64];
        int P = orc_n_params(m);
        if (gU) {
            memset(lgU, 0, sizeof lgU);
            memset(lgW, 0, sizeof lgW);
        }
        pair_mol(m, s, X, &gi, &gj, &o, gU ? lgU : NULL, gU ? lgW : NULL);
        for (int k = 0; k < 3; k++) {
            Fi[k] += o.Fi[k];
            ti[k] += o.ti[k];
            S->Wd[k] += 0.5 * o.Wd[k];
        }
        S->U += 0.5 * o.U;
        S->W += 0.5 * o.W;
        S->absU += 0.5 * fabs(o.U);
        S->absW += 0.5 * fabs(o.W);
        S->nmol += 0.5;
        S->nsite += 0.5 * (double)o.nsite;
        if (gU)
            for (int p = 0; p < P; p++) {
                gU[p] += 0.5 * lgU[p];
                gW[p] += 0.5 * lgW[p];
                aU[p] += 0.5 * fabs(lgU[p]);
                aW[p] += 0.5 * fabs(lgW[p]);
            }
    }
}

static int forces_impl(const orc_model *m, const orc_setup *s, int64_t n, const double *r, const double *q,
                       int use_cells, int n_threads, double *F, double *tau, double *obs, double *gU, double *gW,
                       double *aU, double *aW)
{
    int rcode = check_setup(m, s);
    if (rcode) return rcode;
    int P = orc_n_params(m);
    if (P > 64) return -1;
    cells_t C;
    memset(&C, 0, sizeof C);
    if (use_cells) {
        rcode = cells_build(s, n, r, &C);
        if (rcode) return rcode;
    }
    sums_t S;
    memset(&S, 0, sizeof S);
    if (gU) {
        memset(gU, 0, (size_t)P * sizeof(double));
        memset(gW, 0, (size_t)P * sizeof(double));
        memset(aU, 0, (size_t)P * sizeof(double));
        memset(aW, 0, (size_t)P * sizeof(double));
    }
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
    if (use_cells) {
#pragma omp parallel
        {
            sums_t Sl;
            memset(&Sl, 0, sizeof Sl);
            double lgU[64], lgW[64], laU[64], laW[64];
            memset(lgU, 0, sizeof lgU);
            memset(lgW, 0, sizeof lgW);
            memset(laU, 0, sizeof laU);
            memset(laW, 0, sizeof laW);
#pragma omp for schedule(dynamic, 64)
            for (int64_t i = 0; i < n; i++)
                forces_for_i(m, s, n, r, q, &C, i, &F[3 * i], &tau[3 * i], &Sl, gU ? lgU : NULL, gU ? lgW : NULL,
                             laU, laW);
#pragma omp critical
            {
                S.U += Sl.U;
                S.W += Sl.W;
                for (int k = 0; k < 3; k++) S.Wd[k] += Sl.Wd[k];
                S.nmol += Sl.nmol;
                S.nsite += Sl.nsite;
                S.nexam += Sl.nexam;
                S.absU += Sl.absU;
                S.absW += Sl.absW;
                if (gU)
                    for (int p = 0; p < P; p++) {
                        gU[p] += lgU[p];
                        gW[p] += lgW[p];
                        aU[p] += laU[p];
                        aW[p] += laW[p];
                    }
            }
        }
        cells_free(&C);
    } else {
        /* brute force over all unordered pairs i < j (definition) */
        memset(F, 0, (size_t)n * 3 * sizeof(double));
        memset(tau, 0, (size_t)n * 3 * sizeof(double));
        double rc2 = s->rc * s->rc;
        geom gi, gj;
        for (int64_t i = 0; i < n; i++) {
            mol_geom(m, &q[4 * i], &gi);
            for (int64_t j = i + 1; j < n; j++) {
                double X[3];
                min_image(s->box, &r[3 * i], &r[3 * j], X);
                S.nexam += 1.0;
                if (dot3(X, X) >= rc2) continue;
                mol_geom(m, &q[4 * j], &gj);
                pair_acc o;
                memset(&o, 0, sizeof o);
                double pgU[64], pgW[64];
                if (gU) {
                    memset(pgU, 0, sizeof pgU);
                    memset(pgW, 0, sizeof pgW);
                }
                pair_mol(m, s, X, &gi, &gj, &o, gU ? pgU : NULL, gU ? pgW : NULL);
                if (gU)
                    for (int p = 0; p < P; p++) {
                        gU[p] += pgU[p];
                        gW[p] += pgW[p];
                        aU[p] += fabs(pgU[p]);
                        aW[p] += fabs(pgW[p]);
                    }
                for (int k = 0; k < 3; k++) {
                    F[3 * i + k] += o.Fi[k];
                    F[3 * j + k] -= o.Fi[k];
                    tau[3 * i + k] += o.ti[k];
                    tau[3 * j + k] += o.tj[k];
                    S.Wd[k] += o.Wd[k];
                }
                S.U += o.U;
                S.W += o.W;
                S.absU += fabs(o.U);
                S.absW += fabs(o.W);
                S.nmol += 1.0;
                S.nsite += (double)o.nsite;
            }
        }
    }
    if (obs) {
        memset(obs, 0, ORC_NOBS * sizeof(double));
        obs[ORC_U] = S.U;
        obs[ORC_W] = S.W;
        obs[ORC_WXX] = S.Wd[0];
        obs[ORC_WYY] = S.Wd[1];
        obs[ORC_WZZ] = S.Wd[2];
        obs[ORC_NMOL] = S.nmol;
        obs[ORC_NSITE] = S.nsite;
        obs[ORC_NEXAM] = S.nexam;
        double lrc[3];
        orc_lrc(m, s, n, lrc);
        obs[ORC_ULRC] = lrc[0];
        obs[ORC_WLRC] = lrc[1];
        obs[ORC_URFSELF] = lrc[2];
        obs[ORC_ABSU] = S.absU;
        obs[ORC_ABSW] = S.absW;
    }
    return 0;
}

int orc_forces(const orc_model *m, const orc_setup *s, int64_t n, const double *r, const double *q, int use_cells,
               int n_threads, double *F, double *tau, double *obs)
{
    return forces_impl(m, s, n, r, q, use_cells, n_threads, F, tau, obs, NULL, NULL, NULL, NULL);
}

/* Exact force and torque on selected molecules only (linked cells), for
 * sampled checks of systems too large for a full oracle evaluation. */
int orc_forces_subset(const orc_model *m, const orc_setup *s, int64_t n, const double *r, const double *q,
                      int64_t n_sel, const int64_t *sel, int n_threads, double *F, double *tau)
{
    int rcode = check_setup(m, s);
    if (rcode) return rcode;
    cells_t C;
    memset(&C, 0, sizeof C);
    rcode = cells_build(s, n, r, &C);
    if (rcode) return rcode;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < n_sel; t++) {
        sums_t Sl;
        memset(&Sl, 0, sizeof Sl);
        forces_for_i(m, s, n, r, q, &C, sel[t], &F[3 * t], &tau[3 * t], &Sl, NULL, NULL, NULL, NULL);
    }
    cells_free(&C);
    return 0;
}

/* -------------------------------------------- long-range correction (§3)
 * Isotropic mean-field tail of the LJ interaction beyond rc for every pair
 * of LJ centres (g(r) = 1 beyond the cut-off):
 *   U_LRC = (2 pi N^2 / V) sum_ab 4 eps_ab [sig^12/(9 rc^9) - sig^6/(3 rc^3)]
 *   W_LRC = (2 pi N^2 / V) sum_ab 4 eps_ab [4 sig^12/(3 rc^9) - 2 sig^6/rc^3]
 * (W_LRC is the tail of -sum r u'(r), so P_LRC = W_LRC / (3V)).
 * out[2] = reaction-field self energy -1/2 f N |M|^2 / rc^3 with M the
 * molecule's total point-dipole moment (reported, not part of U). */
int orc_lrc(const orc_model *m, const orc_setup *s, int64_t n, double *out)
{
    double V = s->box[0] * s->box[1] * s->box[2];
    double rc = s->rc, rc3 = rc * rc * rc, rc9 = rc3 * rc3 * rc3;
    double pre = 2.0 * M_PI * (double)n * (double)n / V;
    double U = 0.0, W = 0.0;
    if (s->lj_lrc) {
        for (int a = 0; a < m->n_lj; a++)
            for (int b = 0; b < m->n_lj; b++) {
                double eps, sig;
                lj_mix(m, m->lj_type[a], m->lj_type[b], &eps, &sig);
                double s6 = pow(sig, 6.0), s12 = s6 * s6;
                U += 4.0 * eps * (s12 / (9.0 * rc9) - s6 / (3.0 * rc3));
                W += 4.0 * eps * (4.0 * s12 / (3.0 * rc9) - 2.0 * s6 / rc3);
            }
    }
    out[0] = pre * U;
    out[1] = pre * W;
    double M[3] = {0, 0, 0};
    for (int a = 0; a < m->n_dip; a++)
        for (int k = 0; k < 3; k++) M[k] += m->dip_mu[a] * m->dip_axis[3 * a + k];
    out[2] = -0.5 * rf_factor(s->eps_rf) * (double)n * dot3(M, M) / rc3;
    return 0;
}

/* ------------------------------------------- rigid-body properties ----- */
static void model_inertia(const orc_model *m, double *mass, double *Iinv, double *I)
{
    double M = 0.0, In[9] = {0};
    for (int a = 0; a < m->n_lj; a++) {
        const double *p = &m->lj_pos[3 * a];
        double mm = m->lj_mass[a];
        M += mm;
        double p2 = dot3(p, p);
        for (int r = 0; r < 3; r++)
            for (int c = 0; c < 3; c++) In[3 * r + c] += mm * ((r == c ? p2 : 0.0) - p[r] * p[c]);
    }
    *mass = M;
    for (int k = 0; k < 3; k++) {
        I[k] = In[4 * k];
        Iinv[k] = In[4 * k] > 1e-12 ? 1.0 / In[4 * k] : 0.0;
    }
}

/* q_dot = 1/2 q (x) (0, w_body) */
static void quat_rate(const double *q, const double *w, double *qd)
{
    qd[0] = 0.5 * (-q[1] * w[0] - q[2] * w[1] - q[3] * w[2]);
    qd[1] = 0.5 * (q[0] * w[0] + q[2] * w[2] - q[3] * w[1]);
    qd[2] = 0.5 * (q[0] * w[1] + q[3] * w[0] - q[1] * w[2]);
    qd[3] = 0.5 * (q[0] * w[2] + q[1] * w[1] - q[2] * w[0]);
}

/* body-frame angular velocity from space-frame angular momentum */
static void omega_body(const double *q, const double *jsp, const double *Iinv, double *w)
{
    double R[9], jb[3];
    orc_rotmat(q, R);
    matTvec(R, jsp, jb);
    for (int k = 0; k < 3; k++) w[k] = Iinv[k] * jb[k];
}

static void normalise4(double *q)
{
    double s = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int k = 0; k < 4; k++) q[k] /= s;
}

/* ----------------------------------------------------- leapfrog (§3) ----
 * Translational leapfrog (Eqs. 2-3):
 *   v(t + dt/2) = v(t - dt/2) + dt F(t)/m;  r(t + dt) = r(t) + dt v(t + dt/2)
 * Rotational leapfrog (Eqs. 4-5), read as Fincham's quaternion leapfrog:
 *   j(t)        = j(t - dt/2) + dt/2 tau(t)
 *   q(t + dt/2) = q(t) + dt/2 q_dot(q(t), j(t)), renormalised
 *   j(t + dt/2) = j(t - dt/2) + dt tau(t)
 *   q(t + dt)   = q(t) + dt q_dot(q(t + dt/2), j(t + dt/2)), renormalised
 * where q_dot(q, j) = 1/2 q (x) (0, I^-1 A(q) j), A = R(q)^T; j is the
 * space-frame angular momentum.  Positions are wrapped into [0, L).  Forces
 * and torques at the new configuration are then recomputed. */
int orc_step(const orc_model *m, const orc_setup *s, int64_t n, double dt, int n_steps, int use_cells, int n_threads,
             double *r, double *v, double *q, double *j, double *F, double *tau, double *obs)
{
    return orc_step_T(m, s, n, dt, n_steps, 0.0, use_cells, n_threads, r, v, q, j, F, tau, obs);
}

/* Canonical ensemble by velocity rescaling (§2, ensembles paragraph: the
 * temperature of NVT runs is kept constant by rescaling the velocities).
 * Reading taken: after the leapfrog update of every molecule, the kinetic
 * temperature of the half-step state,
 *   T_half = 2 (K_trans + K_rot) / dof,  dof = 3N - 3 + N * (rotational dof),
 *   K_trans = sum 1/2 m v(t+dt/2)^2,
 *   K_rot   = sum 1/2 w.I w,  w = I^-1 A(q(t+dt)) j(t+dt/2),
 * is brought to T_target by scaling v and j of every molecule by the one
 * factor sqrt(T_target / T_half); positions and orientations of the step
 * are not changed.  T_target <= 0 (or T_half = 0) leaves the state as is. */
static void rescale_to(const orc_model *m, int64_t n, double T_target, double *v, const double *q, double *j)
{
    double mass, Iinv[3], I[3];
    model_inertia(m, &mass, Iinv, I);
    const int rot = (I[0] > 1e-12) + (I[1] > 1e-12) + (I[2] > 1e-12);
    const double dof = 3.0 * (double)n - 3.0 + (double)rot * (double)n;
    double kt = 0.0, kr = 0.0;
    for (int64_t i = 0; i < n; i++) {
        double w[3];
        kt += 0.5 * mass * dot3(&v[3 * i], &v[3 * i]);
        omega_body(&q[4 * i], &j[3 * i], Iinv, w);
        for (int k = 0; k < 3; k++) kr += 0.5 * I[k] * w[k] * w[k];
    }
    if (!(dof > 0.0)) return;
    const double T = 2.0 * (kt + kr) / dof;
    if (!(T > 0.0)) return;
    const double beta = sqrt(T_target / T);
    for (int64_t i = 0; i < 3 * n; i++) {
        v[i] *= beta;
        j[i] *= beta;
    }
}

int orc_step_T(const orc_model *m, const orc_setup *s, int64_t n, double dt, int n_steps, double T_target,
               int use_cells, int n_threads, double *r, double *v, double *q, double *j, double *F, double *tau,
               double *obs)
{
    double mass, Iinv[3], I[3];
    model_inertia(m, &mass, Iinv, I);
    for (int st = 0; st < n_steps; st++) {
        for (int64_t i = 0; i < n; i++) {
            double *ri = &r[3 * i], *vi = &v[3 * i], *qi = &q[4 * i], *ji = &j[3 * i];
            for (int k = 0; k < 3; k++) {
                vi[k] += dt * F[3 * i + k] / mass;
                ri[k] += dt * vi[k];
                ri[k] -= s->box[k] * floor(ri[k] / s->box[k]);
                if (ri[k] >= s->box[k]) ri[k] -= s->box[k];
            }
            double jt[3], w[3], qd[4], qh[4];
            for (int k = 0; k < 3; k++) jt[k] = ji[k] + 0.5 * dt * tau[3 * i + k];
            omega_body(qi, jt, Iinv, w);
            quat_rate(qi, w, qd);
            for (int k = 0; k < 4; k++) qh[k] = qi[k] + 0.5 * dt * qd[k];
            normalise4(qh);
            for (int k = 0; k < 3; k++) ji[k] += dt * tau[3 * i + k];
            omega_body(qh, ji, Iinv, w);
            quat_rate(qh, w, qd);
            for (int k = 0; k < 4; k++) qi[k] += dt * qd[k];
            normalise4(qi);
        }
        if (T_target > 0.0) rescale_to(m, n, T_target, v, q, j);
        int rcode = forces_impl(m, s, n, r, q, use_cells, n_threads, F, tau, obs, NULL, NULL, NULL, NULL);
        if (rcode) return rcode;
    }
    return 0;
}

/* Kinetic energies at time t from the half-step state (v, j at t - dt/2)
 * and F, tau at t:  v(t) = v(t-dt/2) + dt/2 F/m,  j(t) = j(t-dt/2) + dt/2 tau.
 * K[0] = sum 1/2 m v(t)^2, K[1] = sum 1/2 w_b . I w_b with w_b = I^-1 A j(t). */
int orc_kinetic(const orc_model *m, int64_t n, double dt, const double *v, const double *q, const double *j,
                const double *F, const double *tau, double *K)
{
    double mass, Iinv[3], I[3];
    model_inertia(m, &mass, Iinv, I);
    double kt = 0.0, kr = 0.0;
    for (int64_t i = 0; i < n; i++) {
        double vt[3], jt[3], w[3];
        for (int k = 0; k < 3; k++) {
            vt[k] = v[3 * i + k] + 0.5 * dt * F[3 * i + k] / mass;
            jt[k] = j[3 * i + k] + 0.5 * dt * tau[3 * i + k];
        }
        kt += 0.5 * mass * dot3(vt, vt);
        omega_body(&q[4 * i], jt, Iinv, w);
        for (int k = 0; k < 3; k++) kr += 0.5 * I[k] * w[k] * w[k];
    }
    K[0] = kt;
    K[1] = kr;
    return 0;
}

/* ----------------------------------------- parameter derivatives -------
 * d<U>/d theta and d<W>/d theta averaged over n_cfg fixed configurations,
 * theta = (eps_t for each LJ type, sigma_t for each LJ type, each charge q,
 * each dipole mu, each quadrupole Q).  U and W include the long-range
 * correction when it is enabled.  means[0] = <U>, means[1] = <W>.
 * absU/absW: mean over configurations of sum over molecule pairs of
 * |d u_ij / d theta| and |d w_ij / d theta| (the error scale of a sum). */
int orc_param_grad(const orc_model *m, const orc_setup *s, int n_cfg, int64_t n, const double *r_all,
                   const double *q_all, int use_cells, int n_threads, double *dU, double *dW, double *means,
                   double *absU, double *absW)
{
    int P = orc_n_params(m);
    if (P > 64) return -1;
    int T = m->n_types;
    double *F = (double *)malloc((size_t)(n > 0 ? n : 1) * 3 * sizeof(double));
    double *tau = (double *)malloc((size_t)(n > 0 ? n : 1) * 3 * sizeof(double));
    if (!F || !tau) return -5;
    double gU[64], gW[64], aU[64], aW[64], obs[ORC_NOBS];
    memset(dU, 0, (size_t)P * sizeof(double));
    memset(dW, 0, (size_t)P * sizeof(double));
    memset(absU, 0, (size_t)P * sizeof(double));
    memset(absW, 0, (size_t)P * sizeof(double));
    means[0] = means[1] = 0.0;
    for (int c = 0; c < n_cfg; c++) {
        int rcode = forces_impl(m, s, n, &r_all[(size_t)c * n * 3], &q_all[(size_t)c * n * 4], use_cells, n_threads,
                                F, tau, obs, gU, gW, aU, aW);
        if (rcode) {
            free(F);
            free(tau);
            return rcode;
        }
        for (int p = 0; p < P; p++) {
            dU[p] += gU[p] / n_cfg;
            dW[p] += gW[p] / n_cfg;
            absU[p] += aU[p] / n_cfg;
            absW[p] += aW[p] / n_cfg;
        }
        means[0] += (obs[ORC_U] + obs[ORC_ULRC]) / n_cfg;
        means[1] += (obs[ORC_W] + obs[ORC_WLRC]) / n_cfg;
    }
    /* long-range correction derivatives (linear in eps_ab; sigma_ab powers) */
    if (s->lj_lrc) {
        double V = s->box[0] * s->box[1] * s->box[2];
        double rc = s->rc, rc3 = rc * rc * rc, rc9 = rc3 * rc3 * rc3;
        double pre = 2.0 * M_PI * (double)n * (double)n / V;
        for (int a = 0; a < m->n_lj; a++)
            for (int b = 0; b < m->n_lj; b++) {
                int ta = m->lj_type[a], tb = m->lj_type[b];
                double eps, sig;
                lj_mix(m, ta, tb, &eps, &sig);
                double s5 = pow(sig, 5.0), s6 = s5 * sig, s11 = s6 * s5, s12 = s6 * s6;
                double uL = 4.0 * (s12 / (9.0 * rc9) - s6 / (3.0 * rc3));     /* per unit eps */
                double wL = 4.0 * (4.0 * s12 / (3.0 * rc9) - 2.0 * s6 / rc3); /* per unit eps */
                double duL_ds = 4.0 * eps * (12.0 * s11 / (9.0 * rc9) - 6.0 * s5 / (3.0 * rc3));
                double dwL_ds = 4.0 * eps * (48.0 * s11 / (3.0 * rc9) - 12.0 * s5 / rc3);
                for (int t = 0; t < T; t++) {
                    double nt = (double)((ta == t) + (tb == t));
                    if (nt == 0.0) continue;
                    double deps_t = eps * nt / (2.0 * m->eps[t]);
                    double dsig_t = m->eta[ta * T + tb] * nt * 0.5;
                    dU[t] += pre * uL * deps_t;
                    dW[t] += pre * wL * deps_t;
                    dU[T + t] += pre * duL_ds * dsig_t;
                    dW[T + t] += pre * dwL_ds * dsig_t;
                }
            }
    }
    free(F);
    free(tau);
    return 0;
}
