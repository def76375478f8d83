/*
 * md_oracle.h -- plain FP64 CPU oracle for the rigid multi-site molecular
 * dynamics hot path of "ls1 mardyn" (Niethammer et al., arXiv 1408.4599).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the CUDA library and the CUDA library never
 * calls it.
 *
 * What it computes (paper section / equation named per function in the .c):
 *   - short-range pair energy, forces, torques and molecular virial of rigid
 *     molecules made of LJ centres (§2, Eq. 1; LJTS; Lorentz-Berthelot with
 *     binary parameters), point charges, point dipoles and linear point
 *     quadrupoles (§2 multipole expansion), with a centre-of-mass cut-off
 *     and minimum-image periodic boundaries (§3), plus the reaction field
 *     for dipoles and the isotropic LJ long-range correction (§3);
 *   - either by brute force over all pairs or by linked cells (§3);
 *   - the leapfrog integrator, translational (Eqs. 2-3) and rotational
 *     (Eqs. 4-5, read as Fincham's quaternion leapfrog);
 *   - the analytic derivative of the total energy and virial with respect
 *     to the force-field parameters.
 */
#ifndef MD_ORACLE_H
#define MD_ORACLE_H
#include <stdint.h>

#define ORC_MAXT 8   /* LJ types */
#define ORC_MAXE 16  /* entities of one kind per molecule */

typedef struct {
    int32_t n_types;
    double eps[ORC_MAXT], sigma[ORC_MAXT];
    double xi[ORC_MAXT * ORC_MAXT], eta[ORC_MAXT * ORC_MAXT];
    int32_t n_lj;
    double lj_pos[ORC_MAXE * 3];
    int32_t lj_type[ORC_MAXE];
    double lj_mass[ORC_MAXE];
    int32_t n_chg;
    double chg_pos[ORC_MAXE * 3];
    double chg_q[ORC_MAXE];
    int32_t n_dip;
    double dip_pos[ORC_MAXE * 3];
    double dip_axis[ORC_MAXE * 3];
    double dip_mu[ORC_MAXE];
    int32_t n_quad;
    double quad_pos[ORC_MAXE * 3];
    double quad_axis[ORC_MAXE * 3];
    double quad_Q[ORC_MAXE];
} orc_model;

typedef struct {
    double box[3];
    double rc;
    double eps_rf;    /* dielectric constant of the continuum; INFINITY allowed */
    int32_t lj_shift; /* 1: truncated-shifted LJ (LJTS) */
    int32_t lj_lrc;   /* 1: isotropic long-range correction reported */
} orc_setup;

/* obs[] layout returned by orc_forces */
enum {
    ORC_U = 0,       /* pair potential energy inside the cut-off */
    ORC_W = 1,       /* molecular virial sum_{i<j} R_ij . F_ij */
    ORC_WXX = 2, ORC_WYY = 3, ORC_WZZ = 4,
    ORC_NMOL = 5,    /* interacting molecule pairs */
    ORC_NSITE = 6,   /* interacting site (entity) pairs */
    ORC_NEXAM = 7,   /* examined (distance-tested) molecule pairs */
    ORC_ULRC = 8, ORC_WLRC = 9,
    ORC_URFSELF = 10,
    ORC_ABSU = 11,   /* sum over interacting molecule pairs of |u_ij| */
    ORC_ABSW = 12,   /* sum over interacting molecule pairs of |R_ij . F_ij| */
    ORC_NOBS = 16
};

int orc_forces(const orc_model *m, const orc_setup *s, int64_t n, const double *r, const double *q,
               int use_cells, int n_threads, double *F, double *tau, double *obs);
int orc_forces_subset(const orc_model *m, const orc_setup *s, int64_t n, const double *r, const double *q,
                      int64_t n_sel, const int64_t *sel, int n_threads, double *F, double *tau);
int orc_step(const orc_model *m, const orc_setup *s, int64_t n, double dt, int n_steps, int use_cells,
             int n_threads, double *r, double *v, double *q, double *j, double *F, double *tau, double *obs);
/* orc_step with the velocity-rescaling thermostat (T_target > 0; <= 0: NVE) */
int orc_step_T(const orc_model *m, const orc_setup *s, int64_t n, double dt, int n_steps, double T_target,
               int use_cells, int n_threads, double *r, double *v, double *q, double *j, double *F, double *tau,
               double *obs);
int orc_kinetic(const orc_model *m, int64_t n, double dt, const double *v, const double *q, const double *j,
                const double *F, const double *tau, double *K);
int orc_lrc(const orc_model *m, const orc_setup *s, int64_t n, double *out);
int orc_n_params(const orc_model *m);
int orc_param_grad(const orc_model *m, const orc_setup *s, int n_cfg, int64_t n, const double *r_all,
                   const double *q_all, int use_cells, int n_threads, double *dU, double *dW, double *means,
                   double *absU, double *absW);
int orc_rotmat(const double *q, double *R);

#endif
