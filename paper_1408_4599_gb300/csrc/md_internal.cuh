// md_internal.cuh -- device-side data layout and kernel launchers of the
// GB300 rigid multi-site MD library (arXiv 1408.4599: §2 models, §3 linked
// cells and leapfrog).  Not part of the public ABI (see include/md.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define MD_MAX_SITES 8
#define MD_MAX_TYPES 8
#define MD_WARPS 4          // warps per force block (one cell per warp)

// Roles a merged interaction site can carry (§2).  A site has one position
// and at most one axis, shared by its dipole and quadrupole roles.
enum { ROLE_LJ = 1, ROLE_CHG = 2, ROLE_DIP = 4, ROLE_QUAD = 8 };

// Everything the kernels need about the (single) molecular component, as a
// by-value kernel parameter.
struct DevModel {
    int S;                          // merged sites
    int NA;                         // sites carrying an axis
    int roles[MD_MAX_SITES];
    int lj_type[MD_MAX_SITES];
    int axis_slot[MD_MAX_SITES];    // index among axis-carrying sites, -1 if none
    float chg[MD_MAX_SITES], mu[MD_MAX_SITES], Q[MD_MAX_SITES];
    float body[MD_MAX_SITES][3];    // body-frame offsets
    float axis[MD_MAX_SITES][3];    // body-frame unit axis
    float eps4[MD_MAX_TYPES][MD_MAX_TYPES];   // 4 eps_ab
    float eps24[MD_MAX_TYPES][MD_MAX_TYPES];  // 24 eps_ab
    float sig2[MD_MAX_TYPES][MD_MAX_TYPES];   // sigma_ab^2
    float ushift[MD_MAX_TYPES][MD_MAX_TYPES]; // LJTS shift u_ab(rc) (0 if unshifted)
    float isig[MD_MAX_TYPES][MD_MAX_TYPES];     // 1 / sigma_ab
    float ushift_e[MD_MAX_TYPES][MD_MAX_TYPES]; // shift / eps_ab
    float dshift_s[MD_MAX_TYPES][MD_MAX_TYPES]; // d(shift / eps_ab) / d sigma_ab
    float frf;                      // reaction-field factor / rc^3
    int site_pairs_per_mol_pair;    // n_lj^2 + n_el^2 of the user's entities
    int single_lj_at_com;           // 1: one LJ site at the centre of mass, nothing else
    int linear;                     // 1: every site on the body z axis, every axis along +-z: the packed
                                    //    geometry is the space-frame molecular axis alone
    double mass;
    double Iinv[3], I[3];
    int rot_dof;                    // 0, 2 or 3
};

// Linked-cell grid (§3): n_c = floor(L / rc) cells per axis, x fastest.
struct Grid {
    int nc[3];
    long long ncell;
    double L[3];
    int m;                          // stencil radius in cells: 1 (edge >= rc) or 2 (edge >= rc / 2)
    double ell[3];                  // cell edge (>= rc / m)
    double iell[3];                 // 1 / ell
    float ellf[3];
    double rc2;
    float rc2f;
    float bandf;                    // |d^2 - rc^2| below which the test is redone in FP64
};

// Device buffers of one system (storage order = sorted cell order after
// every rebuild).
struct DevState {
    long long n;
    int K;                          // float4 per molecule in geo: S + NA
    double *r, *v, *q, *j;          // current state, n x 3 / n x 4
    double *r2, *v2, *q2, *j2;      // reorder targets
    int *ids, *ids2;                // caller's molecule index of each slot
    double *F, *tau;                // n x 3, storage order
    int *cell;                      // cell of each slot (current order)
    int *cell_count;                // ncell
    int *cell_start;                // ncell + 1
    int *cell_fill;                 // ncell
    int *perm, *perm2;              // new slot -> old slot
    float4 *com;                    // n: centre of mass relative to its cell centre
    float4 *geo;                    // n * K: site offsets then axes (space frame)
    int *scan_tmp;                  // block sums of the scan
    double *partials;               // force-kernel block partials, 8 per block, then one counter slot
    unsigned *cell_ctr;             // in that last slot: cells handed out by the force kernel
    double *kin_partials;           // kinetic partials, 4 per block ([2], [3]: half-step K for the thermostat)
    double *thermo;                 // [0] velocity-rescaling factor of the last step, [1] its T_half
    int *flags;                     // [0] non-finite, [1] overflow, [2] timeout
    float *facc;                    // n x 8 FP32 accumulators per molecule: F (3), 0, tau (3), 0 (half shell)
};

// Compiled model of a system (used by the batched replicas, which compile
// the model once through md_create).
struct md_system;
struct ModelInfo {
    DevModel m;
    Grid g;
    double lrc_u_coef, lrc_w_coef, rf_self_per_mol;
};
void model_info(const md_system *s, ModelInfo *out);

// Accumulator record of one molecule: two 16-byte halves (F, 0) and (tau, 0).
constexpr int FACC_STRIDE = 8;

// Element-wise atomic add of four floats to a 16-byte aligned address (one
// vector reduction instead of four scalar ones).
__device__ __forceinline__ void red_add_v4(float *addr, float a, float b, float c, float d)
{
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}

// Partial-sum layout of the force kernel (per block).
enum { P_U = 0, P_W, P_WXX, P_WYY, P_WZZ, P_NMOL, P_NSITE, P_NEXAM, P_COUNT };

enum { FLAG_NONFINITE = 0, FLAG_OVERFLOW = 1, FLAG_TIMEOUT = 2, FLAG_INPUT = 3 };

// ------------------------------------------------------------- launchers
// (all return cudaGetLastError() of the launch)
cudaError_t launch_cellid(const Grid &g, DevState &d, cudaStream_t s);
// beta (device scalar, may be NULL): factor applied to v and j while they are reordered
// zero_acc (non-deterministic rebuilds): also clear the FP32 accumulator
// records of the new order, for the half-shell force kernel that follows
cudaError_t launch_rebuild(const Grid &g, const DevModel &m, DevState &d, cudaStream_t s,
                           const double *beta = nullptr, int deterministic = 1, int zero_acc = 0);
cudaError_t launch_sort(long long ncell, DevState &d, cudaStream_t s);
void swap_state(DevState &d);
// half shell: the results stay in the FP32 accumulators d.facc until
// launch_force_finalize; full shell: FP64 d.F, d.tau directly.
// acc_zeroed: the records are already clear (the rebuild cleared them)
cudaError_t launch_force(const Grid &g, const DevModel &m, DevState &d, int half_shell, int dynamic_cells, int n_blocks,
                         cudaStream_t s, int acc_zeroed = 0);
// acc32: read the forces from d.facc instead of d.F, d.tau; zero_count:
// clear the histogram first (not needed after a non-deterministic rebuild,
// which leaves it at zero)
cudaError_t launch_integrate(const Grid &g, const DevModel &m, DevState &d, double dt, int acc32, cudaStream_t s,
                             int zero_count = 1);
cudaError_t launch_kinetic(const DevModel &m, DevState &d, double dt_half, int n_blocks, cudaStream_t s);
cudaError_t launch_rescale(const DevModel &m, DevState &d, double fac_v, double fac_j, cudaStream_t s);
// velocity rescaling to T_target: half-step kinetic energies -> d.thermo[0] = sqrt(T_target / T_half)
cudaError_t launch_thermostat(const DevModel &m, DevState &d, int n_blocks, double T_target, double dof,
                              cudaStream_t s);
// r, v, q, j (each may be NULL) in the caller's molecule order, one kernel
cudaError_t launch_scatter_state(const DevState &d, double *r, double *v, double *q, double *j, cudaStream_t s);
cudaError_t launch_scatter_out(const DevState &d, const double *src, int width, double *dst, cudaStream_t s);
cudaError_t launch_gather_in(DevState &d, const double *src, int width, double *dst, cudaStream_t s);
cudaError_t launch_prepare_input(const Grid &g, DevState &d, cudaStream_t s);
int force_blocks_default();
int device_sms();
cudaError_t launch_force_finalize(DevState &d, cudaStream_t s);
int adjoint_nacc(const DevModel &m);
cudaError_t launch_adjoint(const Grid &g, const DevModel &m, const DevState &d, int half_shell, int dynamic_cells,
                           int n_blocks, double *partials, int nacc, cudaStream_t s);
int scan_blocks(long long ncell);
