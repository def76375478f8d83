// md_batch.cu -- many independent replicas of uneven size advanced together
// (one model, one cut-off, each replica its own periodic box and state).
//
// Layout: the replicas' molecules and linked cells are concatenated;
// replica k owns slots [mol0_k, mol0_{k+1}) and cells [cell0_k, cell0_{k+1}).
// The counting sort only permutes molecules inside their own cells, so the
// slot -> replica map never changes.  One launch of each kernel covers all
// replicas:
//   integrate (per-slot replica box) -> one counting sort over all cells ->
//   reorder + pack (per-slot replica grid) -> persistent force kernels.
// The force kernels pull chunks of cells from an atomic work queue ordered
// longest-first by the paper's per-cell cost estimate
// n_d(i) ~ N_i/2 (N_i + sum_neigh N_j) (§4, Eq. 6), evaluated per replica
// from its mean cell occupancy; replicas with >= 3 cells per axis use the
// Newton-3 half stencil, smaller boxes the full stencil (two launches).
// Energies and virials are written per cell and reduced per replica in a
// fixed order.  md_batch_step can replay the steps from a captured CUDA
// graph; md_batch_tune times the work-chunk size and grid occupancy.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/md.h"
#include "md_forceop.cuh"
#include "md_leapfrog.cuh"

using namespace mdk;

// Per-replica grid on the device.
struct RepGrid {
    int nc[3];
    int half;  // 1: half stencil (needs >= 3 cells per axis and options->half_shell; see half_min_occ)
    float ellf[3];
    double L[3];
    double ell[3];
    double iell[3];  // 1 / ell
    long long cell0, mol0;
};

struct md_batch {
    int n_sys = 0;
    md_system *tmpl = nullptr;  // model compiled once (md_create of the first box)
    DevModel m;
    md_options opt;
    double rc = 0.0, lrc_u = 0.0, lrc_w = 0.0, rf_self = 0.0;
    std::vector<RepGrid> grids;
    std::vector<char> half_ok;  // replica may use the half stencil
    std::vector<long long> n_per;
    std::vector<long long> cell_off;
    std::vector<double> rep_cost;  // Eq. 6 cost estimate per replica
    std::vector<int> work_host;    // host copy of the work list
    long long ncell = 0, ntot = 0, cap = 0;
    Grid g;  // shared scalars (rc2, band); ncell = total cells
    DevState d;
    RepGrid *dgrids = nullptr;
    int *rep_of_slot = nullptr, *rep_of_cell = nullptr;
    int *work = nullptr;  // [half list | full list] of cells, longest replicas first
    long long n_work_half = 0, n_work_full = 0;
    int *counters = nullptr;  // work-queue heads (2)
    double *cellE = nullptr;  // 5 per cell
    int *cellN = nullptr;     // 2 per cell
    double *rep_obs = nullptr;  // 8 per replica
    double *rep_kin = nullptr;  // 2 per replica
    double *rep_T = nullptr;    // per-replica thermostat target (<= 0: NVE)
    double *rep_beta = nullptr; // per-replica velocity-rescaling factor of the last step
    bool nvt = false;           // some replica has a target
    bool has_mol = false, forces_valid = false;
    bool f_in_acc = false;  // the latest forces exist only in the FP32 accumulators
    double dt_last = 0.0, time = 0.0;
    long long step = 0;
    int chunk = 2, grid_frac_pct = 100;
    int test_width = NTEST;     // candidates per lane per test round (4 or NTEST)
    double half_min_occ = 0.0;  // replicas below this mean occupancy (molecules per cell) run the full shell
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    double gdt[2] = {0.0, 0.0};
    int parity = 0;
    char err[512];
};

namespace {

__global__ void k_prepare_b(const RepGrid *G, const int *rep, double *r, double *q, int *ids, long long n, int *flags)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const RepGrid &g = G[rep[s]];
    bool bad = false;
    for (int k = 0; k < 3; k++) {
        double x = r[3 * s + k];
        bad |= !isfinite(x);
        x -= g.L[k] * floor(x / g.L[k]);
        if (x >= g.L[k]) x -= g.L[k];
        if (x < 0.0) x = 0.0;
        r[3 * s + k] = x;
    }
    double nn = sqrt(q[4 * s] * q[4 * s] + q[4 * s + 1] * q[4 * s + 1] + q[4 * s + 2] * q[4 * s + 2] +
                     q[4 * s + 3] * q[4 * s + 3]);
    bad |= !(nn > 0.0) || !isfinite(nn);
    for (int k = 0; k < 4; k++) q[4 * s + k] /= nn;
    ids[s] = (int)s;
    if (bad) atomicExch(&flags[FLAG_NONFINITE], 1);
}

__global__ void k_cellid_b(const RepGrid *G, const int *rep, const double *r, int *cell, int *count, long long n)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const RepGrid &g = G[rep[s]];
    const int cx = cell_coord(r[3 * s], g.iell[0], g.nc[0]);
    const int cy = cell_coord(r[3 * s + 1], g.iell[1], g.nc[1]);
    const int cz = cell_coord(r[3 * s + 2], g.iell[2], g.nc[2]);
    const int c = (int)g.cell0 + (cz * g.nc[1] + cy) * g.nc[0] + cx;
    cell[s] = c;
    atomicAdd(&count[c], 1);
}

// Leapfrog of §3 (Eqs. 2-5), the single-system step of md_leapfrog.cuh
// with the slot's replica box; the forces come from the FP32 accumulators,
// which every replica's force pass fills.
__global__ void k_integrate_b(const RepGrid *G, const int *rep, DevModel m, DevState d, LeapArgs a)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= d.n) return;
    const RepGrid &g = G[rep[s]];
    int cc[3];
    if (leapfrog_one<true>(m, d, s, a, g.L, g.iell, g.nc, cc)) atomicExch(&d.flags[FLAG_NONFINITE], 1);
    const int c = (int)g.cell0 + (cc[2] * g.nc[1] + cc[1]) * g.nc[0] + cc[0];
    d.cell[s] = c;
    atomicAdd(&d.cell_count[c], 1);
}

__global__ void k_reorder_pack_b(const RepGrid *G, const int *rep, DevModel m, DevState d, const double *beta)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= d.n) return;
    const int o = d.perm2[s];
    const double rx = d.r[3 * o], ry = d.r[3 * o + 1], rz = d.r[3 * o + 2];
    d.r2[3 * s] = rx;
    d.r2[3 * s + 1] = ry;
    d.r2[3 * s + 2] = rz;
    const double b = beta ? beta[rep[s]] : 1.0;  // velocity rescaling of the slot's replica
    for (int k = 0; k < 3; k++) {
        d.v2[3 * s + k] = b * d.v[3 * o + k];
        d.j2[3 * s + k] = b * d.j[3 * o + k];
    }
    const double qw = d.q[4 * o], qx = d.q[4 * o + 1], qy = d.q[4 * o + 2], qz = d.q[4 * o + 3];
    d.q2[4 * s] = qw;
    d.q2[4 * s + 1] = qx;
    d.q2[4 * s + 2] = qy;
    d.q2[4 * s + 3] = qz;
    d.ids2[s] = d.ids[o];
    const RepGrid &g = G[rep[s]];
    const int c = d.cell[o] - (int)g.cell0;
    const int cx = c % g.nc[0], cy = (c / g.nc[0]) % g.nc[1], cz = c / (g.nc[0] * g.nc[1]);
    // conversions on the integer pipe (md_fpconv.cuh), the same bits as the hardware's
    d.com[s] = make_float4(d2f_bits(rx - int_plus_half(cx) * g.ell[0]), d2f_bits(ry - int_plus_half(cy) * g.ell[1]),
                           d2f_bits(rz - int_plus_half(cz) * g.ell[2]), 0.f);
    if (m.single_lj_at_com) return;
    const float w = d2f_bits(qw), x = d2f_bits(qx), y = d2f_bits(qy), z = d2f_bits(qz);
    const float R[9] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y),
                        2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x),
                        2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)};
    float4 *out = d.geo + s * (long long)d.K;
    if (m.linear) {  // the molecular axis R(q) z carries every site offset and axis
        out[0] = make_float4(R[2], R[5], R[8], 0.f);
        return;
    }
    for (int a = 0; a < m.S; a++) {
        const float *b = m.body[a];
        out[a] = make_float4(R[0] * b[0] + R[1] * b[1] + R[2] * b[2], R[3] * b[0] + R[4] * b[1] + R[5] * b[2],
                             R[6] * b[0] + R[7] * b[1] + R[8] * b[2], 0.f);
        if (m.axis_slot[a] >= 0) {
            const float *e = m.axis[a];
            out[m.S + m.axis_slot[a]] =
                make_float4(R[0] * e[0] + R[1] * e[1] + R[2] * e[2], R[3] * e[0] + R[4] * e[1] + R[5] * e[2],
                            R[6] * e[0] + R[7] * e[1] + R[8] * e[2], 0.f);
        }
    }
}

struct BatchArgs {
    ForceArgs f;  // model, packed data, accumulators (grid fields and cell_ctr unused)
    const RepGrid *grids;
    const int *rep_of_cell;
    const int *work;
    long long n_work;
    int *counter;
    int chunk;
    double *cellE;
    int *cellN;
};

// Persistent force kernel over a work list of cells of many replicas.
template <class SIG, bool HALF, int NT>
__global__ void __launch_bounds__(MD_WARPS * 32) k_force_batch(const __grid_constant__ BatchArgs B)
{
    using Op = ForceOp<SIG, HALF, false>;  // chunked half shell (see ForceOp)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    typename Op::Tile *T = reinterpret_cast<typename Op::Tile *>(smem_raw) + warp;
    const DevModel &m = B.f.m;
    const int K = SIG::kk(m);
    Op op(m, B.f, K, T);
    for (;;) {
        long long w0 = 0;
        if (lane == 0) w0 = atomicAdd(B.counter, B.chunk);
        w0 = __shfl_sync(FULLMASK, w0, 0);
        if (w0 >= B.n_work) break;
        const long long w1 = min(w0 + (long long)B.chunk, B.n_work);
        for (long long w = w0; w < w1; w++) {
            const long long c = B.work[w];
            const RepGrid &rg = B.grids[B.rep_of_cell[c]];
            GridView gv;
            for (int k = 0; k < 3; k++) {
                gv.nc[k] = rg.nc[k];
                gv.ellf[k] = rg.ellf[k];
                gv.L[k] = rg.L[k];
            }
            gv.rc2 = B.f.g.rc2;
            gv.rc2f = B.f.g.rc2f;
            gv.bandf = B.f.g.bandf;
            gv.cell0 = rg.cell0;
            traverse_cell<SIG, HALF, 1, NT>(m, gv, B.f.cell_start, B.f.com, B.f.geo, B.f.r, K, c - rg.cell0, *T, op,
                                            lane);
            double v[5];
            int nm, ne;
            op_warp_totals(op, v, nm, ne);
            if (lane == 0) {
                for (int q = 0; q < 5; q++) B.cellE[5 * c + q] = v[q];
                B.cellN[2 * c] = nm;
                B.cellN[2 * c + 1] = ne;
            }
            op.reset_totals();
        }
    }
}

// One block per replica: energies/virials/counts (fixed summation order).
__global__ void k_rep_reduce(const RepGrid *G, int n_sys, long long ncell, const double *cellE, const int *cellN,
                             int site_pairs, double *out)
{
    const int k = blockIdx.x;
    if (k >= n_sys) return;
    const long long c0 = G[k].cell0, c1 = (k + 1 < n_sys) ? G[k + 1].cell0 : ncell;
    __shared__ double sh[8][32];
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (long long c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
        for (int q = 0; q < 5; q++) acc[q] += cellE[5 * c + q];
        acc[5] += (double)cellN[2 * c];
        acc[7] += (double)cellN[2 * c + 1];
    }
    for (int q = 0; q < 8; q++)
        for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
        for (int q = 0; q < 8; q++) sh[q][warp] = acc[q];
    __syncthreads();
    if (threadIdx.x < 8) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += sh[threadIdx.x][w];
        const double esc = G[k].half ? 1.0 : 0.5;
        if (threadIdx.x == 6) {
            t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += sh[5][w];
            t *= (double)site_pairs;
        }
        out[8 * k + threadIdx.x] = esc * t;
    }
}

// One block per replica: kinetic energies at integer time (FP64).
__global__ void k_rep_kinetic(const RepGrid *G, int n_sys, long long n, DevModel m, DevState d, double dt_half,
                              double *out)
{
    const int k = blockIdx.x;
    if (k >= n_sys) return;
    const long long s0 = G[k].mol0, s1 = (k + 1 < n_sys) ? G[k + 1].mol0 : n;
    __shared__ double sh[2][32];
    double kt = 0.0, kr = 0.0;
    const double im = 1.0 / m.mass;
    const float Iinv[3] = {(float)m.Iinv[0], (float)m.Iinv[1], (float)m.Iinv[2]};
    const float Im[3] = {(float)m.I[0], (float)m.I[1], (float)m.I[2]};
    for (long long s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
        double v2 = 0.0;
        for (int q = 0; q < 3; q++) {
            const double vq = d.v[3 * s + q] + dt_half * d.F[3 * s + q] * im;
            v2 += vq * vq;
        }
        kt += 0.5 * m.mass * v2;
        if (m.rot_dof > 0) {
            const double jt[3] = {d.j[3 * s] + dt_half * d.tau[3 * s], d.j[3 * s + 1] + dt_half * d.tau[3 * s + 1],
                                  d.j[3 * s + 2] + dt_half * d.tau[3 * s + 2]};
            kr += 0.5 * (double)kin_rot2(d.q + 4 * s, jt, Iinv, Im);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        kt += __shfl_xor_sync(0xffffffffu, kt, o);
        kr += __shfl_xor_sync(0xffffffffu, kr, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        sh[0][warp] = kt;
        sh[1][warp] = kr;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += sh[threadIdx.x][w];
        out[2 * k + threadIdx.x] = t;
    }
}

// Velocity rescaling per replica (§2 NVT), one block per replica: half-step
// kinetic temperature (v, j at t + dt/2, q at t + dt; translational part in
// FP64, rotational per molecule in FP32 with FP64 sums) and the factor
// sqrt(T_k / T_half), 1 for replicas without a target.
__global__ void k_rep_thermostat(const RepGrid *G, int n_sys, long long n, DevModel m, DevState d, const double *Tt,
                                 double *beta)
{
    const int k = blockIdx.x;
    if (k >= n_sys) return;
    const long long s0 = G[k].mol0, s1 = (k + 1 < n_sys) ? G[k + 1].mol0 : n;
    __shared__ double sh[32];
    double e = 0.0;  // 2 K
    const float Iinv[3] = {(float)m.Iinv[0], (float)m.Iinv[1], (float)m.Iinv[2]};
    const float Im[3] = {(float)m.I[0], (float)m.I[1], (float)m.I[2]};
    if (Tt[k] > 0.0)
        for (long long s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
            const double v0 = d.v[3 * s], v1 = d.v[3 * s + 1], v2 = d.v[3 * s + 2];
            e += m.mass * (v0 * v0 + v1 * v1 + v2 * v2);
            if (m.rot_dof > 0) {
                const double jh[3] = {d.j[3 * s], d.j[3 * s + 1], d.j[3 * s + 2]};
                e += (double)kin_rot2(d.q + 4 * s, jh, Iinv, Im);
            }
        }
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += sh[w];
        const double N = (double)(s1 - s0), dof = 3.0 * N - 3.0 + (double)m.rot_dof * N;
        const double T = dof > 0.0 ? t / dof : 0.0;
        beta[k] = (Tt[k] > 0.0 && T > 0.0 && isfinite(T)) ? sqrt(Tt[k] / T) : 1.0;
    }
}

struct LaunchBatchForce {
    const BatchArgs &B;
    int half, blocks_cap, nt;
    cudaStream_t s;
    template <class SIG>
    cudaError_t operator()() const
    {
        if (half) return nt == 4 ? run<SIG, true, 4>() : run<SIG, true, NTEST>();
        return nt == 4 ? run<SIG, false, 4>() : run<SIG, false, NTEST>();
    }
    template <class SIG, bool HALF, int NT>
    cudaError_t run() const
    {
        if (B.n_work == 0) return cudaSuccess;
        const size_t sm = sizeof(typename ForceOp<SIG, HALF, false>::Tile) * MD_WARPS;
        cudaFuncSetAttribute(k_force_batch<SIG, HALF, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        int per_sm = 0, dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_force_batch<SIG, HALF, NT>, MD_WARPS * 32, sm);
        long long want = (long long)(per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
        want = want * blocks_cap / 100;
        const long long need = (B.n_work + MD_WARPS - 1) / MD_WARPS;
        if (want > need) want = need;
        if (want < 1) want = 1;
        k_force_batch<SIG, HALF, NT><<<(unsigned)want, MD_WARPS * 32, sm, s>>>(B);
        return cudaGetLastError();
    }
};

void bset_err(md_batch *b, const char *msg) { snprintf(b->err, sizeof b->err, "%s", msg); }

md_status bcuda(md_batch *b, cudaError_t e, const char *where);

// Stencil of every replica (half where allowed and the replica's mean
// occupancy is at least half_min_occ molecules per cell, full otherwise)
// and the work list: half-stencil cells first, each list longest replica
// first by the Eq. 6 cost; copies grids and list to the device on st.
md_status apply_shell_policy(md_batch *b, cudaStream_t st)
{
    for (int k = 0; k < b->n_sys; k++) {
        const double nce = (double)(b->cell_off[k + 1] - b->cell_off[k]);
        const double occ = (double)b->n_per[k] / nce;
        b->grids[k].half = (b->half_ok[k] && occ >= b->half_min_occ) ? 1 : 0;
    }
    std::vector<int> order(b->n_sys);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return b->rep_cost[a] > b->rep_cost[c]; });
    b->work_host.clear();
    b->work_host.reserve((size_t)b->ncell);
    for (int pass = 1; pass >= 0; pass--)
        for (int k : order)
            if (b->grids[k].half == pass)
                for (long long c = b->cell_off[k]; c < b->cell_off[k + 1]; c++) b->work_host.push_back((int)c);
    b->n_work_half = 0;
    for (int k = 0; k < b->n_sys; k++)
        if (b->grids[k].half) b->n_work_half += b->cell_off[k + 1] - b->cell_off[k];
    b->n_work_full = b->ncell - b->n_work_half;
    cudaError_t e = cudaMemcpyAsync(b->dgrids, b->grids.data(), sizeof(RepGrid) * b->n_sys, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->work, b->work_host.data(), sizeof(int) * b->work_host.size(), cudaMemcpyHostToDevice, st);
    // the host vectors must outlive the copies
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? MD_OK : bcuda(b, e, "copy grids / work list");
}

md_status bcuda(md_batch *b, cudaError_t e, const char *where)
{
    snprintf(b->err, sizeof b->err, "%s: %s", where, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? MD_ERR_OOM : MD_ERR_CUDA;
}

#define BCK(call, where)                                      \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return bcuda(b, e_, where);    \
    } while (0)

inline unsigned nb256(long long n) { return (unsigned)((n + 255) / 256); }

BatchArgs batch_args(md_batch *b, bool half_list)
{
    BatchArgs B;
    memset(&B, 0, sizeof B);
    B.f.g = b->g;
    B.f.m = b->m;
    B.f.cell_start = b->d.cell_start;
    B.f.com = b->d.com;
    B.f.geo = b->d.geo;
    B.f.r = b->d.r;
    B.f.F = b->d.F;
    B.f.tau = b->d.tau;
    B.f.acc = b->d.facc;
    B.f.n = b->d.n;
    B.f.partials = nullptr;
    B.f.flags = b->d.flags;
    B.f.to_acc = 1;
    B.f.cell_ctr = nullptr;
    B.f.parts = 1;
    B.grids = b->dgrids;
    B.rep_of_cell = b->rep_of_cell;
    B.work = half_list ? b->work : b->work + b->n_work_half;
    B.n_work = half_list ? b->n_work_half : b->n_work_full;
    B.counter = b->counters + (half_list ? 0 : 1);
    B.chunk = b->chunk;
    B.cellE = b->cellE;
    B.cellN = b->cellN;
    return B;
}

// Forces for all replicas at the current (packed) configuration.
md_status batch_force(md_batch *b, cudaStream_t st)
{
    DevState &d = b->d;
    BCK(cudaMemsetAsync(d.facc, 0, sizeof(float) * FACC_STRIDE * (d.n > 0 ? d.n : 1), st), "zero accumulators");
    BCK(cudaMemsetAsync(b->counters, 0, 2 * sizeof(int), st), "zero work queues");
    for (int h = 1; h >= 0; h--) {
        BatchArgs B = batch_args(b, h == 1);
        BCK(dispatch_sig(b->m, LaunchBatchForce{B, h, b->grid_frac_pct, b->test_width, st}), "batched force kernel");
    }
    b->forces_valid = true;
    b->f_in_acc = true;
    return MD_OK;
}

// FP64 F and tau for the readers outside the step (the integrator reads the
// FP32 accumulators).
md_status batch_forces_to_f64(md_batch *b, cudaStream_t st)
{
    if (!b->f_in_acc) return MD_OK;
    BCK(launch_force_finalize(b->d, st), "force finalize");
    b->f_in_acc = false;
    return MD_OK;
}

md_status batch_rebuild(md_batch *b, cudaStream_t st, bool need_cellid, const double *beta = nullptr)
{
    DevState &d = b->d;
    if (need_cellid) {
        BCK(cudaMemsetAsync(d.cell_count, 0, sizeof(int) * b->ncell, st), "zero counts");
        if (d.n > 0) k_cellid_b<<<nb256(d.n), 256, 0, st>>>(b->dgrids, b->rep_of_slot, d.r, d.cell, d.cell_count, d.n);
    }
    BCK(launch_sort(b->ncell, d, st), "counting sort");
    if (d.n > 0) k_reorder_pack_b<<<nb256(d.n), 256, 0, st>>>(b->dgrids, b->rep_of_slot, b->m, d, beta);
    BCK(cudaGetLastError(), "reorder/pack kernel");
    swap_state(d);
    return MD_OK;
}

md_status batch_one_step(md_batch *b, double dt, cudaStream_t st)
{
    DevState &d = b->d;
    BCK(cudaMemsetAsync(d.cell_count, 0, sizeof(int) * b->ncell, st), "zero counts");
    if (d.n > 0) k_integrate_b<<<nb256(d.n), 256, 0, st>>>(b->dgrids, b->rep_of_slot, b->m, d, leap_args(b->m, dt));
    BCK(cudaGetLastError(), "integrate kernel");
    if (b->nvt) {
        k_rep_thermostat<<<b->n_sys, 256, 0, st>>>(b->dgrids, b->n_sys, d.n, b->m, d, b->rep_T, b->rep_beta);
        BCK(cudaGetLastError(), "thermostat kernel");
    }
    md_status ms = batch_rebuild(b, st, false, b->nvt ? b->rep_beta : nullptr);
    if (ms != MD_OK) return ms;
    return batch_force(b, st);
}

void drop_graphs(md_batch *b)
{
    for (int p = 0; p < 2; p++)
        if (b->gexec[p]) {
            cudaGraphExecDestroy(b->gexec[p]);
            b->gexec[p] = nullptr;
        }
}

void batch_free(md_batch *b)
{
    drop_graphs(b);
    DevState &d = b->d;
    void *ptrs[] = {d.r, d.v, d.q, d.j, d.r2, d.v2, d.q2, d.j2, d.ids, d.ids2, d.F, d.tau, d.cell, d.cell_count,
                    d.cell_start, d.cell_fill, d.perm, d.perm2, d.com, d.geo, d.scan_tmp, d.flags, d.facc,
                    b->dgrids, b->rep_of_slot, b->rep_of_cell, b->work, b->counters, b->cellE, b->cellN,
                    b->rep_obs, b->rep_kin, b->rep_T, b->rep_beta};
    for (void *p : ptrs) cudaFree(p);
    memset(&b->d, 0, sizeof b->d);
    b->dgrids = nullptr;
    b->rep_of_slot = b->rep_of_cell = b->work = b->counters = b->cellN = nullptr;
    b->cellE = nullptr;
    b->rep_obs = b->rep_kin = b->rep_T = b->rep_beta = nullptr;
    b->cap = 0;
}

}  // namespace

extern "C" {

md_status md_batch_create(int32_t n_sys, const double *boxes, double cutoff, const md_site_types *types,
                          const md_options *options, md_batch **out)
{
    if (!out || n_sys < 1 || !boxes || !types) return MD_ERR_ARG;
    *out = nullptr;
    md_batch *b = new (std::nothrow) md_batch();
    if (!b) return MD_ERR_OOM;
    for (int k = 0; k < n_sys; k++)
        for (int a = 0; a < 3; a++)
            if (!(std::isfinite(boxes[3 * k + a]) && boxes[3 * k + a] > 0.0)) {
                delete b;
                return MD_ERR_ARG;
            } else if (boxes[3 * k + a] < 2.0 * cutoff) {
                delete b;
                return MD_ERR_BOX;
            }
    md_options opt = {INFINITY, 0, 0, 1, 1, 1};
    if (options) opt = *options;
    if (opt.cell_div != 0 && opt.cell_div != 1) {  // replicas use cells of edge >= cutoff
        delete b;
        return opt.cell_div == 2 ? MD_ERR_UNSUPPORTED : MD_ERR_ARG;
    }
    md_status st = md_create(boxes, cutoff, types, &opt, &b->tmpl);
    if (st != MD_OK) {
        delete b;
        return st;
    }
    ModelInfo mi;
    model_info(b->tmpl, &mi);
    b->m = mi.m;
    b->g = mi.g;
    b->lrc_u = mi.lrc_u_coef;
    b->lrc_w = mi.lrc_w_coef;
    b->rf_self = mi.rf_self_per_mol;
    b->opt = opt;
    b->rc = cutoff;
    b->n_sys = n_sys;
    b->grids.resize(n_sys);
    b->cell_off.assign(n_sys + 1, 0);
    long long nc_tot = 0;
    for (int k = 0; k < n_sys; k++) {
        RepGrid &g = b->grids[k];
        bool all3 = true;
        for (int a = 0; a < 3; a++) {
            int nc = (int)std::floor(boxes[3 * k + a] / (cutoff * (1.0 + 1e-9)));
            g.nc[a] = nc < 1 ? 1 : nc;
            g.L[a] = boxes[3 * k + a];
            g.ell[a] = g.L[a] / g.nc[a];
            g.iell[a] = 1.0 / g.ell[a];
            g.ellf[a] = (float)g.ell[a];
            all3 = all3 && g.nc[a] >= 3;
        }
        g.half = (opt.half_shell && all3) ? 1 : 0;
        b->half_ok.push_back((char)g.half);
        g.cell0 = nc_tot;
        b->cell_off[k] = nc_tot;
        nc_tot += (long long)g.nc[0] * g.nc[1] * g.nc[2];
    }
    b->cell_off[n_sys] = nc_tot;
    if (nc_tot > (1LL << 31) - 2) {
        md_destroy(b->tmpl);
        delete b;
        return MD_ERR_UNSUPPORTED;
    }
    b->ncell = nc_tot;
    b->g.ncell = nc_tot;
    b->d.K = b->m.single_lj_at_com ? 0 : (b->m.linear ? 1 : b->m.S + b->m.NA);
    DevState &d = b->d;
    cudaError_t e = cudaMalloc((void **)&d.cell_count, sizeof(int) * nc_tot);
    if (e == cudaSuccess) e = cudaMalloc((void **)&d.cell_start, sizeof(int) * (nc_tot + 1));
    if (e == cudaSuccess) e = cudaMalloc((void **)&d.cell_fill, sizeof(int) * nc_tot);
    if (e == cudaSuccess) e = cudaMalloc((void **)&d.scan_tmp, sizeof(int) * (scan_blocks(nc_tot) + 1));
    if (e == cudaSuccess) e = cudaMalloc((void **)&d.flags, sizeof(int) * 4);
    if (e == cudaSuccess) e = cudaMemset(d.flags, 0, sizeof(int) * 4);
    if (e == cudaSuccess) e = cudaMemset(d.cell_start, 0, sizeof(int) * (nc_tot + 1));
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->dgrids, sizeof(RepGrid) * n_sys);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->rep_of_cell, sizeof(int) * nc_tot);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->work, sizeof(int) * nc_tot);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->counters, sizeof(int) * 2);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->cellE, sizeof(double) * 5 * nc_tot);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->cellN, sizeof(int) * 2 * nc_tot);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->rep_obs, sizeof(double) * 8 * n_sys);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->rep_kin, sizeof(double) * 2 * n_sys);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->rep_T, sizeof(double) * n_sys);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->rep_beta, sizeof(double) * n_sys);
    if (e == cudaSuccess) e = cudaMemset(b->rep_T, 0, sizeof(double) * n_sys);
    if (e == cudaSuccess) e = cudaMemset(b->cellE, 0, sizeof(double) * 5 * nc_tot);
    if (e == cudaSuccess) e = cudaMemset(b->cellN, 0, sizeof(int) * 2 * nc_tot);
    if (e == cudaSuccess) {
        std::vector<int> roc(nc_tot);
        for (int k = 0; k < n_sys; k++)
            for (long long c = b->cell_off[k]; c < b->cell_off[k + 1]; c++) roc[c] = k;
        e = cudaMemcpy(b->rep_of_cell, roc.data(), sizeof(int) * nc_tot, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        md_status r = bcuda(b, e, "md_batch_create allocations");
        batch_free(b);
        md_destroy(b->tmpl);
        delete b;
        return r;
    }
    *out = b;
    return MD_OK;
}

void md_batch_destroy(md_batch *b)
{
    if (!b) return;
    cudaDeviceSynchronize();
    batch_free(b);
    md_destroy(b->tmpl);
    delete b;
}

const char *md_batch_last_error(const md_batch *b) { return b ? b->err : "NULL handle"; }

md_status md_batch_set_molecules(md_batch *b, const int64_t *n_per_sys, const double *r, const double *v,
                                 const double *q, const double *j, int32_t on_device, void *cuda_stream)
{
    if (!b || !n_per_sys) return MD_ERR_ARG;
    long long ntot = 0;
    for (int k = 0; k < b->n_sys; k++) {
        if (n_per_sys[k] < 0) return MD_ERR_ARG;
        ntot += n_per_sys[k];
    }
    if (ntot > (1LL << 31) - 1 || (ntot > 0 && (!r || !q))) return MD_ERR_ARG;
    if (!on_device)
        for (long long i = 0; i < 3 * ntot; i++)
            if (!std::isfinite(r[i]) || (v && !std::isfinite(v[i])) || (j && !std::isfinite(j[i]))) {
                bset_err(b, "md_batch_set_molecules: non-finite input");
                return MD_ERR_ARG;
            }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    drop_graphs(b);
    DevState &d = b->d;
    if (ntot > b->cap || !d.r) {
        double **dbl[] = {&d.r, &d.v, &d.j, &d.r2, &d.v2, &d.j2, &d.F, &d.tau};
        for (auto p : dbl) {
            cudaFree(*p);
            *p = nullptr;
        }
        void *others[] = {d.q, d.q2, d.ids, d.ids2, d.cell, d.perm, d.perm2, d.com, d.geo, d.facc, b->rep_of_slot};
        for (void *p : others) cudaFree(p);
        d.q = d.q2 = nullptr;
        d.ids = d.ids2 = d.cell = d.perm = d.perm2 = nullptr;
        d.com = d.geo = nullptr;
        d.facc = nullptr;
        b->rep_of_slot = nullptr;
        const size_t nn = (size_t)(ntot > 0 ? ntot : 1);
        cudaError_t e = cudaSuccess;
        for (auto p : dbl)
            if (e == cudaSuccess) e = cudaMalloc((void **)p, nn * 3 * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc((void **)&d.q, nn * 4 * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc((void **)&d.q2, nn * 4 * sizeof(double));
        int **ints[] = {&d.ids, &d.ids2, &d.cell, &d.perm, &d.perm2, &b->rep_of_slot};
        for (auto p : ints)
            if (e == cudaSuccess) e = cudaMalloc((void **)p, nn * sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc((void **)&d.com, nn * sizeof(float4));
        if (e == cudaSuccess) e = cudaMalloc((void **)&d.geo, nn * (size_t)(d.K > 0 ? d.K : 1) * sizeof(float4));
        if (e == cudaSuccess) e = cudaMalloc((void **)&d.facc, nn * FACC_STRIDE * sizeof(float));
        if (e != cudaSuccess) return bcuda(b, e, "allocating batch molecule buffers");
        b->cap = ntot;
    }
    d.n = ntot;
    b->ntot = ntot;
    b->n_per.assign(n_per_sys, n_per_sys + b->n_sys);
    // per-replica molecule offsets and the longest-first work list
    long long m0 = 0;
    std::vector<int> ros((size_t)(ntot > 0 ? ntot : 1));
    std::vector<double> cost(b->n_sys);
    for (int k = 0; k < b->n_sys; k++) {
        RepGrid &g = b->grids[k];
        g.mol0 = m0;
        for (long long i = 0; i < n_per_sys[k]; i++) ros[m0 + i] = k;
        m0 += n_per_sys[k];
        const double nce = (double)(b->cell_off[k + 1] - b->cell_off[k]);
        const double occ = (double)n_per_sys[k] / nce;  // mean molecules per cell
        cost[k] = nce * 0.5 * occ * (occ + 26.0 * occ);  // sum over cells of n_d (§4, Eq. 6)
    }
    b->rep_cost = cost;
    cudaStream_t st0 = st;
    {
        md_status wm = apply_shell_policy(b, st0);
        if (wm != MD_OK) return wm;
    }
    BCK(cudaMemcpyAsync(b->rep_of_slot, ros.data(), sizeof(int) * ros.size(), cudaMemcpyHostToDevice, st0),
        "copy slot map");
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const size_t b3 = sizeof(double) * 3 * (size_t)ntot, b4 = sizeof(double) * 4 * (size_t)ntot;
    if (ntot > 0) {
        BCK(cudaMemcpyAsync(d.r, r, b3, kind, st), "copy r");
        BCK(cudaMemcpyAsync(d.q, q, b4, kind, st), "copy q");
        if (v) BCK(cudaMemcpyAsync(d.v, v, b3, kind, st), "copy v");
        else BCK(cudaMemsetAsync(d.v, 0, b3, st), "zero v");
        if (j) BCK(cudaMemcpyAsync(d.j, j, b3, kind, st), "copy j");
        else BCK(cudaMemsetAsync(d.j, 0, b3, st), "zero j");
        BCK(cudaMemsetAsync(d.F, 0, b3, st), "zero F");
        BCK(cudaMemsetAsync(d.tau, 0, b3, st), "zero tau");
        k_prepare_b<<<nb256(ntot), 256, 0, st>>>(b->dgrids, b->rep_of_slot, d.r, d.q, d.ids, ntot, d.flags);
        BCK(cudaGetLastError(), "prepare kernel");
    }
    md_status ms = batch_rebuild(b, st, true);
    if (ms != MD_OK) return ms;
    b->has_mol = true;
    b->forces_valid = false;
    b->f_in_acc = false;
    b->dt_last = b->time = 0.0;
    b->step = 0;
    b->parity = 0;
    if (!on_device) BCK(cudaStreamSynchronize(st), "md_batch_set_molecules sync");
    return MD_OK;
}

md_status md_batch_compute_forces(md_batch *b, void *cuda_stream)
{
    if (!b) return MD_ERR_ARG;
    if (!b->has_mol) {
        bset_err(b, "md_batch_compute_forces: call md_batch_set_molecules first");
        return MD_ERR_STATE;
    }
    return batch_force(b, (cudaStream_t)cuda_stream);
}

md_status md_batch_step(md_batch *b, int32_t n_steps, double dt, int32_t use_graph, void *cuda_stream)
{
    if (!b) return MD_ERR_ARG;
    if (!b->has_mol) {
        bset_err(b, "md_batch_step: call md_batch_set_molecules first");
        return MD_ERR_STATE;
    }
    if (n_steps < 0 || !std::isfinite(dt) || !(dt > 0.0) || !(b->m.mass > 0.0)) return MD_ERR_ARG;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (!b->forces_valid) {
        md_status ms = batch_force(b, st);
        if (ms != MD_OK) return ms;
    }
    int k = 0;
    if (use_graph) {
        // a captured pair of steps returns the ping-pong buffers to where they
        // started, so one executable graph per buffer parity is replayed
        for (; k + 2 <= n_steps; k += 2) {
            const int p = b->parity;
            if (!b->gexec[p] || b->gdt[p] != dt) {
                if (b->gexec[p]) cudaGraphExecDestroy(b->gexec[p]);
                b->gexec[p] = nullptr;
                cudaStream_t cs;
                BCK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "capture stream");
                cudaGraph_t graph;
                BCK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal), "begin capture");
                DevState saved = b->d;
                md_status ms = batch_one_step(b, dt, cs);
                if (ms == MD_OK) ms = batch_one_step(b, dt, cs);
                cudaError_t ec = cudaStreamEndCapture(cs, &graph);
                b->d = saved;  // the capture only recorded; the state has not moved
                cudaStreamDestroy(cs);
                if (ms != MD_OK) return ms;
                BCK(ec, "end capture");
                cudaError_t ei = cudaGraphInstantiate(&b->gexec[p], graph, 0);
                cudaGraphDestroy(graph);
                BCK(ei, "graph instantiate");
                b->gdt[p] = dt;
            }
            BCK(cudaGraphLaunch(b->gexec[p], st), "graph launch");
            // two swaps: the buffer assignment is back where it started
        }
    }
    for (; k < n_steps; k++) {
        md_status ms = batch_one_step(b, dt, st);
        if (ms != MD_OK) return ms;
        b->parity ^= 1;
    }
    b->step += n_steps;
    b->time += n_steps * dt;
    b->dt_last = dt;
    b->forces_valid = true;
    // a replayed graph runs no host code: the flag is set here, not by batch_force
    b->f_in_acc = true;
    return MD_OK;
}

md_status md_batch_energy_virial(md_batch *b, md_observables *out, void *cuda_stream)
{
    if (!b || !out) return MD_ERR_ARG;
    if (!b->forces_valid) {
        bset_err(b, "md_batch_energy_virial: no force evaluation yet");
        return MD_ERR_STATE;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    DevState &d = b->d;
    md_status mf = batch_forces_to_f64(b, st);
    if (mf != MD_OK) return mf;
    k_rep_reduce<<<b->n_sys, 256, 0, st>>>(b->dgrids, b->n_sys, b->ncell, b->cellE, b->cellN,
                                            b->m.site_pairs_per_mol_pair, b->rep_obs);
    k_rep_kinetic<<<b->n_sys, 256, 0, st>>>(b->dgrids, b->n_sys, d.n, b->m, d, 0.5 * b->dt_last, b->rep_kin);
    BCK(cudaGetLastError(), "replica reductions");
    std::vector<double> ob(8 * b->n_sys), kn(2 * b->n_sys);
    int fl[4];
    BCK(cudaMemcpyAsync(ob.data(), b->rep_obs, ob.size() * sizeof(double), cudaMemcpyDeviceToHost, st), "copy obs");
    BCK(cudaMemcpyAsync(kn.data(), b->rep_kin, kn.size() * sizeof(double), cudaMemcpyDeviceToHost, st), "copy kin");
    BCK(cudaMemcpyAsync(fl, d.flags, sizeof fl, cudaMemcpyDeviceToHost, st), "copy flags");
    BCK(cudaStreamSynchronize(st), "md_batch_energy_virial sync");
    for (int k = 0; k < b->n_sys; k++) {
        md_observables &o = out[k];
        memset(&o, 0, sizeof o);
        const RepGrid &g = b->grids[k];
        const double N = (double)b->n_per[k], V = g.L[0] * g.L[1] * g.L[2];
        o.U_pot = ob[8 * k + P_U];
        o.W = ob[8 * k + P_W];
        o.W_xx = ob[8 * k + P_WXX];
        o.W_yy = ob[8 * k + P_WYY];
        o.W_zz = ob[8 * k + P_WZZ];
        o.n_mol_pairs = (int64_t)llround(ob[8 * k + P_NMOL]);
        o.n_site_pairs = (int64_t)llround(ob[8 * k + P_NSITE]);
        o.n_examined = (int64_t)llround(ob[8 * k + P_NEXAM]);
        o.U_lrc = b->opt.lj_lrc ? b->lrc_u * N * N / V : 0.0;
        o.W_lrc = b->opt.lj_lrc ? b->lrc_w * N * N / V : 0.0;
        o.U_rf_self = b->rf_self * N;
        o.K_trans = kn[2 * k];
        o.K_rot = kn[2 * k + 1];
        const double dof = 3.0 * N - 3.0 + (double)b->m.rot_dof * N;
        o.T = dof > 0 ? 2.0 * (o.K_trans + o.K_rot) / dof : 0.0;
        o.P = (2.0 * o.K_trans + o.W + o.W_lrc) / (3.0 * V);
        o.time = b->time;
        o.step = b->step;
        o.n_molecules = b->n_per[k];
    }
    if (fl[FLAG_NONFINITE]) {
        bset_err(b, "non-finite force, torque or position detected on the device");
        return MD_ERR_NONFINITE;
    }
    return MD_OK;
}

md_status md_batch_get_molecules(md_batch *b, double *r, double *v, double *q, double *j, int32_t on_device,
                                 void *cuda_stream)
{
    if (!b) return MD_ERR_ARG;
    if (!b->has_mol) return MD_ERR_STATE;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    DevState &d = b->d;
    const double *src[4] = {d.r, d.v, d.q, d.j};
    double *dst[4] = {r, v, q, j}, *tmp[4] = {d.r2, d.v2, d.q2, d.j2};
    const int w[4] = {3, 3, 4, 3};
    for (int k = 0; k < 4; k++) {
        if (!dst[k] || d.n == 0) continue;
        BCK(launch_scatter_out(d, src[k], w[k], on_device ? dst[k] : tmp[k], st), "scatter kernel");
        if (!on_device)
            BCK(cudaMemcpyAsync(dst[k], tmp[k], sizeof(double) * w[k] * (size_t)d.n, cudaMemcpyDeviceToHost, st),
                "copy to host");
    }
    BCK(cudaStreamSynchronize(st), "md_batch_get_molecules sync");
    return MD_OK;
}

md_status md_batch_get_forces(md_batch *b, double *F, double *tau, int32_t on_device, void *cuda_stream)
{
    if (!b) return MD_ERR_ARG;
    if (!b->forces_valid) return MD_ERR_STATE;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    md_status mf = batch_forces_to_f64(b, st);
    if (mf != MD_OK) return mf;
    DevState &d = b->d;
    const double *src[2] = {d.F, d.tau};
    double *dst[2] = {F, tau}, *tmp[2] = {d.r2, d.v2};
    for (int k = 0; k < 2; k++) {
        if (!dst[k] || d.n == 0) continue;
        BCK(launch_scatter_out(d, src[k], 3, on_device ? dst[k] : tmp[k], st), "scatter kernel");
        if (!on_device)
            BCK(cudaMemcpyAsync(dst[k], tmp[k], sizeof(double) * 3 * (size_t)d.n, cudaMemcpyDeviceToHost, st),
                "copy to host");
    }
    BCK(cudaStreamSynchronize(st), "md_batch_get_forces sync");
    return MD_OK;
}

// Times the batched force evaluation for each (work-chunk size, grid
// occupancy) candidate with CUDA events and keeps the fastest.
md_status md_batch_set_thermostat(md_batch *b, const double *T_target, void *cuda_stream)
{
    if (!b) return MD_ERR_ARG;
    std::vector<double> t(b->n_sys, 0.0);
    bool any = false;
    if (T_target)
        for (int k = 0; k < b->n_sys; k++) {
            if (!std::isfinite(T_target[k])) {
                bset_err(b, "md_batch_set_thermostat: non-finite target temperature");
                return MD_ERR_ARG;
            }
            t[k] = T_target[k] > 0.0 ? T_target[k] : 0.0;
            any = any || t[k] > 0.0;
        }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    BCK(cudaMemcpyAsync(b->rep_T, t.data(), sizeof(double) * b->n_sys, cudaMemcpyHostToDevice, st), "copy targets");
    BCK(cudaStreamSynchronize(st), "md_batch_set_thermostat sync");
    if (any != b->nvt) drop_graphs(b);  // the captured step differs with and without the thermostat
    b->nvt = any;
    return MD_OK;
}

// Key of the tuning cache: GPU name | site signature (roles and LJ types of
// the merged sites) | occupancy bucket (half-octaves of the mean molecules
// per cell over all replicas).
static void tune_key(md_batch *b, char *key, size_t cap)
{
    cudaDeviceProp p;
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) snprintf(p.name, sizeof p.name, "unknown");
    unsigned sig = 0, ty = 0;
    for (int a = 0; a < b->m.S && a < 8; a++) {
        sig |= (unsigned)b->m.roles[a] << (4 * a);
        ty |= (unsigned)(b->m.roles[a] & ROLE_LJ ? b->m.lj_type[a] : 0) << (4 * a);
    }
    const double occ = b->ncell > 0 ? (double)b->ntot / (double)b->ncell : 0.0;
    const int bucket = occ > 0.0 ? (int)std::floor(2.0 * std::log2(occ)) : -99;
    snprintf(key, cap, "%s|%08x.%08x|occ%d", p.name, sig, ty, bucket);
    for (char *c = key; *c; c++)
        if (*c == ' ') *c = '_';
}

static bool tune_cache_find(const char *path, const char *key, md_batch_tuning *t)
{
    if (!path) return false;
    FILE *f = fopen(path, "r");
    if (!f) return false;
    char k[256];
    int chunk, grid, nt;
    double occ;
    float ms;
    bool found = false;
    while (fscanf(f, "%255s %d %d %d %lf %f", k, &chunk, &grid, &nt, &occ, &ms) == 6) {
        if (strcmp(k, key) == 0 && chunk >= 1 && chunk <= 64 && (grid == 100 || grid == 50) &&
            (nt == 4 || nt == NTEST) && occ >= 0.0) {
            t->chunk = chunk;
            t->grid_pct = grid;
            t->test_width = nt;
            t->half_min_occ = occ;
            t->ms = ms;
            found = true;
        }
    }
    fclose(f);
    return found;
}

static void tune_cache_store(const char *path, const char *key, const md_batch_tuning *t)
{
    if (!path) return;
    std::vector<std::string> keep;
    if (FILE *f = fopen(path, "r")) {
        char line[512];
        while (fgets(line, sizeof line, f)) {
            char k[256];
            if (sscanf(line, "%255s", k) == 1 && strcmp(k, key) != 0) keep.push_back(line);
        }
        fclose(f);
    }
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = fopen(tmp.c_str(), "w");
    if (!f) return;
    for (const std::string &l : keep) fputs(l.c_str(), f);
    fprintf(f, "%s %d %d %d %.6g %.6g\n", key, t->chunk, t->grid_pct, t->test_width, t->half_min_occ, t->ms);
    fclose(f);
    rename(tmp.c_str(), path);
}

// Mean of 3 batched force evaluations with the current tiles (after one
// untimed one), in ms.
static md_status time_forces(md_batch *b, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, float *ms)
{
    md_status r = batch_force(b, st);
    if (r != MD_OK) return r;
    cudaEventRecord(e0, st);
    for (int rep = 0; rep < 3 && r == MD_OK; rep++) r = batch_force(b, st);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    *ms = t / 3.f;
    return r;
}

md_status md_batch_tune_tiles(md_batch *b, void *cuda_stream, const char *cache_path, md_batch_tuning *out)
{
    if (!b || !out) return MD_ERR_ARG;
    if (!b->has_mol) return MD_ERR_STATE;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    md_batch_tuning t;
    memset(&t, 0, sizeof t);
    tune_key(b, t.key, sizeof t.key);
    cudaEvent_t e0, e1;
    BCK(cudaEventCreate(&e0), "event");
    BCK(cudaEventCreate(&e1), "event");
    auto apply = [&](int chunk, int grid, int nt, double occ) -> md_status {
        b->chunk = chunk;
        b->grid_frac_pct = grid;
        b->test_width = nt;
        if (occ != b->half_min_occ) {
            b->half_min_occ = occ;
            return apply_shell_policy(b, st);
        }
        return MD_OK;
    };
    // the defaults, timed for the comparison
    md_status ms = apply(2, 100, NTEST, 0.0);
    if (ms == MD_OK) ms = time_forces(b, st, e0, e1, &t.default_ms);
    md_batch_tuning cached = t;
    if (ms == MD_OK && tune_cache_find(cache_path, t.key, &cached)) {
        t = cached;
        t.from_cache = 1;
        ms = apply(t.chunk, t.grid_pct, t.test_width, t.half_min_occ);
    } else if (ms == MD_OK) {
        const int chunks[] = {1, 2, 4, 8};
        const int grids[] = {100, 50};
        const int widths[] = {4, NTEST};
        const double occs[] = {0.0, 2.0, 6.0};
        float best = 1e30f;
        for (double occ : occs)
            for (int nt : widths)
                for (int grid : grids)
                    for (int chunk : chunks) {
                        if (ms != MD_OK) break;
                        float tm = 0.f;
                        ms = apply(chunk, grid, nt, occ);
                        if (ms == MD_OK) ms = time_forces(b, st, e0, e1, &tm);
                        if (ms == MD_OK && tm < best) {
                            best = tm;
                            t.chunk = chunk;
                            t.grid_pct = grid;
                            t.test_width = nt;
                            t.half_min_occ = occ;
                            t.ms = tm;
                        }
                    }
        if (ms == MD_OK) ms = apply(t.chunk, t.grid_pct, t.test_width, t.half_min_occ);
        if (ms == MD_OK) tune_cache_store(cache_path, t.key, &t);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    drop_graphs(b);
    b->forces_valid = false;
    *out = t;
    return ms;
}

md_status md_batch_tune(md_batch *b, void *cuda_stream, int32_t *best_chunk, int32_t *best_grid_pct, float *best_ms)
{
    md_batch_tuning t;
    md_status ms = md_batch_tune_tiles(b, cuda_stream, nullptr, &t);
    if (ms != MD_OK) return ms;
    if (best_chunk) *best_chunk = t.chunk;
    if (best_grid_pct) *best_grid_pct = t.grid_pct;
    if (best_ms) *best_ms = t.ms;
    return MD_OK;
}

}  // extern "C"
