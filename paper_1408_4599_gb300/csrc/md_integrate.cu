// md_integrate.cu -- leapfrog integrator (§3, Eqs. 2-3 translational,
// Eqs. 4-5 rotational read as Fincham's quaternion leapfrog), fused with
// the periodic wrap and the cell id + histogram of the next rebuild; the
// kinetic-energy reduction at integer time steps (FP64); velocity
// rescaling.  FP64 state; the precision split is described in
// md_leapfrog.cuh.
#include "md_leapfrog.cuh"

using namespace mdk;

namespace {

// One leapfrog step per molecule (storage order), then the cell id and
// histogram for the rebuild that follows.
template <bool ACC32>
__global__ void k_integrate(Grid g, DevModel m, DevState d, LeapArgs a)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= d.n) return;
    int cc[3];
    if (leapfrog_one<ACC32>(m, d, s, a, g.L, g.iell, g.nc, cc)) atomicExch(&d.flags[FLAG_NONFINITE], 1);
    const int c = (cc[2] * g.nc[1] + cc[1]) * g.nc[0] + cc[0];
    d.cell[s] = c;
    atomicAdd(&d.cell_count[c], 1);
}

// Kinetic energies at integer time: v(t) = v + dt/2 F/m, j(t) = j + dt/2 tau.
// K_trans in FP64; K_rot per molecule in FP32 (w = I^-1 A(q) j(t) from the
// rounded q and j(t), ~1e-7 relative) with FP64 sums.
// Block partials: [0] K_trans, [1] K_rot.
__global__ void k_kinetic(DevModel m, DevState d, double dt_half)
{
    __shared__ double sh[2][32];
    double kt = 0.0, kr = 0.0;
    const double im = 1.0 / m.mass;
    const float Iinv[3] = {(float)m.Iinv[0], (float)m.Iinv[1], (float)m.Iinv[2]};
    const float Im[3] = {(float)m.I[0], (float)m.I[1], (float)m.I[2]};
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < d.n; s += (long long)gridDim.x * blockDim.x) {
        double v2 = 0.0;
        for (int k = 0; k < 3; k++) {
            const double vk = d.v[3 * s + k] + dt_half * d.F[3 * s + k] * im;
            v2 += vk * vk;
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
        d.kin_partials[blockIdx.x * 4 + threadIdx.x] = t;
    }
}

// Velocity rescaling (§2: NVT by rescaling the velocities), step 1: the
// half-step kinetic energies K_trans = sum 1/2 m v^2 (FP64) and
// K_rot = sum 1/2 w.I w with w = I^-1 A(q) j from the rounded state (FP32
// per molecule, FP64 sums), v, j at t + dt/2 and q at t + dt.  Block
// partials in kin_partials[4b + 2], [4b + 3].
__global__ void k_kinetic_half(DevModel m, DevState d)
{
    __shared__ double sh[2][32];
    double kt = 0.0, kr = 0.0;
    const float Iinv[3] = {(float)m.Iinv[0], (float)m.Iinv[1], (float)m.Iinv[2]};
    const float Im[3] = {(float)m.I[0], (float)m.I[1], (float)m.I[2]};
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < d.n; s += (long long)gridDim.x * blockDim.x) {
        const double v0 = d.v[3 * s], v1 = d.v[3 * s + 1], v2 = d.v[3 * s + 2];
        kt += v0 * v0 + v1 * v1 + v2 * v2;
        if (m.rot_dof > 0) {
            const double jh[3] = {d.j[3 * s], d.j[3 * s + 1], d.j[3 * s + 2]};
            kr += (double)kin_rot2(d.q + 4 * s, jh, Iinv, Im);
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
        d.kin_partials[blockIdx.x * 4 + 2 + threadIdx.x] = 0.5 * (threadIdx.x == 0 ? m.mass : 1.0) * t;
    }
}

// Step 2 (one warp, fixed summation order): T_half = 2 (K_trans + K_rot) /
// dof and the factor sqrt(T_target / T_half) (1 if T_half is not positive).
__global__ void k_thermo_factor(DevState d, int n_blocks, double T_target, double dof)
{
    const int lane = threadIdx.x;
    double k = 0.0;
    for (int b = lane; b < n_blocks; b += 32) k += d.kin_partials[4 * b + 2] + d.kin_partials[4 * b + 3];
    for (int o = 16; o > 0; o >>= 1) k += __shfl_xor_sync(0xffffffffu, k, o);
    if (lane == 0) {
        const double T = 2.0 * k / dof;
        d.thermo[0] = (T > 0.0 && isfinite(T)) ? sqrt(T_target / T) : 1.0;
        d.thermo[1] = T;
    }
}

__global__ void k_rescale(DevState d, double fv, double fj)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * d.n) return;
    d.v[t] *= fv;
    d.j[t] *= fj;
}

}  // namespace

cudaError_t launch_integrate(const Grid &g, const DevModel &m, DevState &d, double dt, int acc32, cudaStream_t s,
                             int zero_count)
{
    cudaError_t e = zero_count ? cudaMemsetAsync(d.cell_count, 0, sizeof(int) * g.ncell, s) : cudaSuccess;
    if (e != cudaSuccess || d.n == 0) return e;
    const LeapArgs a = leap_args(m, dt);
    const unsigned nb = (unsigned)((d.n + 127) / 128);
    if (acc32) k_integrate<true><<<nb, 128, 0, s>>>(g, m, d, a);
    else k_integrate<false><<<nb, 128, 0, s>>>(g, m, d, a);
    return cudaGetLastError();
}

cudaError_t launch_kinetic(const DevModel &m, DevState &d, double dt_half, int n_blocks, cudaStream_t s)
{
    k_kinetic<<<n_blocks, 256, 0, s>>>(m, d, dt_half);
    return cudaGetLastError();
}

cudaError_t launch_thermostat(const DevModel &m, DevState &d, int n_blocks, double T_target, double dof, cudaStream_t s)
{
    k_kinetic_half<<<n_blocks, 256, 0, s>>>(m, d);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_thermo_factor<<<1, 32, 0, s>>>(d, n_blocks, T_target, dof);
    return cudaGetLastError();
}

cudaError_t launch_rescale(const DevModel &m, DevState &d, double fv, double fj, cudaStream_t s)
{
    (void)m;
    if (d.n == 0) return cudaSuccess;
    k_rescale<<<(unsigned)((3 * d.n + 255) / 256), 256, 0, s>>>(d, fv, fj);
    return cudaGetLastError();
}
