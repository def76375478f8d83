// md_integrate.cu -- leapfrog integrator (§3, Eqs. 2-3 translational,
// Eqs. 4-5 rotational read as Fincham's quaternion leapfrog), fused with
// the periodic wrap and the cell id + histogram of the next rebuild; the
// kinetic-energy reduction at integer time steps (FP64); velocity
// rescaling.  FP64 state; see k_integrate for the precision split.
#include "md_internal.cuh"

namespace {

__device__ __forceinline__ int cell_axis(double x, double ell, int nc)
{
    int c = (int)floor(x / ell);
    return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

// w_body = I^-1 A(q) j, A = R(q)^T (space -> body)
__device__ __forceinline__ void omega_body(const double q[4], const double j[3], const double Iinv[3], double w[3])
{
    const double qw = q[0], qx = q[1], qy = q[2], qz = q[3];
    const double R00 = 1 - 2 * (qy * qy + qz * qz), R01 = 2 * (qx * qy - qw * qz), R02 = 2 * (qx * qz + qw * qy);
    const double R10 = 2 * (qx * qy + qw * qz), R11 = 1 - 2 * (qx * qx + qz * qz), R12 = 2 * (qy * qz - qw * qx);
    const double R20 = 2 * (qx * qz - qw * qy), R21 = 2 * (qy * qz + qw * qx), R22 = 1 - 2 * (qx * qx + qy * qy);
    w[0] = Iinv[0] * (R00 * j[0] + R10 * j[1] + R20 * j[2]);
    w[1] = Iinv[1] * (R01 * j[0] + R11 * j[1] + R21 * j[2]);
    w[2] = Iinv[2] * (R02 * j[0] + R12 * j[1] + R22 * j[2]);
}

// q_dot = 1/2 q (x) (0, w)
__device__ __forceinline__ void quat_rate(const double q[4], const double w[3], double qd[4])
{
    qd[0] = 0.5 * (-q[1] * w[0] - q[2] * w[1] - q[3] * w[2]);
    qd[1] = 0.5 * (q[0] * w[0] + q[2] * w[2] - q[3] * w[1]);
    qd[2] = 0.5 * (q[0] * w[1] + q[3] * w[0] - q[1] * w[2]);
    qd[3] = 0.5 * (q[0] * w[2] + q[1] * w[1] - q[2] * w[0]);
}

__device__ __forceinline__ void normalise4(double q[4])
{
    const double inv = rsqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    q[0] *= inv;
    q[1] *= inv;
    q[2] *= inv;
    q[3] *= inv;
}

// FP32 helpers for the rotational increments.
__device__ __forceinline__ void omega_body_f(const float q[4], const float j[3], const float Iinv[3], float w[3])
{
    const float qw = q[0], qx = q[1], qy = q[2], qz = q[3];
    const float R00 = 1.f - 2.f * (qy * qy + qz * qz), R01 = 2.f * (qx * qy - qw * qz), R02 = 2.f * (qx * qz + qw * qy);
    const float R10 = 2.f * (qx * qy + qw * qz), R11 = 1.f - 2.f * (qx * qx + qz * qz), R12 = 2.f * (qy * qz - qw * qx);
    const float R20 = 2.f * (qx * qz - qw * qy), R21 = 2.f * (qy * qz + qw * qx), R22 = 1.f - 2.f * (qx * qx + qy * qy);
    w[0] = Iinv[0] * (R00 * j[0] + R10 * j[1] + R20 * j[2]);
    w[1] = Iinv[1] * (R01 * j[0] + R11 * j[1] + R21 * j[2]);
    w[2] = Iinv[2] * (R02 * j[0] + R12 * j[1] + R22 * j[2]);
}

__device__ __forceinline__ void quat_rate_f(const float q[4], const float w[3], float qd[4])
{
    qd[0] = 0.5f * (-q[1] * w[0] - q[2] * w[1] - q[3] * w[2]);
    qd[1] = 0.5f * (q[0] * w[0] + q[2] * w[2] - q[3] * w[1]);
    qd[2] = 0.5f * (q[0] * w[1] + q[3] * w[0] - q[1] * w[2]);
    qd[3] = 0.5f * (q[0] * w[2] + q[1] * w[1] - q[2] * w[0]);
}

// One leapfrog step per molecule (storage order), then wrap into [0, L),
// cell id and histogram for the rebuild that follows.
//
// Precision split (GB300's FP64 pipe is a small fraction of its FP32 rate):
// the state r, v, q, j and every update of it are FP64 (Eqs. 2-5 as
// written); the rotational increment q_dot (from w = I^-1 A(q) j, the
// half-step quaternion and its renormalisation) is formed in FP32 from the
// rounded state, so its relative error (~1e-7) enters q only through the
// dt-scaled update.  The final renormalisation of q uses the series
// (1 + e)^(-1/2) = 1 - e/2 + 3e^2/8 - 5e^3/16 with e = |q|^2 - 1 where it
// is exact to FP64 rounding (|e| < 1e-4, the usual case), 1/sqrt(1 + e)
// otherwise.
__global__ void k_integrate(Grid g, DevModel m, DevState d, double dt)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= d.n) return;
    const double dtm = dt / m.mass;
    int cc[3];
    bool bad = false;
    for (int k = 0; k < 3; k++) {
        const double v = d.v[3 * s + k] + dtm * d.F[3 * s + k];  // Eq. 2
        double r = d.r[3 * s + k] + dt * v;                        // Eq. 3
        bad |= !isfinite(r);
        if (r < 0.0) r += g.L[k];
        else if (r >= g.L[k]) r -= g.L[k];
        if (!(r >= 0.0 && r < g.L[k])) {  // moved more than a box length: general wrap
            r -= g.L[k] * floor(r / g.L[k]);
            if (r >= g.L[k]) r -= g.L[k];
            if (r < 0.0) r = 0.0;
        }
        d.v[3 * s + k] = v;
        d.r[3 * s + k] = r;
        cc[k] = cell_axis(r, g.ell[k], g.nc[k]);
    }
    if (m.rot_dof > 0) {
        double q[4] = {d.q[4 * s], d.q[4 * s + 1], d.q[4 * s + 2], d.q[4 * s + 3]};
        double j[3] = {d.j[3 * s], d.j[3 * s + 1], d.j[3 * s + 2]};
        const double t[3] = {d.tau[3 * s], d.tau[3 * s + 1], d.tau[3 * s + 2]};
        const float Iinv[3] = {(float)m.Iinv[0], (float)m.Iinv[1], (float)m.Iinv[2]};
        const float hdt = (float)(0.5 * dt);
        float qf[4] = {(float)q[0], (float)q[1], (float)q[2], (float)q[3]};
        float tf[3] = {(float)t[0], (float)t[1], (float)t[2]};
        float jt[3], w[3], qd[4], qh[4];
        for (int k = 0; k < 3; k++) jt[k] = (float)j[k] + hdt * tf[k];  // j(t)
        omega_body_f(qf, jt, Iinv, w);
        quat_rate_f(qf, w, qd);
        for (int k = 0; k < 4; k++) qh[k] = qf[k] + hdt * qd[k];  // q(t + dt/2)
        const float nh = rsqrtf(qh[0] * qh[0] + qh[1] * qh[1] + qh[2] * qh[2] + qh[3] * qh[3]);
        for (int k = 0; k < 4; k++) qh[k] *= nh;
        float jh[3];
        for (int k = 0; k < 3; k++) {
            j[k] += dt * t[k];  // Eq. 4: j(t + dt/2), FP64
            jh[k] = (float)j[k];
        }
        omega_body_f(qh, jh, Iinv, w);
        quat_rate_f(qh, w, qd);
        for (int k = 0; k < 4; k++) q[k] += dt * (double)qd[k];  // Eq. 5: q(t + dt)
        const double e = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3] - 1.0;
        // (1 + e)^(-1/2): the cubic series is exact to FP64 rounding for |e| < 1e-4
        const double inv = fabs(e) < 1e-4 ? 1.0 + e * (-0.5 + e * (0.375 - 0.3125 * e)) : 1.0 / sqrt(1.0 + e);
        for (int k = 0; k < 4; k++) d.q[4 * s + k] = q[k] * inv;
        for (int k = 0; k < 3; k++) d.j[3 * s + k] = j[k];
        bad |= !isfinite(e);
    }
    if (bad) atomicExch(&d.flags[FLAG_NONFINITE], 1);
    const int c = (cc[2] * g.nc[1] + cc[1]) * g.nc[0] + cc[0];
    d.cell[s] = c;
    atomicAdd(&d.cell_count[c], 1);
}

// Kinetic energies at integer time: v(t) = v + dt/2 F/m, j(t) = j + dt/2 tau.
// Block partials: [0] K_trans, [1] K_rot.
__global__ void k_kinetic(DevModel m, DevState d, double dt_half)
{
    __shared__ double sh[2][32];
    double kt = 0.0, kr = 0.0;
    const double im = 1.0 / m.mass;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < d.n; s += (long long)gridDim.x * blockDim.x) {
        double v2 = 0.0;
        for (int k = 0; k < 3; k++) {
            const double vk = d.v[3 * s + k] + dt_half * d.F[3 * s + k] * im;
            v2 += vk * vk;
        }
        kt += 0.5 * m.mass * v2;
        if (m.rot_dof > 0) {
            const double q[4] = {d.q[4 * s], d.q[4 * s + 1], d.q[4 * s + 2], d.q[4 * s + 3]};
            double jt[3], w[3];
            for (int k = 0; k < 3; k++) jt[k] = d.j[3 * s + k] + dt_half * d.tau[3 * s + k];
            omega_body(q, jt, m.Iinv, w);
            kr += 0.5 * (m.I[0] * w[0] * w[0] + m.I[1] * w[1] * w[1] + m.I[2] * w[2] * w[2]);
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

__global__ void k_rescale(DevState d, double fv, double fj)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * d.n) return;
    d.v[t] *= fv;
    d.j[t] *= fj;
}

}  // namespace

cudaError_t launch_integrate(const Grid &g, const DevModel &m, DevState &d, double dt, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(d.cell_count, 0, sizeof(int) * g.ncell, s);
    if (e != cudaSuccess || d.n == 0) return e;
    k_integrate<<<(unsigned)((d.n + 127) / 128), 128, 0, s>>>(g, m, d, dt);
    return cudaGetLastError();
}

cudaError_t launch_kinetic(const DevModel &m, DevState &d, double dt_half, int n_blocks, cudaStream_t s)
{
    k_kinetic<<<n_blocks, 256, 0, s>>>(m, d, dt_half);
    return cudaGetLastError();
}

cudaError_t launch_rescale(const DevModel &m, DevState &d, double fv, double fj, cudaStream_t s)
{
    (void)m;
    if (d.n == 0) return cudaSuccess;
    k_rescale<<<(unsigned)((3 * d.n + 255) / 256), 256, 0, s>>>(d, fv, fj);
    return cudaGetLastError();
}
