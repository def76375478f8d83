// md_leapfrog.cuh -- one molecule's leapfrog step (§3: Eqs. 2-3
// translational, Eqs. 4-5 rotational read as Fincham's quaternion
// leapfrog), shared by the single-system and the batched integrators.
//
// Precision split (GB300's FP64 pipe is a small fraction of its FP32 rate):
// the state r, v, q, j and every update of it are FP64 (Eqs. 2-5 as
// written); the rotational increment q_dot (from w = I^-1 A(q) j, the
// half-step quaternion and its renormalisation) is formed in FP32 from the
// rounded state, so its relative error (~1e-7) enters q only through the
// dt-scaled update.  The FP32 <-> FP64 conversions and the cell floor run
// as integer bit operations (md_fpconv.cuh, the same bits as the hardware
// conversions), which keeps them off the FP64 pipe that bounds this step.  The final renormalisation of q uses the series
// (1 + e)^(-1/2) = 1 - e/2 + 3e^2/8 - 5e^3/16 with e = |q|^2 - 1 where it
// is exact to FP64 rounding (|e| < 1e-4, the usual case), 1/sqrt(1 + e)
// otherwise.  No FP64 division is left per molecule: dt/m and 1/ell come
// from the host.
#pragma once

#include "md_fpconv.cuh"
#include "md_internal.cuh"

namespace mdk {

// Per-launch constants of one step.
struct LeapArgs {
    double dt, dtm;  // dt and dt / m
    float hdt;       // dt / 2
    float Iinv[3];   // principal inverse moments
};

inline LeapArgs leap_args(const DevModel &m, double dt)
{
    LeapArgs a;
    a.dt = dt;
    a.dtm = dt / m.mass;
    a.hdt = (float)(0.5 * dt);
    for (int k = 0; k < 3; k++) a.Iinv[k] = (float)m.Iinv[k];
    return a;
}

// Cell coordinate along one axis, floor(x / ell), from the reciprocal edge.
// x * (1/ell) is within a few ulp of x / ell; cell edges are at least
// rc (1 + 1e-9), so a molecule that rounding moves across a face lands in a
// cell from which every partner closer than rc is still in the stencil.
// The floor is taken on the integer pipe (floor_bits).
__device__ __forceinline__ int cell_coord(double x, double iell, int nc)
{
    const int c = floor_bits(x * iell);
    return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

// w_body = I^-1 A(q) j with A = R(q)^T (space -> body), FP32.
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

// q_dot = 1/2 q (x) (0, w), FP32.
__device__ __forceinline__ void quat_rate_f(const float q[4], const float w[3], float qd[4])
{
    qd[0] = 0.5f * (-q[1] * w[0] - q[2] * w[1] - q[3] * w[2]);
    qd[1] = 0.5f * (q[0] * w[0] + q[2] * w[2] - q[3] * w[1]);
    qd[2] = 0.5f * (q[0] * w[1] + q[3] * w[0] - q[1] * w[2]);
    qd[3] = 0.5f * (q[0] * w[2] + q[1] * w[1] - q[2] * w[0]);
}

// Twice the rotational kinetic energy of one molecule, w.I w with
// w = I^-1 A(q) j, in FP32 from the FP64 q and j (every kinetic-energy
// kernel uses this one expression, so their per-molecule values agree).
__device__ __forceinline__ float kin_rot2(const double *q, const double (&j)[3], const float (&Iinv)[3],
                                          const float (&Im)[3])
{
    const float qf[4] = {d2f_bits(q[0]), d2f_bits(q[1]), d2f_bits(q[2]), d2f_bits(q[3])};
    const float jf[3] = {d2f_bits(j[0]), d2f_bits(j[1]), d2f_bits(j[2])};
    float w[3];
    omega_body_f(qf, jf, Iinv, w);
    return Im[0] * w[0] * w[0] + Im[1] * w[1] * w[1] + Im[2] * w[2] * w[2];
}

// One step of molecule s in place; cc receives its cell coordinates after
// the periodic wrap.  ACC32: the forces and torques are read from the FP32
// accumulator records (F, 0, tau, 0 per molecule), otherwise from the FP64
// arrays.
// Returns true if a non-finite value appeared.
template <bool ACC32>
__device__ __forceinline__ bool leapfrog_one(const DevModel &m, const DevState &d, long long s, const LeapArgs &a,
                                             const double (&L)[3], const double (&iell)[3], const int (&nc)[3],
                                             int (&cc)[3])
{
    bool bad = false;
    float4 fa = make_float4(0.f, 0.f, 0.f, 0.f), ta = fa;
    if (ACC32) {
        fa = reinterpret_cast<const float4 *>(d.facc)[2 * s];
        ta = reinterpret_cast<const float4 *>(d.facc)[2 * s + 1];
    }
    const float fav[3] = {fa.x, fa.y, fa.z}, tav[3] = {ta.x, ta.y, ta.z};
    for (int k = 0; k < 3; k++) {
        const double F = ACC32 ? f2d_bits(fav[k]) : d.F[3 * s + k];
        const double v = d.v[3 * s + k] + a.dtm * F;  // Eq. 2
        double r = d.r[3 * s + k] + a.dt * v;         // Eq. 3
        // 0 <= r < L as one unsigned compare of the bit patterns (IEEE order
        // of non-negative doubles; negative values and NaN compare above)
        if ((unsigned long long)__double_as_longlong(r) >= (unsigned long long)__double_as_longlong(L[k])) {
            bad |= !isfinite(r);  // crossed a face (rare): periodic wrap
            r -= L[k] * floor(r / L[k]);
            if (r >= L[k]) r -= L[k];
            if (r < 0.0) r = 0.0;
        }
        d.v[3 * s + k] = v;
        d.r[3 * s + k] = r;
        cc[k] = cell_coord(r, iell[k], nc[k]);
    }
    if (m.rot_dof > 0) {
        double q[4] = {d.q[4 * s], d.q[4 * s + 1], d.q[4 * s + 2], d.q[4 * s + 3]};
        double j[3], t[3];
        float qf[4], tf[3], jh[3], jt[3], w[3], qd[4], qh[4];
        for (int k = 0; k < 4; k++) qf[k] = d2f_bits(q[k]);
        for (int k = 0; k < 3; k++) {
            if (ACC32) {
                tf[k] = tav[k];
                t[k] = f2d_bits(tf[k]);
            } else {
                t[k] = d.tau[3 * s + k];
                tf[k] = (float)t[k];
            }
            j[k] = d.j[3 * s + k] + a.dt * t[k];  // Eq. 4: j(t + dt/2), FP64
            jh[k] = d2f_bits(j[k]);
            jt[k] = jh[k] - a.hdt * tf[k];  // j(t)
        }
        omega_body_f(qf, jt, a.Iinv, w);
        quat_rate_f(qf, w, qd);
        for (int k = 0; k < 4; k++) qh[k] = qf[k] + a.hdt * qd[k];  // q(t + dt/2)
        const float nh = rsqrtf(qh[0] * qh[0] + qh[1] * qh[1] + qh[2] * qh[2] + qh[3] * qh[3]);
        for (int k = 0; k < 4; k++) qh[k] *= nh;
        omega_body_f(qh, jh, a.Iinv, w);
        quat_rate_f(qh, w, qd);
        for (int k = 0; k < 4; k++) q[k] += a.dt * f2d_bits(qd[k]);  // Eq. 5: q(t + dt)
        const double e = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3] - 1.0;
        // (1 + e)^(-1/2): the cubic series is exact to FP64 rounding for |e| < 1e-4
        const double inv = fabs(e) < 1e-4 ? 1.0 + e * (-0.5 + e * (0.375 - 0.3125 * e)) : 1.0 / sqrt(1.0 + e);
        for (int k = 0; k < 4; k++) d.q[4 * s + k] = q[k] * inv;
        for (int k = 0; k < 3; k++) d.j[3 * s + k] = j[k];
        bad |= !isfinite(e);
    }
    return bad;
}

}  // namespace mdk
