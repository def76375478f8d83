// md_pair.cuh -- site-site interaction laws (§2: LJ Eq. 1 with Lorentz-
// Berthelot mixing, point charges, dipoles, linear quadrupoles; §3 reaction
// field) and the linked-cell traversal (§3: 27-cell stencil, or the 14-cell
// Newton-3 half stencil) shared by the force, adjoint and batched kernels.
//
// Traversal (one warp per i-cell):
//   * the stencil cells' slots, counts and image offsets are loaded once
//     (one lane per cell) and their candidate molecules staged in shared
//     memory in windows of JCAP, image offset applied (FP32, i-cell frame);
//   * for each i molecule the lanes test NTEST x 32 candidates per round,
//     or NTEST/2 x 32 when the i's candidates fit (a warp-uniform choice per
//     i: single-site fluids stage ~130 candidates per cell, ~half a full
//     round) (FP32 centre-of-mass distance; a test within a narrow band of
//     r_c^2 is redone in FP64 from the FP64 state, so the pair set is the
//     FP64 definition's);
//   * hits are ballot-compacted into a per-warp queue shared by the i
//     molecules of a pass and handed to the pair operation 32 at a time, so
//     the expensive site-site math runs on packed lanes (only ~16% of the
//     examined pairs interact, §3); the lanes of one i in a chunk are
//     contiguous and their j's distinct.
#pragma once

#include <type_traits>

#include "md_internal.cuh"

namespace mdk {

constexpr int EL_ROLES = ROLE_CHG | ROLE_DIP | ROLE_QUAD;
constexpr int AX_ROLES = ROLE_DIP | ROLE_QUAD;
constexpr unsigned FULLMASK = 0xffffffffu;

__host__ __device__ constexpr int sig_role(unsigned R, int a) { return (int)((R >> (4 * a)) & 15u); }
__host__ __device__ constexpr int sig_slot(unsigned R, int a)
{
    int k = 0;
    for (int b = 0; b < a; b++) k += (sig_role(R, b) & AX_ROLES) ? 1 : 0;
    return (sig_role(R, a) & AX_ROLES) ? k : -1;
}
__host__ __device__ constexpr int sig_na(unsigned R, int S)
{
    int k = 0;
    for (int b = 0; b < S; b++) k += (sig_role(R, b) & AX_ROLES) ? 1 : 0;
    return k;
}
__host__ __device__ constexpr bool sig_has_role(unsigned R, int S, int role)
{
    for (int a = 0; a < S; a++)
        if (sig_role(R, a) & role) return true;
    return false;
}
__host__ __device__ constexpr unsigned sigkey(int r0, int r1 = 0, int r2 = 0, int r3 = 0, int r4 = 0, int r5 = 0,
                                              int r6 = 0, int r7 = 0)
{
    return (unsigned)r0 | ((unsigned)r1 << 4) | ((unsigned)r2 << 8) | ((unsigned)r3 << 12) | ((unsigned)r4 << 16) |
           ((unsigned)r5 << 20) | ((unsigned)r6 << 24) | ((unsigned)r7 << 28);
}

// Signatures compiled ahead of time; any other model runs SigDyn.
constexpr unsigned SIG_2CLJ = sigkey(ROLE_LJ, ROLE_LJ);
constexpr unsigned SIG_2CLJQ = sigkey(ROLE_LJ, ROLE_LJ, ROLE_QUAD);
constexpr unsigned SIG_2CLJDQ = sigkey(ROLE_LJ, ROLE_LJ, ROLE_DIP | ROLE_QUAD);
constexpr unsigned SIG_4SITE = sigkey(ROLE_LJ, ROLE_LJ | ROLE_CHG, ROLE_LJ | ROLE_CHG, ROLE_DIP, ROLE_QUAD);

// Compile-time site-role signature: S sites, 4 role bits per site, and the
// LJ type of each LJ site (4 bits per site), so that the mixing-table
// entries are compile-time constant-bank operands.  LIN: a linear molecule
// (DevModel::linear), whose packed geometry is its space-frame axis u alone;
// site a sits at body_z(a) u and its axis is axis_z(a) u.
template <int S_, unsigned R_, bool SINGLE_ = false, unsigned TY_ = 0, bool LIN_ = false, unsigned COM_ = 0>
struct SigStatic {
    static constexpr int S = S_;
    static constexpr unsigned ROLES = R_;  // 4 role bits per site
    static constexpr bool DYN = false;
    static constexpr bool SINGLE = SINGLE_;
    static constexpr bool LIN = LIN_;
    // bit a: site a sits at the centre of mass (linear signatures)
    __host__ __device__ static constexpr bool at_com(int a) { return ((COM_ >> a) & 1u) != 0; }
    static constexpr int K = LIN_ ? 1 : S_ + sig_na(R_, S_);
    __device__ __forceinline__ static constexpr int role(int a, const DevModel &) { return sig_role(R_, a); }
    __device__ __forceinline__ static constexpr int slot(int a, const DevModel &) { return sig_slot(R_, a); }
    __device__ __forceinline__ static constexpr int type(int a, const DevModel &) { return sig_role(TY_, a); }
    __device__ __forceinline__ static int kk(const DevModel &) { return K; }
    __device__ __forceinline__ static int s_of(const DevModel &) { return S_; }
};

// Run-time signature for any other model (up to MD_MAX_SITES sites).
struct SigDyn {
    static constexpr int S = MD_MAX_SITES;
    static constexpr unsigned ROLES = 0;  // roles known at run time only
    static constexpr bool DYN = true;
    static constexpr bool SINGLE = false;
    static constexpr bool LIN = false;
    __host__ __device__ static constexpr bool at_com(int) { return false; }
    __device__ __forceinline__ static int role(int a, const DevModel &m) { return a < m.S ? m.roles[a] : 0; }
    __device__ __forceinline__ static int slot(int a, const DevModel &m) { return m.axis_slot[a]; }
    __device__ __forceinline__ static int type(int a, const DevModel &m) { return m.lj_type[a]; }
    __device__ __forceinline__ static int kk(const DevModel &m) { return m.S + m.NA; }
    __device__ __forceinline__ static int s_of(const DevModel &m) { return m.S; }
};

constexpr unsigned TY_4SITE = sigkey(0, 1, 1);  // LJ types of the 4-site model's sites

// The compiled signatures by name.  The two-centre models are compiled for
// the linear geometry only, their multipole site at the centre of mass.
using Sig1CLJ = SigStatic<1, ROLE_LJ, true>;
using Sig2CLJ = SigStatic<2, SIG_2CLJ, false, 0, true>;
using Sig2CLJQ = SigStatic<3, SIG_2CLJQ, false, 0, true, 4u>;
using Sig2CLJDQ = SigStatic<3, SIG_2CLJDQ, false, 0, true, 4u>;
using Sig4Site = SigStatic<5, SIG_4SITE, false, TY_4SITE>;

// Dispatch of a model to its compiled signature: f.template operator()<SIG>().
template <class F>
__host__ auto dispatch_sig(const DevModel &m, F &&f)
{
    unsigned key = 0, ty = 0;
    for (int a = 0; a < m.S; a++) {
        key |= (unsigned)m.roles[a] << (4 * a);
        if (m.roles[a] & ROLE_LJ) ty |= (unsigned)m.lj_type[a] << (4 * a);
    }
    if (m.single_lj_at_com && ty == 0) return f.template operator()<Sig1CLJ>();
    if (m.linear && m.S == 2 && key == SIG_2CLJ && ty == 0) return f.template operator()<Sig2CLJ>();
    if (m.linear && m.S == 3 && key == SIG_2CLJQ && ty == 0 && m.body[2][2] == 0.f)
        return f.template operator()<Sig2CLJQ>();
    if (m.linear && m.S == 3 && key == SIG_2CLJDQ && ty == 0 && m.body[2][2] == 0.f)
        return f.template operator()<Sig2CLJDQ>();
    if (m.S == 5 && key == SIG_4SITE && ty == TY_4SITE) return f.template operator()<Sig4Site>();
    return f.template operator()<SigDyn>();
}

// Stencil of M cells per axis around a cell (§3: M = 1 for cells of edge
// >= r_c, the 27-cell stencil; M = 2 for cells of edge >= r_c / 2, the
// 125-cell stencil).  Full stencil index f = (dz+M) W^2 + (dy+M) W + dx+M,
// W = 2M+1.  The half (Newton-3) stencil is the cell itself (index 0) and
// the (W^3 - 1)/2 cells that follow it in (z, y, x) lexicographic order.
template <int M>
struct Stencil {
    static constexpr int W = 2 * M + 1;
    static constexpr int FULL = W * W * W;
    static constexpr int CENTRE = (FULL - 1) / 2;  // full index of the cell itself
    static constexpr int HALFN = CENTRE + 1;       // half stencil size
};

template <int M>
__device__ __forceinline__ void stencil_offset(bool half, int o, int &dx, int &dy, int &dz)
{
    using St = Stencil<M>;
    const int f = half ? St::CENTRE + o : o;  // half index o > 0 is full index CENTRE + o
    dx = f % St::W - M;
    dy = (f / St::W) % St::W - M;
    dz = f / (St::W * St::W) - M;
}

__device__ __forceinline__ int wrap_axis(int c, int d, int nc, int &k)
{
    int x = c + d;
    k = 0;
    if (x < 0) {
        x += nc;
        k = -1;
    } else if (x >= nc) {
        x -= nc;
        k = 1;
    }
    return x;
}

// One electrostatic role pair's unit-strength energy and its partials with
// respect to r (as n U: U is homogeneous of degree -n in r), pa = e_a.xh,
// pb = e_b.xh and cab = e_a.e_b (x = r_a - r_b, xh = x/r, k_C = 1):
//   q q: 1/r;  q mu: pb/r^2;  mu q: -pa/r^2;  mu mu: (cab - 3 pa pb)/r^3;
//   q Q: (3 pb^2 - 1)/(2 r^3);  Q q: (3 pa^2 - 1)/(2 r^3);
//   mu Q: 3/(2 r^4) [-pa (5 pb^2 - 1) + 2 pb cab];
//   Q mu: 3/(2 r^4) [pb (5 pa^2 - 1) - 2 pa cab];
//   Q Q: 3/(4 r^5) [1 - 5 pa^2 - 5 pb^2 - 15 pa^2 pb^2 + 2 (cab - 5 pa pb)^2];
//   reaction field (dipole pairs, §3): -f_RF cab / rc^3 (no r dependence).
struct Law {
    float U, nU, Upa, Upb, Ucab;
};

enum { LAW_QQ, LAW_QMU, LAW_MUQ, LAW_MUMU, LAW_QQUAD, LAW_QUADQ, LAW_MUQUAD, LAW_QUADMU, LAW_QUADQUAD };

template <int L>
__device__ __forceinline__ Law law(float ir, float pa, float pb, float cab, float frf)
{
    Law o{0.f, 0.f, 0.f, 0.f, 0.f};
    const float u2 = ir * ir, u3 = u2 * ir;
    if (L == LAW_QQ) {
        o.U = ir;
        o.nU = ir;
    } else if (L == LAW_QMU) {
        o.U = pb * u2;
        o.nU = 2.f * o.U;
        o.Upb = u2;
    } else if (L == LAW_MUQ) {
        o.U = -pa * u2;
        o.nU = 2.f * o.U;
        o.Upa = -u2;
    } else if (L == LAW_MUMU) {
        const float t = (cab - 3.f * pa * pb) * u3;
        o.U = t - frf * cab;
        o.nU = 3.f * t;
        o.Upa = -3.f * pb * u3;
        o.Upb = -3.f * pa * u3;
        o.Ucab = u3 - frf;
    } else if (L == LAW_QQUAD) {
        o.U = 0.5f * (3.f * pb * pb - 1.f) * u3;
        o.nU = 3.f * o.U;
        o.Upb = 3.f * pb * u3;
    } else if (L == LAW_QUADQ) {
        o.U = 0.5f * (3.f * pa * pa - 1.f) * u3;
        o.nU = 3.f * o.U;
        o.Upa = 3.f * pa * u3;
    } else if (L == LAW_MUQUAD) {
        const float c = 1.5f * u2 * u2;
        o.U = c * (2.f * pb * cab - pa * (5.f * pb * pb - 1.f));
        o.nU = 4.f * o.U;
        o.Upa = c * (1.f - 5.f * pb * pb);
        o.Upb = c * (2.f * cab - 10.f * pa * pb);
        o.Ucab = 2.f * c * pb;
    } else if (L == LAW_QUADMU) {
        const float c = 1.5f * u2 * u2;
        o.U = c * (pb * (5.f * pa * pa - 1.f) - 2.f * pa * cab);
        o.nU = 4.f * o.U;
        o.Upb = c * (5.f * pa * pa - 1.f);
        o.Upa = c * (10.f * pa * pb - 2.f * cab);
        o.Ucab = -2.f * c * pa;
    } else {
        const float c = 0.75f * u2 * u3;
        const float pa2 = pa * pa, pb2 = pb * pb;
        const float tt = cab - 5.f * pa * pb;
        o.U = c * (1.f - 5.f * (pa2 + pb2) - 15.f * pa2 * pb2 + 2.f * tt * tt);
        o.nU = 5.f * o.U;
        o.Upa = -c * (10.f * pa + 30.f * pa * pb2 + 20.f * pb * tt);
        o.Upb = -c * (10.f * pb + 30.f * pa2 * pb + 20.f * pa * tt);
        o.Ucab = 4.f * c * tt;
    }
    return o;
}

__device__ __forceinline__ void law_acc(Law &t, const Law &l, float s)
{
    t.U += s * l.U;
    t.nU += s * l.nU;
    t.Upa += s * l.Upa;
    t.Upb += s * l.Upb;
    t.Ucab += s * l.Ucab;
}

// Electrostatic interaction of site a (on i) with site b (on j) with the
// strengths applied: energy, force on a, orientation torques e x (-dU/de).
template <bool JSIDE>
__device__ __forceinline__ void elec_site(const int ra, const int rb, const float qa, const float mua, const float Qa,
                                          const float qb, const float mub, const float Qb, const float frf,
                                          const float x, const float y, const float z, const float ir,
                                          const float4 &ea, const float4 &eb, float &U, float &fx, float &fy,
                                          float &fz, float (&ti)[3], float (&tj)[3])
{
    const float xh = x * ir, yh = y * ir, zh = z * ir;
    const bool axa = (ra & AX_ROLES) != 0, axb = (rb & AX_ROLES) != 0;
    const float pa = axa ? (ea.x * xh + ea.y * yh + ea.z * zh) : 0.f;
    const float pb = axb ? (eb.x * xh + eb.y * yh + eb.z * zh) : 0.f;
    const float cab = (axa && axb) ? (ea.x * eb.x + ea.y * eb.y + ea.z * eb.z) : 0.f;
    Law t{0.f, 0.f, 0.f, 0.f, 0.f};
    if ((ra & ROLE_CHG) && (rb & ROLE_CHG)) law_acc(t, law<LAW_QQ>(ir, pa, pb, cab, 0.f), qa * qb);
    if ((ra & ROLE_CHG) && (rb & ROLE_DIP)) law_acc(t, law<LAW_QMU>(ir, pa, pb, cab, 0.f), qa * mub);
    if ((ra & ROLE_DIP) && (rb & ROLE_CHG)) law_acc(t, law<LAW_MUQ>(ir, pa, pb, cab, 0.f), mua * qb);
    if ((ra & ROLE_DIP) && (rb & ROLE_DIP)) law_acc(t, law<LAW_MUMU>(ir, pa, pb, cab, frf), mua * mub);
    if ((ra & ROLE_CHG) && (rb & ROLE_QUAD)) law_acc(t, law<LAW_QQUAD>(ir, pa, pb, cab, 0.f), qa * Qb);
    if ((ra & ROLE_QUAD) && (rb & ROLE_CHG)) law_acc(t, law<LAW_QUADQ>(ir, pa, pb, cab, 0.f), Qa * qb);
    if ((ra & ROLE_DIP) && (rb & ROLE_QUAD)) law_acc(t, law<LAW_MUQUAD>(ir, pa, pb, cab, 0.f), mua * Qb);
    if ((ra & ROLE_QUAD) && (rb & ROLE_DIP)) law_acc(t, law<LAW_QUADMU>(ir, pa, pb, cab, 0.f), Qa * mub);
    if ((ra & ROLE_QUAD) && (rb & ROLE_QUAD)) law_acc(t, law<LAW_QUADQUAD>(ir, pa, pb, cab, 0.f), Qa * Qb);
    U += t.U;
    // dU/dx = xh (Ur - (Upa pa + Upb pb)/r) + (Upa e_a + Upb e_b)/r, Ur = -nU/r
    const float cx = -(t.nU + t.Upa * pa + t.Upb * pb) * ir;
    const float ua = t.Upa * ir, ub = t.Upb * ir;
    fx -= cx * xh + ua * ea.x + ub * eb.x;
    fy -= cx * yh + ua * ea.y + ub * eb.y;
    fz -= cx * zh + ua * ea.z + ub * eb.z;
    float cex = 0.f, cey = 0.f, cez = 0.f;
    if (axa && axb) {
        cex = ea.y * eb.z - ea.z * eb.y;
        cey = ea.z * eb.x - ea.x * eb.z;
        cez = ea.x * eb.y - ea.y * eb.x;
    }
    if (axa) {  // e_a x (-(Upa xh + Ucab e_b))
        ti[0] -= t.Upa * (ea.y * zh - ea.z * yh) + t.Ucab * cex;
        ti[1] -= t.Upa * (ea.z * xh - ea.x * zh) + t.Ucab * cey;
        ti[2] -= t.Upa * (ea.x * yh - ea.y * xh) + t.Ucab * cez;
    }
    if (JSIDE && axb) {  // e_b x (-(Upb xh + Ucab e_a))
        tj[0] += -t.Upb * (eb.y * zh - eb.z * yh) + t.Ucab * cex;
        tj[1] += -t.Upb * (eb.z * xh - eb.x * zh) + t.Ucab * cey;
        tj[2] += -t.Upb * (eb.x * yh - eb.y * xh) + t.Ucab * cez;
    }
}

// The i molecule of the current traversal step, in registers.  Linear
// molecules keep only their axis u (site offsets z_a u and axes +-u are
// formed per pair), so that an i held across many pairs costs few registers.
template <class SIG, bool LIN = SIG::LIN>
struct IMol {
    float4 c;                 // centre of mass (cell-centre frame)
    float d[SIG::S][3];       // space-frame site offsets
    float4 e[SIG::S];         // space-frame axes
    float4 e_axis;            // unused
    int slot;
};
template <class SIG>
struct IMol<SIG, true> {
    float4 c;                 // centre of mass (cell-centre frame)
    float4 e_axis;            // the molecular axis u
    int slot;
};

template <class SIG>
__device__ __forceinline__ void load_i(const DevModel &m, const float4 *com, const float4 *geo, int K, int si,
                                       IMol<SIG> &I)
{
    I.slot = si;
    I.c = com[si];
    if constexpr (SIG::LIN) {
        I.e_axis = geo[(long long)si * K];
    } else {
#pragma unroll
        for (int a = 0; a < SIG::S; a++) {
            I.d[a][0] = I.d[a][1] = I.d[a][2] = 0.f;
            I.e[a] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (!SIG::SINGLE && SIG::role(a, m)) {
                const float4 t4 = geo[(long long)si * K + a];
                I.d[a][0] = t4.x;
                I.d[a][1] = t4.y;
                I.d[a][2] = t4.z;
                if (SIG::role(a, m) & AX_ROLES) I.e[a] = geo[(long long)si * K + SIG::s_of(m) + SIG::slot(a, m)];
            }
        }
    }
}

// Paired FP32 arithmetic of sm_100-class GPUs (fma/mul/add.rn.f32x2): two
// independent FP32 operations per instruction on a register pair, the same
// FMA throughput in half the issue slots.
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

// Linear two-centre models whose sites 0 and 1 are plain LJ centres of one
// type (2CLJ, 2CLJQ, 2CLJDQ): their four LJ site pairs are evaluated as two
// f32x2 pairs, P0 = (a0 b0, a1 b1) and P1 = (a0 b1, a1 b0), the low half
// always on i's site 0 and the high half on i's site 1.
template <class SIG>
__host__ __device__ constexpr bool lin_lj2()
{
    return SIG::LIN && !SIG::DYN && SIG::S >= 2 && sig_role(SIG::ROLES, 0) == ROLE_LJ &&
           sig_role(SIG::ROLES, 1) == ROLE_LJ;
}

// Eq. 1 on two site pairs at once: x, y, z hold the two site-site vectors
// (i site minus j site); the force on the i sites is added to fx, fy, fz and
// the unshifted energy to U.
__device__ __forceinline__ void lj_pair2(const float2 x, const float2 y, const float2 z, const float2 sig2,
                                         const float2 eps4, const float2 eps24, float2 &fx, float2 &fy, float2 &fz,
                                         float2 &U)
{
    const float2 r2 = fma2(z, z, fma2(y, y, mul2(x, x)));
    const float2 ir2 = f2(__fdividef(1.f, r2.x), __fdividef(1.f, r2.y));
    const float2 s2 = mul2(sig2, ir2);
    const float2 s6 = mul2(mul2(s2, s2), s2);
    const float2 fr = mul2(mul2(mul2(eps24, s6), fma2(s6, f2(2.f, 2.f), f2(-1.f, -1.f))), ir2);
    U = fma2(eps4, fma2(s6, s6, f2(-s6.x, -s6.y)), U);
    fx = fma2(fr, x, fx);
    fy = fma2(fr, y, fy);
    fz = fma2(fr, z, fz);
}

// Site a of the i molecule: space-frame offset d and axis e (zero unless
// the site carries an axis).
template <class SIG>
__device__ __forceinline__ void imol_site(const DevModel &m, const IMol<SIG> &I, int a, float &d0, float &d1,
                                          float &d2, float4 &e)
{
    if constexpr (SIG::LIN) {
        const float4 u = I.e_axis;
        const float z = m.body[a][2], sa = m.axis[a][2];
        d0 = z * u.x;
        d1 = z * u.y;
        d2 = z * u.z;
        e = (SIG::role(a, m) & AX_ROLES) ? make_float4(sa * u.x, sa * u.y, sa * u.z, 0.f)
                                         : make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
        d0 = I.d[a][0];
        d1 = I.d[a][1];
        d2 = I.d[a][2];
        e = I.e[a];
    }
}

// Pair of molecules: force on i, torque on i (lever arms + orientation),
// energy; with JSIDE also the torque on j from the pair's angular-momentum
// balance, tau_i + tau_j + X x F_ij = 0 (X = R_i - R_j), which holds exactly
// for the rotation-invariant site-site laws of §2.  Site forces are summed
// per site of i inside the pair so that the lever-arm torque costs 6 FMA
// per site of i.
template <class SIG, bool JSIDE, bool UJ = false>  // UJ: the j axis is given (ujv), not read from gj
__device__ __forceinline__ void mol_pair(const DevModel &m, const float X0, const float X1, const float X2,
                                         const IMol<SIG> &I, const float4 *__restrict__ gj, float (&Fo)[3],
                                         float (&to)[3], float (&tj)[3], float &Uo,
                                         const float4 ujv = make_float4(0.f, 0.f, 0.f, 0.f))
{
    constexpr int S = SIG::S;
    float fa[S][3], xa[S][3];
    float4 ea[S];  // space-frame axes of i's sites
#pragma unroll
    for (int a = 0; a < S; a++) {
        fa[a][0] = fa[a][1] = fa[a][2] = 0.f;
        float d0, d1, d2;
        imol_site<SIG>(m, I, a, d0, d1, d2, ea[a]);
        if (SIG::at_com(a)) {  // zero offset: no add (x + 0 is not folded under IEEE rules)
            xa[a][0] = X0;
            xa[a][1] = X1;
            xa[a][2] = X2;
        } else {
            xa[a][0] = X0 + d0;
            xa[a][1] = X1 + d1;
            xa[a][2] = X2 + d2;
        }
    }
    float ti[3] = {0.f, 0.f, 0.f}, tdummy[3];
    float U = 0.f;
    if (SIG::SINGLE) {
        const float r2 = X0 * X0 + X1 * X1 + X2 * X2;
        const float ir2 = __fdividef(1.f, r2);
        const float s2 = m.sig2[0][0] * ir2;
        const float s6 = s2 * s2 * s2;
        const float fr = m.eps24[0][0] * s6 * (2.f * s6 - 1.f) * ir2;
        U = m.eps4[0][0] * s6 * (s6 - 1.f) - m.ushift[0][0];
        fa[0][0] = fr * X0;
        fa[0][1] = fr * X1;
        fa[0][2] = fr * X2;
    } else {
        float4 uj = make_float4(0.f, 0.f, 0.f, 0.f);
        if constexpr (SIG::LIN) uj = UJ ? ujv : __ldg(gj);  // the j molecule's axis
        if constexpr (lin_lj2<SIG>()) {
            // x_ab = X + z_a u_i - z_b u_j for the LJ sites a, b in {0, 1}
            const float4 ui = I.e_axis;
            const float z0 = m.body[0][2], z1 = m.body[1][2];
            const float2 za = f2(z0, z1), nzb0 = f2(-z0, -z1), nzb1 = f2(-z1, -z0);
            const float2 wx = fma2(za, f2(ui.x, ui.x), f2(X0, X0));
            const float2 wy = fma2(za, f2(ui.y, ui.y), f2(X1, X1));
            const float2 wz = fma2(za, f2(ui.z, ui.z), f2(X2, X2));
            const float2 ujx = f2(uj.x, uj.x), ujy = f2(uj.y, uj.y), ujz = f2(uj.z, uj.z);
            const float2 sg = f2(m.sig2[0][0], m.sig2[0][0]), e4 = f2(m.eps4[0][0], m.eps4[0][0]),
                         e24 = f2(m.eps24[0][0], m.eps24[0][0]);
            float2 fx = f2(0.f, 0.f), fy = fx, fz = fx, U2 = fx;
            lj_pair2(fma2(nzb0, ujx, wx), fma2(nzb0, ujy, wy), fma2(nzb0, ujz, wz), sg, e4, e24, fx, fy, fz, U2);
            lj_pair2(fma2(nzb1, ujx, wx), fma2(nzb1, ujy, wy), fma2(nzb1, ujz, wz), sg, e4, e24, fx, fy, fz, U2);
            U += (U2.x + U2.y) - 4.f * m.ushift[0][0];
            fa[0][0] = fx.x;
            fa[0][1] = fy.x;
            fa[0][2] = fz.x;
            fa[1][0] = fx.y;
            fa[1][1] = fy.y;
            fa[1][2] = fz.y;
        }
        // the run-time signature keeps its j-site loop rolled (its i-site
        // loop stays unrolled, so the site totals stay in registers): a fully
        // unrolled 8 x 8 site loop with run-time roles takes minutes to compile
#pragma unroll(SIG::DYN ? 1 : S)
        for (int b = 0; b < S; b++) {
            const int rb = SIG::role(b, m);
            if (rb == 0) continue;
            float4 db, eb = make_float4(0.f, 0.f, 0.f, 0.f);
            if constexpr (SIG::LIN) {
                const float z = m.body[b][2], sb = m.axis[b][2];
                db = SIG::at_com(b) ? make_float4(0.f, 0.f, 0.f, 0.f) : make_float4(z * uj.x, z * uj.y, z * uj.z, 0.f);
                if (rb & AX_ROLES) eb = make_float4(sb * uj.x, sb * uj.y, sb * uj.z, 0.f);
            } else {
                db = __ldg(gj + b);
                if (rb & AX_ROLES) eb = __ldg(gj + SIG::s_of(m) + SIG::slot(b, m));
            }
#pragma unroll
            for (int a = 0; a < S; a++) {
                const int ra = SIG::role(a, m);
                const bool lj = (ra & ROLE_LJ) && (rb & ROLE_LJ) && !(lin_lj2<SIG>() && a < 2 && b < 2);
                const bool el = (ra & EL_ROLES) && (rb & EL_ROLES);
                if (!lj && !el) continue;
                const bool zb = SIG::LIN && SIG::at_com(b);
                const float x = zb ? xa[a][0] : xa[a][0] - db.x;
                const float y = zb ? xa[a][1] : xa[a][1] - db.y;
                const float z = zb ? xa[a][2] : xa[a][2] - db.z;
                const float r2 = x * x + y * y + z * z;
                float fx = 0.f, fy = 0.f, fz = 0.f;
                float ir = 0.f, ir2;
                if (el) {
                    ir = rsqrtf(r2);
                    ir2 = ir * ir;
                } else {
                    ir2 = __fdividef(1.f, r2);
                }
                if (lj) {
                    const int ta = SIG::type(a, m), tb = SIG::type(b, m);
                    const float s2 = m.sig2[ta][tb] * ir2;
                    const float s6 = s2 * s2 * s2;
                    const float fr = m.eps24[ta][tb] * s6 * (2.f * s6 - 1.f) * ir2;
                    U += m.eps4[ta][tb] * s6 * (s6 - 1.f) - m.ushift[ta][tb];
                    fx = fr * x;
                    fy = fr * y;
                    fz = fr * z;
                }
                if (el) {
                    elec_site<false>(ra, rb, m.chg[a], m.mu[a], m.Q[a], m.chg[b], m.mu[b], m.Q[b], m.frf, x, y, z,
                                     ir, ea[a], eb, U, fx, fy, fz, ti, tdummy);
                }
                fa[a][0] += fx;
                fa[a][1] += fy;
                fa[a][2] += fz;
            }
        }
    }
    float F0 = 0.f, F1 = 0.f, F2 = 0.f;
    if constexpr (SIG::LIN) {
        // lever arms z_a u: sum_a z_a u x f_a = u x (sum_a z_a f_a)
        float g0 = 0.f, g1 = 0.f, g2 = 0.f;
#pragma unroll
        for (int a = 0; a < S; a++) {
            F0 += fa[a][0];
            F1 += fa[a][1];
            F2 += fa[a][2];
            if (!SIG::at_com(a)) {
                const float z = m.body[a][2];
                g0 += z * fa[a][0];
                g1 += z * fa[a][1];
                g2 += z * fa[a][2];
            }
        }
        const float4 u = I.e_axis;
        ti[0] += u.y * g2 - u.z * g1;
        ti[1] += u.z * g0 - u.x * g2;
        ti[2] += u.x * g1 - u.y * g0;
    } else {
#pragma unroll
        for (int a = 0; a < S; a++) {
            F0 += fa[a][0];
            F1 += fa[a][1];
            F2 += fa[a][2];
            if constexpr (!SIG::SINGLE && !SIG::LIN) {
                ti[0] += I.d[a][1] * fa[a][2] - I.d[a][2] * fa[a][1];
                ti[1] += I.d[a][2] * fa[a][0] - I.d[a][0] * fa[a][2];
                ti[2] += I.d[a][0] * fa[a][1] - I.d[a][1] * fa[a][0];
            }
        }
    }
    Fo[0] = F0;
    Fo[1] = F1;
    Fo[2] = F2;
    to[0] = ti[0];
    to[1] = ti[1];
    to[2] = ti[2];
    if (JSIDE) {
        if (SIG::SINGLE) {
            tj[0] = tj[1] = tj[2] = 0.f;
        } else {
            tj[0] = -ti[0] - (X1 * F2 - X2 * F1);
            tj[1] = -ti[1] - (X2 * F0 - X0 * F2);
            tj[2] = -ti[2] - (X0 * F1 - X1 * F0);
        }
    }
    Uo = U;
}


// ------------------------------------------------------------- traversal
#ifndef MD_JCAP
#define MD_JCAP 256
#endif
constexpr int JCAP = MD_JCAP;  // staged candidates per segment (a multiple of 32)
#ifndef MD_TEST_UNROLL
#define MD_TEST_UNROLL 8
#endif
constexpr int NTEST = MD_TEST_UNROLL;   // candidates per lane per test round
constexpr int QCAP = 32 * (NTEST + 1);  // hit queue of chunk-drained operations (31 waiting + NTEST x 32 new)
constexpr int QRUN = 1024;              // hit queue of run-drained operations (a window's hits, or a part)

// Stencils wider than a warp (M = 2): each stencil cell's first slot and
// the exclusive prefix of the counts, per warp in shared memory.
struct StencilMeta {
    int j0[Stencil<2>::FULL];
    int pre[Stencil<2>::FULL + 1];
};

// Per-warp staging area; Extra is the pair operation's own shared state, QC
// the capacity of its hit queue.
template <class Extra, int QC = QCAP>
struct WarpTile {
    static constexpr int QCAPACITY = QC;
    static constexpr bool DUP = false;
    static constexpr bool AXES = false;  // no staged axes
    static constexpr int QSHIFT = 16;    // queue entry (i << 16) | k
    float4 jc[JCAP];          // candidate COM + image offset (i-cell frame); w = storage slot bits
    unsigned char jst[JCAP];  // stencil index of the candidate's cell
    int queue[QC];
    Extra x;
    __device__ __forceinline__ float4 cand(int k) const { return jc[k]; }
    __device__ __forceinline__ int cand_slot(int k) const { return __float_as_int(jc[k].w); }
    __device__ __forceinline__ void stage(int t, float x_, float y_, float z_, int js, int o)
    {
        jc[t] = make_float4(x_, y_, z_, __int_as_float(js));
        jst[t] = (unsigned char)o;
    }
    // duplicated layout and staged axes (WarpTileD only)
    __device__ __forceinline__ float4 dxy(int) const { return make_float4(0.f, 0.f, 0.f, 0.f); }
    __device__ __forceinline__ float2 dz(int) const { return make_float2(0.f, 0.f); }
    __device__ __forceinline__ void pad(int, int) {}
    __device__ __forceinline__ void stage_axis(int, float4) {}
    __device__ __forceinline__ float4 axis(int) const { return make_float4(0.f, 0.f, 0.f, 0.f); }
};

// Staging area of the half shell's duplicated-candidate test: each
// candidate's coordinates negated and duplicated, (-x, -x, -y, -y) and
// (-z, -z), so that one f32x2 instruction advances the tests of two i
// molecules against it, and 32 far-away sentinels after the window's last
// candidate, so that test rounds need no range check; queue entries
// (i << 16) | k.  CP (compact): -z stored once (the test duplicates it in a
// register pair) and 16-bit queue entries (i << 8) | k.  AX (linear
// molecules, compact): the candidates' axes staged beside them, so that the
// drained pairs read no global memory, in less shared memory than the wide
// layout without axes (four blocks per SM).  Single-site molecules use the
// compact layout without axes, which lets five blocks fit an SM.
template <class Extra, int QC, bool AX = false, bool CP = AX>
struct WarpTileD {
    static_assert(!CP || JCAP <= 256, "16-bit queue entries hold k in 8 bits");
    static constexpr int QCAPACITY = QC;
    static constexpr bool DUP = true;
    static constexpr bool AXES = AX;
    static constexpr int QSHIFT = CP ? 8 : 16;
    using ZT = std::conditional_t<CP, float, float2>;
    using QT = std::conditional_t<CP, unsigned short, int>;
    float4 jd[JCAP + 32];
    ZT jz[JCAP + 32];
    int jslot[JCAP];               // storage slot of each candidate
    float jax[AX ? 3 * JCAP : 1];  // axis of each candidate (AX)
    unsigned char jst[JCAP];       // stencil index of the candidate's cell
    QT queue[QC];
    Extra x;
    __device__ __forceinline__ float4 cand(int k) const
    {
        const float4 d = jd[k];
        return make_float4(-d.x, -d.z, -dz(k).x, 0.f);
    }
    __device__ __forceinline__ int cand_slot(int k) const { return jslot[k]; }
    __device__ __forceinline__ void stage(int t, float x_, float y_, float z_, int js, int o)
    {
        jd[t] = make_float4(-x_, -x_, -y_, -y_);
        if constexpr (CP) jz[t] = -z_;
        else jz[t] = make_float2(-z_, -z_);
        jslot[t] = js;
        jst[t] = (unsigned char)o;
    }
    __device__ __forceinline__ void stage_axis(int t, float4 u)
    {
        if constexpr (AX) {
            jax[3 * t] = u.x;
            jax[3 * t + 1] = u.y;
            jax[3 * t + 2] = u.z;
        }
    }
    __device__ __forceinline__ float4 axis(int k) const
    {
        if constexpr (AX) return make_float4(jax[3 * k], jax[3 * k + 1], jax[3 * k + 2], 0.f);
        else return make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __device__ __forceinline__ float4 dxy(int k) const { return jd[k]; }
    __device__ __forceinline__ float2 dz(int k) const
    {
        if constexpr (CP) {
            const float z = jz[k];
            return make_float2(z, z);
        } else {
            return jz[k];
        }
    }
    // sentinels at candidates [nj, nj + 32) (all lanes call)
    __device__ __forceinline__ void pad(int nj, int lane)
    {
        jd[nj + lane] = make_float4(-1.0e18f, -1.0e18f, -1.0e18f, -1.0e18f);
        if constexpr (CP) jz[nj + lane] = -1.0e18f;
        else jz[nj + lane] = make_float2(-1.0e18f, -1.0e18f);
    }
};

// The periodic grid a cell belongs to (one system, or one replica of a batch).
struct GridView {
    int nc[3];
    float ellf[3];
    double L[3];
    double rc2;
    float rc2f, bandf;
    long long cell0;          // first global cell index of this grid
};

// Calls visit(c, p) once for every part p < parts of every cell c < ncell,
// each (cell, part) unit by one warp of the grid (warp = the warp's index
// in its block); a part is a contiguous share of the cell's i molecules.
// ctr non-null: units one at a time in counter order (the parts of a cell
// consecutively), the next claimed when the warp has finished its unit
// (cell costs vary with the occupation, so warps that finish early take
// more; claiming ahead balances the tail one unit later and measured
// slower).  ctr null: a fixed grid stride, the same units per warp on every
// launch (fixed summation grouping of the block partials).
template <class Visit>
__device__ __forceinline__ void for_each_cell(long long ncell, int parts, unsigned *ctr, int warp, int lane,
                                              Visit &&visit)
{
    const long long units = ncell * parts;
    if (ctr) {
        for (;;) {
            unsigned u = 0;
            if (lane == 0) u = atomicAdd(ctr, 1u);
            u = __shfl_sync(FULLMASK, u, 0);
            if (u >= units) break;
            visit((long long)(u / parts), (int)(u % parts));
        }
    } else {
        for (long long u = (long long)blockIdx.x * MD_WARPS + warp; u < units; u += (long long)gridDim.x * MD_WARPS)
            visit(u / parts, (int)(u % parts));
    }
}

// Visits every interacting pair (i in cell c, j in the stencil) in chunks
// of <= 32 pairs; with parts > 1 only the i of share `part` of the cell's
// molecules.  The hits of consecutive i molecules of a pass share a
// queue, so a chunk may hold pairs of several i's (contiguous lanes per i,
// in i order) and only the last chunk of a segment is partly filled.
// Op provides:
//   pass_begin(ig, ni, lane) / pass_end(s0, ig, ni, lane)
//   seg_begin(T, nj, lane)            after a segment has been staged
//   seg_end(T, nj, lane)              after all i's of a pass met the segment
//   pair(T, I, k, X0, X1, X2, js)     the lane's queued pair (i molecule I,
//                                     staged candidate k, storage slot js)
//   chunk_end(T, il, k, valid, lane)  all lanes, after the pairs of a chunk;
//                                     il = the lane's i index in the pass
//                                     (lanes of one i are contiguous and
//                                     their k are distinct)
//   count_examined(n)
// An operation with RUNS = true is instead drained in runs: the hits of all
// i's of a pass against the staged window collect in its (larger) queue and
// drain(T, qn, sbase, lane) consumes them at the end of the window (or when
// the queue would overflow); lanes take contiguous runs of entries, so that
// a lane meets one i for many consecutive pairs (sbase = storage slot of
// the pass's first i).  chunk_end is then not called.
// cell_start holds global slots; c is the cell index inside the grid.
// NT: candidates per lane per test round of the chunked pipeline (a tile
// parameter of the batched replicas' autotuner; <= NTEST).
template <class SIG, bool HALF, int M = 1, int NT = NTEST, class Op, class Tile>
__device__ __forceinline__ void traverse_cell(const DevModel &m, const GridView &g, const int *__restrict__ cell_start,
                                              const float4 *__restrict__ com, const float4 *__restrict__ geo,
                                              const double *__restrict__ r64, int K, long long c, Tile &T,
                                              Op &op, int lane, StencilMeta *meta = nullptr, int part = 0,
                                              int parts = 1)
{
    constexpr int IMAX = Op::IMAX;
    static_assert(IMAX <= 32 && JCAP <= 65536, "queue entry packs (i << 16) | k");
    const unsigned lt_mask = (1u << lane) - 1u;
    static_assert(M == 1 || M == 2, "stencil radius 1 or 2 cells");
    constexpr int NOFF = HALF ? Stencil<M>::HALFN : Stencil<M>::FULL;
    constexpr int SELF = HALF ? 0 : Stencil<M>::CENTRE;  // stencil index of the cell itself
    const int cx = (int)(c % g.nc[0]);
    const int cy = (int)((c / g.nc[0]) % g.nc[1]);
    const int cz = (int)(c / ((long long)g.nc[0] * g.nc[1]));
    // M = 1: stencil cell of lane t (< NOFF): first slot, count, offset of
    // its cell centre and the exclusive prefix of the counts (position in the
    // concatenated candidate list); loaded at once, then read by shuffles
    // while staging.  M = 2 (more stencil cells than lanes): first slots and
    // prefixes in shared memory, offsets recomputed from the stencil index.
    int t_j0 = 0, t_cnt = 0, t_pre = 0;
    float t_ox = 0.f, t_oy = 0.f, t_oz = 0.f;
    int n_cand, self_pre, self_cnt, s0;
    if constexpr (M == 1) {
        if (lane < NOFF) {
            int dx, dy, dz, kx, ky, kz;
            stencil_offset<M>(HALF, lane, dx, dy, dz);
            const int nx = wrap_axis(cx, dx, g.nc[0], kx);
            const int ny = wrap_axis(cy, dy, g.nc[1], ky);
            const int nz = wrap_axis(cz, dz, g.nc[2], kz);
            const long long cn = g.cell0 + ((long long)nz * g.nc[1] + ny) * g.nc[0] + nx;
            t_j0 = cell_start[cn];
            t_cnt = cell_start[cn + 1] - t_j0;
            t_ox = dx * g.ellf[0];
            t_oy = dy * g.ellf[1];
            t_oz = dz * g.ellf[2];
        }
        t_pre = t_cnt;  // inclusive scan, then exclusive
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(FULLMASK, t_pre, o);
            if (lane >= o) t_pre += v;
        }
        n_cand = __shfl_sync(FULLMASK, t_pre, NOFF - 1);
        t_pre -= t_cnt;
        self_pre = __shfl_sync(FULLMASK, t_pre, SELF);
        self_cnt = __shfl_sync(FULLMASK, t_cnt, SELF);
        // the i-cell is the stencil's own entry (no separate load round)
        s0 = __shfl_sync(FULLMASK, t_j0, SELF);
        // the table staging reads (shared memory, so that it holds no
        // registers while the pairs are computed); unused entries never match
    } else {
        int carry = 0;
        for (int e0 = 0; e0 < NOFF; e0 += 32) {  // warp-uniform
            const int e = e0 + lane;
            int j0 = 0, cnt = 0;
            if (e < NOFF) {
                int dx, dy, dz, kx, ky, kz;
                stencil_offset<M>(HALF, e, dx, dy, dz);
                const int nx = wrap_axis(cx, dx, g.nc[0], kx);
                const int ny = wrap_axis(cy, dy, g.nc[1], ky);
                const int nz = wrap_axis(cz, dz, g.nc[2], kz);
                const long long cn = g.cell0 + ((long long)nz * g.nc[1] + ny) * g.nc[0] + nx;
                j0 = cell_start[cn];
                cnt = cell_start[cn + 1] - j0;
            }
            int inc = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(FULLMASK, inc, o);
                if (lane >= o) inc += v;
            }
            if (e < NOFF) {
                meta->j0[e] = j0;
                meta->pre[e] = carry + inc - cnt;
            }
            carry += __shfl_sync(FULLMASK, inc, 31);
        }
        if (lane == 0) meta->pre[NOFF] = carry;
        __syncwarp();
        n_cand = carry;
        self_pre = meta->pre[SELF];
        self_cnt = meta->pre[SELF + 1] - self_pre;
        s0 = meta->j0[SELF];
    }
    const int n_i = self_cnt;
    // this unit's share of the cell's i molecules
    const int i_lo = n_i * part / parts, i_hi = n_i * (part + 1) / parts;  // n_i * parts << 2^31
    if (i_lo >= i_hi) return;
    for (int ig = i_lo; ig < i_hi; ig += IMAX) {
        const int ni = min(IMAX, i_hi - ig);
        op.pass_begin(ig, ni, lane);
        // the first nq queue entries as one chunk (all lanes call)
        auto chunk = [&](int nq) {
            const bool valid = lane < nq;
            int il = 32 + lane, k = -1 - lane;  // unique placeholders for idle lanes
            if (valid) {
                const int e = T.queue[lane];
                il = e >> 16;
                k = e & 0xffff;
            }
            if (valid) {
                IMol<SIG> I;
                load_i<SIG>(m, com, geo, K, s0 + ig + il, I);
                const float4 cj = T.cand(k);
                op.pair(T, I, k, I.c.x - cj.x, I.c.y - cj.y, I.c.z - cj.z, T.cand_slot(k));
            }
            op.chunk_end(T, il, k, valid, lane);
        };
        // segments: consecutive windows of <= JCAP entries of the candidate list
        for (int seg0 = 0; seg0 < n_cand; seg0 += JCAP) {
            const int nj = min(JCAP, n_cand - seg0);
            // every lane stages entries x = seg0 + lane + 32 b; its stencil
            // cell is the last one whose prefix is <= x (binary search over
            // the lanes' prefixes for M = 1, over the shared prefixes for
            // M = 2); the loads of all rounds are independent
            if constexpr (M == 1) {
#pragma unroll 4
                for (int tb = 0; tb < nj; tb += 32) {  // warp-uniform trip count: the shuffles need every lane
                    const int t = tb + lane;
                    const int x = seg0 + t;
                    int o = 0;
#pragma unroll
                    for (int st = 16; st > 0; st >>= 1) {
                        const int c2 = o + st;
                        const int p2 = __shfl_sync(FULLMASK, t_pre, c2 < NOFF ? c2 : 0);
                        if (c2 < NOFF && p2 <= x) o = c2;
                    }
                    const int js = __shfl_sync(FULLMASK, t_j0, o) + (x - __shfl_sync(FULLMASK, t_pre, o));
                    const float ox = __shfl_sync(FULLMASK, t_ox, o), oy = __shfl_sync(FULLMASK, t_oy, o),
                                oz = __shfl_sync(FULLMASK, t_oz, o);
                    if (t < nj) {
                        const float4 cj = com[js];
                        if constexpr (Tile::AXES) T.stage_axis(t, geo[(long long)js * K]);
                        T.stage(t, cj.x + ox, cj.y + oy, cj.z + oz, js, o);
                    }
                }
            } else {
#pragma unroll 2
                for (int t = lane; t < nj; t += 32) {
                    const int x = seg0 + t;
                    int o = 0;  // the last stencil cell whose prefix is <= x (an occupied one)
#pragma unroll
                    for (int st = 64; st > 0; st >>= 1) {
                        const int c2 = o + st;
                        if (c2 < NOFF && meta->pre[c2] <= x) o = c2;
                    }
                    int dx, dy, dz;
                    stencil_offset<M>(HALF, o, dx, dy, dz);
                    const int js = meta->j0[o] + (x - meta->pre[o]);
                    const float4 cj = com[js];
                    T.stage(t, cj.x + dx * g.ellf[0], cj.y + dy * g.ellf[1], cj.z + dz * g.ellf[2], js, o);
                }
            }
            T.pad(nj, lane);
            // the i-cell's entries in this window: local index self_lo + (k - self_base)
            const int w_lo = max(self_pre, seg0), w_hi = min(self_pre + self_cnt, seg0 + nj);
            const int self_n = max(0, w_hi - w_lo), self_lo = w_lo - self_pre, self_base = w_lo - seg0;
            op.seg_begin(T, nj, lane);
            __syncwarp();
            // FP64 cut-off decision of the pass's i molecule il and staged
            // candidate k (pairs queued inside the FP32 band)
            auto exact_in = [&](int il, int k) -> bool {
                int dx, dy, dz, kx, ky, kz;
                stencil_offset<M>(HALF, T.jst[k], dx, dy, dz);
                wrap_axis(cx, dx, g.nc[0], kx);
                wrap_axis(cy, dy, g.nc[1], ky);
                wrap_axis(cz, dz, g.nc[2], kz);
                const double *ri = r64 + 3LL * (s0 + ig + il), *rj = r64 + 3LL * T.cand_slot(k);
                const double e0 = __dsub_rn(__dsub_rn(ri[0], rj[0]), (double)kx * g.L[0]);
                const double e1 = __dsub_rn(__dsub_rn(ri[1], rj[1]), (double)ky * g.L[1]);
                const double e2 = __dsub_rn(__dsub_rn(ri[2], rj[2]), (double)kz * g.L[2]);
                return __dadd_rn(__dadd_rn(__dmul_rn(e0, e0), __dmul_rn(e1, e1)), __dmul_rn(e2, e2)) < g.rc2;
            };
            int qn = 0;
            if constexpr (Tile::DUP) {
                // two i molecules per test round (a = il, b = il + 1; b absent
                // at an odd end of the pass) against candidates k = kb + 32 u
                // + lane, with kb the i's first candidate rounded down to a
                // multiple of 32 and as many 32-wide steps as reach the
                // window's end (the sentinels fill the last step); tests
                // against the widened bound rc^2 + band, the FP64 decision
                // inside the band is taken when the pair is drained
                static_assert(JCAP == 256, "the round widths below cover 1 ... 8 steps of 32");
                const float hi = g.rc2f + g.bandf;
                for (int il = ig; il < ig + ni; il += 2) {
                    const bool has_b = il + 1 < ig + ni;
                    const int ib = has_b ? il + 1 : il;
                    auto ci_of = [&](int i) -> float4 {
                        const bool in_seg = self_n > 0 && i >= self_lo && i < self_lo + self_n;
                        return in_seg ? T.cand(self_base + i - self_lo) : com[s0 + i];
                    };
                    auto skip_of = [&](int i) -> int {
                        return (self_n > 0 && HALF) ? max(0, min(self_n, i - self_lo + 1)) : 0;
                    };
                    const float4 ca = ci_of(il), cb = ci_of(ib);
                    const int skip_a = skip_of(il), skip_b = has_b ? skip_of(ib) : nj;
                    const float2 Cx = f2(ca.x, cb.x), Cy = f2(ca.y, cb.y), Cz = f2(ca.z, cb.z);
                    const int kb = skip_a & ~31;
                    const int tag_a = (il - ig) << Tile::QSHIFT, tag_b = (ib - ig) << Tile::QSHIFT;
                    auto round_d = [&](auto ntc) {
                        constexpr int NT = decltype(ntc)::value;
                        bool ha[NT], hb[NT];
#pragma unroll
                        for (int u = 0; u < NT; u++) {
                            const int k = kb + 32 * u + lane;
                            const float4 d = T.dxy(k);
                            const float2 dd = T.dz(k);
                            const float2 dx = __fadd2_rn(Cx, f2(d.x, d.y));
                            const float2 dy = __fadd2_rn(Cy, f2(d.z, d.w));
                            const float2 dz = __fadd2_rn(Cz, dd);
                            const float2 d2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
                            ha[u] = d2.x < hi;
                            hb[u] = d2.y < hi;
                        }
                        // the own cell's candidates up to and including the i
                        ha[0] = ha[0] && kb + lane >= skip_a;
                        hb[0] = hb[0] && kb + lane >= skip_b;
#pragma unroll
                        for (int u = 0; u < NT; u++) {
                            const unsigned bal = __ballot_sync(FULLMASK, ha[u]);
                            if (ha[u]) T.queue[qn + __popc(bal & lt_mask)] = tag_a | (kb + 32 * u + lane);
                            qn += __popc(bal);
                        }
#pragma unroll
                        for (int u = 0; u < NT; u++) {
                            const unsigned bal = __ballot_sync(FULLMASK, hb[u] && has_b);
                            if (hb[u] && has_b) T.queue[qn + __popc(bal & lt_mask)] = tag_b | (kb + 32 * u + lane);
                            qn += __popc(bal);
                        }
                    };
                    if (qn > Tile::QCAPACITY - 64 * (JCAP / 32)) {  // room for a full round of two i's
                        __syncwarp();
                        op.drain(T, qn, s0 + ig, lane, exact_in, g.rc2f - g.bandf);
                        qn = 0;
                        __syncwarp();
                    }
                    switch ((nj - kb + 31) >> 5) {  // warp-uniform, 1 ... JCAP / 32
                    case 1: round_d(std::integral_constant<int, 1>{}); break;
                    case 2: round_d(std::integral_constant<int, 2>{}); break;
                    case 3: round_d(std::integral_constant<int, 3>{}); break;
                    case 4: round_d(std::integral_constant<int, 4>{}); break;
                    case 5: round_d(std::integral_constant<int, 5>{}); break;
                    case 6: round_d(std::integral_constant<int, 6>{}); break;
                    case 7: round_d(std::integral_constant<int, 7>{}); break;
                    default: round_d(std::integral_constant<int, JCAP / 32>{}); break;
                    }
                    if (lane == 0) op.count_examined((nj - skip_a) + (has_b ? nj - skip_b : 0));
                }
            } else {
                for (int il = ig; il < ig + ni; il++) {
                    const int si = s0 + il;
                    const bool in_seg = self_n > 0 && il >= self_lo && il < self_lo + self_n;
                    const float4 ci = in_seg ? T.cand(self_base + il - self_lo) : com[si];
                    const int skip_to = (self_n > 0 && HALF) ? max(0, min(self_n, il - self_lo + 1)) : 0;
                    const int self_k = (!HALF && in_seg) ? self_base + (il - self_lo) : -1;
                    const int tag = (il - ig) << 16;
                    // squared COM distance of candidate k (huge if k is not a candidate of i)
                    auto dist2 = [&](int k) -> float {
                        if (k >= nj || (!HALF && k == self_k)) return 3.0e38f;
                        const float4 cj = T.cand(k);
                        const float X0 = ci.x - cj.x, X1 = ci.y - cj.y, X2 = ci.z - cj.z;
                        return X0 * X0 + X1 * X1 + X2 * X2;
                    };
                    // the same test in FP64 from the FP64 state (pairs near the cut-off)
                    auto test64 = [&](int k) -> bool {
                        int dx, dy, dz, kx, ky, kz;
                        stencil_offset<M>(HALF, T.jst[k], dx, dy, dz);
                        wrap_axis(cx, dx, g.nc[0], kx);
                        wrap_axis(cy, dy, g.nc[1], ky);
                        wrap_axis(cz, dz, g.nc[2], kz);
                        const double *ri = r64 + 3LL * si, *rj = r64 + 3LL * T.cand_slot(k);
                        const double e0 = __dsub_rn(__dsub_rn(ri[0], rj[0]), (double)kx * g.L[0]);
                        const double e1 = __dsub_rn(__dsub_rn(ri[1], rj[1]), (double)ky * g.L[1]);
                        const double e2 = __dsub_rn(__dsub_rn(ri[2], rj[2]), (double)kz * g.L[2]);
                        return __dadd_rn(__dadd_rn(__dmul_rn(e0, e0), __dmul_rn(e1, e1)), __dmul_rn(e2, e2)) < g.rc2;
                    };
                    // one test round: NT candidates per lane (independent tests),
                    // then the hits are appended in candidate order
                    auto round = [&](auto ntc, int kb) {
                        constexpr int NT = decltype(ntc)::value;
                        bool h[NT], near[NT], any_near = false;
    #pragma unroll
                        for (int u = 0; u < NT; u++) {
                            const float d2 = dist2(kb + 32 * u + lane);
                            h[u] = d2 < g.rc2f;
                            near[u] = fabsf(d2 - g.rc2f) < g.bandf;
                            any_near |= near[u];
                        }
                        if (__any_sync(FULLMASK, any_near)) {  // rare: decide in FP64
    #pragma unroll
                            for (int u = 0; u < NT; u++)
                                if (near[u]) h[u] = test64(kb + 32 * u + lane);
                        }
    #pragma unroll
                        for (int u = 0; u < NT; u++) {
                            const unsigned bal = __ballot_sync(FULLMASK, h[u]);
                            if (h[u]) T.queue[qn + __popc(bal & lt_mask)] = tag | (kb + 32 * u + lane);
                            qn += __popc(bal);
                        }
                        if constexpr (!Op::RUNS) {
                            while (qn >= 32) {
                                __syncwarp();
                                chunk(32);
                                __syncwarp();
                                for (int t = lane; t < qn - 32; t += 32) T.queue[t] = T.queue[32 + t];
                                qn -= 32;
                                __syncwarp();
                            }
                        }
                    };
                    // run-drained: keep room for one more full test round
                    auto make_room = [&]() {
                        if constexpr (Op::RUNS) {
                            if (qn > Tile::QCAPACITY - 32 * NTEST) {
                                __syncwarp();
                                op.drain(T, qn, s0 + ig, lane, exact_in, g.rc2f - g.bandf);
                                qn = 0;
                                __syncwarp();
                            }
                        }
                    };
                    {
                        // warp-uniform: half-width rounds when the i's candidates fit
                        static_assert(NT <= NTEST && NT % 2 == 0, "test rounds of 2 ... NTEST candidates per lane");
                        if (nj - skip_to <= 32 * (NT / 2)) {
                            make_room();
                            round(std::integral_constant<int, NT / 2>{}, skip_to);
                        } else {
                            for (int kb = skip_to; kb < nj; kb += 32 * NT) {
                                make_room();
                                round(std::integral_constant<int, NT>{}, kb);
                            }
                        }
                    }
                    if (lane == 0) op.count_examined(nj - skip_to - (self_k >= 0 ? 1 : 0));
                }
            }
            if (qn > 0) {
                __syncwarp();
                if constexpr (Op::RUNS) op.drain(T, qn, s0 + ig, lane, exact_in, g.rc2f - g.bandf);
                else chunk(qn);
            }
            __syncwarp();
            op.seg_end(T, nj, lane);
            __syncwarp();
        }
        op.pass_end(s0, ig, ni, lane);
        __syncwarp();
    }
}

}  // namespace mdk
