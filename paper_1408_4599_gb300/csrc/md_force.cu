// md_force.cu -- linked-cell force / torque / energy / virial kernel (§3:
// "calculation of forces and torques", linked cells with the 27-cell
// stencil, Newton-3 cell enumeration) for rigid molecules of LJ centres
// (Eq. 1, LJTS, Lorentz-Berthelot) and point charges, dipoles and linear
// quadrupoles (§2), reaction field for dipoles (§3).
//
// Design (GB300, CUDA cores -- this is not a dense contraction):
//   * one warp per cell of i molecules; G lanes share one i molecule when
//     the cell holds fewer than 32 (G = 32 / next_pow2(n_i)), each lane
//     testing a 1/G share of the candidate j molecules;
//   * centre-of-mass cut-off test in FP32 on cell-centre-relative
//     coordinates; tests that land within a narrow band around rc^2 are
//     redone in FP64 from the FP64 state, so the set of interacting pairs
//     is the one the FP64 definition selects;
//   * hits go to a per-lane list in shared memory; when any lane's list is
//     full (and at the end) all lanes evaluate their lists in lock step, so
//     the expensive site-site math runs on packed lanes instead of on the
//     15% of lanes that a direct test-and-compute loop would keep busy;
//   * FP32 site-site math, FP32 per-lane partial sums, warp shuffles to
//     combine the G lanes of one molecule, FP64 for the stored force,
//     torque and the block energy / virial partials;
//   * full shell (27 cells, each ordered pair from both sides, no atomics,
//     deterministic) or half shell (14 cells, Newton 3, the reaction on j
//     added with FP64 atomics).
#include "md_internal.cuh"

namespace {

struct ForceArgs {
    Grid g;
    DevModel m;
    const int *cell_start;
    const float4 *com;
    const float4 *geo;
    const double *r;
    double *F, *tau;
    double *partials;
    int *flags;
};

// Half-shell stencil: the cell itself and the 13 neighbours that follow it
// in (z, y, x) lexicographic order.
__constant__ signed char c_half[14][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 1, 0}, {0, 1, 0}, {1, 1, 0},
                                          {-1, -1, 1}, {0, -1, 1}, {1, -1, 1}, {-1, 0, 1}, {0, 0, 1},
                                          {1, 0, 1},  {-1, 1, 1},  {0, 1, 1},  {1, 1, 1}};

constexpr int EL_ROLES = ROLE_CHG | ROLE_DIP | ROLE_QUAD;
constexpr int AX_ROLES = ROLE_DIP | ROLE_QUAD;

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

// Compile-time site-role signature: S sites, 4 role bits per site.
template <int S_, unsigned R_, bool SINGLE_ = false>
struct SigStatic {
    static constexpr int S = S_;
    static constexpr bool DYN = false;
    static constexpr bool SINGLE = SINGLE_;
    static constexpr int K = S_ + sig_na(R_, S_);
    __device__ __forceinline__ static constexpr int role(int a, const DevModel &) { return sig_role(R_, a); }
    __device__ __forceinline__ static constexpr int slot(int a, const DevModel &) { return sig_slot(R_, a); }
    __device__ __forceinline__ static int kk(const DevModel &) { return K; }
};

// Run-time signature for any other model (up to MD_MAX_SITES sites).
struct SigDyn {
    static constexpr int S = MD_MAX_SITES;
    static constexpr bool DYN = true;
    static constexpr bool SINGLE = false;
    __device__ __forceinline__ static int role(int a, const DevModel &m) { return a < m.S ? m.roles[a] : 0; }
    __device__ __forceinline__ static int slot(int a, const DevModel &m) { return m.axis_slot[a]; }
    __device__ __forceinline__ static int kk(const DevModel &m) { return m.S + m.NA; }
};

// Offset of the axis block inside a molecule's geo record.
template <class SIG>
__device__ __forceinline__ int S_of(const DevModel &m)
{
    return SIG::DYN ? m.S : SIG::S;
}

// Electrostatic interaction of site a (on i) with site b (on j), §2
// multipole laws with k_C = 1.  x = r_a - r_b, ir = 1/|x|.  Adds the
// energy, the force on a and the orientation torques (e x -dU/de).
// Laws in terms of pa = e_a.xh, pb = e_b.xh, cab = e_a.e_b:
//   q q: 1/r;  q mu: pb/r^2;  mu q: -pa/r^2;  mu mu: (cab - 3 pa pb)/r^3;
//   q Q: (3 pb^2 - 1)/(2 r^3);  Q q: (3 pa^2 - 1)/(2 r^3);
//   mu Q: 3/(2 r^4) [-pa (5 pb^2 - 1) + 2 pb cab];
//   Q mu: 3/(2 r^4) [pb (5 pa^2 - 1) - 2 pa cab];
//   Q Q: 3/(4 r^5) [1 - 5 pa^2 - 5 pb^2 - 15 pa^2 pb^2 + 2 (cab - 5 pa pb)^2];
//   reaction field (dipole pairs): -f_RF mu mu cab / rc^3.
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
    const float u2 = ir * ir, u3 = u2 * ir;
    float Ut = 0.f, nU = 0.f, Upa = 0.f, Upb = 0.f, Ucab = 0.f;
    if ((ra & ROLE_CHG) && (rb & ROLE_CHG)) {
        const float t = qa * qb * ir;
        Ut += t;
        nU += t;
    }
    if ((ra & ROLE_CHG) && (rb & ROLE_DIP)) {
        const float s = qa * mub * u2;
        const float t = s * pb;
        Ut += t;
        nU += 2.f * t;
        Upb += s;
    }
    if ((ra & ROLE_DIP) && (rb & ROLE_CHG)) {
        const float s = mua * qb * u2;
        const float t = -s * pa;
        Ut += t;
        nU += 2.f * t;
        Upa -= s;
    }
    if ((ra & ROLE_DIP) && (rb & ROLE_DIP)) {
        const float s = mua * mub * u3;
        const float t = s * (cab - 3.f * pa * pb);
        Ut += t;
        nU += 3.f * t;
        Upa -= 3.f * s * pb;
        Upb -= 3.f * s * pa;
        Ucab += s;
        const float sr = mua * mub * frf;
        Ut -= sr * cab;
        Ucab -= sr;
    }
    if ((ra & ROLE_CHG) && (rb & ROLE_QUAD)) {
        const float s = qa * Qb * u3;
        const float t = 0.5f * s * (3.f * pb * pb - 1.f);
        Ut += t;
        nU += 3.f * t;
        Upb += 3.f * s * pb;
    }
    if ((ra & ROLE_QUAD) && (rb & ROLE_CHG)) {
        const float s = Qa * qb * u3;
        const float t = 0.5f * s * (3.f * pa * pa - 1.f);
        Ut += t;
        nU += 3.f * t;
        Upa += 3.f * s * pa;
    }
    if ((ra & ROLE_DIP) && (rb & ROLE_QUAD)) {
        const float c = 1.5f * mua * Qb * u2 * u2;
        const float t = c * (2.f * pb * cab - pa * (5.f * pb * pb - 1.f));
        Ut += t;
        nU += 4.f * t;
        Upa += c * (1.f - 5.f * pb * pb);
        Upb += c * (2.f * cab - 10.f * pa * pb);
        Ucab += 2.f * c * pb;
    }
    if ((ra & ROLE_QUAD) && (rb & ROLE_DIP)) {
        const float c = 1.5f * Qa * mub * u2 * u2;
        const float t = c * (pb * (5.f * pa * pa - 1.f) - 2.f * pa * cab);
        Ut += t;
        nU += 4.f * t;
        Upb += c * (5.f * pa * pa - 1.f);
        Upa += c * (10.f * pa * pb - 2.f * cab);
        Ucab -= 2.f * c * pa;
    }
    if ((ra & ROLE_QUAD) && (rb & ROLE_QUAD)) {
        const float c = 0.75f * Qa * Qb * u2 * u3;
        const float pa2 = pa * pa, pb2 = pb * pb;
        const float tt = cab - 5.f * pa * pb;
        const float B = 1.f - 5.f * (pa2 + pb2) - 15.f * pa2 * pb2 + 2.f * tt * tt;
        Ut += c * B;
        nU += 5.f * c * B;
        Upa -= c * (10.f * pa + 30.f * pa * pb2 + 20.f * pb * tt);
        Upb -= c * (10.f * pb + 30.f * pa2 * pb + 20.f * pa * tt);
        Ucab += 4.f * c * tt;
    }
    U += Ut;
    // dU/dx = xh (Ur - (Upa pa + Upb pb)/r) + (Upa e_a + Upb e_b)/r, Ur = -nU/r
    const float cx = -(nU + Upa * pa + Upb * pb) * ir;
    const float ua = Upa * ir, ub = Upb * ir;
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
        ti[0] -= Upa * (ea.y * zh - ea.z * yh) + Ucab * cex;
        ti[1] -= Upa * (ea.z * xh - ea.x * zh) + Ucab * cey;
        ti[2] -= Upa * (ea.x * yh - ea.y * xh) + Ucab * cez;
    }
    if (JSIDE && axb) {  // e_b x (-(Upb xh + Ucab e_a))
        tj[0] += -Upb * (eb.y * zh - eb.z * yh) + Ucab * cex;
        tj[1] += -Upb * (eb.z * xh - eb.x * zh) + Ucab * cey;
        tj[2] += -Upb * (eb.x * yh - eb.y * xh) + Ucab * cez;
    }
}

// Interaction of molecule i with molecule j at centre-of-mass separation
// X = R_i - R_j (inside the cut-off): all site pairs.  Accumulates the
// per-site forces on i (fa), i's orientation torque (ti), energy and
// virial; with JSIDE also j's torque (tj) and returns the total force on i.
template <class SIG, bool JSIDE>
__device__ __forceinline__ void mol_pair(const DevModel &m, const float X0, const float X1, const float X2,
                                         const float (&di)[SIG::S][3], const float4 (&ei)[SIG::S],
                                         const float4 *__restrict__ gj, const int K, float (&fa)[SIG::S][3],
                                         float (&ti)[3], float &uacc, float &wacc, float (&wd)[3], float (&Fij)[3],
                                         float (&tj)[3])
{
    constexpr int S = SIG::S;
    float Fx = 0.f, Fy = 0.f, Fz = 0.f, U = 0.f;
    if (JSIDE) tj[0] = tj[1] = tj[2] = 0.f;
    if (SIG::SINGLE) {
        const float r2 = X0 * X0 + X1 * X1 + X2 * X2;
        const float ir2 = __fdividef(1.f, r2);
        const float s2 = m.sig2[0][0] * ir2;
        const float s6 = s2 * s2 * s2;
        const float fr = m.eps24[0][0] * s6 * (2.f * s6 - 1.f) * ir2;
        U = m.eps4[0][0] * s6 * (s6 - 1.f) - m.ushift[0][0];
        Fx = fr * X0;
        Fy = fr * X1;
        Fz = fr * X2;
        fa[0][0] += Fx;
        fa[0][1] += Fy;
        fa[0][2] += Fz;
    } else {
#pragma unroll
        for (int b = 0; b < S; b++) {
            const int rb = SIG::role(b, m);
            if (rb == 0) continue;
            const float4 db = __ldg(gj + b);
            float4 eb = make_float4(0.f, 0.f, 0.f, 0.f);
            if (rb & AX_ROLES) eb = __ldg(gj + S_of<SIG>(m) + SIG::slot(b, m));
            float fbx = 0.f, fby = 0.f, fbz = 0.f;
#pragma unroll
            for (int a = 0; a < S; a++) {
                const int ra = SIG::role(a, m);
                const bool lj = (ra & ROLE_LJ) && (rb & ROLE_LJ);
                const bool el = (ra & EL_ROLES) && (rb & EL_ROLES);
                if (!lj && !el) continue;
                const float x = X0 + di[a][0] - db.x;
                const float y = X1 + di[a][1] - db.y;
                const float z = X2 + di[a][2] - db.z;
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
                    const int ta = m.lj_type[a], tb = m.lj_type[b];
                    const float s2 = m.sig2[ta][tb] * ir2;
                    const float s6 = s2 * s2 * s2;
                    const float fr = m.eps24[ta][tb] * s6 * (2.f * s6 - 1.f) * ir2;
                    U += m.eps4[ta][tb] * s6 * (s6 - 1.f) - m.ushift[ta][tb];
                    fx = fr * x;
                    fy = fr * y;
                    fz = fr * z;
                }
                if (el) {
                    elec_site<JSIDE>(ra, rb, m.chg[a], m.mu[a], m.Q[a], m.chg[b], m.mu[b], m.Q[b], m.frf, x, y, z,
                                     ir, ei[a], eb, U, fx, fy, fz, ti, tj);
                }
                fa[a][0] += fx;
                fa[a][1] += fy;
                fa[a][2] += fz;
                fbx += fx;
                fby += fy;
                fbz += fz;
            }
            Fx += fbx;
            Fy += fby;
            Fz += fbz;
            if (JSIDE) {  // lever arm of site b: d_b x (-f_b)
                tj[0] -= db.y * fbz - db.z * fby;
                tj[1] -= db.z * fbx - db.x * fbz;
                tj[2] -= db.x * fby - db.y * fbx;
            }
        }
    }
    uacc += U;
    wacc += X0 * Fx + X1 * Fy + X2 * Fz;
    wd[0] += X0 * Fx;
    wd[1] += X1 * Fy;
    wd[2] += X2 * Fz;
    Fij[0] = Fx;
    Fij[1] = Fy;
    Fij[2] = Fz;
}

// ---------------------------------------------------------------- kernel
// FP64 re-test of a pair whose FP32 squared distance fell inside the guard
// band: minimum image through the known periodic shift of j's cell.
__device__ __noinline__ bool recheck64(const ForceArgs &A, int si, int jj, int kx, int ky, int kz)
{
    const double *ri = A.r + 3LL * si, *rj = A.r + 3LL * jj;
    const double d0 = __dsub_rn(__dsub_rn(ri[0], rj[0]), (double)kx * A.g.L[0]);
    const double d1 = __dsub_rn(__dsub_rn(ri[1], rj[1]), (double)ky * A.g.L[1]);
    const double d2 = __dsub_rn(__dsub_rn(ri[2], rj[2]), (double)kz * A.g.L[2]);
    const double s = __dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)), __dmul_rn(d2, d2));
    return s < A.g.rc2;
}

template <class SIG, bool HALF>
__global__ void __launch_bounds__(MD_WARPS * 32) k_force(const __grid_constant__ ForceArgs A)
{
    constexpr int S = SIG::S;
    constexpr unsigned FULL = 0xffffffffu;
    __shared__ int s_hj[MD_WARPS][MD_HIT_CAP][32];
    __shared__ unsigned char s_ho[MD_WARPS][MD_HIT_CAP][32];
    __shared__ double s_red[MD_WARPS][P_COUNT];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const DevModel &m = A.m;
    const Grid &g = A.g;
    const int K = SIG::kk(m);
    const double esc = HALF ? 1.0 : 0.5;  // full shell visits every pair twice
    double accU = 0.0, accW = 0.0, accWd0 = 0.0, accWd1 = 0.0, accWd2 = 0.0, accNm = 0.0, accNe = 0.0;

    for (long long c = (long long)blockIdx.x * MD_WARPS + warp; c < g.ncell; c += (long long)gridDim.x * MD_WARPS) {
        const int s0 = A.cell_start[c];
        const int n_i = A.cell_start[c + 1] - s0;
        if (n_i == 0) continue;
        const int cx = (int)(c % g.nc[0]);
        const int cy = (int)((c / g.nc[0]) % g.nc[1]);
        const int cz = (int)(c / ((long long)g.nc[0] * g.nc[1]));
        for (int ib = 0; ib < n_i; ib += 32) {
            const int ng = min(32, n_i - ib);
            const int P = ng > 16 ? 32 : ng > 8 ? 16 : ng > 4 ? 8 : ng > 2 ? 4 : ng > 1 ? 2 : 1;
            const int G = 32 / P;
            const int il = lane & (P - 1), sub = lane / P;
            const bool act = il < ng;
            const int si = s0 + ib + (act ? il : 0);
            const float4 ci = A.com[si];
            float di[S][3];
            float4 ei[S];
#pragma unroll
            for (int a = 0; a < S; a++) {
                di[a][0] = di[a][1] = di[a][2] = 0.f;
                ei[a] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (!SIG::SINGLE && SIG::role(a, m)) {
                    const float4 t = A.geo[(long long)si * K + a];
                    di[a][0] = t.x;
                    di[a][1] = t.y;
                    di[a][2] = t.z;
                    if (SIG::role(a, m) & AX_ROLES) ei[a] = A.geo[(long long)si * K + S_of<SIG>(m) + SIG::slot(a, m)];
                }
            }
            float fa[S][3], ti[3] = {0.f, 0.f, 0.f}, uacc = 0.f, wacc = 0.f, wd[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int a = 0; a < S; a++) fa[a][0] = fa[a][1] = fa[a][2] = 0.f;
            int nmol = 0, nexam = 0, cnt = 0;
            const int NOFF = HALF ? 14 : 27;

            auto flush = [&]() {
                const int mx = __reduce_max_sync(FULL, cnt);
                for (int k = 0; k < mx; k++) {
                    if (k < cnt) {
                        const int jj = s_hj[warp][k][lane];
                        const int o = s_ho[warp][k][lane];
                        int dx, dy, dz;
                        if (HALF) {
                            dx = c_half[o][0];
                            dy = c_half[o][1];
                            dz = c_half[o][2];
                        } else {
                            dx = o % 3 - 1;
                            dy = (o / 3) % 3 - 1;
                            dz = o / 9 - 1;
                        }
                        const float4 cj = A.com[jj];
                        const float X0 = ci.x - (cj.x + dx * g.ellf[0]);
                        const float X1 = ci.y - (cj.y + dy * g.ellf[1]);
                        const float X2 = ci.z - (cj.z + dz * g.ellf[2]);
                        float Fij[3], tj[3];
                        mol_pair<SIG, HALF>(m, X0, X1, X2, di, ei, A.geo + (long long)jj * K, K, fa, ti, uacc, wacc,
                                            wd, Fij, tj);
                        nmol++;
                        if (HALF) {
                            double *Fj = A.F + 3LL * jj, *Tj = A.tau + 3LL * jj;
                            atomicAdd(Fj, -(double)Fij[0]);
                            atomicAdd(Fj + 1, -(double)Fij[1]);
                            atomicAdd(Fj + 2, -(double)Fij[2]);
                            atomicAdd(Tj, (double)tj[0]);
                            atomicAdd(Tj + 1, (double)tj[1]);
                            atomicAdd(Tj + 2, (double)tj[2]);
                        }
                    }
                }
                cnt = 0;
            };

            for (int o = 0; o < NOFF; o++) {
                int dx, dy, dz;
                if (HALF) {
                    dx = c_half[o][0];
                    dy = c_half[o][1];
                    dz = c_half[o][2];
                } else {
                    dx = o % 3 - 1;
                    dy = (o / 3) % 3 - 1;
                    dz = o / 9 - 1;
                }
                int nx = cx + dx, ny = cy + dy, nz = cz + dz, kx = 0, ky = 0, kz = 0;
                if (nx < 0) { nx += g.nc[0]; kx = -1; } else if (nx >= g.nc[0]) { nx -= g.nc[0]; kx = 1; }
                if (ny < 0) { ny += g.nc[1]; ky = -1; } else if (ny >= g.nc[1]) { ny -= g.nc[1]; ky = 1; }
                if (nz < 0) { nz += g.nc[2]; kz = -1; } else if (nz >= g.nc[2]) { nz -= g.nc[2]; kz = 1; }
                const long long cn = ((long long)nz * g.nc[1] + ny) * g.nc[0] + nx;
                const int j0 = A.cell_start[cn], j1 = A.cell_start[cn + 1];
                const float ox = dx * g.ellf[0], oy = dy * g.ellf[1], oz = dz * g.ellf[2];
                const bool self = (dx == 0 && dy == 0 && dz == 0);
                for (int jb = j0; jb < j1; jb += G) {
                    const int jj = jb + sub;
                    bool ok = act && jj < j1;
                    if (self) ok = ok && (HALF ? (jj > si) : (jj != si));
                    bool hit = false;
                    if (ok) {
                        nexam++;
                        const float4 cj = A.com[jj];
                        const float X0 = ci.x - (cj.x + ox);
                        const float X1 = ci.y - (cj.y + oy);
                        const float X2 = ci.z - (cj.z + oz);
                        const float d2 = X0 * X0 + X1 * X1 + X2 * X2;
                        hit = d2 < g.rc2f;
                        if (fabsf(d2 - g.rc2f) < g.bandf) hit = recheck64(A, si, jj, kx, ky, kz);
                    }
                    if (hit) {
                        s_hj[warp][cnt][lane] = jj;
                        s_ho[warp][cnt][lane] = (unsigned char)o;
                        cnt++;
                    }
                    if (__any_sync(FULL, cnt == MD_HIT_CAP)) flush();
                }
            }
            flush();

            // molecule totals: F_i = sum_a f_a, tau_i = sum_a d_a x f_a + orientation torque
            float Fi[3] = {0.f, 0.f, 0.f}, Ti[3] = {ti[0], ti[1], ti[2]};
#pragma unroll
            for (int a = 0; a < S; a++) {
                Fi[0] += fa[a][0];
                Fi[1] += fa[a][1];
                Fi[2] += fa[a][2];
                if (!SIG::SINGLE) {
                    Ti[0] += di[a][1] * fa[a][2] - di[a][2] * fa[a][1];
                    Ti[1] += di[a][2] * fa[a][0] - di[a][0] * fa[a][2];
                    Ti[2] += di[a][0] * fa[a][1] - di[a][1] * fa[a][0];
                }
            }
            for (int msk = P; msk < 32; msk <<= 1) {
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    Fi[k] += __shfl_xor_sync(FULL, Fi[k], msk);
                    Ti[k] += __shfl_xor_sync(FULL, Ti[k], msk);
                }
            }
            if (act && sub == 0) {
                double *Fo = A.F + 3LL * si, *To = A.tau + 3LL * si;
                if (HALF) {
                    for (int k = 0; k < 3; k++) {
                        atomicAdd(Fo + k, (double)Fi[k]);
                        atomicAdd(To + k, (double)Ti[k]);
                    }
                } else {
                    for (int k = 0; k < 3; k++) {
                        Fo[k] = (double)Fi[k];
                        To[k] = (double)Ti[k];
                    }
                }
                if (!(isfinite(Fi[0]) && isfinite(Fi[1]) && isfinite(Fi[2]) && isfinite(Ti[0]) && isfinite(Ti[1]) &&
                      isfinite(Ti[2])))
                    atomicExch(&A.flags[FLAG_NONFINITE], 1);
            }
            for (int msk = 1; msk < 32; msk <<= 1) {
                uacc += __shfl_xor_sync(FULL, uacc, msk);
                wacc += __shfl_xor_sync(FULL, wacc, msk);
                wd[0] += __shfl_xor_sync(FULL, wd[0], msk);
                wd[1] += __shfl_xor_sync(FULL, wd[1], msk);
                wd[2] += __shfl_xor_sync(FULL, wd[2], msk);
            }
            const int tm = __reduce_add_sync(FULL, nmol), te = __reduce_add_sync(FULL, nexam);
            accU += esc * (double)uacc;
            accW += esc * (double)wacc;
            accWd0 += esc * (double)wd[0];
            accWd1 += esc * (double)wd[1];
            accWd2 += esc * (double)wd[2];
            accNm += esc * (double)tm;
            accNe += esc * (double)te;
        }
    }
    if (lane == 0) {
        s_red[warp][P_U] = accU;
        s_red[warp][P_W] = accW;
        s_red[warp][P_WXX] = accWd0;
        s_red[warp][P_WYY] = accWd1;
        s_red[warp][P_WZZ] = accWd2;
        s_red[warp][P_NMOL] = accNm;
        s_red[warp][P_NSITE] = accNm * (double)m.site_pairs_per_mol_pair;
        s_red[warp][P_NEXAM] = accNe;
    }
    __syncthreads();
    if (threadIdx.x < P_COUNT) {
        double t = 0.0;
        for (int w = 0; w < MD_WARPS; w++) t += s_red[w][threadIdx.x];
        A.partials[(long long)blockIdx.x * P_COUNT + threadIdx.x] = t;
    }
}

template <class SIG>
cudaError_t launch_sig(const ForceArgs &A, int half, int n_blocks, cudaStream_t s)
{
    if (half)
        k_force<SIG, true><<<n_blocks, MD_WARPS * 32, 0, s>>>(A);
    else
        k_force<SIG, false><<<n_blocks, MD_WARPS * 32, 0, s>>>(A);
    return cudaGetLastError();
}

constexpr unsigned sigkey(int r0, int r1 = 0, int r2 = 0, int r3 = 0, int r4 = 0, int r5 = 0, int r6 = 0,
                          int r7 = 0)
{
    return (unsigned)r0 | ((unsigned)r1 << 4) | ((unsigned)r2 << 8) | ((unsigned)r3 << 12) | ((unsigned)r4 << 16) |
           ((unsigned)r5 << 20) | ((unsigned)r6 << 24) | ((unsigned)r7 << 28);
}

// Signatures compiled ahead of time; any other model runs SigDyn.
constexpr unsigned SIG_2CLJ = sigkey(ROLE_LJ, ROLE_LJ);
constexpr unsigned SIG_2CLJQ = sigkey(ROLE_LJ, ROLE_LJ, ROLE_QUAD);
constexpr unsigned SIG_2CLJDQ = sigkey(ROLE_LJ, ROLE_LJ, ROLE_DIP | ROLE_QUAD);
constexpr unsigned SIG_4SITE =
    sigkey(ROLE_LJ, ROLE_LJ | ROLE_CHG, ROLE_LJ | ROLE_CHG, ROLE_DIP, ROLE_QUAD);

}  // namespace

int force_blocks_default() { return 152 * 8; }

cudaError_t launch_force(const Grid &g, const DevModel &m, DevState &d, int half_shell, int n_blocks, cudaStream_t s)
{
    ForceArgs A;
    A.g = g;
    A.m = m;
    A.cell_start = d.cell_start;
    A.com = d.com;
    A.geo = d.geo;
    A.r = d.r;
    A.F = d.F;
    A.tau = d.tau;
    A.partials = d.partials;
    A.flags = d.flags;
    if (half_shell) {
        cudaError_t e = cudaMemsetAsync(d.F, 0, sizeof(double) * 3 * (d.n > 0 ? d.n : 1), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(d.tau, 0, sizeof(double) * 3 * (d.n > 0 ? d.n : 1), s);
        if (e != cudaSuccess) return e;
    }
    unsigned key = 0;
    for (int a = 0; a < m.S; a++) key |= (unsigned)m.roles[a] << (4 * a);
    if (m.single_lj_at_com) return launch_sig<SigStatic<1, ROLE_LJ, true>>(A, half_shell, n_blocks, s);
    if (m.S == 2 && key == SIG_2CLJ) return launch_sig<SigStatic<2, SIG_2CLJ>>(A, half_shell, n_blocks, s);
    if (m.S == 3 && key == SIG_2CLJQ) return launch_sig<SigStatic<3, SIG_2CLJQ>>(A, half_shell, n_blocks, s);
    if (m.S == 3 && key == SIG_2CLJDQ) return launch_sig<SigStatic<3, SIG_2CLJDQ>>(A, half_shell, n_blocks, s);
    if (m.S == 5 && key == SIG_4SITE) return launch_sig<SigStatic<5, SIG_4SITE>>(A, half_shell, n_blocks, s);
    return launch_sig<SigDyn>(A, half_shell, n_blocks, s);
}
