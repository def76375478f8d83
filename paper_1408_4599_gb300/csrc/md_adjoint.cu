// md_adjoint.cu -- parameter sensitivities of the pair energy and the
// molecular virial for force-field fitting: for every interacting molecule
// pair the site-site terms are recomputed (nothing is stored from a forward
// pass) and their derivatives with respect to the LJ parameters (Eq. 1 with
// the §2 Lorentz-Berthelot rules) and the electrostatic strengths (§2) are
// accumulated.
//
// Per lane and per compiled site-role signature the kernel keeps:
//   * for every ordered pair of LJ sites (a, b): sum u/eps_ab, sum w/eps_ab,
//     sum du/dsigma_ab, sum dw/dsigma_ab  (u, w are linear in eps_ab);
//   * for every ordered pair of electrostatic entities (site, role): the
//     unit-strength energy and virial (the pair terms are bilinear in the
//     two strengths; the reaction field is part of the dipole-dipole law);
//   * the pair energy and virial themselves.
// The host applies the chain rule through the mixing rules and the
// strengths (md_api.cu, md_param_grad).  FP32 terms, FP32 per-lane sums,
// FP64 block partials.
#include "md_pair.cuh"

using namespace mdk;

namespace {

// electrostatic roles in entity order: charge, dipole, quadrupole
__host__ __device__ constexpr int role_order(int t) { return t == 0 ? ROLE_CHG : (t == 1 ? ROLE_DIP : ROLE_QUAD); }

// number of electrostatic entities (site, role) of a signature
__host__ __device__ constexpr int sig_ne(unsigned R, int S)
{
    int k = 0;
    for (int a = 0; a < S; a++)
        for (int t = 0; t < 3; t++) k += (sig_role(R, a) & role_order(t)) ? 1 : 0;
    return k;
}
// entity index of (site a, role t)
__host__ __device__ constexpr int sig_ent(unsigned R, int a, int t)
{
    int k = 0;
    for (int b = 0; b < a; b++)
        for (int u = 0; u < 3; u++) k += (sig_role(R, b) & role_order(u)) ? 1 : 0;
    for (int u = 0; u < t; u++) k += (sig_role(R, a) & role_order(u)) ? 1 : 0;
    return k;
}
__host__ __device__ constexpr int sig_nlj(unsigned R, int S)
{
    int k = 0;
    for (int a = 0; a < S; a++) k += (sig_role(R, a) & ROLE_LJ) ? 1 : 0;
    return k;
}
__host__ __device__ constexpr int sig_lj(unsigned R, int a)
{
    int k = 0;
    for (int b = 0; b < a; b++) k += (sig_role(R, b) & ROLE_LJ) ? 1 : 0;
    return k;
}

template <class SIG>
struct AdjLayout;

template <int S_, unsigned R_, bool SG_, unsigned TY_, bool LIN_, unsigned COM_>
struct AdjLayout<SigStatic<S_, R_, SG_, TY_, LIN_, COM_>> {
    static constexpr int NLJ = sig_nlj(R_, S_);
    static constexpr int NE = sig_ne(R_, S_);
    static constexpr int NACC = 4 * NLJ * NLJ + 2 * NE * NE + 2;  // + U, W
    __device__ static constexpr int lj(int a) { return sig_lj(R_, a); }
    __device__ static constexpr int ent(int a, int t) { return sig_ent(R_, a, t); }
};

struct AdjArgs {
    Grid g;
    DevModel m;
    const int *cell_start;
    const float4 *com;
    const float4 *geo;
    const double *r;
    double *partials;  // [block][NACC]
    int nacc;
    unsigned *cell_ctr;  // non-null: cells handed out from this counter
};

struct AdjExtra {
    char unused;
};

template <class SIG, bool HALF>
struct AdjOp {
    static constexpr int IMAX = 32;
    static constexpr bool RUNS = false;
    using Tile = WarpTile<AdjExtra>;
    using LY = AdjLayout<SIG>;
    static constexpr int S = SIG::S;
    const DevModel &m;
    const AdjArgs &A;
    int K;
    float acc[LY::NACC];
    int nexam;

    __device__ AdjOp(const DevModel &m_, const AdjArgs &A_, int K_) : m(m_), A(A_), K(K_)
    {
#pragma unroll
        for (int q = 0; q < LY::NACC; q++) acc[q] = 0.f;
        nexam = 0;
    }
    __device__ void pass_begin(int, int, int) {}
    __device__ void seg_begin(Tile &, int, int) {}
    __device__ void chunk_end(Tile &, int, int, bool, int) {}
    __device__ void seg_end(Tile &, int, int) {}
    __device__ void pass_end(int, int, int, int) {}
    __device__ void count_examined(int n) { nexam += n; }

    template <int L>
    __device__ __forceinline__ void el_term(int ia, int ib, float ir, float pa, float pb, float cab, float Xxh,
                                            float Xea, float Xeb, float sab, float &U, float &W)
    {
        const Law l = law<L>(ir, pa, pb, cab, m.frf);
        // virial of the unit-strength force: X . F1, F1 = -dU1/dx
        const float w1 = -(Xxh * (-(l.nU + l.Upa * pa + l.Upb * pb) * ir) + ir * (l.Upa * Xea + l.Upb * Xeb));
        acc[4 * LY::NLJ * LY::NLJ + 2 * (ia * LY::NE + ib)] += l.U;
        acc[4 * LY::NLJ * LY::NLJ + 2 * (ia * LY::NE + ib) + 1] += w1;
        U += sab * l.U;
        W += sab * w1;
    }

    __device__ void pair(Tile &, const IMol<SIG> &I, int, float X0, float X1, float X2, int js)
    {
        const float4 *gj = A.geo + (long long)js * K;
        float U = 0.f, W = 0.f;
        float4 uj = make_float4(0.f, 0.f, 0.f, 0.f);
        if constexpr (SIG::LIN) uj = __ldg(gj);  // the j molecule's axis
#pragma unroll
        for (int b = 0; b < S; b++) {
            const int rb = SIG::role(b, m);
            if (rb == 0) continue;
            float4 db = make_float4(0.f, 0.f, 0.f, 0.f), eb = db;
            if constexpr (SIG::LIN) {
                const float z = m.body[b][2], sb = m.axis[b][2];
                db = make_float4(z * uj.x, z * uj.y, z * uj.z, 0.f);
                if (rb & AX_ROLES) eb = make_float4(sb * uj.x, sb * uj.y, sb * uj.z, 0.f);
            } else {
                if (!SIG::SINGLE) db = __ldg(gj + b);
                if (rb & AX_ROLES) eb = __ldg(gj + SIG::s_of(m) + SIG::slot(b, m));
            }
#pragma unroll
            for (int a = 0; a < S; a++) {
                const int ra = SIG::role(a, m);
                const bool lj = (ra & ROLE_LJ) && (rb & ROLE_LJ);
                const bool el = (ra & EL_ROLES) && (rb & EL_ROLES);
                if (!lj && !el) continue;
                float da0, da1, da2;
                float4 ea;
                imol_site<SIG>(m, I, a, da0, da1, da2, ea);
                const float x = X0 + da0 - db.x;
                const float y = X1 + da1 - db.y;
                const float z = X2 + da2 - db.z;
                const float r2 = x * x + y * y + z * z;
                const float Xx = X0 * x + X1 * y + X2 * z;
                if (lj) {
                    const int ta = SIG::type(a, m), tb = SIG::type(b, m);
                    const float ir2 = __fdividef(1.f, r2);
                    const float s2 = m.sig2[ta][tb] * ir2;
                    const float s6 = s2 * s2 * s2, s12 = s6 * s6;
                    const float isig = m.isig[ta][tb];
                    const float u_e = 4.f * (s12 - s6) - m.ushift_e[ta][tb];     // u / eps_ab
                    const float w_e = 24.f * (2.f * s12 - s6) * ir2 * Xx;        // w / eps_ab
                    const float eps = 0.25f * m.eps4[ta][tb];
                    const float du_s = eps * (4.f * isig * (12.f * s12 - 6.f * s6) - m.dshift_s[ta][tb]);
                    const float dw_s = eps * 24.f * isig * (24.f * s12 - 6.f * s6) * ir2 * Xx;
                    const int p = 4 * (LY::lj(a) * LY::NLJ + LY::lj(b));
                    acc[p] += u_e;
                    acc[p + 1] += w_e;
                    acc[p + 2] += du_s;
                    acc[p + 3] += dw_s;
                    U += eps * u_e;
                    W += eps * w_e;
                }
                if (el) {
                    const float ir = rsqrtf(r2);
                    const float xh = x * ir, yh = y * ir, zh = z * ir;
                    const bool axa = (ra & AX_ROLES) != 0, axb = (rb & AX_ROLES) != 0;
                    const float pa = axa ? (ea.x * xh + ea.y * yh + ea.z * zh) : 0.f;
                    const float pb = axb ? (eb.x * xh + eb.y * yh + eb.z * zh) : 0.f;
                    const float cab = (axa && axb) ? (ea.x * eb.x + ea.y * eb.y + ea.z * eb.z) : 0.f;
                    const float Xxh = Xx * ir;
                    const float Xea = X0 * ea.x + X1 * ea.y + X2 * ea.z;
                    const float Xeb = X0 * eb.x + X1 * eb.y + X2 * eb.z;
                    if ((ra & ROLE_CHG) && (rb & ROLE_CHG))
                        el_term<LAW_QQ>(LY::ent(a, 0), LY::ent(b, 0), ir, pa, pb, cab, Xxh, Xea, Xeb, m.chg[a] * m.chg[b], U, W);
                    if ((ra & ROLE_CHG) && (rb & ROLE_DIP))
                        el_term<LAW_QMU>(LY::ent(a, 0), LY::ent(b, 1), ir, pa, pb, cab, Xxh, Xea, Xeb, m.chg[a] * m.mu[b], U, W);
                    if ((ra & ROLE_DIP) && (rb & ROLE_CHG))
                        el_term<LAW_MUQ>(LY::ent(a, 1), LY::ent(b, 0), ir, pa, pb, cab, Xxh, Xea, Xeb, m.mu[a] * m.chg[b], U, W);
                    if ((ra & ROLE_DIP) && (rb & ROLE_DIP))
                        el_term<LAW_MUMU>(LY::ent(a, 1), LY::ent(b, 1), ir, pa, pb, cab, Xxh, Xea, Xeb, m.mu[a] * m.mu[b], U, W);
                    if ((ra & ROLE_CHG) && (rb & ROLE_QUAD))
                        el_term<LAW_QQUAD>(LY::ent(a, 0), LY::ent(b, 2), ir, pa, pb, cab, Xxh, Xea, Xeb, m.chg[a] * m.Q[b], U, W);
                    if ((ra & ROLE_QUAD) && (rb & ROLE_CHG))
                        el_term<LAW_QUADQ>(LY::ent(a, 2), LY::ent(b, 0), ir, pa, pb, cab, Xxh, Xea, Xeb, m.Q[a] * m.chg[b], U, W);
                    if ((ra & ROLE_DIP) && (rb & ROLE_QUAD))
                        el_term<LAW_MUQUAD>(LY::ent(a, 1), LY::ent(b, 2), ir, pa, pb, cab, Xxh, Xea, Xeb, m.mu[a] * m.Q[b], U, W);
                    if ((ra & ROLE_QUAD) && (rb & ROLE_DIP))
                        el_term<LAW_QUADMU>(LY::ent(a, 2), LY::ent(b, 1), ir, pa, pb, cab, Xxh, Xea, Xeb, m.Q[a] * m.mu[b], U, W);
                    if ((ra & ROLE_QUAD) && (rb & ROLE_QUAD))
                        el_term<LAW_QUADQUAD>(LY::ent(a, 2), LY::ent(b, 2), ir, pa, pb, cab, Xxh, Xea, Xeb, m.Q[a] * m.Q[b], U, W);
                }
            }
        }
        acc[LY::NACC - 2] += U;
        acc[LY::NACC - 1] += W;
    }
};

template <class SIG, bool HALF>
__global__ void __launch_bounds__(MD_WARPS * 32) k_adjoint(const __grid_constant__ AdjArgs A)
{
    using Op = AdjOp<SIG, HALF>;
    using LY = AdjLayout<SIG>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    typename Op::Tile *T = reinterpret_cast<typename Op::Tile *>(smem_raw) + warp;
    const DevModel &m = A.m;
    const int K = SIG::kk(m);
    GridView gv;
    for (int k = 0; k < 3; k++) {
        gv.nc[k] = A.g.nc[k];
        gv.ellf[k] = A.g.ellf[k];
        gv.L[k] = A.g.L[k];
    }
    gv.rc2 = A.g.rc2;
    gv.rc2f = A.g.rc2f;
    gv.bandf = A.g.bandf;
    gv.cell0 = 0;
    Op op(m, A, K);
    for_each_cell(A.g.ncell, 1, A.cell_ctr, warp, lane, [&](long long c, int) {
        traverse_cell<SIG, HALF>(m, gv, A.cell_start, A.com, A.geo, A.r, K, c, *T, op, lane);
    });
    __shared__ float s_red[MD_WARPS][LY::NACC];
#pragma unroll
    for (int q = 0; q < LY::NACC; q++) {
        float v = op.acc[q];
        for (int msk = 16; msk > 0; msk >>= 1) v += __shfl_xor_sync(FULLMASK, v, msk);
        if (lane == 0) s_red[warp][q] = v;
    }
    __syncthreads();
    const double esc = HALF ? 1.0 : 0.5;
    for (int q = threadIdx.x; q < LY::NACC; q += blockDim.x) {
        double t = 0.0;
        for (int w = 0; w < MD_WARPS; w++) t += (double)s_red[w][q];
        A.partials[(long long)blockIdx.x * A.nacc + q] = esc * t;
    }
}

struct LaunchAdj {
    const AdjArgs &A;
    int half, n_blocks;
    cudaStream_t s;
    template <class SIG>
    cudaError_t operator()() const
    {
        if constexpr (SIG::DYN) {
            return cudaErrorNotSupported;
        } else {
            if (A.nacc != AdjLayout<SIG>::NACC) return cudaErrorInvalidValue;
            const size_t sm = sizeof(typename AdjOp<SIG, true>::Tile) * MD_WARPS;
            if (half)
                k_adjoint<SIG, true><<<n_blocks, MD_WARPS * 32, sm, s>>>(A);
            else
                k_adjoint<SIG, false><<<n_blocks, MD_WARPS * 32, sm, s>>>(A);
            return cudaGetLastError();
        }
    }
};

struct NaccOf {
    template <class SIG>
    int operator()() const
    {
        if constexpr (SIG::DYN)
            return -1;
        else
            return AdjLayout<SIG>::NACC;
    }
};

}  // namespace

// Accumulator count of the adjoint kernel for this model (-1: not compiled).
int adjoint_nacc(const DevModel &m) { return dispatch_sig(m, NaccOf{}); }

cudaError_t launch_adjoint(const Grid &g, const DevModel &m, const DevState &d, int half_shell, int dynamic_cells,
                           int n_blocks, double *partials, int nacc, cudaStream_t s)
{
    AdjArgs A;
    A.g = g;
    A.m = m;
    A.cell_start = d.cell_start;
    A.com = d.com;
    A.geo = d.geo;
    A.r = d.r;
    A.partials = partials;
    A.nacc = nacc;
    A.cell_ctr = dynamic_cells ? d.cell_ctr : nullptr;
    if (A.cell_ctr) {
        const cudaError_t e = cudaMemsetAsync(A.cell_ctr, 0, sizeof(unsigned), s);
        if (e != cudaSuccess) return e;
    }
    return dispatch_sig(m, LaunchAdj{A, half_shell, n_blocks, s});
}
