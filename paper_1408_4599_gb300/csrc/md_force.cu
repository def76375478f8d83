// md_force.cu -- linked-cell force / torque / energy / virial kernel (§3:
// force and torque calculation over the 27-cell stencil or the 14-cell
// Newton-3 stencil, then summation per molecule) for rigid molecules of LJ
// centres and point charges, dipoles and linear quadrupoles (§2).
//
// GB300 design (CUDA cores -- this is not a dense contraction):
//   * traversal of md_pair.cuh: one warp per i-cell, candidates staged in
//     shared memory, FP32 cut-off test with an FP64 re-test in a narrow band,
//     hits compacted into 32-pair chunks of one i molecule;
//   * FP32 site-site math (rsqrt/rcp on the MUFU pipe);
//   * i side: per-lane FP32 partials, one warp reduction per i, per-pass
//     totals in shared memory;
//   * Newton-3 side (half shell): the j's of a chunk are distinct, so the
//     reactions go into per-warp shared accumulators with plain adds; each
//     segment is flushed to global FP32 accumulators (one red per value per
//     staged candidate) and a finalize kernel converts them to FP64;
//   * full shell: each ordered pair from both sides, plain FP64 stores of
//     the per-molecule totals, bitwise deterministic;
//   * no FP64 arithmetic per pair: GB300's FP64 rate is ~1/70 of FP32.
#include "md_pair.cuh"

using namespace mdk;

namespace {

struct ForceArgs {
    Grid g;
    DevModel m;
    const int *cell_start;
    const float4 *com;
    const float4 *geo;
    const double *r;
    double *F, *tau;  // outputs (FP64, storage order)
    float *acc;       // half shell: 6 x n FP32 accumulators (SoA)
    long long n;
    double *partials;
    int *flags;
};

template <bool HALF>
struct ForceExtra {
    float jacc[HALF ? 6 : 1][JCAP];  // Newton-3 reactions: F (3), tau (3)
    float ipart[32][6];              // i totals of the pass: F (3), tau (3)
};

template <class SIG, bool HALF>
struct ForceOp {
    static constexpr int IMAX = 32;
    using Tile = WarpTile<ForceExtra<HALF>>;
    const DevModel &m;
    const ForceArgs &A;
    int K;
    int ig;
    float pF0, pF1, pF2, pT0, pT1, pT2;
    float cU, cW, cX, cY, cZ;                      // pass sums of energy and virial (FP32)
    float sU, kU, sW, kW, sX, kX, sY, kY, sZ, kZ;  // compensated lane totals
    int nmol, nexam;
    Tile *T;

    __device__ ForceOp(const DevModel &m_, const ForceArgs &A_, int K_, Tile *T_) : m(m_), A(A_), K(K_), T(T_)
    {
        sU = kU = sW = kW = sX = kX = sY = kY = sZ = kZ = 0.f;
        nmol = nexam = 0;
    }
    __device__ void pass_begin(int ig_, int ni, int lane)
    {
        ig = ig_;
        for (int t = lane; t < ni * 6; t += 32) (&T->x.ipart[0][0])[t] = 0.f;
        cU = cW = cX = cY = cZ = 0.f;
    }
    __device__ void seg_begin(Tile &TT, int nj, int lane)
    {
        if (HALF)
            for (int t = lane; t < nj; t += 32)
#pragma unroll
                for (int q = 0; q < 6; q++) TT.x.jacc[q][t] = 0.f;
    }
    __device__ void i_begin(const IMol<SIG> &, int) { pF0 = pF1 = pF2 = pT0 = pT1 = pT2 = 0.f; }
    __device__ void count_examined(int n) { nexam += n; }
    __device__ void pair(Tile &TT, const IMol<SIG> &I, int k, float X0, float X1, float X2, int js, int)
    {
        float Fp[3], tp[3], tq[3], Up;
        mol_pair<SIG, HALF>(m, X0, X1, X2, I, A.geo + (long long)js * K, Fp, tp, tq, Up);
        pF0 += Fp[0];
        pF1 += Fp[1];
        pF2 += Fp[2];
        pT0 += tp[0];
        pT1 += tp[1];
        pT2 += tp[2];
        cU += Up;
        cW += X0 * Fp[0] + X1 * Fp[1] + X2 * Fp[2];
        cX += X0 * Fp[0];
        cY += X1 * Fp[1];
        cZ += X2 * Fp[2];
        nmol++;
        if (HALF) {
            TT.x.jacc[0][k] -= Fp[0];
            TT.x.jacc[1][k] -= Fp[1];
            TT.x.jacc[2][k] -= Fp[2];
            TT.x.jacc[3][k] += tq[0];
            TT.x.jacc[4][k] += tq[1];
            TT.x.jacc[5][k] += tq[2];
        }
    }
    __device__ void i_end(const IMol<SIG> &, int il, int lane)
    {
        for (int msk = 16; msk > 0; msk >>= 1) {
            pF0 += __shfl_xor_sync(FULLMASK, pF0, msk);
            pF1 += __shfl_xor_sync(FULLMASK, pF1, msk);
            pF2 += __shfl_xor_sync(FULLMASK, pF2, msk);
            pT0 += __shfl_xor_sync(FULLMASK, pT0, msk);
            pT1 += __shfl_xor_sync(FULLMASK, pT1, msk);
            pT2 += __shfl_xor_sync(FULLMASK, pT2, msk);
        }
        if (lane == 0) {
            float *ip = T->x.ipart[il - ig];
            ip[0] += pF0;
            ip[1] += pF1;
            ip[2] += pF2;
            ip[3] += pT0;
            ip[4] += pT1;
            ip[5] += pT2;
        }
    }
    __device__ void seg_end(Tile &TT, int nj, int lane)
    {
        if (HALF)
            for (int t = lane; t < nj; t += 32) {
                const int js = __float_as_int(TT.jc[t].w);
#pragma unroll
                for (int q = 0; q < 6; q++) atomicAdd(A.acc + (long long)q * A.n + js, TT.x.jacc[q][t]);
            }
    }
    __device__ void pass_end(int s0, int ig_, int ni, int lane)
    {
        for (int t = lane; t < ni; t += 32) {
            const int si = s0 + ig_ + t;
            const float *ip = T->x.ipart[t];
            if (HALF) {
#pragma unroll
                for (int q = 0; q < 6; q++) atomicAdd(A.acc + (long long)q * A.n + si, ip[q]);
            } else {
                double *Fo = A.F + 3LL * si, *To = A.tau + 3LL * si;
                Fo[0] = ip[0];
                Fo[1] = ip[1];
                Fo[2] = ip[2];
                To[0] = ip[3];
                To[1] = ip[4];
                To[2] = ip[5];
                if (!(isfinite(ip[0]) && isfinite(ip[1]) && isfinite(ip[2]) && isfinite(ip[3]) && isfinite(ip[4]) &&
                      isfinite(ip[5])))
                    atomicExch(&A.flags[FLAG_NONFINITE], 1);
            }
        }
        kahan_add(sU, kU, cU);
        kahan_add(sW, kW, cW);
        kahan_add(sX, kX, cX);
        kahan_add(sY, kY, cY);
        kahan_add(sZ, kZ, cZ);
    }
};

template <class SIG, bool HALF>
__global__ void __launch_bounds__(MD_WARPS * 32) k_force(const __grid_constant__ ForceArgs A)
{
    using Op = ForceOp<SIG, HALF>;
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
    Op op(m, A, K, T);
    for (long long c = (long long)blockIdx.x * MD_WARPS + warp; c < A.g.ncell; c += (long long)gridDim.x * MD_WARPS)
        traverse_cell<SIG, HALF>(m, gv, A.cell_start, A.com, A.geo, A.r, K, c, *T, op, lane);

    // block partials: FP32 warp sums of the compensated lane sums; FP64 only
    // once per value per block
    float v[5] = {op.sU - op.kU, op.sW - op.kW, op.sX - op.kX, op.sY - op.kY, op.sZ - op.kZ};
    for (int q = 0; q < 5; q++)
        for (int msk = 16; msk > 0; msk >>= 1) v[q] += __shfl_xor_sync(FULLMASK, v[q], msk);
    const int wm = __reduce_add_sync(FULLMASK, op.nmol), we = __reduce_add_sync(FULLMASK, op.nexam);
    __shared__ float s_red[MD_WARPS][5];
    __shared__ long long s_cnt[MD_WARPS][2];
    if (lane == 0) {
        for (int q = 0; q < 5; q++) s_red[warp][q] = v[q];
        s_cnt[warp][0] = wm;
        s_cnt[warp][1] = we;
    }
    __syncthreads();
    if (threadIdx.x < P_COUNT) {
        const double esc = HALF ? 1.0 : 0.5;  // the full shell visits every pair twice
        const int q = threadIdx.x;
        double t = 0.0;
        for (int w = 0; w < MD_WARPS; w++) {
            if (q == P_NMOL || q == P_NSITE) t += (double)s_cnt[w][0];
            else if (q == P_NEXAM) t += (double)s_cnt[w][1];
            else t += (double)s_red[w][q];
        }
        if (q == P_NSITE) t *= (double)m.site_pairs_per_mol_pair;
        A.partials[(long long)blockIdx.x * P_COUNT + q] = esc * t;
    }
}

// Half shell: FP32 accumulators (SoA) -> FP64 F, tau; non-finite check.
__global__ void k_force_finalize(const float *acc, long long n, double *F, double *tau, int *flags)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    bool bad = false;
    for (int q = 0; q < 3; q++) {
        const float f = acc[q * n + s], t = acc[(q + 3) * n + s];
        bad |= !isfinite(f) || !isfinite(t);
        F[3 * s + q] = (double)f;
        tau[3 * s + q] = (double)t;
    }
    if (bad) atomicExch(&flags[FLAG_NONFINITE], 1);
}

struct LaunchForce {
    const ForceArgs &A;
    int half, n_blocks;
    cudaStream_t s;
    template <class SIG>
    cudaError_t operator()() const
    {
        if (half) return run<SIG, true>();
        return run<SIG, false>();
    }
    // persistent grid: as many blocks as can be resident (grid-stride over
    // cells), never more than the cells need nor than the partials hold
    template <class SIG, bool HALF>
    cudaError_t run() const
    {
        const size_t sm = sizeof(typename ForceOp<SIG, HALF>::Tile) * MD_WARPS;
        cudaFuncSetAttribute(k_force<SIG, HALF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        int per_sm = 0, dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_force<SIG, HALF>, MD_WARPS * 32, sm);
        long long want = (long long)(per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
        const long long need = (A.g.ncell + MD_WARPS - 1) / MD_WARPS;
        if (want > need) want = need;
        if (want > n_blocks) want = n_blocks;
        if (want < 1) want = 1;
        k_force<SIG, HALF><<<(unsigned)want, MD_WARPS * 32, sm, s>>>(A);
        return cudaGetLastError();
    }
};

}  // namespace

int force_blocks_default() { return 152 * 16; }

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
    A.acc = d.facc;
    A.n = d.n;
    A.partials = d.partials;
    A.flags = d.flags;
    // the grid may be smaller than the partials buffer: unused slots read as 0
    cudaError_t e = cudaMemsetAsync(d.partials, 0, sizeof(double) * P_COUNT * n_blocks, s);
    if (e != cudaSuccess) return e;
    if (half_shell) {
        e = cudaMemsetAsync(d.facc, 0, sizeof(float) * 6 * (d.n > 0 ? d.n : 1), s);
        if (e != cudaSuccess) return e;
    }
    e = dispatch_sig(m, LaunchForce{A, half_shell, n_blocks, s});
    if (e != cudaSuccess || !half_shell || d.n == 0) return e;
    k_force_finalize<<<(unsigned)((d.n + 255) / 256), 256, 0, s>>>(d.facc, d.n, d.F, d.tau, d.flags);
    return cudaGetLastError();
}
