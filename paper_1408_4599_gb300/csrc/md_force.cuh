// md_force.cuh -- linked-cell force / torque / energy / virial kernel (§3:
// force and torque calculation over the 27-cell stencil or the 14-cell
// Newton-3 stencil of cells of edge >= r_c, or the 125- / 63-cell stencils
// of cells of edge >= r_c / 2, then summation per molecule) for rigid
// molecules of LJ centres and point charges, dipoles and linear quadrupoles
// (§2).
//
// GB300 design (CUDA cores -- this is not a dense contraction):
//   * traversal of md_pair.cuh: one warp per i-cell (cells handed out from
//     a counter, or by a fixed grid stride in deterministic runs),
//     candidates staged in shared memory (with their axes, for linear
//     molecules in the half shell), FP32 cut-off test of two i molecules
//     per paired instruction with the FP64 decision in a narrow band;
//   * FP32 site-site math (rsqrt/rcp on the MUFU pipe, f32x2 where the
//     math pairs up);
//   * half shell (Newton-3), cells of edge >= r_c: the hits of a pass
//     collect in a queue drained in runs, one per lane; a lane keeps its i
//     molecule's sums in registers while the i stays the same and adds
//     them to the i's FP32 accumulator record once per run segment, and
//     adds each pair's reaction to the j record (16-byte vector
//     reductions); cells of edge >= r_c / 2 and the batched replicas keep
//     the chunked form (per-pair reductions on both records).  The records
//     are cleared by the rebuild that precedes the kernel (else by a
//     memset), read directly by the integrator and converted to FP64 only
//     on demand;
//   * full shell: each ordered pair from both sides, a segmented warp sum
//     per chunk into per-pass i totals in shared memory, plain FP64 stores of
//     the per-molecule totals, bitwise deterministic;
//   * no FP64 arithmetic per pair: GB300's FP64 rate is ~1/64 of FP32.
#pragma once

#include "md_forceop.cuh"

// Instantiated by md_force_inst.cu, which build.py compiles once per
// compiled signature and stencil radius (one kernel pair per object, all
// compiled in parallel); md_force.cu sees only the declaration of
// launch_force_sig in md_forceop.cuh.
namespace {

using namespace mdk;

// Resident blocks the register budget is sized for: 4 blocks of 4 warps (at
// most 128 registers) for models of up to 3 merged sites (the run-drained
// half shell keeps its i molecule and i sums in registers across the run and
// spills under the 102-register cap of 5 blocks; 3 blocks measured 8% slower
// on the 2CLJQ fluid); 5 for single-site LJ in the half shell (96 registers
// without spills, and its compact tile fits five blocks' shared memory:
// 2.5-5% faster than 4); 3 (168) for the larger compiled signatures, whose
// site loops spill at 128 registers; 2 for the run-time signature.
template <class SIG, bool HALF>
constexpr int force_min_blocks()
{
    return SIG::DYN ? 2 : (SIG::S > 3 ? 3 : (SIG::SINGLE && HALF ? 5 : 4));
}

// Dynamic shared memory of one block: the warps' tiles, then (M = 2) their
// stencil tables.
template <class SIG, bool HALF, int M>
constexpr size_t force_smem()
{
    return sizeof(typename ForceOp<SIG, HALF, M == 1>::Tile) * MD_WARPS + (M == 2 ? sizeof(StencilMeta) * MD_WARPS : 0);
}

// M: stencil radius in cells (1: cells of edge >= r_c; 2: >= r_c / 2).
template <class SIG, bool HALF, int M>
__global__ void __launch_bounds__(MD_WARPS * 32, force_min_blocks<SIG, HALF>()) k_force(const __grid_constant__ ForceArgs A)
{
    // cells of edge >= r_c / 2 hold ~2 molecules: the chunked half shell
    // (the run-drained form's per-window costs measured 2.5-5.6x slower there)
    using Op = ForceOp<SIG, HALF, M == 1>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    typename Op::Tile *T = reinterpret_cast<typename Op::Tile *>(smem_raw) + warp;
    StencilMeta *meta = nullptr;
    if (M == 2) meta = reinterpret_cast<StencilMeta *>(smem_raw + sizeof(typename Op::Tile) * MD_WARPS) + warp;
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
    if (A.parts > 1) {
        for_each_cell(A.g.ncell, A.parts, A.cell_ctr, warp, lane, [&](long long c, int p) {
            traverse_cell<SIG, HALF, M>(m, gv, A.cell_start, A.com, A.geo, A.r, K, c, *T, op, lane, meta, p, A.parts);
        });
    } else {  // whole cells: the traversal with a constant share (the common case, kept free of the split)
        for_each_cell(A.g.ncell, 1, A.cell_ctr, warp, lane, [&](long long c, int) {
            traverse_cell<SIG, HALF, M>(m, gv, A.cell_start, A.com, A.geo, A.r, K, c, *T, op, lane, meta);
        });
    }

    // block partials: FP64 warp sums of the lanes' FP64 totals
    double v[5] = {op.total(0), op.total(1), op.total(2), op.total(3), op.total(4)};
    for (int q = 0; q < 5; q++)
        for (int msk = 16; msk > 0; msk >>= 1) v[q] += __shfl_xor_sync(FULLMASK, v[q], msk);
    const int wm = __reduce_add_sync(FULLMASK, op.nmol), we = __reduce_add_sync(FULLMASK, op.nexam);
    __shared__ double s_red[MD_WARPS][5];
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

// Persistent grid: as many blocks as can be resident, never more than the
// units of work need nor than the partials hold.  With cells handed out
// from the counter and fewer than half as many cells as resident warps
// (small systems), each cell's i molecules are split into up to
// FORCE_MAX_PARTS units so that more warps share the work; deterministic
// runs keep one unit per cell (the split changes the FP32 summation
// grouping).
constexpr int FORCE_MAX_PARTS = 4;

template <class SIG, bool HALF, int M>
cudaError_t run_force(const ForceArgs &A, int n_blocks, cudaStream_t s)
{
    const size_t sm = force_smem<SIG, HALF, M>();
    cudaFuncSetAttribute(k_force<SIG, HALF, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int per_sm = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_force<SIG, HALF, M>, MD_WARPS * 32, sm);
    long long want = (long long)(per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
    ForceArgs B = A;
    B.parts = 1;
    if (B.cell_ctr && A.g.ncell > 0) {
        const long long p = 2 * want * MD_WARPS / A.g.ncell;
        B.parts = (int)(p < 1 ? 1 : (p > FORCE_MAX_PARTS ? FORCE_MAX_PARTS : p));
    }
    const long long need = (A.g.ncell * B.parts + MD_WARPS - 1) / MD_WARPS;
    if (want > need) want = need;
    if (want > n_blocks) want = n_blocks;
    if (want < 1) want = 1;
    k_force<SIG, HALF, M><<<(unsigned)want, MD_WARPS * 32, sm, s>>>(B);
    return cudaGetLastError();
}

}  // namespace

namespace mdk {

template <class SIG, int M>
cudaError_t launch_force_sig(const ForceArgs &A, int half_shell, int n_blocks, cudaStream_t s)
{
    return half_shell ? run_force<SIG, true, M>(A, n_blocks, s) : run_force<SIG, false, M>(A, n_blocks, s);
}

}  // namespace mdk
