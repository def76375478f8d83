// md_forceop.cuh -- the force / torque / energy / virial pair operation of
// the linked-cell traversal (md_pair.cuh), shared by the single-system and
// the batched-replica force kernels.  See md_force.cuh for the design.
#pragma once

#include "md_pair.cuh"

namespace mdk {

struct ForceArgs {
    Grid g;
    DevModel m;
    const int *cell_start;
    const float4 *com;
    const float4 *geo;
    const double *r;
    double *F, *tau;  // outputs (FP64, storage order)
    float *acc;       // half shell: n x FACC_STRIDE FP32 accumulator records
    long long n;
    double *partials;
    int *flags;
    int to_acc;       // full shell: also accumulate into acc (batched replicas of mixed shells)
    unsigned *cell_ctr;  // non-null: cells are handed out one at a time from this counter
    int parts;           // each cell's i molecules split into this many units of work
};

// Launches the single-system force kernel (md_force.cuh) for signature SIG
// and stencil radius M (1: cells of edge >= r_c, 2: >= r_c / 2), half or
// full shell.  Defined in md_force.cuh and explicitly instantiated for every
// compiled signature by md_force_inst.cu.
template <class SIG, int M>
cudaError_t launch_force_sig(const ForceArgs &A, int half_shell, int n_blocks, cudaStream_t s);

struct ForceExtraHalf {
    double tot[5][32];  // per lane: FP64 totals of U, W, W_xx, W_yy, W_zz (FP32 pass sums added once per pass)
};
struct ForceExtra {
    double it[6][32];   // full shell: FP64 totals of F and tau of the pass's i molecules (FP32 chunk sums added)
    double tot[5][32];
};

// RUNS_: drain the half shell in runs (single systems); false keeps the
// chunked pipeline with per-pair reductions on both molecules, which the
// batched replicas use: their many small and dilute cells pay the larger
// staging area and the per-window drain of the run-drained form (measured
// 44% slower batched force evaluations).
template <class SIG, bool HALF, bool RUNS_ = HALF>
struct ForceOp {
    static constexpr int IMAX = 32;
    static constexpr int NQ = SIG::SINGLE ? 3 : 6;  // accumulated values per molecule: F, and tau unless single-site
    // the half shell is drained in runs (drain): a lane keeps its i's force
    // and torque in registers over consecutive pairs of that i
    static constexpr bool RUNS = HALF && RUNS_;
    // linear molecules stage the candidates' axes with their COMs (the
    // drained pairs then read no global memory); linear and single-site
    // molecules use the compact tile
    using Tile = std::conditional_t<RUNS, WarpTileD<ForceExtraHalf, QRUN, SIG::LIN && !SIG::DYN, (SIG::LIN || SIG::SINGLE) && !SIG::DYN>,
                                    WarpTile<ForceExtra, QCAP>>;
    // four blocks of the run-drained kernel fit an SM's shared memory
    static_assert(!RUNS || sizeof(Tile) * MD_WARPS <= 55 * 1024, "run-drained tile grew past 4 blocks per SM");
    const DevModel &m;
    const ForceArgs &A;
    int K;
    int ig;
    float pF0, pF1, pF2, pT0, pT1, pT2;            // the lane's pair of the current chunk (i side)
    float tq0, tq1, tq2;                           // its torque on j (half shell)
    int pjs, psi;                                  // storage slots of its j and i
    float cU, cW, cX, cY, cZ;                      // lane sums of energy and virial since the last FP64 flush
    int nmol, nexam, nflush;
    Tile *T;
    int ln;                                        // the lane (index of its compensated totals)

    // The compensated lane totals live in shared memory (T->x.tot), updated
    // once per pass, which keeps ten registers free for the pair math.
    __device__ ForceOp(const DevModel &m_, const ForceArgs &A_, int K_, Tile *T_) : m(m_), A(A_), K(K_), T(T_)
    {
        ln = threadIdx.x & 31;
        reset_totals();
    }
    __device__ void reset_totals()
    {
#pragma unroll
        for (int q = 0; q < 5; q++) T->x.tot[q][ln] = 0.0;
        cU = cW = cX = cY = cZ = 0.f;
        nmol = nexam = nflush = 0;
    }
    // the lane's total of value q (0 U, 1 W, 2 W_xx, 3 W_yy, 4 W_zz)
    __device__ double total(int q) const
    {
        const float c5[5] = {cU, cW, cX, cY, cZ};
        return T->x.tot[q][ln] + (double)c5[q];
    }
    __device__ void pass_begin(int ig_, int ni, int lane)
    {
        ig = ig_;
        if constexpr (!HALF) {  // the half shell sums its i terms while draining
            float *f = reinterpret_cast<float *>(&T->x.it[0][0]);  // FP32 view (to_acc)
            for (int t = lane; t < ni; t += 32)
#pragma unroll
                for (int q = 0; q < 6; q++) {
                    if (A.to_acc) f[q * 32 + t] = 0.f;
                    else T->x.it[q][t] = 0.0;
                }
        }
    }
    __device__ void seg_begin(Tile &, int, int) {}
    __device__ void count_examined(int n) { nexam += n; }
    __device__ void pair(Tile &, const IMol<SIG> &I, int, float X0, float X1, float X2, int js)
    {
        float Fp[3], tp[3], tq[3], Up;
        mol_pair<SIG, HALF>(m, X0, X1, X2, I, A.geo + (long long)js * K, Fp, tp, tq, Up);
        pF0 = Fp[0];
        pF1 = Fp[1];
        pF2 = Fp[2];
        pT0 = tp[0];
        pT1 = tp[1];
        pT2 = tp[2];
        cU += Up;
        cW += X0 * Fp[0] + X1 * Fp[1] + X2 * Fp[2];
        cX += X0 * Fp[0];
        cY += X1 * Fp[1];
        cZ += X2 * Fp[2];
        nmol++;
        pjs = js;
        psi = I.slot;
        if (HALF) {
            tq0 = tq[0];
            tq1 = tq[1];
            tq2 = tq[2];
        }
    }
    // End of a chunk.  Chunked half shell: each lane adds its pair's terms
    // straight to the FP32 records of i and j (a 16-byte vector reduction
    // for F and one for tau per molecule).  Full shell (deterministic): a
    // segmented suffix sum over the lanes, the first lane of each i adding
    // the i's total to the pass totals in shared memory.
    __device__ void chunk_end(Tile &, int il, int, bool valid, int lane)
    {
        if constexpr (HALF) {
            if (valid) {
                float *a = A.acc + (long long)FACC_STRIDE * psi;
                red_add_v4(a, pF0, pF1, pF2, 0.f);
                if (NQ == 6) red_add_v4(a + 4, pT0, pT1, pT2, 0.f);
                float *b = A.acc + (long long)FACC_STRIDE * pjs;
                red_add_v4(b, -pF0, -pF1, -pF2, 0.f);
                if (NQ == 6) red_add_v4(b + 4, tq0, tq1, tq2, 0.f);
            }
        } else {
        const int nvalid = __popc(__ballot_sync(FULLMASK, valid));  // valid lanes are a prefix
        const int prev = __shfl_up_sync(FULLMASK, il, 1);
        const bool head = valid && (lane == 0 || prev != il);
        const unsigned hm0 = __ballot_sync(FULLMASK, head);
        // lanes after this one in the same i segment
        const unsigned later = hm0 & ~((2u << lane) - 1u);
        const int rem = (later ? __ffs(later) - 1 : nvalid) - lane - 1;
        float v[6] = {pF0, pF1, pF2, pT0, pT1, pT2};
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const bool take = off <= rem;
#pragma unroll
            for (int q = 0; q < NQ; q++) {
                const float o = __shfl_down_sync(FULLMASK, v[q], off);
                if (take) v[q] += o;
            }
        }
        if (head) {  // the segment's FP32 sum (<= 32 pair terms) joins the i's total
            if (A.to_acc) {  // destined for FP32 records (batched replicas): FP32 totals
                float *f = reinterpret_cast<float *>(&T->x.it[0][0]);
#pragma unroll
                for (int q = 0; q < NQ; q++) f[q * 32 + il] += v[q];
            } else {  // FP64 outputs: FP64 totals
#pragma unroll
                for (int q = 0; q < NQ; q++) T->x.it[q][il] += (double)v[q];
            }
        }
        }
    }
    // Half shell, run-drained: the queue's qn entries are split into 32
    // contiguous runs of R entries, one per lane (R odd: the lanes'
    // shared-memory reads of one step fall in distinct banks).  Every pair
    // adds its Newton-3 reaction (-F, tau_j) straight to the j record; the i
    // side is summed in registers while the run's i stays the same and added
    // to the i record when it changes (entries of one i are contiguous), so
    // the i records see ~1/R of the per-pair reductions and the i molecule
    // is loaded once per run segment.
    struct Run {
        int cur;
        IMol<SIG> I;
        float a[6];
    };
    template <class Exact>
    __device__ __forceinline__ void run_step(Tile &Tl, Run &r, int e, int sbase, Exact &exact, float band_lo)
    {
        const int q = Tl.queue[e];
        const int il = q >> Tile::QSHIFT, k = q & ((1 << Tile::QSHIFT) - 1);
        if (il != r.cur) {
            if (r.cur >= 0) flush_i(sbase + r.cur, r.a);
            r.cur = il;
#pragma unroll
            for (int c = 0; c < 6; c++) r.a[c] = 0.f;
            if constexpr (SIG::LIN || SIG::SINGLE) load_i<SIG>(m, A.com, A.geo, K, sbase + il, r.I);
        }
        // models with per-site geometry reload it per pair (L1 hits) rather
        // than hold it across the run
        if constexpr (!(SIG::LIN || SIG::SINGLE)) load_i<SIG>(m, A.com, A.geo, K, sbase + il, r.I);
        const float4 cj = Tl.cand(k);
        const float X0 = r.I.c.x - cj.x, X1 = r.I.c.y - cj.y, X2 = r.I.c.z - cj.z;
        const int js = Tl.cand_slot(k);
        float Fp[3], tp[3], tq[3], Up;
        if constexpr (Tile::AXES)
            mol_pair<SIG, true, true>(m, X0, X1, X2, r.I, nullptr, Fp, tp, tq, Up, Tl.axis(k));
        else
            mol_pair<SIG, true>(m, X0, X1, X2, r.I, A.geo + (long long)js * K, Fp, tp, tq, Up);
        // queued inside the FP32 band around r_c^2: the FP64 test decides
        // (after the pair terms, so that no branch holds back their loads;
        // a pair outside the cut-off is dropped)
        if (Tile::DUP && X0 * X0 + X1 * X1 + X2 * X2 > band_lo && !exact(il, k)) return;
        r.a[0] += Fp[0];
        r.a[1] += Fp[1];
        r.a[2] += Fp[2];
        if (NQ == 6) {
            r.a[3] += tp[0];
            r.a[4] += tp[1];
            r.a[5] += tp[2];
        }
        cU += Up;
        cW += X0 * Fp[0] + X1 * Fp[1] + X2 * Fp[2];
        cX += X0 * Fp[0];
        cY += X1 * Fp[1];
        cZ += X2 * Fp[2];
        nmol++;
        float *b = A.acc + (long long)FACC_STRIDE * js;
        red_add_v4(b, -Fp[0], -Fp[1], -Fp[2], 0.f);
        if (NQ == 6) red_add_v4(b + 4, tq[0], tq[1], tq[2], 0.f);
    }
    template <class Exact>
    __device__ void drain(Tile &Tl, int qn, int sbase, int lane, Exact &exact, float band_lo)
    {
        const int R = ((qn + 31) >> 5) | 1;
        const int e0 = lane * R, e1 = min(e0 + R, qn);
        Run r;
        r.cur = -1;
        r.I.slot = 0;
#pragma unroll
        for (int c = 0; c < 6; c++) r.a[c] = 0.f;
        for (int t = 0; t < R; t++)  // warp-uniform trip count
            if (e0 + t < e1) run_step(Tl, r, e0 + t, sbase, exact, band_lo);
        if (r.cur >= 0) flush_i(sbase + r.cur, r.a);
    }
    __device__ __forceinline__ void flush_i(int si, const float (&v)[6])
    {
        float *a = A.acc + (long long)FACC_STRIDE * si;
        red_add_v4(a, v[0], v[1], v[2], 0.f);
        if (NQ == 6) red_add_v4(a + 4, v[3], v[4], v[5], 0.f);
    }
    __device__ void seg_end(Tile &, int, int) {}
    __device__ void pass_end(int s0, int ig_, int ni, int lane)
    {
        if constexpr (!HALF) {
            for (int t = lane; t < ni; t += 32) {
                const int si = s0 + ig_ + t;
                if (A.to_acc) {
                    const float *f = reinterpret_cast<const float *>(&T->x.it[0][0]);
                    float *a = A.acc + (long long)FACC_STRIDE * si;
                    red_add_v4(a, f[t], f[32 + t], f[64 + t], 0.f);
                    if (NQ == 6) red_add_v4(a + 4, f[96 + t], f[128 + t], f[160 + t], 0.f);
                } else {
                    double ip[6];
#pragma unroll
                    for (int q = 0; q < 6; q++) ip[q] = T->x.it[q][t];
                    double *Fo = A.F + 3LL * si, *To = A.tau + 3LL * si;
                    const double t0 = NQ == 6 ? ip[3] : 0.0, t1 = NQ == 6 ? ip[4] : 0.0, t2 = NQ == 6 ? ip[5] : 0.0;
                    Fo[0] = ip[0];
                    Fo[1] = ip[1];
                    Fo[2] = ip[2];
                    To[0] = t0;
                    To[1] = t1;
                    To[2] = t2;
                    if (!(isfinite(ip[0]) && isfinite(ip[1]) && isfinite(ip[2]) && isfinite(t0) && isfinite(t1) &&
                          isfinite(t2)))
                        atomicExch(&A.flags[FLAG_NONFINITE], 1);
                }
            }
        }
        // the lane's FP32 sums join its FP64 totals once they hold >= 256
        // pair terms (one FP64 add per value then; sparse cells would
        // otherwise pay it per pass)
        if (nmol - nflush >= 256) {
            const float c5[5] = {cU, cW, cX, cY, cZ};
#pragma unroll
            for (int q = 0; q < 5; q++) T->x.tot[q][ln] += (double)c5[q];
            cU = cW = cX = cY = cZ = 0.f;
            nflush = nmol;
        }
    }
};


// Warp totals of the energy / virial sums and pair counts of one op (all
// lanes return the same values).
template <class Op>
// Used per cell by the batched kernel: the lane totals of one cell are sums
// of a few hundred FP32 pair terms, so the warp sum is taken in FP32 (FP64
// shuffles and adds per cell measured 50% slower batched force
// evaluations); the per-replica sums are FP64.
__device__ __forceinline__ void op_warp_totals(Op &op, double (&v)[5], int &nm, int &ne)
{
#pragma unroll
    for (int q = 0; q < 5; q++) {
        float f = (float)op.total(q);
        for (int msk = 16; msk > 0; msk >>= 1) f += __shfl_xor_sync(FULLMASK, f, msk);
        v[q] = f;
    }
    nm = __reduce_add_sync(FULLMASK, op.nmol);
    ne = __reduce_add_sync(FULLMASK, op.nexam);
}

}  // namespace mdk
