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

struct ForceExtra {
    float4 if4[32];  // i totals of the pass: F, tau_x
    float2 it2[32];  // tau_y, tau_z
};

template <class SIG, bool HALF>
struct ForceOp {
    static constexpr int IMAX = 32;
    static constexpr int NQ = SIG::SINGLE ? 3 : 6;  // accumulated values per molecule: F, and tau unless single-site
    using Tile = WarpTile<ForceExtra>;
    const DevModel &m;
    const ForceArgs &A;
    int K;
    int ig;
    float pF0, pF1, pF2, pT0, pT1, pT2;            // the lane's pair of the current chunk (i side)
    float tq0, tq1, tq2;                           // its torque on j (half shell)
    int pjs, psi;                                  // storage slots of its j and i
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
        if (!HALF) {  // the half shell adds its i terms per pair (chunk_end)
            for (int t = lane; t < ni; t += 32) {
                T->x.if4[t] = make_float4(0.f, 0.f, 0.f, 0.f);
                T->x.it2[t] = make_float2(0.f, 0.f);
            }
        }
        cU = cW = cX = cY = cZ = 0.f;
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
    // End of a chunk.  Half shell: each lane adds its pair's terms straight
    // to the FP32 accumulator records of i and j (one 16-byte vector
    // reduction for F and one for tau per molecule; measured faster than
    // per-candidate shared accumulators for the Newton-3 side and than a
    // segmented warp sum for the i side).  Full shell (deterministic): a
    // segmented suffix sum over the lanes, the first lane of each i adding the
    // i's total to the pass totals in shared memory.
    __device__ void chunk_end(Tile &, int il, int, bool valid, int lane)
    {
        if (HALF) {
            if (valid) {
                float *a = A.acc + (long long)FACC_STRIDE * psi;
                red_add_v4(a, pF0, pF1, pF2, 0.f);
                if (NQ == 6) red_add_v4(a + 4, pT0, pT1, pT2, 0.f);
                float *b = A.acc + (long long)FACC_STRIDE * pjs;
                red_add_v4(b, -pF0, -pF1, -pF2, 0.f);
                if (NQ == 6) red_add_v4(b + 4, tq0, tq1, tq2, 0.f);
            }
            return;
        }
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
        if (head) {
            float4 a = T->x.if4[il];
            a.x += v[0];
            a.y += v[1];
            a.z += v[2];
            if (NQ == 6) {
                a.w += v[3];
                float2 b = T->x.it2[il];
                b.x += v[4];
                b.y += v[5];
                T->x.it2[il] = b;
            }
            T->x.if4[il] = a;
        }
    }
    __device__ void seg_end(Tile &, int, int) {}
    __device__ void pass_end(int s0, int ig_, int ni, int lane)
    {
        if (!HALF) {
            for (int t = lane; t < ni; t += 32) {
                const int si = s0 + ig_ + t;
                const float4 i4 = T->x.if4[t];
                const float2 i2 = T->x.it2[t];
                const float ip[6] = {i4.x, i4.y, i4.z, i4.w, i2.x, i2.y};
                if (A.to_acc) {
                    float *a = A.acc + (long long)FACC_STRIDE * si;
                    red_add_v4(a, ip[0], ip[1], ip[2], 0.f);
                    if (NQ == 6) red_add_v4(a + 4, ip[3], ip[4], ip[5], 0.f);
                } else {
                    double *Fo = A.F + 3LL * si, *To = A.tau + 3LL * si;
                    const float t0 = NQ == 6 ? ip[3] : 0.f, t1 = NQ == 6 ? ip[4] : 0.f, t2 = NQ == 6 ? ip[5] : 0.f;
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
        kahan_add(sU, kU, cU);
        kahan_add(sW, kW, cW);
        kahan_add(sX, kX, cX);
        kahan_add(sY, kY, cY);
        kahan_add(sZ, kZ, cZ);
    }
};


// Warp totals of the energy / virial sums and pair counts of one op (all
// lanes return the same values).
template <class Op>
__device__ __forceinline__ void op_warp_totals(Op &op, float (&v)[5], int &nm, int &ne)
{
    v[0] = op.sU - op.kU;
    v[1] = op.sW - op.kW;
    v[2] = op.sX - op.kX;
    v[3] = op.sY - op.kY;
    v[4] = op.sZ - op.kZ;
    for (int q = 0; q < 5; q++)
        for (int msk = 16; msk > 0; msk >>= 1) v[q] += __shfl_xor_sync(FULLMASK, v[q], msk);
    nm = __reduce_add_sync(FULLMASK, op.nmol);
    ne = __reduce_add_sync(FULLMASK, op.nexam);
}

}  // namespace mdk
