// md_force.cu -- launches of the linked-cell force kernel (md_force.cuh,
// instantiated by md_force_inst.cu) for cells of edge >= r_c (27- / 14-cell
// stencils) or >= r_c / 2 (125- / 63-cell stencils), and the FP32 -> FP64
// finalize of the half-shell accumulators.
#include "md_forceop.cuh"

using namespace mdk;

namespace {

// Dispatch target of dispatch_sig: the instantiation for one signature.
template <int M>
struct LaunchForce {
    const ForceArgs &A;
    int half, n_blocks;
    cudaStream_t s;
    template <class SIG>
    cudaError_t operator()() const
    {
        return launch_force_sig<SIG, M>(A, half, n_blocks, s);
    }
};

// Half shell: FP32 accumulator records -> FP64 F, tau; non-finite check.
__global__ void k_force_finalize(const float *acc, long long n, double *F, double *tau, int *flags)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const float4 f = reinterpret_cast<const float4 *>(acc)[2 * s], t = reinterpret_cast<const float4 *>(acc)[2 * s + 1];
    const float fv[3] = {f.x, f.y, f.z}, tv[3] = {t.x, t.y, t.z};
    bool bad = false;
    for (int q = 0; q < 3; q++) {
        bad |= !isfinite(fv[q]) || !isfinite(tv[q]);
        F[3 * s + q] = (double)fv[q];
        tau[3 * s + q] = (double)tv[q];
    }
    if (bad) atomicExch(&flags[FLAG_NONFINITE], 1);
}

}  // namespace

// SMs of the current device (152 on GB300 if the query fails)
int device_sms()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess || sms <= 0) {
        cudaGetLastError();
        return 152;
    }
    return sms;
}

// upper bound of the force grid: 16 blocks per SM (the kernels' occupancy
// is lower; the launch trims the grid to what is resident)
int force_blocks_default() { return device_sms() * 16; }

cudaError_t launch_force(const Grid &g, const DevModel &m, DevState &d, int half_shell, int dynamic_cells, int n_blocks,
                         cudaStream_t s, int acc_zeroed)
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
    A.to_acc = 0;
    A.cell_ctr = dynamic_cells ? d.cell_ctr : nullptr;
    // the grid may be smaller than the partials buffer: unused slots read as
    // 0; the counter slot after the partials is cleared with them
    cudaError_t e = cudaMemsetAsync(d.partials, 0, sizeof(double) * (P_COUNT * (size_t)n_blocks + 1), s);
    if (e != cudaSuccess) return e;
    if (half_shell && !acc_zeroed) {
        e = cudaMemsetAsync(d.facc, 0, sizeof(float) * FACC_STRIDE * (d.n > 0 ? d.n : 1), s);
        if (e != cudaSuccess) return e;
    }
    if (g.m == 2) return dispatch_sig(m, LaunchForce<2>{A, half_shell, n_blocks, s});
    return dispatch_sig(m, LaunchForce<1>{A, half_shell, n_blocks, s});
}

cudaError_t launch_force_finalize(DevState &d, cudaStream_t s)
{
    if (d.n == 0) return cudaSuccess;
    k_force_finalize<<<(unsigned)((d.n + 255) / 256), 256, 0, s>>>(d.facc, d.n, d.F, d.tau, d.flags);
    return cudaGetLastError();
}
