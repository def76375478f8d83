// md_force_m2.cu -- the force kernel of md_force.cuh for cells of edge
// >= r_c / 2 and the 125- / 63-cell stencils (§3: smaller cells examine
// 15.6 r_c^3 instead of 27 r_c^3 around each molecule).  A translation unit
// of its own so that both stencils compile in parallel.
#include "md_force.cuh"

cudaError_t launch_force_radius2(const mdk::ForceArgs &A, int half_shell, int n_blocks, cudaStream_t s)
{
    return mdk::dispatch_sig(A.m, LaunchForce<2>{A, half_shell, n_blocks, s});
}
