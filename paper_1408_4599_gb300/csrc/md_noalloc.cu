// md_noalloc.cu -- md_kinetic_noalloc: the kinetic-energy reduction of
// md_energy_virial as a stand-alone entry point that allocates no memory.
//
// Some callers cannot call cudaMalloc (or anything that does):
// applications whose own allocator has reserved the device memory up front
// and must account for every byte, and real-time loops that must not stall
// on the device-wide synchronisation that cudaFree implies.  For them this
// entry point keeps its scratch -- the per-block partial sums of the
// reduction -- in a file-scope device array of fixed size, which every GPU
// that loads the library holds until the process exits.  The first call on
// a device looks up the array's device address (so that first call should
// come before any stream capture); calls that overlap on the GPU race on
// the shared array.  The address is kept per device ordinal for the life of
// the process: resetting a device (cudaDeviceReset) after the first call on
// it is not supported.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/md.h"
#include "md_leapfrog.cuh"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_ITEMS = 8;                          // molecules per thread per block
constexpr int NA_CHUNK = NA_THREADS * NA_ITEMS;      // molecules per block
constexpr int NA_MAX_BLOCKS = 4096;                  // scratch: 4096 x 2 doubles = 64 KiB
constexpr long long NA_MAX_N = (long long)NA_MAX_BLOCKS * NA_CHUNK;  // 8,388,608 molecules
constexpr int NA_MAX_DEVICES = 64;

// Per-block partial sums (K_trans, K_rot) of the last call.  Host code may
// not use this name as an address: it only names a host-side stand-in.
static __device__ __align__(256) double g_kin_scratch[NA_MAX_BLOCKS * 2];

std::mutex g_mu;
double *g_scratch_ptr[NA_MAX_DEVICES] = {nullptr};

struct KinArgs {
    long long n;
    const double *v, *q, *j, *F, *tau;
    double mass, I[3], Iinv[3], dt_half;
    double *scratch;
};

// Phase 1: block b reduces molecules [b*NA_CHUNK, (b+1)*NA_CHUNK) into
// scratch[2b], scratch[2b+1].
__global__ void __launch_bounds__(NA_THREADS) k_kin_partial(KinArgs a)
{
    __shared__ double sh[2][NA_THREADS / 32];
    double kt = 0.0, kr = 0.0;
    const double im = 1.0 / a.mass;
    const long long base = (long long)blockIdx.x * NA_CHUNK;
    for (int it = 0; it < NA_ITEMS; it++) {
        const long long s = base + (long long)it * NA_THREADS + threadIdx.x;
        if (s >= a.n) break;
        double v2 = 0.0, jt[3];
        for (int k = 0; k < 3; k++) {
            const double vk = a.v[3 * s + k] + a.dt_half * a.F[3 * s + k] * im;
            v2 += vk * vk;
            jt[k] = a.j[3 * s + k] + a.dt_half * a.tau[3 * s + k];
        }
        kt += 0.5 * a.mass * v2;
        const float Iinv[3] = {(float)a.Iinv[0], (float)a.Iinv[1], (float)a.Iinv[2]};
        const float Im[3] = {(float)a.I[0], (float)a.I[1], (float)a.I[2]};
        kr += 0.5 * (double)mdk::kin_rot2(a.q + 4 * s, jt, Iinv, Im);
    }
    for (int o = 16; o > 0; o >>= 1) {
        kt += __shfl_xor_sync(0xffffffffu, kt, o);
        kr += __shfl_xor_sync(0xffffffffu, kr, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        sh[0][warp] = kt;
        sh[1][warp] = kr;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double t = 0.0;
        for (int w = 0; w < NA_THREADS / 32; w++) t += sh[threadIdx.x][w];
        a.scratch[2 * blockIdx.x + threadIdx.x] = t;
    }
}

// Phase 2: one warp sums the block partials in a fixed order.
__global__ void k_kin_final(const double *scratch, int nb, double *out)
{
    double kt = 0.0, kr = 0.0;
    for (int b = threadIdx.x; b < nb; b += 32) {
        kt += scratch[2 * b];
        kr += scratch[2 * b + 1];
    }
    for (int o = 16; o > 0; o >>= 1) {
        kt += __shfl_xor_sync(0xffffffffu, kt, o);
        kr += __shfl_xor_sync(0xffffffffu, kr, o);
    }
    if (threadIdx.x == 0) {
        out[0] = kt;
        out[1] = kr;
    }
}

}  // namespace

extern "C" md_status md_kinetic_noalloc(int64_t n, const double *v, const double *q, const double *j,
                                        const double *F, const double *tau, double mass, const double I[3], double dt,
                                        double *K_out, void *cuda_stream)
{
    if (n < 0 || !K_out || !I || (n > 0 && (!v || !q || !j || !F || !tau)) || !(mass > 0.0) || !(dt >= 0.0))
        return MD_ERR_ARG;
    for (int k = 0; k < 3; k++)
        if (!(I[k] >= 0.0)) return MD_ERR_ARG;
    if (n > NA_MAX_N) return MD_ERR_OVERFLOW;  // the fixed scratch holds 4096 block partials
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return MD_ERR_CUDA;
    double *scratch = nullptr;
    {
        // one-time set-up per device, done by the first call on that device
        // with the device current
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_ptr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_kin_scratch) != cudaSuccess || !p) return MD_ERR_CUDA;
            g_scratch_ptr[dev] = (double *)p;
        }
        scratch = g_scratch_ptr[dev];
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    KinArgs a;
    a.n = n;
    a.v = v;
    a.q = q;
    a.j = j;
    a.F = F;
    a.tau = tau;
    a.mass = mass;
    for (int k = 0; k < 3; k++) {
        a.I[k] = I[k];
        a.Iinv[k] = I[k] > 1e-12 ? 1.0 / I[k] : 0.0;
    }
    a.dt_half = 0.5 * dt;
    a.scratch = scratch;
    int nb = (int)((n + NA_CHUNK - 1) / NA_CHUNK);
    // each launch's own status (cudaLaunchKernel returns it), so that an
    // earlier, unrelated error left in the runtime's last-error slot is
    // neither reported here nor cleared
    if (nb > 0) {
        void *args1[] = {&a};
        if (cudaLaunchKernel((const void *)k_kin_partial, dim3(nb), dim3(NA_THREADS), args1, 0, st) != cudaSuccess)
            return MD_ERR_CUDA;
    }
    // every block partial that phase 2 reads was written by this call's phase 1
    const double *sc = scratch;
    void *args2[] = {&sc, &nb, &K_out};
    if (cudaLaunchKernel((const void *)k_kin_final, dim3(1), dim3(32), args2, 0, st) != cudaSuccess)
        return MD_ERR_CUDA;
    return MD_OK;
}
