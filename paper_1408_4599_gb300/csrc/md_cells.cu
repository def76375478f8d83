// md_cells.cu -- linked-cell rebuild (§3 "linked-cell algorithm"): cell id
// per molecule, counting sort (histogram, exclusive scan, scatter), a
// per-cell rank sort by the caller's molecule index (so that the storage
// order is deterministic), and the reorder + FP32 packing pass that writes
// what the force kernel reads.
//
// HBM-bound kernels: each reads/writes every molecule's record once.
#include "md_leapfrog.cuh"

#include <climits>

using mdk::cell_coord;
using mdk::d2f_bits;
using mdk::int_plus_half;

namespace {

constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// Wrap positions into [0, L) and renormalise quaternions (input hygiene);
// flags[FLAG_INPUT] marks a non-finite r, v, j or a zero / non-finite q.
__global__ void k_prepare(Grid g, double *r, double *q, const double *v, const double *j, long long n, int *flags)
{
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    bool bad = false;
    for (int k = 0; k < 3; k++) bad |= !isfinite(v[3 * s + k]) || !isfinite(j[3 * s + k]);
    for (int k = 0; k < 3; k++) {
        double x = r[3 * s + k];
        bad |= !isfinite(x);
        // 0 <= x < L as one unsigned compare of the bit patterns (negative
        // values and NaN compare above); only a position outside the box
        // pays the FP64 division of the wrap
        if ((unsigned long long)__double_as_longlong(x) >= (unsigned long long)__double_as_longlong(g.L[k])) {
            x -= g.L[k] * floor(x / g.L[k]);
            if (x >= g.L[k]) x -= g.L[k];
            if (x < 0.0) x = 0.0;
            r[3 * s + k] = x;
        }
    }
    double w = q[4 * s], a = q[4 * s + 1], b = q[4 * s + 2], c = q[4 * s + 3];
    const double nn2 = w * w + a * a + b * b + c * c, e = nn2 - 1.0;
    bad |= !(nn2 > 0.0) || !isfinite(nn2);
    // |q|^-1 = (1 + e)^(-1/2): the cubic series is exact to FP64 rounding for
    // |e| < 1e-4 (unit quaternions as given), 1/sqrt otherwise
    const double inv = fabs(e) < 1e-4 ? 1.0 + e * (-0.5 + e * (0.375 - 0.3125 * e)) : 1.0 / sqrt(nn2);
    q[4 * s] = w * inv;
    q[4 * s + 1] = a * inv;
    q[4 * s + 2] = b * inv;
    q[4 * s + 3] = c * inv;
    if (bad) atomicExch(&flags[FLAG_INPUT], 1);
}

__global__ void k_iota(int *ids, long long n)
{
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n) ids[s] = (int)s;
}

// Cell of every molecule (positions already in [0, L)) and the histogram.
__global__ void k_cellid(Grid g, const double *r, int *cell, int *count, long long n)
{
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    int cx = cell_coord(r[3 * s], g.iell[0], g.nc[0]);
    int cy = cell_coord(r[3 * s + 1], g.iell[1], g.nc[1]);
    int cz = cell_coord(r[3 * s + 2], g.iell[2], g.nc[2]);
    int c = (cz * g.nc[1] + cy) * g.nc[0] + cx;
    cell[s] = c;
    atomicAdd(&count[c], 1);
}

__device__ __forceinline__ int block_exclusive_scan(int v, int *smem_warp, int &total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < (blockDim.x >> 5) ? smem_warp[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        smem_warp[lane] = w;
    }
    __syncthreads();
    int warp_off = warp > 0 ? smem_warp[warp - 1] : 0;
    total = smem_warp[(blockDim.x >> 5) - 1];
    __syncthreads();
    return warp_off + x - v;
}

// Scan phase 1: sum of each tile.
__global__ void k_scan_reduce(const int *count, long long ncell, int *block_sums)
{
    __shared__ int sw[32];
    long long base = (long long)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    int v = 0;
    for (int k = 0; k < SCAN_ITEMS; k++)
        if (base + k < ncell) v += count[base + k];
    int total;
    block_exclusive_scan(v, sw, total);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

// Scan phase 2: exclusive scan of the tile sums (one block, looping).
__global__ void k_scan_top(int *block_sums, int nb)
{
    __shared__ int sw[32];
    int carry = 0;
    for (int base = 0; base < nb; base += SCAN_THREADS) {
        int i = base + threadIdx.x;
        int v = i < nb ? block_sums[i] : 0;
        int total;
        int ex = block_exclusive_scan(v, sw, total);
        if (i < nb) block_sums[i] = carry + ex;
        carry += total;
    }
}

// Scan phase 3: exclusive scan inside each tile plus the tile offset.
__global__ void k_scan_down(const int *count, long long ncell, const int *block_sums, int *start)
{
    __shared__ int sw[32];
    long long base = (long long)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    int loc[SCAN_ITEMS];
    int v = 0;
    for (int k = 0; k < SCAN_ITEMS; k++) {
        loc[k] = (base + k < ncell) ? count[base + k] : 0;
        v += loc[k];
    }
    int total;
    int ex = block_exclusive_scan(v, sw, total) + block_sums[blockIdx.x];
    for (int k = 0; k < SCAN_ITEMS; k++) {
        if (base + k < ncell) start[base + k] = ex;
        ex += loc[k];
    }
    // the thread owning the last cell also writes the total at start[ncell]
    if (base <= ncell - 1 && ncell - 1 < base + SCAN_ITEMS) start[ncell] = ex;
}

// Exclusive scan of the histogram by one block, tile after tile (grids of
// up to SCAN_SINGLE_MAX cells: one launch instead of three).
constexpr long long SCAN_SINGLE_MAX = 16LL * SCAN_TILE;

__global__ void k_scan_single(const int *count, long long ncell, int *start)
{
    __shared__ int sw[32];
    int carry = 0;
    for (long long t0 = 0; t0 < ncell; t0 += SCAN_TILE) {
        const long long base = t0 + threadIdx.x * SCAN_ITEMS;
        int loc[SCAN_ITEMS];
        int v = 0;
        for (int k = 0; k < SCAN_ITEMS; k++) {
            loc[k] = (base + k < ncell) ? count[base + k] : 0;
            v += loc[k];
        }
        int total;
        int ex = block_exclusive_scan(v, sw, total) + carry;
        for (int k = 0; k < SCAN_ITEMS; k++) {
            if (base + k < ncell) start[base + k] = ex;
            ex += loc[k];
        }
        carry += total;
    }
    if (threadIdx.x == 0) start[ncell] = carry;
}

// Counting-sort scatter: unstable slot claim inside each cell.
__global__ void k_scatter(const int *cell, const int *start, int *fill, int *perm, long long n)
{
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    int c = cell[s];
    int p = start[c] + atomicAdd(&fill[c], 1);
    perm[p] = (int)s;
}

// One warp per cell: order the cell's slots by the caller's molecule index
// (rank sort; keys are unique), making the storage order independent of
// the scatter's atomic order.
__global__ void k_sort_cells(const int *start, const int *perm, const int *ids, int *perm_out, long long ncell)
{
    const int lane = threadIdx.x & 31;
    long long c = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (c >= ncell) return;
    int st = start[c], n = start[c + 1] - st;
    for (int eb = 0; eb < n; eb += 32) {
        int e = eb + lane;
        int pe = e < n ? perm[st + e] : 0;
        int key = e < n ? ids[pe] : INT_MAX;
        int rank = 0;
        for (int kb = 0; kb < n; kb += 32) {
            int k = kb + lane;
            int keyk = k < n ? ids[perm[st + k]] : INT_MAX;
            int lim = min(32, n - kb);
            for (int t = 0; t < lim; t++) rank += (__shfl_sync(0xffffffffu, keyk, t) < key) ? 1 : 0;
        }
        if (e < n) perm_out[st + rank] = pe;
    }
}

// The FP32 data the force kernel reads for the molecule in slot s of cell
// c: its centre of mass relative to the cell centre (formed in FP64, then
// rounded) and the space-frame site offsets and axes R(q) d, R(q) e.  The
// conversions run on the integer pipe (md_fpconv.cuh: the same bits as the
// hardware's, which would occupy the FP64 pipe).
__device__ __forceinline__ void pack_one(const Grid &g, const DevModel &m, const DevState &d, long long s, int c,
                                         double rx, double ry, double rz, double qw, double qx, double qy, double qz)
{
    int cx = c % g.nc[0], cy = (c / g.nc[0]) % g.nc[1], cz = c / (g.nc[0] * g.nc[1]);
    float4 cm;
    cm.x = d2f_bits(rx - int_plus_half(cx) * g.ell[0]);
    cm.y = d2f_bits(ry - int_plus_half(cy) * g.ell[1]);
    cm.z = d2f_bits(rz - int_plus_half(cz) * g.ell[2]);
    cm.w = 0.0f;
    d.com[s] = cm;
    if (m.single_lj_at_com) return;
    float w = d2f_bits(qw), x = d2f_bits(qx), y = d2f_bits(qy), z = d2f_bits(qz);
    float R[9] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y),
                  2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x),
                  2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)};
    float4 *out = d.geo + s * (long long)d.K;
    if (m.linear) {  // the molecular axis R(q) z carries every site offset and axis
        out[0] = make_float4(R[2], R[5], R[8], 0.0f);
        return;
    }
    for (int a = 0; a < m.S; a++) {
        const float *b = m.body[a];
        out[a] = make_float4(R[0] * b[0] + R[1] * b[1] + R[2] * b[2], R[3] * b[0] + R[4] * b[1] + R[5] * b[2],
                             R[6] * b[0] + R[7] * b[1] + R[8] * b[2], 0.0f);
        if (m.axis_slot[a] >= 0) {
            const float *e = m.axis[a];
            out[m.S + m.axis_slot[a]] =
                make_float4(R[0] * e[0] + R[1] * e[1] + R[2] * e[2], R[3] * e[0] + R[4] * e[1] + R[5] * e[2],
                            R[6] * e[0] + R[7] * e[1] + R[8] * e[2], 0.0f);
        }
    }
}

// Reorder the FP64 state into the new cell order (new slot s <- old slot
// perm2[s]) and pack the force kernel's FP32 data.
__global__ void k_reorder_pack(Grid g, DevModel m, DevState d, const double *beta)
{
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= d.n) return;
    int o = d.perm2[s];
    const double b = beta ? *beta : 1.0;  // velocity-rescaling factor of this step
    double rx = d.r[3 * o], ry = d.r[3 * o + 1], rz = d.r[3 * o + 2];
    d.r2[3 * s] = rx;
    d.r2[3 * s + 1] = ry;
    d.r2[3 * s + 2] = rz;
    for (int k = 0; k < 3; k++) {
        d.v2[3 * s + k] = b * d.v[3 * o + k];
        d.j2[3 * s + k] = b * d.j[3 * o + k];
    }
    // quaternion records are 32-byte aligned: two 16-byte moves
    const double2 q01 = reinterpret_cast<const double2 *>(d.q)[2 * o], q23 = reinterpret_cast<const double2 *>(d.q)[2 * o + 1];
    reinterpret_cast<double2 *>(d.q2)[2 * s] = q01;
    reinterpret_cast<double2 *>(d.q2)[2 * s + 1] = q23;
    d.ids2[s] = d.ids[o];
    pack_one(g, m, d, s, d.cell[o], rx, ry, rz, q01.x, q01.y, q23.x, q23.y);
}

// Counting-sort scatter fused with the reorder and packing (runs without
// the deterministic in-cell order): old slot s claims a slot of its cell by
// counting the cell's histogram entry down (which leaves the histogram at
// zero for the next step) and writes its whole record there.  The reads
// are in storage order; the writes land near s, since molecules rarely
// change cell in one step.
// ZACC: also clear the slot's FP32 accumulator record (half shell), so the
// force kernel that follows needs no separate clearing pass.
template <bool BETA, bool ZACC>  // BETA: apply the velocity-rescaling factor (NVT steps)
__global__ void k_scatter_pack(Grid g, DevModel m, DevState d, const double *beta)
{
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= d.n) return;
    const int c = d.cell[s];
    const long long p = d.cell_start[c] + atomicSub(&d.cell_count[c], 1) - 1;
    const double rx = d.r[3 * s], ry = d.r[3 * s + 1], rz = d.r[3 * s + 2];
    d.r2[3 * p] = rx;
    d.r2[3 * p + 1] = ry;
    d.r2[3 * p + 2] = rz;
    if constexpr (BETA) {
        const double b = *beta;
        for (int k = 0; k < 3; k++) {
            d.v2[3 * p + k] = b * d.v[3 * s + k];
            d.j2[3 * p + k] = b * d.j[3 * s + k];
        }
    } else {  // (FP64 multiplies run at a small fraction of the FP32 rate)
        for (int k = 0; k < 3; k++) {
            d.v2[3 * p + k] = d.v[3 * s + k];
            d.j2[3 * p + k] = d.j[3 * s + k];
        }
    }
    const double2 q01 = reinterpret_cast<const double2 *>(d.q)[2 * s], q23 = reinterpret_cast<const double2 *>(d.q)[2 * s + 1];
    reinterpret_cast<double2 *>(d.q2)[2 * p] = q01;
    reinterpret_cast<double2 *>(d.q2)[2 * p + 1] = q23;
    d.ids2[p] = d.ids[s];
    if constexpr (ZACC) {
        float4 *a = reinterpret_cast<float4 *>(d.facc) + 2 * p;
        a[0] = make_float4(0.f, 0.f, 0.f, 0.f);
        a[1] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    pack_one(g, m, d, p, c, rx, ry, rz, q01.x, q01.y, q23.x, q23.y);
}

// The four state arrays back in the caller's molecule order (a NULL target
// is skipped), one thread per molecule.
__global__ void k_scatter_state(const int *ids, const double *r, const double *v, const double *q, const double *j,
                                double *dr, double *dv, double *dq, double *dj, long long n)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const long long o = ids[s];
    if (dr)
        for (int k = 0; k < 3; k++) dr[3 * o + k] = r[3 * s + k];
    if (dv)
        for (int k = 0; k < 3; k++) dv[3 * o + k] = v[3 * s + k];
    if (dq) {
        const double2 a = reinterpret_cast<const double2 *>(q)[2 * s], b = reinterpret_cast<const double2 *>(q)[2 * s + 1];
        reinterpret_cast<double2 *>(dq)[2 * o] = a;
        reinterpret_cast<double2 *>(dq)[2 * o + 1] = b;
    }
    if (dj)
        for (int k = 0; k < 3; k++) dj[3 * o + k] = j[3 * s + k];
}

__global__ void k_scatter_out(const int *ids, const double *src, int width, double *dst, long long n)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * width) return;
    long long s = t / width;
    int k = (int)(t - s * width);
    dst[(long long)ids[s] * width + k] = src[t];
}

inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

int scan_blocks(long long ncell) { return (int)((ncell + SCAN_TILE - 1) / SCAN_TILE); }

cudaError_t launch_prepare_input(const Grid &g, DevState &d, cudaStream_t s)
{
    if (d.n == 0) return cudaSuccess;
    k_prepare<<<nblk(d.n, 256), 256, 0, s>>>(g, d.r, d.q, d.v, d.j, d.n, d.flags);
    k_iota<<<nblk(d.n, 256), 256, 0, s>>>(d.ids, d.n);
    return cudaGetLastError();
}

cudaError_t launch_cellid(const Grid &g, DevState &d, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(d.cell_count, 0, sizeof(int) * g.ncell, s);
    if (e != cudaSuccess) return e;
    if (d.n == 0) return cudaSuccess;
    k_cellid<<<nblk(d.n, 256), 256, 0, s>>>(g, d.r, d.cell, d.cell_count, d.n);
    return cudaGetLastError();
}

// Exclusive scan of the histogram into cell_start (ncell + 1 entries).
static void launch_scan(long long ncell, DevState &d, cudaStream_t s)
{
    if (ncell <= SCAN_SINGLE_MAX) {
        k_scan_single<<<1, SCAN_THREADS, 0, s>>>(d.cell_count, ncell, d.cell_start);
        return;
    }
    int nb = scan_blocks(ncell);
    k_scan_reduce<<<nb, SCAN_THREADS, 0, s>>>(d.cell_count, ncell, d.scan_tmp);
    k_scan_top<<<1, SCAN_THREADS, 0, s>>>(d.scan_tmp, nb);
    k_scan_down<<<nb, SCAN_THREADS, 0, s>>>(d.cell_count, ncell, d.scan_tmp, d.cell_start);
}

// Counting sort over ncell cells: scan of the histogram, scatter and the
// in-cell sort; leaves the new order (new slot -> old slot) in perm2.
cudaError_t launch_sort(long long ncell, DevState &d, cudaStream_t s)
{
    launch_scan(ncell, d, s);
    cudaError_t e = cudaMemsetAsync(d.cell_fill, 0, sizeof(int) * ncell, s);
    if (e != cudaSuccess) return e;
    if (d.n > 0) {
        k_scatter<<<nblk(d.n, 256), 256, 0, s>>>(d.cell, d.cell_start, d.cell_fill, d.perm, d.n);
        k_sort_cells<<<nblk(ncell * 32, 256), 256, 0, s>>>(d.cell_start, d.perm, d.ids, d.perm2, ncell);
    }
    return cudaGetLastError();
}

// Swap the state buffers after a reorder pass.
void swap_state(DevState &d)
{
    double *t;
    t = d.r; d.r = d.r2; d.r2 = t;
    t = d.v; d.v = d.v2; d.v2 = t;
    t = d.q; d.q = d.q2; d.q2 = t;
    t = d.j; d.j = d.j2; d.j2 = t;
    int *ti = d.ids; d.ids = d.ids2; d.ids2 = ti;
}

// Scan of the histogram, scatter, in-cell sort, reorder + pack, then swap
// the state buffers.  Expects cell[] and cell_count[] of the current order.
// deterministic = 0: the scatter claims slots by counting the histogram
// down and writes the records itself (no in-cell sort, no separate
// reorder), leaving cell_count at zero.
cudaError_t launch_rebuild(const Grid &g, const DevModel &m, DevState &d, cudaStream_t s, const double *beta,
                           int deterministic, int zero_acc)
{
    cudaError_t e = cudaSuccess;
    if (deterministic) {
        e = launch_sort(g.ncell, d, s);
        if (e != cudaSuccess) return e;
        if (d.n > 0) k_reorder_pack<<<nblk(d.n, 256), 256, 0, s>>>(g, m, d, beta);
    } else {
        launch_scan(g.ncell, d, s);
        if (d.n > 0) {
            const unsigned nb = nblk(d.n, 256);
            if (beta) {
                if (zero_acc) k_scatter_pack<true, true><<<nb, 256, 0, s>>>(g, m, d, beta);
                else k_scatter_pack<true, false><<<nb, 256, 0, s>>>(g, m, d, beta);
            } else {
                if (zero_acc) k_scatter_pack<false, true><<<nb, 256, 0, s>>>(g, m, d, beta);
                else k_scatter_pack<false, false><<<nb, 256, 0, s>>>(g, m, d, beta);
            }
        }
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    double *t;
    t = d.r; d.r = d.r2; d.r2 = t;
    t = d.v; d.v = d.v2; d.v2 = t;
    t = d.q; d.q = d.q2; d.q2 = t;
    t = d.j; d.j = d.j2; d.j2 = t;
    int *ti = d.ids; d.ids = d.ids2; d.ids2 = ti;
    return cudaSuccess;
}

cudaError_t launch_scatter_state(const DevState &d, double *r, double *v, double *q, double *j, cudaStream_t s)
{
    if (d.n == 0) return cudaSuccess;
    k_scatter_state<<<nblk(d.n, 256), 256, 0, s>>>(d.ids, d.r, d.v, d.q, d.j, r, v, q, j, d.n);
    return cudaGetLastError();
}

cudaError_t launch_scatter_out(const DevState &d, const double *src, int width, double *dst, cudaStream_t s)
{
    if (d.n == 0) return cudaSuccess;
    k_scatter_out<<<nblk(d.n * width, 256), 256, 0, s>>>(d.ids, src, width, dst, d.n);
    return cudaGetLastError();
}
