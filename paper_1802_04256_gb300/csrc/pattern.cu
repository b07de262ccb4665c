// Stage 1a: integration points, uniform-grid cell list, support search,
// node -> point incidence and the BSR pattern of K, all on the device.
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <string>

#include <atomic>
#include <mutex>

#include "common.cuh"

namespace rpim {

constexpr double kGauss2 = 0.57735026918962576451; // 1/sqrt(3)

// ---------------------------------------------------------------------------
// 2x2x2 Gauss-Legendre points of every node cell. Point 8i + l sits at
// mid + half * (+-1/sqrt(3)) per axis (bit k of l selects +), weight
// hx*hy*hz. Rounded products and sums are spelled out so that the points
// are the same doubles on every compliant implementation.
// ---------------------------------------------------------------------------
__global__ void gauss_points_kernel(int64_t n, const double *lo, const double *hi, double *pts,
                                    double *wj)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < 8 * n;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = t >> 3;
        int l = (int)(t & 7);
        double half[3];
        for (int k = 0; k < 3; k++) {
            double a = lo[3 * i + k], b = hi[3 * i + k];
            double mid = __dmul_rn(__dadd_rn(a, b), 0.5);
            half[k] = __dmul_rn(__dsub_rn(b, a), 0.5);
            double off = __dmul_rn(half[k], ((l >> k) & 1) ? kGauss2 : -kGauss2);
            pts[3 * t + k] = __dadd_rn(mid, off);
        }
        wj[t] = __dmul_rn(__dmul_rn(half[0], half[1]), half[2]);
    }
}

// ---------------------------------------------------------------------------
// bounding box and cell binning
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long ordered(double v)
{
    // order-preserving map of doubles to unsigned integers
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double unordered(unsigned long long u)
{
    unsigned long long b = (u & 0x8000000000000000ull) ? (u & 0x7FFFFFFFFFFFFFFFull) : ~u;
    return __longlong_as_double((long long)b);
}

// bounding box of every instance: one block per instance, block reduction
__global__ void bbox_kernel(const InstGrid *ig, const double *xyz, unsigned long long *bb /*6 per instance*/,
                            int *bad)
{
    __shared__ unsigned long long sm[6][32];
    const InstGrid g = ig[blockIdx.x];
    unsigned long long mn[3] = {~0ull, ~0ull, ~0ull}, mx[3] = {0, 0, 0};
    for (int64_t i = g.node_begin + threadIdx.x; i < g.node_end; i += blockDim.x)
        for (int k = 0; k < 3; k++) {
            double v = xyz[3 * i + k];
            if (!isfinite(v)) atomicExch(bad, 1);
            unsigned long long o = ordered(v);
            mn[k] = min(mn[k], o);
            mx[k] = max(mx[k], o);
        }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int k = 0; k < 3; k++) {
        for (int o = 16; o > 0; o >>= 1) {
            mn[k] = min(mn[k], __shfl_down_sync(0xffffffffu, mn[k], o));
            mx[k] = max(mx[k], __shfl_down_sync(0xffffffffu, mx[k], o));
        }
        if (lane == 0) {
            sm[k][w] = mn[k];
            sm[3 + k][w] = mx[k];
        }
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        const int k = threadIdx.x;
        unsigned long long r = k < 3 ? ~0ull : 0ull;
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) r = k < 3 ? min(r, sm[k][i]) : max(r, sm[k][i]);
        bb[6 * blockIdx.x + k] = r;
    }
}

// instance of every node: one block per instance
__global__ void node_inst_kernel(const InstGrid *ig, int32_t *node_inst)
{
    const InstGrid g = ig[blockIdx.x];
    for (int64_t i = g.node_begin + threadIdx.x; i < g.node_end; i += blockDim.x) node_inst[i] = (int32_t)blockIdx.x;
}

__device__ __forceinline__ int cell_coord(double x, double lo, double inv_edge, int n)
{
    double c = floor((x - lo) * inv_edge);
    if (c < 0) return 0;
    if (c > n - 1) return n - 1;
    return (int)c;
}

__global__ void bin_nodes(int64_t n, const double *xyz, const InstGrid *ig, const int32_t *node_inst,
                          int32_t *node_cell, uint32_t *node_cpk, int32_t *cell_count)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const InstGrid &g = ig[node_inst[i]];
        int cx = cell_coord(xyz[3 * i], g.lo[0], g.inv_edge, g.n[0]);
        int cy = cell_coord(xyz[3 * i + 1], g.lo[1], g.inv_edge, g.n[1]);
        int cz = cell_coord(xyz[3 * i + 2], g.lo[2], g.inv_edge, g.n[2]);
        int64_t c = g.cell_off + cx + (int64_t)g.n[0] * (cy + (int64_t)g.n[1] * cz);
        node_cell[i] = (int32_t)c;
        node_cpk[i] = (uint32_t)cx | ((uint32_t)cy << 11) | ((uint32_t)cz << 22);
        atomicAdd(&cell_count[c], 1);
    }
}

__global__ void fill_cells(int64_t n, const int32_t *node_cell, const int32_t *cell_start,
                           int32_t *cursor, int32_t *sorted_ids)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t c = node_cell[i];
        int k = atomicAdd(&cursor[c], 1);
        sorted_ids[cell_start[c] + k] = (int32_t)i;
    }
}

// one thread per cell: insertion sort of the (few) ids, then coordinates
// in cell order and each node's rank in that order
__global__ void finish_cells(int64_t cells, const int32_t *cell_start, int32_t *sorted_ids,
                             const double *xyz, const InstGrid *ig, const int32_t *node_inst, double *sorted_xyz,
                             float *sorted_loc, int32_t *node_rank, int *max_cell)
{
    int mc = 0;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < cells;
         c += (int64_t)gridDim.x * blockDim.x) {
        int b = cell_start[c], e = cell_start[c + 1];
        mc = max(mc, e - b);
        for (int i = b + 1; i < e; i++) {
            int32_t v = sorted_ids[i];
            int j = i - 1;
            while (j >= b && sorted_ids[j] > v) { sorted_ids[j + 1] = sorted_ids[j]; j--; }
            sorted_ids[j + 1] = v;
        }
        for (int i = b; i < e; i++) {
            int32_t id = sorted_ids[i];
            node_rank[id] = i;
            sorted_xyz[4 * (int64_t)i + 0] = xyz[3 * (int64_t)id + 0];
            sorted_xyz[4 * (int64_t)i + 1] = xyz[3 * (int64_t)id + 1];
            sorted_xyz[4 * (int64_t)i + 2] = xyz[3 * (int64_t)id + 2];
            sorted_xyz[4 * (int64_t)i + 3] = 0.0;
            const InstGrid &g = ig[node_inst[id]];
            sorted_loc[4 * (int64_t)i + 0] = (float)((xyz[3 * (int64_t)id + 0] - g.lo[0]) * g.inv_edge);
            sorted_loc[4 * (int64_t)i + 1] = (float)((xyz[3 * (int64_t)id + 1] - g.lo[1]) * g.inv_edge);
            sorted_loc[4 * (int64_t)i + 2] = (float)((xyz[3 * (int64_t)id + 2] - g.lo[2]) * g.inv_edge);
            sorted_loc[4 * (int64_t)i + 3] = 0.0f;
        }
    }
    for (int o = 16; o > 0; o >>= 1) mc = max(mc, __shfl_down_sync(0xffffffffu, mc, o));
    if ((threadIdx.x & 31) == 0) atomicMax(max_cell, mc);
}

// ---------------------------------------------------------------------------
// Morton order of the nodes: key = instance << 32 | the Morton code of the
// node's cell (bits of cx, cy, cz interleaved, x lowest: 11 + 11 + 10 bits),
// sorted stably so that the nodes of a cell keep ascending ids. Rows taken in
// this order are spatially compact at every scale, so the warps working
// side by side share the integration points (and their shape-function
// records) they read.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t morton3(uint32_t x, uint32_t y, uint32_t z)
{
    uint32_t m = 0;
    for (int b = 0; b < 11; b++) {
        m |= ((x >> b) & 1u) << (3 * b);
        m |= ((y >> b) & 1u) << (3 * b + 1);
        if (b < 10) m |= ((z >> b) & 1u) << (3 * b + 2);
    }
    return m;
}

__global__ void morton_keys_kernel(int64_t n, const uint32_t *node_cpk, const int32_t *node_inst, uint64_t *keys,
                                   int32_t *ids)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t c = node_cpk[i];
        keys[i] = ((uint64_t)(uint32_t)node_inst[i] << 32) | morton3(c & 0x7FF, (c >> 11) & 0x7FF, c >> 22);
        ids[i] = (int32_t)i;
    }
}

// ---------------------------------------------------------------------------
// support search: one warp per point, 9 contiguous runs of 3 cells each.
// The squared distance is ((dx*dx + dy*dy) + dz*dz) in double with every
// operation rounded separately, the same expression on every platform.
// Pass 0 counts, pass 1 writes ids in ascending order.
// ---------------------------------------------------------------------------
constexpr int kSearchCap = 512;  // per-point list capacity in the fill pass

__device__ __forceinline__ double dist2(double4 n, double x, double y, double z)
{
    double dx = __dsub_rn(n.x, x), dy = __dsub_rn(n.y, y), dz = __dsub_rn(n.z, z);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

template <int PASS>
__global__ void __launch_bounds__(256) search_kernel(int64_t n_pts, const double *pts, const int32_t *inst_of,
                                                     int shift, const InstGrid *ig, const int32_t *cell_start,
                                                     const double4 *sorted_xyz, const float4 *sorted_loc,
                                                     const int32_t *sorted_ids,
                                                     int64_t *cnt_or_off, int32_t *sidx,
                                                     int *minmax, DevError *err)
{
    __shared__ int32_t list[8][kSearchCap];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    int mn = 1 << 30, mx = 0;
    for (int64_t p = (int64_t)blockIdx.x * (blockDim.x >> 5) + w; p < n_pts; p += warps) {
        const double x = pts[3 * p], y = pts[3 * p + 1], z = pts[3 * p + 2];
        const InstGrid &g = ig[instance_of(inst_of, shift, p)];
        const double rs2 = g.rs2;
        // cell of the point (may lie outside the grid: clamp the runs)
        int c[3];
        const double xs[3] = {x, y, z};
        for (int k = 0; k < 3; k++) {
            double f = floor((xs[k] - g.lo[k]) * g.inv_edge);
            f = fmin(fmax(f, -2.0), (double)g.n[k] + 1.0);
            c[k] = (int)f;
        }
        // the point in cell edges (FP32) for the prefilter
        const float ux = (float)((x - g.lo[0]) * g.inv_edge), uy = (float)((y - g.lo[1]) * g.inv_edge),
                    uz = (float)((z - g.lo[2]) * g.inv_edge);
        const float q_in = g.q_cell - g.margin, q_out = g.q_cell + g.margin;
        int count = 0;
        for (int dz = -1; dz <= 1; dz++) {
            int cz = c[2] + dz;
            if (cz < 0 || cz >= g.n[2]) continue;
            for (int dy = -1; dy <= 1; dy++) {
                int cy = c[1] + dy;
                if (cy < 0 || cy >= g.n[1]) continue;
                int xa = max(c[0] - 1, 0), xb = min(c[0] + 1, g.n[0] - 1);
                if (xa > xb) continue;
                int64_t row = g.cell_off + (int64_t)g.n[0] * (cy + (int64_t)g.n[1] * cz);
                int b = cell_start[row + xa], e = cell_start[row + xb + 1];
                for (int k0 = b; k0 < e; k0 += 32) {
                    int k = k0 + lane;
                    bool in = false;
                    if (k < e) {
                        const float4 l = sorted_loc[k];
                        const float ex = l.x - ux, ey = l.y - uy, ez = l.z - uz;
                        const float d2 = fmaf(ez, ez, fmaf(ey, ey, ex * ex));
                        in = d2 < q_in || (d2 <= q_out && dist2(sorted_xyz[k], x, y, z) <= rs2);
                    }
                    unsigned m = __ballot_sync(0xffffffffu, in);
                    if (PASS == 1 && in) {
                        int pos = count + __popc(m & ((1u << lane) - 1));
                        if (pos < kSearchCap) list[w][pos] = sorted_ids[k];
                    }
                    count += __popc(m);
                }
            }
        }
        if (PASS == 0) {
            if (lane == 0) cnt_or_off[p] = count;
            mn = min(mn, count);
            mx = max(mx, count);
        } else {
            if (count > kSearchCap) {
                if (lane == 0) dev_fail(err, RPIM_E_SUPPORT, p);
                continue;
            }
            __syncwarp();
            // bitonic sort of the ids, padded to a power of two
            int p2 = 1;
            while (p2 < count) p2 <<= 1;
            for (int i = count + lane; i < p2; i += 32) list[w][i] = INT32_MAX;
            __syncwarp();
            for (int k = 2; k <= p2; k <<= 1)
                for (int j = k >> 1; j > 0; j >>= 1) {
                    for (int i = lane; i < p2; i += 32) {
                        int ixj = i ^ j;
                        if (ixj > i) {
                            int32_t a = list[w][i], bb = list[w][ixj];
                            bool up = (i & k) == 0;
                            if ((a > bb) == up) { list[w][i] = bb; list[w][ixj] = a; }
                        }
                    }
                    __syncwarp();
                }
            int64_t o = cnt_or_off[p];
            for (int i = lane; i < count; i += 32) sidx[o + i] = list[w][i];
            __syncwarp();
        }
    }
    if (PASS == 0 && minmax) {
        for (int o = 16; o > 0; o >>= 1) {
            mn = min(mn, __shfl_down_sync(0xffffffffu, mn, o));
            mx = max(mx, __shfl_down_sync(0xffffffffu, mx, o));
        }
        if (lane == 0) {
            atomicMin(&minmax[0], mn);
            atomicMax(&minmax[1], mx);
        }
    }
}

rpim_status search_supports(rpim_pattern *p, int64_t n_pts, const double *pts, const int32_t *inst_of, int shift,
                            int64_t **soff_out, int32_t **sidx_out, int64_t *n_entries, int32_t *max_n,
                            int32_t *min_n, cudaStream_t s, const char *tag)
{
    int64_t *soff = nullptr, *tmp = nullptr;
    int32_t *sidx = nullptr;
    int *mm = nullptr;
    RPIM_CHECK(dalloc(&soff, n_pts + 1, s));
    RPIM_CHECK(dalloc(&tmp, scan_tmp_size(n_pts), s));
    RPIM_CHECK(dalloc(&mm, 2, s));
    int init[2] = {1 << 30, 0};
    RPIM_CUDA(cudaMemcpyAsync(mm, init, sizeof init, cudaMemcpyHostToDevice, s));
    int grid = grid_size(p->sm_count, 8, n_pts * 32, 256);
    launch(tag, search_kernel<0>, grid, 256, 0, s, n_pts, pts, inst_of, shift, (const InstGrid *)p->ig,
           (const int32_t *)p->cell_start, (const double4 *)p->sorted_xyz, (const float4 *)p->sorted_loc, (const int32_t *)p->sorted_ids, soff,
           (int32_t *)nullptr, mm, p->err);
    RPIM_CUDA(cudaGetLastError());
    RPIM_CHECK(exclusive_scan(soff, n_pts, tmp, s));
    int hm[2];
    int64_t ne = 0;
    RPIM_CUDA(cudaMemcpyAsync(hm, mm, sizeof hm, cudaMemcpyDeviceToHost, s));
    RPIM_CUDA(cudaMemcpyAsync(&ne, soff + n_pts, sizeof ne, cudaMemcpyDeviceToHost, s));
    RPIM_CUDA(cudaStreamSynchronize(s));
    dfree(tmp, s);
    dfree(mm, s);
    if (n_pts > 0 && (hm[0] < 4 || hm[1] > RPIM_MAX_SUPPORT)) {
        dfree(soff, s);
        char buf[160];
        snprintf(buf, sizeof buf, "support sizes %d..%d outside [4, %d]", hm[0], hm[1], RPIM_MAX_SUPPORT);
        return fail(RPIM_E_SUPPORT, buf);
    }
    RPIM_CHECK(dalloc(&sidx, ne, s));
    launch(tag, search_kernel<1>, grid, 256, 0, s, n_pts, pts, inst_of, shift, (const InstGrid *)p->ig,
           (const int32_t *)p->cell_start, (const double4 *)p->sorted_xyz, (const float4 *)p->sorted_loc, (const int32_t *)p->sorted_ids, soff, sidx,
           (int *)nullptr, p->err);
    RPIM_CUDA(cudaGetLastError());
    *soff_out = soff;
    *sidx_out = sidx;
    *n_entries = ne;
    *max_n = hm[1];
    *min_n = n_pts > 0 ? hm[0] : 0;
    return RPIM_OK;
}

// Support search into caller-provided device buffers (no allocation):
// soff [n_pts+1], tmp [scan_tmp_size(n_pts)], minmax [2], sidx [cap].
// Returns RPIM_E_ARG when the supports need more than `cap` entries.
// Synchronises s (the entry count comes back to the host).
rpim_status search_supports_into(rpim_pattern *p, int64_t n_pts, const double *pts, int64_t *soff, int64_t *tmp,
                                 int *minmax, int32_t *sidx, int64_t cap, int64_t *n_entries, int32_t *max_n,
                                 cudaStream_t s, const char *tag)
{
    const int init[2] = {1 << 30, 0};
    RPIM_CUDA(cudaMemcpyAsync(minmax, init, sizeof init, cudaMemcpyHostToDevice, s));
    const int grid = grid_size(p->sm_count, 8, n_pts * 32, 256);
    launch(tag, search_kernel<0>, grid, 256, 0, s, n_pts, pts, (const int32_t *)nullptr, 0, (const InstGrid *)p->ig,
           (const int32_t *)p->cell_start, (const double4 *)p->sorted_xyz, (const float4 *)p->sorted_loc, (const int32_t *)p->sorted_ids, soff,
           (int32_t *)nullptr, minmax, p->err);
    RPIM_CUDA(cudaGetLastError());
    RPIM_CHECK(exclusive_scan(soff, n_pts, tmp, s));
    int hm[2];
    int64_t ne = 0;
    RPIM_CUDA(cudaMemcpyAsync(hm, minmax, sizeof hm, cudaMemcpyDeviceToHost, s));
    RPIM_CUDA(cudaMemcpyAsync(&ne, soff + n_pts, sizeof ne, cudaMemcpyDeviceToHost, s));
    RPIM_CUDA(cudaStreamSynchronize(s));
    if (hm[0] < 4 || hm[1] > RPIM_MAX_SUPPORT) {
        char buf[160];
        snprintf(buf, sizeof buf, "support sizes %d..%d outside [4, %d]", hm[0], hm[1], RPIM_MAX_SUPPORT);
        return fail(RPIM_E_SUPPORT, buf);
    }
    if (ne > cap) {
        char buf[160];
        snprintf(buf, sizeof buf, "%lld support entries exceed the fixed scratch capacity of %lld", (long long)ne,
                 (long long)cap);
        return fail(RPIM_E_ARG, buf);
    }
    launch(tag, search_kernel<1>, grid, 256, 0, s, n_pts, pts, (const int32_t *)nullptr, 0, (const InstGrid *)p->ig,
           (const int32_t *)p->cell_start, (const double4 *)p->sorted_xyz, (const float4 *)p->sorted_loc, (const int32_t *)p->sorted_ids, soff, sidx,
           (int *)nullptr, p->err);
    RPIM_CUDA(cudaGetLastError());
    *n_entries = ne;
    *max_n = hm[1];
    return RPIM_OK;
}

// (packed cell, rank in cell) of every support entry's node: the row-owner
// kernels read it with the entry (one coalesced load) instead of gathering
// node_cpk[J] and node_rank[J] behind the load of J
__global__ void entry_cells_kernel(int64_t n_entries, const int32_t *__restrict__ sidx,
                                   const uint32_t *__restrict__ node_cpk, const int32_t *__restrict__ node_rank,
                                   uint2 *__restrict__ ecell)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_entries; e += stride) {
        const int32_t J = sidx[e];
        ecell[e] = make_uint2(node_cpk[J], (uint32_t)node_rank[J]);
    }
}

__global__ void entry_points_kernel(int64_t n_pts, const int64_t *soff, int32_t *entry_pt)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < n_pts; p += warps)
        for (int64_t e = soff[p] + lane; e < soff[p + 1]; e += 32) entry_pt[e] = (int32_t)p;
}

// ---------------------------------------------------------------------------
// BSR pattern, one warp per row I. The columns of row I are the union of the
// supports of the points whose support contains I; every such node lies
// within 2 r_s of I, i.e. in the 5x5x5 cells around I's cell (cell edge >=
// r_s). Those cells form 25 contiguous runs of the cell-ordered node list;
// the union is marked in a bitmap indexed by the position in these runs.
// Pass 0 marks the bitmap in shared memory, counts it and keeps it in global
// memory; pass 1 extracts the kept bitmap, sorts the ids and writes them.
// ---------------------------------------------------------------------------
// pass 0. The (point, support entry) pairs of row I are walked flat: 32
// incident points at a time, their supports concatenated and dealt to the
// lanes, so that every lane has independent loads in flight (walking one
// point at a time left most lanes idle behind a chain of dependent loads).
__global__ void pattern_bits_kernel(int64_t n_nodes, const InstGrid *ig, const int32_t *node_inst,
                                    const int32_t *cell_start, const uint32_t *node_cpk,
                                    const int64_t *toff, const int64_t *tent, const int32_t *entry_pt,
                                    const int64_t *soff, const uint2 *ecell, int64_t *rowcnt, uint32_t *bm,
                                    int words, int *maxrow, const int32_t *order, DevError *err)
{
    extern __shared__ uint32_t smem[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    uint32_t *bits = smem + (size_t)w * words;
    __shared__ int run_start[8][25], run_pre[8][26];
    const int64_t warps = (int64_t)gridDim.x * nw;
    int mrow = 0;
    for (int64_t rw = (int64_t)blockIdx.x * nw + w; rw < n_nodes; rw += warps) {
        const int64_t I = order ? (int64_t)order[rw] : rw;
        const InstGrid &g = ig[node_inst[I]];
        const uint32_t ci = node_cpk[I];
        const int cx = (int)(ci & 0x7FF), cy = (int)((ci >> 11) & 0x7FF), cz = (int)(ci >> 22);
        const int total = cell_runs(g, cell_start, cx, cy, cz, lane, run_start[w], run_pre[w]);
        const int64_t t_begin = toff[I], t_end = toff[I + 1];
        // a node that no integration point's support reaches would get an
        // empty row without a diagonal block (K singular): rejected here,
        // before any later stage indexes its row
        if (total > words * 32 || t_begin == t_end) {
            if (lane == 0) {
                dev_fail(err, RPIM_E_SUPPORT, I);
                rowcnt[I] = 0;
            }
            continue;
        }
        const int nwords = (total + 31) / 32;
        for (int i = lane; i < nwords; i += 32) bits[i] = 0;
        __syncwarp();
        for (int64_t t0 = t_begin; t0 < t_end; t0 += 32) {
            const int nt = (int)min((int64_t)32, t_end - t0);
            int64_t s0 = 0;
            int len = 0;
            if (lane < nt) {
                const int32_t pt = entry_pt[tent[t0 + lane]];
                s0 = soff[pt];
                len = (int)(soff[pt + 1] - s0);
            }
            int incl = len;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            const int excl = incl - len;     // lanes >= nt hold the total
            const int tot = __shfl_sync(0xffffffffu, incl, 31);
            for (int e0 = 0; e0 < tot; e0 += 32) {
                const int e = e0 + lane;
                int q = 0;                   // last point q with excl_q <= e
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const int ex = __shfl_sync(0xffffffffu, excl, q + step);
                    if (ex <= e) q += step;
                }
                const int64_t sq = __shfl_sync(0xffffffffu, s0, q);
                const int eq = __shfl_sync(0xffffffffu, excl, q);
                if (e < tot) {
                    const int bi = run_bit_cell(ecell[sq + (e - eq)], cx, cy, cz, run_start[w], run_pre[w]);
                    if (bi < 0) dev_fail(err, RPIM_E_ARG, I);
                    else atomicOr(&bits[bi >> 5], 1u << (bi & 31));
                }
            }
        }
        __syncwarp();
        int c = 0;
        uint32_t *out = bm + (size_t)I * words;
        for (int i = lane; i < nwords; i += 32) {
            const uint32_t v = bits[i];
            c += __popc(v);
            out[i] = v;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
        if (lane == 0) rowcnt[I] = c;
        mrow = max(mrow, c);
        __syncwarp();
    }
    for (int o = 16; o > 0; o >>= 1) mrow = max(mrow, __shfl_down_sync(0xffffffffu, mrow, o));
    if (lane == 0) atomicMax(maxrow, mrow);
}

// pass 1: the kept bitmap of row I in bitmap order (cell runs, ids ascending
// inside a cell), mapped to node ids, sorted (bitonic, shared memory) and
// written at rowptr[I]
__global__ void pattern_cols_kernel(int64_t n_nodes, const InstGrid *ig, const int32_t *node_inst,
                                    const int32_t *cell_start, const uint32_t *node_cpk, const int32_t *sorted_ids,
                                    const uint32_t *bm, int words, const int64_t *rowptr, int32_t *cols,
                                    int64_t *diag, int list_cap, const int32_t *order)
{
    extern __shared__ uint32_t smem[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    int32_t *list = (int32_t *)smem + (size_t)w * list_cap;
    __shared__ int run_start[8][25], run_pre[8][26];
    const int64_t warps = (int64_t)gridDim.x * nw;
    for (int64_t rw = (int64_t)blockIdx.x * nw + w; rw < n_nodes; rw += warps) {
        const int64_t I = order ? (int64_t)order[rw] : rw;
        const InstGrid &g = ig[node_inst[I]];
        const uint32_t ci = node_cpk[I];
        const int cx = (int)(ci & 0x7FF), cy = (int)((ci >> 11) & 0x7FF), cz = (int)(ci >> 22);
        const int total = cell_runs(g, cell_start, cx, cy, cz, lane, run_start[w], run_pre[w]);
        const int nwords = (total + 31) / 32;
        const uint32_t *in = bm + (size_t)I * words;
        int base = 0;
        for (int i0 = 0; i0 < nwords; i0 += 32) {
            const int i = i0 + lane;
            uint32_t word = i < nwords ? in[i] : 0u;
            const int pc = __popc(word);
            int incl = pc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            int pos = base + incl - pc;
            while (word) {
                const int bit = __ffs(word) - 1;
                word &= word - 1;
                const int bb = i * 32 + bit;
                int r = 0, hi = 25;  // run_pre[r] <= bb < run_pre[r + 1]
                while (hi - r > 1) {
                    const int mid = (r + hi) >> 1;
                    if (run_pre[w][mid] <= bb) r = mid; else hi = mid;
                }
                if (pos < list_cap) list[pos] = sorted_ids[run_start[w][r] + (bb - run_pre[w][r])];
                pos++;
            }
            base += __shfl_sync(0xffffffffu, incl, 31);
        }
        const int cnt = min(base, list_cap);
        __syncwarp();
        int p2 = 1;
        while (p2 < cnt) p2 <<= 1;
        for (int i = cnt + lane; i < p2; i += 32) list[i] = INT32_MAX;
        __syncwarp();
        for (int k = 2; k <= p2; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = lane; i < p2; i += 32) {
                    const int ixj = i ^ j;
                    if (ixj > i) {
                        const int32_t a = list[i], c = list[ixj];
                        const bool up = (i & k) == 0;
                        if ((a > c) == up) { list[i] = c; list[ixj] = a; }
                    }
                }
                __syncwarp();
            }
        const int64_t o = rowptr[I];
        for (int i = lane; i < cnt; i += 32) {
            cols[o + i] = list[i];
            if (list[i] == (int32_t)I) diag[I] = o + i;
        }
        __syncwarp();
    }
}

} // namespace rpim

using namespace rpim;

static void pattern_release(rpim_pattern *p)
{
    cudaStream_t s = p->stream;
    dfree(p->xyz, s); dfree(p->sorted_xyz, s); dfree(p->sorted_loc, s); dfree(p->sorted_ids, s); dfree(p->cell_start, s);
    dfree(p->node_cell, s); dfree(p->node_cpk, s); dfree(p->node_rank, s); dfree(p->pts, s); dfree(p->wj, s);
    dfree(p->row_order, s);
    dfree(p->soff, s); dfree(p->sidx, s); dfree(p->entry_pt, s); dfree(p->ecell, s); dfree(p->toff, s);
    dfree(p->tent, s); dfree(p->rowptr, s); dfree(p->cols, s); dfree(p->diag, s);
    dfree(p->phi, s); dfree(p->lamw, s); dfree(p->err, s); dfree(p->scal, s); dfree(p->series, s);
    dfree(p->ws.buf, s);
    dfree(p->ig, s); dfree(p->node_inst, s); dfree(p->bucket_order, s); dfree(p->tile_counter, s);
    dfree(p->shape_scratch, s);
    dfree(p->seg_row, s); dfree(p->seg_inst, s); dfree(p->inst_seg, s);
    if (p->asm_exec) cudaGraphExecDestroy(p->asm_exec);
    p->asm_exec = nullptr;
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    p->cap_stream = nullptr;
    p->ws.doubles = 0;
    p->n_seg = 0;
}

extern "C" rpim_status rpim_pattern_free(rpim_pattern *p)
{
    if (!p) return RPIM_OK;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(p->device);
    pattern_release(p);
    cudaStreamSynchronize(p->stream);
    cudaSetDevice(cur);
    delete p;
    return RPIM_OK;
}

extern "C" rpim_status rpim_pattern_get_info(const rpim_pattern *p, rpim_pattern_info *info)
{
    if (!p || !info) return fail(RPIM_E_ARG, "null argument");
    info->n_nodes = p->n_nodes;
    info->n_points = p->n_points;
    info->n_entries = p->n_entries;
    info->nnz_blocks = p->nnzb;
    info->max_support = p->max_support;
    info->min_support = p->min_support;
    info->max_row = p->max_row;
    info->device = p->device;
    return RPIM_OK;
}

extern "C" rpim_status rpim_pattern_csr(const rpim_pattern *p, const int64_t **rowptr,
                                        const int32_t **cols)
{
    if (!p) return fail(RPIM_E_ARG, "null pattern");
    if (rowptr) *rowptr = p->rowptr;
    if (cols) *cols = p->cols;
    return RPIM_OK;
}

extern "C" rpim_status rpim_pattern_points(const rpim_pattern *p, const double **xyz,
                                           const double **wj, const int64_t **soff,
                                           const int32_t **sidx)
{
    if (!p) return fail(RPIM_E_ARG, "null pattern");
    if (xyz) *xyz = p->pts;
    if (wj) *wj = p->wj;
    if (soff) *soff = p->soff;
    if (sidx) *sidx = p->sidx;
    return RPIM_OK;
}

extern "C" rpim_status rpim_pattern_copy_csr(const rpim_pattern *p, int64_t *rowptr, int32_t *cols,
                                             rpim_stream_t stream)
{
    if (!p) return fail(RPIM_E_ARG, "null pattern");
    cudaStream_t s = (cudaStream_t)stream;
    if (rowptr)
        RPIM_CUDA(cudaMemcpyAsync(rowptr, p->rowptr, (p->n_nodes + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    if (cols) RPIM_CUDA(cudaMemcpyAsync(cols, p->cols, p->nnzb * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    return RPIM_OK;
}

extern "C" rpim_status rpim_pattern_copy_row_order(const rpim_pattern *p, int32_t *order, rpim_stream_t stream)
{
    if (!p || !order) return fail(RPIM_E_ARG, "null argument");
    RPIM_CUDA(cudaMemcpyAsync(order, p->row_order, p->n_nodes * sizeof(int32_t), cudaMemcpyDeviceToDevice,
                              (cudaStream_t)stream));
    return RPIM_OK;
}

extern "C" rpim_status rpim_pattern_copy_points(const rpim_pattern *p, double *xyz, double *wj, int64_t *soff,
                                                int32_t *sidx, rpim_stream_t stream)
{
    if (!p) return fail(RPIM_E_ARG, "null pattern");
    cudaStream_t s = (cudaStream_t)stream;
    if (xyz) RPIM_CUDA(cudaMemcpyAsync(xyz, p->pts, 3 * p->n_points * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (wj) RPIM_CUDA(cudaMemcpyAsync(wj, p->wj, p->n_points * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (soff)
        RPIM_CUDA(cudaMemcpyAsync(soff, p->soff, (p->n_points + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    if (sidx) RPIM_CUDA(cudaMemcpyAsync(sidx, p->sidx, p->n_entries * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    return RPIM_OK;
}

// support-size bucket of every integration point; buckets group points for
// the shape kernel, whose shared memory per point grows with the support
__global__ void bucket_count_kernel(int64_t n_pts, const int64_t *soff, const int32_t *bounds, int nb,
                                    unsigned long long *count, int *bmax)
{
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n_pts;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int n = (int)(soff[g + 1] - soff[g]);
        int b = 0;
        while (b < nb - 1 && n > bounds[b]) b++;
        atomicAdd(&count[b], 1ull);
        atomicMax(&bmax[b], n);
    }
}

__global__ void bucket_fill_kernel(int64_t n_pts, const int64_t *soff, const int32_t *bounds, int nb,
                                   const int64_t *start, unsigned long long *cursor, int32_t *order)
{
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n_pts;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int n = (int)(soff[g + 1] - soff[g]);
        int b = 0;
        while (b < nb - 1 && n > bounds[b]) b++;
        order[start[b] + (int64_t)atomicAdd(&cursor[b], 1ull)] = (int32_t)g;
    }
}

static std::atomic<int> g_morton_rows{1};

namespace rpim {
// the order in which the row-owner kernels take their rows (null: node order)
const int32_t *rows_in_order(const rpim_pattern *p) { return g_morton_rows.load() ? p->row_order : nullptr; }
} // namespace rpim

extern "C" rpim_status rpim_set_row_order(int32_t morton)
{
    if (morton != 0 && morton != 1) return fail(RPIM_E_ARG, "row order must be 0 or 1");
    g_morton_rows.store(morton);
    return RPIM_OK;
}

// upper support size of each bucket (the last one is open-ended): the
// built-in bounds, or the process-wide choice of rpim_autotune_buckets
static const int32_t kBucketBounds[] = {40, 56, 72, 96, 128, 160, 1 << 30};
static const int kBuckets = 7;
static std::mutex g_bounds_mu;
static std::vector<int32_t> g_bounds(kBucketBounds, kBucketBounds + kBuckets);

namespace rpim {
void set_default_buckets(const std::vector<int32_t> &b)
{
    std::lock_guard<std::mutex> lk(g_bounds_mu);
    g_bounds = b.empty() ? std::vector<int32_t>(kBucketBounds, kBucketBounds + kBuckets) : b;
}
} // namespace rpim

static std::vector<int32_t> default_buckets()
{
    std::lock_guard<std::mutex> lk(g_bounds_mu);
    return g_bounds;
}

// Groups the integration points by support size: bucket b holds the
// points with bounds[b-1] < n <= bounds[b] (the last bound is open-ended).
// Recomputes the point order, counts and largest support of every bucket.
static rpim_status make_buckets(rpim_pattern *p, const std::vector<int32_t> &bounds_in, cudaStream_t s)
{
    std::vector<int32_t> bounds = bounds_in;
    if (bounds.empty() || bounds.back() < (1 << 30)) bounds.push_back(1 << 30);
    const int nb = (int)bounds.size();
    int32_t *dbounds = nullptr;
    unsigned long long *dcount = nullptr;
    int64_t *dstart = nullptr;
    int *dbmax = nullptr;
    rpim_status st = RPIM_OK;
    if ((st = dalloc(&dbounds, nb, s)) != RPIM_OK || (st = dalloc(&dcount, 2 * nb, s)) != RPIM_OK ||
        (st = dalloc(&dstart, nb, s)) != RPIM_OK || (st = dalloc(&dbmax, nb, s)) != RPIM_OK) {
        dfree(dbounds, s); dfree(dcount, s); dfree(dstart, s); dfree(dbmax, s);
        return st;
    }
    if (!p->bucket_order) RPIM_CHECK(dalloc(&p->bucket_order, p->n_points, s));
    std::vector<unsigned long long> hc(nb);
    std::vector<int> hm(nb);
    std::vector<int64_t> hs(nb);
    cudaError_t e = cudaMemcpyAsync(dbounds, bounds.data(), nb * sizeof(int32_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(dcount, 0, 2 * nb * sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(dbmax, 0, nb * sizeof(int), s);
    const int gsz = grid_size(p->sm_count, 4, p->n_points, 256);
    if (e == cudaSuccess) {
        launch("bucket_count", bucket_count_kernel, gsz, 256, 0, s, p->n_points, (const int64_t *)p->soff,
               (const int32_t *)dbounds, nb, dcount, dbmax);
        e = cudaMemcpyAsync(hc.data(), dcount, nb * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(hm.data(), dbmax, nb * sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) {
        int64_t acc = 0;
        p->bucket_count.assign(nb, 0);
        p->bucket_nc.assign(nb, 0);
        for (int b = 0; b < nb; b++) {
            hs[b] = acc;
            acc += (int64_t)hc[b];
            p->bucket_count[b] = (int64_t)hc[b];
            p->bucket_nc[b] = hm[b];
        }
        p->bucket_bounds = bounds;
        e = cudaMemcpyAsync(dstart, hs.data(), nb * sizeof(int64_t), cudaMemcpyHostToDevice, s);
    }
    if (e == cudaSuccess) {
        launch("bucket_fill", bucket_fill_kernel, gsz, 256, 0, s, p->n_points, (const int64_t *)p->soff,
               (const int32_t *)dbounds, nb, (const int64_t *)dstart, dcount + nb, p->bucket_order);
        e = cudaGetLastError();
    }
    // the host arrays above must outlive the copies that read them
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dfree(dbounds, s); dfree(dcount, s); dfree(dstart, s); dfree(dbmax, s);
    if (e != cudaSuccess) return cuda_fail(e, "support-size buckets");
    return RPIM_OK;
}

static rpim_status build(rpim_pattern *p, const double *xyz, const double *lo, const double *hi)
{
    cudaStream_t s = p->stream;
    const int64_t n = p->n_nodes;
    const int ni = p->n_inst;
    // the series for the largest support radius is valid for all instances
    RPIM_CHECK(build_kernel_series(p->prm.alpha_c, p->series_alpha_s, p->prm.q, &p->series_host));
    RPIM_CHECK(dalloc(&p->series, 1, s));
    RPIM_CUDA(cudaMemcpyAsync(p->series, &p->series_host, sizeof(KernelSeries), cudaMemcpyHostToDevice, s));
    RPIM_CHECK(dalloc(&p->err, 1, s));
    RPIM_CUDA(cudaMemsetAsync(p->err, 0xFF, sizeof(DevError), s));
    RPIM_CHECK(dalloc(&p->scal, 16, s));
    {
        int smem_sm = 0;
        RPIM_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, p->device));
        p->shape_scratch_doubles = (int64_t)p->sm_count * smem_sm / (int64_t)sizeof(double);
        RPIM_CHECK(dalloc(&p->shape_scratch, p->shape_scratch_doubles, s));
    }
    RPIM_CHECK(dalloc(&p->xyz, 3 * n, s));
    RPIM_CUDA(cudaMemcpyAsync(p->xyz, xyz, 3 * n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    RPIM_CHECK(dalloc(&p->ig, ni, s));
    RPIM_CUDA(cudaMemcpyAsync(p->ig, p->ig_host.data(), ni * sizeof(InstGrid), cudaMemcpyHostToDevice, s));
    RPIM_CHECK(dalloc(&p->node_inst, n, s));
    launch("node_inst", node_inst_kernel, ni, 256, 0, s, (const InstGrid *)p->ig, p->node_inst);

    // integration points
    p->n_points = 8 * n;
    RPIM_CHECK(dalloc(&p->pts, 3 * p->n_points, s));
    RPIM_CHECK(dalloc(&p->wj, p->n_points, s));
    launch("gauss_points", gauss_points_kernel, grid_size(p->sm_count, 8, p->n_points, 256), 256, 0, s, n, lo, hi, p->pts, p->wj);

    // bounding box of each instance -> its grid, cell edge >= its r_s
    unsigned long long *bb = nullptr;
    int *bad = nullptr;
    RPIM_CHECK(dalloc(&bb, 6 * ni, s));
    RPIM_CHECK(dalloc(&bad, 1, s));
    RPIM_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
    launch("bbox", bbox_kernel, ni, 256, 0, s, (const InstGrid *)p->ig, xyz, bb, bad);
    std::vector<unsigned long long> hb(6 * (size_t)ni);
    int hbad = 0;
    RPIM_CUDA(cudaMemcpyAsync(hb.data(), bb, hb.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    RPIM_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof hbad, cudaMemcpyDeviceToHost, s));
    RPIM_CUDA(cudaStreamSynchronize(s));
    dfree(bb, s);
    dfree(bad, s);
    if (hbad) return fail(RPIM_E_NONFINITE, "non-finite node coordinate");
    auto un = [](unsigned long long u) {
        unsigned long long b = (u & 0x8000000000000000ull) ? (u & 0x7FFFFFFFFFFFFFFFull) : ~u;
        double d;
        memcpy(&d, &b, 8);
        return d;
    };
    int64_t cell_off = 0;
    for (int i = 0; i < ni; i++) {
        InstGrid &g = p->ig_host[i];
        double bmin[3], bmax[3];
        for (int k = 0; k < 3; k++) {
            bmin[k] = un(hb[6 * i + k]);
            bmax[k] = un(hb[6 * i + 3 + k]);
        }
        double edge = sqrt(g.rs2) * (1.0 + 1e-9);
        int64_t cells = 1;
        for (;;) {
            cells = 1;
            bool ok = true;
            for (int k = 0; k < 3; k++) {
                double span = bmax[k] - bmin[k];
                int64_t nk = (int64_t)floor(span / edge) + 1;
                if (nk > (k == 2 ? 1023 : 2047)) ok = false;
                g.n[k] = (int)std::min<int64_t>(nk, 1 << 20);
                cells *= g.n[k];
            }
            if (ok && cells <= (int64_t)1 << 28) break;
            edge *= 1.25;
        }
        for (int k = 0; k < 3; k++) g.lo[k] = bmin[k];
        g.inv_edge = 1.0 / edge;
        // Single-precision prefilter of the support test. In cell edges the
        // test reads |u_n - u_p|^2 <= q, q = rs2 / edge^2, u = (x - lo) / edge.
        // Nodes and points are rounded to FP32 (|u| <= U = largest extent + 2),
        // every tested node lies within 2 cells of the point per axis, and the
        // squared distance is summed in FP32; the bound below covers these
        // roundings with a 1.5x reserve. Outside [q - margin, q + margin] the
        // FP32 decision equals the exact one; inside it the FP64 test decides.
        {
            const double q = g.rs2 * g.inv_edge * g.inv_edge;
            const double U = (double)std::max(g.n[0], std::max(g.n[1], g.n[2])) + 2.0;
            const double e24 = std::ldexp(1.0, -24), W = 2.0002 * U + 2.01;
            const double m = 3.0 * e24 * (q + 12.2) + 6.0 * 2.01 * e24 * W + 3.0 * e24 * e24 * W * W + 1e-12;
            g.q_cell = (float)q;
            g.margin = (float)(1.5 * m);
        }
        g.cell_off = cell_off;
        cell_off += cells;
    }
    if (cell_off > INT32_MAX) return fail(RPIM_E_ARG, "too many grid cells");
    p->total_cells = cell_off;
    RPIM_CUDA(cudaMemcpyAsync(p->ig, p->ig_host.data(), ni * sizeof(InstGrid), cudaMemcpyHostToDevice, s));

    // cell list (cell-major order per instance, ids ascending inside a cell)
    const int64_t cells = p->total_cells;
    int32_t *cursor = nullptr;
    int64_t *tmp = nullptr;
    int *dmax = nullptr;
    RPIM_CHECK(dalloc(&p->node_cell, n, s));
    RPIM_CHECK(dalloc(&p->node_cpk, n, s));
    RPIM_CHECK(dalloc(&p->node_rank, n, s));
    RPIM_CHECK(dalloc(&p->cell_start, cells + 1, s));
    RPIM_CHECK(dalloc(&cursor, cells + 1, s));
    RPIM_CHECK(dalloc(&tmp, scan_tmp_size(cells), s));
    RPIM_CHECK(dalloc(&p->sorted_ids, n, s));
    RPIM_CHECK(dalloc(&p->sorted_xyz, 4 * n, s));
    RPIM_CHECK(dalloc(&p->sorted_loc, 4 * n, s));
    RPIM_CHECK(dalloc(&dmax, 1, s));
    RPIM_CUDA(cudaMemsetAsync(p->cell_start, 0, (cells + 1) * sizeof(int32_t), s));
    RPIM_CUDA(cudaMemsetAsync(cursor, 0, (cells + 1) * sizeof(int32_t), s));
    RPIM_CUDA(cudaMemsetAsync(dmax, 0, sizeof(int), s));
    launch("bin_nodes", bin_nodes, grid_size(p->sm_count, 4, n, 256), 256, 0, s, n, xyz, (const InstGrid *)p->ig,
           (const int32_t *)p->node_inst, p->node_cell, p->node_cpk, p->cell_start);
    RPIM_CHECK(exclusive_scan32(p->cell_start, cells, tmp, s));
    launch("fill_cells", fill_cells, grid_size(p->sm_count, 4, n, 256), 256, 0, s, n, p->node_cell, p->cell_start, cursor, p->sorted_ids);
    launch("finish_cells", finish_cells, grid_size(p->sm_count, 4, cells, 128), 128, 0, s, cells, p->cell_start, p->sorted_ids, xyz,
           (const InstGrid *)p->ig, (const int32_t *)p->node_inst, p->sorted_xyz, p->sorted_loc, p->node_rank, dmax);
    RPIM_CUDA(cudaGetLastError());
    RPIM_CUDA(cudaMemcpyAsync(&p->max_cell, dmax, sizeof(int), cudaMemcpyDeviceToHost, s));
    dfree(cursor, s);
    dfree(tmp, s);
    dfree(dmax, s);

    // Morton order of the rows (instance first; see morton_keys_kernel)
    {
        uint64_t *keys = nullptr;
        RPIM_CHECK(dalloc(&keys, n, s));
        RPIM_CHECK(dalloc(&p->row_order, n, s));
        launch("morton_keys", morton_keys_kernel, grid_size(p->sm_count, 4, n, 256), 256, 0, s, n,
               (const uint32_t *)p->node_cpk, (const int32_t *)p->node_inst, keys, p->row_order);
        int ibits = 0;
        while ((1ll << ibits) < (long long)ni) ibits++;
        const rpim_status st = radix_sort_pairs(keys, p->row_order, n, 32 + ibits, s);
        dfree(keys, s);
        RPIM_CHECK(st);
    }

    // supports of the integration points (point g belongs to node g/8)
    RPIM_CHECK(search_supports(p, p->n_points, p->pts, p->node_inst, 3, &p->soff, &p->sidx, &p->n_entries,
                               &p->max_support, &p->min_support, s, "search"));
    RPIM_CHECK(dalloc(&p->entry_pt, p->n_entries, s));
    launch("entry_points", entry_points_kernel, grid_size(p->sm_count, 8, p->n_points * 32, 256), 256, 0, s, p->n_points, p->soff, p->entry_pt);
    RPIM_CHECK(dalloc(&p->ecell, p->n_entries, s));
    launch("entry_cells", entry_cells_kernel, grid_size(p->sm_count, 8, p->n_entries, 256), 256, 0, s, p->n_entries,
           (const int32_t *)p->sidx, (const uint32_t *)p->node_cpk, (const int32_t *)p->node_rank, p->ecell);
    RPIM_CHECK(build_incidence(n, p->n_entries, p->sidx, &p->toff, &p->tent, &p->max_incident, s, p->sm_count));

    // support-size buckets
    RPIM_CHECK(make_buckets(p, default_buckets(), s));

    // BSR pattern
    const int words = (125 * p->max_cell + 31) / 32 + 1;
    RPIM_CHECK(dalloc(&p->rowptr, n + 1, s));
    RPIM_CHECK(dalloc(&p->diag, n, s));
    RPIM_CUDA(cudaMemsetAsync(p->diag, 0xFF, n * sizeof(int64_t), s));   // -1: no diagonal block
    RPIM_CHECK(dalloc(&dmax, 1, s));
    RPIM_CHECK(dalloc(&tmp, scan_tmp_size(n), s));
    RPIM_CUDA(cudaMemsetAsync(dmax, 0, sizeof(int), s));
    p->bit_words = words;
    uint32_t *bm = nullptr;   // kept bitmaps of pass 0, [n][words]
    RPIM_CHECK(dalloc(&bm, (int64_t)n * words, s));
    {
        const int wpb = 8;
        size_t smem = (size_t)wpb * words * 4;
        if (smem > 227 * 1024) {
            dfree(bm, s);
            return fail(RPIM_E_SUPPORT, "pattern bitmap too large for shared memory (too many nodes per cell)");
        }
        if (smem > 48 * 1024)
            RPIM_CUDA(cudaFuncSetAttribute(pattern_bits_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        launch("pattern_count", pattern_bits_kernel, grid_size(p->sm_count, 4, n, wpb), wpb * 32, smem, s,
               n, (const InstGrid *)p->ig, (const int32_t *)p->node_inst, (const int32_t *)p->cell_start,
               (const uint32_t *)p->node_cpk, (const int64_t *)p->toff,
               (const int64_t *)p->tent, (const int32_t *)p->entry_pt, (const int64_t *)p->soff,
               (const uint2 *)p->ecell, p->rowptr, bm, words, dmax, rows_in_order(p), p->err);
        RPIM_CUDA(cudaGetLastError());
    }
    RPIM_CHECK(exclusive_scan(p->rowptr, n, tmp, s));
    int hmax = 0;
    RPIM_CUDA(cudaMemcpyAsync(&hmax, dmax, sizeof(int), cudaMemcpyDeviceToHost, s));
    RPIM_CUDA(cudaMemcpyAsync(&p->nnzb, p->rowptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    RPIM_CUDA(cudaStreamSynchronize(s));
    dfree(tmp, s);
    dfree(dmax, s);
    rpim_status st = check_device_error(p, "pattern");
    if (st != RPIM_OK) {
        dfree(bm, s);
        return st;
    }
    p->max_row = hmax;
    st = dalloc(&p->cols, p->nnzb, s);
    if (st == RPIM_OK) {
        int p2 = 1;
        while (p2 < hmax) p2 <<= 1;
        int wpb = 8;
        const size_t per = (size_t)p2 * 4;
        while (wpb > 1 && wpb * per > 200 * 1024) wpb >>= 1;
        const size_t smem = wpb * per;
        if (smem > 227 * 1024) st = fail(RPIM_E_SUPPORT, "pattern row too long for shared memory");
        else if (cudaFuncSetAttribute(pattern_cols_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                 cudaSuccess)
            st = fail(RPIM_E_CUDA, "pattern: shared memory attribute");
        else {
            launch("pattern_fill", pattern_cols_kernel, grid_size(p->sm_count, 4, n, wpb), wpb * 32, smem, s,
                   n, (const InstGrid *)p->ig, (const int32_t *)p->node_inst, (const int32_t *)p->cell_start,
                   (const uint32_t *)p->node_cpk, (const int32_t *)p->sorted_ids, (const uint32_t *)bm, words,
                   (const int64_t *)p->rowptr, p->cols, p->diag, p2, rows_in_order(p));
            if (cudaGetLastError() != cudaSuccess) st = fail(RPIM_E_CUDA, "pattern fill launch");
        }
    }
    dfree(bm, s);
    RPIM_CHECK(st);
    RPIM_CHECK(check_device_error(p, "pattern"));
    return RPIM_OK;
}

static rpim_status create(int32_t n_inst, const rpim_instance *inst, const double *xyz, const double *cell_lo,
                          const double *cell_hi, double alpha_c, double q, int32_t gauss_order, rpim_stream_t stream,
                          rpim_pattern **out, int64_t *nnz_blocks)
{
    if (!out) return fail(RPIM_E_ARG, "out is null");
    *out = nullptr;
    if (n_inst < 1 || !inst || !xyz || !cell_lo || !cell_hi) return fail(RPIM_E_ARG, "bad instance list or null pointer");
    if (gauss_order != 2) return fail(RPIM_E_ARG, "only gauss_order = 2 is implemented");
    if (!(alpha_c > 0) || !(q > 0)) return fail(RPIM_E_ARG, "non-positive RPIM parameter");
    int64_t n = 0;
    double as_max = 0.0;
    for (int i = 0; i < n_inst; i++) {
        if (inst[i].n_nodes < 4 || !(inst[i].h > 0) || !(inst[i].alpha_s > 0))
            return fail(RPIM_E_ARG, "instance with fewer than 4 nodes or a non-positive parameter");
        n += inst[i].n_nodes;
        as_max = std::max(as_max, inst[i].alpha_s);
    }
    if (n > INT32_MAX / 8) return fail(RPIM_E_ARG, "too many nodes");
    rpim_pattern *p = new (std::nothrow) rpim_pattern();
    if (!p) return fail(RPIM_E_OOM, "host allocation");
    p->stream = (cudaStream_t)stream;
    p->prm.alpha_s = inst[0].alpha_s;
    p->prm.h = inst[0].h;
    p->prm.alpha_c = alpha_c;
    p->prm.q = q;
    p->prm.gauss_order = gauss_order;
    p->series_alpha_s = as_max;
    p->n_inst = n_inst;
    p->n_nodes = n;
    p->ig_host.resize(n_inst);
    int64_t nb = 0;
    for (int i = 0; i < n_inst; i++) {
        InstGrid &g = p->ig_host[i];
        memset(&g, 0, sizeof g);
        const double rs = inst[i].alpha_s * inst[i].h;
        g.rs2 = rs * rs;
        g.inv_h = 1.0 / inst[i].h;
        g.node_begin = nb;
        nb += inst[i].n_nodes;
        g.node_end = nb;
    }
    cudaGetDevice(&p->device);
    cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->device);
    {
        // keep freed stream-ordered allocations cached in this process's
        // default pool, so that repeated builds do not remap memory
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, p->device) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
    }
    rpim_status st = build(p, xyz, cell_lo, cell_hi);
    if (st != RPIM_OK) {
        std::string msg = rpim_last_error();
        rpim_pattern_free(p);
        return fail(st, msg);
    }
    if (nnz_blocks) *nnz_blocks = p->nnzb;
    *out = p;
    return RPIM_OK;
}

extern "C" rpim_status rpim_build_pattern(int64_t n_nodes, const double *xyz, const double *cell_lo,
                                          const double *cell_hi, const rpim_params *params,
                                          rpim_stream_t stream, rpim_pattern **out, int64_t *nnz_blocks)
{
    RPIM_STAGE("rpim_build_pattern");
    if (out) *out = nullptr;
    if (!params) return fail(RPIM_E_ARG, "params is null");
    if (n_nodes < 4 || n_nodes > INT32_MAX / 8 || !xyz || !cell_lo || !cell_hi)
        return fail(RPIM_E_ARG, "bad node count or null pointer");
    if (!(params->h > 0) || !(params->alpha_s > 0)) return fail(RPIM_E_ARG, "non-positive RPIM parameter");
    rpim_instance one{n_nodes, params->alpha_s, params->h};
    return create(1, &one, xyz, cell_lo, cell_hi, params->alpha_c, params->q, params->gauss_order, stream, out,
                  nnz_blocks);
}

extern "C" rpim_status rpim_build_pattern_batched(int32_t n_inst, const rpim_instance *inst, const double *xyz,
                                                  const double *cell_lo, const double *cell_hi, double alpha_c,
                                                  double q, int32_t gauss_order, rpim_stream_t stream,
                                                  rpim_pattern **out, int64_t *nnz_blocks)
{
    RPIM_STAGE("rpim_build_pattern_batched");
    return create(n_inst, inst, xyz, cell_lo, cell_hi, alpha_c, q, gauss_order, stream, out, nnz_blocks);
}

extern "C" rpim_status rpim_pattern_set_buckets(rpim_pattern *p, int32_t n_bounds, const int32_t *bounds,
                                                rpim_stream_t stream)
{
    RPIM_STAGE("rpim_pattern_set_buckets");
    if (!p || n_bounds < 1 || n_bounds > 31 || !bounds) return fail(RPIM_E_ARG, "bad bucket bounds");
    for (int i = 0; i < n_bounds; i++)
        if (bounds[i] < 1 || (i > 0 && bounds[i] <= bounds[i - 1])) return fail(RPIM_E_ARG, "bucket bounds must increase");
    cudaStream_t s = (cudaStream_t)stream;
    p->stream = s;
    return make_buckets(p, std::vector<int32_t>(bounds, bounds + n_bounds), s);
}

extern "C" rpim_status rpim_pattern_get_buckets(const rpim_pattern *p, int32_t *n_buckets, int32_t *bounds,
                                                int32_t *max_support, int64_t *counts, int32_t capacity)
{
    if (!p || !n_buckets) return fail(RPIM_E_ARG, "null argument");
    const int nb = (int)p->bucket_count.size();
    *n_buckets = nb;
    for (int b = 0; b < nb && b < capacity; b++) {
        if (bounds) bounds[b] = p->bucket_bounds.empty() ? 0 : p->bucket_bounds[b];
        if (max_support) max_support[b] = p->bucket_nc[b];
        if (counts) counts[b] = p->bucket_count[b];
    }
    return RPIM_OK;
}
