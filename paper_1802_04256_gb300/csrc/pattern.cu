// Stage 1a: integration points, uniform-grid cell list, support search,
// node -> point incidence and the BSR pattern of K, all on the device.
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <string>

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

__global__ void bbox_kernel(int64_t n, const double *xyz, unsigned long long *bb /*6: min xyz, max xyz*/,
                            int *bad)
{
    unsigned long long mn[3] = {~0ull, ~0ull, ~0ull}, mx[3] = {0, 0, 0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        for (int k = 0; k < 3; k++) {
            double v = xyz[3 * i + k];
            if (!isfinite(v)) atomicExch(bad, 1);
            unsigned long long o = ordered(v);
            mn[k] = min(mn[k], o);
            mx[k] = max(mx[k], o);
        }
    for (int k = 0; k < 3; k++) {
        for (int o = 16; o > 0; o >>= 1) {
            mn[k] = min(mn[k], __shfl_down_sync(0xffffffffu, mn[k], o));
            mx[k] = max(mx[k], __shfl_down_sync(0xffffffffu, mx[k], o));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(&bb[k], mn[k]);
            atomicMax(&bb[3 + k], mx[k]);
        }
    }
}

__device__ __forceinline__ int cell_coord(double x, double lo, double inv_edge, int n)
{
    double c = floor((x - lo) * inv_edge);
    if (c < 0) return 0;
    if (c > n - 1) return n - 1;
    return (int)c;
}

__global__ void bin_nodes(int64_t n, const double *xyz, Grid g, int32_t *node_cell, uint32_t *node_cpk,
                          int32_t *cell_count)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int cx = cell_coord(xyz[3 * i], g.lo[0], g.inv_edge, g.n[0]);
        int cy = cell_coord(xyz[3 * i + 1], g.lo[1], g.inv_edge, g.n[1]);
        int cz = cell_coord(xyz[3 * i + 2], g.lo[2], g.inv_edge, g.n[2]);
        int32_t c = cx + g.n[0] * (cy + g.n[1] * cz);
        node_cell[i] = c;
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
                             const double *xyz, double *sorted_xyz, int32_t *node_rank, int *max_cell)
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
        }
    }
    for (int o = 16; o > 0; o >>= 1) mc = max(mc, __shfl_down_sync(0xffffffffu, mc, o));
    if ((threadIdx.x & 31) == 0) atomicMax(max_cell, mc);
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
__global__ void __launch_bounds__(256) search_kernel(int64_t n_pts, const double *pts, Grid g,
                                                     const int32_t *cell_start,
                                                     const double4 *sorted_xyz,
                                                     const int32_t *sorted_ids, double rs2,
                                                     int64_t *cnt_or_off, int32_t *sidx,
                                                     int *minmax, DevError *err)
{
    __shared__ int32_t list[8][kSearchCap];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    int mn = 1 << 30, mx = 0;
    for (int64_t p = (int64_t)blockIdx.x * (blockDim.x >> 5) + w; p < n_pts; p += warps) {
        const double x = pts[3 * p], y = pts[3 * p + 1], z = pts[3 * p + 2];
        // cell of the point (may lie outside the grid: clamp the runs)
        int c[3];
        const double xs[3] = {x, y, z};
        for (int k = 0; k < 3; k++) {
            double f = floor((xs[k] - g.lo[k]) * g.inv_edge);
            f = fmin(fmax(f, -2.0), (double)g.n[k] + 1.0);
            c[k] = (int)f;
        }
        int count = 0;
        for (int dz = -1; dz <= 1; dz++) {
            int cz = c[2] + dz;
            if (cz < 0 || cz >= g.n[2]) continue;
            for (int dy = -1; dy <= 1; dy++) {
                int cy = c[1] + dy;
                if (cy < 0 || cy >= g.n[1]) continue;
                int xa = max(c[0] - 1, 0), xb = min(c[0] + 1, g.n[0] - 1);
                if (xa > xb) continue;
                int64_t row = (int64_t)g.n[0] * (cy + (int64_t)g.n[1] * cz);
                int b = cell_start[row + xa], e = cell_start[row + xb + 1];
                for (int k0 = b; k0 < e; k0 += 32) {
                    int k = k0 + lane;
                    bool in = false;
                    if (k < e) in = dist2(sorted_xyz[k], x, y, z) <= rs2;
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

rpim_status search_supports(rpim_pattern *p, int64_t n_pts, const double *pts, int64_t **soff_out,
                            int32_t **sidx_out, int64_t *n_entries, int32_t *max_n, int32_t *min_n,
                            cudaStream_t s, const char *tag)
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
    launch(tag, search_kernel<0>, grid, 256, 0, s, n_pts, pts, p->grid, p->cell_start,
                                          (const double4 *)p->sorted_xyz, p->sorted_ids, p->rs2,
                                          soff, nullptr, mm, p->err);
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
    launch(tag, search_kernel<1>, grid, 256, 0, s, n_pts, pts, p->grid, p->cell_start,
                                          (const double4 *)p->sorted_xyz, p->sorted_ids, p->rs2,
                                          soff, sidx, nullptr, p->err);
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
    launch(tag, search_kernel<0>, grid, 256, 0, s, n_pts, pts, p->grid, p->cell_start,
           (const double4 *)p->sorted_xyz, p->sorted_ids, p->rs2, soff, (int32_t *)nullptr, minmax, p->err);
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
    launch(tag, search_kernel<1>, grid, 256, 0, s, n_pts, pts, p->grid, p->cell_start,
           (const double4 *)p->sorted_xyz, p->sorted_ids, p->rs2, soff, sidx, (int *)nullptr, p->err);
    RPIM_CUDA(cudaGetLastError());
    *n_entries = ne;
    *max_n = hm[1];
    return RPIM_OK;
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
// the union is marked in a shared-memory bitmap indexed by the position in
// these runs, counted (pass 0), then extracted, sorted and written (pass 1).
// ---------------------------------------------------------------------------
template <int PASS>
__global__ void pattern_kernel(int64_t n_nodes, Grid g, const int32_t *cell_start,
                               const int32_t *node_cell, const uint32_t *node_cpk, const int32_t *node_rank,
                               const int32_t *sorted_ids, const int64_t *toff, const int64_t *tent,
                               const int32_t *entry_pt, const int64_t *soff, const int32_t *sidx,
                               int64_t *rowcnt_or_ptr, int32_t *cols, int64_t *diag, int words,
                               int list_cap, int *maxrow, DevError *err)
{
    extern __shared__ uint32_t smem[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    uint32_t *bits = smem + (size_t)w * words;
    int32_t *list = (int32_t *)(smem + (size_t)nw * words) + (size_t)w * list_cap;
    __shared__ int run_start[8][25], run_pre[8][26];
    const int64_t warps = (int64_t)gridDim.x * nw;
    int mrow = 0;
    for (int64_t I = (int64_t)blockIdx.x * nw + w; I < n_nodes; I += warps) {
        const int32_t ci = node_cell[I];
        const int cx = ci % g.n[0], cy = (ci / g.n[0]) % g.n[1], cz = ci / (g.n[0] * g.n[1]);
        if (lane < 25) {
            int dy = lane % 5 - 2, dz = lane / 5 - 2;
            int yy = cy + dy, zz = cz + dz;
            int st = 0, len = 0;
            if (yy >= 0 && yy < g.n[1] && zz >= 0 && zz < g.n[2]) {
                int xa = max(cx - 2, 0), xb = min(cx + 2, g.n[0] - 1);
                int64_t row = (int64_t)g.n[0] * (yy + (int64_t)g.n[1] * zz);
                st = cell_start[row + xa];
                len = cell_start[row + xb + 1] - st;
            }
            run_start[w][lane] = st;
            run_pre[w][lane + 1] = len;
        }
        __syncwarp();
        if (lane == 0) {
            run_pre[w][0] = 0;
            for (int r = 0; r < 25; r++) run_pre[w][r + 1] += run_pre[w][r];
        }
        __syncwarp();
        const int total = run_pre[w][25];
        if (total > words * 32) {
            if (lane == 0) dev_fail(err, RPIM_E_SUPPORT, I);
            continue;
        }
        for (int i = lane; i < (total + 31) / 32; i += 32) bits[i] = 0;
        __syncwarp();
        for (int64_t t = toff[I]; t < toff[I + 1]; t++) {
            const int32_t pt = entry_pt[tent[t]];
            for (int64_t f = soff[pt] + lane; f < soff[pt + 1]; f += 32) {
                const int32_t J = sidx[f];
                const uint32_t cj = node_cpk[J];
                const int jx = (int)(cj & 0x7FF), jy = (int)((cj >> 11) & 0x7FF), jz = (int)(cj >> 22);
                const int dx = jx - cx, dy = jy - cy, dz = jz - cz;
                if (dx < -2 || dx > 2 || dy < -2 || dy > 2 || dz < -2 || dz > 2) {
                    dev_fail(err, RPIM_E_ARG, I);
                    continue;
                }
                const int r = (dy + 2) + 5 * (dz + 2);
                const int b = run_pre[w][r] + (node_rank[J] - run_start[w][r]);
                atomicOr(&bits[b >> 5], 1u << (b & 31));
            }
        }
        __syncwarp();
        int nwords = (total + 31) / 32;
        if (PASS == 0) {
            int c = 0;
            for (int i = lane; i < nwords; i += 32) c += __popc(bits[i]);
            for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
            if (lane == 0) rowcnt_or_ptr[I] = c;
            mrow = max(mrow, c);
        } else {
            // extract in bitmap order: words in chunks of 32 lanes
            int base = 0;
            for (int i0 = 0; i0 < nwords; i0 += 32) {
                int i = i0 + lane;
                uint32_t word = i < nwords ? bits[i] : 0u;
                int pc = __popc(word), incl = pc;
                for (int o = 1; o < 32; o <<= 1) {
                    int v = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += v;
                }
                int pos = base + incl - pc;
                while (word) {
                    int bit = __ffs(word) - 1;
                    word &= word - 1;
                    int b = i * 32 + bit;
                    int r = 0, hi = 25;  // run_pre[r] <= b < run_pre[r + 1]
                    while (hi - r > 1) {
                        const int mid = (r + hi) >> 1;
                        if (run_pre[w][mid] <= b) r = mid; else hi = mid;
                    }
                    int spos = run_start[w][r] + (b - run_pre[w][r]);
                    if (pos < list_cap) list[pos] = sorted_ids[spos];
                    pos++;
                }
                base += __shfl_sync(0xffffffffu, incl, 31);
            }
            const int cnt = base;
            __syncwarp();
            int p2 = 1;
            while (p2 < cnt) p2 <<= 1;
            for (int i = cnt + lane; i < p2; i += 32) list[i] = INT32_MAX;
            __syncwarp();
            for (int k = 2; k <= p2; k <<= 1)
                for (int j = k >> 1; j > 0; j >>= 1) {
                    for (int i = lane; i < p2; i += 32) {
                        int ixj = i ^ j;
                        if (ixj > i) {
                            int32_t a = list[i], bb = list[ixj];
                            bool up = (i & k) == 0;
                            if ((a > bb) == up) { list[i] = bb; list[ixj] = a; }
                        }
                    }
                    __syncwarp();
                }
            const int64_t o = rowcnt_or_ptr[I];
            for (int i = lane; i < cnt; i += 32) {
                cols[o + i] = list[i];
                if (list[i] == (int32_t)I) diag[I] = o + i;
            }
            __syncwarp();
        }
    }
    if (PASS == 0) {
        for (int o = 16; o > 0; o >>= 1) mrow = max(mrow, __shfl_down_sync(0xffffffffu, mrow, o));
        if (lane == 0) atomicMax(maxrow, mrow);
    }
}

} // namespace rpim

using namespace rpim;

static void pattern_release(rpim_pattern *p)
{
    cudaStream_t s = p->stream;
    dfree(p->xyz, s); dfree(p->sorted_xyz, s); dfree(p->sorted_ids, s); dfree(p->cell_start, s);
    dfree(p->node_cell, s); dfree(p->node_cpk, s); dfree(p->node_rank, s); dfree(p->pts, s); dfree(p->wj, s);
    dfree(p->soff, s); dfree(p->sidx, s); dfree(p->entry_pt, s); dfree(p->toff, s);
    dfree(p->tent, s); dfree(p->rowptr, s); dfree(p->cols, s); dfree(p->diag, s);
    dfree(p->phi, s); dfree(p->lamw, s); dfree(p->err, s); dfree(p->scal, s); dfree(p->series, s);
    dfree(p->ws.buf, s);
    p->ws.doubles = 0;
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

static rpim_status build(rpim_pattern *p, const double *xyz, const double *lo, const double *hi)
{
    cudaStream_t s = p->stream;
    const int64_t n = p->n_nodes;
    RPIM_CHECK(build_kernel_series(p->prm.alpha_c, p->prm.alpha_s, p->prm.q, &p->series_host));
    RPIM_CHECK(dalloc(&p->series, 1, s));
    RPIM_CUDA(cudaMemcpyAsync(p->series, &p->series_host, sizeof(KernelSeries), cudaMemcpyHostToDevice, s));
    RPIM_CHECK(dalloc(&p->err, 1, s));
    RPIM_CUDA(cudaMemsetAsync(p->err, 0xFF, sizeof(DevError), s));
    RPIM_CHECK(dalloc(&p->scal, 16, s));
    RPIM_CHECK(dalloc(&p->xyz, 3 * n, s));
    RPIM_CUDA(cudaMemcpyAsync(p->xyz, xyz, 3 * n * sizeof(double), cudaMemcpyDeviceToDevice, s));

    // integration points
    p->n_points = 8 * n;
    RPIM_CHECK(dalloc(&p->pts, 3 * p->n_points, s));
    RPIM_CHECK(dalloc(&p->wj, p->n_points, s));
    launch("gauss_points", gauss_points_kernel, grid_size(p->sm_count, 8, p->n_points, 256), 256, 0, s, n, lo, hi, p->pts, p->wj);

    // bounding box -> grid with cell edge >= r_s
    unsigned long long *bb = nullptr;
    int *bad = nullptr;
    RPIM_CHECK(dalloc(&bb, 6, s));
    RPIM_CHECK(dalloc(&bad, 1, s));
    unsigned long long init[6] = {~0ull, ~0ull, ~0ull, 0, 0, 0};
    RPIM_CUDA(cudaMemcpyAsync(bb, init, sizeof init, cudaMemcpyHostToDevice, s));
    RPIM_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
    launch("bbox", bbox_kernel, grid_size(p->sm_count, 4, n, 256), 256, 0, s, n, xyz, bb, bad);
    unsigned long long hb[6];
    int hbad = 0;
    RPIM_CUDA(cudaMemcpyAsync(hb, bb, sizeof hb, cudaMemcpyDeviceToHost, s));
    RPIM_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof hbad, cudaMemcpyDeviceToHost, s));
    RPIM_CUDA(cudaStreamSynchronize(s));
    dfree(bb, s);
    dfree(bad, s);
    if (hbad) return fail(RPIM_E_NONFINITE, "non-finite node coordinate");
    double bmin[3], bmax[3];
    for (int k = 0; k < 3; k++) {
        auto un = [](unsigned long long u) {
            unsigned long long b = (u & 0x8000000000000000ull) ? (u & 0x7FFFFFFFFFFFFFFFull) : ~u;
            double d;
            memcpy(&d, &b, 8);
            return d;
        };
        bmin[k] = un(hb[k]);
        bmax[k] = un(hb[3 + k]);
    }
    const double rs = sqrt(p->rs2);
    double edge = rs * (1.0 + 1e-9);
    for (;;) {
        int64_t cells = 1;
        bool ok = true;
        for (int k = 0; k < 3; k++) {
            double span = bmax[k] - bmin[k];
            int64_t nk = (int64_t)floor(span / edge) + 1;
            if (nk > (k == 2 ? 1023 : 2047)) ok = false;
            p->grid.n[k] = (int)std::min<int64_t>(nk, 1 << 20);
            cells *= p->grid.n[k];
        }
        if (ok && cells <= (int64_t)1 << 28) {
            p->grid.cells = cells;
            break;
        }
        edge *= 1.25;
    }
    for (int k = 0; k < 3; k++) p->grid.lo[k] = bmin[k];
    p->grid.inv_edge = 1.0 / edge;

    // cell list (cell-major order, ids ascending inside a cell)
    const int64_t cells = p->grid.cells;
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
    RPIM_CHECK(dalloc(&dmax, 1, s));
    RPIM_CUDA(cudaMemsetAsync(p->cell_start, 0, (cells + 1) * sizeof(int32_t), s));
    RPIM_CUDA(cudaMemsetAsync(cursor, 0, (cells + 1) * sizeof(int32_t), s));
    RPIM_CUDA(cudaMemsetAsync(dmax, 0, sizeof(int), s));
    launch("bin_nodes", bin_nodes, grid_size(p->sm_count, 4, n, 256), 256, 0, s, n, xyz, p->grid, p->node_cell,
           p->node_cpk, p->cell_start);
    RPIM_CHECK(exclusive_scan32(p->cell_start, cells, tmp, s));
    launch("fill_cells", fill_cells, grid_size(p->sm_count, 4, n, 256), 256, 0, s, n, p->node_cell, p->cell_start, cursor, p->sorted_ids);
    launch("finish_cells", finish_cells, grid_size(p->sm_count, 4, cells, 128), 128, 0, s, cells, p->cell_start, p->sorted_ids, xyz,
                                                                        p->sorted_xyz, p->node_rank, dmax);
    RPIM_CUDA(cudaGetLastError());
    RPIM_CUDA(cudaMemcpyAsync(&p->max_cell, dmax, sizeof(int), cudaMemcpyDeviceToHost, s));
    dfree(cursor, s);
    dfree(tmp, s);
    dfree(dmax, s);

    // supports of the integration points
    RPIM_CHECK(search_supports(p, p->n_points, p->pts, &p->soff, &p->sidx, &p->n_entries,
                               &p->max_support, &p->min_support, s, "search"));
    RPIM_CHECK(dalloc(&p->entry_pt, p->n_entries, s));
    launch("entry_points", entry_points_kernel, grid_size(p->sm_count, 8, p->n_points * 32, 256), 256, 0, s, p->n_points, p->soff, p->entry_pt);
    RPIM_CHECK(build_incidence(n, p->n_entries, p->sidx, &p->toff, &p->tent, &p->max_incident, s, p->sm_count));

    // BSR pattern
    const int words = (125 * p->max_cell + 31) / 32 + 1;
    RPIM_CHECK(dalloc(&p->rowptr, n + 1, s));
    RPIM_CHECK(dalloc(&p->diag, n, s));
    RPIM_CHECK(dalloc(&dmax, 1, s));
    RPIM_CHECK(dalloc(&tmp, scan_tmp_size(n), s));
    RPIM_CUDA(cudaMemsetAsync(dmax, 0, sizeof(int), s));
    {
        const int wpb = 8;
        size_t smem = (size_t)wpb * words * 4;
        if (smem > 48 * 1024)
            RPIM_CUDA(cudaFuncSetAttribute(pattern_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        launch("pattern_count", pattern_kernel<0>, grid_size(p->sm_count, 4, n, wpb), wpb * 32, smem, s, 
            n, p->grid, p->cell_start, p->node_cell, p->node_cpk, p->node_rank, p->sorted_ids, p->toff, p->tent,
            p->entry_pt, p->soff, p->sidx, p->rowptr, nullptr, nullptr, words, 0, dmax, p->err);
        RPIM_CUDA(cudaGetLastError());
    }
    RPIM_CHECK(exclusive_scan(p->rowptr, n, tmp, s));
    int hmax = 0;
    RPIM_CUDA(cudaMemcpyAsync(&hmax, dmax, sizeof(int), cudaMemcpyDeviceToHost, s));
    RPIM_CUDA(cudaMemcpyAsync(&p->nnzb, p->rowptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    RPIM_CUDA(cudaStreamSynchronize(s));
    dfree(tmp, s);
    dfree(dmax, s);
    RPIM_CHECK(check_device_error(p, "pattern"));
    p->max_row = hmax;
    RPIM_CHECK(dalloc(&p->cols, p->nnzb, s));
    {
        int p2 = 1;
        while (p2 < hmax) p2 <<= 1;
        int wpb = 8;
        size_t per = (size_t)words * 4 + (size_t)p2 * 4;
        while (wpb > 1 && wpb * per > 200 * 1024) wpb >>= 1;
        size_t smem = wpb * per;
        if (smem > 227 * 1024) return fail(RPIM_E_SUPPORT, "pattern row too long for shared memory");
        RPIM_CUDA(cudaFuncSetAttribute(pattern_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        launch("pattern_fill", pattern_kernel<1>, grid_size(p->sm_count, 4, n, wpb), wpb * 32, smem, s, 
            n, p->grid, p->cell_start, p->node_cell, p->node_cpk, p->node_rank, p->sorted_ids, p->toff, p->tent,
            p->entry_pt, p->soff, p->sidx, p->rowptr, p->cols, p->diag, words, p2, nullptr, p->err);
        RPIM_CUDA(cudaGetLastError());
    }
    RPIM_CHECK(check_device_error(p, "pattern"));
    return RPIM_OK;
}

extern "C" rpim_status rpim_build_pattern(int64_t n_nodes, const double *xyz, const double *cell_lo,
                                          const double *cell_hi, const rpim_params *params,
                                          rpim_stream_t stream, rpim_pattern **out,
                                          int64_t *nnz_blocks)
{
    if (!out) return fail(RPIM_E_ARG, "out is null");
    *out = nullptr;
    if (n_nodes < 4 || n_nodes > INT32_MAX / 8 || !xyz || !cell_lo || !cell_hi || !params)
        return fail(RPIM_E_ARG, "bad node count or null pointer");
    if (params->gauss_order != 2) return fail(RPIM_E_ARG, "only gauss_order = 2 is implemented");
    if (!(params->h > 0) || !(params->alpha_s > 0) || !(params->alpha_c > 0) || !(params->q > 0))
        return fail(RPIM_E_ARG, "non-positive RPIM parameter");
    rpim_pattern *p = new (std::nothrow) rpim_pattern();
    if (!p) return fail(RPIM_E_OOM, "host allocation");
    p->stream = (cudaStream_t)stream;
    p->prm = *params;
    double rs = params->alpha_s * params->h;
    p->rs2 = rs * rs;
    p->inv_h = 1.0 / params->h;
    p->n_nodes = n_nodes;
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
