// Stage 1b: assembly of K and f, surface loads and stress recovery.
//
// K_IJ = sum_g w_g B_I^T D_g B_J. For an isotropic D this 3x3 block is
//   K_ab = sum_g [ lambda_g w_g dI_a dJ_b + mu_g w_g (dI_b dJ_a + delta_ab dI . dJ) ]
// with dI = grad phi_I(x_g). Assembly is row-owner: one warp owns row I, walks
// the points whose support contains I in ascending order and accumulates the
// blocks (I, J) for J >= I of each such point in place in K. Every block is
// therefore a fixed-order sum (no atomics, bitwise reproducible). The lower
// blocks are copied, transposed, from the upper ones.
#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace rpim {

// per point: (lambda w|J|, mu w|J|) from E and nu
__global__ void lame_kernel(int64_t n_pts, const double *E, const double *nu, const double *wj,
                            double *lamw, DevError *err)
{
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n_pts;
         g += (int64_t)gridDim.x * blockDim.x) {
        const double e = E[g], v = nu[g], w = wj[g];
        if (!(e > 0.0) || !(v > -1.0) || !(v < 0.5) || !isfinite(e)) {
            dev_fail(err, RPIM_E_ARG, g);
            lamw[2 * g] = lamw[2 * g + 1] = 0.0;
            continue;
        }
        const double lam = e * v / ((1.0 + v) * (1.0 - 2.0 * v));
        const double mu = e / (2.0 * (1.0 + v));
        lamw[2 * g] = lam * w;
        lamw[2 * g + 1] = mu * w;
    }
}

__device__ __forceinline__ int lower_bound_i32(const int32_t *a, int n, int32_t key)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Row kernel. One warp owns row I and accumulates the upper blocks (J >= I)
// of its row (every block is touched by one lane at a time, in ascending
// point order). The running sums live in K (L2-resident read-modify-write)
// or, while a run of consecutive points keeps touching them, in a per-warp
// shared-memory cache of C blocks: a block enters the cache with its running
// sum from K (from zero at its first update in the row) and is written back
// when the cache fills or the row ends. Moving a sum between K and the cache
// is exact, so every block is the same fused multiply-add sequence as without
// the cache (bitwise), with fewer L2 round trips between consecutive points.
// The warps of a
// wave keep their rows' upper blocks (about 19 KB a row on the cantilever)
// in L2, so the number of resident warps is a trade: 16 per SM (2 blocks,
// 100 registers) measured 27 ms on the cantilever; 8 (shared-memory
// accumulators) 34 ms; 32 (a 64-register split into uniform and general
// kernels) 94 ms, the L2 thrashing on 92 MB of blocks in flight. Per-point scalars
// are prefetched 32 points at a time, one point per lane, and broadcast by
// shuffles. A column J's block is found from J's position in the 25 cell
// runs around I (the same positions as the pattern's bitmap, read per
// support entry from the entry's cell record): the row's upper columns are
// marked in a per-warp bitmap over these positions with the popcount before
// each word, so J's rank among them (its local index) is one word, one
// prefix and one popcount; a table maps local indices to the row's slots.
// The tables take about a tenth of the shared memory of a slot per position,
// which leaves room for a cache of up to 112 blocks per warp also where the
// cells hold many nodes (the layered slope: 54).
//
// Uniform rows (all points of the row have the same nu, hence the same
// kappa = lambda/mu = 2 nu / (1 - 2 nu)) accumulate only
//   V_ab = sum_g mu_g w_g dI_a dJ_b
// (9 fused multiply-adds per pair) and finish with
//   K = kappa V + V^T + tr(V) I.
// Other rows accumulate K_ab directly (lambda and mu terms, 24 FP64
// operations per pair).
__global__ void __launch_bounds__(256, 2) row_kernel(int64_t n_nodes, const int64_t *__restrict__ toff,
                                                     const int64_t *__restrict__ tent,
                                                     const int32_t *__restrict__ entry_pt,
                                                     const int64_t *__restrict__ soff,
                                                     const uint2 *__restrict__ ecell,
                                                     const double *__restrict__ phi,
                                                     const double *__restrict__ lamw,
                                                     const double *__restrict__ wj,
                                                     const double *__restrict__ nu,
                                                     const double *__restrict__ body,
                                                     const int64_t *__restrict__ rowptr,
                                                     const int32_t *__restrict__ cols,
                                                     const int64_t *__restrict__ diag, const InstGrid *__restrict__ ig,
                                                     const int32_t *__restrict__ node_inst,
                                                     const int32_t *__restrict__ cell_start,
                                                     const uint32_t *__restrict__ node_cpk,
                                                     const int32_t *__restrict__ node_rank, int nbits, int max_upper,
                                                     int C, const int32_t *__restrict__ order, double *K,
                                                     double *__restrict__ f, DevError *err)
{
    extern __shared__ __align__(16) unsigned char row_smem[];
    __shared__ int run_start[8][25], run_pre[8][26];
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    // per-warp shared memory: the row's upper columns as a bitmap over the
    // positions of the 25 cell runs around I, with the popcount of the words
    // before each word (a column's rank among the row's upper columns is its
    // local index) | local index -> slot in the row | local index -> cache
    // index | cache index -> local index | block cache [C][9]
    const int nw = nbits >> 5;
    const size_t bits_b = ((size_t)nw * 4 + 15) & ~(size_t)15, pre_b = ((size_t)nw * 2 + 15) & ~(size_t)15,
                 l2s_b = ((size_t)max_upper * 2 + 15) & ~(size_t)15,
                 map_b = C > 0 ? (((size_t)max_upper + 15) & ~(size_t)15) : 0,
                 cs_b = ((size_t)C * 2 + 15) & ~(size_t)15;
    unsigned char *wbase = row_smem + (size_t)wi * (bits_b + pre_b + l2s_b + map_b + cs_b + (size_t)C * 72);
    uint32_t *ubits = (uint32_t *)wbase;
    uint16_t *upre = (uint16_t *)(wbase + bits_b);
    int16_t *l2s = (int16_t *)(wbase + bits_b + pre_b);
    int8_t *lmap = (int8_t *)(wbase + bits_b + pre_b + l2s_b);
    int16_t *cslot = (int16_t *)(wbase + bits_b + pre_b + l2s_b + map_b);
    double *cache = (double *)(wbase + bits_b + pre_b + l2s_b + map_b + cs_b);
    // local index of the column at run position bi, or -1 if the row has no
    // such upper column
    auto local_of = [&](int bi, int total) -> int {
        if (bi < 0 || bi >= total) return -1;
        const uint32_t wv = ubits[bi >> 5], m = 1u << (bi & 31);
        return (wv & m) ? (int)upre[bi >> 5] + __popc(wv & (m - 1u)) : -1;
    };
    const unsigned lt = (1u << lane) - 1u;
    double b0 = 0.0, b1 = 0.0, b2 = 0.0;
    if (body) { b0 = body[0]; b1 = body[1]; b2 = body[2]; }
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t rw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; rw < n_nodes; rw += warps) {
        const int64_t I = order ? (int64_t)order[rw] : rw;
        const int64_t sd = diag[I], rend = rowptr[I + 1];
        const int64_t t0 = toff[I], t1 = toff[I + 1];
        if (sd < 0 || t0 >= t1) {   // no point reaches node I (the pattern build rejects this)
            if (lane == 0) dev_fail(err, RPIM_E_SUPPORT, I);
            continue;
        }
        const int U = (int)(rend - sd);
        const int32_t *ucols = cols + sd;
        double *Ku = K + 9 * sd;
        // without a cache every block is a running sum in K from zero; with
        // one, a block's first update starts from zero itself (map -2)
        if (C == 0)
            for (int64_t i = lane; i < 9 * (int64_t)U; i += 32) Ku[i] = 0.0;
        const uint32_t ci = node_cpk[I];
        const int cx = (int)(ci & 0x7FF), cy = (int)((ci >> 11) & 0x7FF), cz = (int)(ci >> 22);
        const int total = cell_runs(ig[node_inst[I]], cell_start, cx, cy, cz, lane, run_start[wi], run_pre[wi]);
        if (total > nbits || U > max_upper) {
            if (lane == 0) dev_fail(err, RPIM_E_ARG, I);
            continue;
        }
        const int nwr = (total + 31) >> 5;
        for (int i = lane; i < nwr; i += 32) ubits[i] = 0u;
        if (C > 0)
            for (int i = lane; i < U; i += 32) lmap[i] = -2;
        __syncwarp();
        bool bad = false;
        for (int s = lane; s < U; s += 32) {
            const int bi = run_bit(node_cpk, node_rank, ucols[s], cx, cy, cz, run_start[wi], run_pre[wi]);
            if (bi >= 0 && bi < total) atomicOr(&ubits[bi >> 5], 1u << (bi & 31));
            else bad = true;
        }
        // (a column outside the runs cannot come from the pattern build; the
        // row is skipped, so that every local index below has a slot)
        if (__any_sync(0xffffffffu, bad)) {
            if (lane == 0) dev_fail(err, RPIM_E_ARG, I);
            continue;
        }
        __syncwarp();
        {   // prefix popcounts: lane l takes words [l per, (l + 1) per)
            const int per = (nwr + 31) >> 5, w0 = min(nwr, lane * per), w1 = min(nwr, w0 + per);
            int cnt = 0;
            for (int i = w0; i < w1; i++) cnt += __popc(ubits[i]);
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            int run = incl - cnt;
            for (int i = w0; i < w1; i++) {
                upre[i] = (uint16_t)run;
                run += __popc(ubits[i]);
            }
        }
        __syncwarp();
        for (int s = lane; s < U; s += 32) {
            const int li = local_of(run_bit(node_cpk, node_rank, ucols[s], cx, cy, cz, run_start[wi], run_pre[wi]), total);
            if (li >= 0) l2s[li] = (int16_t)s;
        }
        __syncwarp();
        // uniform Poisson ratio over the row's points?
        const double nu0 = nu[entry_pt[tent[t0]]];
        bool uni = true;
        for (int64_t t = t0 + lane; t < t1; t += 32) uni &= nu[entry_pt[tent[t]]] == nu0;
        uni = __all_sync(0xffffffffu, uni);
        __syncwarp();
        int nloc = 0;   // cached blocks (warp-uniform)
        // writes the cached blocks back to K (every block keeps its running
        // sum whether it lives in the cache or in K)
        auto flush = [&]() {
            for (int li = lane; li < nloc; li += 32) {
                const int lx = cslot[li];
                const double *c = cache + 9 * li;
                double *o = Ku + 9 * (int)l2s[lx];
#pragma unroll
                for (int i = 0; i < 9; i++) o[i] = c[i];
                lmap[lx] = -1;
            }
            nloc = 0;
            __syncwarp();
        };
        // body force f_I = b sum_g w_g phi_I(g): lane l sums the points
        // tb + l of every prefetch, the lanes are combined at the end of the
        // row (a fixed order); one FP64 add per point instead of three
        // warp-wide multiply-adds per point
        double fw = 0.0;
        for (int64_t tb = t0; tb < t1; tb += 32) {
            // prefetch: lane l loads the scalars of point tb + l
            int64_t pe = 0, pend = 0;
            double pA0 = 0, pA1 = 0, pA2 = 0, pM0 = 0, pM1 = 0, pM2 = 0, pw = 0;
            if (tb + lane < t1) {
                pe = tent[tb + lane];
                const int32_t g = entry_pt[pe];
                pend = soff[g + 1];
                const double2 pa = *(const double2 *)(phi + 4 * pe);
                const double2 pb = *(const double2 *)(phi + 4 * pe + 2);
                const double lw = lamw[2 * (int64_t)g], mw = lamw[2 * (int64_t)g + 1];
                pA0 = lw * pa.y; pA1 = lw * pb.x; pA2 = lw * pb.y;
                pM0 = mw * pa.y; pM1 = mw * pb.x; pM2 = mw * pb.y;
                pw = pa.x * wj[g];
                if (body) fw += pw;
            }
            // The (point, entry) pairs of the batch's points are walked flat
            // in chunks of 32 lanes: a chunk may hold the end of one point's
            // entries and the start of the next point's, so that the lanes
            // stay busy where the supports' upper parts are short. Within a
            // chunk a block can appear twice only for two different points;
            // such a chunk is accumulated in rounds, one point at a time in
            // ascending order, so every block keeps its ascending-point
            // sequence of multiply-adds (bitwise the same K). The block
            // (local index) and gradient of the next chunk are loaded while
            // the current one is accumulated.
            int len = 0;
            if (tb + lane < t1) len = (int)(pend - pe);
            int incl = len;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            const int excl = incl - len;   // lanes past the batch hold the total
            const int tot = __shfl_sync(0xffffffffu, incl, 31);
            auto fetch = [&](int f0_, int &kl_, int &slot_, double &d0_, double &d1_, double &d2_) {
                const int f = f0_ + lane;
                int kk = 0;   // last point of the batch whose entries start at or before f
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const int ex = __shfl_sync(0xffffffffu, excl, kk + step);
                    if (ex <= f) kk += step;
                }
                kl_ = kk;
                const int64_t q = __shfl_sync(0xffffffffu, pe, kk) + (f - __shfl_sync(0xffffffffu, excl, kk));
                slot_ = -1;
                d0_ = d1_ = d2_ = 0.0;
                if (f < tot) {
                    slot_ = local_of(run_bit_cell(ecell[q], cx, cy, cz, run_start[wi], run_pre[wi]), total);
                    if (slot_ < 0) dev_fail(err, RPIM_E_ARG, I);
                    const double2 qa = *(const double2 *)(phi + 4 * q);
                    const double2 qb2 = *(const double2 *)(phi + 4 * q + 2);
                    d0_ = qa.y;
                    d1_ = qb2.x;
                    d2_ = qb2.y;
                }
            };
            int kl, slot;
            double d0, d1, d2;
            fetch(0, kl, slot, d0, d1, d2);
            for (int f0 = 0; f0 < tot; f0 += 32) {
                int nkl = 0, nslot = -1;
                double n0 = 0.0, n1 = 0.0, n2 = 0.0;
                if (f0 + 32 < tot) fetch(f0 + 32, nkl, nslot, n0, n1, n2);
                const double M0 = __shfl_sync(0xffffffffu, pM0, kl), M1 = __shfl_sync(0xffffffffu, pM1, kl),
                             M2 = __shfl_sync(0xffffffffu, pM2, kl);
                double A0 = 0.0, A1 = 0.0, A2 = 0.0;
                if (!uni) {
                    A0 = __shfl_sync(0xffffffffu, pA0, kl);
                    A1 = __shfl_sync(0xffffffffu, pA1, kl);
                    A2 = __shfl_sync(0xffffffffu, pA2, kl);
                }
                // accumulates the lane's entry into its block (slot < 0: none)
                auto accumulate = [&](const int slot) {
                    {
                        // the block's place: in the cache (li >= 0), or to be
                        // brought in; blocks stay in K when the cache is full.
                        // The map holds the cache index, -1 for a block whose
                        // running sum is in K, -2 for a block not yet updated in
                        // this row (its running sum is zero: no load)
                        int li = -1, lv = -1;
                        bool fresh = false;
                        if (C > 0) {   // (C is uniform: without a cache every block stays in K)
                            lv = slot >= 0 ? (int)lmap[slot] : -1;
                            unsigned need = __ballot_sync(0xffffffffu, slot >= 0 && lv < 0);
                            if (need && nloc + __popc(need) > C) {
                                flush();
                                lv = slot >= 0 ? (int)lmap[slot] : -1;
                                need = __ballot_sync(0xffffffffu, slot >= 0 && lv < 0);
                            }
                            li = lv >= 0 ? lv : -1;
                            if (slot >= 0 && lv < 0) {
                                const int n = nloc + __popc(need & lt);
                                if (n < C) {
                                    li = n;
                                    lmap[slot] = (int8_t)n;
                                    cslot[n] = (int16_t)slot;
                                    fresh = true;
                                }
                            }
                            nloc = min(C, nloc + __popc(need));
                        }
                        if (slot >= 0) {
                            // running sum of the block: zero at its first update,
                            // from K when it enters the cache or stays out of it,
                            // else from the cache
                            double o[9];
                            if (lv == -2) {
#pragma unroll
                                for (int i = 0; i < 9; i++) o[i] = 0.0;
                                if (li < 0) lmap[slot] = -1;   // stays in K from now on
                            } else {
                                const double *src = (li >= 0 && !fresh) ? cache + 9 * li : Ku + 9 * (int)l2s[slot];
#pragma unroll
                                for (int i = 0; i < 9; i++) o[i] = src[i];
                            }
                            if (uni) {
                                o[0] = fma(M0, d0, o[0]); o[1] = fma(M0, d1, o[1]); o[2] = fma(M0, d2, o[2]);
                                o[3] = fma(M1, d0, o[3]); o[4] = fma(M1, d1, o[4]); o[5] = fma(M1, d2, o[5]);
                                o[6] = fma(M2, d0, o[6]); o[7] = fma(M2, d1, o[7]); o[8] = fma(M2, d2, o[8]);
                            } else {
                                const double md = fma(M2, d2, fma(M1, d1, M0 * d0));
                                o[0] = fma(M0, d0, fma(A0, d0, o[0] + md));
                                o[1] = fma(M1, d0, fma(A0, d1, o[1]));
                                o[2] = fma(M2, d0, fma(A0, d2, o[2]));
                                o[3] = fma(M0, d1, fma(A1, d0, o[3]));
                                o[4] = fma(M1, d1, fma(A1, d1, o[4] + md));
                                o[5] = fma(M2, d1, fma(A1, d2, o[5]));
                                o[6] = fma(M0, d2, fma(A2, d0, o[6]));
                                o[7] = fma(M1, d2, fma(A2, d1, o[7]));
                                o[8] = fma(M2, d2, fma(A2, d2, o[8] + md));
                            }
                            double *dst = li >= 0 ? cache + 9 * li : Ku + 9 * (int)l2s[slot];
#pragma unroll
                            for (int i = 0; i < 9; i++) dst[i] = o[i];
                        }
                        __syncwarp();   // cache map and entries visible to the next round's lanes
                    }
                };
                const int kfirst = __shfl_sync(0xffffffffu, kl, 0);
                const int klast = __shfl_sync(0xffffffffu, kl, min(31, tot - 1 - f0));
                bool twice = false;
                if (kfirst != klast) {
                    const unsigned peers = __match_any_sync(0xffffffffu, slot >= 0 ? slot : -2 - lane);
                    twice = __any_sync(0xffffffffu, __popc(peers) > 1);
                }
                if (!twice) {
                    accumulate(slot);
                } else {
                    for (int kk = kfirst; kk <= klast; kk++) accumulate(kl == kk ? slot : -1);
                }
                kl = nkl;
                slot = nslot;
                d0 = n0;
                d1 = n1;
                d2 = n2;
            }
        }
        flush();
        // finish the upper blocks
        const double kappa = 2.0 * nu0 / (1.0 - 2.0 * nu0);
        for (int lx = lane; lx < U; lx += 32) {
            const int s = l2s[lx];
            double *o = Ku + 9 * s;
            double k[9];
            // (every upper block of the pattern is updated by some point of
            // the row; a block that was not would be zero)
            const bool touched = C == 0 || lmap[lx] != -2;
#pragma unroll
            for (int i = 0; i < 9; i++) k[i] = touched ? o[i] : 0.0;
            if (uni) {
                const double tr = (k[0] + k[4]) + k[8];
                double v[9];
#pragma unroll
                for (int i = 0; i < 9; i++) v[i] = k[i];
#pragma unroll
                for (int a = 0; a < 3; a++)
#pragma unroll
                    for (int bb = 0; bb < 3; bb++) k[3 * a + bb] = fma(kappa, v[3 * a + bb], v[3 * bb + a]);
                k[0] += tr; k[4] += tr; k[8] += tr;
            }
            if (s == 0) { k[3] = k[1]; k[6] = k[2]; k[7] = k[5]; } // diagonal block: exact symmetry
#pragma unroll
            for (int i = 0; i < 9; i++) o[i] = k[i];
        }
        if (body) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) fw += __shfl_xor_sync(0xffffffffu, fw, o);
        }
        if (lane == 0) {
            f[3 * I] = fw * b0;
            f[3 * I + 1] = fw * b1;
            f[3 * I + 2] = fw * b2;
        }
        __syncwarp();
    }
}

// lower blocks: K_IJ = (K_JI)^T for J < I
__global__ void mirror_kernel(int64_t n_nodes, const int64_t *rowptr, const int32_t *cols, double *K)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t I = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; I < n_nodes; I += warps) {
        const int64_t r0 = rowptr[I], r1 = rowptr[I + 1];
        for (int64_t t = r0 + lane; t < r1; t += 32) {
            const int32_t J = cols[t];
            if (J >= I) break;
            const int64_t j0 = rowptr[J];
            const int len = (int)(rowptr[J + 1] - j0);
            const int off = lower_bound_i32(cols + j0, len, (int32_t)I);
            if (off >= len || cols[j0 + off] != (int32_t)I) continue;
            const double *src = K + 9 * (j0 + off);
            double *dst = K + 9 * t;
#pragma unroll
            for (int a = 0; a < 3; a++)
#pragma unroll
                for (int b = 0; b < 3; b++) dst[3 * a + b] = src[3 * b + a];
        }
    }
}

// f_I += sum over load entries of node I (ascending) of phi * F_point
__global__ void load_gather_kernel(int64_t n_nodes, const int64_t *toff, const int64_t *tent,
                                   const int32_t *entry_pt, const double *phi, const double *force,
                                   double *f)
{
    for (int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; I < n_nodes;
         I += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t0 = toff[I], t1 = toff[I + 1];
        if (t0 == t1) continue;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
        for (int64_t t = t0; t < t1; t++) {
            const int64_t e = tent[t];
            const int64_t p = entry_pt[e];
            const double ph = phi[4 * e];
            a0 = fma(ph, force[3 * p], a0);
            a1 = fma(ph, force[3 * p + 1], a1);
            a2 = fma(ph, force[3 * p + 2], a2);
        }
        f[3 * I] += a0;
        f[3 * I + 1] += a1;
        f[3 * I + 2] += a2;
    }
}

__device__ __forceinline__ double wsum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// sigma = D(E, nu) sum_j B_j u_j, one warp per point
__global__ void stress_kernel(int64_t n_pts, const int64_t *soff, const int32_t *sidx, const double *phi,
                              const double *u, const double *E, const double *nu, double *sigma,
                              DevError *err)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < n_pts; p += warps) {
        double e[6] = {0, 0, 0, 0, 0, 0};
        for (int64_t q = soff[p] + lane; q < soff[p + 1]; q += 32) {
            const int64_t J = sidx[q];
            const double gx = phi[4 * q + 1], gy = phi[4 * q + 2], gz = phi[4 * q + 3];
            const double ux = u[3 * J], uy = u[3 * J + 1], uz = u[3 * J + 2];
            e[0] = fma(gx, ux, e[0]);
            e[1] = fma(gy, uy, e[1]);
            e[2] = fma(gz, uz, e[2]);
            e[3] = fma(gz, uy, fma(gy, uz, e[3]));
            e[4] = fma(gz, ux, fma(gx, uz, e[4]));
            e[5] = fma(gy, ux, fma(gx, uy, e[5]));
        }
#pragma unroll
        for (int k = 0; k < 6; k++) e[k] = wsum(e[k]);
        if (lane == 0) {
            const double Ev = E[p], v = nu[p];
            if (!(Ev > 0.0) || !(v > -1.0) || !(v < 0.5)) {
                dev_fail(err, RPIM_E_ARG, p);
                continue;
            }
            const double lam = Ev * v / ((1.0 + v) * (1.0 - 2.0 * v));
            const double mu = Ev / (2.0 * (1.0 + v));
            const double tr = e[0] + e[1] + e[2];
            double *o = sigma + 6 * p;
            o[0] = lam * tr + 2.0 * mu * e[0];
            o[1] = lam * tr + 2.0 * mu * e[1];
            o[2] = lam * tr + 2.0 * mu * e[2];
            o[3] = mu * e[3];
            o[4] = mu * e[4];
            o[5] = mu * e[5];
        }
    }
}

// stress kernel on given supports and shape functions (no allocation)
rpim_status launch_stress(rpim_pattern *p, int64_t n_pts, const int64_t *soff, const int32_t *sidx, const double *phi,
                          const double *u, const double *E, const double *nu, double *sigma, cudaStream_t s)
{
    launch("stress", stress_kernel, grid_size(p->sm_count, 8, n_pts * 32, 256), 256, 0, s, n_pts, soff, sidx, phi, u,
           E, nu, sigma, p->err);
    RPIM_CUDA(cudaGetLastError());
    return RPIM_OK;
}

// dL/dtheta_g = -w_g eps_g(lam)^T (dD/dtheta) eps_g(u) for theta = E, nu;
// one warp per point, strains reduced over the support in a fixed tree
__global__ void grad_material_kernel(int64_t n_pts, const int64_t *soff, const int32_t *sidx, const double *phi,
                                     const double *wj, const double *u, const double *lam, const double *E,
                                     const double *nu, double *dE, double *dnu, DevError *err)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < n_pts; p += warps) {
        double eu[6] = {0, 0, 0, 0, 0, 0}, el[6] = {0, 0, 0, 0, 0, 0};
        for (int64_t q = soff[p] + lane; q < soff[p + 1]; q += 32) {
            const int64_t J = sidx[q];
            const double gx = phi[4 * q + 1], gy = phi[4 * q + 2], gz = phi[4 * q + 3];
            const double ux = u[3 * J], uy = u[3 * J + 1], uz = u[3 * J + 2];
            const double lx = lam[3 * J], ly = lam[3 * J + 1], lz = lam[3 * J + 2];
            eu[0] = fma(gx, ux, eu[0]); el[0] = fma(gx, lx, el[0]);
            eu[1] = fma(gy, uy, eu[1]); el[1] = fma(gy, ly, el[1]);
            eu[2] = fma(gz, uz, eu[2]); el[2] = fma(gz, lz, el[2]);
            eu[3] = fma(gz, uy, fma(gy, uz, eu[3])); el[3] = fma(gz, ly, fma(gy, lz, el[3]));
            eu[4] = fma(gz, ux, fma(gx, uz, eu[4])); el[4] = fma(gz, lx, fma(gx, lz, el[4]));
            eu[5] = fma(gy, ux, fma(gx, uy, eu[5])); el[5] = fma(gy, lx, fma(gx, ly, el[5]));
        }
#pragma unroll
        for (int k = 0; k < 6; k++) {
            eu[k] = wsum(eu[k]);
            el[k] = wsum(el[k]);
        }
        if (lane == 0) {
            const double Ev = E[p], v = nu[p], w = wj[p];
            if (!(Ev > 0.0) || !(v > -1.0) || !(v < 0.5)) {
                dev_fail(err, RPIM_E_ARG, p);
                continue;
            }
            const double opv = 1.0 + v, omv = 1.0 - 2.0 * v;
            const double lamE = v / (opv * omv), muE = 1.0 / (2.0 * opv);           // lambda/E, mu/E
            const double dlam = Ev * (1.0 + 2.0 * v * v) / (opv * opv * omv * omv);  // dlambda/dnu
            const double dmu = -Ev / (2.0 * opv * opv);                              // dmu/dnu
            const double tt = (el[0] + el[1] + el[2]) * (eu[0] + eu[1] + eu[2]);
            const double qq = 2.0 * (el[0] * eu[0] + el[1] * eu[1] + el[2] * eu[2]) + el[3] * eu[3] +
                              el[4] * eu[4] + el[5] * eu[5];
            dE[p] = -w * (lamE * tt + muE * qq);
            dnu[p] = -w * (dlam * tt + dmu * qq);
        }
    }
}

static rpim_status ensure_phi(rpim_pattern *p, cudaStream_t s)
{
    if (!p->phi) RPIM_CHECK(dalloc(&p->phi, 4 * p->n_entries, s));
    if (!p->lamw) RPIM_CHECK(dalloc(&p->lamw, 2 * p->n_points, s));
    if (!p->tile_counter) RPIM_CHECK(dalloc(&p->tile_counter, 32, s));   // one work counter per bucket
    return RPIM_OK;
}

} // namespace rpim

using namespace rpim;

extern "C" rpim_status rpim_shape_functions(rpim_pattern *p, double *phi, rpim_stream_t stream)
{
    RPIM_STAGE("rpim_shape_functions");
    if (!p || !phi) return fail(RPIM_E_ARG, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    p->stream = s;
    RPIM_CHECK(shape_functions_all(p, phi, s));
    return check_device_error(p, "shape functions");
}

// The launches of one assembly (no allocation, no synchronisation).
static rpim_status assemble_issue(rpim_pattern *p, const double *E, const double *nu, const double *body, double *K,
                                  double *f, cudaStream_t s)
{
    launch("lame", lame_kernel, grid_size(p->sm_count, 4, p->n_points, 256), 256, 0, s, p->n_points, E, nu, p->wj, p->lamw, p->err);
    RPIM_CHECK(shape_functions_all(p, p->phi, s));
    // per warp: the row's column bitmap over the cell-run positions with its
    // word prefix counts, the local index -> slot table and, with a cache of
    // C blocks, its maps (int8 per upper block of the row, so C <= 127); C is
    // the largest multiple of 16 up to 112 that keeps two blocks of 8 warps
    // per SM
    const int nbits = 32 * p->bit_words;
    const int max_row = std::max(1, p->max_row);
    auto a16 = [](size_t b) { return (b + 15) & ~(size_t)15; };
    auto per_warp = [&](int c) {
        return a16((size_t)nbits / 8) + a16((size_t)nbits / 16) + a16((size_t)max_row * 2) +
               (c > 0 ? a16((size_t)max_row) : 0) + a16((size_t)c * 2) + (size_t)c * 72;
    };
    int C = 112;
    while (C > 0 && 8 * per_warp(C) > 108 * 1024) C -= 16;
    const int max_upper = max_row;
    const size_t smem = 8 * per_warp(C);
    if (max_row > 32767 || smem > 216 * 1024)
        return fail(RPIM_E_SUPPORT, "row tables too large for shared memory (too many nodes per cell)");
    RPIM_CUDA(cudaFuncSetAttribute(row_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    launch("row", row_kernel, grid_size(p->sm_count, 8, p->n_nodes * 32, 256), 256, smem, s, p->n_nodes, p->toff,
           p->tent, p->entry_pt, p->soff, (const uint2 *)p->ecell, p->phi, p->lamw, p->wj, nu, body, p->rowptr, p->cols, p->diag,
           (const InstGrid *)p->ig, (const int32_t *)p->node_inst, (const int32_t *)p->cell_start,
           (const uint32_t *)p->node_cpk, (const int32_t *)p->node_rank, nbits, max_upper, C, rows_in_order(p), K, f,
           p->err);
    RPIM_CUDA(cudaGetLastError());
    launch("mirror", mirror_kernel, grid_size(p->sm_count, 8, p->n_nodes * 32, 256), 256, 0, s, p->n_nodes, p->rowptr, p->cols, K);
    RPIM_CUDA(cudaGetLastError());
    return RPIM_OK;
}

extern "C" rpim_status rpim_assemble(rpim_pattern *p, const double *E, const double *nu, const double *body,
                                     double *K, double *f, rpim_stream_t stream)
{
    RPIM_STAGE("rpim_assemble");
    if (!p || !E || !nu || !K || !f) return fail(RPIM_E_ARG, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    p->stream = s;
    RPIM_CHECK(ensure_phi(p, s));
    RPIM_CHECK(assemble_issue(p, E, nu, body, K, f, s));
    return check_device_error(p, "assemble");
}

// rpim_assemble from a CUDA graph: the launches are captured once on the
// pattern's capture stream (capturing runs nothing) for a given set of
// argument pointers and launch plan, then replayed with one graph launch.
extern "C" rpim_status rpim_assemble_graphed(rpim_pattern *p, const double *E, const double *nu, const double *body,
                                             double *K, double *f, rpim_stream_t stream)
{
    RPIM_STAGE("rpim_assemble_graphed");
    if (!p || !E || !nu || !K || !f) return fail(RPIM_E_ARG, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    p->stream = s;
    RPIM_CHECK(ensure_phi(p, s));
    if (profiling_on()) {   // per-kernel event timing needs plain launches
        RPIM_CHECK(assemble_issue(p, E, nu, body, K, f, s));
        return check_device_error(p, "assemble (graphed)");
    }
    std::vector<unsigned char> key;
    RPIM_CHECK(shape_launch_key(p, &key));
    const void *ptrs[5] = {E, nu, body, K, f};
    key.insert(key.end(), (const unsigned char *)ptrs, (const unsigned char *)ptrs + sizeof ptrs);
    if (!p->asm_exec || key != p->asm_key) {
        if (p->asm_exec) {
            cudaGraphExecDestroy(p->asm_exec);
            p->asm_exec = nullptr;
        }
        if (!p->cap_stream) RPIM_CUDA(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
        const int64_t before = launch_count();
        RPIM_CUDA(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
        const rpim_status st = assemble_issue(p, E, nu, body, K, f, p->cap_stream);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(p->cap_stream, &g);
        p->asm_kernels = launch_count() - before;
        add_launches(-p->asm_kernels);   // counted when the graph runs
        if (st != RPIM_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess) return fail(RPIM_E_CUDA, std::string("assembly graph capture: ") + cudaGetErrorString(e));
        const cudaError_t ei = cudaGraphInstantiate(&p->asm_exec, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) {
            p->asm_exec = nullptr;
            return fail(RPIM_E_CUDA, std::string("assembly graph instantiate: ") + cudaGetErrorString(ei));
        }
        p->asm_key = key;
    }
    add_launches(p->asm_kernels);
    RPIM_CUDA(cudaGraphLaunch(p->asm_exec, s));
    return check_device_error(p, "assemble (graphed)");
}

extern "C" rpim_status rpim_grad_material(rpim_pattern *p, const double *u, const double *lam, const double *E,
                                          const double *nu, double *dE, double *dnu, rpim_stream_t stream)
{
    RPIM_STAGE("rpim_grad_material");
    if (!p || !u || !lam || !E || !nu || !dE || !dnu) return fail(RPIM_E_ARG, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    p->stream = s;
    if (!p->phi) {
        RPIM_CHECK(ensure_phi(p, s));
        RPIM_CHECK(shape_functions_all(p, p->phi, s));
    }
    launch("grad_material", grad_material_kernel, grid_size(p->sm_count, 8, p->n_points * 32, 256), 256, 0, s,
           p->n_points, (const int64_t *)p->soff, (const int32_t *)p->sidx, (const double *)p->phi,
           (const double *)p->wj, u, lam, E, nu, dE, dnu, p->err);
    RPIM_CUDA(cudaGetLastError());
    return check_device_error(p, "grad_material");
}

// every instance id of a point list must name an instance of the pattern:
// the search and shape kernels index the per-instance grids with it
__global__ void instance_ids_kernel(int64_t n, const int32_t *inst, int32_t n_inst, DevError *err)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        if ((uint32_t)inst[k] >= (uint32_t)n_inst) dev_fail(err, RPIM_E_ARG, k);
}

static rpim_status check_instance_ids(rpim_pattern *p, int64_t n, const int32_t *inst, cudaStream_t s,
                                      const char *stage)
{
    if (!inst) return RPIM_OK;
    launch("instance_ids", instance_ids_kernel, grid_size(p->sm_count, 4, n, 256), 256, 0, s, n, inst,
           (int32_t)p->n_inst, p->err);
    RPIM_CUDA(cudaGetLastError());
    return check_device_error(p, stage);
}

// The 2x2 Gauss-Legendre points of every face rectangle, with their forces
// t(x_p) w_p: face k lies in the plane x_a = lo[a] (a = axis[k]) and spans
// [lo, hi] along its tangent axes u < v; point 4k + l sits at
// mid +- half/sqrt(3) along u (bit 0 of l) and v (bit 1), weight
// half_u half_v; component c of the traction is the quadratic polynomial
// coef[18k + 6c + (0..5)] . (1, u, v, u^2, u v, v^2). A face that is not
// planar, has lo > hi along a tangent axis or names no axis is reported
// (RPIM_E_ARG, face index) and contributes nothing.
__global__ void face_points_kernel(int64_t n_faces, const double *__restrict__ lo, const double *__restrict__ hi,
                                   const int8_t *__restrict__ axis, const double *__restrict__ coef,
                                   const int32_t *__restrict__ face_inst, double *pts, double *force,
                                   int32_t *pt_inst, DevError *err)
{
    constexpr double g = 0.57735026918962576451;   // 1/sqrt(3)
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < 4 * n_faces;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = t >> 2;
        const int l = (int)(t & 3);
        const int a = axis[k];
        const double *L = lo + 3 * k, *H = hi + 3 * k;
        double *x = pts + 3 * t, *F = force + 3 * t;
        if (pt_inst) pt_inst[t] = face_inst[k];
        const int ua = a == 0 ? 1 : 0, va = a == 2 ? 1 : 2;
        if (a < 0 || a > 2 || L[a] != H[a] || !(L[ua] <= H[ua]) || !(L[va] <= H[va])) {
            if (l == 0) dev_fail(err, RPIM_E_ARG, k);
            x[0] = x[1] = x[2] = 0.0;
            F[0] = F[1] = F[2] = 0.0;
            continue;
        }
        const double mu = __dmul_rn(__dadd_rn(L[ua], H[ua]), 0.5), hu = __dmul_rn(__dsub_rn(H[ua], L[ua]), 0.5);
        const double mv = __dmul_rn(__dadd_rn(L[va], H[va]), 0.5), hv = __dmul_rn(__dsub_rn(H[va], L[va]), 0.5);
        const double u = __dadd_rn(mu, __dmul_rn(hu, (l & 1) ? g : -g));
        const double v = __dadd_rn(mv, __dmul_rn(hv, (l & 2) ? g : -g));
        x[a] = L[a];
        x[ua] = u;
        x[va] = v;
        const double w = __dmul_rn(hu, hv);
        const double m1 = u, m2 = v, m3 = u * u, m4 = u * v, m5 = v * v;
        for (int c = 0; c < 3; c++) {
            const double *q = coef + 18 * k + 6 * c;
            const double tc = fma(q[5], m5, fma(q[4], m4, fma(q[3], m3, fma(q[2], m2, fma(q[1], m1, q[0])))));
            F[c] = tc * w;
        }
    }
}

// f += x over all 3 n_nodes entries
__global__ void add_vector_kernel(int64_t n, const double *__restrict__ x, double *__restrict__ f)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        f[i] += x[i];
}

static rpim_status add_point_loads(rpim_pattern *p, int64_t n_pts, const double *xyz, const double *force,
                                   const int32_t *inst, double *f, cudaStream_t s);

static rpim_status add_traction(rpim_pattern *p, int64_t n_faces, const double *lo, const double *hi,
                                const int8_t *axis, const double *coef, const int32_t *inst, double *f,
                                cudaStream_t s)
{
    if (!p || n_faces < 0 || (n_faces > 0 && (!lo || !hi || !axis || !coef || !f)))
        return fail(RPIM_E_ARG, "bad argument");
    if (p->n_inst > 1 && !inst && n_faces > 0) return fail(RPIM_E_ARG, "a batched pattern needs the instance of every face");
    if (n_faces == 0) return RPIM_OK;
    if (n_faces > (int64_t)1 << 40) return fail(RPIM_E_ARG, "too many faces");
    p->stream = s;
    const int64_t n_pts = 4 * n_faces;
    double *pts = nullptr, *force = nullptr;
    int32_t *pinst = nullptr;
    rpim_status st = dalloc(&pts, 3 * n_pts, s);
    if (st == RPIM_OK) st = dalloc(&force, 3 * n_pts, s);
    if (st == RPIM_OK && inst) st = dalloc(&pinst, n_pts, s);
    if (st == RPIM_OK) {
        launch("face_points", face_points_kernel, grid_size(p->sm_count, 4, n_pts, 256), 256, 0, s, n_faces, lo, hi,
               axis, coef, inst, pts, force, pinst, p->err);
        st = cudaGetLastError() == cudaSuccess ? check_device_error(p, "traction: faces")
                                               : fail(RPIM_E_CUDA, "face kernel launch");
    }
    if (st == RPIM_OK) st = add_point_loads(p, n_pts, pts, force, pinst, f, s);
    dfree(pts, s); dfree(force, s); dfree(pinst, s);
    return st;
}

static rpim_status add_point_loads(rpim_pattern *p, int64_t n_pts, const double *xyz, const double *force,
                                   const int32_t *inst, double *f, cudaStream_t s)
{
    if (!p || (n_pts > 0 && (!xyz || !force || !f)) || n_pts < 0) return fail(RPIM_E_ARG, "bad argument");
    if (p->n_inst > 1 && !inst) return fail(RPIM_E_ARG, "a batched pattern needs the instance of every load point");
    if (n_pts == 0) return RPIM_OK;
    p->stream = s;
    int64_t *soff = nullptr, *toff = nullptr, *tent = nullptr, ne = 0;
    int32_t *sidx = nullptr, *ept = nullptr, mx = 0, mn = 0, mi = 0;
    double *phi = nullptr;
    RPIM_CHECK(check_instance_ids(p, n_pts, inst, s, "point loads: instance id"));
    RPIM_CHECK(search_supports(p, n_pts, xyz, inst, 0, &soff, &sidx, &ne, &mx, &mn, s, "search_loads"));
    rpim_status st = RPIM_OK;
    if ((st = dalloc(&phi, 4 * ne, s)) == RPIM_OK && (st = dalloc(&ept, ne, s)) == RPIM_OK) {
        st = shape_functions(p, n_pts, xyz, inst, 0, (const int32_t *)nullptr, soff, sidx, mx, phi, s, "shape_loads");
        if (st == RPIM_OK) {
            launch("entry_points_loads", entry_points_kernel, grid_size(p->sm_count, 8, n_pts * 32, 256), 256, 0, s, n_pts, soff, ept);
            st = build_incidence(p->n_nodes, ne, sidx, &toff, &tent, &mi, s, p->sm_count);
        }
        if (st == RPIM_OK) {
            launch("load_gather", load_gather_kernel, grid_size(p->sm_count, 4, p->n_nodes, 256), 256, 0, s, p->n_nodes, toff, tent, ept, phi, force, f);
            if (cudaGetLastError() != cudaSuccess) st = fail(RPIM_E_CUDA, "load kernel launch");
        }
    }
    if (st == RPIM_OK) st = check_device_error(p, "point loads");
    dfree(soff, s); dfree(sidx, s); dfree(phi, s); dfree(ept, s); dfree(toff, s); dfree(tent, s);
    return st;
}

extern "C" rpim_status rpim_add_point_loads(rpim_pattern *p, int64_t n_pts, const double *xyz,
                                            const double *force, double *f, rpim_stream_t stream)
{
    RPIM_STAGE("rpim_add_point_loads");
    return add_point_loads(p, n_pts, xyz, force, nullptr, f, (cudaStream_t)stream);
}

extern "C" rpim_status rpim_add_point_loads_batched(rpim_pattern *p, int64_t n_pts, const double *xyz,
                                                    const double *force, const int32_t *inst, double *f,
                                                    rpim_stream_t stream)
{
    RPIM_STAGE("rpim_add_point_loads_batched");
    if (!inst && n_pts > 0) return fail(RPIM_E_ARG, "inst is null");
    return add_point_loads(p, n_pts, xyz, force, inst, f, (cudaStream_t)stream);
}

extern "C" rpim_status rpim_add_traction(rpim_pattern *p, int64_t n_faces, const double *face_lo,
                                         const double *face_hi, const int8_t *face_axis, const double *coef,
                                         double *f, rpim_stream_t stream)
{
    RPIM_STAGE("rpim_add_traction");
    return add_traction(p, n_faces, face_lo, face_hi, face_axis, coef, nullptr, f, (cudaStream_t)stream);
}

extern "C" rpim_status rpim_add_traction_batched(rpim_pattern *p, int64_t n_faces, const double *face_lo,
                                                 const double *face_hi, const int8_t *face_axis, const double *coef,
                                                 const int32_t *inst, double *f, rpim_stream_t stream)
{
    RPIM_STAGE("rpim_add_traction_batched");
    if (!inst && n_faces > 0) return fail(RPIM_E_ARG, "inst is null");
    return add_traction(p, n_faces, face_lo, face_hi, face_axis, coef, inst, f, (cudaStream_t)stream);
}

extern "C" rpim_status rpim_add_vector(rpim_pattern *p, const double *x, double *f, rpim_stream_t stream)
{
    RPIM_STAGE("rpim_add_vector");
    if (!p || !x || !f) return fail(RPIM_E_ARG, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    p->stream = s;
    const int64_t n = 3 * p->n_nodes;
    launch("add_vector", add_vector_kernel, grid_size(p->sm_count, 4, n, 256), 256, 0, s, n, x, f);
    RPIM_CUDA(cudaGetLastError());
    return RPIM_OK;
}

static rpim_status stress(rpim_pattern *p, const double *u, int64_t n_pts, const double *xyz, const int32_t *inst,
                          const double *E, const double *nu, double *sigma, cudaStream_t s)
{
    if (!p || n_pts < 0 || (n_pts > 0 && (!u || !xyz || !E || !nu || !sigma))) return fail(RPIM_E_ARG, "bad argument");
    if (p->n_inst > 1 && !inst) return fail(RPIM_E_ARG, "a batched pattern needs the instance of every stress point");
    if (n_pts == 0) return RPIM_OK;
    p->stream = s;
    int64_t *soff = nullptr, ne = 0;
    int32_t *sidx = nullptr, mx = 0, mn = 0;
    double *phi = nullptr;
    RPIM_CHECK(check_instance_ids(p, n_pts, inst, s, "stress: instance id"));
    RPIM_CHECK(search_supports(p, n_pts, xyz, inst, 0, &soff, &sidx, &ne, &mx, &mn, s, "search_stress"));
    rpim_status st = dalloc(&phi, 4 * ne, s);
    if (st == RPIM_OK)
        st = shape_functions(p, n_pts, xyz, inst, 0, (const int32_t *)nullptr, soff, sidx, mx, phi, s, "shape_stress");
    if (st == RPIM_OK) st = launch_stress(p, n_pts, soff, sidx, phi, u, E, nu, sigma, s);
    if (st == RPIM_OK) st = check_device_error(p, "stress");
    dfree(soff, s); dfree(sidx, s); dfree(phi, s);
    return st;
}

extern "C" rpim_status rpim_stress(rpim_pattern *p, const double *u, int64_t n_pts, const double *xyz,
                                   const double *E, const double *nu, double *sigma, rpim_stream_t stream)
{
    RPIM_STAGE("rpim_stress");
    return stress(p, u, n_pts, xyz, nullptr, E, nu, sigma, (cudaStream_t)stream);
}

extern "C" rpim_status rpim_stress_batched(rpim_pattern *p, const double *u, int64_t n_pts, const double *xyz,
                                           const int32_t *inst, const double *E, const double *nu, double *sigma,
                                           rpim_stream_t stream)
{
    RPIM_STAGE("rpim_stress_batched");
    if (!inst && n_pts > 0) return fail(RPIM_E_ARG, "inst is null");
    return stress(p, u, n_pts, xyz, inst, E, nu, sigma, (cudaStream_t)stream);
}
