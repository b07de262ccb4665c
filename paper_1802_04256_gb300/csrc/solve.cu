// Stage 2 (penalty) and stage 3 (Jacobi-preconditioned conjugate gradients).
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <string>
#include <vector>

#include "common.cuh"

namespace rpim {

__device__ __forceinline__ unsigned long long ord(double v)
{
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double unord(unsigned long long u)
{
    unsigned long long b = (u & 0x8000000000000000ull) ? (u & 0x7FFFFFFFFFFFFFFFull) : ~u;
    return __longlong_as_double((long long)b);
}

// ---------------------------------------------------------------------------
// penalty: alpha = scale * max_i K_ii; K_dd += alpha, f_d += alpha * value
// (one thread per constrained DOF, Sec. 2)
// ---------------------------------------------------------------------------
// per instance: largest scalar diagonal entry (order-preserving integer max,
// so the result does not depend on the order of the updates), then alpha
struct PenaltyState {
    unsigned long long kmax;
    double alpha;
};

__global__ void max_diag_kernel(int64_t n_nodes, const int64_t *diag, const int32_t *node_inst, const double *K,
                                PenaltyState *st)
{
    for (int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; I < n_nodes;
         I += (int64_t)gridDim.x * blockDim.x) {
        const double *b = K + 9 * diag[I];
        const unsigned long long m = max(ord(b[0]), max(ord(b[4]), ord(b[8])));
        atomicMax(&st[node_inst[I]].kmax, m);
    }
}

__global__ void penalty_alpha_kernel(PenaltyState *st, int n_inst, double scale)
{
    for (int i = threadIdx.x; i < n_inst; i += blockDim.x) st[i].alpha = scale * unord(st[i].kmax);
}

__global__ void penalty_fixed_alpha_kernel(PenaltyState *st, int n_inst, double alpha)
{
    for (int i = threadIdx.x; i < n_inst; i += blockDim.x) st[i].alpha = alpha;
}

__global__ void dof_count_kernel(int64_t m, const int64_t *dofs, int64_t ndof, int *mark, DevError *err)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = dofs[i];
        if (d < 0 || d >= ndof) { dev_fail(err, RPIM_E_ARG, i); continue; }
        if (atomicAdd(&mark[d], 1) != 0) dev_fail(err, RPIM_E_ARG, i);
    }
}

__global__ void penalty_apply_kernel(int64_t m, const int64_t *dofs, const double *values, int64_t ndof,
                                     const int *mark, const int64_t *diag, const int32_t *node_inst,
                                     const PenaltyState *st, double *K, double *f)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = dofs[i];
        if (d < 0 || d >= ndof || mark[d] != 1) continue;
        const int64_t I = d / 3;
        const double alpha = st[node_inst[I]].alpha;
        const int a = (int)(d % 3);
        K[9 * diag[I] + 4 * a] += alpha;
        f[d] += alpha * values[i];
    }
}

// ---------------------------------------------------------------------------
// PCG. Deterministic dot products: fixed grid, fixed in-block tree, and the
// last block to finish sums the per-block partials in index order. The
// preconditioner is the diagonal of K (Jacobi) or its 3x3 diagonal blocks
// (block Jacobi: each node's block inverted once, in pcg_init).
// ---------------------------------------------------------------------------
struct PcgState {
    double rz, pq, alpha, beta, rr, fnorm, relres, rtol;
    int iters, max_iter, done, status;
    unsigned int ticket[2];
};

constexpr int kPcgThreads = 256;

__device__ __forceinline__ double block_reduce(double v, double *sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    return t; // valid in thread 0
}

// sums partial[0..nb) in fixed order (one warp) -- called by the last block
__device__ __forceinline__ double sum_partials(const double *part, int nb)
{
    double t = 0.0;
    if (threadIdx.x < 32) {
        for (int i = threadIdx.x; i < nb; i += 32) t += ((volatile const double *)part)[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    return t;
}

__device__ __forceinline__ bool last_block(unsigned int *ticket)
{
    __shared__ bool amlast;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int t = atomicAdd(ticket, 1u);
        amlast = t == gridDim.x - 1;
        if (amlast) *ticket = 0;
    }
    __syncthreads();
    return amlast;
}

// y_I = (K x)_I for one block row by one warp; returns x_I . y_I (valid in
// lane 0). Lane l multiplies blocks l, l + 32, ... of the row. The product
// is bound by the FP64 pipe on this chip (9 DFMA per 76-byte block against a
// 2 DFMA per clock per SM rate), not by HBM: staging the blocks through
// shared memory for coalesced loads was measured to gain nothing, so the
// loads stay plain, and the three row sums are reduce-scattered (6 FP64
// additions per row instead of 15 for three butterfly reductions).
__device__ __forceinline__ double bsr_row(int64_t I, const int64_t *rowptr, const int32_t *cols, const double *K,
                                          const double *x, double *y, int lane)
{
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    const int64_t r1 = rowptr[I + 1];
    int64_t t = rowptr[I] + lane;
    // two blocks per lane and trip: both column indices, then both x
    // gathers are in flight before the first product (the same sums in the
    // same order as one block per trip)
    for (; t + 32 < r1; t += 64) {
        const int64_t J = cols[t], J2 = cols[t + 32];
        const double *b = K + 9 * t, *c = K + 9 * (t + 32);
        const double x0 = x[3 * J], x1 = x[3 * J + 1], x2 = x[3 * J + 2];
        const double y0 = x[3 * J2], y1 = x[3 * J2 + 1], y2 = x[3 * J2 + 2];
        a0 = fma(b[0], x0, fma(b[1], x1, fma(b[2], x2, a0)));
        a1 = fma(b[3], x0, fma(b[4], x1, fma(b[5], x2, a1)));
        a2 = fma(b[6], x0, fma(b[7], x1, fma(b[8], x2, a2)));
        a0 = fma(c[0], y0, fma(c[1], y1, fma(c[2], y2, a0)));
        a1 = fma(c[3], y0, fma(c[4], y1, fma(c[5], y2, a1)));
        a2 = fma(c[6], y0, fma(c[7], y1, fma(c[8], y2, a2)));
    }
    if (t < r1) {
        const double *b = K + 9 * t;
        const int64_t J = cols[t];
        const double x0 = x[3 * J], x1 = x[3 * J + 1], x2 = x[3 * J + 2];
        a0 = fma(b[0], x0, fma(b[1], x1, fma(b[2], x2, a0)));
        a1 = fma(b[3], x0, fma(b[4], x1, fma(b[5], x2, a1)));
        a2 = fma(b[6], x0, fma(b[7], x1, fma(b[8], x2, a2)));
    }
    // lanes 0-15 keep components (0, 1), lanes 16-31 keep (2, -)
    const bool hi16 = (lane & 16) != 0;
    double s0 = hi16 ? a2 : a0, s1 = hi16 ? 0.0 : a1;
    s0 += __shfl_xor_sync(0xffffffffu, hi16 ? a0 : a2, 16);
    s1 += __shfl_xor_sync(0xffffffffu, hi16 ? a1 : 0.0, 16);
    // lanes with bit 3 clear keep the first of the two, the others the second
    const bool hi8 = (lane & 8) != 0;
    double v = hi8 ? s1 : s0;
    v += __shfl_xor_sync(0xffffffffu, hi8 ? s0 : s1, 8);
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    // lanes 0, 8, 16 now hold components 0, 1, 2 of the row (lanes 24-31: 0)
    const int c = lane >> 3;
    double d = 0.0;
    if ((lane & 7) == 0 && c < 3) {
        y[3 * I + c] = v;
        d = v * x[3 * I + c];
    }
    d += __shfl_xor_sync(0xffffffffu, d, 8);
    d += __shfl_xor_sync(0xffffffffu, d, 16);
    return d;
}

// Inverse of a symmetric positive definite 3x3 block (row-major) from its
// L D L^T factors, inv = L^-T D^-1 L^-1 (9 entries written); false when a
// pivot is not positive (the block is not SPD).
__device__ __forceinline__ bool spd3_inverse(const double *b, double *inv)
{
    const double d0 = b[0];
    if (!(d0 > 0.0)) return false;
    const double l10 = b[3] / d0, l20 = b[6] / d0;
    const double d1 = fma(-l10, b[3], b[4]);
    if (!(d1 > 0.0)) return false;
    const double l21 = fma(-l20, b[3], b[7]) / d1;
    const double d2 = fma(-l21 * l21, d1, fma(-l20, b[6], b[8]));
    if (!(d2 > 0.0)) return false;
    const double e0 = 1.0 / d0, e1 = 1.0 / d1, e2 = 1.0 / d2;
    const double m10 = -l10, m21 = -l21, m20 = fma(l10, l21, -l20);   // L^-1 below the unit diagonal
    const double i00 = fma(m20 * m20, e2, fma(m10 * m10, e1, e0)), i01 = fma(m20 * m21, e2, m10 * e1);
    const double i02 = m20 * e2, i11 = fma(m21 * m21, e2, e1), i12 = m21 * e2, i22 = e2;
    inv[0] = i00; inv[1] = i01; inv[2] = i02;
    inv[3] = i01; inv[4] = i11; inv[5] = i12;
    inv[6] = i02; inv[7] = i12; inv[8] = i22;
    return true;
}

// z_I = B_I r_I with the stored 3x3 inverse B_I of node I's diagonal block
__device__ __forceinline__ void apply3(const double *B, double r0, double r1, double r2, double &z0, double &z1,
                                       double &z2)
{
    z0 = fma(B[0], r0, fma(B[1], r1, B[2] * r2));
    z1 = fma(B[3], r0, fma(B[4], r1, B[5] * r2));
    z2 = fma(B[6], r0, fma(B[7], r1, B[8] * r2));
}

// Preconditioner of node I (lane 0 of the warp that just formed r_I = (K x)_I
// in r): r <- f - r, z = M^-1 r, p = z; accumulates r.z, r.r, f.f. M is the
// diagonal of K (Jacobi: dinv[3n]) or its 3x3 diagonal blocks (block Jacobi:
// dinv[9n] holds each block's inverse).
template <bool BLOCK>
__device__ __forceinline__ void init_node(int64_t I, int lane, const double *K, const int64_t *diag,
                                          const double *f, double *r, double *z, double *p, double *dinv,
                                          double &rz, double &rr, double &ff, DevError *err)
{
    if (!BLOCK) {
        if (lane < 3) {
            const int64_t d = 3 * I + lane;
            const double kd = K[9 * diag[I] + 4 * lane];
            if (!(kd > 0.0)) dev_fail(err, RPIM_E_ARG, d);
            const double di = 1.0 / kd;
            const double rv = f[d] - r[d];
            const double zv = di * rv;
            dinv[d] = di;
            r[d] = rv;
            z[d] = zv;
            p[d] = zv;
            rz += rv * zv;
            rr += rv * rv;
            ff += f[d] * f[d];
        }
    } else if (lane == 0) {
        double *B = dinv + 9 * I;
        if (!spd3_inverse(K + 9 * diag[I], B)) {
            dev_fail(err, RPIM_E_ARG, 3 * I);
            for (int k = 0; k < 9; k++) B[k] = 0.0;
        }
        const double r0 = f[3 * I] - r[3 * I], r1 = f[3 * I + 1] - r[3 * I + 1], r2 = f[3 * I + 2] - r[3 * I + 2];
        double z0, z1, z2;
        apply3(B, r0, r1, r2, z0, z1, z2);
        r[3 * I] = r0; r[3 * I + 1] = r1; r[3 * I + 2] = r2;
        z[3 * I] = z0; z[3 * I + 1] = z1; z[3 * I + 2] = z2;
        p[3 * I] = z0; p[3 * I + 1] = z1; p[3 * I + 2] = z2;
        rz += (r0 * z0 + r1 * z1) + r2 * z2;
        rr += (r0 * r0 + r1 * r1) + r2 * r2;
        ff += (f[3 * I] * f[3 * I] + f[3 * I + 1] * f[3 * I + 1]) + f[3 * I + 2] * f[3 * I + 2];
    }
}

// x += alpha p, r -= alpha q, z = M^-1 r for node or DOF i (Jacobi: DOF i;
// block Jacobi: node i); accumulates r.z, r.r
template <bool BLOCK>
__device__ __forceinline__ void update_unit(int64_t i, double alpha, double *x, double *r, double *z,
                                            const double *p, const double *q, const double *dinv, double &rz,
                                            double &rr)
{
    if (!BLOCK) {
        x[i] = fma(alpha, p[i], x[i]);
        const double rv = fma(-alpha, q[i], r[i]);
        const double zv = dinv[i] * rv;
        r[i] = rv;
        z[i] = zv;
        rz = fma(rv, zv, rz);
        rr = fma(rv, rv, rr);
    } else {
        const int64_t d = 3 * i;
        x[d] = fma(alpha, p[d], x[d]);
        x[d + 1] = fma(alpha, p[d + 1], x[d + 1]);
        x[d + 2] = fma(alpha, p[d + 2], x[d + 2]);
        const double r0 = fma(-alpha, q[d], r[d]), r1 = fma(-alpha, q[d + 1], r[d + 1]),
                     r2 = fma(-alpha, q[d + 2], r[d + 2]);
        double z0, z1, z2;
        apply3(dinv + 9 * i, r0, r1, r2, z0, z1, z2);
        r[d] = r0; r[d + 1] = r1; r[d + 2] = r2;
        z[d] = z0; z[d + 1] = z1; z[d + 2] = z2;
        rz = fma(r2, z2, fma(r1, z1, fma(r0, z0, rz)));
        rr = fma(r2, r2, fma(r1, r1, fma(r0, r0, rr)));
    }
}

// r = f - K x, z = M^-1 r, p = z; partials of r.z, r.r, f.f
template <bool BLOCK>
__global__ void __launch_bounds__(kPcgThreads) pcg_init_kernel(int64_t n_nodes, const int64_t *rowptr,
                                                               const int32_t *cols, const double *K,
                                                               const int64_t *diag, const double *f,
                                                               const double *x, double *r, double *z,
                                                               double *p, double *dinv, double *part,
                                                               PcgState *st, DevError *err)
{
    __shared__ double sh[32];
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    double rz = 0.0, rr = 0.0, ff = 0.0;
    for (int64_t I = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; I < n_nodes; I += warps) {
        bsr_row(I, rowptr, cols, K, x, r, lane);
        __syncwarp();
        init_node<BLOCK>(I, lane, K, diag, f, r, z, p, dinv, rz, rr, ff, err);
    }
    double b_rz = block_reduce(rz, sh), b_rr = block_reduce(rr, sh), b_ff = block_reduce(ff, sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = b_rz;
        part[gridDim.x + blockIdx.x] = b_rr;
        part[2 * gridDim.x + blockIdx.x] = b_ff;
    }
    if (last_block(&st->ticket[0])) {
        double trz = sum_partials(part, gridDim.x);
        double trr = sum_partials(part + gridDim.x, gridDim.x);
        double tff = sum_partials(part + 2 * gridDim.x, gridDim.x);
        if (threadIdx.x == 0) {
            st->rz = trz;
            st->rr = trr;
            st->fnorm = tff > 0.0 ? sqrt(tff) : 1.0;
            st->relres = sqrt(trr) / st->fnorm;
            st->iters = 0;
            st->done = (st->relres <= st->rtol || st->max_iter == 0) ? 1 : 0;
            if (!isfinite(st->relres)) { st->done = 1; st->status = RPIM_E_NONFINITE; }
        }
    }
}

// q = K p, partial p.q; last block: alpha = rz / pq
__global__ void __launch_bounds__(kPcgThreads) pcg_spmv_kernel(int64_t n_nodes, const int64_t *rowptr,
                                                               const int32_t *cols, const double *K,
                                                               const double *p, double *q, double *part,
                                                               PcgState *st)
{
    if (st->done) return;
    __shared__ double sh[32];
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    double pq = 0.0;
    for (int64_t I = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; I < n_nodes; I += warps) {
        double v = bsr_row(I, rowptr, cols, K, p, q, lane);
        if (lane == 0) pq += v;
    }
    double b = block_reduce(pq, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = b;
    if (last_block(&st->ticket[0])) {
        double t = sum_partials(part, gridDim.x);
        if (threadIdx.x == 0) {
            st->pq = t;
            st->alpha = st->rz / t;
            if (!isfinite(st->alpha)) { st->done = 1; st->status = RPIM_E_NONFINITE; }
        }
    }
}

// x += alpha p, r -= alpha q, z = M^-1 r over n units (DOFs for Jacobi,
// nodes for block Jacobi); partials r.z, r.r; last block: beta = rz_new /
// rz, convergence test
template <bool BLOCK>
__global__ void __launch_bounds__(kPcgThreads) pcg_update_kernel(int64_t n, double *x, double *r, double *z,
                                                                 const double *p, const double *q,
                                                                 const double *dinv, double *part,
                                                                 PcgState *st)
{
    if (st->done) return;
    __shared__ double sh[32];
    const double alpha = st->alpha;
    double rz = 0.0, rr = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        update_unit<BLOCK>(i, alpha, x, r, z, p, q, dinv, rz, rr);
    double b_rz = block_reduce(rz, sh), b_rr = block_reduce(rr, sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = b_rz;
        part[gridDim.x + blockIdx.x] = b_rr;
    }
    if (last_block(&st->ticket[1])) {
        double trz = sum_partials(part, gridDim.x);
        double trr = sum_partials(part + gridDim.x, gridDim.x);
        if (threadIdx.x == 0) {
            st->beta = trz / st->rz;
            st->rz = trz;
            st->rr = trr;
            st->relres = sqrt(trr) / st->fnorm;
            st->iters += 1;
            if (st->relres <= st->rtol || st->iters >= st->max_iter) st->done = 1;
            if (!isfinite(st->relres)) { st->done = 1; st->status = RPIM_E_NONFINITE; }
        }
    }
}

__global__ void pcg_direction_kernel(int64_t n, const double *z, double *p, const PcgState *st)
{
    if (st->done) return;
    const double beta = st->beta;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = fma(beta, p[i], z[i]);
}


// ---------------------------------------------------------------------------
// Batched PCG: independent Jacobi-PCG iterations of the instances of a
// batched pattern (K is block diagonal by instance), with every instance's
// own alpha, beta and convergence test on its own ||f_i||. Rows are split
// into segments that never cross an instance; a block reduces each of its
// segments to one partial, and the last block to finish sums every live
// instance's partials in segment order, so the scalars are deterministic.
// Converged instances drop out of the sweeps.
// ---------------------------------------------------------------------------
struct PcgInst {
    double rz, pq, alpha, beta, rr, fnorm, relres, pad;
    int iters, done, status, pad2;
};

struct PcgBatch {
    double rtol;
    int max_iter, active;
    unsigned int ticket[2];
};

constexpr int kSegRows = 64;

// sum of part[b..e) by one warp in a fixed order (valid in every lane)
__device__ __forceinline__ double warp_sum_range(const double *part, int64_t b, int64_t e, int lane)
{
    double t = 0.0;
    for (int64_t i = b + lane; i < e; i += 32) t += ((volatile const double *)part)[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    return t;
}

// instances still iterating, counted by the last block into bst->active
__device__ __forceinline__ void count_active(const PcgInst *inst, int n_inst, PcgBatch *bst)
{
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    int c = 0;
    for (int i = threadIdx.x; i < n_inst; i += blockDim.x) c += ((volatile const PcgInst *)inst)[i].done ? 0 : 1;
    if (c) atomicAdd(&cnt, c);
    __syncthreads();
    if (threadIdx.x == 0) bst->active = cnt;
}

template <bool BLOCK>
__global__ void __launch_bounds__(kPcgThreads) pcgb_init_kernel(int64_t n_seg, const int64_t *seg_row,
                                                                const int32_t *inst_seg, int n_inst,
                                                                const int64_t *rowptr, const int32_t *cols,
                                                                const double *K, const int64_t *diag,
                                                                const double *f, const double *x, double *r,
                                                                double *z, double *p, double *dinv, double *part,
                                                                PcgInst *inst, PcgBatch *bst, DevError *err)
{
    __shared__ double sh[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t s = blockIdx.x; s < n_seg; s += gridDim.x) {
        double rz = 0.0, rr = 0.0, ff = 0.0;
        for (int64_t I = seg_row[s] + warp; I < seg_row[s + 1]; I += nw) {
            bsr_row(I, rowptr, cols, K, x, r, lane);
            __syncwarp();
            init_node<BLOCK>(I, lane, K, diag, f, r, z, p, dinv, rz, rr, ff, err);
        }
        const double b_rz = block_reduce(rz, sh), b_rr = block_reduce(rr, sh), b_ff = block_reduce(ff, sh);
        if (threadIdx.x == 0) {
            part[s] = b_rz;
            part[n_seg + s] = b_rr;
            part[2 * n_seg + s] = b_ff;
        }
    }
    if (last_block(&bst->ticket[0])) {
        for (int i = warp; i < n_inst; i += nw) {
            const double trz = warp_sum_range(part, inst_seg[i], inst_seg[i + 1], lane);
            const double trr = warp_sum_range(part + n_seg, inst_seg[i], inst_seg[i + 1], lane);
            const double tff = warp_sum_range(part + 2 * n_seg, inst_seg[i], inst_seg[i + 1], lane);
            if (lane == 0) {
                PcgInst &st = inst[i];
                st.rz = trz;
                st.rr = trr;
                st.fnorm = tff > 0.0 ? sqrt(tff) : 1.0;
                st.relres = sqrt(trr) / st.fnorm;
                st.iters = 0;
                st.status = 0;
                st.done = (st.relres <= bst->rtol || bst->max_iter == 0) ? 1 : 0;
                if (!isfinite(st.relres)) { st.done = 1; st.status = RPIM_E_NONFINITE; }
            }
        }
        __threadfence_block();
        count_active(inst, n_inst, bst);
    }
}

// q = K p on the live instances; last block: alpha_i = rz_i / (p.q)_i
__global__ void __launch_bounds__(kPcgThreads) pcgb_spmv_kernel(int64_t n_seg, const int64_t *seg_row,
                                                                const int32_t *seg_inst, const int32_t *inst_seg,
                                                                int n_inst, const int64_t *rowptr,
                                                                const int32_t *cols, const double *K,
                                                                const double *p, double *q, double *part,
                                                                PcgInst *inst, PcgBatch *bst)
{
    if (bst->active == 0) return;
    __shared__ double sh[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t s = blockIdx.x; s < n_seg; s += gridDim.x) {
        if (inst[seg_inst[s]].done) continue;
        double pq = 0.0;
        for (int64_t I = seg_row[s] + warp; I < seg_row[s + 1]; I += nw) {
            const double v = bsr_row(I, rowptr, cols, K, p, q, lane);
            if (lane == 0) pq += v;
        }
        const double bpq = block_reduce(pq, sh);
        if (threadIdx.x == 0) part[s] = bpq;
    }
    if (last_block(&bst->ticket[0])) {
        for (int i = warp; i < n_inst; i += nw) {
            if (inst[i].done) continue;
            const double t = warp_sum_range(part, inst_seg[i], inst_seg[i + 1], lane);
            if (lane == 0) {
                PcgInst &st = inst[i];
                st.pq = t;
                st.alpha = st.rz / t;
                if (!isfinite(st.alpha)) { st.done = 1; st.status = RPIM_E_NONFINITE; }
            }
        }
    }
}

// x += alpha_i p, r -= alpha_i q, z = Dinv r on the live instances; last
// block: beta_i, residuals, convergence, count of live instances
template <bool BLOCK>
__global__ void __launch_bounds__(kPcgThreads) pcgb_update_kernel(int64_t n_seg, const int64_t *seg_row,
                                                                  const int32_t *seg_inst, const int32_t *inst_seg,
                                                                  int n_inst, double *x, double *r, double *z,
                                                                  const double *p, const double *q,
                                                                  const double *dinv, double *part, PcgInst *inst,
                                                                  PcgBatch *bst)
{
    if (bst->active == 0) return;
    __shared__ double sh[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t s = blockIdx.x; s < n_seg; s += gridDim.x) {
        const PcgInst &st = inst[seg_inst[s]];
        if (st.done) continue;
        const double alpha = st.alpha;
        double rz = 0.0, rr = 0.0;
        const int64_t u0 = BLOCK ? seg_row[s] : 3 * seg_row[s], u1 = BLOCK ? seg_row[s + 1] : 3 * seg_row[s + 1];
        for (int64_t i = u0 + threadIdx.x; i < u1; i += blockDim.x)
            update_unit<BLOCK>(i, alpha, x, r, z, p, q, dinv, rz, rr);
        const double b_rz = block_reduce(rz, sh), b_rr = block_reduce(rr, sh);
        if (threadIdx.x == 0) {
            part[s] = b_rz;
            part[n_seg + s] = b_rr;
        }
    }
    if (last_block(&bst->ticket[1])) {
        for (int i = warp; i < n_inst; i += nw) {
            if (inst[i].done) continue;
            const double trz = warp_sum_range(part, inst_seg[i], inst_seg[i + 1], lane);
            const double trr = warp_sum_range(part + n_seg, inst_seg[i], inst_seg[i + 1], lane);
            if (lane == 0) {
                PcgInst &st = inst[i];
                st.beta = trz / st.rz;
                st.rz = trz;
                st.rr = trr;
                st.relres = sqrt(trr) / st.fnorm;
                st.iters += 1;
                if (st.relres <= bst->rtol || st.iters >= bst->max_iter) st.done = 1;
                if (!isfinite(st.relres)) { st.done = 1; st.status = RPIM_E_NONFINITE; }
            }
        }
        __threadfence_block();
        count_active(inst, n_inst, bst);
    }
}

// p = z + beta_i p on the live instances (an instance that converged in the
// update above is skipped: its p is no longer used)
__global__ void __launch_bounds__(kPcgThreads) pcgb_direction_kernel(int64_t n_seg, const int64_t *seg_row,
                                                                     const int32_t *seg_inst, const double *z,
                                                                     double *p, const PcgInst *inst,
                                                                     const PcgBatch *bst)
{
    if (bst->active == 0) return;
    for (int64_t s = blockIdx.x; s < n_seg; s += gridDim.x) {
        const PcgInst &st = inst[seg_inst[s]];
        if (st.done) continue;
        const double beta = st.beta;
        for (int64_t i = 3 * seg_row[s] + threadIdx.x; i < 3 * seg_row[s + 1]; i += blockDim.x)
            p[i] = fma(beta, p[i], z[i]);
    }
}


// The launches of one chunk of PCG iterations as a CUDA graph: captured once
// per solve on the pattern's capture stream (capturing runs nothing), then
// replayed on the caller's stream, which removes the per-launch host cost
// from the many short iterations of small systems. With per-kernel timing
// on, the launches are issued directly so that every kernel keeps its events.
class ChunkGraph {
public:
    ChunkGraph() = default;
    ChunkGraph(const ChunkGraph &) = delete;
    ChunkGraph &operator=(const ChunkGraph &) = delete;
    ~ChunkGraph()
    {
        if (exec_) cudaGraphExecDestroy(exec_);
    }
    template <class F>
    rpim_status run(rpim_pattern *p, cudaStream_t s, F issue)
    {
        if (profiling_on()) {
            issue(s);
            RPIM_CUDA(cudaGetLastError());
            return RPIM_OK;
        }
        if (!exec_) {
            if (!p->cap_stream) RPIM_CUDA(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
            const int64_t before = launch_count();
            RPIM_CUDA(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
            issue(p->cap_stream);
            cudaGraph_t g = nullptr;
            const cudaError_t e = cudaStreamEndCapture(p->cap_stream, &g);
            kernels_ = launch_count() - before;
            add_launches(-kernels_);   // counted when the graph runs
            if (e != cudaSuccess) return fail(RPIM_E_CUDA, std::string("pcg graph capture: ") + cudaGetErrorString(e));
            const cudaError_t ei = cudaGraphInstantiate(&exec_, g, 0);
            cudaGraphDestroy(g);
            if (ei != cudaSuccess) {
                exec_ = nullptr;
                return fail(RPIM_E_CUDA, std::string("pcg graph instantiate: ") + cudaGetErrorString(ei));
            }
        }
        add_launches(kernels_);
        RPIM_CUDA(cudaGraphLaunch(exec_, s));
        return RPIM_OK;
    }

private:
    cudaGraphExec_t exec_ = nullptr;
    int64_t kernels_ = 0;
};

} // namespace rpim

using namespace rpim;

// alpha_in < 0: alpha = scale * max diag per instance; otherwise alpha_in
static rpim_status apply_penalty(rpim_pattern *p, double *K, double *f, int64_t m, const int64_t *dofs,
                                 const double *values, double scale, double alpha_in, double *alpha_out,
                                 cudaStream_t s)
{
    if (!p || !K || !f || m < 0 || (m > 0 && (!dofs || !values))) return fail(RPIM_E_ARG, "bad argument");
    p->stream = s;
    const int64_t ndof = 3 * p->n_nodes;
    const int ni = p->n_inst;
    PenaltyState *st = nullptr;
    int *mark = nullptr;
    RPIM_CHECK(dalloc(&st, ni, s));
    RPIM_CHECK(dalloc(&mark, ndof, s));
    RPIM_CUDA(cudaMemsetAsync(st, 0, ni * sizeof(PenaltyState), s));
    RPIM_CUDA(cudaMemsetAsync(mark, 0, ndof * sizeof(int), s));
    if (alpha_in < 0) {
        launch("max_diag", max_diag_kernel, grid_size(p->sm_count, 4, p->n_nodes, 256), 256, 0, s, p->n_nodes,
               (const int64_t *)p->diag, (const int32_t *)p->node_inst, (const double *)K, st);
        launch("penalty_alpha", penalty_alpha_kernel, 1, 256, 0, s, st, ni, scale);
    } else {
        launch("penalty_alpha", penalty_fixed_alpha_kernel, 1, 256, 0, s, st, ni, alpha_in);
    }
    if (m > 0) {
        launch("dof_count", dof_count_kernel, grid_size(p->sm_count, 4, m, 256), 256, 0, s, m, dofs, ndof, mark, p->err);
        launch("penalty_apply", penalty_apply_kernel, grid_size(p->sm_count, 4, m, 256), 256, 0, s, m, dofs, values,
               ndof, (const int *)mark, (const int64_t *)p->diag, (const int32_t *)p->node_inst,
               (const PenaltyState *)st, K, f);
    }
    RPIM_CUDA(cudaGetLastError());
    std::vector<PenaltyState> hs(ni);
    RPIM_CUDA(cudaMemcpyAsync(hs.data(), st, ni * sizeof(PenaltyState), cudaMemcpyDeviceToHost, s));
    dfree(st, s);
    dfree(mark, s);
    rpim_status r = check_device_error(p, "penalty");
    if (alpha_out)
        for (int i = 0; i < ni; i++) alpha_out[i] = hs[i].alpha;
    return r;
}

extern "C" rpim_status rpim_apply_penalty_bc(rpim_pattern *p, double *K, double *f, int64_t m, const int64_t *dofs,
                                             const double *values, double scale, double *alpha_out,
                                             rpim_stream_t stream)
{
    RPIM_STAGE("rpim_apply_penalty_bc");
    if (!p) return fail(RPIM_E_ARG, "null pattern");
    std::vector<double> a(p->n_inst);
    rpim_status st = apply_penalty(p, K, f, m, dofs, values, scale, -1.0, a.data(), (cudaStream_t)stream);
    if (alpha_out) *alpha_out = a[0];
    return st;
}

extern "C" rpim_status rpim_apply_penalty_bc_batched(rpim_pattern *p, double *K, double *f, int64_t m,
                                                     const int64_t *dofs, const double *values, double scale,
                                                     double *alpha_out, rpim_stream_t stream)
{
    RPIM_STAGE("rpim_apply_penalty_bc_batched");
    return apply_penalty(p, K, f, m, dofs, values, scale, -1.0, alpha_out, (cudaStream_t)stream);
}

extern "C" rpim_status rpim_apply_penalty_alpha(rpim_pattern *p, double *K, double *f, int64_t m, const int64_t *dofs,
                                                const double *values, double alpha, rpim_stream_t stream)
{
    RPIM_STAGE("rpim_apply_penalty_alpha");
    if (!(alpha >= 0.0)) return fail(RPIM_E_ARG, "negative penalty");
    return apply_penalty(p, K, f, m, dofs, values, 0.0, alpha, nullptr, (cudaStream_t)stream);
}

extern "C" rpim_status rpim_pattern_set_precond(rpim_pattern *p, int32_t kind)
{
    if (!p || (kind != RPIM_PRECOND_JACOBI && kind != RPIM_PRECOND_BLOCK_JACOBI))
        return fail(RPIM_E_ARG, "unknown preconditioner");
    p->precond = kind;
    return RPIM_OK;
}

extern "C" rpim_status rpim_pattern_get_precond(const rpim_pattern *p, int32_t *kind)
{
    if (!p || !kind) return fail(RPIM_E_ARG, "null argument");
    *kind = p->precond;
    return RPIM_OK;
}

extern "C" rpim_status rpim_solve_pcg(rpim_pattern *p, const double *K, const double *f, double *u, double rtol,
                                      int32_t max_iter, int32_t *iters, double *relres, rpim_stream_t stream)
{
    RPIM_STAGE("rpim_solve_pcg");
    if (!p || !K || !f || !u || max_iter < 0 || !(rtol >= 0)) return fail(RPIM_E_ARG, "bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    p->stream = s;
    const int64_t n = 3 * p->n_nodes;
    const int nb = std::max(1, p->sm_count * 6);   // six 256-thread blocks per SM fit the product's 40 registers
    const bool block = p->precond == RPIM_PRECOND_BLOCK_JACOBI;
    const int64_t nd = block ? 3 * n : n;   // preconditioner: 3x3 inverses or diagonal inverses
    const int64_t need = 4 * n + nd + 3 * (int64_t)nb;
    if (p->ws.doubles < need) {
        dfree(p->ws.buf, s);
        RPIM_CHECK(dalloc(&p->ws.buf, need, s));
        p->ws.doubles = need;
    }
    double *r = p->ws.buf, *z = r + n, *pp = z + n, *q = pp + n, *dinv = q + n, *part = dinv + nd;
    PcgState hs{};
    hs.rtol = rtol;
    hs.max_iter = max_iter;
    PcgState *st = (PcgState *)p->scal;
    static_assert(sizeof(PcgState) <= 16 * sizeof(double), "state fits the scalar block");
    RPIM_CUDA(cudaMemcpyAsync(st, &hs, sizeof hs, cudaMemcpyHostToDevice, s));
    const int tpb = kPcgThreads;
    launch("pcg_init", block ? pcg_init_kernel<true> : pcg_init_kernel<false>, nb, tpb, 0, s, p->n_nodes, p->rowptr,
           p->cols, K, p->diag, f, u, r, z, pp, dinv, part, st, p->err);
    RPIM_CUDA(cudaGetLastError());
    const int64_t nu = block ? p->n_nodes : n;   // units of the update kernel
    const int chunk = 32;
    int it = 0;
    ChunkGraph graph;
    auto issue = [&](cudaStream_t cs) {
        for (int k = 0; k < chunk; k++) {
            launch("pcg_spmv", pcg_spmv_kernel, nb, tpb, 0, cs, p->n_nodes, p->rowptr, p->cols, K, pp, q, part, st);
            launch("pcg_update", block ? pcg_update_kernel<true> : pcg_update_kernel<false>, nb, tpb, 0, cs, nu, u,
                   r, z, pp, q, dinv, part, st);
            launch("pcg_direction", pcg_direction_kernel, nb, tpb, 0, cs, n, z, pp, st);
        }
    };
    for (;;) {
        RPIM_CHECK(graph.run(p, s, issue));
        RPIM_CUDA(cudaMemcpyAsync(&hs, st, sizeof hs, cudaMemcpyDeviceToHost, s));
        RPIM_CUDA(cudaStreamSynchronize(s));
        it += chunk;
        if (hs.done || it > max_iter + chunk) break;
    }
    if (iters) *iters = hs.iters;
    if (relres) *relres = hs.relres;
    RPIM_CHECK(check_device_error(p, "pcg"));
    if (hs.status) return fail((rpim_status)hs.status, "pcg: non-finite value");
    if (!(hs.relres <= rtol)) {
        char buf[128];
        snprintf(buf, sizeof buf, "pcg: relative residual %.3e after %d iterations", hs.relres, hs.iters);
        return fail(RPIM_E_NOCONV, buf);
    }
    return RPIM_OK;
}

// segments that never cross an instance: 64 rows (8 per warp), or up to
// 512 when the rows are plentiful enough to give every block of the grid
// several segments (fewer block-wide reductions and barrier waits)
static rpim_status build_segments(rpim_pattern *p, cudaStream_t s)
{
    if (p->seg_row) return RPIM_OK;
    const int64_t nb = (int64_t)p->sm_count * 4;
    int64_t rows = kSegRows;
    while (rows < 512 && p->n_nodes >= 8 * nb * (2 * rows)) rows *= 2;
    std::vector<int64_t> row;
    std::vector<int32_t> sinst, iseg;
    for (int i = 0; i < p->n_inst; i++) {
        iseg.push_back((int32_t)sinst.size());
        const rpim::InstGrid &g = p->ig_host[i];
        for (int64_t r = g.node_begin; r < g.node_end; r += rows) {
            row.push_back(r);
            sinst.push_back(i);
        }
    }
    iseg.push_back((int32_t)sinst.size());
    row.push_back(p->n_nodes);
    const int64_t ns = (int64_t)sinst.size();
    RPIM_CHECK(dalloc(&p->seg_row, ns + 1, s));
    RPIM_CHECK(dalloc(&p->seg_inst, ns, s));
    RPIM_CHECK(dalloc(&p->inst_seg, p->n_inst + 1, s));
    RPIM_CUDA(cudaMemcpyAsync(p->seg_row, row.data(), (ns + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    if (ns) RPIM_CUDA(cudaMemcpyAsync(p->seg_inst, sinst.data(), ns * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    RPIM_CUDA(cudaMemcpyAsync(p->inst_seg, iseg.data(), iseg.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    RPIM_CUDA(cudaStreamSynchronize(s));   // host vectors go out of scope
    p->n_seg = ns;
    return RPIM_OK;
}

extern "C" rpim_status rpim_solve_pcg_batched(rpim_pattern *p, const double *K, const double *f, double *u,
                                              double rtol, int32_t max_iter, int32_t *iters, double *relres,
                                              rpim_stream_t stream)
{
    RPIM_STAGE("rpim_solve_pcg_batched");
    if (!p || !K || !f || !u || max_iter < 0 || !(rtol >= 0)) return fail(RPIM_E_ARG, "bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    p->stream = s;
    RPIM_CHECK(build_segments(p, s));
    const int64_t n = 3 * p->n_nodes, ns = p->n_seg;
    const int ni = p->n_inst;
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(ns, (int64_t)p->sm_count * 4));
    const int64_t inst_doubles = (ni * (int64_t)sizeof(PcgInst) + sizeof(PcgBatch) + 7) / 8;
    const bool block = p->precond == RPIM_PRECOND_BLOCK_JACOBI;
    const int64_t nd = block ? 3 * n : n;
    const int64_t need = 4 * n + nd + 3 * ns + inst_doubles;
    if (p->ws.doubles < need) {
        dfree(p->ws.buf, s);
        RPIM_CHECK(dalloc(&p->ws.buf, need, s));
        p->ws.doubles = need;
    }
    double *r = p->ws.buf, *z = r + n, *pp = z + n, *q = pp + n, *dinv = q + n, *part = dinv + nd;
    PcgBatch *bst = (PcgBatch *)(part + 3 * ns);
    PcgInst *inst = (PcgInst *)(bst + 1);
    static_assert(sizeof(PcgBatch) % 8 == 0 && sizeof(PcgInst) % 8 == 0, "8-byte state records");
    PcgBatch hb{};
    hb.rtol = rtol;
    hb.max_iter = max_iter;
    hb.active = ni;
    RPIM_CUDA(cudaMemcpyAsync(bst, &hb, sizeof hb, cudaMemcpyHostToDevice, s));
    const int tpb = kPcgThreads;
    launch("pcgb_init", block ? pcgb_init_kernel<true> : pcgb_init_kernel<false>, nb, tpb, 0, s, ns,
           (const int64_t *)p->seg_row,
           (const int32_t *)p->inst_seg, ni, (const int64_t *)p->rowptr, (const int32_t *)p->cols, K,
           (const int64_t *)p->diag, f, (const double *)u, r, z, pp, dinv, part, inst, bst, p->err);
    RPIM_CUDA(cudaGetLastError());
    const int chunk = 32;
    int it = 0;
    ChunkGraph graph;
    auto issue = [&](cudaStream_t cs) {
        for (int k = 0; k < chunk; k++) {
            launch("pcgb_spmv", pcgb_spmv_kernel, nb, tpb, 0, cs, ns, (const int64_t *)p->seg_row,
                   (const int32_t *)p->seg_inst, (const int32_t *)p->inst_seg, ni, (const int64_t *)p->rowptr,
                   (const int32_t *)p->cols, K, (const double *)pp, q, part, inst, bst);
            launch("pcgb_update", block ? pcgb_update_kernel<true> : pcgb_update_kernel<false>, nb, tpb, 0, cs, ns,
                   (const int64_t *)p->seg_row,
                   (const int32_t *)p->seg_inst, (const int32_t *)p->inst_seg, ni, u, r, z, (const double *)pp,
                   (const double *)q, (const double *)dinv, part, inst, bst);
            launch("pcgb_direction", pcgb_direction_kernel, nb, tpb, 0, cs, ns, (const int64_t *)p->seg_row,
                   (const int32_t *)p->seg_inst, (const double *)z, pp, (const PcgInst *)inst,
                   (const PcgBatch *)bst);
        }
    };
    for (;;) {
        RPIM_CHECK(graph.run(p, s, issue));
        RPIM_CUDA(cudaMemcpyAsync(&hb, bst, sizeof hb, cudaMemcpyDeviceToHost, s));
        RPIM_CUDA(cudaStreamSynchronize(s));
        it += chunk;
        if (hb.active == 0 || it > max_iter + chunk) break;
    }
    std::vector<PcgInst> hi(ni);
    RPIM_CUDA(cudaMemcpyAsync(hi.data(), inst, ni * sizeof(PcgInst), cudaMemcpyDeviceToHost, s));
    RPIM_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < ni; i++) {
        if (iters) iters[i] = hi[i].iters;
        if (relres) relres[i] = hi[i].relres;
    }
    RPIM_CHECK(check_device_error(p, "pcg batched"));
    for (int i = 0; i < ni; i++) {
        char buf[160];
        if (hi[i].status) {
            snprintf(buf, sizeof buf, "pcg batched: non-finite value in instance %d", i);
            return fail((rpim_status)hi[i].status, buf);
        }
        if (!(hi[i].relres <= rtol)) {
            snprintf(buf, sizeof buf, "pcg batched: instance %d at relative residual %.3e after %d iterations", i,
                     hi[i].relres, hi[i].iters);
            return fail(RPIM_E_NOCONV, buf);
        }
    }
    return RPIM_OK;
}
