// Stage 2 (penalty) and stage 3 (Jacobi-preconditioned conjugate gradients).
#include <math.h>
#include <stdio.h>

#include <algorithm>

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
struct PenaltyState {
    unsigned long long kmax;
    double alpha;
};

__global__ void max_diag_kernel(int64_t n_nodes, const int64_t *diag, const double *K, PenaltyState *st)
{
    unsigned long long m = 0;
    for (int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; I < n_nodes;
         I += (int64_t)gridDim.x * blockDim.x) {
        const double *b = K + 9 * diag[I];
        m = max(m, max(ord(b[0]), max(ord(b[4]), ord(b[8]))));
    }
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&st->kmax, m);
}

__global__ void penalty_alpha_kernel(PenaltyState *st, double scale)
{
    st->alpha = scale * unord(st->kmax);
}

__global__ void penalty_fixed_alpha_kernel(PenaltyState *st, double alpha) { st->alpha = alpha; }

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
                                     const int *mark, const int64_t *diag, const PenaltyState *st,
                                     double *K, double *f)
{
    const double alpha = st->alpha;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = dofs[i];
        if (d < 0 || d >= ndof || mark[d] != 1) continue;
        const int64_t I = d / 3;
        const int a = (int)(d % 3);
        K[9 * diag[I] + 4 * a] += alpha;
        f[d] += alpha * values[i];
    }
}

// ---------------------------------------------------------------------------
// PCG. Deterministic dot products: fixed grid, fixed in-block tree, and the
// last block to finish sums the per-block partials in index order.
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

// y = K x for the rows of this warp; returns x_I . y_I contribution (lane 0)
__device__ __forceinline__ double bsr_row(int64_t I, const int64_t *rowptr, const int32_t *cols, const double *K,
                                          const double *x, double *y, int lane)
{
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    const int64_t r1 = rowptr[I + 1];
    for (int64_t t = rowptr[I] + lane; t < r1; t += 32) {
        const double *b = K + 9 * t;
        const int64_t J = cols[t];
        const double x0 = x[3 * J], x1 = x[3 * J + 1], x2 = x[3 * J + 2];
        a0 = fma(b[0], x0, fma(b[1], x1, fma(b[2], x2, a0)));
        a1 = fma(b[3], x0, fma(b[4], x1, fma(b[5], x2, a1)));
        a2 = fma(b[6], x0, fma(b[7], x1, fma(b[8], x2, a2)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a0 += __shfl_xor_sync(0xffffffffu, a0, o);
        a1 += __shfl_xor_sync(0xffffffffu, a1, o);
        a2 += __shfl_xor_sync(0xffffffffu, a2, o);
    }
    if (lane == 0) {
        y[3 * I] = a0;
        y[3 * I + 1] = a1;
        y[3 * I + 2] = a2;
    }
    return a0 * x[3 * I] + a1 * x[3 * I + 1] + a2 * x[3 * I + 2];
}

// r = f - K x, z = Dinv r, p = z; partials of r.z, r.r, f.f
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

// x += alpha p, r -= alpha q, z = Dinv r; partials r.z, r.r; last block:
// beta = rz_new / rz, convergence test
__global__ void __launch_bounds__(kPcgThreads) pcg_update_kernel(int64_t n, double *x, double *r, double *z,
                                                                 const double *p, const double *q,
                                                                 const double *dinv, double *part,
                                                                 PcgState *st)
{
    if (st->done) return;
    __shared__ double sh[32];
    const double alpha = st->alpha;
    double rz = 0.0, rr = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        x[i] = fma(alpha, p[i], x[i]);
        const double rv = fma(-alpha, q[i], r[i]);
        const double zv = dinv[i] * rv;
        r[i] = rv;
        z[i] = zv;
        rz = fma(rv, zv, rz);
        rr = fma(rv, rv, rr);
    }
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

} // namespace rpim

using namespace rpim;

extern "C" rpim_status rpim_apply_penalty_bc(rpim_pattern *p, double *K, double *f, int64_t m, const int64_t *dofs,
                                             const double *values, double scale, double *alpha_out,
                                             rpim_stream_t stream)
{
    if (!p || !K || !f || m < 0 || (m > 0 && (!dofs || !values))) return fail(RPIM_E_ARG, "bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    p->stream = s;
    const int64_t ndof = 3 * p->n_nodes;
    PenaltyState *st = nullptr;
    int *mark = nullptr;
    RPIM_CHECK(dalloc(&st, 1, s));
    RPIM_CHECK(dalloc(&mark, ndof, s));
    RPIM_CUDA(cudaMemsetAsync(st, 0, sizeof(PenaltyState), s));
    RPIM_CUDA(cudaMemsetAsync(mark, 0, ndof * sizeof(int), s));
    launch("max_diag", max_diag_kernel, grid_size(p->sm_count, 4, p->n_nodes, 256), 256, 0, s, p->n_nodes, p->diag, K, st);
    launch("penalty_alpha", penalty_alpha_kernel, 1, 1, 0, s, st, scale);
    if (m > 0) {
        launch("dof_count", dof_count_kernel, grid_size(p->sm_count, 4, m, 256), 256, 0, s, m, dofs, ndof, mark, p->err);
        launch("penalty_apply", penalty_apply_kernel, grid_size(p->sm_count, 4, m, 256), 256, 0, s, m, dofs, values, ndof, mark,
                                                                                 p->diag, st, K, f);
    }
    RPIM_CUDA(cudaGetLastError());
    double alpha = 0.0;
    RPIM_CUDA(cudaMemcpyAsync(&alpha, &st->alpha, sizeof(double), cudaMemcpyDeviceToHost, s));
    dfree(st, s);
    dfree(mark, s);
    rpim_status r = check_device_error(p, "penalty");
    if (alpha_out) *alpha_out = alpha;
    return r;
}

extern "C" rpim_status rpim_apply_penalty_alpha(rpim_pattern *p, double *K, double *f, int64_t m, const int64_t *dofs,
                                                const double *values, double alpha, rpim_stream_t stream)
{
    if (!p || !K || !f || m < 0 || (m > 0 && (!dofs || !values)) || !(alpha >= 0.0))
        return fail(RPIM_E_ARG, "bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    p->stream = s;
    const int64_t ndof = 3 * p->n_nodes;
    PenaltyState *st = nullptr;
    int *mark = nullptr;
    RPIM_CHECK(dalloc(&st, 1, s));
    RPIM_CHECK(dalloc(&mark, ndof, s));
    RPIM_CUDA(cudaMemsetAsync(mark, 0, ndof * sizeof(int), s));
    launch("penalty_alpha", penalty_fixed_alpha_kernel, 1, 1, 0, s, st, alpha);
    if (m > 0) {
        launch("dof_count", dof_count_kernel, grid_size(p->sm_count, 4, m, 256), 256, 0, s, m, dofs, ndof, mark, p->err);
        launch("penalty_apply", penalty_apply_kernel, grid_size(p->sm_count, 4, m, 256), 256, 0, s, m, dofs, values, ndof,
               (const int *)mark, (const int64_t *)p->diag, (const PenaltyState *)st, K, f);
    }
    RPIM_CUDA(cudaGetLastError());
    dfree(st, s);
    dfree(mark, s);
    return check_device_error(p, "penalty");
}

extern "C" rpim_status rpim_solve_pcg(rpim_pattern *p, const double *K, const double *f, double *u, double rtol,
                                      int32_t max_iter, int32_t *iters, double *relres, rpim_stream_t stream)
{
    if (!p || !K || !f || !u || max_iter < 0 || !(rtol >= 0)) return fail(RPIM_E_ARG, "bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    p->stream = s;
    const int64_t n = 3 * p->n_nodes;
    const int nb = std::max(1, p->sm_count * 4);
    const int64_t need = 5 * n + 3 * (int64_t)nb;
    if (p->ws.doubles < need) {
        dfree(p->ws.buf, s);
        RPIM_CHECK(dalloc(&p->ws.buf, need, s));
        p->ws.doubles = need;
    }
    double *r = p->ws.buf, *z = r + n, *pp = z + n, *q = pp + n, *dinv = q + n, *part = dinv + n;
    PcgState hs{};
    hs.rtol = rtol;
    hs.max_iter = max_iter;
    PcgState *st = (PcgState *)p->scal;
    static_assert(sizeof(PcgState) <= 16 * sizeof(double), "state fits the scalar block");
    RPIM_CUDA(cudaMemcpyAsync(st, &hs, sizeof hs, cudaMemcpyHostToDevice, s));
    const int tpb = kPcgThreads;
    launch("pcg_init", pcg_init_kernel, nb, tpb, 0, s, p->n_nodes, p->rowptr, p->cols, K, p->diag, f, u, r, z, pp, dinv, part, st, p->err);
    RPIM_CUDA(cudaGetLastError());
    const int chunk = 32;
    int it = 0;
    for (;;) {
        for (int k = 0; k < chunk; k++) {
            launch("pcg_spmv", pcg_spmv_kernel, nb, tpb, 0, s, p->n_nodes, p->rowptr, p->cols, K, pp, q, part, st);
            launch("pcg_update", pcg_update_kernel, nb, tpb, 0, s, n, u, r, z, pp, q, dinv, part, st);
            launch("pcg_direction", pcg_direction_kernel, nb, tpb, 0, s, n, z, pp, st);
        }
        RPIM_CUDA(cudaGetLastError());
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
