// Moving least-squares (MLS) and Shepard shape functions and gradients,
// FP64, one thread per point.
//
// The paper lists MLS among the shape functions it intends to add next to
// RPIM (Sec. 4). This is the textbook MLS with the linear basis
// p(y) = [1, (y - x)/h] (origin at the evaluation point x, so p(x) = e0) and
// the cubic-spline weight of sb = |x_i - x| / r_s on the RPIM support radius:
//     w(sb) = 2/3 - 4 sb^2 + 4 sb^3            (sb <= 1/2)
//     w(sb) = 4/3 - 4 sb + 4 sb^2 - 4/3 sb^3   (1/2 < sb <= 1), 0 beyond.
// With A = sum_i w_i p_i p_i^T (4x4, symmetric) and gamma = A^-1 p(x):
//     phi_i          = w_i p_i . gamma
//     dgamma/dx_k    = A^-1 (e_{k+1}/h - dA/dx_k gamma),  dA/dx_k = sum_i dw_i/dx_k p_i p_i^T
//     dphi_i/dx_k    = dw_i/dx_k p_i . gamma + w_i p_i . dgamma/dx_k
// (the shape functions do not depend on the basis origin, so the origin is
// held fixed while differentiating and then placed at x).
//
// The work is O(n) per point (about 90 FP64 operations per support node and
// a 4x4 solve), against O(n^3) for the RPIM moment problem; one thread owns a
// point and keeps A and the three dA/dx_k (40 sums) in registers. Pass 1
// writes (w_i, dw_i/dx) into the output records and accumulates the sums;
// pass 2 reads them back and overwrites them with (phi, dphi/dx).
#include <math.h>

#include "common.cuh"

namespace rpim {

// LU factorisation with partial pivoting (largest magnitude, lowest row on
// ties) of a 4x4 matrix in place; piv[k] = row swapped into position k,
// rinv[k] = 1 / U_kk. Returns false when a pivot is below 1e-13 times the
// largest entry.
__device__ __forceinline__ bool lu4(double M[4][4], int piv[4], double rinv[4])
{
    double amax = 0.0;
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) amax = fmax(amax, fabs(M[i][j]));
#pragma unroll
    for (int k = 0; k < 4; k++) {
        int pr = k;
        double best = fabs(M[k][k]);
#pragma unroll
        for (int i = k + 1; i < 4; i++)
            if (fabs(M[i][k]) > best) { best = fabs(M[i][k]); pr = i; }
        piv[k] = pr;
        if (!(best >= 1e-13 * amax)) return false;
#pragma unroll
        for (int i = k + 1; i < 4; i++)   // row exchange with compile-time indices (registers)
            if (i == pr) {
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    const double t = M[k][j];
                    M[k][j] = M[i][j];
                    M[i][j] = t;
                }
            }
        rinv[k] = 1.0 / M[k][k];
#pragma unroll
        for (int i = k + 1; i < 4; i++) {
            const double l = M[i][k] * rinv[k];
            M[i][k] = l;
#pragma unroll
            for (int j = k + 1; j < 4; j++) M[i][j] = fma(-l, M[k][j], M[i][j]);
        }
    }
    return true;
}

// solves (the factorised) M y = r in place, same row exchanges and
// multipliers as the factorisation
__device__ __forceinline__ void lu4_solve(const double M[4][4], const int piv[4], const double rinv[4], double r[4])
{
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const int pr = piv[k];
        double t = r[k];
#pragma unroll
        for (int i = 0; i < 4; i++)
            if (i == pr) { r[k] = r[i]; r[i] = t; }
#pragma unroll
        for (int i = k + 1; i < 4; i++) r[i] = fma(-M[i][k], r[k], r[i]);
    }
#pragma unroll
    for (int k = 3; k >= 0; k--) {
        double s = r[k];
#pragma unroll
        for (int i = k + 1; i < 4; i++) s = fma(-M[k][i], r[i], s);
        r[k] = s * rinv[k];
    }
}

// cubic-spline weight w(sb) and its slope w'(sb), zero beyond sb = 1
__device__ __forceinline__ void spline_weight(double sb, double &w, double &dws)
{
    if (sb <= 0.5) {
        w = fma(sb * sb, fma(4.0, sb, -4.0), 2.0 / 3.0);
        dws = sb * fma(12.0, sb, -8.0);
    } else if (sb <= 1.0) {
        w = fma(sb, fma(sb, fma(-4.0 / 3.0, sb, 4.0), -4.0), 4.0 / 3.0);
        dws = fma(sb, fma(-4.0, sb, 8.0), -4.0);
    } else {
        w = 0.0;
        dws = 0.0;
    }
}

// symmetric 4x4 from its 10 upper entries, order (00 01 02 03 11 12 13 22 23 33)
__device__ __forceinline__ void sym4(const double *a, double M[4][4])
{
    M[0][0] = a[0]; M[0][1] = M[1][0] = a[1]; M[0][2] = M[2][0] = a[2]; M[0][3] = M[3][0] = a[3];
    M[1][1] = a[4]; M[1][2] = M[2][1] = a[5]; M[1][3] = M[3][1] = a[6];
    M[2][2] = a[7]; M[2][3] = M[3][2] = a[8];
    M[3][3] = a[9];
}

__global__ void __launch_bounds__(128) mls_shape_kernel(int64_t n_pts, const double *__restrict__ pts,
                                                        const int32_t *__restrict__ inst_of, int shift,
                                                        const InstGrid *__restrict__ ig,
                                                        const int32_t *__restrict__ order,
                                                        const int64_t *__restrict__ soff,
                                                        const int32_t *__restrict__ sidx,
                                                        const double *__restrict__ xyz, double *__restrict__ phi,
                                                        DevError *err)
{
    for (int64_t pk = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; pk < n_pts;
         pk += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = order ? (int64_t)order[pk] : pk;
        const InstGrid &g = ig[instance_of(inst_of, shift, p)];
        const double inv_h = g.inv_h;
        const double inv_rs = 1.0 / sqrt(g.rs2);          // 1 / r_s
        const double inv_as = inv_rs / inv_h;              // 1 / alpha_s (r_s = alpha_s h)
        const int64_t b = soff[p], e = soff[p + 1];
        if (e - b < 4) {
            dev_fail(err, RPIM_E_SUPPORT, p);
            continue;
        }
        const double gx = pts[3 * p], gy = pts[3 * p + 1], gz = pts[3 * p + 2];
        double A[10], dA[3][10];
#pragma unroll
        for (int t = 0; t < 10; t++) A[t] = dA[0][t] = dA[1][t] = dA[2][t] = 0.0;
        // pass 1: weights, their gradients, and the moment sums
        for (int64_t q = b; q < e; q++) {
            const int64_t J = sidx[q];
            const double x0 = (xyz[3 * J] - gx) * inv_h, x1 = (xyz[3 * J + 1] - gy) * inv_h,
                         x2 = (xyz[3 * J + 2] - gz) * inv_h;
            const double d2 = fma(x2, x2, fma(x1, x1, x0 * x0));
            const double rd = d2 > 0.0 ? rsqrt(d2) : 0.0;   // 1 / |xi| (0 for a node at the point)
            const double sb = d2 * rd * inv_as;
            double w, dws;
            spline_weight(sb, w, dws);
            // dw/dx_k = w'(sb) d sb/dx_k = -w'(sb) xi_k / (alpha_s h |xi|)
            const double c = -dws * inv_as * inv_h * rd;
            const double w0 = c * x0, w1 = c * x1, w2 = c * x2;
            *(double2 *)(phi + 4 * q) = make_double2(w, w0);
            *(double2 *)(phi + 4 * q + 2) = make_double2(w1, w2);
            const double pp[10] = {1.0, x0, x1, x2, x0 * x0, x0 * x1, x0 * x2, x1 * x1, x1 * x2, x2 * x2};
#pragma unroll
            for (int t = 0; t < 10; t++) {
                A[t] = fma(w, pp[t], A[t]);
                dA[0][t] = fma(w0, pp[t], dA[0][t]);
                dA[1][t] = fma(w1, pp[t], dA[1][t]);
                dA[2][t] = fma(w2, pp[t], dA[2][t]);
            }
        }
        double M[4][4], rinv[4];
        int piv[4];
        sym4(A, M);
        if (!lu4(M, piv, rinv)) {
            dev_fail(err, RPIM_E_SINGULAR, p);
            continue;
        }
        double gam[4] = {1.0, 0.0, 0.0, 0.0};
        lu4_solve(M, piv, rinv, gam);
        double dg[3][4];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            double D[4][4];
            sym4(dA[k], D);
#pragma unroll
            for (int a = 0; a < 4; a++) {
                double s = a == k + 1 ? inv_h : 0.0;
#pragma unroll
                for (int c2 = 0; c2 < 4; c2++) s = fma(-D[a][c2], gam[c2], s);
                dg[k][a] = s;
            }
            lu4_solve(M, piv, rinv, dg[k]);
        }
        // pass 2: phi_i = w_i p_i.gamma, dphi_i/dx_k = dw_i/dx_k p_i.gamma + w_i p_i.dgamma_k
        bool finite = true;
        for (int64_t q = b; q < e; q++) {
            const int64_t J = sidx[q];
            const double x0 = (xyz[3 * J] - gx) * inv_h, x1 = (xyz[3 * J + 1] - gy) * inv_h,
                         x2 = (xyz[3 * J + 2] - gz) * inv_h;
            const double2 r0 = *(const double2 *)(phi + 4 * q);
            const double2 r1 = *(const double2 *)(phi + 4 * q + 2);
            const double w = r0.x;
            const double pg = fma(gam[3], x2, fma(gam[2], x1, fma(gam[1], x0, gam[0])));
            double o[4];
            o[0] = w * pg;
            const double dw[3] = {r0.y, r1.x, r1.y};
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const double pd = fma(dg[k][3], x2, fma(dg[k][2], x1, fma(dg[k][1], x0, dg[k][0])));
                o[1 + k] = fma(dw[k], pg, w * pd);
            }
            finite &= isfinite(o[0]) && isfinite(o[1]) && isfinite(o[2]) && isfinite(o[3]);
            *(double2 *)(phi + 4 * q) = make_double2(o[0], o[1]);
            *(double2 *)(phi + 4 * q + 2) = make_double2(o[2], o[3]);
        }
        if (!finite) dev_fail(err, RPIM_E_NONFINITE, p);
    }
}

// Shepard shape functions (the constant-basis member of the same family):
// phi_i = w_i / W, W = sum_j w_j, dphi_i/dx_k = (dw_i/dx_k - phi_i dW/dx_k) / W
// with the cubic-spline weights above. One thread per point, two passes as
// in the MLS kernel; W = 0 (no node strictly inside the radius) is singular.
__global__ void __launch_bounds__(128) shepard_shape_kernel(int64_t n_pts, const double *__restrict__ pts,
                                                            const int32_t *__restrict__ inst_of, int shift,
                                                            const InstGrid *__restrict__ ig,
                                                            const int32_t *__restrict__ order,
                                                            const int64_t *__restrict__ soff,
                                                            const int32_t *__restrict__ sidx,
                                                            const double *__restrict__ xyz,
                                                            double *__restrict__ phi, DevError *err)
{
    for (int64_t pk = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; pk < n_pts;
         pk += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = order ? (int64_t)order[pk] : pk;
        const InstGrid &g = ig[instance_of(inst_of, shift, p)];
        const double inv_h = g.inv_h;
        const double inv_as = 1.0 / (sqrt(g.rs2) * inv_h);
        const int64_t b = soff[p], e = soff[p + 1];
        if (e - b < 1) {
            dev_fail(err, RPIM_E_SUPPORT, p);
            continue;
        }
        const double gx = pts[3 * p], gy = pts[3 * p + 1], gz = pts[3 * p + 2];
        double W = 0.0, W0 = 0.0, W1 = 0.0, W2 = 0.0;
        for (int64_t q = b; q < e; q++) {
            const int64_t J = sidx[q];
            const double x0 = (xyz[3 * J] - gx) * inv_h, x1 = (xyz[3 * J + 1] - gy) * inv_h,
                         x2 = (xyz[3 * J + 2] - gz) * inv_h;
            const double d2 = fma(x2, x2, fma(x1, x1, x0 * x0));
            const double rd = d2 > 0.0 ? rsqrt(d2) : 0.0;
            const double sb = d2 * rd * inv_as;
            double w, dws;
            spline_weight(sb, w, dws);
            const double c = -dws * inv_as * inv_h * rd;
            *(double2 *)(phi + 4 * q) = make_double2(w, c * x0);
            *(double2 *)(phi + 4 * q + 2) = make_double2(c * x1, c * x2);
            W += w;
            W0 = fma(c, x0, W0);
            W1 = fma(c, x1, W1);
            W2 = fma(c, x2, W2);
        }
        if (!(W > 0.0)) {
            dev_fail(err, RPIM_E_SINGULAR, p);
            continue;
        }
        const double iW = 1.0 / W;
        bool finite = true;
        for (int64_t q = b; q < e; q++) {
            const double2 r0 = *(const double2 *)(phi + 4 * q);
            const double2 r1 = *(const double2 *)(phi + 4 * q + 2);
            const double ph = r0.x * iW;
            const double o1 = fma(-ph, W0, r0.y) * iW, o2 = fma(-ph, W1, r1.x) * iW, o3 = fma(-ph, W2, r1.y) * iW;
            finite &= isfinite(ph) && isfinite(o1) && isfinite(o2) && isfinite(o3);
            *(double2 *)(phi + 4 * q) = make_double2(ph, o1);
            *(double2 *)(phi + 4 * q + 2) = make_double2(o2, o3);
        }
        if (!finite) dev_fail(err, RPIM_E_NONFINITE, p);
    }
}

rpim_status mls_shape_functions(rpim_pattern *p, int64_t n_pts, const double *pts, const int32_t *inst_of, int shift,
                                const int32_t *order, const int64_t *soff, const int32_t *sidx, double *phi,
                                cudaStream_t s, const char *tag)
{
    if (n_pts == 0) return RPIM_OK;
    if (p->shape_kind == RPIM_SHAPE_SHEPARD) {
        launch(tag, shepard_shape_kernel, grid_size(p->sm_count, 8, n_pts, 128), 128, 0, s, n_pts, pts, inst_of,
               shift, (const InstGrid *)p->ig, order, soff, sidx, (const double *)p->xyz, phi, p->err);
        RPIM_CUDA(cudaGetLastError());
        return RPIM_OK;
    }
    launch(tag, mls_shape_kernel, grid_size(p->sm_count, 8, n_pts, 128), 128, 0, s, n_pts, pts, inst_of, shift,
           (const InstGrid *)p->ig, order, soff, sidx, (const double *)p->xyz, phi, p->err);
    RPIM_CUDA(cudaGetLastError());
    return RPIM_OK;
}

} // namespace rpim

using namespace rpim;

extern "C" rpim_status rpim_pattern_set_shape(rpim_pattern *p, int32_t kind)
{
    if (!p) return fail(RPIM_E_ARG, "null pattern");
    if (kind != RPIM_SHAPE_RPIM && kind != RPIM_SHAPE_MLS && kind != RPIM_SHAPE_SHEPARD)
        return fail(RPIM_E_ARG, "unknown shape-function kind");
    p->shape_kind = kind;
    return RPIM_OK;
}

extern "C" rpim_status rpim_pattern_get_shape(const rpim_pattern *p, int32_t *kind)
{
    if (!p || !kind) return fail(RPIM_E_ARG, "null argument");
    *kind = p->shape_kind;
    return RPIM_OK;
}
