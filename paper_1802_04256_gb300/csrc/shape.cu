// RPIM shape functions and gradients, one warp per point, FP64.
//
// For a point x with support nodes x_1..x_n and local coordinates
// xi_i = (x_i - x)/h, the RPIM shape functions (Sec. 1, refs. [23,24]) are the
// first n entries of the solution of the moment problem
//     [A  P] [a]   [r]
//     [P' 0] [b] = [s]
// with A_ij = R(s_ij), s_ij = |xi_i - xi_j|^2 + alpha_c^2, P_i = [1, xi_i],
// r_i = R(s_i(x)), s = p(x) = [1, 0, 0, 0] for phi and the derivatives of
// both sides for dphi/dxi_k. This kernel solves it as follows.
//
//  1. Kernel: R(s) = s^q is replaced by A(s) = s^q - alpha - beta s (the chord
//     removed). The linear constraints annihilate the removed part exactly, so
//     phi is unchanged, while A is ~1000x smaller than R and its rounding
//     perturbs the ill-conditioned problem correspondingly less. A(s) comes
//     from a piecewise binomial series evaluated by Horner's rule: the
//     high powers, whose terms are below 1e-12, in FP32, the rest in FP64.
//  2. Null space: four support nodes forming a large tetrahedron are chosen
//     greedily (pivots p). With M = P_p^{-T}, C = M P_r^T and d = M s, every
//     admissible a is a = [d - C a_r; a_r], and a_r solves the symmetric
//     positive definite system
//        S a_r = rhs,  S = A_rr - Y C - C' Y',  Y = A_rp - C' A_pp / 2,
//        rhs = v_r - C' v_p,  v = r - A_:p d.
//  3. S (packed lower triangle, shared memory) is factored S = L D L' by a
//     warp-wide right-looking elimination (no square roots); the four
//     right-hand sides are solved with lane-owned rows in registers, so the
//     triangular solves need no per-step scalar arithmetic.
// On this GPU the FP64 pipe occupies a whole warp slot whatever the lane
// mask, so warp-uniform scalar FP64 work (square roots, divisions, a 4x4
// inverse on one lane) costs as much as 32 lanes of useful work; it is kept
// to one reciprocal per elimination step.
#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace rpim {

// Reciprocal by Newton-Raphson iteration r <- r (2 - d r) from a
// single-precision seed: the relative error squares at each step
// (2^-23 -> 2^-46 -> below double rounding), so two steps give a result
// within an ulp or two of 1/d for |d| inside the single-precision range.
__device__ __forceinline__ double recip_nr(double d)
{
    double r = (double)__frcp_rn((float)d);
    double e = fma(-d, r, 1.0);
    r = fma(r, e, r);
    e = fma(-d, r, 1.0);
    return fma(r, e, r);
}

__device__ __forceinline__ int piece_of(const KernelSeries &ks, double s)
{
    const float f = (__log2f((float)s) - ks.log2_lo) * ks.inv_log2r;
    const int k = (int)f;
    return min(max(k, 0), ks.pieces - 1);
}

__device__ __forceinline__ double series_A(const KernelSeries &ks, double s)
{
    const int k = piece_of(ks, s);
    const double t = (s - ks.centre[k]) * ks.inv_w[k];
    double v = 0.0;
    if (ks.n64 <= ks.degree) {
        const float tf = (float)t;
        const float *cf = ks.coef_f[k];
        float h = cf[ks.degree];
        for (int j = ks.degree - 1; j >= ks.n64; j--) h = fmaf(h, tf, cf[j]);
        v = (double)h;
    }
    const double *c = ks.coef[k];
    for (int j = ks.n64 - 1; j >= 0; j--) v = fma(v, t, c[j]);
    return v;
}

__device__ __forceinline__ void series_A_dA(const KernelSeries &ks, double s, double &A, double &dA)
{
    A = series_A(ks, s);
    const int k = piece_of(ks, s);
    const double t = (s - ks.centre[k]) * ks.inv_w[k];
    const double *dc = ks.dcoef[k];
    double dv = dc[ks.degree - 1];
    for (int j = ks.degree - 2; j >= 0; j--) dv = fma(dv, t, dc[j]);
    dA = dv;
}

struct WarpSmem {
    double *xi;     // [3][NC]
    float *xf;      // [3][NC] single-precision copy for the pivot search
    double *C;      // [4][NC]  C[k][r]
    double *Y;      // [4][NC]  A_rp then Y
    double *v;      // [4][NC]  v[rhs][j] (original order); column buffer later
    double *invd;   // [NC]     1 / D_kk
    double *S;      // packed lower triangle, (NC-4)(NC-3)/2
    double *M;      // [16] P_p^{-T}, row-major
    double *App;    // [16]
    int *r2o;       // [NC] rest index -> original index
};

__host__ __device__ inline int64_t warp_smem_doubles(int NC)
{
    int64_t m = NC - 4;
    return 3 * NC + (3 * NC + 1) / 2 + 4 * NC + 4 * NC + 4 * NC + NC + m * (m + 1) / 2 + 32 + (NC + 1) / 2 + 2;
}

__device__ __forceinline__ WarpSmem carve(double *base, int NC)
{
    WarpSmem w;
    int64_t m = NC - 4;
    double *p = base;
    w.xi = p; p += 3 * NC;
    w.xf = (float *)p; p += (3 * NC + 1) / 2;
    w.C = p; p += 4 * NC;
    w.Y = p; p += 4 * NC;
    w.v = p; p += 4 * NC;
    w.invd = p; p += NC;
    w.S = p; p += m * (m + 1) / 2;
    w.M = p; p += 16;
    w.App = p; p += 16;
    w.r2o = (int *)p;
    return w;
}

// warp argmax of (value, index): larger value, then smaller index
__device__ __forceinline__ void warp_argmax(float &v, int &j)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float ov = __shfl_xor_sync(0xffffffffu, v, o);
        int oj = __shfl_xor_sync(0xffffffffu, j, o);
        if (ov > v || (ov == v && oj < j)) { v = ov; j = oj; }
    }
}

__device__ __forceinline__ double det3(double a, double b, double c, double d, double e, double f, double g,
                                       double h, double i)
{
    return a * fma(e, i, -f * h) - b * fma(d, i, -f * g) + c * fma(d, h, -e * g);
}

// position (i, j), i >= j, of linear index u of a packed lower triangle
__device__ __forceinline__ void tri_decode(int u, int &i, int &j)
{
    int r = (int)((sqrtf(8.0f * (float)u + 1.0f) - 1.0f) * 0.5f);
    while ((r + 1) * (r + 2) / 2 <= u) r++;
    while (r * (r + 1) / 2 > u) r--;
    i = r;
    j = u - r * (r + 1) / 2;
}

template <int R>
__global__ void __launch_bounds__(256) shape_kernel(int64_t n_pts, const double *__restrict__ pts,
                                                    const int64_t *__restrict__ soff,
                                                    const int32_t *__restrict__ sidx,
                                                    const double *__restrict__ xyz, double inv_h,
                                                    const KernelSeries *__restrict__ ks_g,
                                                    double *__restrict__ phi, int NC, DevError *err)
{
    extern __shared__ double dsm[];
    __shared__ KernelSeries ks;
    {
        const int nw = sizeof(KernelSeries) / sizeof(int);
        const int *src = (const int *)ks_g;
        int *dst = (int *)&ks;
        for (int i = threadIdx.x; i < nw; i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    WarpSmem W = carve(dsm + (size_t)wid * warp_smem_doubles(NC), NC);
    const double c2 = ks.c2;
    const int64_t stride = (int64_t)gridDim.x * nwarps;

    for (int64_t p = (int64_t)blockIdx.x * nwarps + wid; p < n_pts; p += stride) {
        const int64_t base = soff[p];
        const int n = (int)(soff[p + 1] - base);
        if (n < 4 || n > NC) {
            if (lane == 0) dev_fail(err, RPIM_E_SUPPORT, p);
            continue;
        }
        const int m = n - 4;
        const double gx = pts[3 * p], gy = pts[3 * p + 1], gz = pts[3 * p + 2];

        // 1. local coordinates (FP64) and a single-precision copy
        for (int j = lane; j < n; j += 32) {
            const int64_t J = sidx[base + j];
            const double a = (xyz[3 * J] - gx) * inv_h, b = (xyz[3 * J + 1] - gy) * inv_h,
                         c = (xyz[3 * J + 2] - gz) * inv_h;
            W.xi[j] = a;
            W.xi[NC + j] = b;
            W.xi[2 * NC + j] = c;
            W.xf[j] = (float)a;
            W.xf[NC + j] = (float)b;
            W.xf[2 * NC + j] = (float)c;
        }
        __syncwarp();

        // 2. greedy pivot tetrahedron (single precision is enough to choose)
        const float *X = W.xf, *Yc = W.xf + NC, *Z = W.xf + 2 * NC;
        int p0, p1, p2, p3;
        {
            float bv = -INFINITY;
            int bj = 0x7fffffff;
            for (int j = lane; j < n; j += 32)
                if (-X[j] > bv) { bv = -X[j]; bj = j; }
            warp_argmax(bv, bj);
            p0 = bj;
        }
        const float ax = X[p0], ay = Yc[p0], az = Z[p0];
        {
            float bv = -1.0f;
            int bj = 0x7fffffff;
            for (int j = lane; j < n; j += 32) {
                float dx = X[j] - ax, dy = Yc[j] - ay, dz = Z[j] - az;
                float d = dx * dx + dy * dy + dz * dz;
                if (d > bv) { bv = d; bj = j; }
            }
            warp_argmax(bv, bj);
            p1 = bj;
        }
        const float ux = X[p1] - ax, uy = Yc[p1] - ay, uz = Z[p1] - az;
        {
            float bv = -1.0f;
            int bj = 0x7fffffff;
            for (int j = lane; j < n; j += 32) {
                float dx = X[j] - ax, dy = Yc[j] - ay, dz = Z[j] - az;
                float cx = dy * uz - dz * uy, cy = dz * ux - dx * uz, cz = dx * uy - dy * ux;
                float d = cx * cx + cy * cy + cz * cz;
                if (d > bv) { bv = d; bj = j; }
            }
            warp_argmax(bv, bj);
            p2 = bj;
        }
        {
            const float vx = X[p2] - ax, vy = Yc[p2] - ay, vz = Z[p2] - az;
            const float nx = uy * vz - uz * vy, ny = uz * vx - ux * vz, nz = ux * vy - uy * vx;
            float bv = -1.0f;
            int bj = 0x7fffffff;
            for (int j = lane; j < n; j += 32) {
                float d = fabsf((X[j] - ax) * nx + (Yc[j] - ay) * ny + (Z[j] - az) * nz);
                if (d > bv) { bv = d; bj = j; }
            }
            warp_argmax(bv, bj);
            p3 = bj;
            const float ulen2 = ux * ux + uy * uy + uz * uz;
            if (!(bv > 1e-5f * ulen2 * sqrtf(ulen2))) {
                if (lane == 0) dev_fail(err, RPIM_E_SINGULAR, p);
                continue;
            }
        }
        // rest ordering: original order without the pivots
        for (int j = lane; j < n; j += 32) {
            int less = (p0 < j) + (p1 < j) + (p2 < j) + (p3 < j);
            bool isp = j == p0 || j == p1 || j == p2 || j == p3;
            if (!isp) W.r2o[j - less] = j;
        }
        auto pivot = [&](int k) { return k == 0 ? p0 : k == 1 ? p1 : k == 2 ? p2 : p3; };

        // 3. M = P_p^{-T} = cofactor matrix / det, one cofactor per lane 0..15
        {
            const int ri = (lane >> 2) & 3, cj = lane & 3;
            double e[3][3];
            int rr = 0;
            for (int r = 0; r < 4; r++) {
                if (r == ri) continue;
                const int pr = pivot(r);
                const double row[4] = {1.0, W.xi[pr], W.xi[NC + pr], W.xi[2 * NC + pr]};
                int cc = 0;
                for (int c = 0; c < 4; c++)
                    if (c != cj) e[rr][cc++] = row[c];
                rr++;
            }
            double cof = det3(e[0][0], e[0][1], e[0][2], e[1][0], e[1][1], e[1][2], e[2][0], e[2][1], e[2][2]);
            if ((ri + cj) & 1) cof = -cof;
            // det = sum_j P_p[0][j] cof(0, j) from lanes 0..3
            const int p0r = p0;
            const double prow = cj == 0 ? 1.0 : W.xi[(cj - 1) * NC + p0r];
            double part = lane < 4 ? prow * cof : 0.0;
            part += __shfl_xor_sync(0xffffffffu, part, 1);
            part += __shfl_xor_sync(0xffffffffu, part, 2);
            const double det = __shfl_sync(0xffffffffu, part, 0);
            const double idet = recip_nr(det);
            if (lane < 16) W.M[lane] = cof * idet;
        }
        __syncwarp();

        // 4. A_pp (lanes 0..15), C and A_rp (lanes over rest rows)
        if (lane < 16) {
            const int a = lane >> 2, b = lane & 3;
            const int ia = pivot(a), ib = pivot(b);
            double val = ks.diag;
            if (a != b) {
                double dx = W.xi[ia] - W.xi[ib], dy = W.xi[NC + ia] - W.xi[NC + ib], dz = W.xi[2 * NC + ia] - W.xi[2 * NC + ib];
                val = series_A(ks, fma(dz, dz, fma(dy, dy, fma(dx, dx, c2))));
            }
            W.App[lane] = val;
        }
        for (int r = lane; r < m; r += 32) {
            const int j = W.r2o[r];
            const double x0 = W.xi[j], x1 = W.xi[NC + j], x2 = W.xi[2 * NC + j];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                W.C[k * NC + r] = fma(W.M[4 * k + 3], x2, fma(W.M[4 * k + 2], x1, fma(W.M[4 * k + 1], x0, W.M[4 * k])));
                const int ik = pivot(k);
                double dx = x0 - W.xi[ik], dy = x1 - W.xi[NC + ik], dz = x2 - W.xi[2 * NC + ik];
                W.Y[k * NC + r] = series_A(ks, fma(dz, dz, fma(dy, dy, fma(dx, dx, c2))));
            }
        }
        __syncwarp();

        // 5. right-hand sides v = r - A_:p d  (d = columns of M), all nodes
        for (int j = lane; j < n; j += 32) {
            const double x0 = W.xi[j], x1 = W.xi[NC + j], x2 = W.xi[2 * NC + j];
            double Aj, dAj;
            series_A_dA(ks, fma(x2, x2, fma(x1, x1, fma(x0, x0, c2))), Aj, dAj);
            const double m2 = -2.0 * dAj;
            const double rr[4] = {Aj, m2 * x0, m2 * x1, m2 * x2};
            double Ajp[4];
            int kp = -1;
#pragma unroll
            for (int k = 0; k < 4; k++)
                if (pivot(k) == j) kp = k;
            if (kp >= 0) {
#pragma unroll
                for (int k = 0; k < 4; k++) Ajp[k] = W.App[4 * kp + k];
            } else {
                const int r = j - (p0 < j) - (p1 < j) - (p2 < j) - (p3 < j);
#pragma unroll
                for (int k = 0; k < 4; k++) Ajp[k] = W.Y[k * NC + r];
            }
#pragma unroll
            for (int q = 0; q < 4; q++) {
                double acc = rr[q];
#pragma unroll
                for (int k = 0; k < 4; k++) acc = fma(-Ajp[k], W.M[4 * k + q], acc);
                W.v[q * NC + j] = acc;
            }
        }
        __syncwarp();
        // Y = A_rp - C' A_pp / 2
        for (int r = lane; r < m; r += 32) {
            double y[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                double acc = 0.0;
#pragma unroll
                for (int t = 0; t < 4; t++) acc = fma(W.C[t * NC + r], W.App[4 * t + k], acc);
                y[k] = fma(-0.5, acc, W.Y[k * NC + r]);
            }
#pragma unroll
            for (int k = 0; k < 4; k++) W.Y[k * NC + r] = y[k];
        }
        __syncwarp();

        // 6. S = A_rr - Y C - C' Y' (packed lower triangle)
        {
            const int T = m * (m + 1) / 2;
            int i, j;
            tri_decode(lane, i, j);
            for (int u = lane; u < T; u += 32) {
                const int oi = W.r2o[i], oj = W.r2o[j];
                double a;
                if (i == j) {
                    a = ks.diag;
                } else {
                    double dx = W.xi[oi] - W.xi[oj], dy = W.xi[NC + oi] - W.xi[NC + oj], dz = W.xi[2 * NC + oi] - W.xi[2 * NC + oj];
                    a = series_A(ks, fma(dz, dz, fma(dy, dy, fma(dx, dx, c2))));
                }
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    a = fma(-W.Y[k * NC + i], W.C[k * NC + j], a);
                    a = fma(-W.C[k * NC + i], W.Y[k * NC + j], a);
                }
                W.S[u] = a;
                j += 32;
                while (j > i) { j -= i + 1; i++; }
            }
        }
        // reduced right-hand sides into lane-owned rows
        double b[R][4];
#pragma unroll
        for (int s = 0; s < R; s++) {
            const int r = lane + 32 * s;
#pragma unroll
            for (int q = 0; q < 4; q++) b[s][q] = 0.0;
            if (r < m) {
                const int j = W.r2o[r];
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    double acc = W.v[q * NC + j];
#pragma unroll
                    for (int k = 0; k < 4; k++) acc = fma(-W.C[k * NC + r], W.v[q * NC + pivot(k)], acc);
                    b[s][q] = acc;
                }
            }
        }
        __syncwarp();

        // 7. S = L D L' (right-looking, packed, in place; W.v holds the
        //    unscaled column of the current step)
        double *col = W.v;
        bool ok = true;
        for (int k = 0; k < m; k++) {
            const int kb = k * (k + 1) / 2;
            const double dkk = W.S[kb + k];
            if (!(dkk > 0.0)) { ok = false; break; }
            const double iv = recip_nr(dkk);
            if (lane == 0) W.invd[k] = iv;
            for (int i = k + 1 + lane; i < m; i += 32) {
                const int ik = i * (i + 1) / 2 + k;
                const double a = W.S[ik];
                col[i] = a;
                W.S[ik] = a * iv;
            }
            __syncwarp();
            const int tk = m - k - 1;
            const int T = tk * (tk + 1) / 2;
            if (T > 0) {
                int ri, rj;
                tri_decode(lane, ri, rj);
                int i = k + 1 + ri, j = k + 1 + rj;
                for (int u = lane; u < T; u += 32) {
                    const int ib = i * (i + 1) / 2;
                    W.S[ib + j] = fma(-W.S[ib + k], col[j], W.S[ib + j]);
                    j += 32;
                    while (j > i) { j -= i - k; i++; }
                }
            }
            __syncwarp();
        }
        if (!ok) {
            if (lane == 0) dev_fail(err, RPIM_E_SINGULAR, p);
            __syncwarp();
            continue;
        }

        // 8. L y = b (unit diagonal), y /= D, L' a = y (lane-owned rows)
        for (int k = 0; k < m - 1; k++) {
            const int owner = k & 31, slot = k >> 5;
            double y[4];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                double mine = 0.0;
#pragma unroll
                for (int s = 0; s < R; s++)
                    if (s == slot) mine = b[s][q];
                y[q] = __shfl_sync(0xffffffffu, mine, owner);
            }
#pragma unroll
            for (int s = 0; s < R; s++) {
                const int i = lane + 32 * s;
                if (i > k && i < m) {
                    const double l = W.S[i * (i + 1) / 2 + k];
#pragma unroll
                    for (int q = 0; q < 4; q++) b[s][q] = fma(-l, y[q], b[s][q]);
                }
            }
        }
#pragma unroll
        for (int s = 0; s < R; s++) {
            const int i = lane + 32 * s;
            if (i < m) {
                const double iv = W.invd[i];
#pragma unroll
                for (int q = 0; q < 4; q++) b[s][q] *= iv;
            }
        }
        for (int k = m - 1; k > 0; k--) {
            const int owner = k & 31, slot = k >> 5;
            double a[4];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                double mine = 0.0;
#pragma unroll
                for (int s = 0; s < R; s++)
                    if (s == slot) mine = b[s][q];
                a[q] = __shfl_sync(0xffffffffu, mine, owner);
            }
            const int kb = k * (k + 1) / 2;
#pragma unroll
            for (int s = 0; s < R; s++) {
                const int i = lane + 32 * s;
                if (i < k) {
                    const double l = W.S[kb + i];
#pragma unroll
                    for (int q = 0; q < 4; q++) b[s][q] = fma(-l, a[q], b[s][q]);
                }
            }
        }

        // 9. pivot values a_p = d - C a_r: 16 sums over the rest rows,
        //    reduce-scattered so that lane l ends with sum number l >> 1
        double v[16];
#pragma unroll
        for (int k = 0; k < 4; k++)
#pragma unroll
            for (int q = 0; q < 4; q++) {
                double acc = 0.0;
#pragma unroll
                for (int s = 0; s < R; s++) {
                    const int r = lane + 32 * s;
                    if (r < m) acc = fma(W.C[k * NC + r], b[s][q], acc);
                }
                v[4 * k + q] = acc;
            }
#pragma unroll
        for (int half = 8, bit = 16; half >= 1; half >>= 1, bit >>= 1) {
            const bool up = (lane & bit) != 0;
#pragma unroll
            for (int i = 0; i < half; i++) {
                const double mine = up ? v[i + half] : v[i];
                const double theirs = up ? v[i] : v[i + half];
                v[i] = mine + __shfl_xor_sync(0xffffffffu, theirs, bit);
            }
        }
        v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);

        double *out = phi + 4 * base;
        bool finite = true;
#pragma unroll
        for (int s = 0; s < R; s++) {
            const int r = lane + 32 * s;
            if (r < m) {
                const int j = W.r2o[r];
                double2 lo2 = make_double2(b[s][0], b[s][1] * inv_h);
                double2 hi2 = make_double2(b[s][2] * inv_h, b[s][3] * inv_h);
                finite &= isfinite(lo2.x) && isfinite(lo2.y) && isfinite(hi2.x) && isfinite(hi2.y);
                *(double2 *)(out + 4 * j) = lo2;
                *(double2 *)(out + 4 * j + 2) = hi2;
            }
        }
        if ((lane & 1) == 0) {
            const int idx = lane >> 1, k = idx >> 2, q = idx & 3;
            double val = W.M[4 * k + q] - v[0];
            if (q) val *= inv_h;
            finite &= isfinite(val);
            out[4 * pivot(k) + q] = val;
        }
        if (!__all_sync(0xffffffffu, finite) && lane == 0) dev_fail(err, RPIM_E_NONFINITE, p);
        __syncwarp();
    }
}

template <int R>
static rpim_status launch_shape(rpim_pattern *p, int64_t n_pts, const double *pts, const int64_t *soff,
                                const int32_t *sidx, int NC, double *phi, cudaStream_t s, const char *tag)
{
    const size_t per = (size_t)warp_smem_doubles(NC) * sizeof(double);
    const size_t budget = 216 * 1024;
    int wpb = (int)std::min<size_t>(8, budget / per);
    if (wpb < 1) return fail(RPIM_E_SUPPORT, "support too large for shared memory");
    const size_t smem = (size_t)wpb * per;
    RPIM_CUDA(cudaFuncSetAttribute(shape_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int bps = 0;
    RPIM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, shape_kernel<R>, wpb * 32, smem));
    if (bps < 1) bps = 1;
    int64_t blocks = std::min<int64_t>((int64_t)p->sm_count * bps, (n_pts + wpb - 1) / wpb);
    if (blocks < 1) blocks = 1;
    launch(tag, shape_kernel<R>, (unsigned)blocks, wpb * 32, smem, s, n_pts, pts, soff, sidx, p->xyz, p->inv_h,
                                                              p->series, phi, NC, p->err);
    RPIM_CUDA(cudaGetLastError());
    return RPIM_OK;
}

rpim_status shape_functions(rpim_pattern *p, int64_t n_pts, const double *pts, const int64_t *soff,
                            const int32_t *sidx, int32_t max_n, double *phi, cudaStream_t s, const char *tag)
{
    if (n_pts == 0) return RPIM_OK;
    if (max_n > RPIM_MAX_SUPPORT) return fail(RPIM_E_SUPPORT, "support larger than RPIM_MAX_SUPPORT");
    const int NC = std::max(8, (int)max_n);
    const int m = NC - 4;
    if (m <= 32) return launch_shape<1>(p, n_pts, pts, soff, sidx, NC, phi, s, tag);
    if (m <= 64) return launch_shape<2>(p, n_pts, pts, soff, sidx, NC, phi, s, tag);
    if (m <= 128) return launch_shape<4>(p, n_pts, pts, soff, sidx, NC, phi, s, tag);
    return launch_shape<7>(p, n_pts, pts, soff, sidx, NC, phi, s, tag);
}

} // namespace rpim
