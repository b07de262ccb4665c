/*
 * RPIM oracle: a plain, slow, obviously correct CPU implementation of the
 * global stiffness assembly of the radial point interpolation method (RPIM)
 * and the stages around it, written to check the GPU path.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, load or
 * call this file; the tests, the package's smoke check and the benchmark's
 * CPU-baseline leg are its only users. It shares no code with the CUDA path.
 *
 * What it computes (the paper describes the pipeline in Sec. 2 and names the
 * method -- Liu's RPIM, refs. [23,24] -- in Sec. 1; it prints no formulas, so
 * the textbook definition is written out here):
 *
 *  - Integration: every field node owns a box cell; each cell is integrated
 *    with the 2x2x2 Gauss-Legendre rule (points mid +- half/sqrt(3), weight
 *    |J| = product of the half extents). Sec. 2 ("element stiffness matrix of
 *    each field node").
 *  - Support of a point x: every node i with |x_i - x|^2 <= r_s^2,
 *    r_s = alpha_s * h, found by brute force over all nodes, ascending id.
 *  - Shape functions (RPIM with linear polynomial augmentation, m = 4): with
 *    local coordinates xi = (x_i - x)/h, the multiquadric
 *    R(r) = (r^2 + alpha_c^2)^q, moment matrix
 *        G = [[R_Q, P], [P^T, 0]],  R_Q[i][j] = R(|xi_i - xi_j|),
 *        P[i] = [1, xi_i],
 *    solve G z = [R(x); p(x)] and its derivatives; phi = the first n entries.
 *    Own Gaussian elimination with partial pivoting.
 *  - Shape functions, MLS variant (the paper names moving least squares only
 *    as future work, Sec. 4; selected with orc_set_shape(1)): textbook MLS
 *    with the linear basis p = [1, xi] and the cubic-spline weight
 *    w(r / r_s) on the same support radius. A(x) = sum_i w_i p_i p_i^T,
 *    gamma = A^-1 p(x), phi_i = w_i p_i^T gamma, and for the derivatives
 *    dgamma/dx_k = A^-1 (dp/dx_k - dA/dx_k gamma),
 *    dphi_i/dx_k = dw_i/dx_k p_i^T gamma + w_i p_i^T dgamma/dx_k.
 *    Own Gaussian elimination with partial pivoting on the 4x4 system.
 *  - Shape functions, Shepard variant (also named as future work, Sec. 4;
 *    orc_set_shape(2)): inverse-distance weighting with the same cubic-spline
 *    weight, phi_i = w_i / sum_j w_j, i.e. moving least squares with the
 *    constant basis p = [1]; reproduces constants only.
 *  - Point stiffness: K_IJ += w |J| B_I^T D B_J with the 6x3 strain matrix B_I
 *    (Voigt xx, yy, zz, yz, xz, xy; engineering shear strains) and isotropic
 *    D(E, nu). Every block (I, J) is formed on its own (no mirroring), and
 *    blocks are summed in ascending point order.
 *  - Body force f_I += phi_I b w|J|; surface loads f_I += phi_I F at given
 *    points, or tractions integrated over face rectangles (2x2 Gauss-Legendre
 *    per face).
 *  - Penalty (Sec. 2, second stage): alpha = scale * max_i K_ii,
 *    K_dd += alpha, f_d += alpha * u_d for each constrained DOF d.
 *  - Solve (Sec. 2, third stage): Jacobi-preconditioned conjugate gradients.
 *  - Stress: sigma = D sum_I B_I u_I at given points.
 *
 * Precision: every floating-point step after the integration points runs in
 * the type `real`, which is double by default and long double when built
 * with -DORC_LONG (extended precision, used to measure the FP64 floor).
 * The integration points and the support test use double arithmetic without
 * fused multiply-add, so that support sets are a well-defined integer result.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifdef ORC_LONG
typedef long double real;
#define RPOW powl
#define RSQRT sqrtl
#define RABS fabsl
#else
typedef double real;
#define RPOW pow
#define RSQRT sqrt
#define RABS fabs
#endif

/* status codes shared in meaning with the library's public header */
enum { ORC_OK = 0, ORC_E_ARG = 1, ORC_E_OOM = 3, ORC_E_SUPPORT = 4, ORC_E_SINGULAR = 5,
       ORC_E_NOCONV = 6 };

static int g_threads = 1;
static int g_shape = 0;   /* 0: RPIM, 1: MLS, 2: Shepard */

int orc_real_bytes(void) { return (int)sizeof(real); }
void orc_set_threads(int t) { g_threads = t > 0 ? t : 1; }
void orc_set_shape(int kind) { g_shape = (kind == 1 || kind == 2) ? kind : 0; }
int orc_get_shape(void) { return g_shape; }

/* ---------------------------------------------------------------------------
 * Integration points: 2x2x2 Gauss-Legendre rule on every node cell.
 * Point 8*i + l, l = a + 2b + 4c, sits at mid + half * (+-1/sqrt(3)) with the
 * sign of each axis given by bit a, b, c (0 -> minus). Weight = hx*hy*hz.
 * ------------------------------------------------------------------------- */
#define GAUSS2 0.57735026918962576451

void orc_gauss_points(int64_t n_cells, const double *lo, const double *hi,
                      double *pts, double *wj)
{
    for (int64_t i = 0; i < n_cells; i++) {
        double mid[3], half[3];
        for (int k = 0; k < 3; k++) {
            mid[k] = (lo[3 * i + k] + hi[3 * i + k]) * 0.5;
            half[k] = (hi[3 * i + k] - lo[3 * i + k]) * 0.5;
        }
        for (int l = 0; l < 8; l++) {
            for (int k = 0; k < 3; k++) {
                double s = ((l >> k) & 1) ? GAUSS2 : -GAUSS2;
                double off = half[k] * s;
                pts[3 * (8 * i + l) + k] = mid[k] + off;
            }
            wj[8 * i + l] = (half[0] * half[1]) * half[2];
        }
    }
}

/* ---------------------------------------------------------------------------
 * Support of a point by brute force: nodes with squared distance <= rs2,
 * in ascending node id. The squared distance is ((dx*dx + dy*dy) + dz*dz),
 * evaluated in double with no contraction. Returns the count (may exceed cap;
 * only the first cap ids are written).
 * ------------------------------------------------------------------------- */
int64_t orc_support(int64_t n_nodes, const double *xyz, const double *x, double rs2,
                    int32_t *out, int64_t cap)
{
    int64_t cnt = 0;
    for (int64_t i = 0; i < n_nodes; i++) {
        double dx = xyz[3 * i] - x[0];
        double dy = xyz[3 * i + 1] - x[1];
        double dz = xyz[3 * i + 2] - x[2];
        double dxx = dx * dx, dyy = dy * dy, dzz = dz * dz;
        double d2 = (dxx + dyy) + dzz;
        if (d2 <= rs2) {
            if (cnt < cap) out[cnt] = (int32_t)i;
            cnt++;
        }
    }
    return cnt;
}

double orc_support_radius2(double alpha_s, double h)
{
    double rs = alpha_s * h;
    return rs * rs;
}

/* ---------------------------------------------------------------------------
 * RPIM shape functions at x from the n support nodes `supp`.
 * Output phi[4*n]: phi[j], dphi/dx[j], dphi/dy[j], dphi/dz[j] at offsets
 * 0, n, 2n, 3n.  Returns ORC_E_SINGULAR when a pivot falls below
 * 1e-13 * max|G|.
 * ------------------------------------------------------------------------- */
static int shape_rpim_real(const double *xyz, const int32_t *supp, int n, const double *x,
                           double h, double alpha_c, double q, real *phi_out /* 4*n */)
{
    const int N = n + 4;
    real *G = (real *)calloc((size_t)N * N, sizeof(real));
    real *Z = (real *)calloc((size_t)N * 4, sizeof(real));
    real *xi = (real *)malloc((size_t)n * 3 * sizeof(real));
    if (!G || !Z || !xi) { free(G); free(Z); free(xi); return ORC_E_OOM; }
    const real hr = (real)h, c2 = (real)alpha_c * (real)alpha_c, qr = (real)q;

    for (int j = 0; j < n; j++)
        for (int k = 0; k < 3; k++)
            xi[3 * j + k] = ((real)xyz[3 * (int64_t)supp[j] + k] - (real)x[k]) / hr;

    /* moment matrix G = [[R_Q, P], [P^T, 0]] */
    for (int i = 0; i < n; i++) {
        for (int j = 0; j < n; j++) {
            real r2 = 0;
            for (int k = 0; k < 3; k++) {
                real d = xi[3 * i + k] - xi[3 * j + k];
                r2 += d * d;
            }
            G[(size_t)i * N + j] = RPOW(r2 + c2, qr);
        }
        G[(size_t)i * N + n] = 1;
        G[(size_t)n * N + i] = 1;
        for (int k = 0; k < 3; k++) {
            G[(size_t)i * N + n + 1 + k] = xi[3 * i + k];
            G[(size_t)(n + 1 + k) * N + i] = xi[3 * i + k];
        }
    }
    /* right-hand sides: [R(x); p(x)] and d/dx_k of it; x is the origin of xi */
    for (int i = 0; i < n; i++) {
        real r2 = 0;
        for (int k = 0; k < 3; k++) r2 += xi[3 * i + k] * xi[3 * i + k];
        Z[(size_t)i * 4 + 0] = RPOW(r2 + c2, qr);
        real dR = 2 * qr * RPOW(r2 + c2, qr - 1); /* dR/ds times ds/dr^2 = 1 */
        for (int k = 0; k < 3; k++)
            Z[(size_t)i * 4 + 1 + k] = dR * (0 - xi[3 * i + k]); /* d(r^2)/dx_k = 2(x - x_i)_k */
    }
    Z[(size_t)n * 4 + 0] = 1;
    for (int k = 0; k < 3; k++) Z[(size_t)(n + 1 + k) * 4 + 1 + k] = 1;

    /* Gaussian elimination with partial pivoting (largest |entry| in the
     * column, lowest row on ties), applied to the 4 right-hand sides. */
    real gmax = 0;
    for (size_t t = 0; t < (size_t)N * N; t++) if (RABS(G[t]) > gmax) gmax = RABS(G[t]);
    int status = ORC_OK;
    for (int k = 0; k < N && status == ORC_OK; k++) {
        int p = k;
        real best = RABS(G[(size_t)k * N + k]);
        for (int i = k + 1; i < N; i++) {
            real v = RABS(G[(size_t)i * N + k]);
            if (v > best) { best = v; p = i; }
        }
        if (best < (real)1e-13 * gmax) { status = ORC_E_SINGULAR; break; }
        if (p != k) {
            for (int j = 0; j < N; j++) {
                real t = G[(size_t)k * N + j]; G[(size_t)k * N + j] = G[(size_t)p * N + j];
                G[(size_t)p * N + j] = t;
            }
            for (int j = 0; j < 4; j++) {
                real t = Z[(size_t)k * 4 + j]; Z[(size_t)k * 4 + j] = Z[(size_t)p * 4 + j];
                Z[(size_t)p * 4 + j] = t;
            }
        }
        for (int i = k + 1; i < N; i++) {
            real l = G[(size_t)i * N + k] / G[(size_t)k * N + k];
            if (l == 0) continue;
            for (int j = k; j < N; j++) G[(size_t)i * N + j] -= l * G[(size_t)k * N + j];
            for (int j = 0; j < 4; j++) Z[(size_t)i * 4 + j] -= l * Z[(size_t)k * 4 + j];
        }
    }
    if (status == ORC_OK) {
        for (int k = N - 1; k >= 0; k--)
            for (int j = 0; j < 4; j++) {
                real s = Z[(size_t)k * 4 + j];
                for (int i = k + 1; i < N; i++) s -= G[(size_t)k * N + i] * Z[(size_t)i * 4 + j];
                Z[(size_t)k * 4 + j] = s / G[(size_t)k * N + k];
            }
        for (int j = 0; j < n; j++) {
            phi_out[j] = Z[(size_t)j * 4 + 0];
            for (int k = 0; k < 3; k++) phi_out[(size_t)(1 + k) * n + j] = Z[(size_t)j * 4 + 1 + k] / hr;
        }
    }
    free(G); free(Z); free(xi);
    return status;
}

int orc_shape(const double *xyz, const int32_t *supp, int n, const double *x, double h,
              double alpha_c, double q, double *phi)
{
    if (n < 1) return ORC_E_SUPPORT;
    real *tmp = (real *)malloc((size_t)4 * n * sizeof(real));
    if (!tmp) return ORC_E_OOM;
    int st = shape_rpim_real(xyz, supp, n, x, h, alpha_c, q, tmp);
    if (st == ORC_OK)
        for (int t = 0; t < 4 * n; t++) phi[t] = (double)tmp[t];
    free(tmp);
    return st;
}

/* ---------------------------------------------------------------------------
 * MLS shape functions at x (the variant; see the header). Cubic spline
 * weight of sb = |x_i - x| / r_s:
 *   w = 2/3 - 4 sb^2 + 4 sb^3             (sb <= 1/2)
 *   w = 4/3 - 4 sb + 4 sb^2 - 4/3 sb^3    (1/2 < sb <= 1),  0 beyond,
 * and w'(sb) its derivative. Output layout as for RPIM. Returns
 * ORC_E_SINGULAR when a pivot of A falls below 1e-13 * max|A|.
 * ------------------------------------------------------------------------- */
static void spline(real sb, real *w, real *dw)
{
    if (sb <= (real)0.5) {
        *w = (real)2 / 3 - 4 * sb * sb + 4 * sb * sb * sb;
        *dw = -8 * sb + 12 * sb * sb;
    } else if (sb <= 1) {
        *w = (real)4 / 3 - 4 * sb + 4 * sb * sb - (real)4 / 3 * sb * sb * sb;
        *dw = -4 + 8 * sb - 4 * sb * sb;
    } else {
        *w = 0;
        *dw = 0;
    }
}

/* solve the 4x4 system M y = r for 4 right-hand sides (columns of R, 4x4,
 * overwritten with the solutions); partial pivoting, lowest row on ties */
static int solve4(real M[4][4], real R[4][4])
{
    real amax = 0;
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) if (RABS(M[i][j]) > amax) amax = RABS(M[i][j]);
    for (int k = 0; k < 4; k++) {
        int p = k;
        for (int i = k + 1; i < 4; i++) if (RABS(M[i][k]) > RABS(M[p][k])) p = i;
        if (RABS(M[p][k]) < (real)1e-13 * amax) return ORC_E_SINGULAR;
        for (int j = 0; j < 4; j++) {
            real t = M[k][j]; M[k][j] = M[p][j]; M[p][j] = t;
            t = R[k][j]; R[k][j] = R[p][j]; R[p][j] = t;
        }
        for (int i = k + 1; i < 4; i++) {
            real l = M[i][k] / M[k][k];
            for (int j = k; j < 4; j++) M[i][j] -= l * M[k][j];
            for (int j = 0; j < 4; j++) R[i][j] -= l * R[k][j];
        }
    }
    for (int k = 3; k >= 0; k--)
        for (int j = 0; j < 4; j++) {
            real s = R[k][j];
            for (int i = k + 1; i < 4; i++) s -= M[k][i] * R[i][j];
            R[k][j] = s / M[k][k];
        }
    return ORC_OK;
}

static int shape_mls_real(const double *xyz, const int32_t *supp, int n, const double *x, double h,
                          double alpha_s, real *phi_out /* 4*n */)
{
    real *xi = (real *)malloc((size_t)n * 3 * sizeof(real));
    real *w = (real *)malloc((size_t)n * 4 * sizeof(real)); /* w_i, dw_i/dx_k */
    if (!xi || !w) { free(xi); free(w); return ORC_E_OOM; }
    const real hr = (real)h, as = (real)alpha_s;
    real A[4][4], dA[3][4][4];
    memset(A, 0, sizeof A);
    memset(dA, 0, sizeof dA);
    for (int i = 0; i < n; i++) {
        real d2 = 0;
        for (int k = 0; k < 3; k++) {
            xi[3 * i + k] = ((real)xyz[3 * (int64_t)supp[i] + k] - (real)x[k]) / hr;
            d2 += xi[3 * i + k] * xi[3 * i + k];
        }
        const real d = RSQRT(d2), sb = d / as;
        real wv, dws;
        spline(sb, &wv, &dws);
        w[4 * i] = wv;
        for (int k = 0; k < 3; k++) /* d sb / d x_k = -xi_k / (alpha_s h |xi|) */
            w[4 * i + 1 + k] = d > 0 ? dws * (-xi[3 * i + k]) / (as * hr * d) : 0;
        const real p[4] = {1, xi[3 * i], xi[3 * i + 1], xi[3 * i + 2]};
        for (int a = 0; a < 4; a++)
            for (int c = 0; c < 4; c++) {
                A[a][c] += wv * p[a] * p[c];
                for (int k = 0; k < 3; k++) dA[k][a][c] += w[4 * i + 1 + k] * p[a] * p[c];
            }
    }
    /* gamma = A^-1 p(x), p(x) = e0 (x is the origin of xi) */
    real M[4][4], R[4][4];
    memcpy(M, A, sizeof M);
    memset(R, 0, sizeof R);
    R[0][0] = 1;
    int st = solve4(M, R);
    real gam[4], dgam[3][4];
    if (st == ORC_OK) {
        for (int a = 0; a < 4; a++) gam[a] = R[a][0];
        /* dgamma/dx_k = A^-1 (dp/dx_k - dA/dx_k gamma), dp/dx_k = e_{k+1} / h */
        memcpy(M, A, sizeof M);
        memset(R, 0, sizeof R);
        for (int k = 0; k < 3; k++)
            for (int a = 0; a < 4; a++) {
                real s = (a == k + 1) ? 1 / hr : 0;
                for (int c = 0; c < 4; c++) s -= dA[k][a][c] * gam[c];
                R[a][k] = s;
            }
        st = solve4(M, R);
        for (int k = 0; k < 3; k++)
            for (int a = 0; a < 4; a++) dgam[k][a] = R[a][k];
    }
    if (st == ORC_OK)
        for (int i = 0; i < n; i++) {
            const real p[4] = {1, xi[3 * i], xi[3 * i + 1], xi[3 * i + 2]};
            real pg = 0;
            for (int a = 0; a < 4; a++) pg += p[a] * gam[a];
            phi_out[i] = w[4 * i] * pg;
            for (int k = 0; k < 3; k++) {
                real pdg = 0;
                for (int a = 0; a < 4; a++) pdg += p[a] * dgam[k][a];
                phi_out[(size_t)(1 + k) * n + i] = w[4 * i + 1 + k] * pg + w[4 * i] * pdg;
            }
        }
    free(xi); free(w);
    return st;
}

int orc_shape_mls(const double *xyz, const int32_t *supp, int n, const double *x, double h,
                  double alpha_s, double *phi)
{
    if (n < 1) return ORC_E_SUPPORT;
    real *tmp = (real *)malloc((size_t)4 * n * sizeof(real));
    if (!tmp) return ORC_E_OOM;
    int st = shape_mls_real(xyz, supp, n, x, h, alpha_s, tmp);
    if (st == ORC_OK)
        for (int t = 0; t < 4 * n; t++) phi[t] = (double)tmp[t];
    free(tmp);
    return st;
}

/* ---------------------------------------------------------------------------
 * Shepard shape functions at x: phi_i = w_i / W with W = sum_j w_j and the
 * cubic-spline weights of the MLS variant; by the quotient rule
 *   dphi_i/dx_k = (dw_i/dx_k - phi_i dW/dx_k) / W.
 * Returns ORC_E_SINGULAR when no node carries a positive weight.
 * ------------------------------------------------------------------------- */
static int shape_shepard_real(const double *xyz, const int32_t *supp, int n, const double *x, double h,
                              double alpha_s, real *phi_out /* 4*n */)
{
    const real hr = (real)h, as = (real)alpha_s;
    real W = 0, dW[3] = {0, 0, 0};
    for (int pass = 0; pass < 2; pass++) {
        for (int i = 0; i < n; i++) {
            real xi[3], d2 = 0;
            for (int k = 0; k < 3; k++) {
                xi[k] = ((real)xyz[3 * (int64_t)supp[i] + k] - (real)x[k]) / hr;
                d2 += xi[k] * xi[k];
            }
            const real d = RSQRT(d2), sb = d / as;
            real wv, dws, dw[3];
            spline(sb, &wv, &dws);
            for (int k = 0; k < 3; k++) dw[k] = d > 0 ? dws * (-xi[k]) / (as * hr * d) : 0;
            if (pass == 0) {
                W += wv;
                for (int k = 0; k < 3; k++) dW[k] += dw[k];
            } else {
                const real ph = wv / W;
                phi_out[i] = ph;
                for (int k = 0; k < 3; k++) phi_out[(size_t)(1 + k) * n + i] = (dw[k] - ph * dW[k]) / W;
            }
        }
        if (pass == 0 && !(W > 0)) return ORC_E_SINGULAR;
    }
    return ORC_OK;
}

int orc_shape_shepard(const double *xyz, const int32_t *supp, int n, const double *x, double h,
                      double alpha_s, double *phi)
{
    if (n < 1) return ORC_E_SUPPORT;
    real *tmp = (real *)malloc((size_t)4 * n * sizeof(real));
    if (!tmp) return ORC_E_OOM;
    int st = shape_shepard_real(xyz, supp, n, x, h, alpha_s, tmp);
    if (st == ORC_OK)
        for (int t = 0; t < 4 * n; t++) phi[t] = (double)tmp[t];
    free(tmp);
    return st;
}

/* the shape functions selected by orc_set_shape */
static int shape_real(const double *xyz, const int32_t *supp, int n, const double *x, double h,
                      double alpha_s, double alpha_c, double q, real *phi_out)
{
    if (g_shape == 1) return shape_mls_real(xyz, supp, n, x, h, alpha_s, phi_out);
    if (g_shape == 2) return shape_shepard_real(xyz, supp, n, x, h, alpha_s, phi_out);
    return shape_rpim_real(xyz, supp, n, x, h, alpha_c, q, phi_out);
}

/* ---------------------------------------------------------------------------
 * Isotropic elasticity in Voigt form (xx, yy, zz, yz, xz, xy), engineering
 * shear strains: lambda = E nu / ((1 + nu)(1 - 2 nu)), mu = E / (2 (1 + nu)).
 * ------------------------------------------------------------------------- */
static void elastic_D(real E, real nu, real D[6][6])
{
    real lam = E * nu / ((1 + nu) * (1 - 2 * nu));
    real mu = E / (2 * (1 + nu));
    memset(D, 0, sizeof(real) * 36);
    for (int a = 0; a < 3; a++) {
        for (int b = 0; b < 3; b++) D[a][b] = lam;
        D[a][a] = lam + 2 * mu;
        D[3 + a][3 + a] = mu;
    }
}

/* strain matrix of node I from its gradient g = (phi_x, phi_y, phi_z) */
static void strain_B(const real g[3], real B[6][3])
{
    memset(B, 0, sizeof(real) * 18);
    B[0][0] = g[0];
    B[1][1] = g[1];
    B[2][2] = g[2];
    B[3][1] = g[2]; B[3][2] = g[1]; /* gamma_yz */
    B[4][0] = g[2]; B[4][2] = g[0]; /* gamma_xz */
    B[5][0] = g[1]; B[5][1] = g[0]; /* gamma_xy */
}

/* ---------------------------------------------------------------------------
 * Assembly of K (3x3-block CSR) and the body-force vector over a list of
 * integration points. The pattern holds block (I, J) iff some point has both
 * I and J in its support (block symmetric by construction). Blocks are accumulated point by point in the given
 * (ascending) point order.
 * ------------------------------------------------------------------------- */
typedef struct {
    int64_t n_nodes, nnzb;
    int64_t *rowptr;
    int32_t *cols;
    real *vals;  /* 9 per block, row-major 3x3 */
    real *f;     /* 3 per node */
    int64_t *soff; /* support offsets per point */
    int32_t *sidx; /* support ids */
    int64_t n_pts;
    int status;
    int64_t bad_point;
} orc_model;

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

static int64_t find_col(const orc_model *m, int64_t I, int32_t J)
{
    int64_t lo = m->rowptr[I], hi = m->rowptr[I + 1] - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (m->cols[mid] == J) return mid;
        if (m->cols[mid] < J) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

void orc_free(orc_model *m)
{
    if (!m) return;
    free(m->rowptr); free(m->cols); free(m->vals); free(m->f); free(m->soff); free(m->sidx);
    free(m);
}

orc_model *orc_assemble(int64_t n_nodes, const double *xyz, int64_t n_pts, const double *pts,
                        const double *wj, const double *E, const double *nu, const double *body,
                        double alpha_s, double alpha_c, double q, double h, int max_support,
                        const uint8_t *row_mask)
{
    orc_model *m = (orc_model *)calloc(1, sizeof(orc_model));
    if (!m) return NULL;
    m->n_nodes = n_nodes;
    m->n_pts = n_pts;
    m->bad_point = -1;
    const double rs2 = orc_support_radius2(alpha_s, h);

    /* supports by brute force */
    m->soff = (int64_t *)malloc((size_t)(n_pts + 1) * sizeof(int64_t));
    int32_t *tmp = (int32_t *)malloc((size_t)max_support * sizeof(int32_t));
    if (!m->soff || !tmp) { free(tmp); m->status = ORC_E_OOM; return m; }
    m->soff[0] = 0;
    for (int64_t g = 0; g < n_pts; g++) {
        int64_t c = orc_support(n_nodes, xyz, pts + 3 * g, rs2, tmp, max_support);
        if (c > max_support || c < 4) { m->status = ORC_E_SUPPORT; m->bad_point = g; free(tmp); return m; }
        m->soff[g + 1] = m->soff[g] + c;
    }
    m->sidx = (int32_t *)malloc((size_t)m->soff[n_pts] * sizeof(int32_t) + 4);
    if (!m->sidx) { free(tmp); m->status = ORC_E_OOM; return m; }
    for (int64_t g = 0; g < n_pts; g++)
        orc_support(n_nodes, xyz, pts + 3 * g, rs2, m->sidx + m->soff[g], max_support);
    free(tmp);

    /* pattern: row I holds J iff some point has both I and J in its support.
     * Rows are collected through the node -> point incidence lists with a
     * marker array, then sorted. */
    int64_t *ioff = (int64_t *)calloc((size_t)n_nodes + 1, sizeof(int64_t));
    int64_t *ipts = (int64_t *)malloc((size_t)m->soff[n_pts] * sizeof(int64_t) + 8);
    int64_t *mark = (int64_t *)malloc((size_t)n_nodes * sizeof(int64_t));
    int64_t *cnt = (int64_t *)calloc((size_t)n_nodes + 1, sizeof(int64_t));
    if (!ioff || !ipts || !mark || !cnt) {
        free(ioff); free(ipts); free(mark); free(cnt); m->status = ORC_E_OOM; return m;
    }
    for (int64_t e = 0; e < m->soff[n_pts]; e++) ioff[m->sidx[e] + 1]++;
    for (int64_t i = 0; i < n_nodes; i++) ioff[i + 1] += ioff[i];
    for (int64_t g = 0; g < n_pts; g++)
        for (int64_t e = m->soff[g]; e < m->soff[g + 1]; e++) {
            int64_t I = m->sidx[e];
            ipts[ioff[I] + cnt[I]++] = g;
        }
    for (int64_t i = 0; i < n_nodes; i++) mark[i] = -1;
    m->rowptr = (int64_t *)calloc((size_t)n_nodes + 1, sizeof(int64_t));
    for (int pass = 0; pass < 2; pass++) {
        for (int64_t i = 0; i < n_nodes; i++) mark[i] = -1;
        for (int64_t I = 0; I < n_nodes; I++) {
            int64_t c = 0;
            for (int64_t t = ioff[I]; t < ioff[I + 1]; t++) {
                int64_t g = ipts[t];
                for (int64_t e = m->soff[g]; e < m->soff[g + 1]; e++) {
                    int32_t J = m->sidx[e];
                    if (mark[J] != I) {
                        mark[J] = I;
                        if (pass == 1) m->cols[m->rowptr[I] + c] = J;
                        c++;
                    }
                }
            }
            if (pass == 0) m->rowptr[I + 1] = c;
            else qsort(m->cols + m->rowptr[I], (size_t)c, sizeof(int32_t), cmp_i32);
        }
        if (pass == 0) {
            for (int64_t i = 0; i < n_nodes; i++) m->rowptr[i + 1] += m->rowptr[i];
            m->nnzb = m->rowptr[n_nodes];
            m->cols = (int32_t *)malloc((size_t)m->nnzb * sizeof(int32_t) + 4);
            m->vals = (real *)calloc((size_t)m->nnzb * 9 + 1, sizeof(real));
            m->f = (real *)calloc((size_t)n_nodes * 3, sizeof(real));
            if (!m->cols || !m->vals || !m->f) {
                free(ioff); free(ipts); free(mark); free(cnt); m->status = ORC_E_OOM; return m;
            }
        }
    }
    free(mark); free(cnt);

    /* shape functions of every point (independent per point; the paper's CPU
     * scheme runs these in parallel with OpenMP, Sec. 2) */
    real *phis = (real *)malloc((size_t)m->soff[n_pts] * 4 * sizeof(real) + 8);
    if (!phis) { free(ioff); free(ipts); m->status = ORC_E_OOM; return m; }
    int64_t bad = -1;
    int bad_status = ORC_OK;
#pragma omp parallel for schedule(dynamic, 16) num_threads(g_threads)
    for (int64_t g = 0; g < n_pts; g++) {
        int n = (int)(m->soff[g + 1] - m->soff[g]);
        int st = shape_real(xyz, m->sidx + m->soff[g], n, pts + 3 * g, h, alpha_s, alpha_c, q,
                            phis + 4 * m->soff[g]);
        if (st != ORC_OK) {
#pragma omp critical
            { if (bad < 0 || g < bad) { bad = g; bad_status = st; } }
        }
    }
    if (bad >= 0) { free(ioff); free(ipts); free(phis); m->status = bad_status; m->bad_point = bad; return m; }

    /* accumulate w|J| B_I^T D B_J for every ordered pair (I, J) of every
     * point's support, each block over the points in ascending order. Row I
     * takes its points from the incidence list (ascending) and is formed by
     * one thread, so rows can be formed in parallel and each block is the
     * same sum in the same order as a point-by-point sweep. With row_mask,
     * only the rows I with row_mask[I] != 0 are formed (the others stay 0). */
#pragma omp parallel for schedule(dynamic, 16) num_threads(g_threads)
    for (int64_t I = 0; I < n_nodes; I++) {
        if (row_mask && !row_mask[I]) continue;
        for (int64_t t = ioff[I]; t < ioff[I + 1]; t++) {
            const int64_t g = ipts[t];
            const int n = (int)(m->soff[g + 1] - m->soff[g]);
            const int32_t *s = m->sidx + m->soff[g];
            const real *ph = phis + 4 * m->soff[g];
            real D[6][6];
            elastic_D((real)E[g], (real)nu[g], D);
            const real w = (real)wj[g];
            int a = 0;
            while (s[a] != (int32_t)I) a++;   /* I's place in the support of g */
            real ga[3] = {ph[n + a], ph[2 * n + a], ph[3 * n + a]};
            real Ba[6][3];
            strain_B(ga, Ba);
            for (int b = 0; b < n; b++) {
                real gb[3] = {ph[n + b], ph[2 * n + b], ph[3 * n + b]};
                real Bb[6][3], DBb[6][3];
                strain_B(gb, Bb);
                for (int r = 0; r < 6; r++)
                    for (int cc = 0; cc < 3; cc++) {
                        real acc = 0;
                        for (int k = 0; k < 6; k++) acc += D[r][k] * Bb[k][cc];
                        DBb[r][cc] = acc;
                    }
                int64_t slot = find_col(m, s[a], s[b]);
                real *kv = m->vals + 9 * slot;
                for (int al = 0; al < 3; al++)
                    for (int be = 0; be < 3; be++) {
                        real acc = 0;
                        for (int k = 0; k < 6; k++) acc += Ba[k][al] * DBb[k][be];
                        kv[3 * al + be] += w * acc;
                    }
            }
            if (body)
                for (int k = 0; k < 3; k++) m->f[3 * (int64_t)s[a] + k] += ph[a] * (real)body[k] * w;
        }
    }
    free(ioff); free(ipts); free(phis);
    return m;
}

int orc_status(const orc_model *m) { return m ? m->status : ORC_E_OOM; }
int64_t orc_bad_point(const orc_model *m) { return m ? m->bad_point : -1; }
int64_t orc_nnzb(const orc_model *m) { return m ? m->nnzb : -1; }
int64_t orc_support_total(const orc_model *m) { return m ? m->soff[m->n_pts] : -1; }

void orc_copy_csr(const orc_model *m, int64_t *rowptr, int32_t *cols, double *vals, double *f)
{
    if (rowptr) memcpy(rowptr, m->rowptr, (size_t)(m->n_nodes + 1) * sizeof(int64_t));
    if (cols) memcpy(cols, m->cols, (size_t)m->nnzb * sizeof(int32_t));
    if (vals) for (int64_t i = 0; i < 9 * m->nnzb; i++) vals[i] = (double)m->vals[i];
    if (f) for (int64_t i = 0; i < 3 * m->n_nodes; i++) f[i] = (double)m->f[i];
}

void orc_copy_support(const orc_model *m, int64_t *off, int32_t *idx)
{
    if (off) memcpy(off, m->soff, (size_t)(m->n_pts + 1) * sizeof(int64_t));
    if (idx) memcpy(idx, m->sidx, (size_t)m->soff[m->n_pts] * sizeof(int32_t));
}

/* ---------------------------------------------------------------------------
 * Surface loads lumped at points: f_I += phi_I(x_p) F_p (F_p = traction x
 * quadrature weight), points in the given order.
 * ------------------------------------------------------------------------- */
int orc_point_loads(int64_t n_nodes, const double *xyz, int64_t n, const double *pts,
                    const double *force, double alpha_s, double alpha_c, double q, double h,
                    int max_support, double *f)
{
    const double rs2 = orc_support_radius2(alpha_s, h);
    int32_t *s = (int32_t *)malloc((size_t)max_support * sizeof(int32_t));
    real *ph = (real *)malloc((size_t)max_support * 4 * sizeof(real));
    real *acc = (real *)calloc((size_t)n_nodes * 3, sizeof(real));
    if (!s || !ph || !acc) { free(s); free(ph); free(acc); return ORC_E_OOM; }
    int st = ORC_OK;
    for (int64_t p = 0; p < n && st == ORC_OK; p++) {
        int64_t c = orc_support(n_nodes, xyz, pts + 3 * p, rs2, s, max_support);
        if (c < 4 || c > max_support) { st = ORC_E_SUPPORT; break; }
        st = shape_real(xyz, s, (int)c, pts + 3 * p, h, alpha_s, alpha_c, q, ph);
        if (st != ORC_OK) break;
        for (int64_t a = 0; a < c; a++)
            for (int k = 0; k < 3; k++) acc[3 * (int64_t)s[a] + k] += ph[a] * (real)force[3 * p + k];
    }
    if (st == ORC_OK)
        for (int64_t i = 0; i < 3 * n_nodes; i++) f[i] += (double)acc[i];
    free(s); free(ph); free(acc);
    return st;
}

/* ---------------------------------------------------------------------------
 * Surface tractions on axis-aligned face rectangles (the pressure and shear
 * loads of the verification examples, Sec. 3): face k lies in the plane
 * x_a = lo[a] (a = axis[k]) and spans [lo, hi] along the two other axes
 * u < v. The traction component c is the polynomial
 *     t_c(u, v) = C0 + C1 u + C2 v + C3 u^2 + C4 u v + C5 v^2
 * (coef[18 k + 6 c + j]) in global coordinates. Each face is integrated with
 * the 2x2 Gauss-Legendre rule: points mid +- half/sqrt(3) along u and v
 * (point l = a + 2b, bit a for u, b for v, 0 -> minus), weight
 * half_u * half_v, so f_I += sum over points of phi_I(x_p) t(x_p) w_p,
 * faces in order, points in order. Exact for tractions of degree <= 3 in
 * each tangent coordinate times polynomial shape functions.
 * ------------------------------------------------------------------------- */
int orc_traction(int64_t n_nodes, const double *xyz, int64_t n_faces, const double *lo,
                 const double *hi, const int8_t *axis, const double *coef, double alpha_s,
                 double alpha_c, double q, double h, int max_support, double *f)
{
    const double rs2 = orc_support_radius2(alpha_s, h);
    int32_t *s = (int32_t *)malloc((size_t)max_support * sizeof(int32_t));
    real *ph = (real *)malloc((size_t)max_support * 4 * sizeof(real));
    real *acc = (real *)calloc((size_t)n_nodes * 3, sizeof(real));
    if (!s || !ph || !acc) { free(s); free(ph); free(acc); return ORC_E_OOM; }
    int st = ORC_OK;
    for (int64_t k = 0; k < n_faces && st == ORC_OK; k++) {
        const int a = axis[k];
        if (a < 0 || a > 2) { st = ORC_E_ARG; break; }
        const int ua = a == 0 ? 1 : 0, va = a == 2 ? 1 : 2;   /* tangent axes, ascending */
        const double *l = lo + 3 * k, *u = hi + 3 * k;
        if (l[a] != u[a] || !(l[ua] <= u[ua]) || !(l[va] <= u[va])) { st = ORC_E_ARG; break; }
        const double mu = (l[ua] + u[ua]) * 0.5, hu = (u[ua] - l[ua]) * 0.5;
        const double mv = (l[va] + u[va]) * 0.5, hv = (u[va] - l[va]) * 0.5;
        const double w = hu * hv;
        for (int pt = 0; pt < 4 && st == ORC_OK; pt++) {
            double x[3];
            x[a] = l[a];
            x[ua] = mu + hu * ((pt & 1) ? GAUSS2 : -GAUSS2);
            x[va] = mv + hv * ((pt & 2) ? GAUSS2 : -GAUSS2);
            const double U = x[ua], V = x[va];
            const double m[6] = {1.0, U, V, U * U, U * V, V * V};
            real F[3];
            for (int c = 0; c < 3; c++) {
                real t = 0;
                for (int j = 0; j < 6; j++) t += (real)coef[18 * k + 6 * c + j] * (real)m[j];
                F[c] = t * (real)w;
            }
            int64_t cnt = orc_support(n_nodes, xyz, x, rs2, s, max_support);
            if (cnt < 4 || cnt > max_support) { st = ORC_E_SUPPORT; break; }
            st = shape_real(xyz, s, (int)cnt, x, h, alpha_s, alpha_c, q, ph);
            if (st != ORC_OK) break;
            for (int64_t i = 0; i < cnt; i++)
                for (int c = 0; c < 3; c++) acc[3 * (int64_t)s[i] + c] += ph[i] * F[c];
        }
    }
    if (st == ORC_OK)
        for (int64_t i = 0; i < 3 * n_nodes; i++) f[i] += (double)acc[i];
    free(s); free(ph); free(acc);
    return st;
}

/* ---------------------------------------------------------------------------
 * Penalty enforcement of prescribed displacements (Sec. 2, second stage).
 * alpha = scale * max_i K_ii over all scalar diagonal entries;
 * K_dd += alpha and f_d += alpha * value for each listed DOF.
 * ------------------------------------------------------------------------- */
int orc_penalty(int64_t n_nodes, const int64_t *rowptr, const int32_t *cols, double *vals,
                double *f, int64_t m, const int64_t *dofs, const double *values, double scale,
                double *alpha_out)
{
    /* scale < 0: alpha = -scale is given by the caller (frozen penalty) */
    double kmax = 0.0;
    for (int64_t I = 0; I < n_nodes; I++)
        for (int64_t t = rowptr[I]; t < rowptr[I + 1]; t++)
            if (cols[t] == I)
                for (int a = 0; a < 3; a++)
                    if (vals[9 * t + 4 * a] > kmax) kmax = vals[9 * t + 4 * a];
    double alpha = scale < 0 ? -scale : scale * kmax;
    for (int64_t i = 0; i < m; i++) {
        int64_t d = dofs[i], I = d / 3;
        int a = (int)(d % 3);
        if (d < 0 || I >= n_nodes) return ORC_E_ARG;
        int64_t slot = -1;
        for (int64_t t = rowptr[I]; t < rowptr[I + 1]; t++) if (cols[t] == I) slot = t;
        if (slot < 0) return ORC_E_ARG;
        vals[9 * slot + 4 * a] += alpha;
        f[d] += alpha * values[i];
    }
    if (alpha_out) *alpha_out = alpha;
    return ORC_OK;
}

/* y = K x on the 3x3-block CSR matrix */
static void spmv(int64_t n_nodes, const int64_t *rowptr, const int32_t *cols, const double *vals,
                 const real *x, real *y)
{
    for (int64_t I = 0; I < n_nodes; I++) {
        real acc[3] = {0, 0, 0};
        for (int64_t t = rowptr[I]; t < rowptr[I + 1]; t++) {
            const double *b = vals + 9 * t;
            const real *xj = x + 3 * (int64_t)cols[t];
            for (int a = 0; a < 3; a++)
                acc[a] += (real)b[3 * a] * xj[0] + (real)b[3 * a + 1] * xj[1] + (real)b[3 * a + 2] * xj[2];
        }
        for (int a = 0; a < 3; a++) y[3 * I + a] = acc[a];
    }
}

static real dot(int64_t n, const real *a, const real *b)
{
    real s = 0;
    for (int64_t i = 0; i < n; i++) s += a[i] * b[i];
    return s;
}

/* inverse of a 3x3 matrix by Gauss-Jordan elimination with partial pivoting
 * (row-major in and out); ORC_E_SINGULAR on a zero pivot */
static int inverse3(const double *a, real *inv)
{
    real m[3][6];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 6; j++) m[i][j] = j < 3 ? (real)a[3 * i + j] : (real)(j - 3 == i);
    for (int k = 0; k < 3; k++) {
        int p = k;
        for (int i = k + 1; i < 3; i++) if (RABS(m[i][k]) > RABS(m[p][k])) p = i;
        if (m[p][k] == 0) return ORC_E_SINGULAR;
        for (int j = 0; j < 6; j++) { real t = m[k][j]; m[k][j] = m[p][j]; m[p][j] = t; }
        const real piv = m[k][k];
        for (int j = 0; j < 6; j++) m[k][j] /= piv;
        for (int i = 0; i < 3; i++) {
            if (i == k) continue;
            const real l = m[i][k];
            for (int j = 0; j < 6; j++) m[i][j] -= l * m[k][j];
        }
    }
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) inv[3 * i + j] = m[i][3 + j];
    return ORC_OK;
}

/* z = M^-1 r: Jacobi (dinv[i] = 1 / K_ii) or block Jacobi (dinv[9I..] the
 * inverse of node I's 3x3 diagonal block) */
static void precondition(int block, int64_t n_nodes, const real *dinv, const real *r, real *z)
{
    if (!block) {
        for (int64_t i = 0; i < 3 * n_nodes; i++) z[i] = dinv[i] * r[i];
        return;
    }
    for (int64_t I = 0; I < n_nodes; I++)
        for (int a = 0; a < 3; a++) {
            real s = 0;
            for (int b = 0; b < 3; b++) s += dinv[9 * I + 3 * a + b] * r[3 * I + b];
            z[3 * I + a] = s;
        }
}

/* ---------------------------------------------------------------------------
 * Preconditioned conjugate gradients (Sec. 2, third stage; the paper calls a
 * library solver, this is the textbook PCG) with the Jacobi (block = 0) or
 * 3x3 block-Jacobi (block = 1) preconditioner: stops when
 * ||r|| <= rtol ||f|| or after max_iter iterations. u holds the initial guess
 * on entry and the solution on exit.
 * ------------------------------------------------------------------------- */
int orc_pcg(int64_t n_nodes, const int64_t *rowptr, const int32_t *cols, const double *vals,
            const double *f, double *u, double rtol, int max_iter, int *iters, double *relres, int block)
{
    const int64_t n = 3 * n_nodes;
    real *x = (real *)malloc((size_t)n * sizeof(real)), *r = (real *)malloc((size_t)n * sizeof(real));
    real *z = (real *)malloc((size_t)n * sizeof(real)), *p = (real *)malloc((size_t)n * sizeof(real));
    real *qv = (real *)malloc((size_t)n * sizeof(real));
    real *dinv = (real *)malloc((size_t)(block ? 3 : 1) * n * sizeof(real));
    if (!x || !r || !z || !p || !qv || !dinv) {
        free(x); free(r); free(z); free(p); free(qv); free(dinv);
        return ORC_E_OOM;
    }
    for (int64_t I = 0; I < n_nodes; I++)
        for (int64_t t = rowptr[I]; t < rowptr[I + 1]; t++)
            if (cols[t] == I) {
                if (block) {
                    if (inverse3(vals + 9 * t, dinv + 9 * I) != ORC_OK) {
                        free(x); free(r); free(z); free(p); free(qv); free(dinv);
                        return ORC_E_SINGULAR;
                    }
                } else {
                    for (int a = 0; a < 3; a++) dinv[3 * I + a] = 1 / (real)vals[9 * t + 4 * a];
                }
            }
    for (int64_t i = 0; i < n; i++) x[i] = (real)u[i];
    spmv(n_nodes, rowptr, cols, vals, x, qv);
    real fn = 0;
    for (int64_t i = 0; i < n; i++) { r[i] = (real)f[i] - qv[i]; fn += (real)f[i] * (real)f[i]; }
    fn = RSQRT(fn);
    if (fn == 0) fn = 1;
    precondition(block, n_nodes, dinv, r, z);
    for (int64_t i = 0; i < n; i++) p[i] = z[i];
    real rz = dot(n, r, z);
    real rn = RSQRT(dot(n, r, r));
    int it = 0;
    while (rn > (real)rtol * fn && it < max_iter) {
        spmv(n_nodes, rowptr, cols, vals, p, qv);
        real alpha = rz / dot(n, p, qv);
        for (int64_t i = 0; i < n; i++) { x[i] += alpha * p[i]; r[i] -= alpha * qv[i]; }
        precondition(block, n_nodes, dinv, r, z);
        real rz_new = dot(n, r, z);
        real beta = rz_new / rz;
        rz = rz_new;
        for (int64_t i = 0; i < n; i++) p[i] = z[i] + beta * p[i];
        rn = RSQRT(dot(n, r, r));
        it++;
    }
    for (int64_t i = 0; i < n; i++) u[i] = (double)x[i];
    if (iters) *iters = it;
    if (relres) *relres = (double)(rn / fn);
    free(x); free(r); free(z); free(p); free(qv); free(dinv);
    return rn <= (real)rtol * fn ? ORC_OK : ORC_E_NOCONV;
}

/* ---------------------------------------------------------------------------
 * Material gradient of a solved system (back-analysis). With K(theta) u = f
 * and the adjoint K lam = dL/du (K symmetric, penalty frozen), the gradient
 * of L with respect to the parameters of point g is
 *     dL/dtheta_g = - w_g eps_g(lam)^T (dD/dtheta) eps_g(u),
 * eps_g(v) = sum_I B_I(x_g) v_I, for theta = E and theta = nu, with
 *     dD/dE = D/E,
 *     dD/dnu = dlambda/dnu (1 1 1 0 0 0)^T (1 1 1 0 0 0)
 *              + dmu/dnu diag(2, 2, 2, 1, 1, 1),
 *     dlambda/dnu = E (1 + 2 nu^2) / ((1 + nu)^2 (1 - 2 nu)^2),
 *     dmu/dnu = -E / (2 (1 + nu)^2).
 * ------------------------------------------------------------------------- */
static void elastic_dD(real E, real nu, real dDE[6][6], real dDnu[6][6])
{
    real D[6][6];
    elastic_D(E, nu, D);
    for (int a = 0; a < 6; a++)
        for (int b = 0; b < 6; b++) dDE[a][b] = D[a][b] / E;
    real dlam = E * (1 + 2 * nu * nu) / ((1 + nu) * (1 + nu) * (1 - 2 * nu) * (1 - 2 * nu));
    real dmu = -E / (2 * (1 + nu) * (1 + nu));
    memset(dDnu, 0, sizeof(real) * 36);
    for (int a = 0; a < 3; a++) {
        for (int b = 0; b < 3; b++) dDnu[a][b] = dlam;
        dDnu[a][a] = dlam + 2 * dmu;
        dDnu[3 + a][3 + a] = dmu;
    }
}

int orc_grad_material(int64_t n_nodes, const double *xyz, int64_t n_pts, const double *pts,
                      const double *wj, const double *E, const double *nu, const double *u,
                      const double *lam, double alpha_s, double alpha_c, double q, double h,
                      int max_support, double *dE, double *dnu)
{
    const double rs2 = orc_support_radius2(alpha_s, h);
    int32_t *s = (int32_t *)malloc((size_t)max_support * sizeof(int32_t));
    real *ph = (real *)malloc((size_t)max_support * 4 * sizeof(real));
    if (!s || !ph) { free(s); free(ph); return ORC_E_OOM; }
    int st = ORC_OK;
    for (int64_t p = 0; p < n_pts; p++) {
        int64_t c = orc_support(n_nodes, xyz, pts + 3 * p, rs2, s, max_support);
        if (c < 4 || c > max_support) { st = ORC_E_SUPPORT; break; }
        st = shape_real(xyz, s, (int)c, pts + 3 * p, h, alpha_s, alpha_c, q, ph);
        if (st != ORC_OK) break;
        real eu[6] = {0, 0, 0, 0, 0, 0}, el[6] = {0, 0, 0, 0, 0, 0};
        for (int64_t a = 0; a < c; a++) {
            real g[3] = {ph[c + a], ph[2 * c + a], ph[3 * c + a]};
            real B[6][3];
            strain_B(g, B);
            for (int r = 0; r < 6; r++)
                for (int k = 0; k < 3; k++) {
                    eu[r] += B[r][k] * (real)u[3 * (int64_t)s[a] + k];
                    el[r] += B[r][k] * (real)lam[3 * (int64_t)s[a] + k];
                }
        }
        real dDE[6][6], dDnu[6][6];
        elastic_dD((real)E[p], (real)nu[p], dDE, dDnu);
        real ge = 0, gn = 0;
        for (int a = 0; a < 6; a++)
            for (int b = 0; b < 6; b++) {
                ge += el[a] * dDE[a][b] * eu[b];
                gn += el[a] * dDnu[a][b] * eu[b];
            }
        dE[p] = (double)(-(real)wj[p] * ge);
        dnu[p] = (double)(-(real)wj[p] * gn);
    }
    free(s); free(ph);
    return st;
}

/* ---------------------------------------------------------------------------
 * Stress at points: sigma = D(E_p, nu_p) sum_I B_I(x_p) u_I, Voigt order
 * xx, yy, zz, yz, xz, xy.
 * ------------------------------------------------------------------------- */
int orc_stress(int64_t n_nodes, const double *xyz, const double *u, int64_t n_pts,
               const double *pts, const double *E, const double *nu, double alpha_s,
               double alpha_c, double q, double h, int max_support, double *sigma)
{
    const double rs2 = orc_support_radius2(alpha_s, h);
    int32_t *s = (int32_t *)malloc((size_t)max_support * sizeof(int32_t));
    real *ph = (real *)malloc((size_t)max_support * 4 * sizeof(real));
    if (!s || !ph) { free(s); free(ph); return ORC_E_OOM; }
    int st = ORC_OK;
    for (int64_t p = 0; p < n_pts; p++) {
        int64_t c = orc_support(n_nodes, xyz, pts + 3 * p, rs2, s, max_support);
        if (c < 4 || c > max_support) { st = ORC_E_SUPPORT; break; }
        st = shape_real(xyz, s, (int)c, pts + 3 * p, h, alpha_s, alpha_c, q, ph);
        if (st != ORC_OK) break;
        real eps[6] = {0, 0, 0, 0, 0, 0};
        for (int64_t a = 0; a < c; a++) {
            real g[3] = {ph[c + a], ph[2 * c + a], ph[3 * c + a]};
            real B[6][3];
            strain_B(g, B);
            for (int r = 0; r < 6; r++)
                for (int k = 0; k < 3; k++) eps[r] += B[r][k] * (real)u[3 * (int64_t)s[a] + k];
        }
        real D[6][6];
        elastic_D((real)E[p], (real)nu[p], D);
        for (int r = 0; r < 6; r++) {
            real acc = 0;
            for (int k = 0; k < 6; k++) acc += D[r][k] * eps[k];
            sigma[6 * p + r] = (double)acc;
        }
    }
    free(s); free(ph);
    return st;
}
