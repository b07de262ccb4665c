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
#include <atomic>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace rpim {

// Conversions between double and float by bit manipulation on the integer
// pipe (the FP64 pipe is the bottleneck of this kernel). Both truncate and
// flush values outside the single-precision normal range to zero.
__device__ __forceinline__ float f32_from_f64(double d)
{
    const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
    const int e = (int)((hi >> 20) & 0x7FF) - 1023 + 127;
    if (e <= 0 || e >= 255) return 0.0f;
    return __uint_as_float((hi & 0x80000000u) | ((unsigned)e << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29));
}

__device__ __forceinline__ double f64_from_f32(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xFF;
    if (e == 0) return 0.0;
    const unsigned hi = (u & 0x80000000u) | ((e - 127 + 1023) << 20) | ((u & 0x7FFFFFu) >> 3);
    return __hiloint2double((int)hi, (int)(u << 29));
}

// true for a positive, finite, normal double (integer test)
__device__ __forceinline__ bool positive_normal(double d)
{
    const int hi = __double2hiint(d);
    return hi > 0x000FFFFF && hi < 0x7FF00000;
}

// Small integers to float and back without a conversion instruction (the
// conversions do not run on the FP32 pipe): for 0 <= x < 2^23 the float
// 2^23 + x has the bits 0x4B000000 | x, and adding 2^23 to 0 <= f < 2^22
// leaves the nearest integer of f in the low mantissa bits.
__device__ __forceinline__ float small_int_to_float(int x)
{
    return __fsub_rn(__int_as_float(0x4B000000 | x), 8388608.0f);
}

__device__ __forceinline__ int small_float_to_int(float f)
{
    return __float_as_int(__fadd_rn(f, 8388608.0f)) & 0x7FFFFF;
}

// Reciprocal by Newton-Raphson iteration r <- r (2 - d r) from a
// single-precision seed: the relative error squares at each step
// (2^-22 -> 2^-44 -> below double rounding), so two steps give a result
// within an ulp of 1/d (tested against correctly rounded division through
// rpim_probe_recip). |d| must lie in [2^-126, 2^126], where both d and the
// seed 1/d are single-precision normal numbers; either sign. (Pivots and
// determinants in this kernel are of order 1e-9 to 1e3.)
__device__ __forceinline__ double recip_nr(double d)
{
    double r = f64_from_f32(__frcp_rn(f32_from_f64(d)));
    double e = fma(-d, r, 1.0);
    r = fma(r, e, r);
    e = fma(-d, r, 1.0);
    return fma(r, e, r);
}

// ---------------------------------------------------------------------------
// Double-single ("float-float") arithmetic for the refined solver: a value is
// the unevaluated sum hi + lo of two FP32 numbers with |lo| <= ulp(hi) / 2,
// about 48 significant bits. Sums use Knuth's TwoSum and products Dekker's
// exact product in its FMA form (fmaf(a, b, -a*b) is the rounding error of
// a*b exactly); both are error-free transformations (Knuth, TAOCP vol. 2,
// 4.2.2; Dekker, Numer. Math. 18, 1971). Every operation is spelled with the
// round-to-nearest intrinsics, which the compiler neither contracts into
// fused operations nor reorders. On this GPU an FP32 operation costs 1/64 of
// an FP64 one, so the ~15 FP32 operations of a float-float multiply-add are
// still several times cheaper than one FP64 FMA.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return make_float2(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}

// a + b for |a| >= |b| (or a == 0)
__device__ __forceinline__ float2 fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ float2 ff_mul(float2 x, float2 y)
{
    const float p = __fmul_rn(x.x, y.x);
    float e = __fmaf_rn(x.x, y.x, -p);
    e = __fmaf_rn(x.x, y.y, e);
    e = __fmaf_rn(x.y, y.x, e);
    return fast_two_sum(p, e);
}

// c - x * y
__device__ __forceinline__ float2 ff_fnma(float2 x, float2 y, float2 c)
{
    const float p = __fmul_rn(x.x, y.x);
    float pe = __fmaf_rn(x.x, y.x, -p);
    pe = __fmaf_rn(x.x, y.y, pe);
    pe = __fmaf_rn(x.y, y.x, pe);
    const float2 s = two_sum(c.x, -p);
    const float e = __fadd_rn(s.y, __fsub_rn(c.y, pe));
    return two_sum(s.x, e);
}

// hi + lo of a double on the integer pipe: hi is d truncated to 24 bits,
// lo the next 24 bits of the remainder (truncated); d outside the FP32
// normal range, and remainders below it, flush to zero.
__device__ __forceinline__ float2 ff_from_f64(double d)
{
    const float hi = f32_from_f64(d);
    if (hi == 0.0f) return make_float2(0.0f, 0.0f);
    const unsigned hw = (unsigned)__double2hiint(d), lw = (unsigned)__double2loint(d);
    const int e = (int)((hw >> 20) & 0x7FF) - 1023 - 52 + 127;   // biased FP32 exponent of the lowest bit
    const unsigned rem = lw & 0x1FFFFFFFu;                         // the 29 bits below hi
    float lo = 0.0f;
    if (rem) {   // normalise rem by its leading bit (integer pipe)
        const int lz = __clz(rem);          // 3..31
        const int eb = e + (31 - lz);       // biased exponent of that bit
        if (eb >= 1) {
            const unsigned mant = lz >= 8 ? rem << (lz - 8) : rem >> (8 - lz);
            lo = __uint_as_float(((unsigned)eb << 23) | (mant & 0x7FFFFFu));
        }
    }
    return make_float2(hi, (hw & 0x80000000u) ? -lo : lo);
}

__device__ __forceinline__ double ff_to_f64(float2 a) { return f64_from_f32(a.x) + f64_from_f32(a.y); }

// positive with a normal FP32 leading word (a usable pivot)
__device__ __forceinline__ bool ff_pivot_ok(float2 a) { return a.x >= 1.17549435e-38f && a.x < 3.0e38f; }

// 1/d for a positive pivot: the FP32 reciprocal q and one Newton step
// q + q (1 - d q), the residual 1 - d q formed from Dekker's exact product
// (relative error about 2^-46)
__device__ __forceinline__ float2 ff_recip(float2 d)
{
    const float q = __frcp_rn(d.x);
    const float p = __fmul_rn(d.x, q);
    float pe = __fmaf_rn(d.x, q, -p);
    pe = __fmaf_rn(d.y, q, pe);
    const float r = __fsub_rn(__fsub_rn(1.0f, p), pe);   // 1 - p is exact (p lies within 2^-23 of 1)
    return fast_two_sum(q, __fmul_rn(q, r));
}

// (i, j), i >= j, of the linear index u < 2^20 of a packed lower triangle,
// from the single-instruction approximate square root (no conversion
// instruction) and one integer correction each way
__device__ __forceinline__ void tri_decode_fast(int u, int &i, int &j)
{
    float f;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(f) : "f"(small_int_to_float(8 * u + 1)));
    int r = small_float_to_int(__fmul_rn(__fsub_rn(f, 1.0f), 0.5f));
    if ((r + 1) * (r + 2) / 2 <= u) r++;
    if (r * (r + 1) / 2 > u) r--;
    i = r;
    j = u - r * (r + 1) / 2;
}

// piece of s: floor((log2 s - log2_lo) / log2 r), clamped to the pieces, as
// the nearest integer of f + 1/2 minus one (the argument of the rounding
// stays >= 1/2; an f that is an exact integer may give the piece below, whose
// series the host check also covers: it reaches |t| = 1.02)
__device__ __forceinline__ int piece_of(const KernelSeries &ks, double s)
{
    const float f = fminf(fmaxf((__log2f(f32_from_f64(s)) - ks.log2_lo) * ks.inv_log2r, 0.0f), 64.0f);
    const int k = small_float_to_int(__fadd_rn(f, 0.5f)) - 1;
    return min(max(k, 0), ks.pieces - 1);
}

__device__ __forceinline__ double series_A(const KernelSeries &ks, double s)
{
    const int k = piece_of(ks, s);
    const double t = (s - ks.centre[k]) * ks.inv_w[k];
    double v = 0.0;
    if (ks.n64 <= ks.degree) {
        const float tf = f32_from_f64(t);
        const float *cf = ks.coef_f[k];
        float h = cf[ks.degree];
        for (int j = ks.degree - 1; j >= ks.n64; j--) h = fmaf(h, tf, cf[j]);
        v = f64_from_f32(h);
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

// Shared memory of one point group: fields at fixed offsets (in doubles)
// from one base; each accessor computes its address where it is used, so
// the group's sixteen arrays cost no registers between uses.
//   xi   [3][NC]  local coordinates
//   xf   [3][NC]  single-precision copy for the pivot search
//   C    [4][NC]  C[k][r]
//   Y    [4][NC]  A_rp then Y
//   v    [4][NC]  v[rhs][j] (original order); column buffers later
//   S    packed lower triangle of order NC: S, then 4 rhs rows (float-float
//        pairs in the refined solver)
//   M    [16] P_p^{-T}, row-major;  App [16];  red [4 * 16] partial sums of
//        the pivot values;  redv/redj [4 passes][16 warps] argmax values and
//        indices;  r2o [NC] rest index -> original index;  piv [16] pivot
//        block of the next elimination step
//   refined solver only: rhs [4][NC] reduced right-hand sides (FP64),
//        a [4][NC] solution a_r (FP64), ivs [NC] reciprocal pivots
struct PointSmem {
    double *base;
    int NC;
    __device__ __forceinline__ int64_t o_xf() const { return 3 * NC; }
    __device__ __forceinline__ int64_t o_C() const { return o_xf() + (3 * NC + 1) / 2; }
    __device__ __forceinline__ int64_t o_Y() const { return o_C() + 4 * NC; }
    __device__ __forceinline__ int64_t o_v() const { return o_Y() + 4 * NC; }
    __device__ __forceinline__ int64_t o_S() const { return o_v() + 4 * NC; }
    __device__ __forceinline__ int64_t o_M() const { return o_S() + (int64_t)NC * (NC + 1) / 2; }
    __device__ __forceinline__ double *xi() const { return base; }
    __device__ __forceinline__ float *xf() const { return (float *)(base + o_xf()); }
    __device__ __forceinline__ double *C() const { return base + o_C(); }
    __device__ __forceinline__ double *Y() const { return base + o_Y(); }
    __device__ __forceinline__ double *v() const { return base + o_v(); }
    __device__ __forceinline__ double *S() const { return base + o_S(); }
    __device__ __forceinline__ double *M() const { return base + o_M(); }
    __device__ __forceinline__ double *App() const { return base + o_M() + 16; }
    __device__ __forceinline__ double *red() const { return base + o_M() + 32; }
    __device__ __forceinline__ float *redv() const { return (float *)(base + o_M() + 96); }
    __device__ __forceinline__ int *redj() const { return (int *)(base + o_M() + 128); }
    __device__ __forceinline__ int *r2o() const { return (int *)(base + o_M() + 160); }
    __device__ __forceinline__ double *piv() const { return base + o_M() + 160 + (NC + 1) / 2; }
    __device__ __forceinline__ double *rhs() const { return piv() + 16; }
    __device__ __forceinline__ double *a() const { return rhs() + 4 * NC; }
    __device__ __forceinline__ float2 *ivs() const { return (float2 *)(a() + 4 * NC); }
};

// shared memory of one point group (doubles); the refined solver adds the
// FP64 right-hand sides and solution and the reciprocal pivots
__host__ __device__ inline int64_t point_smem_doubles(int NC, bool refine)
{
    return 3 * NC + (3 * NC + 1) / 2 + 4 * NC + 4 * NC + 4 * NC + (int64_t)NC * (NC + 1) / 2 + 32 + 64 + 32 + 32 +
           (NC + 1) / 2 + 16 + (refine ? 9 * NC : 0);
}

// global scratch of one point group in the refined solver: the FP64 reduced
// matrix S (packed lower triangle of order NC - 4)
__host__ __device__ inline int64_t point_scratch_doubles(int NC)
{
    return (int64_t)(NC - 4) * (NC - 3) / 2;
}

__device__ __forceinline__ PointSmem carve(double *base, int NC, bool)
{
    PointSmem w;
    w.base = base;
    w.NC = NC;
    return w;
}

struct ArgMax {
    float v;
    int j;
};

// named barrier over the `count` threads of one point group
__device__ __forceinline__ void group_sync(int bar, int count)
{
    asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(count) : "memory");
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

// Thread roles inside one point group of G warps.
struct Group {
    int GT, gt, lane, wig, G, bar;
};

// columns per elimination step
constexpr int kElimCols = 2;

// threads per block of the shape kernels: the FP64 solver runs up to 768
// (80 registers a thread: at 1024 threads and 64 registers it spilled inside
// the elimination, 1.3% slower on the layered slope, where the tuned shapes
// use at most 768 threads anyway); the float-float solver, whose long
// dependent FP32 chains need registers for overlap, up to 512 (128 registers)
constexpr int kShapeMaxThreads[2] = {768, 512};

// Arithmetic of the elimination: FP64, or float-float pairs.
struct F64Ops {
    typedef double T;
    static constexpr int kUnroll = 1;   // trailing-update entries interleaved per thread
    static __device__ __forceinline__ T zero() { return 0.0; }
    static __device__ __forceinline__ T mul(T a, T b) { return a * b; }
    static __device__ __forceinline__ T fnma(T x, T y, T c) { return fma(-x, y, c); }   // c - x y
    static __device__ __forceinline__ T inv_pivot(T d) { return positive_normal(d) ? recip_nr(d) : 0.0; }
    static __device__ __forceinline__ bool usable(T iv) { return iv > 0.0; }
};

struct FFOps {
    typedef float2 T;
    static constexpr int kUnroll = 2;
    static __device__ __forceinline__ T zero() { return make_float2(0.0f, 0.0f); }
    static __device__ __forceinline__ T mul(T a, T b) { return ff_mul(a, b); }
    static __device__ __forceinline__ T fnma(T x, T y, T c) { return ff_fnma(x, y, c); }
    static __device__ __forceinline__ T inv_pivot(T d) { return ff_pivot_ok(d) ? ff_recip(d) : zero(); }
    static __device__ __forceinline__ bool usable(T iv) { return iv.x > 0.0f; }
};

// Right-looking A = L D L' of the packed lower triangle A (order M2, in
// place), the first m columns, B columns per step:
//  - the B x B pivot block of the step is factored by one thread (lane 0 of
//    the group's first warp) at the end of the previous step: reciprocal
//    pivots piv[t] and the updated unscaled block entries piv[B + t(t-1)/2 + s]
//    (t > s);
//  - every row i below the block forms its B updated unscaled entries
//    (col[t][i]) and their scaled values L_{i,k+t} (one thread per row);
//  - every entry of the trailing triangle gets its B updates in one pass.
// Each value is the same sequence of multiply-adds as in the elimination one
// column at a time (same order), so B does not change the result; it divides
// the barriers and index decodes by B. col: B arrays of NC values. ivs
// (optional) receives 1/D of every column. Returns false (for the whole
// group) at a pivot that is not positive.
// The B x B pivot block of the step at column k (nb <= B columns) by one
// thread: reciprocal pivots piv[t] and updated unscaled entries
// piv[B + t(t-1)/2 + s] (t > s), each the multiply-add sequence of the
// column-at-a-time elimination. Not inlined: one thread runs it per step,
// and inlined its registers would be reserved by every thread.
template <class Ops, int B>
__device__ __noinline__ void pivot_block(const typename Ops::T *A, typename Ops::T *piv, int k, int nb)
{
    typedef typename Ops::T T;
    T iv[B];
#pragma unroll
    for (int t = 0; t < B; t++) {
        if (t < nb) {
            const int rt = (k + t) * (k + t + 1) / 2 + k;   // row k + t, column k
            T d = A[rt + t];
#pragma unroll
            for (int s = 0; s < B; s++) {
                if (s < t) {
                    // updated entry (k + t, k + s): the block's columns r < s first
                    T c = A[rt + s];
#pragma unroll
                    for (int r = 0; r < B; r++)
                        if (r < s) c = Ops::fnma(Ops::mul(piv[B + t * (t - 1) / 2 + r], iv[r]), piv[B + s * (s - 1) / 2 + r], c);
                    piv[B + t * (t - 1) / 2 + s] = c;
                    d = Ops::fnma(Ops::mul(c, iv[s]), c, d);
                }
            }
            iv[t] = Ops::inv_pivot(d);
            piv[t] = iv[t];
        }
    }
}

// Right-looking A = L D L' of the packed lower triangle A (order M2, in
// place), the first m columns, B columns per step:
//  - the B x B pivot block of the step is factored by one thread (lane 0 of
//    the group's first warp) at the end of the previous step (pivot_block);
//  - every row i below the block forms its B updated unscaled entries
//    (col[t][i]) and their scaled values L_{i,k+t} (one thread per row);
//  - every entry of the trailing triangle gets its B updates in one pass.
// Each value is the same sequence of multiply-adds as in the elimination one
// column at a time (same order), so B does not change the result; it divides
// the barriers and index decodes by B. col: B arrays of NC values. ivs
// (optional) receives 1/D of every column. Returns false (for the whole
// group) at a pivot that is not positive.
template <class Ops, int B>
__device__ __forceinline__ bool eliminate(typename Ops::T *A, typename Ops::T *col, int NC, typename Ops::T *piv,
                                          typename Ops::T *ivs, int m, int M2, const Group &gr)
{
    typedef typename Ops::T T;
    const int GT = gr.GT, gt = gr.gt, bar = gr.bar;
    if (gr.wig == 0 && gr.lane == 0) pivot_block<Ops, B>(A, piv, 0, min(B, m));
    group_sync(bar, GT);
    for (int k = 0; k < m; k += B) {
        const int nb = min(B, m - k);
        T iv[B];
        bool ok = true;
#pragma unroll
        for (int t = 0; t < B; t++) {
            iv[t] = t < nb ? piv[t] : Ops::zero();
            if (t < nb) ok &= Ops::usable(iv[t]);
        }
        if (!ok) return false;   // (every thread read the same pivots)
        if (ivs && gt == 0)
            for (int t = 0; t < nb; t++) ivs[k + t] = iv[t];
        // scale: rows i > k; a row inside the block has only the columns s < i - k
#pragma unroll 1
        for (int i = k + 1 + gt; i < M2; i += GT) {
            const int ik = i * (i + 1) / 2 + k;
            const int nt = min(nb, i - k);
            T l[B];
#pragma unroll
            for (int t = 0; t < B; t++) {
                if (t < nt) {
                    T a = A[ik + t];
#pragma unroll
                    for (int s = 0; s < B; s++)
                        if (s < t) a = Ops::fnma(l[s], piv[B + t * (t - 1) / 2 + s], a);
                    col[t * NC + i] = a;
                    l[t] = Ops::mul(a, iv[t]);
                    A[ik + t] = l[t];
                }
            }
        }
        group_sync(bar, GT);
        // trailing triangle: rows and columns >= k + nb
        const int k1 = k + nb, tk = M2 - k1, T2 = tk * (tk + 1) / 2;
#pragma unroll (Ops::kUnroll)
        for (int u = gt; u < T2; u += GT) {
            int ri, rj;
            tri_decode_fast(u, ri, rj);
            const int i = k1 + ri, j = k1 + rj, ib = i * (i + 1) / 2;
            T nv = A[ib + j];
#pragma unroll
            for (int t = 0; t < B; t++)
                if (t < nb) nv = Ops::fnma(A[ib + k + t], col[t * NC + j], nv);
            A[ib + j] = nv;
        }
        // the next pivot block: its entries (u < 10 above) were updated by
        // lanes of the first warp
        if (k1 < m && gr.wig == 0) {
            __syncwarp();
            if (gr.lane == 0) pivot_block<Ops, B>(A, piv, k1, min(B, m - k1));
        }
        group_sync(bar, GT);
    }
    return true;
}

// Shape functions of point p by one group (all G*32 threads of the group
// call it; the phases are separated by the group's named barrier).
//
// REFINE selects the solver of step 7 onwards: false factors S in FP64;
// true factors it in float-float arithmetic and recovers FP64 accuracy by
// one step of iterative refinement with the residual in FP64 (Sg: the
// group's global scratch, which holds S in FP64 for the residual).
template <bool REFINE>
__device__ __forceinline__ void shape_point(const int64_t p, const KernelSeries &ks, const PointSmem &W, const int NC,
                                            const Group &gr, const double *__restrict__ pts,
                                            const int32_t *__restrict__ inst_of, int shift,
                                            const InstGrid *__restrict__ ig, const int64_t *__restrict__ soff,
                                            const int32_t *__restrict__ sidx, const double *__restrict__ xyz,
                                            double *__restrict__ phi, double *__restrict__ Sg, DevError *err)
{
    const int GT = gr.GT, gt = gr.gt, lane = gr.lane, wig = gr.wig, G = gr.G, bar = gr.bar;
    const double c2 = ks.c2;
    const double inv_h = ig[instance_of(inst_of, shift, p)].inv_h;
    const int64_t base = soff[p];
    const int n = (int)(soff[p + 1] - base);
    if (n < 4 || n > NC) {
        if (gt == 0) dev_fail(err, RPIM_E_SUPPORT, p);
        return;
    }
    const int m = n - 4;
    const double gx = pts[3 * p], gy = pts[3 * p + 1], gz = pts[3 * p + 2];

    // 1. local coordinates (FP64) and a single-precision copy
    for (int j = gt; j < n; j += GT) {
        const int64_t J = sidx[base + j];
        const double a = (xyz[3 * J] - gx) * inv_h, b = (xyz[3 * J + 1] - gy) * inv_h,
                     c = (xyz[3 * J + 2] - gz) * inv_h;
        W.xi()[j] = a;
        W.xi()[NC + j] = b;
        W.xi()[2 * NC + j] = c;
        W.xf()[j] = f32_from_f64(a);
        W.xf()[NC + j] = f32_from_f64(b);
        W.xf()[2 * NC + j] = f32_from_f64(c);
    }
    group_sync(bar, GT);

    // 2. greedy pivot tetrahedron (single precision is enough to choose);
    //    each pass: warp argmax, then the group combines the G warps in
    //    order
    const float *X = W.xf(), *Yc = W.xf() + NC, *Z = W.xf() + 2 * NC;
    auto group_argmax = [&](float bv, int bj, int pass) {
        warp_argmax(bv, bj);
        if (lane == 0) {
            W.redv()[16 * pass + wig] = bv;
            W.redj()[16 * pass + wig] = bj;
        }
        group_sync(bar, GT);
        float v = W.redv()[16 * pass];
        int j = W.redj()[16 * pass];
        for (int w = 1; w < G; w++) {
            const float ov = W.redv()[16 * pass + w];
            const int oj = W.redj()[16 * pass + w];
            if (ov > v || (ov == v && oj < j)) { v = ov; j = oj; }
        }
        return ArgMax{v, j};
    };
    int p0, p1, p2, p3;
    {
        float bv = -INFINITY;
        int bj = 0x7fffffff;
        for (int j = gt; j < n; j += GT)
            if (-X[j] > bv) { bv = -X[j]; bj = j; }
        p0 = group_argmax(bv, bj, 0).j;
    }
    const float ax = X[p0], ay = Yc[p0], az = Z[p0];
    {
        float bv = -1.0f;
        int bj = 0x7fffffff;
        for (int j = gt; j < n; j += GT) {
            float dx = X[j] - ax, dy = Yc[j] - ay, dz = Z[j] - az;
            float d = dx * dx + dy * dy + dz * dz;
            if (d > bv) { bv = d; bj = j; }
        }
        p1 = group_argmax(bv, bj, 1).j;
    }
    const float ux = X[p1] - ax, uy = Yc[p1] - ay, uz = Z[p1] - az;
    {
        float bv = -1.0f;
        int bj = 0x7fffffff;
        for (int j = gt; j < n; j += GT) {
            float dx = X[j] - ax, dy = Yc[j] - ay, dz = Z[j] - az;
            float cx = dy * uz - dz * uy, cy = dz * ux - dx * uz, cz = dx * uy - dy * ux;
            float d = cx * cx + cy * cy + cz * cz;
            if (d > bv) { bv = d; bj = j; }
        }
        p2 = group_argmax(bv, bj, 2).j;
    }
    {
        const float vx = X[p2] - ax, vy = Yc[p2] - ay, vz = Z[p2] - az;
        const float nx = uy * vz - uz * vy, ny = uz * vx - ux * vz, nz = ux * vy - uy * vx;
        float bv = -1.0f;
        int bj = 0x7fffffff;
        for (int j = gt; j < n; j += GT) {
            float d = fabsf((X[j] - ax) * nx + (Yc[j] - ay) * ny + (Z[j] - az) * nz);
            if (d > bv) { bv = d; bj = j; }
        }
        auto r = group_argmax(bv, bj, 3);
        p3 = r.j;
        const float ulen2 = ux * ux + uy * uy + uz * uz;
        if (!(r.v > 1e-5f * ulen2 * sqrtf(ulen2))) {
            if (gt == 0) dev_fail(err, RPIM_E_SINGULAR, p);
            group_sync(bar, GT);
            return;
        }
    }
    // rest ordering: original order without the pivots
    for (int j = gt; j < n; j += GT) {
        int less = (p0 < j) + (p1 < j) + (p2 < j) + (p3 < j);
        bool isp = j == p0 || j == p1 || j == p2 || j == p3;
        if (!isp) W.r2o()[j - less] = j;
    }
    auto pivot = [&](int k) { return k == 0 ? p0 : k == 1 ? p1 : k == 2 ? p2 : p3; };

    // 3. M = P_p^{-T} = cofactor matrix / det, one cofactor per lane 0..15
    //    of the group's first warp
    if (wig == 0) {
        const int ri = (lane >> 2) & 3, cj = lane & 3;
        double e[3][3];
        int rr = 0;
        for (int r = 0; r < 4; r++) {
            if (r == ri) continue;
            const int pr = pivot(r);
            const double row[4] = {1.0, W.xi()[pr], W.xi()[NC + pr], W.xi()[2 * NC + pr]};
            int cc = 0;
            for (int c = 0; c < 4; c++)
                if (c != cj) e[rr][cc++] = row[c];
            rr++;
        }
        double cof = det3(e[0][0], e[0][1], e[0][2], e[1][0], e[1][1], e[1][2], e[2][0], e[2][1], e[2][2]);
        if ((ri + cj) & 1) cof = -cof;
        const double prow = cj == 0 ? 1.0 : W.xi()[(cj - 1) * NC + p0];
        double part = lane < 4 ? prow * cof : 0.0;
        part += __shfl_xor_sync(0xffffffffu, part, 1);
        part += __shfl_xor_sync(0xffffffffu, part, 2);
        const double det = __shfl_sync(0xffffffffu, part, 0);
        const double idet = recip_nr(det);
        if (lane < 16) W.M()[lane] = cof * idet;
    }
    group_sync(bar, GT);

    // 4. A_pp, C and A_rp
    if (gt < 16) {
        const int a = gt >> 2, b = gt & 3;
        const int ia = pivot(a), ib = pivot(b);
        double val = ks.diag;
        if (a != b) {
            double dx = W.xi()[ia] - W.xi()[ib], dy = W.xi()[NC + ia] - W.xi()[NC + ib], dz = W.xi()[2 * NC + ia] - W.xi()[2 * NC + ib];
            val = series_A(ks, fma(dz, dz, fma(dy, dy, fma(dx, dx, c2))));
        }
        W.App()[gt] = val;
    }
    for (int t = gt; t < 4 * m; t += GT) {
        const int r = t >> 2, k = t & 3;
        const int j = W.r2o()[r];
        const double x0 = W.xi()[j], x1 = W.xi()[NC + j], x2 = W.xi()[2 * NC + j];
        W.C()[k * NC + r] = fma(W.M()[4 * k + 3], x2, fma(W.M()[4 * k + 2], x1, fma(W.M()[4 * k + 1], x0, W.M()[4 * k])));
        const int ik = pivot(k);
        double dx = x0 - W.xi()[ik], dy = x1 - W.xi()[NC + ik], dz = x2 - W.xi()[2 * NC + ik];
        W.Y()[k * NC + r] = series_A(ks, fma(dz, dz, fma(dy, dy, fma(dx, dx, c2))));
    }
    group_sync(bar, GT);

    // 5. right-hand sides v = r - A_:p d  (d = columns of M), all nodes
    for (int j = gt; j < n; j += GT) {
        const double x0 = W.xi()[j], x1 = W.xi()[NC + j], x2 = W.xi()[2 * NC + j];
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
            for (int k = 0; k < 4; k++) Ajp[k] = W.App()[4 * kp + k];
        } else {
            const int r = j - (p0 < j) - (p1 < j) - (p2 < j) - (p3 < j);
#pragma unroll
            for (int k = 0; k < 4; k++) Ajp[k] = W.Y()[k * NC + r];
        }
#pragma unroll
        for (int q = 0; q < 4; q++) {
            double acc = rr[q];
#pragma unroll
            for (int k = 0; k < 4; k++) acc = fma(-Ajp[k], W.M()[4 * k + q], acc);
            W.v()[q * NC + j] = acc;
        }
    }
    group_sync(bar, GT);
    // Y = A_rp - C' A_pp / 2
    for (int t = gt; t < 4 * m; t += GT) {
        const int r = t >> 2, k = t & 3;
        double acc = 0.0;
#pragma unroll
        for (int s2 = 0; s2 < 4; s2++) acc = fma(W.C()[s2 * NC + r], W.App()[4 * s2 + k], acc);
        W.Y()[k * NC + r] = fma(-0.5, acc, W.Y()[k * NC + r]);  // each thread owns its element
    }
    group_sync(bar, GT);

    // 6. S = A_rr - Y C - C' Y' (packed lower triangle, rows 0..m-1),
    //    then the reduced right-hand sides as rows m..m+3 (entries
    //    j < m), so that the elimination below also performs the
    //    forward substitution. The refined solver keeps S and the
    //    right-hand sides in FP64 as well (S in the group's global scratch,
    //    which stays in L2) for the residual of step 8.
    float2 *SF = (float2 *)W.S();     // the triangle as float-float pairs (refined solver)
    float2 *PF = (float2 *)W.piv();   // reciprocal of the next pivot (refined solver)
    {
        const int T = m * (m + 1) / 2;
        for (int u = gt; u < T; u += GT) {
            int i, j;
            tri_decode_fast(u, i, j);
            const int oi = W.r2o()[i], oj = W.r2o()[j];
            double a;
            if (i == j) {
                a = ks.diag;
            } else {
                double dx = W.xi()[oi] - W.xi()[oj], dy = W.xi()[NC + oi] - W.xi()[NC + oj], dz = W.xi()[2 * NC + oi] - W.xi()[2 * NC + oj];
                a = series_A(ks, fma(dz, dz, fma(dy, dy, fma(dx, dx, c2))));
            }
#pragma unroll
            for (int k = 0; k < 4; k++) {
                a = fma(-W.Y()[k * NC + i], W.C()[k * NC + j], a);
                a = fma(-W.C()[k * NC + i], W.Y()[k * NC + j], a);
            }
            if constexpr (REFINE) {
                Sg[u] = a;
                SF[u] = ff_from_f64(a);
            } else {
                W.S()[u] = a;
            }
        }
    }
    for (int t = gt; t < 4 * (m + 4); t += GT) {
        const int q = t / (m + 4), r = t - q * (m + 4);
        double acc = 0.0;
        if (r < m) {
            const int j = W.r2o()[r];
            acc = W.v()[q * NC + j];
#pragma unroll
            for (int k = 0; k < 4; k++) acc = fma(-W.C()[k * NC + r], W.v()[q * NC + pivot(k)], acc);
        }
        if constexpr (REFINE) {
            if (r < m) W.rhs()[q * NC + r] = acc;
            if (r <= m + q) SF[(m + q) * (m + q + 1) / 2 + r] = ff_from_f64(acc);
        } else {
            if (r <= m + q) W.S()[(m + q) * (m + q + 1) / 2 + r] = acc;
        }
    }
    group_sync(bar, GT);

    // 7. S = L D L' (right-looking, packed, in place) on the order-(m+4)
    //    triangle, kElimCols columns per step; W.v() holds the unscaled
    //    columns of the current step. After the last step the rhs rows hold
    //    z = D^-1 L^-1 rhs. The reciprocal pivots are computed once per
    //    step, by one thread, and read from shared memory by the group:
    //    replicated in every warp they would cost each warp a full FP64
    //    issue slot per instruction.
    const int M2 = m + 4;
    bool ok;
    if constexpr (REFINE)
        ok = eliminate<FFOps, kElimCols>(SF, (float2 *)W.v(), NC, PF, W.ivs(), m, M2, gr);
    else
        ok = eliminate<F64Ops, kElimCols>(W.S(), W.v(), NC, W.piv(), nullptr, m, M2, gr);
    if (!ok) {
        if (gt == 0) dev_fail(err, RPIM_E_SINGULAR, p);
        group_sync(bar, GT);
        return;
    }

    // 8. L' a = z, column by column; threads over (row, rhs) pairs
    double *Z0 = W.S() + (size_t)m * (m + 1) / 2;  // rhs row q starts at Z0 + q*m + q*(q+1)/2
    if constexpr (REFINE) {
        float2 *Z0f = SF + (size_t)m * (m + 1) / 2;
        for (int k = m - 1; k > 0; k--) {
            const int kb = k * (k + 1) / 2;
            for (int t = gt; t < 4 * k; t += GT) {
                const int q = t & 3, i = t >> 2;
                float2 *zq = Z0f + q * m + q * (q + 1) / 2;
                zq[i] = ff_fnma(SF[kb + i], zq[k], zq[i]);
            }
            group_sync(bar, GT);
        }
        for (int t = gt; t < 4 * m; t += GT) {
            const int q = t & 3, i = t >> 2;
            W.a()[q * NC + i] = ff_to_f64(Z0f[q * m + q * (q + 1) / 2 + i]);
        }
        group_sync(bar, GT);
        //    One step of iterative refinement: the residual rhs - S a in
        //    FP64 (one thread per row, ascending column order), then the
        //    correction from the float-float factors (L y = r, D z = y,
        //    L' e = z) added to a in FP64.
        float2 *R = (float2 *)W.v();   // [4][NC]
        for (int i = gt; i < m; i += GT) {
            double r0 = W.rhs()[i], r1 = W.rhs()[NC + i], r2 = W.rhs()[2 * NC + i], r3 = W.rhs()[3 * NC + i];
            // row i of S: (i, j) for j <= i, then (j, i) for j > i (not
            // unrolled: unrolling spills the kernel's registers)
            const double *srow = Sg + i * (i + 1) / 2;
#pragma unroll 1
            for (int j = 0; j <= i; j++) {
                const double sv = srow[j];
                r0 = fma(-sv, W.a()[j], r0);
                r1 = fma(-sv, W.a()[NC + j], r1);
                r2 = fma(-sv, W.a()[2 * NC + j], r2);
                r3 = fma(-sv, W.a()[3 * NC + j], r3);
            }
            int pos = (i + 1) * (i + 2) / 2 + i;   // (i + 1, i)
#pragma unroll 1
            for (int j = i + 1; j < m; j++) {
                const double sv = Sg[pos];
                pos += j + 1;
                r0 = fma(-sv, W.a()[j], r0);
                r1 = fma(-sv, W.a()[NC + j], r1);
                r2 = fma(-sv, W.a()[2 * NC + j], r2);
                r3 = fma(-sv, W.a()[3 * NC + j], r3);
            }
            R[i] = ff_from_f64(r0);
            R[NC + i] = ff_from_f64(r1);
            R[2 * NC + i] = ff_from_f64(r2);
            R[3 * NC + i] = ff_from_f64(r3);
        }
        group_sync(bar, GT);
        for (int k = 0; k + 1 < m; k++) {
            for (int t = gt; t < 4 * (m - 1 - k); t += GT) {
                const int q = t & 3, i = k + 1 + (t >> 2);
                R[q * NC + i] = ff_fnma(SF[i * (i + 1) / 2 + k], R[q * NC + k], R[q * NC + i]);
            }
            group_sync(bar, GT);
        }
        for (int t = gt; t < 4 * m; t += GT) {
            const int q = t & 3, i = t >> 2;
            R[q * NC + i] = ff_mul(R[q * NC + i], W.ivs()[i]);
        }
        group_sync(bar, GT);
        for (int k = m - 1; k > 0; k--) {
            const int kb = k * (k + 1) / 2;
            for (int t = gt; t < 4 * k; t += GT) {
                const int q = t & 3, i = t >> 2;
                R[q * NC + i] = ff_fnma(SF[kb + i], R[q * NC + k], R[q * NC + i]);
            }
            group_sync(bar, GT);
        }
        for (int t = gt; t < 4 * m; t += GT) {
            const int q = t & 3, i = t >> 2;
            W.a()[q * NC + i] += ff_to_f64(R[q * NC + i]);
        }
        group_sync(bar, GT);
    } else {
        for (int k = m - 1; k > 0; k--) {
            const int kb = k * (k + 1) / 2;
            for (int t = gt; t < 4 * k; t += GT) {
                const int q = t & 3, i = t >> 2;
                double *zq = Z0 + q * m + q * (q + 1) / 2;
                zq[i] = fma(-W.S()[kb + i], zq[k], zq[i]);
            }
            group_sync(bar, GT);
        }
    }
    // a_r of right-hand side q (r < m)
    auto ar_of = [&](int q, int r) -> double {
        if constexpr (REFINE) return W.a()[q * NC + r];
        else return Z0[q * m + q * (q + 1) / 2 + r];
    };

    // 9. pivot values a_p = d - C a_r: 16 sums over the rest rows, by the
    //    group's first warp alone (lane-strided partial sums, then
    //    reduce-scattered so that lane l ends with sum l >> 1). The
    //    summation order is therefore the same for every group width G,
    //    and the other warps issue no FP64 work here.
    if (wig == 0) {
        double v[16];
#pragma unroll
        for (int k = 0; k < 16; k++) v[k] = 0.0;
        for (int r = lane; r < m; r += 32) {
            double ar[4];
#pragma unroll
            for (int q = 0; q < 4; q++) ar[q] = ar_of(q, r);
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const double c = W.C()[k * NC + r];
#pragma unroll
                for (int q = 0; q < 4; q++) v[4 * k + q] = fma(c, ar[q], v[4 * k + q]);
            }
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
        if ((lane & 1) == 0) W.red()[lane >> 1] = v[0];
    }

    double *out = phi + 4 * base;
    bool finite = true;
    for (int r = gt; r < m; r += GT) {
        const int j = W.r2o()[r];
        double2 lo2 = make_double2(ar_of(0, r), ar_of(1, r) * inv_h);
        double2 hi2 = make_double2(ar_of(2, r) * inv_h, ar_of(3, r) * inv_h);
        finite &= isfinite(lo2.x) && isfinite(lo2.y) && isfinite(hi2.x) && isfinite(hi2.y);
        *(double2 *)(out + 4 * j) = lo2;
        *(double2 *)(out + 4 * j + 2) = hi2;
    }
    group_sync(bar, GT);
    if (gt < 16) {
        const int k = gt >> 2, q = gt & 3;
        double val = W.M()[4 * k + q] - W.red()[gt];
        if (q) val *= inv_h;
        finite &= isfinite(val);
        out[4 * pivot(k) + q] = val;
    }
    if (!__all_sync(0xffffffffu, finite) && lane == 0) dev_fail(err, RPIM_E_NONFINITE, p);
    group_sync(bar, GT);
}

// recip_nr over an array (the accuracy probe of rpim_probe_recip)
__global__ void recip_probe_kernel(int64_t n, const double *__restrict__ d, double *__restrict__ r)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        r[i] = recip_nr(d[i]);
}

// One group of G warps per point. Every loop below is a flattened parallel
// loop over the group's G*32 threads; the phases are separated by a named
// barrier of the group. Groups of one block are independent.
// scratch: the refined solver's FP64 copy of S, point_scratch_doubles(NC)
// per point group, group g of block b at (b * ppb + g) (unused otherwise;
// every block of this kernel works with the same NC and ppb).
template <bool REFINE>
__global__ void __launch_bounds__(kShapeMaxThreads[REFINE]) shape_kernel(int64_t n_pts, const double *__restrict__ pts,
                                                     const int32_t *__restrict__ inst_of, int shift,
                                                     const InstGrid *__restrict__ ig,
                                                     const int32_t *__restrict__ order,
                                                     const int64_t *__restrict__ soff,
                                                     const int32_t *__restrict__ sidx,
                                                     const double *__restrict__ xyz,
                                                     const KernelSeries *__restrict__ ks_g,
                                                     double *__restrict__ phi, int NC, int G,
                                                     double *__restrict__ scratch, DevError *err)
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
    const int GT = G * 32;
    const int grp = threadIdx.x / GT, gt = threadIdx.x - grp * GT;
    const int lane = threadIdx.x & 31, wig = gt >> 5;
    const int ppb = blockDim.x / GT;
    const int bar = 1 + grp;
    PointSmem W = carve(dsm + (size_t)grp * point_smem_doubles(NC, REFINE), NC, REFINE);
    double *Sg = REFINE ? scratch + ((size_t)blockIdx.x * ppb + grp) * point_scratch_doubles(NC) : nullptr;
    const int64_t stride = (int64_t)gridDim.x * ppb;

    const Group gr{GT, gt, lane, wig, G, bar};
    for (int64_t pk = (int64_t)blockIdx.x * ppb + grp; pk < n_pts; pk += stride) {
        const int64_t p = order ? (int64_t)order[pk] : pk;
        shape_point<REFINE>(p, ks, W, NC, gr, pts, inst_of, shift, ig, soff, sidx, xyz, phi, Sg, err);
    }
}

// Work plan of the persistent shape kernel: the support-size buckets, largest
// supports first, each with its launch shape (ppb groups of G warps per block,
// NC-sized point buffers) and its slice [start, start + count) of the point
// order.
constexpr int kMaxTileBuckets = 32;
struct BucketPlan {
    int nb;
    int pad;
    long long total;                       // points of all buckets
    long long block_scratch;               // refined solver: scratch doubles of one block (largest bucket)
    int NC[kMaxTileBuckets], G[kMaxTileBuckets], ppb[kMaxTileBuckets];
    long long start[kMaxTileBuckets];      // first position of the bucket in the order list
    long long count[kMaxTileBuckets];      // points of the bucket
};

// Persistent shape kernel: one launch over a (bucket, point) work list. The
// blocks walk the buckets in the plan's order; for each bucket a block lays
// its shared memory out for that bucket's launch shape, and each of its
// point groups takes the bucket's next point from a device counter until the
// bucket is exhausted, independently of the other groups (no block-wide
// wait per point). A block-wide barrier separates buckets, since group roles
// and buffers change between them. Every value is computed by the same
// thread-level formula as in shape_kernel, whatever the launch shape, so the
// results are bitwise those of the per-bucket launches.
template <bool REFINE>
__global__ void __launch_bounds__(kShapeMaxThreads[REFINE]) shape_tiles_kernel(const BucketPlan plan, unsigned long long *counters,
                                                           const double *__restrict__ pts,
                                                           const int32_t *__restrict__ inst_of, int shift,
                                                           const InstGrid *__restrict__ ig,
                                                           const int32_t *__restrict__ order,
                                                           const int64_t *__restrict__ soff,
                                                           const int32_t *__restrict__ sidx,
                                                           const double *__restrict__ xyz,
                                                           const KernelSeries *__restrict__ ks_g,
                                                           double *__restrict__ phi, double *__restrict__ scratch,
                                                           DevError *err)
{
    extern __shared__ double dsm[];
    __shared__ KernelSeries ks;
    __shared__ long long s_next[32];
    {
        const int nw = sizeof(KernelSeries) / sizeof(int);
        const int *src = (const int *)ks_g;
        int *dst = (int *)&ks;
        for (int i = threadIdx.x; i < nw; i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    // every block owns one fixed region of the scratch, sized for its largest
    // bucket (blocks work on different buckets at the same time)
    for (int b = 0; b < plan.nb; b++) {
        const int G = plan.G[b], ppb = plan.ppb[b], NC = plan.NC[b];
        const int GT = G * 32;
        const int grp = threadIdx.x / GT;
        if (grp < ppb) {
            const int gt = threadIdx.x - grp * GT;
            const Group gr{GT, gt, lane, gt >> 5, G, 1 + grp};
            const PointSmem W = carve(dsm + (size_t)grp * point_smem_doubles(NC, REFINE), NC, REFINE);
            double *Sg = REFINE ? scratch + (size_t)blockIdx.x * plan.block_scratch +
                                      (size_t)grp * point_scratch_doubles(NC)
                                : nullptr;
            for (;;) {
                if (gt == 0) s_next[grp] = (long long)atomicAdd(&counters[b], 1ull);
                group_sync(1 + grp, GT);
                const long long pk = s_next[grp];
                group_sync(1 + grp, GT);   // every thread holds pk before the next fetch
                if (pk >= plan.count[b]) break;
                const int64_t p = (int64_t)order[plan.start[b] + pk];
                shape_point<REFINE>(p, ks, W, NC, gr, pts, inst_of, shift, ig, soff, sidx, xyz, phi, Sg, err);
            }
        }
        __syncthreads();
    }
}

// Launch shape of the shape kernel for supports up to NC: ppb point groups
// of G warps per block. The results do not depend on it (every value is
// computed by one thread with a fixed formula, the argmax passes break ties
// by index, and the one reduction runs in the first warp alone), so it is a
// pure speed choice: a default rule, or what rpim_autotune_shape measured.
struct ShapeCfg {
    int ppb = 0, G = 0;
};

static std::mutex g_tune_mu;
static ShapeCfg g_tuned[2][RPIM_MAX_SUPPORT + 1];   // per solver

static std::atomic<int> g_solver{RPIM_SOLVER_FP64};

static bool refined() { return g_solver.load() == RPIM_SOLVER_REFINED; }

// (every host path reads the solver once and passes it down, so that the
// shared memory it sizes and the kernel it launches always agree)
static size_t point_bytes(int NC, bool ref) { return (size_t)point_smem_doubles(NC, ref) * sizeof(double); }

constexpr size_t kShapeSmemBudget = 216 * 1024;
constexpr int kMaxGroupWarps = 16;   // warps per point group (argmax buffers hold 16)

static bool cfg_valid(int NC, ShapeCfg c, bool ref)
{
    return c.G >= 1 && c.G <= kMaxGroupWarps && c.ppb >= 1 && c.ppb <= 15 && c.ppb * c.G * 32 <= kShapeMaxThreads[ref] &&
           (size_t)c.ppb * point_bytes(NC, ref) <= kShapeSmemBudget;
}

static ShapeCfg default_cfg(int NC, bool ref)
{
    ShapeCfg c;
    c.ppb = (int)std::min<size_t>(15, kShapeSmemBudget / point_bytes(NC, ref));  // points (groups) per block
    // warps per point: about 24 warps per block, at most 8 per point (the
    // launch shapes the autotuner picked on supports of 40-130 nodes)
    c.G = std::max(1, std::min(8, (ref ? 12 : 24) / std::max(1, c.ppb)));
    return c;
}

static ShapeCfg shape_cfg(int NC, bool ref)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const ShapeCfg t = g_tuned[ref][std::min(NC, RPIM_MAX_SUPPORT)];
    return cfg_valid(NC, t, ref) ? t : default_cfg(NC, ref);
}

static rpim_status launch_shape(rpim_pattern *p, int64_t n_pts, const double *pts, const int32_t *inst_of, int shift,
                                const int32_t *order, const int64_t *soff, const int32_t *sidx, int NC, ShapeCfg c,
                                bool ref, double *phi, cudaStream_t s, const char *tag)
{
    const size_t smem = (size_t)c.ppb * point_bytes(NC, ref);
    int64_t blocks = std::min<int64_t>((int64_t)p->sm_count, (n_pts + c.ppb - 1) / c.ppb);
    if (blocks < 1) blocks = 1;
    if (ref) {
        if (blocks * c.ppb * point_scratch_doubles(NC) > p->shape_scratch_doubles)
            return fail(RPIM_E_ARG, "shape scratch too small for the launch");
        RPIM_CUDA(cudaFuncSetAttribute(shape_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        launch(tag, shape_kernel<true>, (unsigned)blocks, c.ppb * c.G * 32, smem, s, n_pts, pts, inst_of, shift,
               (const InstGrid *)p->ig, order, soff, sidx, (const double *)p->xyz, (const KernelSeries *)p->series,
               phi, NC, c.G, p->shape_scratch, p->err);
    } else {
        RPIM_CUDA(cudaFuncSetAttribute(shape_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        launch(tag, shape_kernel<false>, (unsigned)blocks, c.ppb * c.G * 32, smem, s, n_pts, pts, inst_of, shift,
               (const InstGrid *)p->ig, order, soff, sidx, (const double *)p->xyz, (const KernelSeries *)p->series,
               phi, NC, c.G, (double *)nullptr, p->err);
    }
    RPIM_CUDA(cudaGetLastError());
    return RPIM_OK;
}

rpim_status shape_functions(rpim_pattern *p, int64_t n_pts, const double *pts, const int32_t *inst_of, int shift,
                            const int32_t *order, const int64_t *soff, const int32_t *sidx, int32_t max_n,
                            double *phi, cudaStream_t s, const char *tag)
{
    if (n_pts == 0) return RPIM_OK;
    if (max_n > RPIM_MAX_SUPPORT) return fail(RPIM_E_SUPPORT, "support larger than RPIM_MAX_SUPPORT");
    if (p->shape_kind != RPIM_SHAPE_RPIM)   // MLS or Shepard
        return mls_shape_functions(p, n_pts, pts, inst_of, shift, order, soff, sidx, phi, s, tag);
    const int NC = std::max(8, (int)max_n);
    const bool ref = refined();
    if (point_bytes(NC, ref) > kShapeSmemBudget) return fail(RPIM_E_SUPPORT, "support too large for shared memory");
    return launch_shape(p, n_pts, pts, inst_of, shift, order, soff, sidx, NC, shape_cfg(NC, ref), ref, phi, s, tag);
}

static std::atomic<int> g_persistent{1};

static rpim_status shape_functions_buckets(rpim_pattern *p, double *phi, cudaStream_t s)
{
    int64_t start = 0;
    for (size_t b = 0; b < p->bucket_count.size(); b++) {
        const int64_t cnt = p->bucket_count[b];
        if (cnt > 0)
            RPIM_CHECK(shape_functions(p, cnt, p->pts, p->node_inst, 3, p->bucket_order + start, p->soff, p->sidx,
                                       p->bucket_nc[b], phi, s, "shape"));
        start += cnt;
    }
    return RPIM_OK;
}

// Plan of the persistent launch over the pattern's buckets (a sample of
// `frac` of every bucket when tuning). Returns the shared memory and threads
// per block and the largest number of blocks with work.
static rpim_status bucket_plan(const rpim_pattern *p, double frac, bool ref, BucketPlan *plan, size_t *smem_out,
                               int *threads_out, int64_t *blocks_out)
{
    *plan = BucketPlan{};
    struct B { int NC; ShapeCfg c; int64_t start, count; };
    std::vector<B> bs;
    int64_t start = 0;
    for (size_t b = 0; b < p->bucket_count.size(); b++) {
        const int64_t full = p->bucket_count[b];
        const int64_t cnt = frac >= 1.0 ? full : std::min<int64_t>(full, (int64_t)(full * frac) + 1);
        if (cnt > 0) {
            if (p->bucket_nc[b] > RPIM_MAX_SUPPORT) return fail(RPIM_E_SUPPORT, "support larger than RPIM_MAX_SUPPORT");
            const int NC = std::max(8, (int)p->bucket_nc[b]);
            if (point_bytes(NC, ref) > kShapeSmemBudget) return fail(RPIM_E_SUPPORT, "support too large for shared memory");
            bs.push_back(B{NC, shape_cfg(NC, ref), start, cnt});
        }
        start += full;
    }
    if ((int)bs.size() > kMaxTileBuckets) return fail(RPIM_E_ARG, "too many support-size buckets");
    std::stable_sort(bs.begin(), bs.end(), [](const B &a, const B &b) { return a.NC > b.NC; });
    size_t smem = 0;
    int threads = 32;
    int64_t blocks = 1;
    plan->nb = (int)bs.size();
    for (int b = 0; b < plan->nb; b++) {
        plan->NC[b] = bs[b].NC;
        plan->G[b] = bs[b].c.G;
        plan->ppb[b] = bs[b].c.ppb;
        plan->start[b] = bs[b].start;
        plan->count[b] = bs[b].count;
        plan->total += bs[b].count;
        smem = std::max(smem, (size_t)bs[b].c.ppb * point_bytes(bs[b].NC, ref));
        plan->block_scratch = std::max<long long>(plan->block_scratch, (long long)bs[b].c.ppb * point_scratch_doubles(bs[b].NC));
        threads = std::max(threads, bs[b].c.ppb * bs[b].c.G * 32);
        blocks = std::max<int64_t>(blocks, (bs[b].count + bs[b].c.ppb - 1) / bs[b].c.ppb);
    }
    *smem_out = smem;
    *threads_out = threads;
    *blocks_out = blocks;
    return RPIM_OK;
}

static rpim_status shape_functions_tiles(rpim_pattern *p, double *phi, cudaStream_t s, double frac = 1.0)
{
    BucketPlan plan;
    size_t smem = 0;
    int threads = 0;
    int64_t need = 0;
    const bool ref = refined();
    RPIM_CHECK(bucket_plan(p, frac, ref, &plan, &smem, &threads, &need));
    if (plan.total == 0) return RPIM_OK;
    if (!p->tile_counter) RPIM_CHECK(dalloc(&p->tile_counter, kMaxTileBuckets, s));
    RPIM_CUDA(cudaMemsetAsync(p->tile_counter, 0, kMaxTileBuckets * sizeof(unsigned long long), s));
    auto kern = ref ? shape_tiles_kernel<true> : shape_tiles_kernel<false>;
    RPIM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    RPIM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((int64_t)p->sm_count * std::max(1, per_sm), need));
    if (ref && blocks * plan.block_scratch > p->shape_scratch_doubles)
        return fail(RPIM_E_ARG, "shape scratch too small for the launch");
    launch("shape", kern, (unsigned)blocks, threads, smem, s, plan, p->tile_counter, (const double *)p->pts,
           (const int32_t *)p->node_inst, 3, (const InstGrid *)p->ig, (const int32_t *)p->bucket_order,
           (const int64_t *)p->soff, (const int32_t *)p->sidx, (const double *)p->xyz,
           (const KernelSeries *)p->series, phi, ref ? p->shape_scratch : (double *)nullptr, p->err);
    RPIM_CUDA(cudaGetLastError());
    return RPIM_OK;
}

// Everything that decides what shape_functions_all launches for a pattern
// (kind, schedule, the tile plan with its tuned launch shapes): a captured
// assembly graph stays valid while this key is unchanged.
rpim_status shape_launch_key(const rpim_pattern *p, std::vector<unsigned char> *key)
{
    key->clear();
    auto put = [&](const void *a, size_t n) {
        const unsigned char *c = (const unsigned char *)a;
        key->insert(key->end(), c, c + n);
    };
    const int kind = p->shape_kind, sched = g_persistent.load(), solver = g_solver.load();
    put(&kind, sizeof kind);
    put(&sched, sizeof sched);
    put(&solver, sizeof solver);
    if (kind == RPIM_SHAPE_RPIM) {
        if (sched) {
            BucketPlan plan;
            size_t smem = 0;
            int threads = 0;
            int64_t blocks = 0;
            RPIM_CHECK(bucket_plan(p, 1.0, solver == RPIM_SOLVER_REFINED, &plan, &smem, &threads, &blocks));
            put(&plan, sizeof plan);
        } else {
            for (size_t b = 0; b < p->bucket_count.size(); b++) {
                const int NC = std::max(8, (int)p->bucket_nc[b]);
                const ShapeCfg c = shape_cfg(NC, solver == RPIM_SOLVER_REFINED);
                put(&p->bucket_count[b], sizeof(int64_t));
                put(&NC, sizeof NC);
                put(&c, sizeof c);
            }
        }
    }
    return RPIM_OK;
}

rpim_status shape_functions_all(rpim_pattern *p, double *phi, cudaStream_t s)
{
    // MLS and Shepard: one launch over all points in their natural order (the
    // eight points of a cell, which share most of their support, run side by
    // side)
    if (p->shape_kind != RPIM_SHAPE_RPIM)
        return mls_shape_functions(p, p->n_points, p->pts, p->node_inst, 3, nullptr, p->soff, p->sidx, phi, s,
                                   p->shape_kind == RPIM_SHAPE_MLS ? "mls_shape" : "shepard_shape");
    return g_persistent.load() ? shape_functions_tiles(p, phi, s) : shape_functions_buckets(p, phi, s);
}

} // namespace rpim

using namespace rpim;

extern "C" rpim_status rpim_autotune_shape(rpim_pattern *p, int64_t max_points, int32_t *table, int32_t *n_table,
                                           rpim_stream_t stream)
{
    RPIM_STAGE("rpim_autotune_shape");
    if (!p || max_points < 1) return fail(RPIM_E_ARG, "bad argument");
    if (p->shape_kind != RPIM_SHAPE_RPIM) {   // only the RPIM kernel has launch shapes to tune
        if (n_table) *n_table = 0;
        return RPIM_OK;
    }
    cudaStream_t s = (cudaStream_t)stream;
    p->stream = s;
    if (!p->phi) RPIM_CHECK(dalloc(&p->phi, 4 * p->n_entries, s));
    cudaEvent_t e0, e1;
    RPIM_CUDA(cudaEventCreate(&e0));
    RPIM_CUDA(cudaEventCreate(&e1));
    int nt = 0;
    int64_t start = 0;
    rpim_status st = RPIM_OK;
    const bool ref = refined();
    for (size_t bk = 0; bk < p->bucket_count.size() && st == RPIM_OK; bk++) {
        const int64_t cnt = std::min<int64_t>(p->bucket_count[bk], max_points);
        const int NC = std::max(8, (int)p->bucket_nc[bk]);
        const int32_t *order = p->bucket_order + start;
        start += p->bucket_count[bk];
        if (cnt == 0 || point_bytes(NC, ref) > kShapeSmemBudget) continue;
        ShapeCfg best = default_cfg(NC, ref);
        float best_ms = 1e30f;
        for (int G : {1, 2, 3, 4, 6, 8, 12, 16})
            for (int ppb = 1; ppb <= 15 && st == RPIM_OK; ppb++) {
                const ShapeCfg c{ppb, G};
                if (!cfg_valid(NC, c, ref)) continue;
                // skip launch shapes that cannot fill the SMs' warp slots
                if (ppb * G < 4 && !(ppb == default_cfg(NC, ref).ppb && G == default_cfg(NC, ref).G)) continue;
                float ms = 1e30f;
                for (int rep = 0; rep < 3 && st == RPIM_OK; rep++) {
                    if (cudaEventRecord(e0, s) != cudaSuccess) { st = fail(RPIM_E_CUDA, "tune: event"); break; }
                    st = launch_shape(p, cnt, p->pts, p->node_inst, 3, order, p->soff, p->sidx, NC, c, ref, p->phi, s,
                                      "tune");
                    if (st != RPIM_OK) break;
                    if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
                        st = fail(RPIM_E_CUDA, "tune: event");
                        break;
                    }
                    float t = 0.f;
                    cudaEventElapsedTime(&t, e0, e1);
                    if (rep > 0) ms = std::min(ms, t);   // the first run warms up
                }
                if (ms < best_ms) { best_ms = ms; best = c; }
            }
        if (st != RPIM_OK) break;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tuned[ref][std::min(NC, RPIM_MAX_SUPPORT)] = best;
        }
        if (table && nt < 16) {
            table[3 * nt] = NC;
            table[3 * nt + 1] = best.G;
            table[3 * nt + 2] = best.ppb;
        }
        nt++;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (n_table) *n_table = nt;
    RPIM_CHECK(st);
    return check_device_error(p, "autotune");
}

extern "C" rpim_status rpim_probe_recip(int64_t n, const double *d, double *r, rpim_stream_t stream)
{
    if (n < 0 || (n > 0 && (!d || !r))) return fail(RPIM_E_ARG, "bad argument");
    if (n == 0) return RPIM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    RPIM_CUDA(cudaGetDevice(&dev));
    RPIM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    launch("recip_probe", recip_probe_kernel, grid_size(sms, 4, n, 256), 256, 0, s, n, d, r);
    RPIM_CUDA(cudaGetLastError());
    RPIM_CUDA(cudaStreamSynchronize(s));
    return RPIM_OK;
}

extern "C" rpim_status rpim_autotune_set(int32_t max_support, int32_t warps_per_point, int32_t points_per_block)
{
    const int NC = std::max(8, (int)max_support);
    const ShapeCfg c{points_per_block, warps_per_point};
    const bool ref = refined();
    if (max_support < 1 || max_support > RPIM_MAX_SUPPORT || !cfg_valid(NC, c, ref))
        return fail(RPIM_E_ARG, "launch shape not admissible for this support size");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[ref][NC] = c;
    return RPIM_OK;
}

extern "C" rpim_status rpim_autotune_reset(void)
{
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (auto &t : g_tuned)
            for (auto &c : t) c = ShapeCfg{};
    }
    set_default_buckets({});
    return RPIM_OK;
}

extern "C" rpim_status rpim_set_shape_solver(int32_t solver)
{
    if (solver != RPIM_SOLVER_FP64 && solver != RPIM_SOLVER_REFINED) return fail(RPIM_E_ARG, "unknown solver");
    g_solver.store(solver);
    return RPIM_OK;
}

extern "C" rpim_status rpim_get_shape_solver(int32_t *solver)
{
    if (!solver) return fail(RPIM_E_ARG, "null argument");
    *solver = g_solver.load();
    return RPIM_OK;
}

extern "C" rpim_status rpim_set_shape_schedule(int32_t persistent)
{
    if (persistent != 0 && persistent != 1) return fail(RPIM_E_ARG, "schedule must be 0 or 1");
    g_persistent.store(persistent);
    return RPIM_OK;
}

// Bucket bounds autotuner: candidate bound sets (the built-in one and
// uniform widths of 4-32 support sizes between the smallest and largest
// support) are each applied to the pattern and the persistent shape pass is
// timed on a sample of every bucket (CUDA events); the fastest set stays.
extern "C" rpim_status rpim_autotune_buckets(rpim_pattern *p, int64_t max_points, int32_t *bounds_out,
                                             int32_t *n_bounds_out, rpim_stream_t stream)
{
    RPIM_STAGE("rpim_autotune_buckets");
    if (!p || max_points < 1) return fail(RPIM_E_ARG, "bad argument");
    if (p->shape_kind != RPIM_SHAPE_RPIM) {
        if (n_bounds_out) *n_bounds_out = 0;
        return RPIM_OK;
    }
    cudaStream_t s = (cudaStream_t)stream;
    p->stream = s;
    if (!p->phi) RPIM_CHECK(dalloc(&p->phi, 4 * p->n_entries, s));
    std::vector<std::vector<int32_t>> cands;
    cands.push_back({40, 56, 72, 96, 128, 160});
    for (int w : {4, 8, 12, 16, 24, 32}) {
        std::vector<int32_t> b;
        for (int v = std::max(8, (int)p->min_support + w - 1); v < (int)p->max_support; v += w) b.push_back(v);
        if (b.empty()) b.push_back((int32_t)p->max_support);
        if ((int)b.size() <= 31) cands.push_back(b);
    }
    {
        // occupancy bounds: the largest support for which ppb point groups
        // fit one block's shared memory, ppb = 1..15 (a bucket just below
        // such a bound runs one more point per block than a bucket above it),
        // alone and merged with the width-16 bounds
        const bool ref = refined();
        std::vector<int32_t> occ;
        for (int ppb = 15; ppb >= 1; ppb--) {
            int nc = 8;
            while (nc + 1 <= RPIM_MAX_SUPPORT && (size_t)ppb * point_bytes(nc + 1, ref) <= kShapeSmemBudget) nc++;
            if ((size_t)ppb * point_bytes(nc, ref) <= kShapeSmemBudget && nc > (int)p->min_support &&
                nc < (int)p->max_support && (occ.empty() || nc > occ.back()))
                occ.push_back(nc);
        }
        if (!occ.empty()) {
            cands.push_back(occ);
            std::vector<int32_t> merged = occ;
            for (int v = std::max(8, (int)p->min_support + 15); v < (int)p->max_support; v += 16) merged.push_back(v);
            std::sort(merged.begin(), merged.end());
            merged.erase(std::unique(merged.begin(), merged.end()), merged.end());
            if ((int)merged.size() <= 31) cands.push_back(merged);
        }
    }
    const double frac = std::min(1.0, (double)max_points / (double)std::max<int64_t>(1, p->n_points));
    cudaEvent_t e0, e1;
    RPIM_CUDA(cudaEventCreate(&e0));
    RPIM_CUDA(cudaEventCreate(&e1));
    rpim_status st = RPIM_OK;
    float best_ms = 1e30f;
    size_t best = 0;
    for (size_t c = 0; c < cands.size() && st == RPIM_OK; c++) {
        st = rpim_pattern_set_buckets(p, (int32_t)cands[c].size(), cands[c].data(), stream);
        float ms = 1e30f;
        for (int rep = 0; rep < 3 && st == RPIM_OK; rep++) {
            if (cudaEventRecord(e0, s) != cudaSuccess) { st = fail(RPIM_E_CUDA, "tune: event"); break; }
            st = shape_functions_tiles(p, p->phi, s, frac);
            if (st != RPIM_OK) break;
            if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
                st = fail(RPIM_E_CUDA, "tune: event");
                break;
            }
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            if (rep > 0) ms = std::min(ms, t);
        }
        if (st == RPIM_OK && ms < best_ms) { best_ms = ms; best = c; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st == RPIM_OK) st = rpim_pattern_set_buckets(p, (int32_t)cands[best].size(), cands[best].data(), stream);
    RPIM_CHECK(st);
    set_default_buckets(cands[best]);
    if (n_bounds_out) *n_bounds_out = (int32_t)cands[best].size();
    if (bounds_out)
        for (size_t i = 0; i < cands[best].size(); i++) bounds_out[i] = cands[best][i];
    return check_device_error(p, "autotune buckets");
}
