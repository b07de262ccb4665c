// Errors, device-wide scans, node -> entry incidence and the kernel-basis
// series of librpim.
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/rpim_probe.h"
#include "common.cuh"

namespace rpim {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

rpim_status fail(rpim_status st, const std::string &msg)
{
    g_last_error = msg;
    return st;
}

rpim_status cuda_fail(cudaError_t e, const char *what)
{
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? RPIM_E_OOM : RPIM_E_CUDA;
}

// ---------------------------------------------------------------------------
// launch bookkeeping
// ---------------------------------------------------------------------------
namespace {
struct LaunchRecord {
    const char *name;
    cudaEvent_t a, b;
};
std::atomic<long long> g_launches{0};
std::atomic<long long> g_device_allocs{0};
std::atomic<int> g_profile{0};
std::mutex g_mu;
std::vector<LaunchRecord> g_pending;
std::vector<cudaEvent_t> g_pool;
std::map<std::string, std::pair<long long, double>> g_stats;

cudaEvent_t pool_get()
{
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}
} // namespace

int64_t launch_begin(const char *name, cudaStream_t s)
{
    g_launches.fetch_add(1);
    if (!g_profile.load()) return -1;
    std::lock_guard<std::mutex> lk(g_mu);
    LaunchRecord r{name, pool_get(), pool_get()};
    cudaEventRecord(r.a, s);
    g_pending.push_back(r);
    return (int64_t)g_pending.size() - 1;
}

bool profiling_on() { return g_profile.load() != 0; }

void add_launches(int64_t n) { g_launches.fetch_add(n); }

void note_device_alloc() { g_device_allocs.fetch_add(1); }

int64_t launch_count() { return g_launches.load(); }

void launch_end(int64_t tok, cudaStream_t s)
{
    if (tok < 0) return;
    std::lock_guard<std::mutex> lk(g_mu);
    if (tok < (int64_t)g_pending.size()) cudaEventRecord(g_pending[tok].b, s);
}

static void drain_pending()
{
    for (auto &r : g_pending) {
        float ms = 0.f;
        cudaEventSynchronize(r.b);
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            auto &st = g_stats[r.name];
            st.first += 1;
            st.second += ms;
        }
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_pending.clear();
}

int grid_size(int sm_count, int blocks_per_sm, int64_t work, int threads)
{
    int64_t need = (work + threads - 1) / threads;
    int64_t cap = (int64_t)sm_count * blocks_per_sm;
    if (need < 1) need = 1;
    return (int)std::min(need, cap);
}

// ---------------------------------------------------------------------------
// exclusive scan (3 kernels: block sums, scan of block sums, block scans)
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

template <class T>
__device__ __forceinline__ int64_t block_sum(int64_t v)
{
    __shared__ int64_t warp_sums[kScanThreads / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) warp_sums[w] = v;
    __syncthreads();
    int64_t t = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < kScanThreads / 32; i++) t += warp_sums[i];
    __syncthreads();
    return t;
}

template <class T>
__global__ void scan_block_sums(const T *data, int64_t n, int64_t *sums)
{
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t v = 0;
    for (int i = 0; i < kScanItems; i++) {
        int64_t k = base + (int64_t)i * kScanThreads + threadIdx.x;
        if (k < n) v += (int64_t)data[k];
    }
    int64_t t = block_sum<T>(v);
    if (threadIdx.x == 0) sums[blockIdx.x] = t;
}

__global__ void scan_sums_serial(int64_t *sums, int64_t nb)
{
    // one block: exclusive scan of nb block sums, in chunks of blockDim
    __shared__ int64_t buf[1024];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < nb; base += blockDim.x) {
        int64_t k = base + threadIdx.x;
        buf[threadIdx.x] = k < nb ? sums[k] : 0;
        __syncthreads();
        for (int o = 1; o < (int)blockDim.x; o <<= 1) {
            int64_t add = threadIdx.x >= (unsigned)o ? buf[threadIdx.x - o] : 0;
            __syncthreads();
            buf[threadIdx.x] += add;
            __syncthreads();
        }
        int64_t incl = buf[threadIdx.x];
        int64_t excl = incl - (k < nb ? sums[k] : 0);
        __syncthreads();
        if (k < nb) sums[k] = carry + excl;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[nb] = carry;
}

template <class T>
__global__ void scan_blocks(T *data, int64_t n, const int64_t *sums)
{
    // each thread scans kScanItems consecutive items; then block scan
    __shared__ int64_t tsum[kScanThreads];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t loc[kScanItems];
    int64_t acc = 0;
    for (int i = 0; i < kScanItems; i++) {
        int64_t k = base + i;
        int64_t v = k < n ? (int64_t)data[k] : 0;
        loc[i] = acc;
        acc += v;
    }
    tsum[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 1; o < kScanThreads; o <<= 1) {
        int64_t add = threadIdx.x >= (unsigned)o ? tsum[threadIdx.x - o] : 0;
        __syncthreads();
        tsum[threadIdx.x] += add;
        __syncthreads();
    }
    int64_t off = sums[blockIdx.x] + tsum[threadIdx.x] - acc;
    for (int i = 0; i < kScanItems; i++) {
        int64_t k = base + i;
        if (k < n) data[k] = (T)(off + loc[i]);
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) data[n] = (T)sums[gridDim.x];
}

int64_t scan_tmp_size(int64_t n) { return (n + kScanTile - 1) / kScanTile + 2; }

template <class T>
static rpim_status scan_impl(T *data, int64_t n, int64_t *tmp, cudaStream_t s)
{
    int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb < 1) nb = 1;
    launch("scan_block_sums", scan_block_sums<T>, (unsigned)nb, kScanThreads, 0, s, data, n, tmp);
    launch("scan_sums_serial", scan_sums_serial, 1, 1024, 0, s, tmp, nb);
    launch("scan_blocks", scan_blocks<T>, (unsigned)nb, kScanThreads, 0, s, data, n, tmp);
    RPIM_CUDA(cudaGetLastError());
    return RPIM_OK;
}

rpim_status exclusive_scan(int64_t *data, int64_t n, int64_t *tmp, cudaStream_t s)
{
    return scan_impl<int64_t>(data, n, tmp, s);
}
rpim_status exclusive_scan32(int32_t *data, int64_t n, int64_t *tmp, cudaStream_t s)
{
    return scan_impl<int32_t>(data, n, tmp, s);
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort of (key, value) pairs, 8-bit digits from bit 0 up to
// `bits`. Every pass: the digit histogram of every tile of kSortTile
// elements; an exclusive scan of the histograms in digit-major order (the
// first output slot of every (digit, tile)); a scatter in which an element's
// place among the equal digits of its tile follows its position (warp
// match, per-warp counts, running counts per round), so equal keys keep
// their input order.
// ---------------------------------------------------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortTile = 16 * kSortThreads;

__global__ void __launch_bounds__(kSortThreads) radix_hist_kernel(const uint64_t *keys, int64_t n, int shift,
                                                                  int64_t *hist)
{
    __shared__ int cnt[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) cnt[i] = 0;
    __syncthreads();
    const int64_t b0 = (int64_t)blockIdx.x * kSortTile, b1 = min(n, b0 + kSortTile);
    for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) atomicAdd(&cnt[(keys[i] >> shift) & 255], 1);
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[(int64_t)d * gridDim.x + blockIdx.x] = cnt[d];
}

__global__ void __launch_bounds__(kSortThreads) radix_scatter_kernel(const uint64_t *kin, const int32_t *vin,
                                                                     int64_t n, int shift, const int64_t *off,
                                                                     uint64_t *kout, int32_t *vout)
{
    __shared__ int base[256];                 // elements of each digit placed by earlier rounds
    __shared__ int wcnt[kSortWarps][256];     // this round's count of each digit per warp
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < 256; d += blockDim.x) base[d] = 0;
    const int64_t b0 = (int64_t)blockIdx.x * kSortTile, b1 = min(n, b0 + kSortTile);
    for (int64_t r0 = b0; r0 < b1; r0 += kSortThreads) {
        for (int i = threadIdx.x; i < kSortWarps * 256; i += blockDim.x) (&wcnt[0][0])[i] = 0;
        __syncthreads();
        const int64_t i = r0 + threadIdx.x;
        const bool valid = i < b1;
        uint64_t k = 0;
        int32_t v = 0;
        int dig = 256;   // past the digits: lanes without an element
        if (valid) {
            k = kin[i];
            v = vin[i];
            dig = (int)((k >> shift) & 255);
        }
        const unsigned peers = __match_any_sync(0xffffffffu, dig);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && lane == __ffs(peers) - 1) wcnt[w][dig] = __popc(peers);
        __syncthreads();
        if (valid) {
            int before = 0;
            for (int ww = 0; ww < w; ww++) before += wcnt[ww][dig];
            const int64_t pos = off[(int64_t)dig * gridDim.x + blockIdx.x] + base[dig] + before + rank;
            kout[pos] = k;
            vout[pos] = v;
        }
        __syncthreads();
        for (int d = threadIdx.x; d < 256; d += blockDim.x) {
            int t = 0;
            for (int ww = 0; ww < kSortWarps; ww++) t += wcnt[ww][d];
            base[d] += t;
        }
        __syncthreads();
    }
}

rpim_status radix_sort_pairs(uint64_t *keys, int32_t *vals, int64_t n, int bits, cudaStream_t s)
{
    if (n <= 1 || bits <= 0) return RPIM_OK;
    const int64_t nb = (n + kSortTile - 1) / kSortTile;
    const int64_t nh = 256 * nb;
    uint64_t *k2 = nullptr;
    int32_t *v2 = nullptr;
    int64_t *hist = nullptr, *tmp = nullptr;
    rpim_status st = dalloc(&k2, n, s);
    if (st == RPIM_OK) st = dalloc(&v2, n, s);
    if (st == RPIM_OK) st = dalloc(&hist, nh + 1, s);
    if (st == RPIM_OK) st = dalloc(&tmp, scan_tmp_size(nh), s);
    uint64_t *ka = keys, *kb = k2;
    int32_t *va = vals, *vb = v2;
    int passes = 0;
    for (int shift = 0; shift < bits && st == RPIM_OK; shift += 8, passes++) {
        launch("radix_hist", radix_hist_kernel, (unsigned)nb, kSortThreads, 0, s, (const uint64_t *)ka, n, shift, hist);
        st = exclusive_scan(hist, nh, tmp, s);
        if (st != RPIM_OK) break;
        launch("radix_scatter", radix_scatter_kernel, (unsigned)nb, kSortThreads, 0, s, (const uint64_t *)ka,
               (const int32_t *)va, n, shift, (const int64_t *)hist, kb, vb);
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (st == RPIM_OK && cudaGetLastError() != cudaSuccess) st = fail(RPIM_E_CUDA, "radix sort launch");
    if (st == RPIM_OK && (passes & 1)) {   // the result sits in the scratch buffers
        cudaError_t e = cudaMemcpyAsync(keys, ka, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(vals, va, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) st = cuda_fail(e, "radix sort copy");
    }
    dfree(k2, s); dfree(v2, s); dfree(hist, s); dfree(tmp, s);
    return st;
}

// ---------------------------------------------------------------------------
// device error word
// ---------------------------------------------------------------------------
static const char *status_name(int c)
{
    switch (c) {
    case RPIM_E_ARG: return "invalid argument";
    case RPIM_E_SUPPORT: return "support size out of range, or a node in no support";
    case RPIM_E_SINGULAR: return "singular moment problem";
    case RPIM_E_NONFINITE: return "non-finite value";
    case RPIM_E_NOCONV: return "no convergence";
    case RPIM_E_TIMEOUT: return "timeout";
    default: return "error";
    }
}

rpim_status check_device_error(rpim_pattern *p, const char *stage)
{
    unsigned long long w = 0;
    RPIM_CUDA(cudaMemcpyAsync(&w, &p->err->word, sizeof(w), cudaMemcpyDeviceToHost, p->stream));
    RPIM_CUDA(cudaStreamSynchronize(p->stream));
    if (w == ~0ull) return RPIM_OK;
    int code = (int)(w >> 48);
    long long idx = (long long)(w & 0xFFFFFFFFFFFFull);
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s at index %lld", stage, status_name(code), idx);
    // reset for the next call
    unsigned long long clean = ~0ull;
    RPIM_CUDA(cudaMemcpyAsync(&p->err->word, &clean, sizeof(clean), cudaMemcpyHostToDevice, p->stream));
    RPIM_CUDA(cudaStreamSynchronize(p->stream));
    return fail((rpim_status)code, buf);
}

// ---------------------------------------------------------------------------
// node -> entries incidence: counting sort by node, then a bitonic sort of
// every node's segment so that entries (hence points) ascend.
// ---------------------------------------------------------------------------
__global__ void count_nodes(const int32_t *sidx, int64_t ne, unsigned long long *cnt)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne;
         e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[sidx[e]], 1ull);
}

__global__ void fill_nodes(const int32_t *sidx, int64_t ne, const int64_t *toff,
                           unsigned long long *cursor, int64_t *tent)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne;
         e += (int64_t)gridDim.x * blockDim.x) {
        int32_t I = sidx[e];
        unsigned long long k = atomicAdd(&cursor[I], 1ull);
        tent[toff[I] + (int64_t)k] = e;
    }
}

__global__ void max_segment(const int64_t *off, int64_t n, int *out)
{
    int m = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, (int)(off[i + 1] - off[i]));
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// one warp per segment; segment padded to `pow2` in shared memory
__global__ void sort_segments(const int64_t *off, int64_t n, int64_t *vals, int pow2)
{
    extern __shared__ int64_t sm[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t *buf = sm + (size_t)w * pow2;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t seg = (int64_t)blockIdx.x * (blockDim.x >> 5) + w; seg < n; seg += warps) {
        int64_t b = off[seg], len = off[seg + 1] - b;
        if (len <= 1) continue;
        int p2 = 1;
        while (p2 < len) p2 <<= 1;
        for (int i = lane; i < p2; i += 32) buf[i] = i < len ? vals[b + i] : INT64_MAX;
        __syncwarp();
        for (int k = 2; k <= p2; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = lane; i < p2; i += 32) {
                    int ixj = i ^ j;
                    if (ixj > i) {
                        int64_t a = buf[i], c = buf[ixj];
                        bool up = (i & k) == 0;
                        if ((a > c) == up) { buf[i] = c; buf[ixj] = a; }
                    }
                }
                __syncwarp();
            }
        for (int i = lane; i < len; i += 32) vals[b + i] = buf[i];
        __syncwarp();
    }
}

rpim_status build_incidence(int64_t n_nodes, int64_t ne, const int32_t *sidx, int64_t **toff_out,
                            int64_t **tent_out, int32_t *max_incident, cudaStream_t s, int sm_count)
{
    int64_t *toff = nullptr, *tent = nullptr, *tmp = nullptr;
    unsigned long long *cursor = nullptr;
    int *dmax = nullptr;
    RPIM_CHECK(dalloc(&toff, n_nodes + 1, s));
    RPIM_CHECK(dalloc(&tent, ne, s));
    RPIM_CHECK(dalloc(&cursor, n_nodes + 1, s));
    RPIM_CHECK(dalloc(&tmp, scan_tmp_size(n_nodes), s));
    RPIM_CHECK(dalloc(&dmax, 1, s));
    RPIM_CUDA(cudaMemsetAsync(toff, 0, (n_nodes + 1) * sizeof(int64_t), s));
    RPIM_CUDA(cudaMemsetAsync(cursor, 0, (n_nodes + 1) * sizeof(unsigned long long), s));
    RPIM_CUDA(cudaMemsetAsync(dmax, 0, sizeof(int), s));
    int g = grid_size(sm_count, 8, ne, 256);
    launch("count_nodes", count_nodes, g, 256, 0, s, sidx, ne, (unsigned long long *)toff);
    RPIM_CHECK(exclusive_scan(toff, n_nodes, tmp, s));
    launch("fill_nodes", fill_nodes, g, 256, 0, s, sidx, ne, toff, cursor, tent);
    launch("max_segment", max_segment, grid_size(sm_count, 4, n_nodes, 256), 256, 0, s, toff, n_nodes, dmax);
    int hmax = 0;
    RPIM_CUDA(cudaMemcpyAsync(&hmax, dmax, sizeof(int), cudaMemcpyDeviceToHost, s));
    RPIM_CUDA(cudaStreamSynchronize(s));
    int p2 = 1;
    while (p2 < hmax) p2 <<= 1;
    if (p2 > 8192) {
        dfree(toff, s); dfree(tent, s); dfree(cursor, s); dfree(tmp, s); dfree(dmax, s);
        return fail(RPIM_E_SUPPORT, "node incidence larger than 8192 entries");
    }
    int wpb = std::max(1, std::min(8, (int)(48 * 1024 / ((size_t)p2 * 8))));
    size_t smem = (size_t)wpb * p2 * 8;
    if (smem > 48 * 1024) RPIM_CUDA(cudaFuncSetAttribute(sort_segments, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    launch("sort_segments", sort_segments, grid_size(sm_count, 4, n_nodes, wpb), wpb * 32, smem, s, toff, n_nodes, tent, p2);
    RPIM_CUDA(cudaGetLastError());
    dfree(cursor, s);
    dfree(tmp, s);
    dfree(dmax, s);
    *toff_out = toff;
    *tent_out = tent;
    *max_incident = hmax;
    return RPIM_OK;
}

// ---------------------------------------------------------------------------
// Kernel-basis series.
//
// With the linear polynomial constraints sum_i a_i p(x_i) = 0, any kernel of
// the form alpha + beta (|x - y|^2 + c^2) adds nothing to the interpolant:
// its constant part, its f(x) + f(y) part and its bilinear -2 beta x.y part
// are all annihilated, and the right-hand sides change consistently. The
// shape functions are therefore unchanged when the multiquadric s^q
// (s = r^2 + c^2) is replaced by  A(s) = s^q - alpha - beta s,  the
// multiquadric minus its chord over the range of s met in a support. A(s) is
// a few hundredths in size instead of tens, so its FP64 rounding perturbs the
// (ill-conditioned) moment problem hundreds of times less.
//
// A(s) is evaluated as a power series in t = (s - m_k)/w_k on geometric
// pieces [b_k, b_k+1] of the range, from the binomial series
//   s^q = sum_j C(q, j) m^(q-j) (s - m)^j,  |s - m| < m,
// whose j = 0, 1 terms are merged with the chord. All coefficients are
// computed in long double and the truncated series is checked against
// powl() on a dense sample.
// ---------------------------------------------------------------------------
static rpim_status build_kernel_series_uncached(double alpha_c, double alpha_s, double q, KernelSeries *ks);

// The series depends on (alpha_c, alpha_s, q) only; it is built (and
// checked against the closed form in long double, a few milliseconds where
// long double is emulated in software) once per parameter set and process.
rpim_status build_kernel_series(double alpha_c, double alpha_s, double q, KernelSeries *ks)
{
    static std::mutex mu;
    static std::map<std::tuple<double, double, double>, KernelSeries> cache;
    const auto key = std::make_tuple(alpha_c, alpha_s, q);
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) {
            *ks = it->second;
            return RPIM_OK;
        }
    }
    rpim_status st = build_kernel_series_uncached(alpha_c, alpha_s, q, ks);
    if (st == RPIM_OK) {
        std::lock_guard<std::mutex> lk(mu);
        cache[key] = *ks;
    }
    return st;
}

static rpim_status build_kernel_series_uncached(double alpha_c, double alpha_s, double q, KernelSeries *ks)
{
    if (!(alpha_c > 0) || !(alpha_s > 0) || !(q > 0) || q == 1.0 || q >= 2.0)
        return fail(RPIM_E_ARG, "kernel parameters out of range (need alpha_c, alpha_s > 0, 0 < q < 2, q != 1)");
    typedef long double L;
    memset(ks, 0, sizeof(*ks));
    const L c2 = (L)alpha_c * (L)alpha_c, ql = (L)q;
    const L s_lo = c2 * (1 - 1e-9L);
    const L s_hi = (c2 + 4 * (L)alpha_s * (L)alpha_s) * (1 + 1e-6L);
    const L beta = (powl(s_hi, ql) - powl(s_lo, ql)) / (s_hi - s_lo);
    const L alpha0 = powl(s_lo, ql) - beta * s_lo;
    const L ratio = s_hi / s_lo;
    ks->c2 = (double)c2;
    // |coefficient of t^j| on the worst (first) piece: |C(q,j)| m^q x^j
    auto coef_bound = [&](L m, L x, int j) {
        L cj = 1;
        for (int i = 1; i <= j; i++) cj *= (ql - i + 1) / i;
        return fabsl(cj) * powl(m, ql) * powl(x, (L)j);
    };
    // most pieces whose series reaches a tail below 1e-19 within kMaxDegree
    int P = 0, D = 0, H = 0;
    for (int pieces = kMaxPieces; pieces >= 2 && !P; pieces /= 2) {
        L r = powl(ratio, 1.0L / pieces);
        L m = s_lo * (1 + r) / 2, x = (r - 1) / (1 + r) * 1.01L; // |t| <= 1.01
        for (int d = 2; d <= kMaxDegree; d++) {
            if (coef_bound(m, x, d + 1) / (1 - x) < 1e-19L) {
                P = pieces;
                D = d;
                break;
            }
        }
        // FP32 for the powers whose coefficients are below 2^-24 * 1e-19 * ...
        if (P) {
            H = D + 1;
            for (int j = 2; j <= D; j++)
                if (coef_bound(m, x, j) < 1.7e-12L) { H = j; break; }
            if (H > kMaxHead) H = kMaxHead;
        }
    }
    if (!P) return fail(RPIM_E_ARG, "kernel series: support radius too large for the series");
    ks->pieces = P;
    ks->degree = D;
    ks->n64 = H;
    const L r = powl(ratio, 1.0L / P);
    ks->log2_lo = (float)log2l(s_lo);
    ks->inv_log2r = (float)(1.0L / log2l(r));
    for (int k = 0; k < P; k++) {
        L b0 = s_lo * powl(r, (L)k), b1 = s_lo * powl(r, (L)(k + 1));
        // the device forms t = (s - centre) * inv_w with the rounded centre
        // and inverse half-width (s - centre is exact: Sterbenz); the
        // coefficients are taken at exactly those values
        ks->centre[k] = (double)((b0 + b1) / 2);
        ks->inv_w[k] = (double)(2 / (b1 - b0));
        const L m = (L)ks->centre[k], w = 1 / (L)ks->inv_w[k];
        L a[kMaxDegree + 2];
        a[0] = powl(m, ql) - alpha0 - beta * m;
        a[1] = (ql * powl(m, ql - 1) - beta) * w;
        L cj = ql; // C(q,1)
        for (int j = 2; j <= D + 1; j++) {
            cj *= (ql - j + 1) / j;
            a[j] = cj * powl(m, ql - j) * powl(w, (L)j);
        }
        for (int j = 0; j <= D; j++) {
            if (j < H) ks->coef[k][j] = (double)a[j];
            else ks->coef_f[k][j] = (float)a[j];
        }
        for (int j = 0; j < D; j++) ks->dcoef[k][j] = (double)((j + 1) * a[j + 1] / w);
    }
    // check the device evaluation order (piece from a single-precision log2,
    // FP32 tail, FP64 head) against the closed form
    auto eval = [&](L s, L &v, L &dv) {
        float f = (log2f((float)s) - ks->log2_lo) * ks->inv_log2r;
        int k = (int)f;
        k = k < 0 ? 0 : (k > P - 1 ? P - 1 : k);
        double t = ((double)s - ks->centre[k]) * ks->inv_w[k];
        float tf = (float)t, h = ks->coef_f[k][D];
        for (int j = D - 1; j >= H; j--) h = h * tf + ks->coef_f[k][j];
        v = H <= D ? (L)h : 0;
        for (int j = H - 1; j >= 0; j--) v = v * (L)t + (L)ks->coef[k][j];
        dv = 0;
        for (int j = D - 1; j >= 0; j--) dv = dv * (L)t + (L)ks->dcoef[k][j];
    };
    // Sample points: 129 per piece, evenly spaced in t over [-1.02, 1.02]
    // (a truncated series errs most at the ends of its piece, and the
    // single-precision piece choice may move a point just across a piece
    // boundary), clipped to the range of s the device evaluates. Long double
    // is emulated in software on some hosts, so the sample is kept to a few
    // thousand closed-form evaluations.
    L worst = 0, worst_d = 0;
    const int NT = 128;
    for (int k = 0; k < P; k++) {
        const L m = (L)ks->centre[k], w = 1 / (L)ks->inv_w[k];
        for (int i = 0; i <= NT; i++) {
            L sl = m + w * (-1.02L + 2.04L * (L)i / NT);
            sl = sl < c2 ? c2 : (sl > s_hi ? s_hi : sl);
            // sample at doubles: the device only ever sees double arguments
            L s = (L)(double)sl, v, dv;
            eval(s, v, dv);
            L want = powl(s, ql) - alpha0 - beta * s;
            L dwant = ql * powl(s, ql - 1) - beta;
            worst = fmaxl(worst, fabsl(v - want));
            worst_d = fmaxl(worst_d, fabsl(dv - dwant));
        }
    }
    ks->check_err = (double)fmaxl(worst, worst_d);
    if (worst > 5e-17L || worst_d > 5e-17L) {
        char buf[160];
        snprintf(buf, sizeof buf, "kernel series check failed: %.3Le %.3Le", worst, worst_d);
        return fail(RPIM_E_ARG, buf);
    }
    {
        L v, dv;
        eval(c2, v, dv);
        ks->diag = (double)v;
    }
    return RPIM_OK;
}

} // namespace rpim

extern "C" const char *rpim_last_error(void) { return rpim::g_last_error.c_str(); }
extern "C" rpim_status rpim_kernel_series_info(double alpha_c, double alpha_s, double q, int32_t *pieces,
                                               int32_t *degree, int32_t *fp64_terms, double *max_err)
{
    rpim::KernelSeries ks;
    rpim_status st = rpim::build_kernel_series_uncached(alpha_c, alpha_s, q, &ks);
    if (pieces) *pieces = ks.pieces;
    if (degree) *degree = ks.degree;
    if (fp64_terms) *fp64_terms = ks.n64;
    if (max_err) *max_err = ks.check_err;
    return st;
}

extern "C" int64_t rpim_kernel_launches(void) { return rpim::g_launches.load(); }

extern "C" int64_t rpim_device_allocations(void) { return rpim::g_device_allocs.load(); }

extern "C" rpim_status rpim_pool_used_bytes(int64_t *bytes)
{
    if (!bytes) return rpim::fail(RPIM_E_ARG, "null argument");
    int dev = 0;
    RPIM_CUDA(cudaGetDevice(&dev));
    cudaMemPool_t pool;
    RPIM_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
    uint64_t used = 0;
    RPIM_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used));
    *bytes = (int64_t)used;
    return RPIM_OK;
}

extern "C" rpim_status rpim_profile_enable(int32_t on)
{
    std::lock_guard<std::mutex> lk(rpim::g_mu);
    rpim::drain_pending();
    rpim::g_profile.store(on ? 1 : 0);
    return RPIM_OK;
}

extern "C" rpim_status rpim_profile_read(char *buf, int64_t cap, int32_t reset)
{
    if (!buf || cap <= 0) return rpim::fail(RPIM_E_ARG, "null buffer");
    std::lock_guard<std::mutex> lk(rpim::g_mu);
    rpim::drain_pending();
    std::string js = "{";
    char item[256];
    bool first = true;
    for (auto &kv : rpim::g_stats) {
        snprintf(item, sizeof item, "%s\"%s\": [%lld, %.6f]", first ? "" : ", ", kv.first.c_str(),
                 kv.second.first, kv.second.second);
        js += item;
        first = false;
    }
    js += "}";
    if (reset) rpim::g_stats.clear();
    if ((int64_t)js.size() + 1 > cap) return rpim::fail(RPIM_E_ARG, "profile buffer too small");
    memcpy(buf, js.c_str(), js.size() + 1);
    return RPIM_OK;
}

extern "C" const char *rpim_version(void) { return "rpim-gb300 0.1 (sm_103a)"; }
