// Internal definitions shared by the translation units of librpim.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/rpim.h"

namespace rpim {

// ---------------------------------------------------------------------------
// error reporting
// ---------------------------------------------------------------------------
void set_error(const std::string &msg);
rpim_status fail(rpim_status st, const std::string &msg);
rpim_status cuda_fail(cudaError_t e, const char *what);

#define RPIM_CUDA(call)                                         \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return ::rpim::cuda_fail(e_, #call); \
    } while (0)

// An NVTX range around one call of the C ABI, named after the call, so that
// profilers (Nsight Systems, ncu --nvtx) show the pipeline's stages; without
// a tool attached a push/pop is a no-op call.
struct StageRange {
    explicit StageRange(const char *name) { nvtxRangePushA(name); }
    ~StageRange() { nvtxRangePop(); }
    StageRange(const StageRange &) = delete;
    StageRange &operator=(const StageRange &) = delete;
};
#define RPIM_STAGE(name) ::rpim::StageRange rpim_stage_range_(name)

#define RPIM_CHECK(st)                       \
    do {                                     \
        rpim_status s_ = (st);               \
        if (s_ != RPIM_OK) return s_;        \
    } while (0)

// Device error record: the first failing (code, index) pair wins, encoded as
// code << 48 | index so that atomicMin keeps the lowest code, then the lowest
// index (deterministic report).
struct DevError {
    unsigned long long word; // 0xFFFF... when clean
};

__device__ __forceinline__ void dev_fail(DevError *err, int code, long long index)
{
    unsigned long long w = ((unsigned long long)code << 48) | ((unsigned long long)index & 0xFFFFFFFFFFFFull);
    atomicMin(&err->word, w);
}

// ---------------------------------------------------------------------------
// kernel-basis series: the multiquadric with its affine-in-s part removed,
// as piecewise power series in t = (s - centre) / half_width, s = r^2 + c^2.
// ---------------------------------------------------------------------------
constexpr int kMaxPieces = 16;
constexpr int kMaxHead = 16;   // FP64 (head) terms of the value series
constexpr int kMaxDegree = 24;

struct KernelSeries {
    int pieces;
    int degree;                         // highest power kept
    int n64;                            // powers 0..n64-1 in FP64, n64..degree in FP32
    float log2_lo;                      // piece = floor((log2 s - log2_lo) * inv_log2r)
    float inv_log2r;
    double c2;                          // alpha_c^2
    double diag;                        // value at s = c2 (r = 0)
    double check_err;                   // largest error of the host check
    double centre[kMaxPieces];          // centre of each piece
    double inv_w[kMaxPieces];           // 1 / half_width
    double coef[kMaxPieces][kMaxHead];          // value series, powers 0..n64-1
    float coef_f[kMaxPieces][kMaxDegree + 1];   // value series, powers n64..degree
    double dcoef[kMaxPieces][kMaxDegree + 1];   // d/ds series, powers 0..degree-1
};

// Builds the series on the host (long double arithmetic) and checks it
// against the closed form on a dense sample.
rpim_status build_kernel_series(double alpha_c, double alpha_s, double q, KernelSeries *ks);

// ---------------------------------------------------------------------------
// pattern object
// ---------------------------------------------------------------------------
// One independent instance (node cloud) of a pattern: its own uniform grid
// (cell edge >= its support radius), support radius and nodal spacing.
// Instances are consecutive node ranges; a plain pattern has one.
struct InstGrid {
    double lo[3];
    double inv_edge;     // 1 / cell edge
    double rs2;          // support radius squared
    double inv_h;        // 1 / nodal spacing
    int n[3];            // cells per axis
    float q_cell;        // rs2 in squared cell edges (single precision)
    float margin;        // bound on the single-precision error of a squared distance in cell units
    int pad;
    int64_t cell_off;    // first global cell of the instance
    int64_t node_begin, node_end;
};

// the 25 runs of cells (dy, dz in [-2, 2], dx in [-2, 2] contiguous) around
// I's cell: start in the cell-ordered list and exclusive prefix of lengths
__device__ __forceinline__ int cell_runs(const InstGrid &g, const int32_t *cell_start, int cx, int cy, int cz,
                                         int lane, int *run_start, int *run_pre)
{
    if (lane < 25) {
        const int dy = lane % 5 - 2, dz = lane / 5 - 2;
        const int yy = cy + dy, zz = cz + dz;
        int st = 0, len = 0;
        if (yy >= 0 && yy < g.n[1] && zz >= 0 && zz < g.n[2]) {
            const int xa = max(cx - 2, 0), xb = min(cx + 2, g.n[0] - 1);
            const int64_t row = g.cell_off + (int64_t)g.n[0] * (yy + (int64_t)g.n[1] * zz);
            st = cell_start[row + xa];
            len = cell_start[row + xb + 1] - st;
        }
        run_start[lane] = st;
        run_pre[lane + 1] = len;
    }
    __syncwarp();
    if (lane == 0) {
        run_pre[0] = 0;
        for (int r = 0; r < 25; r++) run_pre[r + 1] += run_pre[r];
    }
    __syncwarp();
    return run_pre[25];
}

// position of node J in the 25 runs around the cell (cx, cy, cz) (the bit
// of J in a row's bitmap), or -1 when J lies outside the 5x5x5 cells
__device__ __forceinline__ int run_bit(const uint32_t *node_cpk, const int32_t *node_rank, int32_t J, int cx, int cy,
                                       int cz, const int *run_start, const int *run_pre)
{
    const uint32_t cj = node_cpk[J];
    const int dx = (int)(cj & 0x7FF) - cx, dy = (int)((cj >> 11) & 0x7FF) - cy, dz = (int)(cj >> 22) - cz;
    if (dx < -2 || dx > 2 || dy < -2 || dy > 2 || dz < -2 || dz > 2) return -1;
    const int r = (dy + 2) + 5 * (dz + 2);
    return run_pre[r] + (node_rank[J] - run_start[r]);
}

// the same from a node's (packed cell, rank in cell) pair, as stored per
// support entry (rpim_pattern::ecell)
__device__ __forceinline__ int run_bit_cell(uint2 cj_rank, int cx, int cy, int cz, const int *run_start,
                                            const int *run_pre)
{
    const uint32_t cj = cj_rank.x;
    const int dx = (int)(cj & 0x7FF) - cx, dy = (int)((cj >> 11) & 0x7FF) - cy, dz = (int)(cj >> 22) - cz;
    if (dx < -2 || dx > 2 || dy < -2 || dy > 2 || dz < -2 || dz > 2) return -1;
    const int r = (dy + 2) + 5 * (dz + 2);
    return run_pre[r] + ((int)cj_rank.y - run_start[r]);
}

// instance of point k of a list: inst_of[k >> shift], or 0 without a map
__device__ __forceinline__ int instance_of(const int32_t *inst_of, int shift, int64_t k)
{
    return inst_of ? inst_of[k >> shift] : 0;
}

struct Workspace {      // PCG vectors and reduction scratch (lazily sized)
    double *buf = nullptr;
    int64_t doubles = 0;
};

} // namespace rpim

struct rpim_pattern {
    int device = 0;
    cudaStream_t stream = nullptr;
    rpim_params prm{};     // alpha_c, q (common); alpha_s, h of the first instance
    int n_inst = 1;
    int shape_kind = RPIM_SHAPE_RPIM;   // shape functions of every stage (rpim_pattern_set_shape)
    int precond = RPIM_PRECOND_JACOBI;  // PCG preconditioner (rpim_pattern_set_precond)
    double series_alpha_s = 0.0;    // support radius the kernel series covers
    std::vector<rpim::InstGrid> ig_host;
    rpim::InstGrid *ig = nullptr;   // [n_inst] device copy
    int32_t *node_inst = nullptr;   // [n_nodes] instance of each node
    int64_t total_cells = 0;
    // support-size buckets of the integration points for the shape kernel
    std::vector<int64_t> bucket_count;   // points per bucket
    std::vector<int32_t> bucket_nc;      // largest support in the bucket
    int32_t *bucket_order = nullptr;     // [n_points] point ids grouped by bucket
    std::vector<int32_t> bucket_bounds;  // upper support size of each bucket (last open-ended)
    unsigned long long *tile_counter = nullptr;  // [32] per-bucket work counters of the persistent shape kernel
    // FP64 copies of the reduced moment matrices of the refined shape solver:
    // one slice per resident point group (multiprocessors x their shared
    // memory bounds every launch), allocated with the pattern
    double *shape_scratch = nullptr;
    int64_t shape_scratch_doubles = 0;

    int64_t n_nodes = 0, n_points = 0, n_entries = 0, nnzb = 0;
    int32_t max_support = 0, min_support = 0, max_row = 0;
    int32_t max_incident = 0;  // largest number of (point, entry) pairs per node
    int32_t max_cell = 0;      // largest node count of a grid cell
    int32_t bit_words = 0;     // 32-bit words of a row bitmap over the 5x5x5 cells around a node

    // nodes
    double *xyz = nullptr;          // [n_nodes*3] copy of the coordinates
    double *sorted_xyz = nullptr;   // [n_nodes*4] coordinates in cell order (x,y,z,pad)
    float *sorted_loc = nullptr;    // [n_nodes*4] the same in cell edges from the grid origin, FP32
    int32_t *sorted_ids = nullptr;  // [n_nodes] node ids in cell order
    int32_t *cell_start = nullptr;  // [cells+1]
    int32_t *node_cell = nullptr;   // [n_nodes] linear cell index of each node
    uint32_t *node_cpk = nullptr;   // [n_nodes] cell coordinates packed x | y << 11 | z << 22
    int32_t *node_rank = nullptr;   // [n_nodes] position of the node in its cell
    int32_t *row_order = nullptr;   // [n_nodes] nodes by Morton key of their cell (instance first), ids ascending
    // integration points
    double *pts = nullptr;          // [n_points*3]
    double *wj = nullptr;           // [n_points]
    // supports
    int64_t *soff = nullptr;        // [n_points+1]
    int32_t *sidx = nullptr;        // [n_entries]
    int32_t *entry_pt = nullptr;    // [n_entries] point of each entry
    uint2 *ecell = nullptr;         // [n_entries] (packed cell, rank in cell) of each entry's node
    // node -> entries incidence, ascending entry (hence ascending point)
    int64_t *toff = nullptr;        // [n_nodes+1]
    int64_t *tent = nullptr;        // [n_entries]
    // BSR pattern of K
    int64_t *rowptr = nullptr;      // [n_nodes+1]
    int32_t *cols = nullptr;        // [nnzb]
    int64_t *diag = nullptr;        // [n_nodes] slot of the diagonal block
    // assembly scratch
    double *phi = nullptr;          // [n_entries*4]
    double *lamw = nullptr;         // [n_points*2] (lambda w|J|, mu w|J|)
    // device scalars
    rpim::DevError *err = nullptr;
    double *scal = nullptr;         // [16] device scalars (penalty, PCG)
    rpim::KernelSeries *series = nullptr; // device copy
    rpim::KernelSeries series_host{};
    rpim::Workspace ws;
    // row segments of the batched solver: rows [seg_row[s], seg_row[s+1])
    // belong to instance seg_inst[s]; instance i owns the segments
    // [inst_seg[i], inst_seg[i+1]) (built on the first batched solve)
    cudaStream_t cap_stream = nullptr;   // capture-only stream of the PCG and assembly graphs
    cudaGraphExec_t asm_exec = nullptr;  // captured assembly (rpim_assemble_graphed)
    std::vector<unsigned char> asm_key;  // what the captured assembly was built for
    int64_t asm_kernels = 0;             // kernels in the captured assembly
    int64_t n_seg = 0;
    int64_t *seg_row = nullptr;     // [n_seg+1]
    int32_t *seg_inst = nullptr;    // [n_seg]
    int32_t *inst_seg = nullptr;    // [n_inst+1]
    int sm_count = 0;
};

namespace rpim {

// every device allocation the library makes is counted (rpim_device_allocations)
void note_device_alloc();

// allocation helpers (stream ordered)
template <class T>
rpim_status dalloc(T **p, int64_t count, cudaStream_t s)
{
    if (count <= 0) count = 1;
    note_device_alloc();
    cudaError_t e = cudaMallocAsync((void **)p, (size_t)count * sizeof(T), s);
    if (e != cudaSuccess) {
        *p = nullptr;
        return fail(RPIM_E_OOM, std::string("device allocation failed: ") + cudaGetErrorString(e));
    }
    return RPIM_OK;
}
template <class T>
void dfree(T *&p, cudaStream_t s)
{
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
}

// device-wide exclusive scan of int64 counts (in place on `data`, n+1
// entries: data[n] receives the total). Uses `tmp` of scan_tmp_size(n).
int64_t scan_tmp_size(int64_t n);
rpim_status exclusive_scan(int64_t *data, int64_t n, int64_t *tmp, cudaStream_t s);
rpim_status exclusive_scan32(int32_t *data, int64_t n, int64_t *tmp, cudaStream_t s);

// stable LSD radix sort of (key, value) pairs on the low `bits` bits of the
// keys (in place; scratch allocated stream ordered)
rpim_status radix_sort_pairs(uint64_t *keys, int32_t *vals, int64_t n, int bits, cudaStream_t s);

// reads the device error word; returns RPIM_OK or the recorded status
rpim_status check_device_error(rpim_pattern *p, const char *stage);

// support search for arbitrary points (count + fill); output offsets/ids
// are allocated here (stream ordered) and owned by the caller. The instance
// of point k is inst_of[k >> shift] (inst_of NULL: instance 0).
rpim_status search_supports(rpim_pattern *p, int64_t n_pts, const double *pts, const int32_t *inst_of, int shift,
                            int64_t **soff, int32_t **sidx, int64_t *n_entries,
                            int32_t *max_n, int32_t *min_n, cudaStream_t s, const char *tag);

// support search into caller-provided buffers (no allocation)
rpim_status search_supports_into(rpim_pattern *p, int64_t n_pts, const double *pts, int64_t *soff, int64_t *tmp,
                                 int *minmax, int32_t *sidx, int64_t cap, int64_t *n_entries, int32_t *max_n,
                                 cudaStream_t s, const char *tag);  // single-instance patterns

// stress kernel on given supports and shape functions (no allocation)
rpim_status launch_stress(rpim_pattern *p, int64_t n_pts, const int64_t *soff, const int32_t *sidx, const double *phi,
                          const double *u, const double *E, const double *nu, double *sigma, cudaStream_t s);

// shape functions of n_pts points with given supports -> phi [entries*4];
// instance of point k as for search_supports; `order` (optional) lists the
// points to process (n_pts of them), all with supports <= max_n
rpim_status shape_functions(rpim_pattern *p, int64_t n_pts, const double *pts, const int32_t *inst_of, int shift,
                            const int32_t *order, const int64_t *soff, const int32_t *sidx, int32_t max_n,
                            double *phi, cudaStream_t s, const char *tag);

// shape functions of all integration points of a pattern, one launch per
// support-size bucket
rpim_status shape_functions_all(rpim_pattern *p, double *phi, cudaStream_t s);

// the order in which the row-owner kernels (pattern, row) take their rows:
// the pattern's Morton order, or null (node order), per rpim_set_row_order
const int32_t *rows_in_order(const rpim_pattern *p);

// bucket bounds that new patterns start with (empty: the built-in ones)
void set_default_buckets(const std::vector<int32_t> &bounds);

// key of what shape_functions_all launches for this pattern (see shape.cu)
rpim_status shape_launch_key(const rpim_pattern *p, std::vector<unsigned char> *key);

// MLS variant of shape_functions (one thread per point, any support size)
rpim_status mls_shape_functions(rpim_pattern *p, int64_t n_pts, const double *pts, const int32_t *inst_of, int shift,
                                const int32_t *order, const int64_t *soff, const int32_t *sidx, double *phi,
                                cudaStream_t s, const char *tag);

// node -> entries incidence (stable: ascending entry) of a support list
rpim_status build_incidence(int64_t n_nodes, int64_t n_entries, const int32_t *sidx,
                            int64_t **toff, int64_t **tent, int32_t *max_incident,
                            cudaStream_t s, int sm_count);

int grid_size(int sm_count, int blocks_per_sm_hint, int64_t work, int threads);

// kernel launch bookkeeping: every launch of the library is counted, and
// when profiling is on (rpim_profile_enable) bracketed by CUDA events on its
// stream so that per-kernel device times can be read back.
int64_t launch_begin(const char *name, cudaStream_t s);
void launch_end(int64_t token, cudaStream_t s);
bool profiling_on();            // per-kernel event timing enabled
void add_launches(int64_t n);   // kernels run by a replayed CUDA graph
int64_t launch_count();

template <typename... KArgs, typename... Args>
inline void launch(const char *name, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                   cudaStream_t s, Args... args)
{
    const int64_t tok = launch_begin(name, s);
    kernel<<<grid, block, smem, s>>>(args...);
    launch_end(tok, s);
}

// entry -> point map of a support list (one warp per point)
__global__ void entry_points_kernel(int64_t n_pts, const int64_t *soff, int32_t *entry_pt);

} // namespace rpim
