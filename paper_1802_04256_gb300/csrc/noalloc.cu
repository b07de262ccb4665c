// Stress recovery without any device allocation.
//
// Some callers must not allocate device memory once they are running: hosts
// that fix their device-memory budget at start-up and account every byte, or
// loops that keep other streams busy and cannot afford the device-wide
// synchronisation that cudaMalloc/cudaFree may imply. rpim_stress allocates
// its per-call scratch (support lists and shape functions of the stress
// points); rpim_stress_noalloc does the same work in a fixed scratch array
// that lives in the library's own device memory for as long as the library
// is loaded.
#include <stdio.h>

#include <mutex>

#include "common.cuh"

namespace rpim {
namespace {

// scratch layout (bytes, each part 256-byte aligned):
//   support offsets  int64 [kMaxPoints + 1]
//   scan scratch     int64 [scan_tmp_size(kMaxPoints)]
//   min/max support  int32 [2]
//   support ids      int32 [kMaxEntries]
//   shape functions  double [4 * kMaxEntries]
constexpr int64_t kMaxPoints = RPIM_NOALLOC_MAX_POINTS;
constexpr int64_t kMaxEntries = RPIM_NOALLOC_MAX_ENTRIES;

constexpr int64_t align256(int64_t b) { return (b + 255) / 256 * 256; }
constexpr int64_t kOffSoff = 0;
constexpr int64_t kOffTmp = align256(kOffSoff + 8 * (kMaxPoints + 1));
constexpr int64_t kOffMinMax = align256(kOffTmp + 8 * ((kMaxPoints + 4095) / 4096 + 2));
constexpr int64_t kOffSidx = align256(kOffMinMax + 8);
constexpr int64_t kOffPhi = align256(kOffSidx + 4 * kMaxEntries);
constexpr int64_t kScratchBytes = align256(kOffPhi + 32 * kMaxEntries);

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of the scratch array for each device, taken once per
// device with that device current. In host code the array's name is only a
// host-side stand-in, so kernels get this address, never the name.
std::mutex g_mu;
unsigned char *g_addr[64] = {nullptr};

rpim_status scratch_address(int device, unsigned char **out)
{
    if (device < 0 || device >= 64) return fail(RPIM_E_ARG, "device index out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[device]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_addr[device] = (unsigned char *)ptr;
    }
    *out = g_addr[device];
    return RPIM_OK;
}

} // namespace
} // namespace rpim

using namespace rpim;

extern "C" rpim_status rpim_stress_noalloc(rpim_pattern *p, const double *u, int64_t n_pts, const double *xyz,
                                           const double *E, const double *nu, double *sigma, rpim_stream_t stream)
{
    if (!p || n_pts < 0 || (n_pts > 0 && (!u || !xyz || !E || !nu || !sigma))) return fail(RPIM_E_ARG, "bad argument");
    if (n_pts > kMaxPoints) {
        char buf[128];
        snprintf(buf, sizeof buf, "%lld stress points exceed the fixed limit of %lld per call", (long long)n_pts,
                 (long long)kMaxPoints);
        return fail(RPIM_E_ARG, buf);
    }
    if (n_pts == 0) return RPIM_OK;
    int dev = 0;
    RPIM_CUDA(cudaGetDevice(&dev));
    if (dev != p->device) return fail(RPIM_E_ARG, "pattern belongs to another device");
    if (p->n_inst != 1) return fail(RPIM_E_ARG, "the allocation-free variant takes single-instance patterns");
    unsigned char *base = nullptr;
    RPIM_CHECK(scratch_address(dev, &base));
    cudaStream_t s = (cudaStream_t)stream;
    p->stream = s;
    int64_t *soff = (int64_t *)(base + kOffSoff);
    int64_t *tmp = (int64_t *)(base + kOffTmp);
    int *minmax = (int *)(base + kOffMinMax);
    int32_t *sidx = (int32_t *)(base + kOffSidx);
    double *phi = (double *)(base + kOffPhi);
    int64_t ne = 0;
    int32_t mx = 0;
    // every part the kernels read is written first in this call: the count
    // pass fills soff, the scan fills tmp, min/max is reset from the host,
    // the fill pass writes the ids and the shape kernel writes phi
    RPIM_CHECK(search_supports_into(p, n_pts, xyz, soff, tmp, minmax, sidx, kMaxEntries, &ne, &mx, s,
                                    "search_stress_noalloc"));
    RPIM_CHECK(shape_functions(p, n_pts, xyz, (const int32_t *)nullptr, 0, (const int32_t *)nullptr, soff, sidx, mx,
                               phi, s, "shape_stress_noalloc"));
    RPIM_CHECK(launch_stress(p, n_pts, soff, sidx, phi, u, E, nu, sigma, s));
    return check_device_error(p, "stress (no allocation)");
}
