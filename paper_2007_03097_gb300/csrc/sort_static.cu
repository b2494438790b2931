// sph_sort_keys_noalloc: the (key, id) sort of sph_sort_keys for callers that
// cannot allocate device memory.  Its scratch (key and index ping-pong
// buffers, digit histograms, scan partials, status word) lives in one
// file-scope static device array of fixed size; the caller passes only its
// inputs and the output permutation.  No context, no cudaMalloc/cudaFree.
//
// The kernels are those of the context path (tree.cu, scan.cu): this file
// points a context-shaped view at the static array and runs the same sort.
#include <string>

#include "sph_internal.cuh"

// message of the last failing context-free call of this thread
// (sph_last_error(NULL) returns it)
void noalloc_fail(const std::string &msg);

namespace {

constexpr int64_t NOALLOC_MAX = SPH_SORT_NOALLOC_MAX;
constexpr size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr int64_t NOALLOC_TILES = (NOALLOC_MAX + 4095) / 4096;
constexpr size_t OFF_KA = 0;
constexpr size_t OFF_KB = OFF_KA + align256(8 * (size_t)NOALLOC_MAX);
constexpr size_t OFF_VA = OFF_KB + align256(8 * (size_t)NOALLOC_MAX);
constexpr size_t OFF_VB = OFF_VA + align256(4 * (size_t)NOALLOC_MAX);
constexpr size_t OFF_HIST = OFF_VB + align256(4 * (size_t)NOALLOC_MAX);
constexpr size_t OFF_SCAN = OFF_HIST + align256(4 * 256 * (size_t)NOALLOC_TILES);
constexpr size_t SCAN_BYTES = 4096;                 // scan partials of 256 x 64 histogram entries
constexpr size_t OFF_CNT = OFF_SCAN + SCAN_BYTES;
constexpr size_t SCRATCH_BYTES = OFF_CNT + align256(sizeof(DevCounters));

// ~6.1 MB, held by every device that loads the library until the process exits
static __device__ __align__(256) unsigned char g_sort_scratch[SCRATCH_BYTES];

// Device address of the static array on the current device.  In host code
// the symbol is only a host-side stand-in, so its device address is looked up
// with cudaGetSymbolAddress on every call, with the device current: the first
// call on a device also loads the library's device code there, and a device
// reset gives the array a new address, so none is kept between calls.
int scratch_address(unsigned char **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_sort_scratch);
    if (e != cudaSuccess || !p) {
        noalloc_fail(std::string("cudaGetSymbolAddress of the sort scratch: ") + cudaGetErrorString(e));
        return SPH_ERR_CUDA;
    }
    *out = (unsigned char *)p;
    return SPH_OK;
}

// nullptr if ptr is device (or managed) memory of device dev, else the reason
const char *not_on_device(const void *ptr, int dev)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();                       // clear the error the failed query recorded
        return "is not a CUDA pointer";
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return "is not device memory";
    if (at.device != dev) return "lives on another device than the current one";
    return nullptr;
}

}  // namespace

extern "C" int sph_sort_keys_noalloc(int64_t n, const uint64_t *keys, const uint32_t *ids, uint32_t *perm,
                                     void *stream)
{
    if (n < 1 || !keys || !perm) {
        noalloc_fail("sph_sort_keys_noalloc: n must be >= 1 and keys, perm must not be NULL");
        return SPH_ERR_ARG;
    }
    if (n > NOALLOC_MAX) {
        noalloc_fail("sph_sort_keys_noalloc: n = " + std::to_string(n) + " exceeds the static scratch (at most " +
                     std::to_string(NOALLOC_MAX) + " keys)");
        return SPH_ERR_CAPACITY;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        noalloc_fail("sph_sort_keys_noalloc: no current CUDA device");
        return SPH_ERR_CUDA;
    }
    const void *ptrs[3] = {keys, ids, perm};
    const char *names[3] = {"keys", "ids", "perm"};
    for (int k = 0; k < 3; ++k) {
        if (!ptrs[k]) continue;                   // ids may be NULL
        if (const char *why = not_on_device(ptrs[k], dev)) {
            noalloc_fail(std::string("sph_sort_keys_noalloc: ") + names[k] + " " + why + " (device " +
                         std::to_string(dev) + ")");
            return SPH_ERR_ARG;
        }
    }
    unsigned char *base = nullptr;
    const int st = scratch_address(&base);
    if (st != SPH_OK) return st;
    // a context-shaped view over the static scratch (host object only)
    sph_ctx view;
    view.n_max = NOALLOC_MAX;
    view.key_a = (uint64_t *)(base + OFF_KA);
    view.key_b = (uint64_t *)(base + OFF_KB);
    view.val_a = (uint32_t *)(base + OFF_VA);
    view.val_b = (uint32_t *)(base + OFF_VB);
    view.hist = (uint32_t *)(base + OFF_HIST);
    view.hist_cap = 256 * NOALLOC_TILES;
    view.scan_tmp = base + OFF_SCAN;
    view.scan_tmp_bytes = SCAN_BYTES;
    view.dcnt = (DevCounters *)(base + OFF_CNT);
    DevCounters host_counters{};
    view.hcnt = &host_counters;
    const int r = tree_sort(&view, n, keys, ids, perm, (cudaStream_t)stream);
    if (r != SPH_OK) noalloc_fail(view.err.empty() ? std::string("sph_sort_keys_noalloc failed") : view.err);
    return r;
}
