// sph_sort_keys_noalloc: the (key, id) sort of sph_sort_keys for callers that
// cannot allocate device memory.  Its scratch (key and index ping-pong
// buffers, digit histograms, scan partials, status word) lives in one
// file-scope static device array of fixed size; the caller passes only its
// inputs and the output permutation.  No context, no cudaMalloc/cudaFree.
//
// The kernels are those of the context path (tree.cu, scan.cu): this file
// points a context-shaped view at the static array and runs the same sort.
#include <mutex>

#include "sph_internal.cuh"

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

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void *g_addr[MAX_DEVICES] = {};

// Device address of the static array on the current device.  In host code
// the symbol is only a host-side stand-in, so it is looked up once per device
// with cudaGetSymbolAddress (the first call on a device does this).
int scratch_address(int dev, unsigned char **out)
{
    if (dev < 0 || dev >= MAX_DEVICES) return SPH_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_sort_scratch) != cudaSuccess || !p) return SPH_ERR_CUDA;
        g_addr[dev] = p;
    }
    *out = (unsigned char *)g_addr[dev];
    return SPH_OK;
}

}  // namespace

extern "C" int sph_sort_keys_noalloc(int64_t n, const uint64_t *keys, const uint32_t *ids, uint32_t *perm,
                                     void *stream)
{
    if (n < 1 || !keys || !perm) return SPH_ERR_ARG;
    if (n > NOALLOC_MAX) return SPH_ERR_CAPACITY;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SPH_ERR_CUDA;
    unsigned char *base = nullptr;
    const int st = scratch_address(dev, &base);
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
    return tree_sort(&view, n, keys, ids, perm, (cudaStream_t)stream);
}
