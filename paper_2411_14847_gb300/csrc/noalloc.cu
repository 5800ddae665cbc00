// dass_bin_sort_static: the tile binning + radix sort of dass_bin_sort for callers that cannot
// allocate device memory. Such callers exist when a host application owns every device
// allocation through its own pool and does not let libraries call cudaMalloc (real-time render
// plugins, engines with a fixed memory budget), or when an allocation on the calling path would
// block or synchronise the device at a moment the caller cannot afford. They still pass the
// inputs and outputs; the sort's scratch lives in a fixed device array compiled into this file.
#include <mutex>

#include "common.cuh"

namespace dass {
size_t bin_sort_workspace_bytes(long long n_rec, long long cap);
int bin_sort_launch(const dass_splat* splats, long long n_rec, const CamTable& ct, uint32_t* pair_rec, long long cap,
                    uint32_t* tile_ranges, long long* counters, void* ws, size_t ws_bytes, cudaStream_t st);
void set_error_message(const char* msg);
}  // namespace dass

using namespace dass;

namespace {

constexpr size_t kScratchBytes = (size_t)DASS_BIN_SORT_STATIC_BYTES;
constexpr int kMaxDevices = 64;

// One copy per device that loads this library, resident until the process exits.
static __device__ __align__(256) unsigned char g_sort_scratch[kScratchBytes];

std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_sort_scratch on the current device, looked up once per device. In host
// code the symbol names a host-side stand-in, so only this address may be given to kernels.
// The cached address belongs to the device's context at lookup time: a cudaDeviceReset (or any
// teardown of the primary context) reloads the module at another address, so this entry point
// must not be used across such a reset.
int scratch_for_current_device(void** out) {
    int dev = -1;
    DASS_CHECK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return DASS_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (g_scratch_ptr[dev] == nullptr) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_sort_scratch);
        if (e != cudaSuccess || p == nullptr) {
            set_last_error("cudaGetSymbolAddress(g_sort_scratch)", e);
            return DASS_ERR_CUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return DASS_OK;
}

}  // namespace

DASS_API int dass_bin_sort_static(const dass_splat* splats, int64_t rec_stride, const dass_camera* cams, int n_cams,
                                  int tile, uint32_t* pair_rec, int64_t pair_capacity, uint32_t* tile_ranges,
                                  int64_t* counters, void* stream) {
    if (rec_stride < 0 || pair_capacity < 0 || !tile_ranges || !counters) return DASS_ERR_INVALID_ARG;
    static thread_local CamTable ct;
    if (!make_cam_table(cams, n_cams, tile, rec_stride, &ct)) return DASS_ERR_INVALID_ARG;
    long long n_rec = (long long)n_cams * rec_stride;
    if (n_rec >= (1ll << 32) || pair_capacity >= (1ll << 31)) return DASS_ERR_INVALID_ARG;
    if (n_rec > 0 && (!splats || !pair_rec)) return DASS_ERR_INVALID_ARG;
    size_t need = bin_sort_workspace_bytes(n_rec, pair_capacity);
    if (need > kScratchBytes) {
        set_error_message("dass_bin_sort_static: records and pair capacity need more scratch than the "
                          "DASS_BIN_SORT_STATIC_BYTES static array; use dass_bin_sort with a workspace");
        return DASS_ERR_OOM;
    }
    void* scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc) return rc;
    return bin_sort_launch(splats, n_rec, ct, pair_rec, pair_capacity, tile_ranges, (long long*)counters, scratch,
                           kScratchBytes, as_stream(stream));
}
