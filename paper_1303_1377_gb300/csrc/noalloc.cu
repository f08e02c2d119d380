// Allocation-free variant of ddamg_apply_Dc.
//
// Some callers cannot let this library call cudaMalloc at the moment they apply
// the coarse operator. Examples are a code that has handed almost all device
// memory to its own pool (PyTorch's caching allocator, a serving process with a
// fixed memory budget), or a latency-critical loop that cannot afford the
// implicit device synchronisation of cudaMalloc/cudaFree. For them this entry
// point takes its working memory from a fixed, file-scope device array instead of
// allocating: the caller passes device input and output vectors, and the two
// internal-layout staging buffers live in the array below.
#include "kernels.h"

struct ddamg_handle;

namespace ddamg {
int apply_Dc_into_scratch(ddamg_handle* h, const double* in, double* out, int n_rhs, void* scratch, size_t scratch_bytes);
int handle_device(const ddamg_handle* h);
}

namespace {

// 16 MiB of scratch, held by every GPU that loads the library until the process exits.
constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the array per device (host code cannot use the symbol itself:
// in host code it names a host-side stand-in, not device memory).
constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};

}  // namespace

extern "C" int ddamg_apply_Dc_noalloc(ddamg_handle* h, const double* in, double* out, int n_rhs) {
    if (!h) {
        ddamg::set_error("ddamg_apply_Dc_noalloc: null handle");
        return DDAMG_ERR_INVALID_ARG;
    }
    // The kernels run on the handle's stream, which lives on the device the handle was created on;
    // the scratch address must be that device's copy of the array.
    const int hdev = ddamg::handle_device(h);
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        ddamg::set_error(std::string("ddamg_apply_Dc_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
        return DDAMG_ERR_CUDA;
    }
    if (dev != hdev) {
        ddamg::set_error("ddamg_apply_Dc_noalloc: the current device (" + std::to_string(dev) + ") is not the handle's device (" +
                         std::to_string(hdev) + "); make the handle's device current first");
        return DDAMG_ERR_INVALID_ARG;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        ddamg::set_error("ddamg_apply_Dc_noalloc: device index " + std::to_string(dev) + " is beyond the " +
                         std::to_string(kMaxDevices) + " devices this entry point keeps a scratch address for");
        return DDAMG_ERR_INVALID_ARG;
    }
    if (!g_scratch_addr[dev]) {
        // one-time set-up on this device (with this device current)
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            ddamg::set_error(std::string("ddamg_apply_Dc_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return DDAMG_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    return ddamg::apply_Dc_into_scratch(h, in, out, n_rhs, g_scratch_addr[dev], kNoAllocScratchBytes);
}
