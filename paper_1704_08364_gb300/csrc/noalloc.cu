// noalloc.cu -- bst_fbp_noalloc: the BST filtered backprojection with its
// scratch memory in a fixed, file-scope device array instead of a
// caller-provided workspace.
//
// For callers that cannot allocate device memory at the point where they
// reconstruct: code running under an external memory manager that owns all
// of the device's memory, or a latency-sensitive loop where a cudaMalloc /
// cudaFree (which may synchronise the device) is not acceptable.  The call
// itself allocates nothing; the plan (created beforehand with
// bst_plan_create, which does allocate its tables) is reused as is.
//
// Limit: the scratch array holds BST_NOALLOC_SCRATCH_BYTES = 8 MiB on every
// GPU that loads the library, for as long as the process lives.  Its device
// address is looked up when a plan is created on a device (see
// bst_noalloc_setup_current_device), so a call does no set-up of its own.  A call is
// accepted when one slice pair's workspace, (V M + 4 ceil(N/4) M) * 8 bytes,
// fits in it (for example N = V = 512 at pad factor 2); larger plans are
// rejected with BST_ERR_WORKSPACE_TOO_SMALL.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "bst_internal.h"

#define BST_NOALLOC_SCRATCH_BYTES ((size_t)8 << 20)
#define BST_NOALLOC_MAX_DEVICES 64

// The scratch shared by every bst_fbp_noalloc call on a device.  In host
// code this name is only a host-side stand-in for the symbol, never a
// device address: the address is taken once per device with
// cudaGetSymbolAddress below and passed to the kernels.
static __device__ __align__(256) unsigned char bst_noalloc_scratch[BST_NOALLOC_SCRATCH_BYTES];

namespace {

std::mutex g_mu;
void* g_addr[BST_NOALLOC_MAX_DEVICES] = {nullptr};

// Look up the scratch array's device address on the current device and
// cache it (refresh = true replaces a cached address).
bst_status_t resolve(bool refresh, void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return BST_ERR_CUDA;
    if (dev < 0 || dev >= BST_NOALLOC_MAX_DEVICES) return BST_ERR_INVALID_ARGUMENT;
    std::lock_guard<std::mutex> lock(g_mu);
    if (refresh || !g_addr[dev]) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, bst_noalloc_scratch) != cudaSuccess || !ptr) {
            g_addr[dev] = nullptr;
            return BST_ERR_CUDA;
        }
        g_addr[dev] = ptr;
    }
    if (out) *out = g_addr[dev];
    return BST_OK;
}

}  // namespace

// Set-up for the current device, called by bst_plan_create with the plan's
// device current: the first symbol lookup loads this file's device code on
// that device (which places the scratch array in device memory), so that it
// happens when the caller creates a plan, not inside a bst_fbp_noalloc call.
// A new plan re-reads the address, which keeps it valid after a
// cudaDeviceReset (which also ends every plan made before it).
bst_status_t bst_noalloc_setup_current_device() { return resolve(true, nullptr); }

extern "C" {

size_t bst_noalloc_scratch_bytes(void) { return BST_NOALLOC_SCRATCH_BYTES; }

bst_status_t bst_fbp_noalloc(bst_plan_t p, const float* d_sino, int slices, const float* d_g, float* d_volume,
                             bst_stream_t stream) {
    if (!p || !d_sino || !d_volume || slices <= 0) return BST_ERR_INVALID_ARGUMENT;
    if (!bsth::on_plan_device(p)) return BST_ERR_INVALID_ARGUMENT;
    const size_t ns = (size_t)slices * p->V * p->N * sizeof(float);
    const size_t nv = (size_t)slices * p->N * p->N * sizeof(float);
    const uintptr_t a0 = (uintptr_t)d_sino, b0 = (uintptr_t)d_volume;
    if (a0 < b0 + nv && b0 < a0 + ns) return BST_ERR_INVALID_ARGUMENT;
    const size_t per_pair = bsth::fwd_bytes_per_pair(p);
    if (per_pair > BST_NOALLOC_SCRATCH_BYTES) return BST_ERR_WORKSPACE_TOO_SMALL;
    void* ws = nullptr;
    const bst_status_t s = resolve(false, &ws);   // normally cached by bst_plan_create
    if (s != BST_OK) return s;
    // every scratch byte a call reads is written earlier in the same call, so
    // nothing needs clearing between calls
    const int max_chunk = (int)std::min<size_t>((size_t)p->chunk_pairs, BST_NOALLOC_SCRATCH_BYTES / per_pair);
    return bst_launch_forward_chunked(p, d_sino, slices, BSTK_FILTER, d_g, d_volume, ws, (cudaStream_t)stream,
                                      max_chunk, 1);
}

}  // extern "C"
