// host.cu -- bst_fbp_host: filtered backprojection of a volume held in host
// memory, with the host->device copies, the BST path and the device->host
// copies overlapped in double-buffered chunks of slices.
//
// The paper's pipeline overlaps data movement with GPU stages on separate
// threads and streams (Sec. 3); here one call enqueues the whole overlap on
// three streams: the caller's stream computes, two plan-owned streams copy.
// Chunk c uses staging buffer c % 2: its upload waits until the compute of
// chunk c - 2 has consumed that input buffer; its compute waits for its upload
// and for the download of chunk c - 2 from that output buffer; its download
// waits for its compute.  One cudaMemcpyAsync per chunk and direction.
#include <cuda_runtime.h>

#include <algorithm>

#include "bst_internal.h"

namespace {

// slices per staging chunk: an even number, about 512 MiB of input
int host_chunk_slices(const bst_plan_s* p, int slices) {
    const size_t per_slice = (size_t)p->V * p->N * sizeof(float);
    size_t c = ((size_t)512 << 20) / per_slice;
    c = std::max<size_t>(2, c & ~(size_t)1);
    return (int)std::min<size_t>(c, (size_t)slices);
}

bool ensure_host_streams(bst_plan_s* p) {
    for (int i = 0; i < 2; ++i) {
        if (!p->hs[i] && cudaStreamCreateWithFlags(&p->hs[i], cudaStreamNonBlocking) != cudaSuccess) return false;
    }
    for (int i = 0; i < 7; ++i) {
        if (!p->hev[i] && cudaEventCreateWithFlags(&p->hev[i], cudaEventDisableTiming) != cudaSuccess) return false;
    }
    return true;
}

}  // namespace

extern "C" {

size_t bst_host_workspace_bytes(bst_plan_t p, int slices) {
    if (!p || slices <= 0) return 0;
    const size_t C = (size_t)host_chunk_slices(p, slices);
    const size_t in = C * p->V * p->N * sizeof(float);
    const size_t out = C * p->N * p->N * sizeof(float);
    return 2 * (in + out) + bst_workspace_bytes(p, (int)C) + 256;
}

bst_status_t bst_fbp_host(bst_plan_t p, const float* h_sino, int slices, const float* d_g, float* h_volume,
                          void* d_ws, size_t ws_bytes, bst_stream_t stream) {
    if (!p || !h_sino || !h_volume || slices <= 0) return BST_ERR_INVALID_ARGUMENT;
    if (!bsth::on_plan_device(p)) return BST_ERR_INVALID_ARGUMENT;
    if (!d_ws || ws_bytes < bst_host_workspace_bytes(p, slices)) return BST_ERR_WORKSPACE_TOO_SMALL;
    if (!ensure_host_streams(p)) return BST_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    const int C = host_chunk_slices(p, slices);
    const size_t in_elems = (size_t)C * p->V * p->N, out_elems = (size_t)C * p->N * p->N;
    float* in_buf[2] = {(float*)d_ws, (float*)d_ws + in_elems};
    float* out_buf[2] = {(float*)d_ws + 2 * in_elems, (float*)d_ws + 2 * in_elems + out_elems};
    void* fwd_ws = (void*)((float*)d_ws + 2 * (in_elems + out_elems));
    const size_t fwd_bytes = bst_workspace_bytes(p, C);
    cudaEvent_t& start = p->hev[0];
    cudaEvent_t* comp_done = &p->hev[1];   // [2]
    cudaEvent_t* in_ready = &p->hev[3];    // [2]
    cudaEvent_t* out_done = &p->hev[5];    // [2]
    cudaStream_t up = p->hs[0], down = p->hs[1];
    bool ok = cudaEventRecord(start, st) == cudaSuccess && cudaStreamWaitEvent(up, start, 0) == cudaSuccess &&
              cudaStreamWaitEvent(down, start, 0) == cudaSuccess;
    const int nchunks = (slices + C - 1) / C;
    for (int c = 0; ok && c < nchunks; ++c) {
        const int b = c & 1;
        const int s0 = c * C;
        const int ns = std::min(C, slices - s0);
        if (c >= 2) ok = ok && cudaStreamWaitEvent(up, comp_done[b], 0) == cudaSuccess;
        ok = ok && cudaMemcpyAsync(in_buf[b], h_sino + (size_t)s0 * p->V * p->N, (size_t)ns * p->V * p->N * sizeof(float),
                                   cudaMemcpyHostToDevice, up) == cudaSuccess;
        ok = ok && cudaEventRecord(in_ready[b], up) == cudaSuccess;
        ok = ok && cudaStreamWaitEvent(st, in_ready[b], 0) == cudaSuccess;
        if (c >= 2) ok = ok && cudaStreamWaitEvent(st, out_done[b], 0) == cudaSuccess;
        if (!ok) break;
        const bst_status_t s = bst_launch_forward(p, in_buf[b], ns, BSTK_FILTER, d_g, out_buf[b], fwd_ws, fwd_bytes, st);
        if (s != BST_OK) return s;
        ok = ok && cudaEventRecord(comp_done[b], st) == cudaSuccess;
        ok = ok && cudaStreamWaitEvent(down, comp_done[b], 0) == cudaSuccess;
        ok = ok && cudaMemcpyAsync(h_volume + (size_t)s0 * p->N * p->N, out_buf[b], (size_t)ns * p->N * p->N * sizeof(float),
                                   cudaMemcpyDeviceToHost, down) == cudaSuccess;
        ok = ok && cudaEventRecord(out_done[b], down) == cudaSuccess;
    }
    // the caller's stream completes only after the last download
    for (int b = 0; ok && b < std::min(2, nchunks); ++b) ok = cudaStreamWaitEvent(st, out_done[b], 0) == cudaSuccess;
    return ok && cudaGetLastError() == cudaSuccess ? BST_OK : BST_ERR_CUDA;
}

}  // extern "C"
