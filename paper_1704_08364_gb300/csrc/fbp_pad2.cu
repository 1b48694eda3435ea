// fbp_pad2.cu -- the forward-path kernels instantiated for pad factor 2
// (ray count N = M / 2 as a compile-time constant).
#include "bst_launch.cuh"

#define BST_FOR_EACH_M(X) \
    X(16) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048) X(4096) X(48) X(96) X(192) X(384) X(768) X(1536) X(3072)

bst_status_t bst_forward_pad2(bst_plan_s* p, const float* sino, int slices, int mode, const float* g, float* vol,
                               void* ws, cudaStream_t st, int max_chunk, int lanes, const bst::PrepArgs* prep) {
    switch (p->M) {
#define BST_CASE(m)                                                                                        \
    case m:                                                                                                \
        return p->maxr == 8                                                                                \
                   ? bst::launch_forward_M<m, 8, m / 2>(p, sino, slices, mode, g, vol, ws, st, max_chunk, lanes, prep) \
                   : bst::launch_forward_M<m, 16, m / 2>(p, sino, slices, mode, g, vol, ws, st, max_chunk, lanes, prep);
        BST_FOR_EACH_M(BST_CASE)
#undef BST_CASE
    }
    return BST_ERR_UNSUPPORTED_SIZE;
}
