// ragged.cu -- a batch of sinograms of mixed sizes reconstructed by one
// persistent launch (optionally replayed from a CUDA graph).
//
// Items that share a plan are paired (two slices per complex line, as in the
// per-size path).  Every pair-item is cut into units of the three stages of
// the forward path (ray FFT, gridding + column inverse FFT, row inverse FFT),
// each unit filling a 1024-thread block.  One block per SM claims units from
// a queue in which every unit comes after the units it depends on: stage s
// of pair-item p is queued at step p + s, so neighbouring items overlap.  A
// unit of stage 2 or 3 first waits until the previous stage of its item has
// completed: one thread spins on the item's completion counter with an acquire
// load and a bounded number of iterations; if the bound is reached it records
// BST_ERR_TIMEOUT in the batch's error word and the block leaves the loop, so
// the launch always ends.  The launch is cooperative, which guarantees that all
// blocks are resident (a unit is only waited on after it has been claimed by a
// running block).  Each pair-item owns its own workspace region, so no block
// can hold stale cached lines of data another block writes in the launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <new>
#include <vector>

#include "bst_stages.cuh"

namespace bst {

struct RItem {
    const float* sa;  // slice a sinogram [V][N]
    const float* sb;  // slice b sinogram or null
    float* va;        // slice a volume [N][N]
    float* vb;        // slice b volume or null
    const float* g;   // filter taps [M/2] or null (ramp)
    float2* Z;        // [V][M]
    float2* T;        // [ceil(N/4)][M][4]
    const float2* tw;
    const int* gJ;
    const float2* gF;
    int M, N, V, maxr;
    float scale, two_alpha;
    int n[3];         // units per stage
};

constexpr int RAGGED_THREADS = 1024;

template <int M> __host__ __device__ constexpr int r_lines() { return RAGGED_THREADS / tpl_of<M>(); }

template <int M> __host__ __device__ constexpr size_t r_smem() {
    return (size_t)(r_lines<M>() * smem_line_len(M) > 4 * (r_lines<M>() / 4) * row_line_stride<M>()
                        ? r_lines<M>() * smem_line_len(M)
                        : 4 * (r_lines<M>() / 4) * row_line_stride<M>()) *
           sizeof(float2);
}

// stage units, not inlined, so that every (length, schedule, stage) variant
// keeps its own register allocation inside the 64-register budget of the kernel
template <int M, int MAXR>
__device__ __noinline__ void ray_u(float2* smem, const RItem& it, int u) {
    constexpr int TPL = tpl_of<M>(), L = r_lines<M>();
    ray_unit<M, TPL, L, MAXR>(smem, u * L, it.V, it.N, it.sa, it.sb, BSTK_FILTER, it.g, it.two_alpha, it.Z, it.tw);
}
template <int M, int MAXR>
__device__ __noinline__ void grid_u(float2* smem, const RItem& it, int u) {
    constexpr int TPL = tpl_of<M>(), L = r_lines<M>();
    grid_unit<M, TPL, L, MAXR>(smem, u * L, it.V, it.N, it.Z, it.gJ, it.gF, it.T, it.tw);
}
template <int M, int MAXR>
__device__ __noinline__ void row_u(float2* smem, const RItem& it, int u) {
    constexpr int TPL = tpl_of<M>(), L = r_lines<M>();
    row_unit<M, TPL, L / 4, MAXR>(smem, u * (L / 4), it.N, it.T, it.va, it.vb, it.scale, it.tw);
}
template <int M, int MAXR>
__device__ __forceinline__ void run_unit(float2* smem, const RItem& it, int stage, int u) {
    if (stage == 0) ray_u<M, MAXR>(smem, it, u);
    else if (stage == 1) grid_u<M, MAXR>(smem, it, u);
    else row_u<M, MAXR>(smem, it, u);
}

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

#define BST_RAGGED_SIZES(X) X(256) X(512) X(768) X(1024) X(1536) X(2048) X(3072) X(4096)

__global__ void __launch_bounds__(RAGGED_THREADS, 1)
    k_ragged(const RItem* __restrict__ items, const int4* __restrict__ queue, int nq, int* __restrict__ next,
             int* __restrict__ done, int* __restrict__ err, int spin_limit) {
    extern __shared__ float2 smem[];
    __shared__ int s_u, s_ok;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_u = atomicAdd(next, 1);
        __syncthreads();
        const int u = s_u;
        if (u >= nq) break;
        const int4 w = queue[u];   // (pair-item, stage, unit)
        const RItem& it = items[w.x];
        if (w.y > 0) {
            if (threadIdx.x == 0) {
                const int need = it.n[w.y - 1];
                const int* c = done + 3 * w.x + (w.y - 1);
                int ok = 1, n = 0;
                while (ld_acquire(c) < need) {
                    if (++n > spin_limit || *(volatile int*)err != 0) {
                        atomicCAS(err, 0, (int)BST_ERR_TIMEOUT);
                        ok = 0;
                        break;
                    }
                    __nanosleep(256);
                }
                s_ok = ok;
            }
            __syncthreads();
            if (!s_ok) break;
        }
        switch (it.M) {
#define BST_UNIT(m)                                         \
    case m:                                                 \
        if (it.maxr == 8) run_unit<m, 8>(smem, it, w.y, w.z); \
        else run_unit<m, 16>(smem, it, w.y, w.z);           \
        break;
            BST_RAGGED_SIZES(BST_UNIT)
#undef BST_UNIT
            default:
                break;
        }
        __syncthreads();
        if (threadIdx.x == 0 && w.y < 2) {
            // release: the block's writes of this unit (ordered before by the
            // barrier) become visible to a unit that acquires the counter
            asm volatile("red.release.gpu.global.add.s32 [%0], 1;" ::"l"(done + 3 * w.x + w.y) : "memory");
        }
    }
}

__host__ size_t ragged_smem_bytes() {
    size_t m = 0;
#define BST_SM(mm) m = std::max(m, r_smem<mm>());
    BST_RAGGED_SIZES(BST_SM)
#undef BST_SM
    return m;
}

__host__ bool ragged_supported(int M) {
    switch (M) {
#define BST_C(mm) case mm: return true;
        BST_RAGGED_SIZES(BST_C)
#undef BST_C
    }
    return false;
}

__host__ int ragged_lines(int M) { return RAGGED_THREADS / ((M % 3 == 0) ? M / 12 : M / 16); }

}  // namespace bst

struct bst_ragged_s {
    int items = 0;
    std::vector<bst_plan_t> plans;             // per item
    std::vector<int> first, second;            // items of each pair-item (second -1: none)
    std::vector<size_t> ws_off;                // element offset (float2) of each pair-item's workspace
    size_t ws_elems = 0;
    bst::RItem* d_items = nullptr;
    int4* d_queue = nullptr;
    int nq = 0;
    int* d_ctr = nullptr;                      // next, then 3 counters per pair-item
    int* d_err = nullptr;
    int spin_limit = 1 << 22;
    int grid = 0;
    size_t smem = 0;
    bool bound = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

void drop_graph(bst_ragged_s* r) {
    if (r->exec) cudaGraphExecDestroy(r->exec);
    if (r->graph) cudaGraphDestroy(r->graph);
    r->exec = nullptr;
    r->graph = nullptr;
}

bst_status_t enqueue(bst_ragged_s* r, cudaStream_t st) {
    const int pairs = (int)r->first.size();
    if (cudaMemsetAsync(r->d_ctr, 0, (size_t)(1 + 3 * pairs) * sizeof(int), st) != cudaSuccess) return BST_ERR_CUDA;
    int* next = r->d_ctr;
    int* done = r->d_ctr + 1;
    const bst::RItem* items = r->d_items;
    const int4* queue = r->d_queue;
    int nq = r->nq;
    int* err = r->d_err;
    int spin = r->spin_limit;
    void* args[] = {(void*)&items, (void*)&queue, (void*)&nq, (void*)&next, (void*)&done, (void*)&err, (void*)&spin};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(r->grid);
    cfg.blockDim = dim3(bst::RAGGED_THREADS);
    cfg.dynamicSmemBytes = r->smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelExC(&cfg, (const void*)bst::k_ragged, args) != cudaSuccess) return BST_ERR_CUDA;
    return BST_OK;
}

}  // namespace

extern "C" {

bst_status_t bst_ragged_create(bst_ragged_t* out, int items, const bst_plan_t* plans) {
    if (!out) return BST_ERR_INVALID_ARGUMENT;
    *out = nullptr;
    if (items <= 0 || !plans) return BST_ERR_INVALID_ARGUMENT;
    for (int i = 0; i < items; ++i) {
        if (!plans[i] || !bsth::on_plan_device(plans[i])) return BST_ERR_INVALID_ARGUMENT;
        if (!bst::ragged_supported(plans[i]->M)) return BST_ERR_UNSUPPORTED_SIZE;
    }
    bst_ragged_s* r = new (std::nothrow) bst_ragged_s();
    if (!r) return BST_ERR_OUT_OF_MEMORY;
    r->items = items;
    r->plans.assign(plans, plans + items);
    // pair items of the same plan in input order
    std::vector<int> open_slot(items, -1);
    for (int i = 0; i < items; ++i) {
        int slot = -1;
        for (size_t k = 0; k < r->first.size(); ++k)
            if (r->second[k] < 0 && r->plans[r->first[k]] == plans[i]) {
                slot = (int)k;
                break;
            }
        if (slot >= 0) {
            r->second[slot] = i;
        } else {
            r->first.push_back(i);
            r->second.push_back(-1);
        }
    }
    for (size_t k = 0; k < r->first.size(); ++k) {
        const bst_plan_s* p = plans[r->first[k]];
        r->ws_off.push_back(r->ws_elems);
        r->ws_elems += (size_t)p->V * p->M + (size_t)((p->N + 3) / 4) * 4 * p->M;
        r->ws_elems = (r->ws_elems + 31) & ~(size_t)31;
    }
    if (const char* e = std::getenv("BST_SPIN_LIMIT")) r->spin_limit = std::max(1, atoi(e));
    r->smem = bst::ragged_smem_bytes();
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaFuncSetAttribute((const void*)bst::k_ragged, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)r->smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)bst::k_ragged, bst::RAGGED_THREADS,
                                                      r->smem) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        delete r;
        return BST_ERR_CUDA;
    }
    r->grid = sms * per_sm;
    const int pairs = (int)r->first.size();
    if (cudaMalloc((void**)&r->d_ctr, (size_t)(1 + 3 * pairs) * sizeof(int)) != cudaSuccess ||
        cudaMalloc((void**)&r->d_err, sizeof(int)) != cudaSuccess ||
        cudaMalloc((void**)&r->d_items, (size_t)pairs * sizeof(bst::RItem)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(r->d_ctr);
        cudaFree(r->d_err);
        delete r;
        return BST_ERR_OUT_OF_MEMORY;
    }
    cudaMemset(r->d_err, 0, sizeof(int));
    *out = r;
    return BST_OK;
}

size_t bst_ragged_workspace_bytes(bst_ragged_t r) { return r ? r->ws_elems * sizeof(float2) + 256 : 0; }

int bst_ragged_pair_items(bst_ragged_t r) { return r ? (int)r->first.size() : 0; }

bst_status_t bst_ragged_bind(bst_ragged_t r, const float* const* d_sinos, const float* const* d_g,
                             float* const* d_volumes, void* d_ws, size_t ws_bytes, int flags) {
    if (!r || !d_sinos || !d_volumes) return BST_ERR_INVALID_ARGUMENT;
    if (!bsth::on_plan_device(r->plans[0])) return BST_ERR_INVALID_ARGUMENT;
    if (!d_ws || ws_bytes < bst_ragged_workspace_bytes(r)) return BST_ERR_WORKSPACE_TOO_SMALL;
    for (int i = 0; i < r->items; ++i)
        if (!d_sinos[i] || !d_volumes[i]) return BST_ERR_INVALID_ARGUMENT;
    const int pairs = (int)r->first.size();
    std::vector<bst::RItem> it(pairs);
    for (int k = 0; k < pairs; ++k) {
        const int a = r->first[k], b = r->second[k];
        const bst_plan_s* p = r->plans[a];
        if (p->grid_kind != BST_GRID_BILINEAR) return BST_ERR_INVALID_ARGUMENT;
        const float* ga = d_g ? d_g[a] : nullptr;
        const float* gb = (d_g && b >= 0) ? d_g[b] : nullptr;
        if (b >= 0 && ga != gb) return BST_ERR_INVALID_ARGUMENT;   // a pair shares its filter
        bst::RItem& x = it[k];
        x.sa = d_sinos[a];
        x.sb = b >= 0 ? d_sinos[b] : nullptr;
        x.va = d_volumes[a];
        x.vb = b >= 0 ? d_volumes[b] : nullptr;
        x.g = ga;
        x.Z = (float2*)d_ws + r->ws_off[k];
        x.T = x.Z + (size_t)p->V * p->M;
        x.tw = p->tw;
        x.gJ = p->geo_J;
        x.gF = p->geo_f;
        x.M = p->M;
        x.N = p->N;
        x.V = p->V;
        x.maxr = p->maxr;
        x.scale = (float)((double)p->N / (2.0 * (double)p->M * (double)p->M));
        x.two_alpha = (float)(2 * p->alpha);
        const int L = bst::ragged_lines(p->M);
        x.n[0] = (p->V + L - 1) / L;
        x.n[1] = (p->M / 2 + L - 1) / L;
        x.n[2] = ((p->N + 3) / 4 + L / 4 - 1) / (L / 4);
    }
    // queue; a unit always follows its dependencies.  Default: phases (every
    // ray unit, then every gridding unit, then every row unit), the largest
    // pair-items first within a phase (measured 6 % faster on a 64-item batch).
    // Flag bit 1: stage s of pair-item k at step k + s (neighbouring items overlap).
    std::vector<int4> q;
    const bool skip0 = (flags & 1) != 0;   // diagnostic: leave pair-item 0's ray stage unqueued
    if (!(flags & 2)) {
        std::vector<int> order(pairs);
        for (int k = 0; k < pairs; ++k) order[k] = k;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
            return (size_t)it[a].M * it[a].V > (size_t)it[b].M * it[b].V;
        });
        for (int s = 0; s < 3; ++s)
            for (int k : order) {
                if (s == 0 && k == 0 && skip0) continue;
                for (int u = 0; u < it[k].n[s]; ++u) q.push_back(make_int4(k, s, u, 0));
            }
    } else {
        for (int step = 0; step < pairs + 2; ++step)
            for (int s = 0; s < 3; ++s) {
                const int k = step - s;
                if (k < 0 || k >= pairs) continue;
                if (s == 0 && k == 0 && skip0) continue;
                for (int u = 0; u < it[k].n[s]; ++u) q.push_back(make_int4(k, s, u, 0));
            }
    }
    int4* dq = nullptr;
    if (cudaMalloc((void**)&dq, std::max<size_t>(1, q.size()) * sizeof(int4)) != cudaSuccess)
        return BST_ERR_OUT_OF_MEMORY;
    if (cudaMemcpy(dq, q.data(), q.size() * sizeof(int4), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(r->d_items, it.data(), it.size() * sizeof(bst::RItem), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(dq);
        return BST_ERR_CUDA;
    }
    cudaFree(r->d_queue);
    r->d_queue = dq;
    r->nq = (int)q.size();
    drop_graph(r);
    r->bound = true;
    return BST_OK;
}

bst_status_t bst_ragged_set_spin_limit(bst_ragged_t r, int iterations) {
    if (!r || iterations < 1) return BST_ERR_INVALID_ARGUMENT;
    r->spin_limit = iterations;
    drop_graph(r);
    return BST_OK;
}

bst_status_t bst_ragged_fbp(bst_ragged_t r, int use_graph, bst_stream_t stream) {
    if (!r || !r->bound) return BST_ERR_INVALID_ARGUMENT;
    if (!bsth::on_plan_device(r->plans[0])) return BST_ERR_INVALID_ARGUMENT;
    cudaStream_t st = (cudaStream_t)stream;
    if (!use_graph) return enqueue(r, st);
    if (!r->exec) {
        cudaStream_t cap;
        if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return BST_ERR_CUDA;
        bst_status_t s = BST_OK;
        if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) s = BST_ERR_CUDA;
        if (s == BST_OK) s = enqueue(r, cap);
        cudaGraph_t g = nullptr;
        if (cudaStreamEndCapture(cap, &g) != cudaSuccess || !g) s = BST_ERR_CUDA;
        cudaStreamDestroy(cap);
        if (s != BST_OK) {
            cudaGetLastError();
            if (g) cudaGraphDestroy(g);
            return s;
        }
        if (cudaGraphInstantiate(&r->exec, g, 0) != cudaSuccess) {
            cudaGraphDestroy(g);
            cudaGetLastError();
            return BST_ERR_CUDA;
        }
        r->graph = g;
    }
    return cudaGraphLaunch(r->exec, st) == cudaSuccess ? BST_OK : BST_ERR_CUDA;
}

bst_status_t bst_ragged_status(bst_ragged_t r, bst_stream_t stream) {
    if (!r) return BST_ERR_INVALID_ARGUMENT;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return BST_ERR_CUDA;
    int code = 0;
    if (cudaMemcpy(&code, r->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return BST_ERR_CUDA;
    if (code != 0) cudaMemset(r->d_err, 0, sizeof(int));
    return (bst_status_t)code;
}

bst_status_t bst_ragged_destroy(bst_ragged_t r) {
    if (!r) return BST_OK;
    cudaDeviceSynchronize();
    drop_graph(r);
    cudaFree(r->d_items);
    cudaFree(r->d_queue);
    cudaFree(r->d_ctr);
    cudaFree(r->d_err);
    delete r;
    return BST_OK;
}

}  // extern "C"
