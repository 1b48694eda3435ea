// ragged.cu -- a batch of sinograms of mixed sizes reconstructed by one
// persistent launch (optionally replayed from a CUDA graph).
//
// Items that share a plan are paired (two slices per complex line, as in the
// per-size path).  Every pair-item is cut into units of the three stages of
// the forward path (ray FFT, gridding + column inverse FFT, row inverse FFT).
// One 1024-thread block per SM runs two independent 512-thread workers; each
// worker claims units from a queue in which every unit comes after the units
// it depends on, and synchronises its threads with its own named barrier, so
// the two workers of an SM never wait on each other's FFT passes.  A unit
// fills one worker: for FFT length M (TPL = M/16 or M/12 threads per line)
// 512 / TPL ray lines, 256 / TPL Cartesian column pairs of the paired
// spectrum layout (the per-size path's faster gridding kernel), or 512 / TPL
// rows (tiles of four rows, or of two where four lines exceed the worker).
// A unit of stage 2 or 3 first waits until the previous stage of its item has
// completed: the worker's first thread spins on the item's completion counter
// with an acquire load and a bounded number of iterations; if the bound is
// reached it records BST_ERR_TIMEOUT in the batch's error word and the worker
// leaves its loop, so the launch always ends.  The launch is cooperative,
// which guarantees that all blocks are resident (a unit is only waited on
// after it has been claimed by a running worker).  Each pair-item owns its own
// workspace region, so no block can hold stale cached lines of data another
// block writes in the launch.
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
    float2* Z;        // [V][M] (paired layout)
    float2* T;        // [ceil(N/4)][M][4]
    const float2* tw;
    const int* gJ;
    const float2* gF;
    int M, N, V, maxr;
    float scale, two_alpha;
    int n[3];         // units per stage
};

constexpr int RAGGED_THREADS = 1024;
constexpr int RAGGED_WORKERS = 2;
constexpr int RAGGED_WT = RAGGED_THREADS / RAGGED_WORKERS;   // threads per worker

// unit shapes per FFT length
template <int M> __host__ __device__ constexpr int r_ray_lines() { return RAGGED_WT / tpl_of<M>(); }
template <int M> __host__ __device__ constexpr int r_grid_pairs() { return RAGGED_WT / (2 * tpl_of<M>()); }
template <int M> __host__ __device__ constexpr int r_row_rpt() { return 4 * tpl_of<M>() <= RAGGED_WT ? 4 : 2; }
template <int M> __host__ __device__ constexpr int r_row_tiles() { return RAGGED_WT / (r_row_rpt<M>() * tpl_of<M>()); }

// shared memory of one worker (float2 elements): the largest of its units
template <int M> __host__ __device__ constexpr size_t r_worker_smem() {
    const size_t a = (size_t)r_ray_lines<M>() * smem_line_len(M);
    const size_t b = (size_t)2 * r_grid_pairs<M>() * smem_line_len(M);
    const size_t c = (size_t)r_row_rpt<M>() * r_row_tiles<M>() * row_line_stride<M>();
    return a > b ? (a > c ? a : c) : (b > c ? b : c);
}

#define BST_RAGGED_SIZES(X) X(256) X(512) X(768) X(1024) X(1536) X(2048) X(3072) X(4096)

__host__ __device__ constexpr size_t r_max_worker_smem() {
    size_t m = 0;
#define BST_SM(mm) m = m > r_worker_smem<mm>() ? m : r_worker_smem<mm>();
    BST_RAGGED_SIZES(BST_SM)
#undef BST_SM
    return m;
}

// stage units, not inlined, so that every (length, schedule, stage) variant
// keeps its own register allocation inside the 64-register budget of the
// kernel (inlining them all spills kilobytes).  NC = M/2 serves items of pad
// factor 2 (N known at compile time: the first pass skips the zero padding and
// the last the dropped outputs, as in the per-size kernels); NC = 0 the others.
template <int M, int MAXR, int NC>
__device__ __noinline__ void ray_u(float2* smem, const RItem& it, int u, const WorkerSync& sync, int tid) {
    constexpr int TPL = tpl_of<M>(), L = r_ray_lines<M>();
    ray_unit<M, TPL, L, MAXR, NC, WorkerSync>(smem, u * L, it.V, it.N, it.sa, it.sb, BSTK_FILTER | BSTK_PAIRED, it.g,
                                              it.two_alpha, it.Z, it.tw, sync, tid);
}
template <int M, int MAXR, int NC>
__device__ __noinline__ void grid_u(float2* smem, const RItem& it, int u, const WorkerSync& sync, int tid) {
    constexpr int TPL = tpl_of<M>(), CP = r_grid_pairs<M>();
    grid_unit_paired<M, TPL, CP, MAXR, NC, 2, WorkerSync>(smem, u * CP, it.V, it.N,
                                                          reinterpret_cast<const float4*>(it.Z), it.gJ, it.gF, it.T,
                                                          it.tw, sync, tid);
}
template <int M, int MAXR, int NC>
__device__ __noinline__ void row_u(float2* smem, const RItem& it, int u, const WorkerSync& sync, int tid) {
    constexpr int TPL = tpl_of<M>(), TT = r_row_tiles<M>(), RPT = r_row_rpt<M>();
    row_unit<M, TPL, TT, MAXR, NC, WorkerSync, RPT>(smem, u * TT, it.N, it.T, it.va, it.vb, it.scale, it.tw,
                                                    nullptr, sync, tid);
}
template <int M, int MAXR, int NC>
__device__ __forceinline__ void run_unit_nc(float2* smem, const RItem& it, int stage, int u, const WorkerSync& sync,
                                            int tid) {
    if (stage == 0) ray_u<M, MAXR, NC>(smem, it, u, sync, tid);
    else if (stage == 1) grid_u<M, MAXR, NC>(smem, it, u, sync, tid);
    else row_u<M, MAXR, NC>(smem, it, u, sync, tid);
}
template <int M, int MAXR>
__device__ __forceinline__ void run_unit(float2* smem, const RItem& it, int stage, int u, const WorkerSync& sync,
                                         int tid) {
    if (2 * it.N == M) run_unit_nc<M, MAXR, M / 2>(smem, it, stage, u, sync, tid);
    else run_unit_nc<M, MAXR, 0>(smem, it, stage, u, sync, tid);
}

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__global__ void __launch_bounds__(RAGGED_THREADS, 1)
    k_ragged(const RItem* __restrict__ items, const int4* __restrict__ queue, int nq, int* __restrict__ next,
             int* __restrict__ done, int* __restrict__ err, int spin_limit) {
    extern __shared__ float2 smem[];
    __shared__ int s_u[RAGGED_WORKERS], s_ok[RAGGED_WORKERS];
    const int wk = threadIdx.x / RAGGED_WT;
    const int tid = threadIdx.x % RAGGED_WT;
    const WorkerSync sync{1 + wk, RAGGED_WT};
    float2* wsm = smem + (size_t)wk * r_max_worker_smem();
    int claimed = -1;   // thread 0: the entry claimed ahead of time
    for (;;) {
        sync();   // the worker's previous entry is done with its shared memory and s_u
        if (tid == 0) s_u[wk] = claimed >= 0 ? claimed : atomicAdd(next, 1);
        sync();
        const int u = s_u[wk];
        if (u >= nq) break;
        // claim the next entry now, so that the atomic's latency overlaps this
        // entry's work (claims stay in queue order per worker: the oldest
        // claimed, unfinished entry is always some worker's current one)
        if (tid == 0) claimed = atomicAdd(next, 1);
        const int4 w = queue[u];   // (pair-item, stage, first unit, units)
        const RItem& it = items[w.x];
        if (w.y > 0) {
            if (tid == 0) {
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
                s_ok[wk] = ok;
            }
            sync();
            if (!s_ok[wk]) break;
        }
        for (int k = 0; k < w.w; ++k) {
            if (k > 0) sync();   // the previous unit is done with the shared memory
            switch (it.M) {
#define BST_UNIT(m)                                                                \
    case m:                                                                        \
        if (it.maxr == 8) run_unit<m, 8>(wsm, it, w.y, w.z + k, sync, tid);        \
        else run_unit<m, 16>(wsm, it, w.y, w.z + k, sync, tid);                    \
        break;
                BST_RAGGED_SIZES(BST_UNIT)
#undef BST_UNIT
                default:
                    break;
            }
        }
        sync();
        if (tid == 0 && w.y < 2) {
            // release: the worker's writes of these units (ordered before by its
            // barrier) become visible to a unit that acquires the counter
            asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(done + 3 * w.x + w.y), "r"(w.w)
                         : "memory");
        }
    }
}

__host__ size_t ragged_smem_bytes() { return (size_t)RAGGED_WORKERS * r_max_worker_smem() * sizeof(float2); }

__host__ bool ragged_supported(int M) {
    switch (M) {
#define BST_C(mm) case mm: return true;
        BST_RAGGED_SIZES(BST_C)
#undef BST_C
    }
    return false;
}

// units per stage of an item of FFT length M, N rays and V angles
__host__ void ragged_units(int M, int N, int V, int* n) {
    const int tpl = (M % 3 == 0) ? M / 12 : M / 16;
    const int lines = RAGGED_WT / tpl;                  // ray lines per unit
    const int pairs = RAGGED_WT / (2 * tpl);            // column pairs per unit
    const int rows = RAGGED_WT / tpl;                   // rows per unit (tiles x rows per tile)
    n[0] = (V + lines - 1) / lines;
    n[1] = (M / 2 + pairs - 1) / pairs;
    n[2] = (N + rows - 1) / rows;
}

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
        bst::ragged_units(p->M, p->N, p->V, x.n);
    }
    // queue of entries (pair-item, stage, first unit, units), each entry a run
    // of up to RAGGED_RUN units of one stage (every unit is 8192 points of FFT
    // work whatever the length, so entries are of about equal size); an entry
    // always follows the entries it depends on.  Default: phases (every ray
    // entry, then every gridding entry, then every row entry), the largest
    // pair-items first within a phase.  Flag bit 1: stage s of pair-item k at
    // step k + s (neighbouring items overlap).
    // (runs of RAGGED_RUN units for lengths of 2048 and more, whose items have
    // units enough to fill every worker; single units for the others)
    constexpr int RAGGED_RUN = 4;
    std::vector<int4> q;
    const bool skip0 = (flags & 1) != 0;   // diagnostic: leave pair-item 0's ray stage unqueued
    auto push_stage = [&](int k, int s) {
        if (s == 0 && k == 0 && skip0) return;
        const int run = it[k].M >= 2048 ? RAGGED_RUN : 1;
        for (int u = 0; u < it[k].n[s]; u += run) q.push_back(make_int4(k, s, u, std::min(run, it[k].n[s] - u)));
    };
    if (!(flags & 2)) {
        std::vector<int> order(pairs);
        for (int k = 0; k < pairs; ++k) order[k] = k;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
            return (size_t)it[a].M * it[a].V > (size_t)it[b].M * it[b].V;
        });
        for (int s = 0; s < 3; ++s)
            for (int k : order) push_stage(k, s);
    } else {
        for (int step = 0; step < pairs + 2; ++step)
            for (int s = 0; s < 3; ++s) {
                const int k = step - s;
                if (k >= 0 && k < pairs) push_stage(k, s);
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
