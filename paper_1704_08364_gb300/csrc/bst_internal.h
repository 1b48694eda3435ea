// bst_internal.h -- plan object and host-side helpers shared by the
// translation units of libbst (not part of the public ABI).
#pragma once
#include <cuda_runtime.h>

#include <atomic>

#include <vector>

#include "../../include/bst.h"
#include "bst_geo.cuh"

struct bst_plan_s {
    int N = 0, V = 0, M = 0, alpha = 0;
    int device = 0;
    std::vector<double> theta;      // angles as given (float32 widened exactly)
    // device tables owned by the plan
    float2* tw = nullptr;           // [M] exp(-2 pi i m / M)
    float4* dir = nullptr;          // [V+2] angle directions, double-float
    float* invdth = nullptr;        // [V+1]
    int* lut = nullptr;             // [L]
    int L = 0;
    float lut_scale = 0.f;
    int uniform = 0;                // evenly spaced angles (bracket estimate by arithmetic)
    float th0 = 0.f, inv_step = 0.f;
    double2* cs64 = nullptr;        // [V] (cos, sin) in double, slant-stack tile origins
    float2* cs32 = nullptr;         // [V] (cos, sin) in float, slant-stack tile offsets
    float* wq = nullptr;            // [V] trapezoid weights of Eq. 2
    int* err = nullptr;             // sticky device error word
    // gridding geometry of the half grid c' in [0, M/2), [M/2][M], built at plan
    // creation: (bracket J << 16) | floor(rho) (J = -2: the point is zero) and
    // (angle fraction, radius fraction)
    int* geo_J = nullptr;
    float2* geo_f = nullptr;
    // P5 gridding kernel (BST_GRID_BILINEAR or BST_GRID_KAISER_BESSEL) and the
    // KB tables: kernel table, deapodization 1/C per output index, per-strip
    // sample lists and work items (built by bst_plan_set_gridding)
    int grid_kind = 0;
    int kb_w = 0;
    float kb_poly[13] = {0};        // phi as a degree-12 polynomial in t = 2 (2x/W)^2 - 1
    float* kb_dk = nullptr;         // [N]
    int* kb_start = nullptr;        // [kb_nstrips + 1] first work item of each strip
    int* kb_list = nullptr;         // [kb_n] sample ids
    int4* kb_items = nullptr;       // (band, first entry, end entry, 0)
    size_t kb_n = 0;
    int kb_nstrips = 0;
    int chunk_pairs = 1;            // slice pairs per chunk of the forward path
    int chunk_default = 1;          // the chunk sized to about 64 MiB of workspace
    int maxr = 16;                  // FFT radix schedule of the forward path (16 or 8; autotuned)
    int fwd_layout = 0;             // BST_LAYOUT_PACKED or BST_LAYOUT_PAIRED (autotuned)
    int pair_fast = 0;              // gridding blocks ordered pair-fastest (autotuned)
    int max_lanes = 2;              // streams alternating chunks (1 or 2)
    int grid_xchg = 0;              // register-fed paired gridding (0 or 1; autotuned)
    // two plan-owned streams that alternate chunks of the forward path (fork
    // from and join back to the caller's stream with events), created on first use
    cudaStream_t lane[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_join[3] = {nullptr, nullptr, nullptr};
    // bst_fbp_host: upload and download streams and their events, created on first use
    cudaStream_t hs[2] = {nullptr, nullptr};
    cudaEvent_t hev[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    // gridding cell lists for the adjoint, built on first use
    int* cell_start = nullptr;      // [(V+1) M + 1]
    int* cell_pts = nullptr;        // [n] index c * M + r of each Cartesian point
    float2* cell_w = nullptr;       // [n] (fth, frac) of each point
    int cell_n = 0;
    bool cells_built = false;
    // optional per-stage timing: an event after every launch (see bst_plan_set_timing)
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<int> ev_stage;     // stage that ended at each recorded event (-1: start mark)
    size_t ev_used = 0;
    double stage_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    long long stage_launches[8] = {0, 0, 0, 0, 0, 0, 0, 0};

    bst::Geo geo() const {
        bst::Geo g;
        g.dir = dir;
        g.invdth = invdth;
        g.lut = lut;
        g.V = V;
        g.M = M;
        g.L = L;
        g.lut_scale = lut_scale;
        g.uniform = uniform;
        g.th0 = th0;
        g.inv_step = inv_step;
        return g;
    }
};

namespace bsth {

// chunks of the forward path in flight at once, each on its own stream with its
// own workspace (a third one measured no faster than two at 2048^3)
constexpr int kMaxLanes = 2;
static_assert(kMaxLanes <= (int)(sizeof(bst_plan_s::lane) / sizeof(cudaStream_t)) &&
                  kMaxLanes <= (int)(sizeof(bst_plan_s::ev_join) / sizeof(cudaEvent_t)),
              "the plan holds a stream and a join event per lane");

// A plan's tables live on the device that was current at its creation; the
// calls that launch work or build tables for it check that it is current.
inline bool on_plan_device(const bst_plan_s* p) {
    int dev = -1;
    return cudaGetDevice(&dev) == cudaSuccess && dev == p->device;
}

// The opt-in to more than 48 KB of dynamic shared memory is an attribute of a
// kernel on one device.  A launch site keeps one bit per device in `done` and
// runs `set` (which sets its kernels' attributes on the current device) the
// first time it launches on that device; on devices beyond 63 it runs `set`
// every time.
template <class F>
inline bool once_per_device(std::atomic<unsigned long long>& done, F&& set) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    const unsigned long long bit = (dev >= 0 && dev < 64) ? 1ull << dev : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return true;
    if (!set()) return false;
    if (bit) done.fetch_or(bit, std::memory_order_release);
    return true;
}

inline bool supported_fft_length(int M) {
    int m = M;
    if (m % 3 == 0) m /= 3;
    if (m < 16 || (m & (m - 1)) != 0) return false;
    return M >= 16 && M <= 4096;
}

inline bool check_cuda(cudaError_t e) { return e == cudaSuccess; }

// byte sizes of the per-pair workspace of the forward path (one lane)
inline size_t fwd_bytes_per_pair(const bst_plan_s* p) {
    const size_t rows_t = (size_t)((p->N + 3) / 4) * 4;
    return ((size_t)p->V * p->M + rows_t * p->M) * sizeof(float2);
}

}  // namespace bsth

// Record a timing mark on `st` after a launch of `stage` (or a start mark
// with stage -1).  No-op unless timing is enabled on the plan.
void bst_timing_mark(bst_plan_s* p, cudaStream_t st, int stage);

// launchers (one dispatch on M each), defined in the kernel translation units
bst_status_t bst_launch_forward(bst_plan_s* p, const float* sino, int slices, int mode, const float* g,
                                float* vol, void* ws, size_t ws_bytes, cudaStream_t st);
// as bst_launch_forward, with at most max_chunk slice pairs per chunk of the
// workspace and up to `lanes` (1 or 2) streams alternating the chunks
bst_status_t bst_launch_forward_chunked(bst_plan_s* p, const float* sino, int slices, int mode, const float* g,
                                        float* vol, void* ws, cudaStream_t st, int max_chunk, int lanes);
namespace bst {
struct PrepArgs;
}
// as bst_launch_forward (filter mode) with the pre-reconstruction stages in the ray kernel
bst_status_t bst_launch_forward_prep(bst_plan_s* p, const float* sino, int slices, const bst::PrepArgs& prep,
                                     const float* g, float* vol, void* ws, size_t ws_bytes, cudaStream_t st);
// the forward path for pad factor 1 or 2 (fbp_pad1.cu, fbp_pad2.cu); prep may be null
bst_status_t bst_forward_pad1(bst_plan_s* p, const float* sino, int slices, int mode, const float* g, float* vol,
                              void* ws, cudaStream_t st, int max_chunk, int lanes, const bst::PrepArgs* prep);
bst_status_t bst_forward_pad2(bst_plan_s* p, const float* sino, int slices, int mode, const float* g, float* vol,
                              void* ws, cudaStream_t st, int max_chunk, int lanes, const bst::PrepArgs* prep);
// create the plan's two chunk streams and their events (false on failure)
bool bst_ensure_lanes(bst_plan_s* p);
bst_status_t bst_launch_adjoint(bst_plan_s* p, int mode, const float* g, const float* vol, int slices,
                                float* sino, void* ws, size_t ws_bytes, cudaStream_t st);
bst_status_t bst_launch_filter_grad(bst_plan_s* p, const float* sino, const float* gvol, int slices,
                                    float* grad_g, void* ws, size_t ws_bytes, cudaStream_t st);
bst_status_t bst_launch_backward(bst_plan_s* p, const float* sino, const float* gvol, int slices, const float* g,
                                 float* grad_sino, float* grad_g, void* ws, cudaStream_t st);
bst_status_t bst_launch_brute(bst_plan_s* p, const float* sino, int slices, const float* g, float* vol,
                              void* ws, size_t ws_bytes, cudaStream_t st);
bst_status_t bst_build_cells(bst_plan_s* p, cudaStream_t st);
bst_status_t bst_build_geo_table(bst_plan_s* p);
// KB gridding + column inverse FFT of np pairs (kb.cu)
bst_status_t bst_launch_kb_col(bst_plan_s* p, const float2* Z, float2* T, int np, cudaStream_t st);
void bst_free_kb(bst_plan_s* p);
double bst_bessel_i0(double x);
// look up (and cache) the device address of bst_fbp_noalloc's scratch array
// on the current device (noalloc.cu); called by bst_plan_create
bst_status_t bst_noalloc_setup_current_device();
size_t bst_adjoint_ws(const bst_plan_s* p, int slices);
size_t bst_brute_ws(const bst_plan_s* p, int slices, int filtered);

// mode values shared by the launchers
enum { BSTK_FILTER = 0, BSTK_BACKPROJECT = 1, BSTK_RAW = 2 };
// flag or-ed into the ray-stage mode: also multiply by the polar cell area
// |k| (1/4 at k = 0) for KB gridding
enum { BSTK_KBW = 8 };
// flag or-ed into the ray-stage mode: write the spectrum in the paired
// (Z[k], Z[-k]) layout read by the paired bilinear gridding kernel
enum { BSTK_PAIRED = 16 };
