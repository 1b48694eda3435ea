// plan.cu -- plan creation (device tables), argument validation and the
// public entry points of libbst.  The kernels live in bst_forward.cuh (forward BST),
// adjoint.cu (Fourier-slice adjoint and filter gradient) and brute.cu
// (slant-stack comparator).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "bst_internal.h"
#include "bst_twiddle.h"

namespace {

template <class T>
bool upload(T** dptr, const std::vector<T>& host) {
    if (cudaMalloc((void**)dptr, host.size() * sizeof(T)) != cudaSuccess) return false;
    return cudaMemcpy(*dptr, host.data(), host.size() * sizeof(T), cudaMemcpyHostToDevice) == cudaSuccess;
}

void free_plan(bst_plan_s* p) {
    if (!p) return;
    for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
    for (int i = 0; i < bsth::kMaxLanes; ++i) {
        if (p->lane[i]) cudaStreamDestroy(p->lane[i]);
        if (p->ev_join[i]) cudaEventDestroy(p->ev_join[i]);
    }
    if (p->ev_fork) cudaEventDestroy(p->ev_fork);
    for (int i = 0; i < 2; ++i)
        if (p->hs[i]) cudaStreamDestroy(p->hs[i]);
    for (int i = 0; i < 7; ++i)
        if (p->hev[i]) cudaEventDestroy(p->hev[i]);
    cudaFree(p->tw);
    cudaFree(p->dir);
    cudaFree(p->invdth);
    cudaFree(p->lut);
    cudaFree(p->cs64);
    cudaFree(p->cs32);
    cudaFree(p->wq);
    cudaFree(p->err);
    cudaFree(p->cell_start);
    cudaFree(p->cell_pts);
    cudaFree(p->cell_w);
    cudaFree(p->geo_J);
    cudaFree(p->geo_f);
    bst_free_kb(p);
    delete p;
}

float4 split_dir(double c, double s) {
    const float ch = (float)c, sh = (float)s;
    return make_float4(ch, (float)(c - (double)ch), sh, (float)(s - (double)sh));
}

bool ranges_overlap(const void* a, size_t na, const void* b, size_t nb) {
    const uintptr_t a0 = (uintptr_t)a, b0 = (uintptr_t)b;
    return a0 < b0 + nb && b0 < a0 + na;
}

}  // namespace

bool bst_ensure_lanes(bst_plan_s* p) {
    if (p->lane[bsth::kMaxLanes - 1]) return true;
    for (int i = 0; i < bsth::kMaxLanes; ++i) {
        if (!p->lane[i] && cudaStreamCreateWithFlags(&p->lane[i], cudaStreamNonBlocking) != cudaSuccess) return false;
        if (!p->ev_join[i] && cudaEventCreateWithFlags(&p->ev_join[i], cudaEventDisableTiming) != cudaSuccess)
            return false;
    }
    if (!p->ev_fork && cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming) != cudaSuccess) return false;
    return true;
}

void bst_timing_mark(bst_plan_s* p, cudaStream_t st, int stage) {
    if (!p->timing) return;
    if (p->ev_used == p->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        p->ev_pool.push_back(e);
        p->ev_stage.push_back(-1);
    }
    p->ev_stage[p->ev_used] = stage;
    cudaEventRecord(p->ev_pool[p->ev_used], st);
    ++p->ev_used;
}

extern "C" {

bst_status_t bst_plan_set_timing(bst_plan_t p, int enable) {
    if (!p) return BST_ERR_INVALID_ARGUMENT;
    p->timing = enable != 0;
    return BST_OK;
}

bst_status_t bst_plan_timing(bst_plan_t p, double* stage_ms, long long* launches, int n) {
    if (!p || n < 0 || n > 8 || (n > 0 && (!stage_ms || !launches))) return BST_ERR_INVALID_ARGUMENT;
    for (size_t i = 0; i < p->ev_used; ++i)
        if (cudaEventSynchronize(p->ev_pool[i]) != cudaSuccess) return BST_ERR_CUDA;
    for (size_t i = 1; i < p->ev_used; ++i) {
        const int s = p->ev_stage[i];
        if (s < 0) continue;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p->ev_pool[i - 1], p->ev_pool[i]) != cudaSuccess) return BST_ERR_CUDA;
        if (s < 8) {
            p->stage_ms[s] += ms;
            p->stage_launches[s] += 1;
        }
    }
    for (int s = 0; s < n; ++s) {
        stage_ms[s] = p->stage_ms[s];
        launches[s] = p->stage_launches[s];
    }
    for (int s = 0; s < 8; ++s) {
        p->stage_ms[s] = 0.0;
        p->stage_launches[s] = 0;
    }
    p->ev_used = 0;
    return BST_OK;
}

const char* bst_status_string(bst_status_t s) {
    switch (s) {
        case BST_OK: return "ok";
        case BST_ERR_INVALID_ARGUMENT: return "invalid argument";
        case BST_ERR_UNSUPPORTED_SIZE: return "unsupported size (FFT length M = alpha N must be 2^a in [16, 4096] or 3*2^a in [48, 3072], N even)";
        case BST_ERR_WORKSPACE_TOO_SMALL: return "workspace too small";
        case BST_ERR_CUDA: return "CUDA error";
        case BST_ERR_TIMEOUT: return "device-side wait timed out";
        case BST_ERR_OUT_OF_MEMORY: return "out of device memory";
    }
    return "unknown status";
}

bst_status_t bst_plan_create(bst_plan_t* out, int rays, int angles, const float* angles_rad_host, int pad_factor) {
    if (!out) return BST_ERR_INVALID_ARGUMENT;
    *out = nullptr;
    if (!angles_rad_host || angles < 2 || rays < 2) return BST_ERR_INVALID_ARGUMENT;
    if (pad_factor != 1 && pad_factor != 2) return BST_ERR_UNSUPPORTED_SIZE;
    if (rays % 2 != 0) return BST_ERR_UNSUPPORTED_SIZE;
    const int M = pad_factor * rays;
    if (!bsth::supported_fft_length(M)) return BST_ERR_UNSUPPORTED_SIZE;
    std::vector<double> th(angles);
    for (int j = 0; j < angles; ++j) {
        const double v = (double)angles_rad_host[j];
        if (!std::isfinite(v) || v < 0.0 || v >= M_PI) return BST_ERR_INVALID_ARGUMENT;
        if (j > 0 && !(v > th[j - 1])) return BST_ERR_INVALID_ARGUMENT;
        th[j] = v;
    }
    bst_plan_s* p = new (std::nothrow) bst_plan_s();
    if (!p) return BST_ERR_OUT_OF_MEMORY;
    p->N = rays;
    p->V = angles;
    p->M = M;
    p->alpha = pad_factor;
    p->theta = th;
    cudaGetDevice(&p->device);
    const int V = angles;

    // twiddles: the base table, then each radix schedule's per-pass tables
    const std::vector<float2> tw = bst::make_twiddles(M);
    std::vector<double> ext(V + 2);
    ext[0] = th[V - 1] - M_PI;
    for (int j = 0; j < V; ++j) ext[j + 1] = th[j];
    ext[V + 1] = th[0] + M_PI;
    std::vector<float4> dir(V + 2);
    for (int j = 0; j < V; ++j) dir[j + 1] = split_dir(std::cos(th[j]), std::sin(th[j]));
    dir[0] = split_dir(-std::cos(th[V - 1]), -std::sin(th[V - 1]));
    dir[V + 1] = split_dir(-std::cos(th[0]), -std::sin(th[0]));
    std::vector<float> invdth(V + 1);
    for (int J = -1; J <= V - 1; ++J) invdth[J + 1] = (float)(1.0 / (ext[J + 2] - ext[J + 1]));
    const int L = std::max(64, 4 * V);
    std::vector<int> lut(L);
    {
        int cnt = 0;
        for (int b = 0; b < L; ++b) {
            const double start = (double)b * M_PI / (double)L;
            while (cnt < V && th[cnt] <= start) ++cnt;
            lut[b] = cnt - 1;
        }
    }
    std::vector<double2> cs64(V);
    std::vector<float2> cs32(V);
    std::vector<float> wq(V);
    for (int j = 0; j < V; ++j) {
        cs64[j] = make_double2(std::cos(th[j]), std::sin(th[j]));
        cs32[j] = make_float2((float)cs64[j].x, (float)cs64[j].y);
        wq[j] = (float)((ext[j + 2] - ext[j]) / 2.0);
    }
    p->L = L;
    p->lut_scale = (float)((double)L / M_PI);
    {
        // evenly spaced angles: the gridding estimates the bracket arithmetically
        // (the estimate only saves a table lookup; exact tests decide the bracket)
        const double step = (th[V - 1] - th[0]) / (double)(V - 1);
        double dev = 0.0;
        for (int j = 0; j < V; ++j) dev = std::max(dev, std::fabs(th[j] - (th[0] + j * step)));
        p->uniform = (step > 0.0 && dev <= 1e-3 * step) ? 1 : 0;
        p->th0 = (float)th[0];
        p->inv_step = (float)(1.0 / step);
    }
    bool ok = upload(&p->tw, tw) && upload(&p->dir, dir) && upload(&p->invdth, invdth) && upload(&p->lut, lut) &&
              upload(&p->cs64, cs64) && upload(&p->cs32, cs32) && upload(&p->wq, wq);
    if (ok) ok = cudaMalloc((void**)&p->err, sizeof(int)) == cudaSuccess && cudaMemset(p->err, 0, sizeof(int)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_plan(p);
        return BST_ERR_OUT_OF_MEMORY;
    }
    {
        const bst_status_t gs = bst_build_geo_table(p);
        if (gs != BST_OK) {
            cudaGetLastError();
            free_plan(p);
            return gs;
        }
    }
    const size_t per_pair = bsth::fwd_bytes_per_pair(p);
    const size_t budget = (size_t)64 << 20;
    p->chunk_pairs = (int)std::max<size_t>(1, std::min<size_t>(256, budget / per_pair));
    p->chunk_default = p->chunk_pairs;
    // bst_fbp_noalloc's set-up for this device (a failure here leaves the
    // plan usable; bst_fbp_noalloc then retries and reports it)
    if (bst_noalloc_setup_current_device() != BST_OK) cudaGetLastError();
    *out = p;
    return BST_OK;
}

bst_status_t bst_plan_destroy(bst_plan_t p) {
    if (!p) return BST_OK;
    cudaDeviceSynchronize();
    free_plan(p);
    return BST_OK;
}

int bst_plan_fft_length(bst_plan_t p) { return p ? p->M : 0; }

size_t bst_workspace_bytes(bst_plan_t p, int slices) {
    if (!p || slices <= 0) return 0;
    const int pairs = (slices + 1) / 2;
    const int chunk = std::min(pairs, p->chunk_pairs);
    const int nchunks = (pairs + chunk - 1) / chunk;
    const int lanes = std::min(std::min(nchunks, bsth::kMaxLanes), std::max(p->max_lanes, 1));   // chunks in flight
    return (size_t)lanes * chunk * bsth::fwd_bytes_per_pair(p);
}

size_t bst_adjoint_workspace_bytes(bst_plan_t p, int slices) {
    if (!p || slices <= 0) return 0;
    return bst_adjoint_ws(p, slices);
}

size_t brute_workspace_bytes(bst_plan_t p, int slices, int filtered) {
    if (!p || slices <= 0) return 0;
    return bst_brute_ws(p, slices, filtered);
}

static bst_status_t check_io(bst_plan_t p, const float* sino, int slices, const float* vol) {
    if (!p || !sino || !vol || slices <= 0) return BST_ERR_INVALID_ARGUMENT;
    if (!bsth::on_plan_device(p)) return BST_ERR_INVALID_ARGUMENT;
    const size_t ns = (size_t)slices * p->V * p->N * sizeof(float);
    const size_t nv = (size_t)slices * p->N * p->N * sizeof(float);
    if (ranges_overlap(sino, ns, vol, nv)) return BST_ERR_INVALID_ARGUMENT;
    return BST_OK;
}

bst_status_t bst_fbp(bst_plan_t p, const float* d_sino, int slices, const float* d_g, float* d_volume, void* d_ws,
                     size_t ws_bytes, bst_stream_t stream) {
    bst_status_t s = check_io(p, d_sino, slices, d_volume);
    if (s != BST_OK) return s;
    const size_t need = bst_workspace_bytes(p, slices);
    if (!d_ws || ws_bytes < need) return BST_ERR_WORKSPACE_TOO_SMALL;
    return bst_launch_forward(p, d_sino, slices, BSTK_FILTER, d_g, d_volume, d_ws, ws_bytes, (cudaStream_t)stream);
}

bst_status_t bst_backproject(bst_plan_t p, const float* d_sino, int slices, float* d_volume, void* d_ws,
                             size_t ws_bytes, bst_stream_t stream) {
    bst_status_t s = check_io(p, d_sino, slices, d_volume);
    if (s != BST_OK) return s;
    const size_t need = bst_workspace_bytes(p, slices);
    if (!d_ws || ws_bytes < need) return BST_ERR_WORKSPACE_TOO_SMALL;
    return bst_launch_forward(p, d_sino, slices, BSTK_BACKPROJECT, nullptr, d_volume, d_ws, ws_bytes,
                              (cudaStream_t)stream);
}

bst_status_t radon_adjoint(bst_plan_t p, bst_mode_t mode, const float* d_g, const float* d_volume, int slices,
                           float* d_sino, void* d_ws, size_t ws_bytes, bst_stream_t stream) {
    bst_status_t s = check_io(p, d_sino, slices, d_volume);
    if (s != BST_OK) return s;
    if (mode != BST_W_FILTER && mode != BST_W_BACKPROJECT) return BST_ERR_INVALID_ARGUMENT;
    if (p->grid_kind != BST_GRID_BILINEAR) return BST_ERR_INVALID_ARGUMENT;
    const size_t need = bst_adjoint_ws(p, slices);
    if (!d_ws || ws_bytes < need) return BST_ERR_WORKSPACE_TOO_SMALL;
    return bst_launch_adjoint(p, mode == BST_W_FILTER ? BSTK_FILTER : BSTK_BACKPROJECT,
                              mode == BST_W_FILTER ? d_g : nullptr, d_volume, slices, d_sino, d_ws, ws_bytes,
                              (cudaStream_t)stream);
}

bst_status_t bst_fbp_filter_grad(bst_plan_t p, const float* d_sino, const float* d_grad_vol, int slices,
                                 float* d_grad_g, void* d_ws, size_t ws_bytes, bst_stream_t stream) {
    bst_status_t s = check_io(p, d_sino, slices, d_grad_vol);
    if (s != BST_OK) return s;
    if (!d_grad_g || p->grid_kind != BST_GRID_BILINEAR) return BST_ERR_INVALID_ARGUMENT;
    const size_t need = bst_adjoint_ws(p, slices);
    if (!d_ws || ws_bytes < need) return BST_ERR_WORKSPACE_TOO_SMALL;
    return bst_launch_filter_grad(p, d_sino, d_grad_vol, slices, d_grad_g, d_ws, ws_bytes, (cudaStream_t)stream);
}

bst_status_t bst_fbp_backward(bst_plan_t p, const float* d_sino, const float* d_grad_vol, int slices,
                              const float* d_g, float* d_grad_sino, float* d_grad_g, void* d_ws, size_t ws_bytes,
                              bst_stream_t stream) {
    if (!p || !d_grad_vol || slices <= 0 || (!d_grad_sino && !d_grad_g)) return BST_ERR_INVALID_ARGUMENT;
    if (!bsth::on_plan_device(p)) return BST_ERR_INVALID_ARGUMENT;
    if (d_grad_g && !d_sino) return BST_ERR_INVALID_ARGUMENT;
    if (p->grid_kind != BST_GRID_BILINEAR) return BST_ERR_INVALID_ARGUMENT;
    const size_t nv = (size_t)slices * p->N * p->N * sizeof(float), ns = (size_t)slices * p->V * p->N * sizeof(float);
    if (d_grad_sino && ranges_overlap(d_grad_sino, ns, d_grad_vol, nv)) return BST_ERR_INVALID_ARGUMENT;
    if (!d_ws || ws_bytes < bst_adjoint_ws(p, slices)) return BST_ERR_WORKSPACE_TOO_SMALL;
    return bst_launch_backward(p, d_sino, d_grad_vol, slices, d_g, d_grad_sino, d_grad_g, d_ws, (cudaStream_t)stream);
}

bst_status_t brute_backproject(bst_plan_t p, const float* d_sino, int slices, const float* d_g, float* d_volume,
                               void* d_ws, size_t ws_bytes, bst_stream_t stream) {
    bst_status_t s = check_io(p, d_sino, slices, d_volume);
    if (s != BST_OK) return s;
    const size_t need = bst_brute_ws(p, slices, d_g != nullptr);
    if (need > 0 && (!d_ws || ws_bytes < need)) return BST_ERR_WORKSPACE_TOO_SMALL;
    return bst_launch_brute(p, d_sino, slices, d_g, d_volume, d_ws, ws_bytes, (cudaStream_t)stream);
}

bst_status_t bst_plan_set_schedule(bst_plan_t p, int max_radix) {
    if (!p || (max_radix != 8 && max_radix != 16)) return BST_ERR_INVALID_ARGUMENT;
    p->maxr = max_radix;
    return BST_OK;
}

int bst_plan_get_schedule(bst_plan_t p) { return p ? p->maxr : 0; }

bst_status_t bst_plan_set_forward_config(bst_plan_t p, const bst_fwd_config_t* c) {
    if (!p || !c) return BST_ERR_INVALID_ARGUMENT;
    if ((c->max_radix != 8 && c->max_radix != 16) ||
        (c->layout != BST_LAYOUT_PACKED && c->layout != BST_LAYOUT_PAIRED) || c->chunk_pairs < 1 ||
        c->chunk_pairs > 256 || (c->pair_fast != 0 && c->pair_fast != 1) || c->max_lanes < 1 ||
        c->max_lanes > bsth::kMaxLanes || (c->grid_xchg != 0 && c->grid_xchg != 1))
        return BST_ERR_INVALID_ARGUMENT;
    p->maxr = c->max_radix;
    p->fwd_layout = c->layout;
    p->chunk_pairs = c->chunk_pairs;
    p->pair_fast = c->pair_fast;
    p->max_lanes = c->max_lanes;
    p->grid_xchg = c->grid_xchg;
    return BST_OK;
}

bst_status_t bst_plan_get_forward_config(bst_plan_t p, bst_fwd_config_t* c) {
    if (!p || !c) return BST_ERR_INVALID_ARGUMENT;
    c->max_radix = p->maxr;
    c->layout = p->fwd_layout;
    c->chunk_pairs = p->chunk_pairs;
    c->pair_fast = p->pair_fast;
    c->max_lanes = p->max_lanes;
    c->grid_xchg = p->grid_xchg;
    return BST_OK;
}

// The candidate launch shapes of the autotuner: radix 16 or 8, the packed or
// (bilinear plans) paired spectrum layout, for the paired layout the gather
// through shared memory or into registers, and the default chunk in column-fastest
// order or pair-fastest order; where the default chunk is a single pair (the
// workspace of one pair exceeds L2), also chunks of 2, 4 and 8 pairs: the
// launches then fill more waves of blocks, at the price of a workspace (and
// intermediates in HBM) that grows with the chunk.  The lane count stays the
// plan's.
static std::vector<bst_fwd_config_t> tune_candidates(const bst_plan_s* p) {
    std::vector<bst_fwd_config_t> out;
    const int layouts = p->grid_kind == BST_GRID_BILINEAR ? 3 : 1;   // packed, paired, paired + exchange
    for (int r : {16, 8})
        for (int lg = 0; lg < layouts; ++lg) {
            const int l = lg == 0 ? BST_LAYOUT_PACKED : BST_LAYOUT_PAIRED;
            bst_fwd_config_t c{r, l, p->chunk_default, 0, p->max_lanes, lg == 2 ? 1 : 0};
            out.push_back(c);
            if (p->chunk_default == 1) {
                for (int ch : {2, 4, 8}) {
                    c.chunk_pairs = ch;
                    c.pair_fast = 0;
                    out.push_back(c);
                    c.pair_fast = 1;
                    out.push_back(c);
                }
            } else {
                c.pair_fast = 1;
                out.push_back(c);
            }
        }
    return out;
}

bst_status_t bst_plan_autotune(bst_plan_t p, int slices, int* chosen) {
    if (!p) return BST_ERR_INVALID_ARGUMENT;
    if (!bsth::on_plan_device(p)) return BST_ERR_INVALID_ARGUMENT;
    if (slices <= 0) {
        const size_t per = (size_t)p->V * p->N * sizeof(float);
        slices = (int)std::max<size_t>(4, std::min<size_t>(4096, (((size_t)256 << 20) / per) & ~(size_t)1));
    }
    // at least two chunks of the largest candidate on each lane
    slices = std::max(slices, p->chunk_default == 1 ? 2 * 2 * 8 * 2 : 4);
    bst_fwd_config_t old{};
    bst_plan_get_forward_config(p, &old);
    const std::vector<bst_fwd_config_t> cand = tune_candidates(p);
    // workspace for the largest candidate chunk
    size_t nws = 0;
    for (const bst_fwd_config_t& c : cand) {
        bst_plan_set_forward_config(p, &c);
        nws = std::max(nws, bst_workspace_bytes(p, slices));
    }
    bst_plan_set_forward_config(p, &old);
    const size_t nin = (size_t)slices * p->V * p->N, nout = (size_t)slices * p->N * p->N;
    float *in = nullptr, *out = nullptr;
    void* ws = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    bst_status_t st = BST_OK;
    if (cudaMalloc((void**)&in, nin * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void**)&out, nout * sizeof(float)) != cudaSuccess || cudaMalloc(&ws, nws) != cudaSuccess) {
        st = BST_ERR_OUT_OF_MEMORY;
    }
    if (st == BST_OK && (cudaMemset(in, 0, nin * sizeof(float)) != cudaSuccess ||
                         cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        st = BST_ERR_CUDA;
    const bool timing = p->timing;
    p->timing = false;
    bst_fwd_config_t best = old;
    float best_ms = 1e30f;
    for (size_t c = 0; st == BST_OK && c < cand.size(); ++c) {
        bst_plan_set_forward_config(p, &cand[c]);
        float ms_min = 1e30f;
        for (int rep = 0; rep < 4 && st == BST_OK; ++rep) {
            cudaEventRecord(e0, nullptr);
            st = bst_launch_forward(p, in, slices, BSTK_FILTER, nullptr, out, ws, nws, nullptr);
            cudaEventRecord(e1, nullptr);
            if (cudaEventSynchronize(e1) != cudaSuccess) st = BST_ERR_CUDA;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) ms_min = std::min(ms_min, ms);   // the first run warms up
        }
        if (st == BST_OK && ms_min < best_ms) {
            best_ms = ms_min;
            best = cand[c];
        }
    }
    bst_plan_set_forward_config(p, st == BST_OK ? &best : &old);
    p->timing = timing;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(in);
    cudaFree(out);
    cudaFree(ws);
    if (chosen) *chosen = p->maxr;
    return st;
}

bst_status_t bst_plan_status(bst_plan_t p, bst_stream_t stream) {
    if (!p) return BST_ERR_INVALID_ARGUMENT;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return BST_ERR_CUDA;
    int code = 0;
    if (cudaMemcpy(&code, p->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return BST_ERR_CUDA;
    return (bst_status_t)code;
}

}  // extern "C"
