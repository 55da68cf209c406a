// Host entry points of libdiffcloud.so (declared in include/diffcloud.h).
#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "dc_internal.cuh"

namespace dc {

// ---------------------------------------------------------------------------------------
// bookkeeping: launch count, Chamfer-kernel event timing
// ---------------------------------------------------------------------------------------
static std::atomic<long long> g_launches{0};
void count_launch(int n) { g_launches += n; }

static std::mutex g_prof_mu;
static bool g_prof_on = false;
static int g_prof_cap = 0, g_prof_n = 0;
static std::vector<cudaEvent_t> g_prof_ev;

void prof_before(cudaStream_t s) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (g_prof_on && g_prof_n < g_prof_cap) cudaEventRecord(g_prof_ev[2 * g_prof_n], s);
}
void prof_after(cudaStream_t s) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (g_prof_on && g_prof_n < g_prof_cap) {
        cudaEventRecord(g_prof_ev[2 * g_prof_n + 1], s);
        ++g_prof_n;
    }
}

// ---------------------------------------------------------------------------------------
// workspace layout
// ---------------------------------------------------------------------------------------
Layout make_layout(const Sizes& s) {
    Layout L{};
    size_t off = 0;
    auto take = [&](long long bytes) {
        size_t o = off;
        off += ((size_t)(bytes > 0 ? bytes : 0) + 255) / 256 * 256;
        return o;
    };
    L.hdr = take(sizeof(WsHeader));
    L.frames = take(s.n_frames * (long long)sizeof(FrameDesc));
    L.rowpre = take((s.n_frames + 1) * 4);
    L.colpre = take((s.n_frames + 1) * 4);
    L.unit_frame = take(s.n_units * 4);
    L.unit_rb = take(s.n_units * 4);
    L.unit_pre = take((s.n_units + 1) * 4);
    L.cdf = take(s.sum_f * 4);
    L.x = take(s.rows * 16);
    L.fw = take(s.rows * 16);
    L.tsoa = take(6 * s.cols * 4);
    L.tpl = take(3 * s.cols * 4);
    L.pab = take(s.rows * 8);
    L.pba = take(s.cols * 8);
    L.nnab = take(s.rows * 4);
    L.nnba = take(s.cols * 4);
    L.loss = take(s.n_frames * 4);
    L.part = take(s.n_frames * s.slices * 2 * 4);
    L.frame_err = take(s.n_frames * 4);
    L.fbox = take(s.n_frames * 16);
    const long long tcp = s.tc_units > 0 ? s.rows + s.cols : 0;  // points with forms
    L.tc_ufr = take(s.tc_units * 4);
    L.tc_urb = take(s.tc_units * 4);
    L.tc_upre = take(s.tc_units > 0 ? (s.tc_units + 1) * 4 : 0);
    L.tca = take(tcp * 32);
    L.tcb = take(tcp * 32);
    L.kab = take(s.tc_units > 0 ? s.rows * TC_KEYS * 4 : 0);
    L.kba = take(s.tc_units > 0 ? s.cols * TC_KEYS * 4 : 0);
    L.kpart = take(s.tc_units > 0 ? s.tc_slots * 2 * TC_UNIT_ROWS * TC_KEYS * 4 : 0);
    L.tcfb = take(tcp * 4);
    L.tcfn = take(s.tc_units > 0 ? s.n_frames * 8 : 0);
    L.total = off;
    return L;
}

Ws make_ws(void* base, const Layout& L) {
    char* p = static_cast<char*>(base);
    Ws w;
    w.hdr = reinterpret_cast<WsHeader*>(p + L.hdr);
    w.frames = reinterpret_cast<FrameDesc*>(p + L.frames);
    w.rowpre = reinterpret_cast<int*>(p + L.rowpre);
    w.colpre = reinterpret_cast<int*>(p + L.colpre);
    w.unit_frame = reinterpret_cast<int*>(p + L.unit_frame);
    w.unit_rb = reinterpret_cast<int*>(p + L.unit_rb);
    w.unit_pre = reinterpret_cast<int*>(p + L.unit_pre);
    w.cdf = reinterpret_cast<float*>(p + L.cdf);
    w.x = reinterpret_cast<float4*>(p + L.x);
    w.fw = reinterpret_cast<int4*>(p + L.fw);
    w.tsoa = reinterpret_cast<float*>(p + L.tsoa);
    w.tpl = reinterpret_cast<float*>(p + L.tpl);
    w.pab = reinterpret_cast<unsigned long long*>(p + L.pab);
    w.pba = reinterpret_cast<unsigned long long*>(p + L.pba);
    w.nnab = reinterpret_cast<int*>(p + L.nnab);
    w.nnba = reinterpret_cast<int*>(p + L.nnba);
    w.loss = reinterpret_cast<float*>(p + L.loss);
    w.part = reinterpret_cast<float*>(p + L.part);
    w.frame_err = reinterpret_cast<int*>(p + L.frame_err);
    w.fbox = reinterpret_cast<float4*>(p + L.fbox);
    w.tc_ufr = reinterpret_cast<int*>(p + L.tc_ufr);
    w.tc_urb = reinterpret_cast<int*>(p + L.tc_urb);
    w.tc_upre = reinterpret_cast<int*>(p + L.tc_upre);
    w.tca = reinterpret_cast<uint4*>(p + L.tca);
    w.tcb = reinterpret_cast<uint4*>(p + L.tcb);
    w.kab = reinterpret_cast<unsigned*>(p + L.kab);
    w.kba = reinterpret_cast<unsigned*>(p + L.kba);
    w.kpart = reinterpret_cast<unsigned*>(p + L.kpart);
    w.tcfb = reinterpret_cast<int*>(p + L.tcfb);
    w.tcfn = reinterpret_cast<int*>(p + L.tcfn);
    return w;
}

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char* where) {
    return fail(DC_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

constexpr long long INT_LIMIT = 0x7fffffffLL;

// Sizes of a uniform trajectory; false if any derived count overflows int32. The unit
// arrays are sized for the narrowest CTA (the most units); sub[w] is the Chamfer work
// (sub-chunks) at CTA width 1, 2 and 4 (indices 0, 1, 2).
bool uniform_sizes(int T, int V, int F, int N, int M, Sizes& s, long long sub[3], int& spu,
                   bool with_tc = true) {
    const long long Npad = (long long)div_up(N, ROW_PAD) * ROW_PAD;
    const long long Mpad = M > 0 ? (long long)div_up(M, COL_PAD) * COL_PAD : 0;
    spu = M > 0 ? div_up(M, SUB) : 0;
    for (int i = 0; i < 3; ++i)
        sub[i] = (long long)T * div_up(N, ROWS_PER_WARP << i) * spu;
    s.n_frames = T;
    s.n_units = (long long)T * div_up(N, ROWS_PER_WARP);
    s.sum_f = (long long)T * F;
    s.rows = (long long)T * Npad;
    s.cols = (long long)T * Mpad;
    s.slices = epilogue_slices(T);
    // tensor-core regions, sized for both sides (the mode is not known here), when the frame
    // fits the key format; none for calls without targets
    s.tc_units = s.tc_slots = 0;
    if (with_tc && M > 0 && Npad <= TC_MAX_COLS && Mpad <= TC_MAX_COLS) {
        const long long u0 = div_up(N, TC_UNIT_ROWS), u1 = div_up(M, TC_UNIT_ROWS);
        s.tc_units = (long long)T * (u0 + u1);
        const long long chunks = (long long)T * (u0 * (Mpad / TC_CHUNK) + u1 * (Npad / TC_CHUNK));
        if (chunks >= INT_LIMIT) return false;
        s.tc_slots = tc_grid(chunks);  // the pass's CTAs (partial-key slots are per CTA)
    }
    return s.rows < INT_LIMIT && s.cols < INT_LIMIT && s.sum_f < INT_LIMIT &&
           sub[0] < INT_LIMIT && s.rows * 3 < INT_LIMIT * 16 && s.cols * 6 < INT_LIMIT * 16 &&
           3LL * V < INT_LIMIT && (s.rows + s.cols) * 2 < INT_LIMIT;
}

enum : unsigned {
    PH_AREA = 1,
    PH_SAMPLE = 2,
    PH_TARGETS = 4,
    PH_CHAMFER = 8,
};

int check_ws(void* ws, size_t ws_bytes, size_t need) {
    if (!ws) return fail(DC_EINVAL, "workspace is NULL");
    if (!aligned(ws, 256)) return fail(DC_EINVAL, "workspace must be 256-byte aligned");
    if (ws_bytes < need)
        return fail(DC_ENOSPC, "workspace has %zu bytes, %zu needed", ws_bytes, need);
    return DC_OK;
}

int g_engine = ENGINE_AUTO;  // process-wide engine set by dc_tune_set

// The Chamfer engine of a call: a tensor-core filter when the problem fits its key format
// (tcgen05 by default, the warp-level MMA one when asked for), else, or when the direct
// engine is requested, the CUDA-core direct form.
// The default is the warp-level tensor-core filter for calls large enough to pay back its
// fixed costs (candidate recovery, the fallback scans, the merge of split units): at least
// 1e9 pairs and 5e7 per frame on average. Measured on one GB300 against the direct engine:
// 1 frame of 32 768 points 329 vs 330 us, 10 frames of 10 000 282 vs 302 us, 40 frames of
// 10 000 0.909 vs 1.028 ms, but 100 frames of 4096 497 vs 483 us and 1 frame of 16 384
// 139 vs 119 us. The tcgen05 filter measured slower than the warp-level one on every
// workload (at K = 16 each distance tile is one isolated tcgen05 MMA, whose issue and
// synchronisation cost the folds cannot hide); it stays available on request.
constexpr double TC_AUTO_MIN_PAIRS = 1e9;
constexpr double TC_AUTO_MIN_FRAME_PAIRS = 5e7;

int choose_engine(bool tc_fits, double pairs, long long frames) {
    if (g_engine == ENGINE_DIRECT || !tc_fits) return ENGINE_DIRECT;
    if (g_engine == ENGINE_TC5) return ENGINE_TC5;
    if (g_engine == ENGINE_TC) return ENGINE_TC;
    const bool big = pairs >= TC_AUTO_MIN_PAIRS &&
                     pairs >= TC_AUTO_MIN_FRAME_PAIRS * (double)(frames > 0 ? frames : 1);
    return big ? ENGINE_TC : ENGINE_DIRECT;
}

int keyed_grid(int engine, long long chunks) {
    return engine == ENGINE_TC5 ? tc5_grid(chunks) : tc_grid(chunks);
}

int run_uniform(UniformArgs a, unsigned phases, int epi_flags, float* loss_total, void* ws,
                size_t ws_bytes, cudaStream_t st, bool direct_only = false) {
    Sizes sz;
    long long sub[3];
    int spu = 0;
    if (!uniform_sizes(a.T, a.V, a.F, a.N, a.M, sz, sub, spu, !direct_only))
        return fail(DC_EINVAL, "problem too large for 32-bit offsets");
    const bool chamfer = (phases & PH_CHAMFER) != 0;
    const int engine =
        chamfer && !direct_only
            ? choose_engine(sz.tc_units > 0, (double)a.T * (double)a.N * (double)a.M, a.T)
            : ENGINE_DIRECT;
    const int warps =
        (chamfer && engine == ENGINE_DIRECT) ? choose_warps(a.mode, sub[2], sub[1], sub[0]) : 1;
    a.engine = engine;
    a.warps = warps;
    a.units_per_frame = div_up(a.N, ROWS_PER_WARP * warps);
    a.subs_per_unit = spu;
    a.slices = (int)sz.slices;
    const Layout L = make_layout(sz);
    int rc = check_ws(ws, ws_bytes, L.total);
    if (rc) return rc;
    const Ws w = make_ws(ws, L);
    const int T = a.T, rows = (int)sz.rows, cols = (int)sz.cols;
    const bool tc = chamfer && keyed(engine);
    // with sampling to follow, the tables and the area CDFs (and the frame boxes of the
    // tensor-core forms) share one launch
    const bool fused = (phases & PH_AREA) && (phases & PH_SAMPLE);
    cudaError_t e = fused ? launch_build_area(a, w, st) : launch_build_uniform(a, w, st);
    if (!e && (phases & PH_AREA) && !fused) e = launch_area_cdf(w, T, st);
    if (!e && tc && !fused) e = launch_bbox(w, T, st);
    if (!e && (phases & (PH_SAMPLE | PH_TARGETS)))
        e = launch_stage(w, T, (int)sz.slices, a.pts ? 0 : a.F, (phases & PH_SAMPLE) ? rows : 0,
                         (phases & PH_TARGETS) ? cols : 0, fused ? 1 : 0, tc ? 1 : 0, st);
    int grid = 0;
    if (!e && chamfer) {
        if (tc) {
            const long long Npad = (long long)div_up(a.N, ROW_PAD) * ROW_PAD;
            const long long Mpad = (long long)div_up(a.M, COL_PAD) * COL_PAD;
            const long long u1 = a.mode == DC_BIDIR_MEAN ? div_up(a.M, TC_UNIT_ROWS) : 0;
            const long long chunks =
                (long long)T * (div_up(a.N, TC_UNIT_ROWS) * (Mpad / TC_CHUNK) + u1 * (Npad / TC_CHUNK));
            grid = keyed_grid(engine, chunks);
            const int units =
                T * (div_up(a.N, TC_UNIT_ROWS) +
                     (a.mode == DC_BIDIR_MEAN ? div_up(a.M, TC_UNIT_ROWS) : 0));
            e = launch_tcpass(w, engine, grid, chunks, units, rows, cols, a.mode, T, st);
        } else {
            const long long units = (long long)T * a.units_per_frame;
            e = launch_chamfer(w, (int)units, (int)(units * spu), a.mode, warps, st);
        }
    }
    if (!e && epi_flags)
        e = launch_epilogue(w, T, (int)sz.slices, a.grad ? a.V : 0, a.mode, epi_flags,
                            loss_total, tc ? grid : 0, st);
    if (e) return cuda_fail(e, "kernel launch");
    return DC_OK;
}

int check_common(int T, int N, int M, int mode) {
    if (T <= 0 || N <= 0 || M <= 0) return fail(DC_EINVAL, "T, N and M must be positive");
    if (mode != DC_BIDIR_MEAN && mode != DC_UNIDIR_SUM) return fail(DC_EINVAL, "bad mode");
    return DC_OK;
}

int check_ptrs(std::initializer_list<const void*> ps, const char* what) {
    for (const void* p : ps) {
        if (!p) return fail(DC_EINVAL, "%s: required pointer is NULL", what);
        if (!aligned(p, 4)) return fail(DC_EINVAL, "%s: pointer not 4-byte aligned", what);
    }
    return DC_OK;
}

// dc_loss_traj; direct_only runs the direct engine on a workspace laid out without the
// tensor-core regions (the smaller footprint of the built-in scratch of the no-allocation
// entry point)
int loss_traj_impl(const float* verts, const int32_t* faces, const uint8_t* face_mask,
                   const float* draws, const float* targets, int T, int V, int F, int N, int M,
                   int mode, const float* frame_w, float* loss_total, float* loss_frames,
                   float* grad_verts, int32_t* nn_ab, int32_t* nn_ba, void* ws,
                   size_t ws_bytes, dc_stream_t stream, bool direct_only) {
    int rc = check_common(T, N, M, mode);
    if (rc) return rc;
    if (V <= 0 || F <= 0) return fail(DC_EINVAL, "V and F must be positive");
    rc = check_ptrs({verts, faces, draws, targets, loss_frames}, "dc_loss_traj");
    if (rc) return rc;
    UniformArgs a{};
    a.verts = verts;
    a.faces = faces;
    a.mask = face_mask;
    a.draws = draws;
    a.tgt = targets;
    a.loss = loss_frames;
    a.nn_ab = nn_ab;
    a.nn_ba = mode == DC_BIDIR_MEAN ? nn_ba : nullptr;
    a.grad = grad_verts;
    a.weight = frame_w;
    a.T = T;
    a.V = V;
    a.F = F;
    a.N = N;
    a.M = M;
    a.mode = mode;
    const unsigned ph = PH_AREA | PH_SAMPLE | PH_TARGETS | PH_CHAMFER;
    const int epi = EPI_RESCAN | EPI_LOSS | (grad_verts ? EPI_GRAD : 0);
    return run_uniform(a, ph, epi, loss_total, ws, ws_bytes, static_cast<cudaStream_t>(stream),
                       direct_only);
}

// bytes of a uniform workspace laid out for the direct engine only
size_t direct_workspace_size(int T, int V, int F, int N, int M) {
    if (T <= 0 || V <= 0 || F <= 0 || N <= 0 || M < 0) return 0;
    Sizes sz;
    long long sub[3];
    int spu;
    if (!uniform_sizes(T, V, F, N, M, sz, sub, spu, false)) return 0;
    return make_layout(sz).total;
}

// ---- batch plans (host copy of what dc_batch_run needs to launch) ----
struct Plan {
    Sizes sz;
    int mode, any_grad, max_v, max_f, total_sub, n_units, warps, engine, tc_grid, tc_units;
    long long tc_chunks;
    size_t bytes;
};
std::mutex g_plan_mu;
std::unordered_map<const void*, Plan> g_plans;

int plan_impl(const dc_frame* frames, int n_frames, int mode, void* ws, size_t ws_bytes,
              char* host_staging, size_t staging_bytes, size_t* size_only, cudaStream_t stream);

}  // namespace
}  // namespace dc

using namespace dc;

extern "C" {

const char* dc_last_error(void) { return g_err; }

long long dc_launch_count(void) { return g_launches.load(); }

int dc_prof_start(int cap) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (cap <= 0) return fail(DC_EINVAL, "cap must be positive");
    for (cudaEvent_t e : g_prof_ev) cudaEventDestroy(e);
    g_prof_ev.assign(2 * (size_t)cap, nullptr);
    for (auto& e : g_prof_ev) {
        cudaError_t r = cudaEventCreate(&e);
        if (r) return cuda_fail(r, "cudaEventCreate");
    }
    g_prof_cap = cap;
    g_prof_n = 0;
    g_prof_on = true;
    return DC_OK;
}

int dc_prof_stop(float* total_ms, int* launches) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_on = false;
    float sum = 0.f;
    for (int i = 0; i < g_prof_n; ++i) {
        cudaError_t r = cudaEventSynchronize(g_prof_ev[2 * i + 1]);
        if (r) return cuda_fail(r, "cudaEventSynchronize");
        float ms = 0.f;
        r = cudaEventElapsedTime(&ms, g_prof_ev[2 * i], g_prof_ev[2 * i + 1]);
        if (r) return cuda_fail(r, "cudaEventElapsedTime");
        sum += ms;
    }
    if (total_ms) *total_ms = sum;
    if (launches) *launches = g_prof_n;
    return DC_OK;
}

int dc_tune_set(const dc_tune* tune) {
    const int w = tune ? tune->warps_per_cta : 0;
    const int en = tune ? tune->engine : DC_ENGINE_AUTO;
    if (w != 0 && w != 1 && w != 2 && w != 4)
        return fail(DC_EINVAL, "warps_per_cta must be 0 (automatic), 1, 2 or 4");
    if (en != DC_ENGINE_AUTO && en != DC_ENGINE_DIRECT && en != DC_ENGINE_TENSOR &&
        en != DC_ENGINE_TCGEN05)
        return fail(DC_EINVAL, "engine must be DC_ENGINE_AUTO, DC_ENGINE_DIRECT, "
                               "DC_ENGINE_TENSOR or DC_ENGINE_TCGEN05");
    set_tuned_warps(w);
    g_engine = en == DC_ENGINE_DIRECT    ? ENGINE_DIRECT
               : en == DC_ENGINE_TENSOR  ? ENGINE_TC
               : en == DC_ENGINE_TCGEN05 ? ENGINE_TC5
                                         : ENGINE_AUTO;
    return DC_OK;
}

int dc_tune_get(dc_tune* tune) {
    if (!tune) return fail(DC_EINVAL, "tune is NULL");
    tune->warps_per_cta = tuned_warps();
    tune->engine = g_engine == ENGINE_DIRECT ? DC_ENGINE_DIRECT
                   : g_engine == ENGINE_TC   ? DC_ENGINE_TENSOR
                   : g_engine == ENGINE_TC5  ? DC_ENGINE_TCGEN05
                                             : DC_ENGINE_AUTO;
    return DC_OK;
}

size_t dc_workspace_size(int T, int V, int F, int N, int M) {
    if (T <= 0 || V <= 0 || F <= 0 || N <= 0 || M < 0) return 0;
    Sizes sz;
    long long sub[3];
    int spu;
    if (!uniform_sizes(T, V, F, N, M, sz, sub, spu)) return 0;
    return make_layout(sz).total;
}

int dc_loss_total(const float* loss_frames, const float* frame_w, int T, float* loss_total,
                  dc_stream_t stream) {
    if (T <= 0) return fail(DC_EINVAL, "T must be positive");
    int rc = check_ptrs({loss_frames, loss_total}, "dc_loss_total");
    if (rc) return rc;
    if (frame_w && !aligned(frame_w, 4)) return fail(DC_EINVAL, "frame_w not 4-byte aligned");
    cudaError_t e = launch_loss_total(loss_frames, frame_w, T, loss_total,
                                      static_cast<cudaStream_t>(stream));
    if (e) return cuda_fail(e, "dc_loss_total");
    return DC_OK;
}

int dc_ws_status(const void* ws, dc_stream_t stream) {
    if (!ws) return fail(DC_EINVAL, "workspace is NULL");
    int st = 0;
    const WsHeader* h = static_cast<const WsHeader*>(ws);
    cudaError_t e = cudaMemcpyAsync(&st, &h->status, sizeof(int), cudaMemcpyDeviceToHost, stream);
    if (!e) e = cudaStreamSynchronize(stream);
    if (e) return cuda_fail(e, "dc_ws_status");
    if (st != DC_OK) fail(st, "device-side error %d recorded in the workspace", st);
    return st;
}

int dc_area_cdf(const float* verts, const int32_t* faces, const uint8_t* face_mask, int T,
                int V, int F, float* cdf, void* ws, size_t ws_bytes, dc_stream_t stream) {
    if (T <= 0 || V <= 0 || F <= 0) return fail(DC_EINVAL, "sizes must be positive");
    int rc = check_ptrs({verts, faces, cdf}, "dc_area_cdf");
    if (rc) return rc;
    UniformArgs a{};
    a.verts = verts;
    a.faces = faces;
    a.mask = face_mask;
    a.T = T;
    a.V = V;
    a.F = F;
    a.N = 1;  // no sampling: the smallest valid layout
    a.M = 0;
    a.mode = DC_BIDIR_MEAN;
    rc = run_uniform(a, PH_AREA, 0, nullptr, ws, ws_bytes, stream);
    if (rc) return rc;
    // the CDFs of the frames lie back to back in the workspace (frame t at t F)
    Sizes sz;
    long long sub[3];
    int spu = 0;
    uniform_sizes(T, V, F, 1, 0, sz, sub, spu);
    const Ws w = make_ws(ws, make_layout(sz));
    cudaError_t e = cudaMemcpyAsync(cdf, w.cdf, sizeof(float) * (size_t)T * F,
                                    cudaMemcpyDeviceToDevice, stream);
    if (e) return cuda_fail(e, "dc_area_cdf");
    return DC_OK;
}

int dc_sample(const float* verts, const int32_t* faces, const uint8_t* face_mask,
              const float* draws, int T, int V, int F, int N, float* points, int32_t* face_idx,
              float* bary, void* ws, size_t ws_bytes, dc_stream_t stream) {
    if (T <= 0 || V <= 0 || F <= 0 || N <= 0) return fail(DC_EINVAL, "sizes must be positive");
    int rc = check_ptrs({verts, faces, draws, points}, "dc_sample");
    if (rc) return rc;
    UniformArgs a{};
    a.verts = verts;
    a.faces = faces;
    a.mask = face_mask;
    a.draws = draws;
    a.out_pts = points;
    a.out_face = face_idx;
    a.out_bary = bary;
    a.T = T;
    a.V = V;
    a.F = F;
    a.N = N;
    a.M = 0;
    a.mode = DC_BIDIR_MEAN;
    return run_uniform(a, PH_AREA | PH_SAMPLE, 0, nullptr, ws, ws_bytes, stream);
}

int dc_chamfer_fwd(const float* a_pts, const float* b, int T, int N, int M, int mode,
                   float* loss, int32_t* nn_ab, int32_t* nn_ba, void* ws, size_t ws_bytes,
                   dc_stream_t stream) {
    int rc = check_common(T, N, M, mode);
    if (rc) return rc;
    rc = check_ptrs({a_pts, b, loss}, "dc_chamfer_fwd");
    if (rc) return rc;
    UniformArgs a{};
    a.pts = a_pts;
    a.tgt = b;
    a.loss = loss;
    a.nn_ab = nn_ab;
    a.nn_ba = mode == DC_BIDIR_MEAN ? nn_ba : nullptr;
    a.T = T;
    a.V = 1;
    a.F = 0;
    a.N = N;
    a.M = M;
    a.mode = mode;
    return run_uniform(a, PH_SAMPLE | PH_TARGETS | PH_CHAMFER, EPI_RESCAN | EPI_LOSS, nullptr,
                       ws, ws_bytes, stream);
}

int dc_chamfer_bwd(const float* a, const float* b, const int32_t* nn_ab, const int32_t* nn_ba,
                   int T, int N, int M, int mode, const float* grad_loss, float* grad_a,
                   dc_stream_t stream) {
    int rc = check_common(T, N, M, mode);
    if (rc) return rc;
    rc = check_ptrs({a, b, nn_ab, grad_loss, grad_a}, "dc_chamfer_bwd");
    if (rc) return rc;
    if (mode == DC_BIDIR_MEAN && !nn_ba) return fail(DC_EINVAL, "nn_ba is required in Eq. 1");
    cudaError_t e = launch_chamfer_bwd_points(a, b, nn_ab, nn_ba, T, N, M, mode, grad_loss,
                                              grad_a, stream);
    if (e) return cuda_fail(e, "dc_chamfer_bwd");
    return DC_OK;
}

int dc_loss_traj(const float* verts, const int32_t* faces, const uint8_t* face_mask,
                 const float* draws, const float* targets, int T, int V, int F, int N, int M,
                 int mode,
                 const float* frame_w, float* loss_total, float* loss_frames, float* grad_verts,
                 int32_t* nn_ab, int32_t* nn_ba, void* ws, size_t ws_bytes,
                 dc_stream_t stream) {
    return loss_traj_impl(verts, faces, face_mask, draws, targets, T, V, F, N, M, mode, frame_w,
                          loss_total, loss_frames, grad_verts, nn_ab, nn_ba, ws, ws_bytes,
                          stream, false);
}

int dc_loss_traj_bwd(const float* verts, const int32_t* faces, const uint8_t* face_mask,
                     const float* draws, const float* targets, int T, int V, int F, int N, int M,
                     int mode, const int32_t* nn_ab, const int32_t* nn_ba, const float* frame_w,
                     const float* grad_total, const float* grad_frames, float* grad_verts,
                     void* ws, size_t ws_bytes, dc_stream_t stream) {
    int rc = check_common(T, N, M, mode);
    if (rc) return rc;
    if (V <= 0 || F <= 0) return fail(DC_EINVAL, "V and F must be positive");
    rc = check_ptrs({verts, faces, draws, targets, nn_ab, grad_verts}, "dc_loss_traj_bwd");
    if (rc) return rc;
    if (mode == DC_BIDIR_MEAN && !nn_ba) return fail(DC_EINVAL, "nn_ba is required in Eq. 1");
    if (!grad_total && !grad_frames)
        return fail(DC_EINVAL, "dc_loss_traj_bwd: grad_total or grad_frames is required");
    UniformArgs a{};
    a.verts = verts;
    a.faces = faces;
    a.mask = face_mask;
    a.draws = draws;
    a.tgt = targets;
    a.nn_ab = const_cast<int32_t*>(nn_ab);
    a.nn_ba = mode == DC_BIDIR_MEAN ? const_cast<int32_t*>(nn_ba) : nullptr;
    a.grad = grad_verts;
    a.weight = frame_w;
    a.gtotal = grad_total;
    a.gframes = grad_frames;
    a.bwd = 1;
    a.T = T;
    a.V = V;
    a.F = F;
    a.N = N;
    a.M = M;
    a.mode = mode;
    // targets are staged too: the gradient reads them from the compact planes
    return run_uniform(a, PH_AREA | PH_SAMPLE | PH_TARGETS, EPI_GRAD, nullptr, ws, ws_bytes,
                       stream);
}

// ---------------------------------------------------------------------------------------
// batches
// ---------------------------------------------------------------------------------------
static bool batch_sizes(const dc_frame* fr, int n, Sizes& s, long long sub[3]) {
    s = Sizes{n, 0, 0, 0, 0, epilogue_slices(n), 0, 0};
    sub[0] = sub[1] = sub[2] = 0;
    long long max_v = 0, tc_units = 0, tc_chunks = 0;
    bool tc_fits = true;
    for (int k = 0; k < n; ++k) {
        const long long spu = div_up(fr[k].M, SUB);
        s.n_units += div_up(fr[k].N, ROWS_PER_WARP);
        for (int i = 0; i < 3; ++i) sub[i] += (long long)div_up(fr[k].N, ROWS_PER_WARP << i) * spu;
        s.sum_f += fr[k].F;
        const long long Npad = (long long)div_up(fr[k].N, ROW_PAD) * ROW_PAD;
        const long long Mpad = (long long)div_up(fr[k].M, COL_PAD) * COL_PAD;
        s.rows += Npad;
        s.cols += Mpad;
        if (fr[k].grad_verts && fr[k].V > max_v) max_v = fr[k].V;
        tc_fits = tc_fits && Npad <= TC_MAX_COLS && Mpad <= TC_MAX_COLS;
        const long long u0 = div_up(fr[k].N, TC_UNIT_ROWS), u1 = div_up(fr[k].M, TC_UNIT_ROWS);
        tc_units += u0 + u1;
        tc_chunks += u0 * (Mpad / TC_CHUNK) + u1 * (Npad / TC_CHUNK);
    }
    if (tc_fits && tc_chunks < INT_LIMIT) {
        s.tc_units = tc_units;
        s.tc_slots = tc_grid(tc_chunks);
    }
    return s.rows < INT_LIMIT && s.cols < INT_LIMIT && s.sum_f < INT_LIMIT &&
           sub[0] < INT_LIMIT && s.n_units < INT_LIMIT && s.cols * 6 < INT_LIMIT * 16 &&
           3 * max_v < INT_LIMIT && tc_chunks < INT_LIMIT && (s.rows + s.cols) * 2 < INT_LIMIT;
}

size_t dc_batch_workspace_size(const dc_frame* frames, int n_frames) {
    if (!frames || n_frames <= 0) return 0;
    for (int k = 0; k < n_frames; ++k)
        if (frames[k].N <= 0 || frames[k].M <= 0 || frames[k].F <= 0 || frames[k].V <= 0)
            return 0;
    Sizes sz;
    long long sub[3];
    if (!batch_sizes(frames, n_frames, sz, sub)) return 0;
    return make_layout(sz).total;
}

int dc_batch_plan(const dc_frame* frames, int n_frames, int mode, void* ws, size_t ws_bytes,
                  dc_stream_t stream) {
    return plan_impl(frames, n_frames, mode, ws, ws_bytes, nullptr, 0, nullptr, stream);
}

size_t dc_batch_plan_bytes(const dc_frame* frames, int n_frames, int mode) {
    size_t need = 0;
    if (plan_impl(frames, n_frames, mode, nullptr, 0, nullptr, 0, &need, nullptr) != DC_OK)
        return 0;
    return need;
}

int dc_batch_plan_async(const dc_frame* frames, int n_frames, int mode, void* ws,
                        size_t ws_bytes, void* host_staging, size_t staging_bytes,
                        dc_stream_t stream) {
    if (!host_staging) return fail(DC_EINVAL, "dc_batch_plan_async: host_staging is NULL");
    return plan_impl(frames, n_frames, mode, ws, ws_bytes, static_cast<char*>(host_staging),
                     staging_bytes, nullptr, stream);
}

}  // extern "C"

namespace dc {
namespace {

// dc_batch_plan and its variants. With host_staging the tables are built there and copied
// without waiting for the stream; without it the copy is made from the library's own host
// memory and the stream is synchronised. With size_only (and no workspace) only the bytes of
// the staging image are returned.
int plan_impl(const dc_frame* frames, int n_frames, int mode, void* ws, size_t ws_bytes,
              char* host_staging, size_t staging_bytes, size_t* size_only, cudaStream_t stream) {
    if (!frames || n_frames <= 0) return fail(DC_EINVAL, "no frames");
    if (mode != DC_BIDIR_MEAN && mode != DC_UNIDIR_SUM) return fail(DC_EINVAL, "bad mode");
    for (int k = 0; k < n_frames; ++k) {
        const dc_frame& f = frames[k];
        if (f.N <= 0 || f.M <= 0 || f.F <= 0 || f.V <= 0)
            return fail(DC_EINVAL, "frame %d: sizes must be positive", k);
        if (!f.verts || !f.faces || !f.draws || !f.targets)
            return fail(DC_EINVAL, "frame %d: verts, faces, draws and targets are required", k);
        if (!aligned(f.verts, 4) || !aligned(f.faces, 4) || !aligned(f.draws, 4) ||
            !aligned(f.targets, 4))
            return fail(DC_EINVAL, "frame %d: pointers must be 4-byte aligned", k);
    }
    Sizes sz;
    long long sub[3];
    if (!batch_sizes(frames, n_frames, sz, sub))
        return fail(DC_EINVAL, "batch too large for 32-bit offsets");
    double pairs = 0.0;
    for (int k = 0; k < n_frames; ++k) pairs += (double)frames[k].N * (double)frames[k].M;
    const int engine = choose_engine(sz.tc_units > 0, pairs, n_frames);
    const int warps = engine == ENGINE_DIRECT ? choose_warps(mode, sub[2], sub[1], sub[0]) : 1;
    const Layout L = make_layout(sz);
    // the staging image: the table regions [hdr, cdf), then the tensor-core unit tables
    const size_t img_bytes = L.cdf + (keyed(engine) ? L.tca - L.tc_ufr : 0);
    if (size_only) {
        *size_only = img_bytes;
        return DC_OK;
    }
    int rc = check_ws(ws, ws_bytes, L.total);
    if (rc) return rc;
    if (host_staging && staging_bytes < img_bytes)
        return fail(DC_ENOSPC, "host staging has %zu bytes, %zu needed", staging_bytes,
                    img_bytes);
    const Ws w = make_ws(ws, L);

    // host image of the table regions [hdr, cdf)
    std::vector<char> img(L.cdf, 0);
    WsHeader* h = reinterpret_cast<WsHeader*>(img.data() + L.hdr);
    FrameDesc* fd = reinterpret_cast<FrameDesc*>(img.data() + L.frames);
    int* rowpre = reinterpret_cast<int*>(img.data() + L.rowpre);
    int* colpre = reinterpret_cast<int*>(img.data() + L.colpre);
    int* ufr = reinterpret_cast<int*>(img.data() + L.unit_frame);
    int* urb = reinterpret_cast<int*>(img.data() + L.unit_rb);
    int* upre = reinterpret_cast<int*>(img.data() + L.unit_pre);
    // the tensor-core unit tables follow in the workspace; they get a host image of their own
    const size_t tc_beg = L.tc_ufr, tc_end = L.tca;
    std::vector<char> tcimg(keyed(engine) ? tc_end - tc_beg : 0, 0);
    int* tufr = reinterpret_cast<int*>(tcimg.data() + (L.tc_ufr - tc_beg));
    int* turb = reinterpret_cast<int*>(tcimg.data() + (L.tc_urb - tc_beg));
    int* tupre = reinterpret_cast<int*>(tcimg.data() + (L.tc_upre - tc_beg));
    int tunit = 0, tchunk = 0;
    int row0 = 0, col0 = 0, cdf0 = 0, unit = 0, subc = 0, any_grad = 0, max_v = 0, max_f = 0;
    // The table lists the frames largest first (N + M, ties in the caller's order). The
    // sampling and epilogue kernels run one CTA per (frame, slice) in table order, so the
    // long CTAs of big frames start first and the small ones fill in behind them instead of
    // leaving a tail (measured on 64 trajectories of uneven sizes).
    std::vector<int> order(n_frames);
    for (int k = 0; k < n_frames; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [frames](int a, int b) {
        return (long long)frames[a].N + frames[a].M > (long long)frames[b].N + frames[b].M;
    });
    for (int k = 0; k < n_frames; ++k) {
        const dc_frame& f = frames[order[k]];
        FrameDesc d{};
        d.verts = f.verts;
        d.faces = f.faces;
        d.mask = f.face_mask;
        d.draws = f.draws;
        d.tgt = f.targets;
        d.loss = f.loss ? f.loss : w.loss + k;
        d.Npad = div_up(f.N, ROW_PAD) * ROW_PAD;
        d.Mpad = div_up(f.M, COL_PAD) * COL_PAD;
        d.nn_ab = f.nn_ab ? f.nn_ab : w.nnab + row0;
        d.nn_ba = f.nn_ba ? f.nn_ba : w.nnba + col0;
        d.grad = f.grad_verts;
        d.V = f.V;
        d.F = f.F;
        d.N = f.N;
        d.M = f.M;
        d.weight = f.weight;
        d.gscale = f.weight;
        d.skip = f.weight == 0.0f;
        d.row0 = row0;
        d.col0 = col0;
        d.cdf0 = cdf0;
        d.unit0 = unit;
        d.tc_unit0 = tunit;
        fd[k] = d;
        if (keyed(engine)) {
            // sim rows against the targets, then (Eq. 1) the targets against the sim points
            const int u0 = div_up(f.N, TC_UNIT_ROWS);
            const int u1 = mode == DC_BIDIR_MEAN ? div_up(f.M, TC_UNIT_ROWS) : 0;
            for (int r = 0; r < u0 + u1; ++r, ++tunit) {
                const int side = r >= u0 ? 1 : 0, rb = side ? r - u0 : r;
                tufr[tunit] = k;
                turb[tunit] = (side << 30) | rb;
                tupre[tunit] = tchunk;
                if (!d.skip) tchunk += (side ? d.Npad : d.Mpad) / TC_CHUNK;
            }
        }
        rowpre[k] = row0;
        colpre[k] = col0;
        const int upf = div_up(f.N, ROWS_PER_WARP * warps);
        const int spu = d.skip ? 0 : div_up(f.M, SUB);  // a skipped frame carries no work
        for (int r = 0; r < upf; ++r, ++unit) {
            ufr[unit] = k;
            urb[unit] = r;
            upre[unit] = subc;
            subc += spu;
        }
        if (f.F > max_f) max_f = f.F;
        if (f.grad_verts) {
            any_grad = 1;
            if (f.V > max_v) max_v = f.V;
        }
        row0 += d.Npad;
        col0 += d.Mpad;
        cdf0 += f.F;
    }
    rowpre[n_frames] = row0;
    colpre[n_frames] = col0;
    upre[unit] = subc;
    if (keyed(engine)) tupre[tunit] = tchunk;
    h->status = DC_OK;
    h->n_frames = n_frames;
    h->n_units = unit;
    h->total_sub = subc;
    h->total_rows = row0;
    h->total_cols = col0;
    h->sum_f = cdf0;
    h->mode = mode;
    h->planned = 1;
    h->any_grad = any_grad;
    h->max_v = max_v;
    h->slices = (int)sz.slices;
    h->warps = warps;
    h->engine = engine;
    h->tc_units = keyed(engine) ? tunit : 0;
    h->tc_total = keyed(engine) ? tchunk : 0;
    h->tc_fallback = 0;
    h->tc_next = 0;
    const char* src_img = img.data();
    const char* src_tc = tcimg.data();
    if (host_staging) {  // the caller's (pinned) memory: the copies need no host wait
        memcpy(host_staging, img.data(), img.size());
        if (!tcimg.empty()) memcpy(host_staging + img.size(), tcimg.data(), tcimg.size());
        src_img = host_staging;
        src_tc = host_staging + img.size();
    }
    cudaError_t e = cudaMemcpyAsync(ws, src_img, img.size(), cudaMemcpyHostToDevice, stream);
    if (!e && !tcimg.empty())
        e = cudaMemcpyAsync(static_cast<char*>(ws) + tc_beg, src_tc, tcimg.size(),
                            cudaMemcpyHostToDevice, stream);
    if (!e && !host_staging) e = cudaStreamSynchronize(stream);
    if (e) return cuda_fail(e, "dc_batch_plan copy");
    Plan p;
    p.sz = sz;
    p.mode = mode;
    p.any_grad = any_grad;
    p.max_v = max_v;
    p.max_f = max_f;
    p.total_sub = subc;
    p.n_units = unit;
    p.warps = warps;
    p.engine = engine;
    p.tc_grid = keyed(engine) ? keyed_grid(engine, tchunk) : 0;
    p.tc_units = keyed(engine) ? tunit : 0;
    p.tc_chunks = tchunk;
    p.bytes = L.total;
    std::lock_guard<std::mutex> lk(g_plan_mu);
    g_plans[ws] = p;
    return DC_OK;
}

}  // namespace
}  // namespace dc

extern "C" {

int dc_batch_run(void* ws, float* loss_total, dc_stream_t stream) {
    Plan p;
    {
        std::lock_guard<std::mutex> lk(g_plan_mu);
        auto it = g_plans.find(ws);
        if (it == g_plans.end()) return fail(DC_EINVAL, "workspace holds no batch plan");
        p = it->second;
    }
    const Layout L = make_layout(p.sz);
    const Ws w = make_ws(ws, L);
    const int n = (int)p.sz.n_frames, rows = (int)p.sz.rows, cols = (int)p.sz.cols;
    const bool tc = keyed(p.engine);
    cudaError_t e = launch_reset(w, stream);
    if (!e) e = launch_area_cdf(w, n, stream);  // and the frame boxes
    if (!e) e = launch_stage(w, n, (int)p.sz.slices, p.max_f, rows, cols, 0, tc ? 1 : 0, stream);
    if (!e)
        e = tc ? launch_tcpass(w, p.engine, p.tc_grid, p.tc_chunks, p.tc_units, rows, cols,
                               p.mode, n, stream)
               : launch_chamfer(w, p.n_units, p.total_sub, p.mode, p.warps, stream);
    if (!e)
        e = launch_epilogue(w, n, (int)p.sz.slices, p.any_grad ? p.max_v : 0, p.mode,
                            EPI_RESCAN | EPI_LOSS | (p.any_grad ? EPI_GRAD : 0), loss_total,
                            tc ? p.tc_grid : 0, stream);
    if (e) return cuda_fail(e, "dc_batch_run");
    return DC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// dc_loss_traj_noalloc: dc_loss_traj with built-in scratch memory instead of a workspace
// ---------------------------------------------------------------------------------------
// Some callers cannot call cudaMalloc at the point where they need the loss: a plug-in inside
// a host framework whose memory pool owns all device memory, or a real-time control loop that
// forbids allocator calls after start-up (an allocation can synchronise the device and take
// unbounded time). For them the scratch lives in this file-scope device array, reserved once
// when the library's module is loaded on a GPU and held until the process exits.
#define DC_NOALLOC_SCRATCH_BYTES (16u << 20)

static __device__ __align__(256) unsigned char g_noalloc_scratch[DC_NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[64];  // device address of g_noalloc_scratch, per device
}  // namespace

extern "C" int dc_loss_traj_noalloc(const float* verts, const int32_t* faces,
                                    const uint8_t* face_mask, const float* draws,
                                    const float* targets, int T, int V, int F,
                                    int N, int M, int mode, const float* frame_w,
                                    float* loss_total, float* loss_frames, float* grad_verts,
                                    int32_t* nn_ab, int32_t* nn_ba, int32_t* status,
                                    dc_stream_t stream) {
    int rc = check_common(T, N, M, mode);
    if (rc) return rc;
    if (V <= 0 || F <= 0) return fail(DC_EINVAL, "V and F must be positive");
    // the size check comes first: a problem that does not fit is refused before any pointer
    // is looked at or any CUDA call is made
    // the built-in scratch runs the direct engine, whose layout has no tensor-core regions
    const size_t need = direct_workspace_size(T, V, F, N, M);
    if (need == 0) return fail(DC_EINVAL, "problem too large for 32-bit offsets");
    if (need > DC_NOALLOC_SCRATCH_BYTES)
        return fail(DC_ENOSPC,
                    "dc_loss_traj_noalloc: this problem needs %zu bytes of scratch; the built-in "
                    "scratch holds %u bytes (use dc_loss_traj with a workspace)",
                    need, DC_NOALLOC_SCRATCH_BYTES);
    rc = check_ptrs({verts, faces, draws, targets, loss_frames}, "dc_loss_traj_noalloc");
    if (rc) return rc;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(DC_EINVAL, "device index %d out of range", dev);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(static_cast<cudaStream_t>(stream), &cap);
    if (e) return cuda_fail(e, "cudaStreamIsCapturing");
    void* ws = nullptr;
    {
        // The array's device address, with this device current. It is looked up again on every
        // call outside a stream capture (the lookup allocates nothing), so that a context that
        // was reset and reloaded the module is followed; inside a capture the address from the
        // last call outside one is used, so the first call on a device must precede any capture.
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (cap == cudaStreamCaptureStatusNone || !g_noalloc_ptr[dev]) {
            if (cap != cudaStreamCaptureStatusNone)
                return fail(DC_EINVAL, "dc_loss_traj_noalloc: the first call on a device must "
                                       "come before any stream capture");
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
            g_noalloc_ptr[dev] = p;
        }
        ws = g_noalloc_ptr[dev];
    }
    // Every region of the scratch that a call reads is written earlier in the same call (the
    // status word included), so nothing needs clearing between calls.
    rc = loss_traj_impl(verts, faces, face_mask, draws, targets, T, V, F, N, M, mode, frame_w,
                        loss_total, loss_frames, grad_verts, nn_ab, nn_ba, ws,
                        DC_NOALLOC_SCRATCH_BYTES, stream, true);
    if (rc) return rc;
    if (status) {
        e = cudaMemcpyAsync(status, &static_cast<const WsHeader*>(ws)->status, sizeof(int32_t),
                            cudaMemcpyDeviceToDevice, stream);
        if (e) return cuda_fail(e, "status copy");
    }
    return DC_OK;
}

// ---------------------------------------------------------------------------------------
// test of the device-side failure detection
// ---------------------------------------------------------------------------------------
extern "C" int dc_test_inject_stall(void) {
    dc::inject_stall();
    return DC_OK;
}
