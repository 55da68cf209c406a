// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/diffcloud.h"

namespace dc {

// ---------------------------------------------------------------------------------------
// Chamfer tiling. A CTA of WARPS warps owns one "unit": ROWS_PER_UNIT consecutive sim points
// of one frame, ROWS_PER_THREAD per thread held in registers as packed pairs {x_i, x_i+1}.
// Targets stream through shared memory in chunks of CHUNK points: structure-of-arrays planes
// holding every coordinate negated and twice, {-X_j, -X_j}, bulk-copied. The per-row minimum
// is tracked per sub-chunk of SUB targets, so that a row's nearest neighbour can later be
// found again by re-scanning one sub-chunk, and a target's by re-scanning one thread's rows.
// ---------------------------------------------------------------------------------------
#ifndef DC_ROWS_PER_THREAD
#define DC_ROWS_PER_THREAD 16
#endif
constexpr int ROWS_PER_THREAD = DC_ROWS_PER_THREAD;  // even
constexpr int ROWS_PER_WARP = 32 * ROWS_PER_THREAD;       // 512
// A Chamfer CTA has 1, 2 or 4 warps (units of 512, 1024 or 2048 sim points): wide CTAs
// amortise the target staging and the column merges over more rows, narrow ones give
// small problems enough work items to fill the GPU.
constexpr int MAX_WARPS = 4;
#ifndef DC_SUB
#define DC_SUB 32
#endif
constexpr int SUB = DC_SUB;                               // targets per tracked sub-chunk
#ifndef DC_CHUNK
#define DC_CHUNK 256
#endif
constexpr int CHUNK = DC_CHUNK;                           // targets per staged chunk
constexpr int SUBS_PER_CHUNK = CHUNK / SUB;
constexpr int ROW_PAD = ROWS_PER_WARP;                    // sim points padded to this
constexpr int COL_PAD = CHUNK;                            // target points padded to this
constexpr int EPI_THREADS = 256;                          // epilogue CTA size
constexpr int EPI_CTAS = 608;                             // epilogue CTAs resident at once
constexpr int MAX_SLICES = 32;                            // epilogue slices per frame

constexpr float COORD_MAX = 1e15f;
constexpr unsigned long long EMPTY = ~0ull;

// ---------------------------------------------------------------------------------------
// Tensor-core filter (tcpass.cu). Every point p of a frame is centred on the frame's box
// centre c and scaled by a power of two sig (|(p - c) sig| < 64 per coordinate), and each
// scaled coordinate s is split into two halves h = fp16(s), l = fp16(s - h) (22 significant
// bits). With n = |s|^2 (float32, split the same way), the K = 16 vectors
//   A(p) = (h0 h0 l0 l0  h1 h1 l1 l1  h2 h2 l2 l2  1  1  nh nl)
//   B(q) = (-2h0 -2l0 -2h0 -2l0  -2h1 -2l1 -2h1 -2l1  -2h2 -2l2 -2h2 -2l2  nh nl 1 1)
// give A(p).B(q) = |p - q|^2 sig^2 up to a small bound (the expanded form, used only to
// select candidates; the reported minimum is recomputed exactly in the direct form). The
// four quad lanes that share a row each see a quarter of its columns; a lane's minimum over
// its columns of a block of TC_BLOCK becomes a 32-bit key, (value bits truncated to 20) |
// block, and every (row, lane) keeps its three smallest keys in a slot of its own.
// Both forms are stored per group of 8 points as the two 8 x 16-byte halves of K (256 B),
// in the order tc_form_pos gives within each block of TC_BLOCK points.
// ---------------------------------------------------------------------------------------
#ifndef DC_TC_WARPS
#define DC_TC_WARPS 4
#endif
#ifndef DC_TC_ROWS_PER_WARP
#define DC_TC_ROWS_PER_WARP 128
#endif
constexpr int TC_WARPS = DC_TC_WARPS;                       // warps per CTA
constexpr int TC_ROWS_PER_WARP = DC_TC_ROWS_PER_WARP;       // rows per warp (16 per m16 tile)
constexpr int TC_UNIT_ROWS = TC_WARPS * TC_ROWS_PER_WARP;   // rows per work unit (512)
constexpr int TC_CHUNK = 256;                               // columns per staged chunk
constexpr int TC_BLOCK = 128;                               // columns per key block
constexpr int TC_MAX_BLOCKS = 4096;                         // block ids a key can hold (12 bits)
constexpr int TC_MAX_COLS = TC_MAX_BLOCKS * TC_BLOCK;       // 524 288 points per side
constexpr int TC_MAX_GRID = 1024;                           // partial-key slots sized for it
constexpr int TC_KEYS = 12;                                 // keys per row: 3 per quad lane
constexpr unsigned TC_VALUE_MASK = 0xFFFFF000u;             // sign, exponent, 11 mantissa bits
constexpr unsigned TC_EMPTY = 0xFFFFFFFFu;
constexpr float TC_PAD_NORM = 60000.0f;                     // norm of a padding column
constexpr float TC_SCALE_LIMIT = 64.0f;                     // |scaled coordinate| below this
// Error bound of the filter in units of u = 2^-24, per unit of (|sp| + |sq|)^2: measured
// on GB300 at most 6.7 over 6.7e7 pairs of cloth-like clouds (accumulation at most 5.4 ulp
// of the largest product, split residuals below 2^-21 |sp||sq| per coordinate).
constexpr float TC_KAPPA = 32.0f;
// the tensor-core pass hands out whole units on demand when there are at least this many
// units per CTA (else it splits the chunk list evenly between its CTAs). Measured: the
// 100-frame 32 768-point trajectory (28 units per CTA) 18.30 -> 17.39 ms per step on demand,
// the 40-frame 10 000-point one (3.5 per CTA) 0.937 -> 0.965 ms, so the cut lies between.
constexpr long long TC_DYN_UNITS_PER_CTA = 16;
static_assert(ROW_PAD % TC_UNIT_ROWS == 0 && COL_PAD % TC_CHUNK == 0 &&
                  TC_CHUNK % TC_BLOCK == 0 && TC_ROWS_PER_WARP % 16 == 0,
              "the tensor-core tiles nest in the padded sizes");

// Form position of the point with form index p. Within a block of TC_BLOCK columns the MMA
// fragments give quad lane t the positions 8 g + 2 t + e (g < 16, e < 2); the point
// 32 t + 2 g + e is stored there, so that every lane's quarter of a block is 32 consecutive
// points, which the recovery re-reads as whole lines (with the quarters interleaved, a
// quarter's 32 points spanned the block's 128). Frames start at multiples of TC_BLOCK rows
// and columns, so the map stays inside each frame, and rows are permuted the same way.
__host__ __device__ inline long long tc_form_pos(long long p) {
    const int b = (int)(p & (TC_BLOCK - 1));
    return (p & ~(long long)(TC_BLOCK - 1)) | (((b >> 1) & 15) << 3) | ((b >> 5) << 1) | (b & 1);
}
// The point that staging thread slot p handles when the forms are written: within a block
// the bit fields [6:5] and [4:3] of p are swapped, so that the 32 lanes of a warp (slots
// 32 w .. 32 w + 31) take the points 32 t + 8 w + x (t < 4, x < 8), whose forms fill the 32
// consecutive positions 32 w .. 32 w + 31 (whole lines), and whose other per-point records
// are four runs of 8 consecutive points. An involution, inside each block.
__host__ __device__ inline int tc_stage_point(int p) {
    return (p & ~(TC_BLOCK - 1)) | (((p >> 3) & 3) << 5) | (((p >> 5) & 3) << 3) | (p & 7);
}
static_assert(TC_BLOCK == 128, "tc_form_pos splits a block into 4 quarters of 16 pairs");
static_assert(ROW_PAD % TC_BLOCK == 0 && COL_PAD % TC_BLOCK == 0,
              "frames start at block boundaries of the forms");
static_assert(TC_BLOCK % TC_ROWS_PER_WARP == 0 || TC_ROWS_PER_WARP % TC_BLOCK == 0,
              "a warp's rows are part of a block or whole blocks");

// ENGINE_TC: the filter on warp-level MMAs; ENGINE_TC5: on tcgen05 MMAs into tensor memory.
// Both write the same keys, which the same kernels merge and resolve.
enum : int { ENGINE_AUTO = 0, ENGINE_DIRECT = 1, ENGINE_TC = 2, ENGINE_TC5 = 3 };
__host__ __device__ inline bool keyed(int engine) {
    return engine == ENGINE_TC || engine == ENGINE_TC5;
}

// (k1, k2, k3) stays the three smallest of the keys inserted
__device__ __forceinline__ void top3_insert(unsigned& k1, unsigned& k2, unsigned& k3,
                                            unsigned v) {
    const unsigned x1 = max(k1, v);
    k1 = min(k1, v);
    const unsigned x2 = max(k2, x1);
    k2 = min(k2, x1);
    k3 = min(k3, x2);
}

// Everything a kernel needs to know about one frame. Built on the device for uniform
// trajectories, on the host for batches.
struct FrameDesc {
    const float* verts;   // [V][3]; NULL for a frame given as points (Chamfer only)
    const int* faces;     // [F][3]
    const uint8_t* mask;  // [F] nullable: faces with a zero entry get area weight 0
    const float* draws;   // [N][3]
    const float* pts;     // [N][3] sim points given directly; NULL when sampled
    const float* tgt;     // [M][3]
    float* loss;          // [1] out
    int* nn_ab;           // [N] out (user buffer or workspace)
    int* nn_ba;           // [M] out (user buffer or workspace)
    float* grad;          // [V][3] out, NULL: no gradient
    float* out_pts;       // [N][3] out of dc_sample, nullable
    int* out_face;        // [N] out of dc_sample, nullable
    float* out_bary;      // [N][3] out of dc_sample, nullable
    int V, F, N, M;
    int Npad, Mpad;       // N rounded up to ROW_PAD, M to COL_PAD
    float weight;         // w_t in the total loss
    float gscale;         // multiplier of dL_t in the gradient
    int row0;             // offset of this frame's sim points in the padded row buffers
    int col0;             // offset of this frame's targets in the padded column buffers
    int cdf0;             // offset of this frame's CDF
    int unit0;            // first Chamfer unit of this frame
    int skip;             // weight (or gradient multiplier) 0: no work, L reported as 0
    int tc_unit0;         // first tensor-core unit of this frame (sim rows, then targets)
};

// Header at the start of every workspace.
struct WsHeader {
    int status;       // first device-detected error (DC_OK if none)
    int n_frames;
    int n_units;
    int total_sub;    // sum over units of their sub-chunk count
    int total_rows;   // sum of Npad
    int total_cols;   // sum of Mpad
    int sum_f;        // sum of F
    int mode;
    int planned;      // batch plan written
    int any_grad;
    int max_v;        // largest V among frames with a gradient
    int slices;       // epilogue slices per frame
    int warps;        // warps per Chamfer CTA (units of warps * ROWS_PER_WARP sim points)
    int engine;       // ENGINE_DIRECT, ENGINE_TC or ENGINE_TC5
    int tc_units;     // tensor-core work units (frame, side, 512 rows)
    int tc_total;     // their chunks of TC_CHUNK columns (live frames only)
    int tc_fallback;  // rows whose keys certified no candidate set (scanned in full)
    int tc_next;      // next unit to take, when the pass hands out whole units on demand
    int pad[46];
};

// Byte offsets of every region of a workspace (computed on the host).
struct Layout {
    size_t hdr, frames, rowpre, colpre, unit_frame, unit_rb, unit_pre, cdf, x, fw, tsoa, tpl,
        pab, pba, nnab, nnba, loss, part, frame_err, fbox, tc_ufr, tc_urb, tc_upre, tca, tcb,
        kab, kba, kpart, tcfb, tcfn, total;
};

struct Sizes {
    long long n_frames, n_units, sum_f, rows, cols;
    long long slices;    // epilogue slices per frame
    long long tc_units;  // tensor-core units (0: no tensor-core regions)
    long long tc_slots;  // CTAs the partial-key buffer is sized for
};

// Epilogue slices per frame: as many as keep all (frame, slice) CTAs in one wave, at most
// MAX_SLICES.
inline int epilogue_slices(long long n_frames) {
    long long s = EPI_CTAS / n_frames;
    return (int)(s < 1 ? 1 : (s > MAX_SLICES ? MAX_SLICES : s));
}

Layout make_layout(const Sizes& s);

// Typed views of a workspace.
struct Ws {
    WsHeader* hdr;
    FrameDesc* frames;
    int* rowpre;       // [n_frames + 1] prefix of Npad
    int* colpre;       // [n_frames + 1] prefix of Mpad
    int* unit_frame;   // [n_units]
    int* unit_rb;      // [n_units] row block of the unit within its frame
    int* unit_pre;     // [n_units + 1] prefix of sub-chunk counts
    float* cdf;        // [sum F]
    float4* x;         // [rows] sampled points (w lane unused), NaN beyond N
    int4* fw;          // [rows] (face, w0, w1, w2 bits)
    float* tsoa;       // [6 * cols] per frame: X2[2 Mpad], Y2, Z2 = {-v, -v} pairs, sentinel beyond M
    float* tpl;        // [3 * cols] per frame: X[Mpad], Y, Z (the targets as given), 0 beyond M
    unsigned long long* pab;  // [rows] packed (d bits << 32 | sub-chunk)
    unsigned long long* pba;  // [cols] packed (d bits << 32 | first row of the lane group)
    int* nnab;         // [rows] fallback neighbour buffers
    int* nnba;         // [cols]
    float* loss;       // [n_frames] fallback loss buffer
    int* frame_err;    // [n_frames] error code of the fused build + area launch, per frame
    float* part;       // [n_frames][slices][2] loss partial sums
    float4* fbox;      // [n_frames] (centre x, y, z, scale) of the tensor-core forms
    int* tc_ufr;       // [tc_units] frame of each tensor-core unit
    int* tc_urb;       // [tc_units] side << 30 | row block
    int* tc_upre;      // [tc_units + 1] prefix of chunk counts
    uint4* tca;        // [(rows + cols) * 2] A forms (sim points, then targets), 32 B each
    uint4* tcb;        // [(rows + cols) * 2] B forms
    unsigned* kab;     // [rows][4 lanes][3] the smallest keys of every sim point
    unsigned* kba;     // [cols][4][3] the same of every target
    unsigned* kpart;   // [tc_slots][2][TC_UNIT_ROWS][4][3] keys of units split between CTAs
    int* tcfb;         // [rows + cols] frame-local indices of the rows the keys did not
                       // certify, each frame's list at its own row (rows + column) range
    int* tcfn;         // [n_frames][2] lengths of those lists (zeroed by the staging)
};

Ws make_ws(void* base, const Layout& L);

// ---------------------------------------------------------------------------------------
// Programmatic dependent launch. Every kernel of the library is launched with programmatic
// stream serialisation and starts with pdl_entry(): it first waits until the grid before it
// on the stream has completed and its memory is visible (so the stream order holds for every
// access), then lets the next grid be launched. The next grid's launch latency thus overlaps
// this grid's run instead of following its end. A kernel launched without the attribute (or
// after a copy or an event) passes the wait at once.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void pdl_entry() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
// The long persistent passes wait the same way but let the next grid be launched only as each
// CTA finishes its work (pdl_trigger at the end; a CTA that exits counts as having let it):
// a next grid launched at their start had its CTAs placed on SMs while the pass still ran,
// which cost 7% (stream-K) to 15% (whole units on demand) of the pass on 64 batched
// trajectories.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

__host__ __device__ inline int round_up(int a, int b) { return (a + b - 1) / b * b; }
__host__ __device__ inline int div_up(int a, int b) { return (a + b - 1) / b; }

// ---------------------------------------------------------------------------------------
// kernel launchers (kernels.cu); each returns cudaGetLastError()
// ---------------------------------------------------------------------------------------
struct UniformArgs {
    const float* verts;
    const int* faces;
    const uint8_t* mask;
    const float* draws;
    const float* pts;
    const float* tgt;
    float* loss;
    int* nn_ab;
    int* nn_ba;
    float* grad;
    float* out_pts;
    int* out_face;
    float* out_bary;
    const float* weight;   // [T] nullable: w_t, default 1
    const float* gtotal;   // [1] nullable (backward only): dJ/dL_total
    const float* gframes;  // [T] nullable (backward only): dJ/dL_t directly
    int bwd;               // 1: gradient multipliers g_t = w_t gtotal + gframes[t]
    int T, V, F, N, M, mode, units_per_frame, subs_per_unit, slices, warps;
    int engine;            // ENGINE_DIRECT, ENGINE_TC or ENGINE_TC5 (calls with a Chamfer)
};

cudaError_t launch_build_uniform(const UniformArgs& a, const Ws& w, cudaStream_t s);
// the frame tables and every frame's area CDF in one launch (block 0 builds the tables, block
// 1 + t computes frame t's CDF from the arguments); the area errors go to w.frame_err, which
// the sampling launch that follows (fold = 1) turns into the status word
cudaError_t launch_build_area(const UniformArgs& a, const Ws& w, cudaStream_t s);
cudaError_t launch_reset(const Ws& w, cudaStream_t s);
cudaError_t launch_area_cdf(const Ws& w, int n_frames, cudaStream_t s);
// tc = 1 also writes the tensor-core forms of the points (the frame boxes must be ready)
cudaError_t launch_sample(const Ws& w, int n_frames, int rows, int fold, int tc, cudaStream_t s);
cudaError_t launch_targets(const Ws& w, int n_frames, int cols, int tc, cudaStream_t s);
// sampling + target staging in one (frame, slice) launch when the largest CDF (max_f
// floats) fits in shared memory, else launch_sample + launch_targets
cudaError_t launch_stage(const Ws& w, int n_frames, int slices, int max_f, int rows, int cols,
                         int fold, int tc, cudaStream_t s);
// frame boxes for the tensor-core forms when no area launch computes them (given points)
cudaError_t launch_bbox(const Ws& w, int n_frames, cudaStream_t s);
// the tensor-core filter over every unit (both sides in Eq. 1) on `grid` CTAs, then the merge
// of the keys of units split between CTAs (n_units: the units the call can have), then the
// exact recovery of every row's minimum and neighbour from its keys into pab (and pba in
// Eq. 1) as (distance bits << 32 | index)
cudaError_t launch_tcpass(const Ws& w, int engine, int grid, long long total_chunks,
                          int n_units, int rows, int cols, int mode, int n_frames,
                          cudaStream_t s);
// CTAs of the tcgen05 pass (one per SM) for an upper bound of its chunk count
int tc5_grid(long long total_chunks);
// CTAs of the tensor-core pass for an upper bound of its chunk count
int tc_grid(long long total_chunks);
cudaError_t launch_chamfer(const Ws& w, int n_units, int total_sub, int mode, int warps,
                           cudaStream_t s);
// resident Chamfer CTAs on the current device for a CTA width (persistent grid size)
int chamfer_grid(int mode, int warps);
// CTA width for a problem: the tuned default if one is set, else the widest width that gives
// every resident CTA at least a few sub-chunks; sub_w4 is the work at width 4
int choose_warps(int mode, long long sub_w4, long long sub_w2, long long sub_w1);
void set_tuned_warps(int warps);  // 0: automatic
void inject_stall();              // the next Chamfer launch never gets its first chunk
int take_stall();                 // 1 once after inject_stall (read by the Chamfer launchers)
int tuned_warps();
// epilogue: neighbour recovery (rescan), loss partials, gradient scatter
enum : int { EPI_RESCAN = 1, EPI_LOSS = 2, EPI_GRAD = 4 };
cudaError_t launch_epilogue(const Ws& w, int n_frames, int slices, int max_v, int mode,
                            int flags, float* total, int tc_grid, cudaStream_t s);
// sum_t w_t L_t of given per-frame losses, in the fixed order of the trajectory calls
cudaError_t launch_loss_total(const float* lf, const float* w, int T, float* total,
                              cudaStream_t s);
cudaError_t launch_chamfer_bwd_points(const float* a, const float* b, const int* nn_ab,
                                      const int* nn_ba, int T, int N, int M, int mode,
                                      const float* g, float* grad_a, cudaStream_t s);

void count_launch(int n = 1);

// Chamfer-kernel event timing hooks (api.cu)
void prof_before(cudaStream_t s);
void prof_after(cudaStream_t s);

}  // namespace dc
