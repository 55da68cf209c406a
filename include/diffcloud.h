/*
 * diffcloud.h -- C ABI of the GB300 (sm_103a) DiffCloud loss library, libdiffcloud.so.
 *
 * The library computes the differentiable mesh-to-point-cloud loss of DiffCloud
 * (Sundaresan et al., "DiffCloud: Real-to-Sim from Point Clouds with Differentiable
 * Simulation and Rendering of Deformable Objects", 2022) and its gradient with respect to
 * every mesh vertex, over a trajectory of T frames:
 *
 *   1. area-weighted surface sampling (Sec. III-B): face f_i = min{ f : C_f > r_f,i A },
 *      C the inclusive prefix sum of the face areas, A = C_{F-1};
 *      point x_i = w0 p_f0 + w1 p_f1 + w2 p_f2 (Eq. 3) with
 *      w = (1 - sqrt(r1), sqrt(r1) (1 - r2), sqrt(r1) r2);
 *   2. Chamfer distance against the frame's observed cloud by brute-force nearest
 *      neighbours, bidirectional mean (Eq. 1) or unidirectional sim->real sum (Eq. 2);
 *   3. the adjoint: dL/dx_i along the chosen neighbours, scattered to the face's vertices
 *      with the barycentric weights as partial derivatives (Eq. 4). The face pick is
 *      piecewise constant in the vertices and contributes nothing.
 *
 * Conventions shared by every entry point:
 *   - Arithmetic is float32. Squared distances are evaluated as dx = a - b per coordinate,
 *     d = fma(dz, dz, fma(dy, dy, dx * dx)); ties go to the lowest index.
 *   - Every array pointer is a DEVICE pointer owned by the caller, C-contiguous, float32 or
 *     int32 as typed, at least 4-byte aligned. The library never allocates device memory:
 *     scratch comes from the caller's workspace `ws` (256-byte aligned, at least the size
 *     the matching *_workspace_size function returns). A workspace serves one call at a
 *     time; calls that overlap on the GPU need separate workspaces.
 *   - Layouts: verts [T][V][3], faces [F][3] (0-based vertex indices, shared by all
 *     frames), draws [T][N][3] holding (r_f, r1, r2) in [0, 1), targets [T][M][3].
 *   - Coordinates must be finite with magnitude at most 1e15.
 *   - Every call is asynchronous on `stream` (a cudaStream_t; NULL is the legacy default
 *     stream) and does not synchronise. Host-side argument errors are returned at once.
 *     Errors found on the device (a face index out of range, a frame of zero total area,
 *     a non-finite or oversized coordinate, a bounded wait that gave up) are recorded in
 *     the workspace and read with dc_ws_status().
 *   - Return value: DC_OK or a negative DC_E* code; dc_last_error() describes the last
 *     failure of the calling thread.
 */
#ifndef DIFFCLOUD_H
#define DIFFCLOUD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* dc_stream_t; /* the same type as cudaStream_t */

enum {
    DC_OK = 0,
    DC_EINVAL = -1,       /* bad argument: null pointer, size <= 0, bad alignment, bad index */
    DC_EDEGENERATE = -2,  /* a frame's total surface area is zero or not finite */
    DC_ECUDA = -3,        /* a CUDA runtime call failed */
    DC_ETIMEOUT = -4,     /* a bounded device-side wait gave up */
    DC_EDEVICE = -5,      /* a device-side consistency check failed */
    DC_ENOSPC = -6        /* the workspace is smaller than required */
};

enum {
    DC_BIDIR_MEAN = 0, /* Eq. 1: mean_i min_j |x_i - y_j|^2 + mean_j min_i |y_j - x_i|^2 */
    DC_UNIDIR_SUM = 1  /* Eq. 2: sum_i min_j |x_i - y_j|^2 (sim -> real only) */
};

/* Bytes of workspace the uniform-trajectory entry points need for T frames of V vertices,
 * F faces, N samples and M target points (M may be 0 for dc_sample). */
size_t dc_workspace_size(int T, int V, int F, int N, int M);

/*
 * Face subsets. The entry points that sample take face_mask [F] (uint8, nullable: every
 * face): only faces with a nonzero entry are sampled. A face outside the subset gets area
 * weight 0 before the prefix sum, so the inverse-CDF pick never selects it -- the paper
 * samples the simulated cloud from the visible half of the cloth in its fold scenario
 * (Sec. IV-F) and from a face subset to mimic occlusion (Sec. IV-C). A subset of zero total
 * area is reported as DC_EDEGENERATE, like a zero-area frame.
 */

/*
 * dc_area_cdf -- the per-frame area weighting of the sampler (Sec. III-B): the face areas
 * A_f = 1/2 |(p1 - p0) x (p2 - p0)| (0 outside face_mask, nullable) and their inclusive prefix
 * sum, cdf [T][F] out (float32, the rounding of the exact prefix sum of the float32 areas;
 * cdf[t][F-1] is the frame's total area A). ws sized by dc_workspace_size(T, V, F, 1, 0).
 * A frame of zero total area is recorded as DC_EDEGENERATE (dc_ws_status).
 */
int dc_area_cdf(const float* verts, const int32_t* faces, const uint8_t* face_mask, int T,
                int V, int F, float* cdf, void* ws, size_t ws_bytes, dc_stream_t stream);

/*
 * dc_sample -- area-weighted surface sampling (Sec. III-B, Eq. 3).
 *   face_mask [F] nullable: sample only these faces (see above).
 *   points   [T][N][3] out: x_i of every frame.
 *   face_idx [T][N] out, nullable: the picked face f_i.
 *   bary     [T][N][3] out, nullable: (w0, w1, w2).
 * Uses ws for the per-frame area CDF.
 */
int dc_sample(const float* verts, const int32_t* faces, const uint8_t* face_mask,
              const float* draws, int T, int V, int F, int N, float* points, int32_t* face_idx,
              float* bary, void* ws, size_t ws_bytes, dc_stream_t stream);

/*
 * dc_chamfer_fwd -- Chamfer distance of given clouds, per frame (Eq. 1 or Eq. 2).
 *   a [T][N][3], b [T][M][3]; mode DC_BIDIR_MEAN or DC_UNIDIR_SUM.
 *   loss  [T] out: L_t.
 *   nn_ab [T][N] out, nullable: index into b of the nearest neighbour of each a point.
 *   nn_ba [T][M] out, nullable (ignored in DC_UNIDIR_SUM): index into a of each b point's.
 * ws sized by dc_workspace_size(T, 1, 1, N, M).
 */
int dc_chamfer_fwd(const float* a, const float* b, int T, int N, int M, int mode, float* loss,
                   int32_t* nn_ab, int32_t* nn_ba, void* ws, size_t ws_bytes,
                   dc_stream_t stream);

/*
 * dc_chamfer_bwd -- gradient of sum_t g_t L_t with respect to a (derivative of Eq. 1 / 2:
 * 2 (a_i - b_j) along each chosen pair, scaled by 1/N, 1/M or 1).
 *   nn_ab [T][N], nn_ba [T][M] (ignored in DC_UNIDIR_SUM) from dc_chamfer_fwd.
 *   grad_loss [T]: g_t.   grad_a [T][N][3] out, overwritten.
 * Needs no workspace. Accumulates with float atomics: the last bits may vary run to run.
 */
int dc_chamfer_bwd(const float* a, const float* b, const int32_t* nn_ab, const int32_t* nn_ba,
                   int T, int N, int M, int mode, const float* grad_loss, float* grad_a,
                   dc_stream_t stream);

/*
 * dc_loss_traj -- the whole loss over a trajectory, and optionally its vertex gradient
 * (Sec. III-B, Eq. 1-4; the per-frame loss of Sec. III-C).
 *   face_mask   [F] nullable: sample only these faces (see above).
 *   frame_w     [T] nullable (all ones): weights w_t. A frame whose weight is 0 is skipped:
 *               no sampling, Chamfer or gradient work is done for it, its L_t is reported as
 *               0 and its gradient rows are 0 (the paper mostly optimises one frame, Sec. III-C).
 *   loss_total  [1] out, nullable: sum_t w_t L_t (fixed summation order).
 *   loss_frames [T] out: L_t.
 *   grad_verts  [T][V][3] out, nullable: w_t dL_t/dverts_t (overwritten). When NULL only
 *               the forward runs.
 *   nn_ab [T][N], nn_ba [T][M] out, nullable: the neighbours (kept for dc_loss_traj_bwd).
 * ws sized by dc_workspace_size(T, V, F, N, M). Sampled points live in ws only.
 */
int dc_loss_traj(const float* verts, const int32_t* faces, const uint8_t* face_mask,
                 const float* draws, const float* targets, int T, int V, int F, int N, int M,
                 int mode,
                 const float* frame_w, float* loss_total, float* loss_frames, float* grad_verts,
                 int32_t* nn_ab, int32_t* nn_ba, void* ws, size_t ws_bytes,
                 dc_stream_t stream);

/*
 * dc_loss_traj_bwd -- vertex gradient of an objective J(L_total, L_1 .. L_T) given the
 * neighbours a previous dc_loss_traj returned: the derivative of Eq. 1 (or Eq. 2) with
 * respect to each sampled point, 2 (x_i - y_nn(i)) / N for every sim point and
 * 2 (x_nn(j) - y_j) / M for every target (Eq. 2: 2 (x_i - y_nn(i)) and no target term),
 * scattered to the picked face's vertices with the barycentric weights of Eq. 3 as partial
 * derivatives (Eq. 4). The face pick is piecewise constant in the vertices and contributes
 * nothing. The sampled points are recomputed from the draws (nothing from the forward is
 * stored but nn_ab / nn_ba). face_mask as in that call.
 *   frame_w     [T] nullable (all ones): the weights w_t of the forward call.
 *   grad_total  [1] nullable: dJ/dL_total, with L_total = sum_t w_t L_t.
 *   grad_frames [T] nullable: dJ/dL_t through the per-frame losses directly.
 *               The library forms g_t = w_t grad_total + grad_frames[t] (a missing one counts
 *               as 0; at least one is required) and g_t = 0 for a frame of weight 0, whose
 *               forward L_t is the constant 0. Frames with g_t = 0 are skipped (zero rows).
 *   grad_verts [T][V][3] out, overwritten: g_t dL_t/dverts_t.
 */
int dc_loss_traj_bwd(const float* verts, const int32_t* faces, const uint8_t* face_mask,
                     const float* draws, const float* targets, int T, int V, int F, int N, int M,
                     int mode, const int32_t* nn_ab, const int32_t* nn_ba, const float* frame_w,
                     const float* grad_total, const float* grad_frames, float* grad_verts,
                     void* ws, size_t ws_bytes, dc_stream_t stream);

/*
 * Batched frames of uneven sizes (many trajectories, one launch sequence).
 * One dc_frame per frame; pointers are device pointers; outputs are nullable.
 */
typedef struct dc_frame {
    const float* verts;   /* [V][3] */
    const int32_t* faces; /* [F][3] */
    const uint8_t* face_mask; /* [F], nullable: sample only these faces (see above) */
    const float* draws;   /* [N][3] */
    const float* targets; /* [M][3] */
    int32_t V, F, N, M;
    float weight;         /* w: weight of L in loss_total and multiplier of its gradient;
                             0 skips the frame (L reported as 0, gradient 0) */
    int32_t tag;          /* caller's label (e.g. trajectory id); not read by the library */
    float* loss;          /* [1] out: L */
    float* grad_verts;    /* [V][3] out, overwritten; NULL: no gradient for this frame */
    int32_t* nn_ab;       /* [N] out, nullable */
    int32_t* nn_ba;       /* [M] out, nullable */
} dc_frame;

/* Bytes of workspace a batch of n_frames frames needs. */
size_t dc_batch_workspace_size(const dc_frame* frames, int n_frames);

/*
 * dc_batch_plan -- validate the frames (host array), lay them out in ws and copy the
 * descriptor tables into it (a host-to-device copy on `stream`). The plan stays valid
 * while the frames' buffers stay where they are; it can be run many times. The layout
 * orders the frames by decreasing N + M (ties keep the order of `frames`); every frame's
 * outputs go to its own buffers, so the order shows only in the rounding of loss_total.
 */
int dc_batch_plan(const dc_frame* frames, int n_frames, int mode, void* ws, size_t ws_bytes,
                  dc_stream_t stream);

/* Bytes of host staging memory dc_batch_plan_async needs for these frames and mode (with
 * the engine that the current dc_tune_set selects); 0 if the frames are invalid. */
size_t dc_batch_plan_bytes(const dc_frame* frames, int n_frames, int mode);

/*
 * dc_batch_plan_async -- dc_batch_plan that does not wait for `stream`: the tables are built
 * in the caller's host_staging (host memory of at least dc_batch_plan_bytes bytes; pinned, for
 * the copy to be asynchronous) and copied from there on `stream`. The caller keeps
 * host_staging unchanged until that copy has completed (e.g. until an event recorded on
 * `stream` after the call, or after the batch's first run, has completed).
 */
int dc_batch_plan_async(const dc_frame* frames, int n_frames, int mode, void* ws,
                        size_t ws_bytes, void* host_staging, size_t staging_bytes,
                        dc_stream_t stream);

/*
 * dc_batch_run -- forward (and the gradient of every frame whose grad_verts is set) of a
 * planned batch: sampling, one persistent Chamfer launch over all frames, neighbours,
 * losses, gradient scatter. loss_total [1] out, nullable: sum of w L over the frames.
 * Reads only device memory, so the launch sequence can be captured in a CUDA graph.
 */
int dc_batch_run(void* ws, float* loss_total, dc_stream_t stream);

/*
 * Tuning of the nearest-neighbour search. Three engines compute the same neighbours and losses
 * (the float32 direct form, lowest index among equal distances):
 *   DC_ENGINE_TENSOR -- a tensor-core filter: the expanded form |p|^2 - 2 p.q + |q|^2 on
 *     split-fp16 operands, warp-level MMAs (16 points x 8 candidates each), keeps per point
 *     and quarter of the candidates the three best blocks of 128, and the direct form
 *     re-checks only the blocks that an error bound cannot exclude (every candidate when it
 *     cannot certify the blocks). Frames of at most 524 288 points per side.
 *     DC_ENGINE_AUTO takes it for calls (and batch plans) of at least 1e9 pairs and 5e7
 *     pairs per frame on average, where it pays back its fixed costs; else the direct engine.
 *   DC_ENGINE_TCGEN05 -- the same filter on tcgen05 MMAs (128 points x 128 candidates each)
 *     into tensor memory; same keys, same recovery, same results.
 *   DC_ENGINE_DIRECT -- every pair in the direct form on the CUDA cores; a CTA of w warps
 *     (w = 1, 2 or 4) holds w * 512 sim points in registers while target chunks stream
 *     through it. warps_per_cta = 0 picks two warps when that gives every resident CTA
 *     several work items, else one.
 * dc_tune_set sets both for every later call and plan in the process (an autotuner times
 * them per problem size and sets the winner before its calls); batch plans keep the choice
 * they were planned with.
 */
enum { DC_ENGINE_AUTO = 0, DC_ENGINE_DIRECT = 1, DC_ENGINE_TENSOR = 2, DC_ENGINE_TCGEN05 = 3 };

typedef struct dc_tune {
    int32_t warps_per_cta; /* direct engine: 0 (automatic), 1, 2 or 4 */
    int32_t engine;        /* DC_ENGINE_AUTO, _DIRECT, _TENSOR or _TCGEN05 */
} dc_tune;

int dc_tune_set(const dc_tune* tune); /* NULL restores automatic */
int dc_tune_get(dc_tune* tune);

/*
 * dc_loss_total -- the weighted total of given per-frame losses, sum_t w_t L_t (the
 * objective over a trajectory, Sec. III-C), in the same fixed summation order as the
 * loss_total of dc_loss_traj: a caller that computed a trajectory's frames in several
 * batches gets the total the whole trajectory would have given in one call.
 *   loss_frames [T] device; frame_w [T] device, nullable (all ones); loss_total [1] device out.
 */
int dc_loss_total(const float* loss_frames, const float* frame_w, int T, float* loss_total,
                  dc_stream_t stream);

/*
 * dc_ws_status -- synchronise `stream` and return the first device-side error recorded in
 * ws by the calls issued so far (DC_OK if none). The next call on ws clears it.
 */
int dc_ws_status(const void* ws, dc_stream_t stream);

/*
 * dc_loss_traj_noalloc -- dc_loss_traj for callers that cannot allocate device memory when
 * they need the loss (a plug-in whose host framework owns all device memory, a real-time
 * loop that forbids allocator calls after start-up). The paper has no counterpart: this is
 * an interface convenience.
 *   Arguments and outputs as in dc_loss_traj; instead of a workspace it uses a built-in
 *   16 MiB scratch array in device memory, which every GPU that loads the library holds
 *   until the process exits.
 *   status [1] device, nullable: receives the device-side error code of this call
 *   (DC_OK, DC_EINVAL, DC_EDEGENERATE, ...), since the scratch is not visible to the caller.
 *   Returns DC_ENOSPC when dc_workspace_size(T, V, F, N, M) exceeds 16 MiB (seventeen frames
 *   of 10 000 samples against 10 000 targets on a 2 500-vertex mesh); that check comes
 *   before any pointer is examined or any CUDA call is made.
 *   It calls no allocator. Outside a stream capture every call looks up the scratch array's
 *   device address with the current device (the lookup allocates nothing), so a context that
 *   was reset is followed; a call inside a capture reuses the address of the last call made
 *   outside one, so make the first call on a device before any stream capture (a capturing
 *   first call returns DC_EINVAL).
 *   All calls on a device share the one array and each overwrites it: calls that may overlap
 *   on the GPU (different streams, or threads without ordering) race and must not be issued.
 */
int dc_loss_traj_noalloc(const float* verts, const int32_t* faces, const uint8_t* face_mask,
                         const float* draws, const float* targets, int T, int V, int F, int N,
                         int M, int mode,
                         const float* frame_w, float* loss_total, float* loss_frames,
                         float* grad_verts, int32_t* nn_ab, int32_t* nn_ba, int32_t* status,
                         dc_stream_t stream);

/*
 * dc_fp32_fma_rate -- measured FP32 FMA throughput of the current device, in flop/s (an FMA
 * counts 2). The paper has no counterpart: this is the measured cross-check of the peak the
 * Chamfer kernel's roofline fraction is reported against. packed = 0 times scalar FMAs,
 * packed = 1 packed f32x2 FMAs; every SM runs independent chains at full occupancy for `iters`
 * iterations (16 lane operations per thread each; 20000 takes a few milliseconds). Runs on
 * `stream` and waits for it; allocates nothing.
 */
int dc_fp32_fma_rate(int packed, int iters, double* flop_per_s, dc_stream_t stream);

/*
 * dc_test_inject_stall -- for testing the failure detection (the paper has no counterpart).
 * The next Chamfer launch in the process never requests the first target chunk of each CTA,
 * so the bounded waits on it give up after 2 s: the call completes, its workspace reports
 * DC_ETIMEOUT (dc_ws_status), and the device stays usable for the next call.
 */
int dc_test_inject_stall(void);

/* Description of the last failure on the calling thread ("" if none). */
const char* dc_last_error(void);

/* Number of kernels this library has launched in this process (host-side count). */
long long dc_launch_count(void);

/*
 * Timing of the Chamfer kernel: dc_prof_start(cap) makes the next (up to cap) Chamfer
 * launches record a CUDA event pair on their stream; dc_prof_stop synchronises those
 * events and returns their summed duration (ms) and count, and ends recording.
 */
int dc_prof_start(int cap);
int dc_prof_stop(float* total_ms, int* launches);

#ifdef __cplusplus
}
#endif

#endif /* DIFFCLOUD_H */
