// Frame tables, area CDF, area-weighted sampling and target staging (Sec. III-B, Eq. 3).
#include <cuda_fp16.h>
#include <math.h>

#include "dc_internal.cuh"

namespace dc {

namespace {

constexpr float ROW_SENTINEL = 1e18f;   // coordinate of padded sim points
constexpr float COL_SENTINEL = -1e18f;  // coordinate of padded target points

__device__ __forceinline__ void set_status(int* st, int code) { atomicCAS(st, DC_OK, code); }

// largest k in [0, n) with pre[k] <= g (pre is non-decreasing, pre[0] = 0)
__device__ __forceinline__ int last_le(const int* pre, int n, int g) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= g)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ bool coord_ok(float v) { return fabsf(v) <= COORD_MAX; }

// Frame k's weight w_t in the total and the multiplier of its gradient. The forward uses w_t
// for both. The recomputing backward gets the objective's derivatives: g_t = dJ/dL_t =
// w_t dJ/dL_total + dJ/dL_t(direct), and 0 for a frame of weight 0, whose forward L_t is the
// constant 0.
__device__ __forceinline__ void frame_scales(const UniformArgs& a, int k, float& w, float& gs) {
    w = a.weight ? a.weight[k] : 1.0f;
    if (a.bwd) {
        const float gt = a.gtotal ? a.gtotal[0] : 0.0f;
        const float gf = a.gframes ? a.gframes[k] : 0.0f;
        gs = w == 0.0f ? 0.0f : __fadd_rn(__fmul_rn(w, gt), gf);
    } else {
        gs = w;
    }
}

// ---------------------------------------------------------------------------------------
// tensor-core forms (see dc_internal.cuh): frame box, centre and scale, and the A / B forms
// ---------------------------------------------------------------------------------------
// Centre and scale of a frame over its sim-side points P[np] (vertices or given points) and
// its targets Y[ny]: the centre of their bounding box and the power of two sig with
// |(p - c) sig| < TC_SCALE_LIMIT. Coordinates that fail the range check are left out (they
// are reported as DC_EINVAL elsewhere). The whole block (a multiple of 32 threads) calls it.
__device__ void frame_box(const float* __restrict__ P, int np, const float* __restrict__ Y,
                          int ny, float4* out) {
    __shared__ float s_box[32][6];
    float b[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
    for (int side = 0; side < 2; ++side) {
        const float* Q = side ? Y : P;
        const int n = side ? ny : np;
        if (!Q) continue;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float v = Q[3LL * i + k];
                if (coord_ok(v)) {
                    b[k] = fminf(b[k], v);
                    b[3 + k] = fmaxf(b[3 + k], v);
                }
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            b[k] = fminf(b[k], __shfl_xor_sync(0xffffffffu, b[k], o));
            b[3 + k] = fmaxf(b[3 + k], __shfl_xor_sync(0xffffffffu, b[3 + k], o));
        }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0)
        for (int k = 0; k < 6; ++k) s_box[warp][k] = b[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < nw; ++q)
            for (int k = 0; k < 3; ++k) {
                b[k] = fminf(b[k], s_box[q][k]);
                b[3 + k] = fmaxf(b[3 + k], s_box[q][3 + k]);
            }
        float c[3], R = 0.0f;
        for (int k = 0; k < 3; ++k) {
            c[k] = b[k] <= b[3 + k] ? 0.5f * b[k] + 0.5f * b[3 + k] : 0.0f;
            if (b[k] <= b[3 + k]) R = fmaxf(R, fmaxf(b[3 + k] - c[k], c[k] - b[k]));
        }
        R *= 1.0f + 0x1p-20f;  // covers the rounding of c
        float sig = 1.0f;
        if (R > 0.0f && R < 1e30f) {
            int e = 0;
            frexpf(R, &e);  // R < 2^e
            sig = ldexpf(1.0f, 6 - e);  // R sig < 64 = TC_SCALE_LIMIT
        }
        *out = make_float4(c[0], c[1], c[2], sig);
    }
    __syncthreads();
}

__device__ __forceinline__ unsigned pack_h2(__half lo, __half hi) {
    return (unsigned)__half_as_ushort(lo) | ((unsigned)__half_as_ushort(hi) << 16);
}

// The A and B forms of form index p for the point (x, y, z) of a frame with box `box`,
// stored at position tc_form_pos(p); a padding point gets forms that never win a minimum
// (A = 0; B adds TC_PAD_NORM, above any real scaled squared distance, 4 * 3 * 64^2).
__device__ __forceinline__ void write_forms(const Ws& w, long long p, float x, float y, float z,
                                            float4 box, bool real) {
    uint4 a0, a1, b0, b1;
    const __half one = __float2half_rn(1.0f);
    if (real) {
        const float sc[3] = {__fmul_rn(__fsub_rn(x, box.x), box.w),
                             __fmul_rn(__fsub_rn(y, box.y), box.w),
                             __fmul_rn(__fsub_rn(z, box.z), box.w)};
        __half h[3], l[3], H[3], L[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            h[k] = __float2half_rn(sc[k]);
            l[k] = __float2half_rn(__fsub_rn(sc[k], __half2float(h[k])));
            H[k] = __float2half_rn(-2.0f * __half2float(h[k]));  // exact
            L[k] = __float2half_rn(-2.0f * __half2float(l[k]));
        }
        const float n = __fmaf_rn(sc[2], sc[2], __fmaf_rn(sc[1], sc[1], __fmul_rn(sc[0], sc[0])));
        const __half nh = __float2half_rn(n), nl = __float2half_rn(__fsub_rn(n, __half2float(nh)));
        a0 = make_uint4(pack_h2(h[0], h[0]), pack_h2(l[0], l[0]), pack_h2(h[1], h[1]),
                        pack_h2(l[1], l[1]));
        a1 = make_uint4(pack_h2(h[2], h[2]), pack_h2(l[2], l[2]), pack_h2(one, one),
                        pack_h2(nh, nl));
        b0 = make_uint4(pack_h2(H[0], L[0]), pack_h2(H[0], L[0]), pack_h2(H[1], L[1]),
                        pack_h2(H[1], L[1]));
        b1 = make_uint4(pack_h2(H[2], L[2]), pack_h2(H[2], L[2]), pack_h2(nh, nl),
                        pack_h2(one, one));
    } else {
        const __half zero = __float2half_rn(0.0f), pad = __float2half_rn(TC_PAD_NORM);
        a0 = a1 = b0 = make_uint4(0u, 0u, 0u, 0u);
        b1 = make_uint4(0u, 0u, pack_h2(pad, zero), pack_h2(one, one));
    }
    // group of 8 positions = 16 uint4: K 0..7 of the 8 points, then K 8..15
    const long long s = tc_form_pos(p);
    const long long q = (s >> 3) * 16 + (s & 7);
    w.tca[q] = a0;
    w.tca[q + 8] = a1;
    w.tcb[q] = b0;
    w.tcb[q + 8] = b1;
}

// ---------------------------------------------------------------------------------------
// uniform trajectory -> frame table, row/column prefixes and Chamfer units. One block: the
// Chamfer work of a frame whose weight (or gradient multiplier) is 0 is left out, which
// needs a prefix count of the live frames.
// ---------------------------------------------------------------------------------------
constexpr int BUILD_THREADS = 1024;

// the whole block (blockDim.x threads, a multiple of 32, at most BUILD_THREADS) builds
__device__ void build_uniform(const UniformArgs& a, const Ws& w) {
    __shared__ int s_warp[BUILD_THREADS / 32];
    __shared__ int s_carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int Npad = ((a.N + ROW_PAD - 1) / ROW_PAD) * ROW_PAD;
    const int Mpad = ((a.M + COL_PAD - 1) / COL_PAD) * COL_PAD;
    const int upf = a.units_per_frame, spu = a.subs_per_unit;
    const int n_units = a.T * upf;
    if (tid == 0) s_carry = 0;
    __syncthreads();
    const int nt = blockDim.x;  // a multiple of 32, at most BUILD_THREADS
    // frames, in chunks of nt, with a running count of live frames
    for (int k0 = 0; k0 < a.T; k0 += nt) {
        const int k = k0 + tid;
        bool live = false;
        if (k < a.T) {
            FrameDesc f;
            f.verts = a.verts ? a.verts + 3LL * k * a.V : nullptr;
            f.faces = a.faces;
            f.mask = a.mask;
            f.draws = a.draws ? a.draws + 3LL * k * a.N : nullptr;
            f.pts = a.pts ? a.pts + 3LL * k * a.N : nullptr;
            f.tgt = a.tgt ? a.tgt + 3LL * k * a.M : nullptr;
            f.loss = a.loss ? a.loss + k : w.loss + k;
            f.nn_ab = a.nn_ab ? a.nn_ab + (long long)k * a.N : w.nnab + (long long)k * Npad;
            f.nn_ba = a.nn_ba ? a.nn_ba + (long long)k * a.M : w.nnba + (long long)k * Mpad;
            f.grad = a.grad ? a.grad + 3LL * k * a.V : nullptr;
            f.out_pts = a.out_pts ? a.out_pts + 3LL * k * a.N : nullptr;
            f.out_face = a.out_face ? a.out_face + (long long)k * a.N : nullptr;
            f.out_bary = a.out_bary ? a.out_bary + 3LL * k * a.N : nullptr;
            f.V = a.V;
            f.F = a.F;
            f.N = a.N;
            f.M = a.M;
            f.Npad = Npad;
            f.Mpad = Mpad;
            frame_scales(a, k, f.weight, f.gscale);
            f.skip = f.weight == 0.0f || f.gscale == 0.0f;
            live = !f.skip;
            f.row0 = k * Npad;
            f.col0 = k * Mpad;
            f.cdf0 = k * a.F;
            f.unit0 = 0;  // set below: live frames before this one
            w.frames[k] = f;
            w.rowpre[k] = k * Npad;
            w.colpre[k] = k * Mpad;
        }
        // exclusive prefix of live flags over the chunk
        const unsigned bal = __ballot_sync(0xffffffffu, live);
        const int in_warp = __popc(bal & ((1u << lane) - 1u));
        if (lane == 0) s_warp[warp] = __popc(bal);
        __syncthreads();
        int before = s_carry;
        for (int q = 0; q < warp; ++q) before += s_warp[q];
        if (k < a.T) w.frames[k].unit0 = before + in_warp;
        __syncthreads();
        if (tid == nt - 1) s_carry = before + in_warp + (live ? 1 : 0);
        __syncthreads();
    }
    if (tid == 0) {
        w.rowpre[a.T] = a.T * Npad;
        w.colpre[a.T] = a.T * Mpad;
        WsHeader* h = w.hdr;
        h->status = DC_OK;
        h->n_frames = a.T;
        h->n_units = n_units;
        h->total_sub = s_carry * upf * spu;
        h->total_rows = a.T * Npad;
        h->total_cols = a.T * Mpad;
        h->sum_f = a.T * a.F;
        h->mode = a.mode;
        h->planned = 0;
        h->any_grad = a.grad != nullptr;
        h->max_v = a.V;
        h->slices = a.slices;
        h->warps = a.warps;
        h->engine = keyed(a.engine) ? a.engine : ENGINE_DIRECT;
        h->tc_units = 0;
        h->tc_total = 0;
        h->tc_fallback = 0;
        h->tc_next = 0;
    }
    __syncthreads();  // the frames' live counts are written
    // units: a skipped frame's units carry no sub-chunks
    for (int u = tid; u <= n_units; u += nt) {
        if (u == n_units) {
            w.unit_pre[u] = s_carry * upf * spu;
            continue;
        }
        const int k = u / upf, rb = u - k * upf;
        const FrameDesc* f = w.frames + k;
        w.unit_frame[u] = k;
        w.unit_rb[u] = rb;
        w.unit_pre[u] = (f->unit0 * upf + (f->skip ? 0 : rb)) * spu;
    }
    // tensor-core units: per frame the sim rows (side 0) against the targets, then in Eq. 1
    // the targets (side 1) against the sim points; a skipped frame's units carry no chunks
    const int tu0 = div_up(a.N, TC_UNIT_ROWS);
    const int tu1 = a.mode == DC_BIDIR_MEAN ? div_up(a.M, TC_UNIT_ROWS) : 0;
    const int tupf = tu0 + tu1;
    if (keyed(a.engine)) {
        const int c0 = Mpad / TC_CHUNK, c1 = Npad / TC_CHUNK;  // chunks per unit, by side
        const int per_frame = tu0 * c0 + tu1 * c1;
        const int n_tc = a.T * tupf;
        for (int u = tid; u <= n_tc; u += nt) {
            if (u == n_tc) {
                w.tc_upre[u] = s_carry * per_frame;
                continue;
            }
            const int k = u / tupf, r = u - k * tupf;
            const int side = r >= tu0 ? 1 : 0, rb = side ? r - tu0 : r;
            const FrameDesc* f = w.frames + k;
            w.tc_ufr[u] = k;
            w.tc_urb[u] = (side << 30) | rb;
            w.tc_upre[u] = f->unit0 * per_frame +
                           (f->skip ? 0 : (side ? tu0 * c0 + rb * c1 : rb * c0));
        }
        if (tid == 0) {
            w.hdr->tc_units = n_tc;
            w.hdr->tc_total = s_carry * per_frame;
        }
    }
    // unit0 now holds "live frames before"; restore its documented meaning
    __syncthreads();
    for (int k = tid; k < a.T; k += nt) {
        w.frames[k].unit0 = k * upf;
        w.frames[k].tc_unit0 = k * tupf;
    }
}

__global__ void __launch_bounds__(BUILD_THREADS) k_build_uniform(UniformArgs a, Ws w) {
    pdl_entry();
    build_uniform(a, w);
}

// ---------------------------------------------------------------------------------------
// area CDF: two-float (compensated) prefix sum of the float32 face areas, so that the
// stored C_f is the float32 rounding of the exact prefix sum of those areas
// ---------------------------------------------------------------------------------------
struct FF {
    float hi, lo;
};

__device__ __forceinline__ FF ff_norm(float s, float e) {
    float h = __fadd_rn(s, e);
    return {h, __fsub_rn(e, __fsub_rn(h, s))};
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ FF ff_add(FF a, FF b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    return ff_norm(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ FF ff_add1(FF a, float b) {
    float s, e;
    two_sum(a.hi, b, s, e);
    return ff_norm(s, __fadd_rn(e, a.lo));
}

// area of face f = 1/2 |(p1 - p0) x (p2 - p0)|; flags bad indices / coordinates
__device__ __forceinline__ float face_area(const float* __restrict__ verts,
                                           const int* __restrict__ faces, int V, int f,
                                           bool& bad_idx, bool& bad_val) {
    const int i0 = faces[3 * f], i1 = faces[3 * f + 1], i2 = faces[3 * f + 2];
    if ((unsigned)i0 >= (unsigned)V || (unsigned)i1 >= (unsigned)V ||
        (unsigned)i2 >= (unsigned)V) {
        bad_idx = true;
        return 0.0f;
    }
    const float* p0 = verts + 3LL * i0;
    const float* p1 = verts + 3LL * i1;
    const float* p2 = verts + 3LL * i2;
    float q[9] = {p0[0], p0[1], p0[2], p1[0], p1[1], p1[2], p2[0], p2[1], p2[2]};
#pragma unroll
    for (int k = 0; k < 9; ++k) bad_val |= !coord_ok(q[k]);
    // explicit roundings: both passes of the scan must see bit-identical areas
    const float e1x = __fsub_rn(q[3], q[0]), e1y = __fsub_rn(q[4], q[1]),
                e1z = __fsub_rn(q[5], q[2]);
    const float e2x = __fsub_rn(q[6], q[0]), e2y = __fsub_rn(q[7], q[1]),
                e2z = __fsub_rn(q[8], q[2]);
    const float cx = __fsub_rn(__fmul_rn(e1y, e2z), __fmul_rn(e1z, e2y));
    const float cy = __fsub_rn(__fmul_rn(e1z, e2x), __fmul_rn(e1x, e2z));
    const float cz = __fsub_rn(__fmul_rn(e1x, e2y), __fmul_rn(e1y, e2x));
    const float n2 = __fmaf_rn(cz, cz, __fmaf_rn(cy, cy, __fmul_rn(cx, cx)));
    return __fmul_rn(0.5f, __fsqrt_rn(n2));
}

// The area weight of face f: its area, or 0 for a face outside the sampled subset
// (Sec. IV-F). The face is still checked, so that bad indices are reported either way.
__device__ __forceinline__ float face_weight(const float* __restrict__ verts,
                                             const int* __restrict__ faces,
                                             const uint8_t* __restrict__ mask, int V, int f,
                                             bool& bad_idx, bool& bad_val) {
    const float a = face_area(verts, faces, V, f, bad_idx, bad_val);
    return (mask && mask[f] == 0) ? 0.0f : a;
}

constexpr int CDF_THREADS = 1024;

// What the area step needs to know about one frame.
struct AreaFrame {
    const float* verts;   // [V][3]
    const int* faces;     // [F][3]
    const uint8_t* mask;  // [F] nullable
    float* grad;          // [V][3] nullable: zeroed here for the epilogue's accumulation
    float* cdf;           // [F] out
    int F, V;
    bool skip;            // weight 0: only the gradient (zero) is written
};

// One block (CDF_THREADS threads) computes one frame's area CDF; errors go to *err with
// atomicCAS(DC_OK -> code), so the first one stays.
__device__ void area_cdf(const AreaFrame& fr, int* err) {
    __shared__ FF s_w[32];
    if (fr.skip) {
        if (fr.grad)
            for (int e = threadIdx.x; e < 3 * fr.V; e += CDF_THREADS) fr.grad[e] = 0.0f;
        return;
    }
    const float* verts = fr.verts;
    const int* faces = fr.faces;
    const uint8_t* mask = fr.mask;
    const int F = fr.F, V = fr.V;
    float* cdf = fr.cdf;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (F + CDF_THREADS - 1) / CDF_THREADS;
    const int f0 = min(F, tid * per), f1 = min(F, f0 + per);
    bool bad_idx = false, bad_val = false;

    FF v = {0.0f, 0.0f};
    // pass 1: the segment's area weights, kept in the thread's own slots of the CDF buffer
    for (int f = f0; f < f1; ++f) {
        const float a = face_weight(verts, faces, mask, V, f, bad_idx, bad_val);
        cdf[f] = a;
        v = ff_add1(v, a);
    }

    // block-wide inclusive scan of the segment sums
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        FF u = {__shfl_up_sync(0xffffffffu, v.hi, o), __shfl_up_sync(0xffffffffu, v.lo, o)};
        if (lane >= o) v = ff_add(u, v);
    }
    if (lane == 31) s_w[warp] = v;
    __syncthreads();
    if (warp == 0) {
        FF t = s_w[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            FF u = {__shfl_up_sync(0xffffffffu, t.hi, o), __shfl_up_sync(0xffffffffu, t.lo, o)};
            if (lane >= o) t = ff_add(u, t);
        }
        s_w[lane] = t;
    }
    __syncthreads();
    FF ex = {__shfl_up_sync(0xffffffffu, v.hi, 1), __shfl_up_sync(0xffffffffu, v.lo, 1)};
    if (lane == 0) ex = {0.0f, 0.0f};
    FF run = warp > 0 ? ff_add(s_w[warp - 1], ex) : ex;

    for (int f = f0; f < f1; ++f) {
        run = ff_add1(run, cdf[f]);  // pass 2 reads back this thread's own area weights
        cdf[f] = run.hi;
    }
    if (bad_idx || bad_val) set_status(err, DC_EINVAL);
    // the gradient of this frame starts from zero (accumulated by the epilogue)
    if (fr.grad)
        for (int e = tid; e < 3 * V; e += CDF_THREADS) fr.grad[e] = 0.0f;
    if (f1 == F && f0 < f1) {
        const float A = run.hi;
        if (!(A > 0.0f) || !isfinite(A)) set_status(err, DC_EDEGENERATE);
    }
}

// one block per frame of the table
__global__ void __launch_bounds__(CDF_THREADS) k_area_cdf(Ws w) {
    pdl_entry();
    const FrameDesc* fr = w.frames + blockIdx.x;
    if (!fr->verts) return;
    const AreaFrame af{fr->verts, fr->faces, fr->mask, fr->grad, w.cdf + fr->cdf0,
                       fr->F, fr->V, fr->skip != 0};
    area_cdf(af, &w.hdr->status);
    if (keyed(w.hdr->engine) && !fr->skip)
        frame_box(fr->verts, fr->V, fr->tgt, fr->M, &w.fbox[blockIdx.x]);
}

// Uniform trajectory: block 0 builds the tables (as k_build_uniform) while block 1 + t
// computes frame t's CDF from the arguments, which is where the table's entry would point.
// The tables' builder resets the status word, so the area blocks keep their errors apart,
// one code per frame in w.frame_err, for the sampling launch to report.
__global__ void __launch_bounds__(CDF_THREADS) k_build_area(UniformArgs a, Ws w) {
    pdl_entry();
    if (blockIdx.x == 0) {
        build_uniform(a, w);
        return;
    }
    __shared__ int s_err;
    const int t = blockIdx.x - 1;
    if (threadIdx.x == 0) s_err = DC_OK;
    __syncthreads();
    float wt, gs;
    frame_scales(a, t, wt, gs);
    const AreaFrame af{a.verts + 3LL * t * a.V, a.faces, a.mask,
                       a.grad ? a.grad + 3LL * t * a.V : nullptr, w.cdf + (long long)t * a.F,
                       a.F, a.V, wt == 0.0f || gs == 0.0f};
    area_cdf(af, &s_err);
    __syncthreads();
    if (threadIdx.x == 0) w.frame_err[t] = s_err;
    if (keyed(a.engine) && !af.skip)
        frame_box(af.verts, a.V, a.tgt ? a.tgt + 3LL * t * a.M : nullptr, a.M, &w.fbox[t]);
}

// frame boxes of frames given as points (no area launch)
__global__ void __launch_bounds__(512) k_bbox(Ws w) {
    pdl_entry();
    const FrameDesc* fr = w.frames + blockIdx.x;
    if (fr->skip) return;
    frame_box(fr->pts ? fr->pts : fr->verts, fr->pts ? fr->N : fr->V, fr->tgt, fr->M,
              &w.fbox[blockIdx.x]);
}

// ---------------------------------------------------------------------------------------
// sampling: face pick by inverse CDF (Sec. III-B) and barycentric point (Eq. 3)
// ---------------------------------------------------------------------------------------
// Row g (frame-local index i) of frame fr, with the frame's CDF at `cdf` (global or shared).
__device__ __forceinline__ void sample_row(const Ws& w, const FrameDesc* fr, int i, int g,
                                           const float* cdf, bool tc, float4 box) {
    float4 x = make_float4(ROW_SENTINEL, ROW_SENTINEL, ROW_SENTINEL, 0.0f);
    int4 q = make_int4(-1, 0, 0, 0);
    if (i < fr->N) {
        if (fr->pts) {
            const float* p = fr->pts + 3LL * i;
            x = make_float4(p[0], p[1], p[2], 0.0f);
            if (!coord_ok(x.x) || !coord_ok(x.y) || !coord_ok(x.z))
                set_status(&w.hdr->status, DC_EINVAL);
        } else {
            const float* r = fr->draws + 3LL * i;
            const float rf = r[0], r1 = r[1], r2 = r[2];
            if (!(rf >= 0.0f && rf <= 1.0f && r1 >= 0.0f && r1 <= 1.0f && r2 >= 0.0f &&
                  r2 <= 1.0f))
                set_status(&w.hdr->status, DC_EINVAL);
            const int F = fr->F;
            const float t = __fmul_rn(rf, cdf[F - 1]);
            int lo = 0, hi = F;  // first f with cdf[f] > t
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (cdf[mid] > t)
                    hi = mid;
                else
                    lo = mid + 1;
            }
            const int f = min(lo, F - 1);
            const int i0 = fr->faces[3 * f], i1 = fr->faces[3 * f + 1], i2 = fr->faces[3 * f + 2];
            const int V = fr->V;
            if ((unsigned)i0 < (unsigned)V && (unsigned)i1 < (unsigned)V &&
                (unsigned)i2 < (unsigned)V) {
                const float* p0 = fr->verts + 3LL * i0;
                const float* p1 = fr->verts + 3LL * i1;
                const float* p2 = fr->verts + 3LL * i2;
                const float s = __fsqrt_rn(r1);
                const float w0 = __fsub_rn(1.0f, s);
                const float w1 = __fmul_rn(s, __fsub_rn(1.0f, r2));
                const float w2 = __fmul_rn(s, r2);
                x.x = __fmaf_rn(w2, p2[0], __fmaf_rn(w1, p1[0], __fmul_rn(w0, p0[0])));
                x.y = __fmaf_rn(w2, p2[1], __fmaf_rn(w1, p1[1], __fmul_rn(w0, p0[1])));
                x.z = __fmaf_rn(w2, p2[2], __fmaf_rn(w1, p1[2], __fmul_rn(w0, p0[2])));
                q = make_int4(f, __float_as_int(w0), __float_as_int(w1), __float_as_int(w2));
                if (fr->out_face) fr->out_face[i] = f;
                if (fr->out_bary) {
                    fr->out_bary[3LL * i] = w0;
                    fr->out_bary[3LL * i + 1] = w1;
                    fr->out_bary[3LL * i + 2] = w2;
                }
            } else {
                set_status(&w.hdr->status, DC_EINVAL);
                x = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            }
            if (fr->out_pts) {
                fr->out_pts[3LL * i] = x.x;
                fr->out_pts[3LL * i + 1] = x.y;
                fr->out_pts[3LL * i + 2] = x.z;
            }
        }
    }
    w.x[g] = x;
    w.fw[g] = q;
    w.pab[g] = EMPTY;
    if (tc) write_forms(w, g, x.x, x.y, x.z, box, i < fr->N);
}

// Target j (frame-local) of frame fr at padded column g: the negated duplicated planes the
// Chamfer kernel stages, the compact planes the epilogue re-scans, and the column minimum.
__device__ __forceinline__ void stage_target(const Ws& w, const FrameDesc* fr, int j, int g,
                                             bool tc, float4 box) {
    float vx = COL_SENTINEL, vy = COL_SENTINEL, vz = COL_SENTINEL;
    const bool real = j < fr->M;
    if (real) {
        const float* p = fr->tgt + 3LL * j;
        vx = p[0];
        vy = p[1];
        vz = p[2];
        if (!coord_ok(vx) || !coord_ok(vy) || !coord_ok(vz)) set_status(&w.hdr->status, DC_EINVAL);
    }
    // planes of negated {-v, -v} pairs: X2 [2 Mpad], Y2 [2 Mpad], Z2 [2 Mpad]; the Chamfer
    // kernel forms x - v as x + (-v), which rounds identically
    float2* P = reinterpret_cast<float2*>(w.tsoa + 6LL * fr->col0);
    P[j] = make_float2(-vx, -vx);
    P[fr->Mpad + j] = make_float2(-vy, -vy);
    P[2 * fr->Mpad + j] = make_float2(-vz, -vz);
    // compact planes as given (0 beyond M) for the epilogue's re-scans
    float* Q = w.tpl + 3LL * fr->col0;
    Q[j] = real ? vx : 0.0f;
    Q[fr->Mpad + j] = real ? vy : 0.0f;
    Q[2 * fr->Mpad + j] = real ? vz : 0.0f;
    w.pba[g] = EMPTY;
    if (tc) write_forms(w, (long long)w.hdr->total_rows + g, vx, vy, vz, box, real);
}

// the area errors that a fused build + area launch left for frame k
__device__ __forceinline__ void fold_area_err(const Ws& w, int k) {
    const int code = w.frame_err[k];
    if (code != DC_OK) set_status(&w.hdr->status, code);
}

__global__ void __launch_bounds__(256) k_sample(Ws w, int n_frames, int rows, int fold, int tc) {
    pdl_entry();
    // rows is a whole number of blocks, so the staging order covers every row once
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < rows; s += gridDim.x * blockDim.x) {
        const int g = tc ? tc_stage_point(s) : s;
        const int k = last_le(w.rowpre, n_frames, g);
        const FrameDesc* fr = w.frames + k;
        if (fold && g == fr->row0) fold_area_err(w, k);
        if (!fr->skip)
            sample_row(w, fr, g - fr->row0, g, w.cdf + fr->cdf0, tc != 0,
                       tc ? w.fbox[k] : make_float4(0.f, 0.f, 0.f, 1.f));
    }
}

__global__ void __launch_bounds__(256) k_targets(Ws w, int n_frames, int cols, int tc) {
    pdl_entry();
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < cols; s += gridDim.x * blockDim.x) {
        const int g = tc ? tc_stage_point(s) : s;
        const int k = last_le(w.colpre, n_frames, g);
        const FrameDesc* fr = w.frames + k;
        if (tc && g == fr->col0) {  // the frame's fallback lists start empty
            w.tcfn[2 * k] = 0;
            w.tcfn[2 * k + 1] = 0;
        }
        if (!fr->skip)
            stage_target(w, fr, g - fr->col0, g, tc != 0,
                         tc ? w.fbox[k] : make_float4(0.f, 0.f, 0.f, 1.f));
    }
}

// Sampling and target staging in one launch: one CTA per (frame, slice), the frame's CDF
// copied to shared memory so that the binary searches stay on chip.
constexpr int STAGE_THREADS = 512;

__global__ void __launch_bounds__(STAGE_THREADS) k_stage(Ws w, int slices, int rows, int cols,
                                                        int fold, int tc) {
    pdl_entry();
    extern __shared__ float s_cdf[];
    const int k = blockIdx.x / slices, sl = blockIdx.x - k * slices;
    const FrameDesc* fr = w.frames + k;
    if (fold && sl == 0 && threadIdx.x == 0) fold_area_err(w, k);
    if (tc && sl == 0 && threadIdx.x == 0) {  // the frame's fallback lists start empty
        w.tcfn[2 * k] = 0;
        w.tcfn[2 * k + 1] = 0;
    }
    if (fr->skip) return;
    const float4 box = tc ? w.fbox[k] : make_float4(0.f, 0.f, 0.f, 1.f);
    const bool sampled = fr->verts && !fr->pts;
    if (sampled)
        for (int f = threadIdx.x; f < fr->F; f += STAGE_THREADS) s_cdf[f] = w.cdf[fr->cdf0 + f];
    __syncthreads();
    // slices of whole blocks, so that the staging order stays inside each slice
    if (rows) {
        const int nb = fr->Npad / TC_BLOCK;
        const int a = (int)((long long)nb * sl / slices) * TC_BLOCK;
        const int b = (int)((long long)nb * (sl + 1) / slices) * TC_BLOCK;
        for (int s = a + threadIdx.x; s < b; s += STAGE_THREADS) {
            const int i = tc ? tc_stage_point(s) : s;
            sample_row(w, fr, i, fr->row0 + i, s_cdf, tc != 0, box);
        }
    }
    if (cols) {
        const int nb = fr->Mpad / TC_BLOCK;
        const int a = (int)((long long)nb * sl / slices) * TC_BLOCK;
        const int b = (int)((long long)nb * (sl + 1) / slices) * TC_BLOCK;
        for (int s = a + threadIdx.x; s < b; s += STAGE_THREADS) {
            const int j = tc ? tc_stage_point(s) : s;
            stage_target(w, fr, j, fr->col0 + j, tc != 0, box);
        }
    }
}

int g_stage_smem[64];

int grid_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    return (int)(b < 1 ? 1 : (b > 65535LL * 16 ? 65535LL * 16 : b));
}

}  // namespace

cudaError_t launch_build_uniform(const UniformArgs& a, const Ws& w, cudaStream_t s) {
    // as many threads as frames or units (whichever is more), in whole warps: a block of
    // 1024 threads costs several microseconds of barriers for a single frame
    const long long n_units = (long long)a.T * a.units_per_frame;
    long long nt = a.T > n_units + 1 ? a.T : n_units + 1;
    nt = (nt + 31) / 32 * 32;
    if (nt > BUILD_THREADS) nt = BUILD_THREADS;
    cudaError_t e = launch_pdl(k_build_uniform, 1, (int)nt, 0, s, a, w);
    count_launch();
    return e ? e : cudaGetLastError();
}

cudaError_t launch_reset(const Ws& w, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(&w.hdr->status, 0, sizeof(int), s);
    static_assert(offsetof(WsHeader, tc_next) == offsetof(WsHeader, tc_fallback) + sizeof(int),
                  "one memset clears both");
    return e ? e : cudaMemsetAsync(&w.hdr->tc_fallback, 0, 2 * sizeof(int), s);
}

cudaError_t launch_build_area(const UniformArgs& a, const Ws& w, cudaStream_t s) {
    cudaError_t e = launch_pdl(k_build_area, a.T + 1, CDF_THREADS, 0, s, a, w);
    count_launch();
    return e ? e : cudaGetLastError();
}

cudaError_t launch_bbox(const Ws& w, int n_frames, cudaStream_t s) {
    cudaError_t e = launch_pdl(k_bbox, n_frames, 512, 0, s, w);
    count_launch();
    return e ? e : cudaGetLastError();
}

cudaError_t launch_area_cdf(const Ws& w, int n_frames, cudaStream_t s) {
    cudaError_t e = launch_pdl(k_area_cdf, n_frames, CDF_THREADS, 0, s, w);
    count_launch();
    return e ? e : cudaGetLastError();
}

cudaError_t launch_sample(const Ws& w, int n_frames, int rows, int fold, int tc, cudaStream_t s) {
    cudaError_t e =
        launch_pdl(k_sample, grid_for(rows, 256), 256, 0, s, w, n_frames, rows, fold, tc);
    count_launch();
    return e ? e : cudaGetLastError();
}

cudaError_t launch_targets(const Ws& w, int n_frames, int cols, int tc, cudaStream_t s) {
    cudaError_t e = launch_pdl(k_targets, grid_for(cols, 256), 256, 0, s, w, n_frames, cols, tc);
    count_launch();
    return e ? e : cudaGetLastError();
}

cudaError_t launch_stage(const Ws& w, int n_frames, int slices, int max_f, int rows, int cols,
                         int fold, int tc, cudaStream_t s) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (g_stage_smem[dev] == 0) {
        int optin = 0;
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (optin <= 0) optin = 48 * 1024;
        cudaError_t e = cudaFuncSetAttribute(k_stage, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             optin);
        if (e != cudaSuccess) return e;
        g_stage_smem[dev] = optin;
    }
    const size_t need = (size_t)max_f * sizeof(float);
    if (need > (size_t)g_stage_smem[dev]) {
        // the CDF does not fit on chip: one kernel per step, searching the CDF in global memory
        cudaError_t e = cudaSuccess;
        if (rows) e = launch_sample(w, n_frames, rows, fold, tc, s);
        if (!e && cols) e = launch_targets(w, n_frames, cols, tc, s);
        return e;
    }
    cudaError_t e = launch_pdl(k_stage, n_frames * slices, STAGE_THREADS, need, s, w, slices,
                               (int)(rows > 0), (int)(cols > 0), fold, tc);
    count_launch();
    return e ? e : cudaGetLastError();
}

}  // namespace dc
