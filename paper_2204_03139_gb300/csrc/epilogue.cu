// After the Chamfer pass: nearest-neighbour recovery, the loss (Eq. 1 / Eq. 2) and the
// adjoint -- dL/dx_i along the chosen neighbours scattered to the picked face's vertices with
// the barycentric weights (Eq. 4).
//
// One CTA per (frame, slice): the frame's sim points and target points are cut into
// `slices` equal ranges so that the whole GPU works even on few frames. Each CTA
//   - re-scans the sub-chunk (rows) or the thread's row group (targets) that the packed minimum
//     points at, with the same float32 operations as the Chamfer kernel, to find the first
//     index attaining it (ties go to the lowest index);
//   - sums its minimum distances (fixed order) into a per-slice partial;
//   - scatters the gradient: with one slice per frame into a shared-memory copy of the
//     frame's V x 3 gradient that it then writes out; with several slices straight into the
//     output with global float atomics (the area kernel zeroed it), which costs the big
//     frames nothing against per-slice copies and a reduction launch, and lets few frames
//     use more slices.
#include "dc_internal.cuh"

namespace dc {

namespace {

typedef unsigned long long u64;

__device__ __forceinline__ void set_status(int* st, int code) { atomicCAS(st, DC_OK, code); }

// dx = a - b, d = fma(dz, dz, fma(dy, dy, dx * dx)): the scalar twin of the packed distance
__device__ __forceinline__ float dist2(float ax, float ay, float az, float bx, float by,
                                       float bz) {
    const float dx = __fsub_rn(ax, bx), dy = __fsub_rn(ay, by), dz = __fsub_rn(az, bz);
    return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
}

__device__ __forceinline__ void kahan_add(float& s, float& c, float v) {
    const float y = __fsub_rn(v, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

struct EpiArgs {
    int slices;
    int flags;     // EPI_RESCAN | EPI_LOSS | EPI_GRAD
    int bidir;
    int use_smem;  // one slice per frame and the V x 3 accumulator fits in shared memory
    int exact;     // the packed minima hold the neighbour's index itself (tensor-core path)
};

__device__ __forceinline__ float block_sum_fixed(float v, float* s_red) {
    // fixed-order tree: warp shuffles, then warp 0 over the per-warp sums
    for (int o = 16; o > 0; o >>= 1) v = __fadd_rn(v, __shfl_down_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s_red[warp] = v;
    __syncthreads();
    float r = 0.f;
    if (warp == 0) {
        r = lane < (int)(blockDim.x >> 5) ? s_red[lane] : 0.f;
        for (int o = 16; o > 0; o >>= 1) r = __fadd_rn(r, __shfl_down_sync(0xffffffffu, r, o));
    }
    __syncthreads();
    return r;  // valid in thread 0
}

// THREADS = 256 when frames are cut into slices; 1024 when every frame is one CTA with a
// shared-memory gradient copy (large batches). The copy's size caps the CTAs per SM, and a
// launch with more frames than resident CTAs ends with its largest frames: more warps per
// CTA carry more independent load chains through each frame (on 64 uneven trajectories
// 292.5 -> 287.7 ms per batch with 512 threads, 286.4 ms with 1024; the 40-frame
// trajectory, cut into slices, was 0.7% slower with 512).
template <int THREADS>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS) k_epilogue(Ws w, EpiArgs e) {
    pdl_entry();
    extern __shared__ float s_acc[];
    __shared__ float s_red[THREADS / 32];
    const int k = blockIdx.x / e.slices, sl = blockIdx.x - k * e.slices;
    const int tid = threadIdx.x;
    const FrameDesc* fr = w.frames + k;
    if (fr->skip) {  // weight 0: nothing to recover, L reported as 0, gradient left at 0
        if (tid == 0 && (e.flags & EPI_LOSS)) {
            w.part[2 * (k * e.slices + sl)] = 0.0f;
            w.part[2 * (k * e.slices + sl) + 1] = 0.0f;
        }
        return;
    }
    const int N = fr->N, M = fr->M, V = fr->V, row0 = fr->row0, col0 = fr->col0;
    const bool grad = (e.flags & EPI_GRAD) && fr->grad && fr->verts;
    const bool rescan = (e.flags & EPI_RESCAN) != 0, want_loss = (e.flags & EPI_LOSS) != 0;
    const int* faces = fr->faces;
    
    float* G = nullptr;
    if (grad) {
        if (e.use_smem) {
            G = s_acc;
            for (int v = tid; v < 3 * V; v += THREADS) G[v] = 0.0f;
        } else {
            G = fr->grad;  // zeroed by the area kernel
        }
    }
    __syncthreads();

    const float gs = fr->gscale;
    const float cab = e.bidir ? __fdiv_rn(__fmul_rn(2.0f, gs), (float)N) : __fmul_rn(2.0f, gs);
    const float cba = __fdiv_rn(__fmul_rn(2.0f, gs), (float)M);

    // ---- sim points of this slice, 8 rows per warp step, 4 lanes per row ----
    // A row's minimum points at one sub-chunk of SUB targets; lane q of the row's group
    // checks candidates CPL q .. CPL q + CPL - 1 with contiguous loads, and two xor-shuffles
    // give the group the first candidate that matches. The three vertices of the gradient
    // scatter go to lanes 0..2 of the group.
    constexpr int CPL = SUB / 4;  // re-scan candidates per lane
    static_assert(SUB % 16 == 0, "four lanes of whole float4 groups per row");
    const int lane = tid & 31, warp = tid >> 5, grp = lane >> 2, q = lane & 3;
    constexpr int NW = THREADS / 32;
    const float* PX = w.tpl + 3LL * col0;  // compact target planes X[Mpad], Y, Z
    const float* PY = PX + fr->Mpad;
    const float* PZ = PY + fr->Mpad;
    const int i0 = (int)((long long)N * sl / e.slices);
    const int i1 = (int)((long long)N * (sl + 1) / e.slices);
    const bool exact = e.exact != 0 && rescan;
    constexpr int STEP = NW * 8;  // rows of one warp step of the CTA
    float sab = 0.f, cab_c = 0.f;
    if (exact) {
        // The recovery kernels left (distance bits << 32 | neighbour) for every row. Two warp
        // steps at a time, every load of both before any store: each lane keeps its rows and
        // their order (the loss partials are those of one step at a time), and both rows'
        // chains of dependent loads are in flight together.
        for (int base = i0 + warp * 8; base < i1; base += 2 * STEP) {
            int ir[2], nr[2];
            bool vr[2];
            u64 pr[2];
            float4 xr[2];
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                ir[r] = base + r * STEP + grp;
                vr[r] = ir[r] < i1;
                const int g = row0 + (vr[r] ? ir[r] : i0);
                pr[r] = vr[r] ? __ldg(&w.pab[g]) : EMPTY;
                xr[r] = __ldg(&w.x[g]);
            }
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                int nn = -1;
                if (vr[r] && pr[r] != EMPTY) nn = (int)(pr[r] & 0xffffffffu);
                if (vr[r] && q == 0) {
                    if (pr[r] != EMPTY && want_loss)
                        kahan_add(sab, cab_c, __uint_as_float((unsigned)(pr[r] >> 32)));
                    if (pr[r] == EMPTY || (unsigned)nn >= (unsigned)M)
                        set_status(&w.hdr->status, DC_EDEVICE);
                    fr->nn_ab[ir[r]] = nn;
                }
                nr[r] = vr[r] && (unsigned)nn < (unsigned)M && q < 3 ? nn : -1;
            }
            if (grad) {
                float yr[2][3] = {};
                int4 fr4[2];
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    fr4[r] = make_int4(-1, 0, 0, 0);
                    if (nr[r] >= 0) {
                        yr[r][0] = __ldg(&PX[nr[r]]);
                        yr[r][1] = __ldg(&PY[nr[r]]);
                        yr[r][2] = __ldg(&PZ[nr[r]]);
                        fr4[r] = __ldg(&w.fw[row0 + ir[r]]);
                    }
                }
                int vv[2];
#pragma unroll
                for (int r = 0; r < 2; ++r)
                    vv[r] = fr4[r].x >= 0 ? __ldg(&faces[3 * fr4[r].x + q]) : -1;
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const int v = vv[r];
                    if ((unsigned)v < (unsigned)V) {
                        const int4 fq = fr4[r];
                        const float wq = __int_as_float(q == 0 ? fq.y : (q == 1 ? fq.z : fq.w));
                        const float4 x = xr[r];
                        atomicAdd(&G[3 * v + 0],
                                  __fmul_rn(wq, __fmul_rn(cab, __fsub_rn(x.x, yr[r][0]))));
                        atomicAdd(&G[3 * v + 1],
                                  __fmul_rn(wq, __fmul_rn(cab, __fsub_rn(x.y, yr[r][1]))));
                        atomicAdd(&G[3 * v + 2],
                                  __fmul_rn(wq, __fmul_rn(cab, __fsub_rn(x.z, yr[r][2]))));
                    }
                }
            }
        }
    }
    for (int base = i0 + warp * 8; !exact && base < i1; base += STEP) {
        const int i = base + grp;
        const bool valid = i < i1;
        const int g = row0 + (valid ? i : i0);
        const float4 x = w.x[g];
        int nn = -1;
        float dmin = 0.f;
        if (rescan) {
            const u64 p = valid ? w.pab[g] : EMPTY;
            int first = 0x7fffffff;
            if (p != EMPTY) {
                const unsigned dq = (unsigned)(p >> 32);
                dmin = __uint_as_float(dq);
                const int jb = (int)(p & 0xffffffffu) * SUB + CPL * q;
                float cx[CPL], cy[CPL], cz[CPL];
#pragma unroll
                for (int k = 0; k < CPL; k += 4) {
                    const float4 a = *reinterpret_cast<const float4*>(PX + jb + k);
                    const float4 b = *reinterpret_cast<const float4*>(PY + jb + k);
                    const float4 c = *reinterpret_cast<const float4*>(PZ + jb + k);
                    cx[k] = a.x, cx[k + 1] = a.y, cx[k + 2] = a.z, cx[k + 3] = a.w;
                    cy[k] = b.x, cy[k + 1] = b.y, cy[k + 2] = b.z, cy[k + 3] = b.w;
                    cz[k] = c.x, cz[k + 1] = c.y, cz[k + 2] = c.z, cz[k + 3] = c.w;
                }
#pragma unroll
                for (int t = CPL - 1; t >= 0; --t)
                    if (jb + t < M &&
                        __float_as_uint(dist2(x.x, x.y, x.z, cx[t], cy[t], cz[t])) == dq)
                        first = jb + t;
            }
            first = min(first, __shfl_xor_sync(0xffffffffu, first, 1));
            first = min(first, __shfl_xor_sync(0xffffffffu, first, 2));
            if (valid && p != EMPTY) nn = first == 0x7fffffff ? -1 : first;
            if (valid && q == 0) {
                if (p != EMPTY && want_loss) kahan_add(sab, cab_c, dmin);
                if (nn < 0) set_status(&w.hdr->status, DC_EDEVICE);
                fr->nn_ab[i] = nn;
            }
        } else if (valid) {
            nn = fr->nn_ab[i];
            if ((unsigned)nn >= (unsigned)M) {
                if (q == 0) set_status(&w.hdr->status, DC_EINVAL);
                nn = -1;
            }
        }
        if (grad && valid && nn >= 0 && q < 3) {
            const float y0 = PX[nn], y1 = PY[nn], y2 = PZ[nn];
            const int4 fq = w.fw[g];
            if (fq.x >= 0) {
                const int v = faces[3 * fq.x + q];
                const float wq = __int_as_float(q == 0 ? fq.y : (q == 1 ? fq.z : fq.w));
                if ((unsigned)v < (unsigned)V) {
                    atomicAdd(&G[3 * v + 0], __fmul_rn(wq, __fmul_rn(cab, __fsub_rn(x.x, y0))));
                    atomicAdd(&G[3 * v + 1], __fmul_rn(wq, __fmul_rn(cab, __fsub_rn(x.y, y1))));
                    atomicAdd(&G[3 * v + 2], __fmul_rn(wq, __fmul_rn(cab, __fsub_rn(x.z, y2))));
                }
            }
        }
    }

    // ---- target points of this slice (Eq. 1 only), 8 per warp step, 4 lanes per target ----
    // A target's minimum points at the first row of one lane's group of sim points (16 rows,
    // or 12 or 8 in a frame's last warp): lane q of the target's group checks rows
    // RPL q .. RPL q + RPL - 1 from there. A shorter group is followed by rows of the next
    // group or padding, whose indices are higher, so the first match is still the lowest
    // index attaining the minimum.
    static_assert(ROWS_PER_THREAD % 4 == 0, "four lanes share a row group");
    constexpr int RPL = ROWS_PER_THREAD / 4;
    float sba = 0.f, cba_c = 0.f;
    if (e.bidir) {
        const int j0 = (int)((long long)M * sl / e.slices);
        const int j1 = (int)((long long)M * (sl + 1) / e.slices);
        if (exact) {
            // as for the rows: two warp steps at a time, every load of both before any store
            for (int base = j0 + warp * 8; base < j1; base += 2 * STEP) {
                int jr[2], nr[2];
                bool vr[2];
                u64 pr[2];
                float tr[2][3];
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    jr[r] = base + r * STEP + grp;
                    vr[r] = jr[r] < j1;
                    const int jj = vr[r] ? jr[r] : j0;
                    pr[r] = vr[r] ? __ldg(&w.pba[col0 + jj]) : EMPTY;
                    tr[r][0] = __ldg(&PX[jj]);
                    tr[r][1] = __ldg(&PY[jj]);
                    tr[r][2] = __ldg(&PZ[jj]);
                }
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    int nn = -1;
                    if (vr[r] && pr[r] != EMPTY) nn = (int)(pr[r] & 0xffffffffu);
                    if (vr[r] && q == 0) {
                        if (pr[r] != EMPTY && want_loss)
                            kahan_add(sba, cba_c, __uint_as_float((unsigned)(pr[r] >> 32)));
                        if (pr[r] == EMPTY || (unsigned)nn >= (unsigned)N)
                            set_status(&w.hdr->status, DC_EDEVICE);
                        fr->nn_ba[jr[r]] = nn;
                    }
                    nr[r] = vr[r] && (unsigned)nn < (unsigned)N && q < 3 ? nn : -1;
                }
                if (grad) {
                    float4 xm[2];
                    int4 fr4[2];
#pragma unroll
                    for (int r = 0; r < 2; ++r) {
                        xm[r] = make_float4(0.f, 0.f, 0.f, 0.f);
                        fr4[r] = make_int4(-1, 0, 0, 0);
                        if (nr[r] >= 0) {
                            xm[r] = __ldg(&w.x[row0 + nr[r]]);
                            fr4[r] = __ldg(&w.fw[row0 + nr[r]]);
                        }
                    }
                    int vv[2];
#pragma unroll
                    for (int r = 0; r < 2; ++r)
                        vv[r] = fr4[r].x >= 0 ? __ldg(&faces[3 * fr4[r].x + q]) : -1;
#pragma unroll
                    for (int r = 0; r < 2; ++r) {
                        const int v = vv[r];
                        if ((unsigned)v < (unsigned)V) {
                            const int4 fq = fr4[r];
                            const float wq =
                                __int_as_float(q == 0 ? fq.y : (q == 1 ? fq.z : fq.w));
                            atomicAdd(&G[3 * v + 0],
                                      __fmul_rn(wq, __fmul_rn(cba, __fsub_rn(xm[r].x, tr[r][0]))));
                            atomicAdd(&G[3 * v + 1],
                                      __fmul_rn(wq, __fmul_rn(cba, __fsub_rn(xm[r].y, tr[r][1]))));
                            atomicAdd(&G[3 * v + 2],
                                      __fmul_rn(wq, __fmul_rn(cba, __fsub_rn(xm[r].z, tr[r][2]))));
                        }
                    }
                }
            }
        }
        for (int base = j0 + warp * 8; !exact && base < j1; base += STEP) {
            const int j = base + grp;
            const bool valid = j < j1;
            const int jj = valid ? j : j0;
            const float tx = PX[jj], ty = PY[jj], tz = PZ[jj];
            int nn = -1;
            float dmin = 0.f;
            if (rescan) {
                const u64 p = valid ? w.pba[col0 + jj] : EMPTY;
                int first = 0x7fffffff;
                if (p != EMPTY) {
                    const unsigned dq = (unsigned)(p >> 32);
                    dmin = __uint_as_float(dq);
                    const int rb = (int)(p & 0xffffffffu) + RPL * q;
                    float4 xr[RPL];
#pragma unroll
                    for (int t = 0; t < RPL; ++t)
                        xr[t] = w.x[row0 + min(rb + t, N - 1)];
#pragma unroll
                    for (int t = RPL - 1; t >= 0; --t)
                        if (rb + t < N &&
                            __float_as_uint(dist2(xr[t].x, xr[t].y, xr[t].z, tx, ty, tz)) == dq)
                            first = rb + t;
                }
                first = min(first, __shfl_xor_sync(0xffffffffu, first, 1));
                first = min(first, __shfl_xor_sync(0xffffffffu, first, 2));
                if (valid && p != EMPTY) nn = first == 0x7fffffff ? -1 : first;
                if (valid && q == 0) {
                    if (p != EMPTY && want_loss) kahan_add(sba, cba_c, dmin);
                    if (nn < 0) set_status(&w.hdr->status, DC_EDEVICE);
                    fr->nn_ba[j] = nn;
                }
            } else if (valid) {
                nn = fr->nn_ba[j];
                if ((unsigned)nn >= (unsigned)N) {
                    if (q == 0) set_status(&w.hdr->status, DC_EINVAL);
                    nn = -1;
                }
            }
            if (grad && valid && nn >= 0 && q < 3) {
                const float4 xm = w.x[row0 + nn];
                const int4 fq = w.fw[row0 + nn];
                if (fq.x >= 0) {
                    const int v = faces[3 * fq.x + q];
                    const float wq = __int_as_float(q == 0 ? fq.y : (q == 1 ? fq.z : fq.w));
                    if ((unsigned)v < (unsigned)V) {
                        atomicAdd(&G[3 * v + 0], __fmul_rn(wq, __fmul_rn(cba, __fsub_rn(xm.x, tx))));
                        atomicAdd(&G[3 * v + 1], __fmul_rn(wq, __fmul_rn(cba, __fsub_rn(xm.y, ty))));
                        atomicAdd(&G[3 * v + 2], __fmul_rn(wq, __fmul_rn(cba, __fsub_rn(xm.z, tz))));
                    }
                }
            }
        }
    }

    if (want_loss) {
        const float a = block_sum_fixed(sab, s_red);
        const float b = block_sum_fixed(sba, s_red);
        if (tid == 0) {
            w.part[2 * (k * e.slices + sl)] = a;
            w.part[2 * (k * e.slices + sl) + 1] = b;
        }
    }
    if (grad && e.use_smem) {
        __syncthreads();
        for (int v = tid; v < 3 * V; v += THREADS) fr->grad[v] = s_acc[v];
    }
}

// L_k from its slice partials (Eq. 1: means, Eq. 2: sum) and the weighted total, all in a
// fixed order
constexpr int LOSS_THREADS = 1024;

__global__ void __launch_bounds__(LOSS_THREADS) k_frame_loss(Ws w, int n_frames, int slices,
                                                             int bidir, float* total) {
    pdl_entry();
    __shared__ float s_red[LOSS_THREADS / 32];
    float t = 0.f, tc = 0.f;
    for (int k = threadIdx.x; k < n_frames; k += LOSS_THREADS) {
        const FrameDesc* fr = w.frames + k;
        float sab = 0.f, sba = 0.f;
        for (int q = 0; q < slices; ++q) {
            sab = __fadd_rn(sab, w.part[2 * (k * slices + q)]);
            sba = __fadd_rn(sba, w.part[2 * (k * slices + q) + 1]);
        }
        const float L = bidir ? __fadd_rn(__fdiv_rn(sab, (float)fr->N), __fdiv_rn(sba, (float)fr->M))
                              : sab;
        fr->loss[0] = L;
        kahan_add(t, tc, __fmul_rn(fr->weight, L));
    }
    const float s = block_sum_fixed(t, s_red);
    if (threadIdx.x == 0 && total) total[0] = s;
}

// sum_t w_t L_t of given per-frame losses in the same fixed order as k_frame_loss
__global__ void __launch_bounds__(LOSS_THREADS) k_loss_total(const float* lf, const float* w,
                                                             int T, float* total) {
    pdl_entry();
    __shared__ float s_red[LOSS_THREADS / 32];
    float t = 0.f, tc = 0.f;
    for (int k = threadIdx.x; k < T; k += LOSS_THREADS)
        kahan_add(t, tc, __fmul_rn(w ? w[k] : 1.0f, lf[k]));
    const float s = block_sum_fixed(t, s_red);
    if (threadIdx.x == 0) total[0] = s;
}

// ---- gradient with respect to given sim points (dc_chamfer_bwd) ----
__global__ void __launch_bounds__(256) k_cbwd_rows(const float* a, const float* b,
                                                   const int* nn_ab, int T, int N, int M,
                                                   int bidir, const float* g, float* grad) {
    pdl_entry();
    const long long n = (long long)T * N;
    for (long long e = blockIdx.x * 256LL + threadIdx.x; e < n; e += (long long)gridDim.x * 256) {
        const int t = (int)(e / N);
        const int j = nn_ab[e];
        float gx = 0.f, gy = 0.f, gz = 0.f;
        if ((unsigned)j < (unsigned)M) {
            const float c = bidir ? __fdiv_rn(__fmul_rn(2.0f, g[t]), (float)N)
                                  : __fmul_rn(2.0f, g[t]);
            const float* y = b + 3LL * ((long long)t * M + j);
            gx = __fmul_rn(c, __fsub_rn(a[3 * e], y[0]));
            gy = __fmul_rn(c, __fsub_rn(a[3 * e + 1], y[1]));
            gz = __fmul_rn(c, __fsub_rn(a[3 * e + 2], y[2]));
        }
        grad[3 * e] = gx;
        grad[3 * e + 1] = gy;
        grad[3 * e + 2] = gz;
    }
}

__global__ void __launch_bounds__(256) k_cbwd_cols(const float* a, const float* b,
                                                   const int* nn_ba, int T, int N, int M,
                                                   const float* g, float* grad) {
    pdl_entry();
    const long long n = (long long)T * M;
    for (long long e = blockIdx.x * 256LL + threadIdx.x; e < n; e += (long long)gridDim.x * 256) {
        const int t = (int)(e / M);
        const int i = nn_ba[e];
        if ((unsigned)i >= (unsigned)N) continue;
        const float c = __fdiv_rn(__fmul_rn(2.0f, g[t]), (float)M);
        const long long ia = (long long)t * N + i;
        const float* x = a + 3 * ia;
        atomicAdd(&grad[3 * ia], __fmul_rn(c, __fsub_rn(x[0], b[3 * e])));
        atomicAdd(&grad[3 * ia + 1], __fmul_rn(c, __fsub_rn(x[1], b[3 * e + 1])));
        atomicAdd(&grad[3 * ia + 2], __fmul_rn(c, __fsub_rn(x[2], b[3 * e + 2])));
    }
}

int grid_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    return (int)(b < 1 ? 1 : (b > 65535LL * 16 ? 65535LL * 16 : b));
}

int g_smem_limit[64];

}  // namespace

// CTA size of the one-CTA-per-frame form (see k_epilogue)
constexpr int EPI_THREADS_ONE_SLICE = 4 * EPI_THREADS;

cudaError_t launch_epilogue(const Ws& w, int n_frames, int slices, int max_v, int mode,
                            int flags, float* total, int tc_grid, cudaStream_t s) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (g_smem_limit[dev] == 0) {
        int optin = 0;
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (optin <= 0) optin = 48 * 1024;
        optin -= 1024;  // room for the static reduction buffer
        cudaError_t e = cudaFuncSetAttribute(k_epilogue<EPI_THREADS_ONE_SLICE>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
        if (e != cudaSuccess) return e;
        g_smem_limit[dev] = optin;
    }
    EpiArgs a;
    a.slices = slices;
    a.flags = flags;
    a.bidir = mode == DC_BIDIR_MEAN;
    a.exact = tc_grid > 0;
    const bool grad = (flags & EPI_GRAD) && max_v > 0;
    const size_t need = (size_t)max_v * 3 * sizeof(float);
    a.use_smem = grad && slices == 1 && need <= (size_t)g_smem_limit[dev];
    cudaError_t e = a.use_smem ? launch_pdl(k_epilogue<EPI_THREADS_ONE_SLICE>, n_frames * slices,
                                            EPI_THREADS_ONE_SLICE, need, s, w, a)
                               : launch_pdl(k_epilogue<EPI_THREADS>, n_frames * slices,
                                            EPI_THREADS, 0, s, w, a);
    count_launch();
    if (!e && (flags & EPI_LOSS)) {
        e = launch_pdl(k_frame_loss, 1, LOSS_THREADS, 0, s, w, n_frames, slices, (int)a.bidir,
                       total);
        count_launch();
    }
    return e ? e : cudaGetLastError();
}

cudaError_t launch_loss_total(const float* lf, const float* w, int T, float* total,
                              cudaStream_t s) {
    cudaError_t e = launch_pdl(k_loss_total, 1, LOSS_THREADS, 0, s, lf, w, T, total);
    count_launch();
    return e ? e : cudaGetLastError();
}

cudaError_t launch_chamfer_bwd_points(const float* a, const float* b, const int* nn_ab,
                                      const int* nn_ba, int T, int N, int M, int mode,
                                      const float* g, float* grad_a, cudaStream_t s) {
    const int bidir = mode == DC_BIDIR_MEAN;
    cudaError_t e = launch_pdl(k_cbwd_rows, grid_for((long long)T * N, 256), 256, 0, s, a, b,
                               nn_ab, T, N, M, bidir, g, grad_a);
    count_launch();
    if (!e && bidir) {
        e = launch_pdl(k_cbwd_cols, grid_for((long long)T * M, 256), 256, 0, s, a, b, nn_ba, T,
                       N, M, g, grad_a);
        count_launch();
    }
    if (e) return e;
    return cudaGetLastError();
}

}  // namespace dc
