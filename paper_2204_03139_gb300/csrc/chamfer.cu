// Brute-force bidirectional nearest neighbours and the Chamfer loss (Eq. 1, Eq. 2).
//
// One pass over every (sim point, target point) pair of every frame computes both the
// row minima (sim -> target) and the column minima (target -> sim). The work is the set of
// "units" (ROWS_PER_UNIT sim points of one frame) times their sub-chunks of SUB targets,
// flattened and split evenly over a persistent grid, so that every CTA gets the same number
// of sub-chunks whatever the frame sizes. Partial minima of different CTAs merge through
// 64-bit atomicMin on (distance bits << 32 | position), which keeps the smallest distance
// and, among equal distances, the lowest position. The inner loop tracks minima only; the
// argmin is recovered afterwards by re-scanning the one sub-chunk (rows) or the one 8-row
// group (columns) that holds it, with bit-identical arithmetic.
#include <math.h>

#include "dc_internal.cuh"

namespace dc {

namespace {

typedef unsigned long long u64;

__device__ __forceinline__ void set_status(int* st, int code) { atomicCAS(st, DC_OK, code); }

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

// ---- packed float32 pairs (sm_100+ f32x2 arithmetic, each lane IEEE round-to-nearest) ----
__device__ __forceinline__ u64 pk(float lo, float hi) {
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk(u64 v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ u64 sub2(u64 a, u64 b) {
    u64 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ u64 mul2(u64 a, u64 b) {
    u64 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {
    u64 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ float min3(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// The scalar twin of the packed distance: dx = a - b, d = fma(dz, dz, fma(dy, dy, dx*dx)).
__device__ __forceinline__ float dist2(float ax, float ay, float az, float bx, float by,
                                       float bz) {
    const float dx = __fsub_rn(ax, bx), dy = __fsub_rn(ay, by), dz = __fsub_rn(az, bz);
    return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
}

// ---- mbarrier + bulk copy (global -> shared), all waits bounded ----
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(u64* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(u64* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, u64* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
        "[%3];" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try(u64* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; "
        "selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ u64 globaltimer() {
    u64 t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
constexpr u64 WAIT_LIMIT_NS = 2000000000ull;  // 2 s

// Wait for phase `parity` of `bar`; gives up after WAIT_LIMIT_NS and returns false.
__device__ __forceinline__ bool mbar_wait(u64* bar, uint32_t parity) {
    if (mbar_try(bar, parity)) return true;
    const u64 t0 = globaltimer();
    for (;;) {
        for (int i = 0; i < 64; ++i)
            if (mbar_try(bar, parity)) return true;
        if (globaltimer() - t0 > WAIT_LIMIT_NS) return false;
    }
}

// ---------------------------------------------------------------------------------------
// the fused bidirectional kernel
// ---------------------------------------------------------------------------------------
template <bool BIDIR>
__global__ void __launch_bounds__(THREADS, 4)
    k_chamfer(Ws w, int n_units, int total_sub) {
    __shared__ __align__(128) float s_t[2][3][CHUNK];
    __shared__ __align__(16) u64 s_col[BIDIR ? 2 : 1][BIDIR ? WARPS : 1][BIDIR ? CHUNK : 1];
    __shared__ __align__(8) u64 s_bar[2];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (total_sub + gridDim.x - 1) / gridDim.x;
    int s = blockIdx.x * per;
    const int s_end = min(total_sub, s + per);
    if (s >= s_end) return;
    int u = last_le(w.unit_pre, n_units, s);

    if (tid == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    uint32_t par = 0;     // bit b: the phase parity to wait for on buffer b
    uint32_t pending = 0; // bit b: a copy into buffer b is in flight
    int seq = 0;          // chunks consumed so far; buffer = seq & 1
    bool abort = false;

    while (s < s_end) {
        const int k = w.unit_frame[u], rb = w.unit_rb[u];
        const FrameDesc* fr = w.frames + k;
        const int N = fr->N, M = fr->M, Mpad = fr->Mpad, row0 = fr->row0, col0 = fr->col0;
        const int upre = w.unit_pre[u], unext = w.unit_pre[u + 1];
        const int sub_lo = s - upre, sub_hi = min(s_end, unext) - upre;
        const float* TX = w.tsoa + 3LL * col0;
        const int c_lo = sub_lo / SUBS_PER_CHUNK, c_hi = (sub_hi - 1) / SUBS_PER_CHUNK;

        // stage the first two chunks of this unit (both buffers are free here)
        if (tid == 0) {
            for (int c = c_lo; c <= min(c_hi, c_lo + 1); ++c) {
                const int b = (seq + c - c_lo) & 1;
                mbar_expect_tx(&s_bar[b], 3 * CHUNK * sizeof(float));
                for (int p = 0; p < 3; ++p)
                    bulk_g2s(&s_t[b][p][0], TX + (long long)p * Mpad + (long long)c * CHUNK,
                             CHUNK * sizeof(float), &s_bar[b]);
                pending |= 1u << b;
            }
        }

        // this thread's ROWS_PER_THREAD sim points, duplicated into both f32x2 lanes
        const int wrow0 = rb * ROWS_PER_UNIT + warp * ROWS_PER_WARP;
        const bool wactive = wrow0 < N;
        const int trow0 = wrow0 + lane * ROWS_PER_THREAD;
        const unsigned rg_base = (unsigned)(wrow0 / ROWS_PER_THREAD);
        const int n_active = min(WARPS, div_up(N - rb * ROWS_PER_UNIT, ROWS_PER_WARP));
        u64 rx[ROWS_PER_THREAD], ry[ROWS_PER_THREAD], rz[ROWS_PER_THREAD];
        float best[ROWS_PER_THREAD];
        unsigned bidx[ROWS_PER_THREAD];
#pragma unroll
        for (int r = 0; r < ROWS_PER_THREAD; ++r) {
            float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
            if (wactive) p = w.x[row0 + trow0 + r];
            rx[r] = pk(p.x, p.x);
            ry[r] = pk(p.y, p.y);
            rz[r] = pk(p.z, p.z);
            best[r] = INFINITY;
            bidx[r] = 0;
        }

        for (int c = c_lo; c <= c_hi; ++c, ++seq) {
            const int b = seq & 1;
            // every lane of a warp must agree before the warp-wide reductions below
            const bool ok = __all_sync(0xffffffffu, mbar_wait(&s_bar[b], (par >> b) & 1u));
            if (ok) par ^= 1u << b;
            const int sc0 = max(sub_lo, c * SUBS_PER_CHUNK);
            const int sc1 = min(sub_hi, (c + 1) * SUBS_PER_CHUNK);
            if (ok && wactive) {
                for (int sc = sc0; sc < sc1; ++sc) {
                    const int off = (sc - c * SUBS_PER_CHUNK) * SUB;
                    float cm[ROWS_PER_THREAD];
#pragma unroll
                    for (int r = 0; r < ROWS_PER_THREAD; ++r) cm[r] = INFINITY;
#pragma unroll 2
                    for (int jj = 0; jj < SUB; jj += 4) {
                        const float4 xq = *reinterpret_cast<const float4*>(&s_t[b][0][off + jj]);
                        const float4 yq = *reinterpret_cast<const float4*>(&s_t[b][1][off + jj]);
                        const float4 zq = *reinterpret_cast<const float4*>(&s_t[b][2][off + jj]);
                        const u64 X01 = pk(xq.x, xq.y), X23 = pk(xq.z, xq.w);
                        const u64 Y01 = pk(yq.x, yq.y), Y23 = pk(yq.z, yq.w);
                        const u64 Z01 = pk(zq.x, zq.y), Z23 = pk(zq.z, zq.w);
                        float c0 = INFINITY, c1 = INFINITY, c2 = INFINITY, c3 = INFINITY;
#pragma unroll
                        for (int r = 0; r < ROWS_PER_THREAD; r += 2) {
                            float a[2][4];
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                u64 dx = sub2(rx[r + h], X01), dy = sub2(ry[r + h], Y01),
                                    dz = sub2(rz[r + h], Z01);
                                const u64 d01 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
                                dx = sub2(rx[r + h], X23);
                                dy = sub2(ry[r + h], Y23);
                                dz = sub2(rz[r + h], Z23);
                                const u64 d23 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
                                upk(d01, a[h][0], a[h][1]);
                                upk(d23, a[h][2], a[h][3]);
                                cm[r + h] = min3(cm[r + h], a[h][0], a[h][1]);
                                cm[r + h] = min3(cm[r + h], a[h][2], a[h][3]);
                            }
                            if (BIDIR) {
                                c0 = min3(c0, a[0][0], a[1][0]);
                                c1 = min3(c1, a[0][1], a[1][1]);
                                c2 = min3(c2, a[0][2], a[1][2]);
                                c3 = min3(c3, a[0][3], a[1][3]);
                            }
                        }
                        if (BIDIR) {
                            const float cc[4] = {c0, c1, c2, c3};
#pragma unroll
                            for (int t = 0; t < 4; ++t) {
                                const unsigned v = __float_as_uint(cc[t]);
                                const unsigned m = __reduce_min_sync(0xffffffffu, v);
                                const unsigned bal = __ballot_sync(0xffffffffu, v == m);
                                if (lane == 0)
                                    s_col[b][warp][off + jj + t] =
                                        ((u64)m << 32) | (u64)(rg_base + (__ffs(bal) - 1));
                            }
                        }
                    }
#pragma unroll
                    for (int r = 0; r < ROWS_PER_THREAD; ++r)
                        if (cm[r] < best[r]) {
                            best[r] = cm[r];
                            bidx[r] = (unsigned)sc;
                        }
                }
            }
            abort = __syncthreads_or(!ok) != 0;
            if (abort) break;
            pending &= ~(1u << b);
            // buffer b is free again: stage chunk c + 2 into it
            if (tid == 0 && c + 2 <= c_hi) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_expect_tx(&s_bar[b], 3 * CHUNK * sizeof(float));
                for (int p = 0; p < 3; ++p)
                    bulk_g2s(&s_t[b][p][0],
                             TX + (long long)p * Mpad + (long long)(c + 2) * CHUNK,
                             CHUNK * sizeof(float), &s_bar[b]);
                pending |= 1u << b;
            }
            if (BIDIR) {
                const int j0 = sc0 * SUB - c * CHUNK;
                const int jend = min(sc1 * SUB, M) - c * CHUNK;
                for (int j = j0 + tid; j < jend; j += THREADS) {
                    u64 v = s_col[b][0][j];
                    for (int q = 1; q < n_active; ++q) v = min(v, s_col[b][q][j]);
                    atomicMin(&w.pba[col0 + c * CHUNK + j], v);
                }
            }
        }
        if (abort) break;
        if (wactive) {
#pragma unroll
            for (int r = 0; r < ROWS_PER_THREAD; ++r) {
                const int row = trow0 + r;
                if (row < N)
                    atomicMin(&w.pab[row0 + row],
                              ((u64)__float_as_uint(best[r]) << 32) | (u64)bidx[r]);
            }
        }
        s = unext;
        ++u;
    }

    if (abort) {
        if (tid == 0) {
            set_status(&w.hdr->status, DC_ETIMEOUT);
            // let copies still in flight land before the CTA's shared memory goes away
            for (int b = 0; b < 2; ++b)
                if (pending & (1u << b)) (void)mbar_wait(&s_bar[b], (par >> b) & 1u);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------------
// argmin recovery: rows re-scan their winning sub-chunk, columns their winning row group
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_finalize(Ws w, int n_frames, int rows, int cols,
                                                  int bidir) {
    const int total = rows + (bidir ? cols : 0);
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
        if (g < rows) {
            const int k = last_le(w.rowpre, n_frames, g);
            const FrameDesc* fr = w.frames + k;
            const int i = g - fr->row0;
            if (i >= fr->N) continue;
            const u64 p = w.pab[g];
            int found = -1;
            if (p != EMPTY) {
                const unsigned d = (unsigned)(p >> 32);
                const int j0 = (int)(p & 0xffffffffu) * SUB, j1 = min(j0 + SUB, fr->M);
                const float4 x = w.x[g];
                const float* X = w.tsoa + 3LL * fr->col0;
                const float* Y = X + fr->Mpad;
                const float* Z = Y + fr->Mpad;
                for (int j = j0; j < j1; ++j)
                    if (__float_as_uint(dist2(x.x, x.y, x.z, X[j], Y[j], Z[j])) == d) {
                        found = j;
                        break;
                    }
            }
            if (found < 0) set_status(&w.hdr->status, DC_EDEVICE);
            fr->nn_ab[i] = found;
        } else {
            const int gc = g - rows;
            const int k = last_le(w.colpre, n_frames, gc);
            const FrameDesc* fr = w.frames + k;
            const int j = gc - fr->col0;
            if (j >= fr->M) continue;
            const u64 p = w.pba[gc];
            int found = -1;
            if (p != EMPTY) {
                const unsigned d = (unsigned)(p >> 32);
                const int r0 = (int)(p & 0xffffffffu) * ROWS_PER_THREAD;
                const int r1 = min(r0 + ROWS_PER_THREAD, fr->N);
                const float* X = w.tsoa + 3LL * fr->col0;
                const float tx = X[j], ty = X[fr->Mpad + j], tz = X[2 * fr->Mpad + j];
                for (int r = r0; r < r1; ++r) {
                    const float4 x = w.x[fr->row0 + r];
                    if (__float_as_uint(dist2(x.x, x.y, x.z, tx, ty, tz)) == d) {
                        found = r;
                        break;
                    }
                }
            }
            if (found < 0) set_status(&w.hdr->status, DC_EDEVICE);
            fr->nn_ba[j] = found;
        }
    }
}

// ---------------------------------------------------------------------------------------
// per-frame loss (Eq. 1 / Eq. 2): fixed-order compensated sums of the minimum distances
// ---------------------------------------------------------------------------------------
constexpr int LOSS_THREADS = 256;

__device__ __forceinline__ float block_sum_fixed(float v, float* s_red) {
    const int tid = threadIdx.x;
    s_red[tid] = v;
    __syncthreads();
    for (int o = LOSS_THREADS / 2; o > 0; o >>= 1) {
        if (tid < o) s_red[tid] = __fadd_rn(s_red[tid], s_red[tid + o]);
        __syncthreads();
    }
    const float r = s_red[0];
    __syncthreads();
    return r;
}

__device__ __forceinline__ void kahan_add(float& s, float& c, float v) {
    const float y = __fsub_rn(v, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

__global__ void __launch_bounds__(LOSS_THREADS) k_loss(Ws w, int bidir) {
    __shared__ float s_red[LOSS_THREADS];
    const FrameDesc* fr = w.frames + blockIdx.x;
    const int N = fr->N, M = fr->M;
    float s = 0.f, c = 0.f;
    for (int i = threadIdx.x; i < N; i += LOSS_THREADS)
        kahan_add(s, c, __uint_as_float((unsigned)(w.pab[fr->row0 + i] >> 32)));
    const float sab = block_sum_fixed(s, s_red);
    float L = 0.f;
    if (bidir) {
        s = 0.f;
        c = 0.f;
        for (int j = threadIdx.x; j < M; j += LOSS_THREADS)
            kahan_add(s, c, __uint_as_float((unsigned)(w.pba[fr->col0 + j] >> 32)));
        const float sba = block_sum_fixed(s, s_red);
        L = __fadd_rn(__fdiv_rn(sab, (float)N), __fdiv_rn(sba, (float)M));
    } else {
        L = sab;
    }
    if (threadIdx.x == 0) fr->loss[0] = L;
}

// total = sum_k w_k L_k in a fixed order (lane-strided partial sums, then a fixed tree)
__global__ void k_total(Ws w, int n_frames, float* total) {
    const int lane = threadIdx.x;
    float s = 0.f, c = 0.f;
    for (int k = lane; k < n_frames; k += 32) {
        const FrameDesc* fr = w.frames + k;
        kahan_add(s, c, __fmul_rn(fr->weight, fr->loss[0]));
    }
    for (int o = 16; o > 0; o >>= 1) s = __fadd_rn(s, __shfl_down_sync(0xffffffffu, s, o));
    if (lane == 0) total[0] = s;
}

int grid_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    return (int)(b < 1 ? 1 : (b > 65535LL * 16 ? 65535LL * 16 : b));
}

int g_chamfer_ctas[64][2];  // per device, per mode: resident CTAs for the persistent grid

int chamfer_ctas(int mode) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    int& n = g_chamfer_ctas[dev][mode == DC_BIDIR_MEAN ? 0 : 1];
    if (n == 0) {
        int sms = 0, occ = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (mode == DC_BIDIR_MEAN)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_chamfer<true>, THREADS, 0);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_chamfer<false>, THREADS, 0);
        n = (sms > 0 ? sms : 1) * (occ > 0 ? occ : 1);
    }
    return n;
}

}  // namespace

cudaError_t launch_chamfer(const Ws& w, int n_units, int total_sub, int mode, cudaStream_t s) {
    if (total_sub <= 0) return cudaSuccess;
    int grid = chamfer_ctas(mode);
    if (grid > total_sub) grid = total_sub;
    prof_before(s);
    if (mode == DC_BIDIR_MEAN)
        k_chamfer<true><<<grid, THREADS, 0, s>>>(w, n_units, total_sub);
    else
        k_chamfer<false><<<grid, THREADS, 0, s>>>(w, n_units, total_sub);
    prof_after(s);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_finalize(const Ws& w, int n_frames, int rows, int cols, int mode,
                            cudaStream_t s) {
    const int bidir = mode == DC_BIDIR_MEAN;
    k_finalize<<<grid_for(rows + (bidir ? cols : 0), 256), 256, 0, s>>>(w, n_frames, rows, cols,
                                                                         bidir);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_loss(const Ws& w, int n_frames, int mode, float* total, cudaStream_t s) {
    k_loss<<<n_frames, LOSS_THREADS, 0, s>>>(w, mode == DC_BIDIR_MEAN);
    count_launch();
    if (total) {
        k_total<<<1, 32, 0, s>>>(w, n_frames, total);
        count_launch();
    }
    return cudaGetLastError();
}

}  // namespace dc
