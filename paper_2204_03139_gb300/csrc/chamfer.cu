// Brute-force bidirectional nearest neighbours and the Chamfer loss (Eq. 1, Eq. 2).
//
// One pass over every (sim point, target point) pair of every frame computes both the
// row minima (sim -> target) and the column minima (target -> sim). The work is the set of
// "units" (ROWS_PER_UNIT sim points of one frame) times their sub-chunks of SUB targets,
// flattened and split evenly over a persistent grid, so that every CTA gets the same number
// of sub-chunks whatever the frame sizes. Partial minima of different CTAs merge through
// 64-bit atomicMin on (distance bits << 32 | position), which keeps the smallest distance
// and, among equal distances, the lowest position. The inner loop tracks minima only; the
// argmin is recovered afterwards (epilogue.cu) by re-scanning the one sub-chunk (rows) or
// the one thread's group of rows (columns) that holds it, with bit-identical arithmetic.
#include <math.h>

#include <atomic>
#include <type_traits>

#include "dc_internal.cuh"
#include "dc_async.cuh"

namespace dc {

namespace {

// ---------------------------------------------------------------------------------------
// the fused bidirectional kernel
// ---------------------------------------------------------------------------------------
constexpr int PAIRS = ROWS_PER_THREAD / 2;  // packed row pairs per thread

// Rows per lane of a warp whose frame has `left` rows from the warp's first row on: the full
// 16, or 12 or 8 for a frame's last warp when 32 lanes of that many rows cover what is left
// (the warp then computes 3/4 or 1/2 of a full tile instead of a tile of mostly padding).
__device__ __forceinline__ int lane_rows(int left) {
    static_assert(ROWS_PER_THREAD == 16, "the short tiles assume 16 rows per lane");
    return left > 12 * 32 ? 16 : (left > 8 * 32 ? 12 : 8);
}

// What the CTA knows about the unit segment it is working on (kept in shared memory so that
// the inner loop's registers go to the rows and the running minima).
struct UnitState {
    const float* tx;  // the frame's negated, duplicated target planes (-X2, -Y2, -Z2)
    int N, M, Mpad, row0, col0, rb, sub_lo, sub_hi;
};

#ifndef DC_TARGETS_PER_STEP
#define DC_TARGETS_PER_STEP 2
#endif
constexpr int TPS = DC_TARGETS_PER_STEP;  // targets per inner step (2 or 4)
// unroll of the step loop after a sub-chunk's first step: 3 divides its 15 remaining steps
// (measured 0.6% faster than 2 bidirectional, 1.3% rows only; 5 and 15 were slower)
#ifndef DC_STEP_UNROLL
#define DC_STEP_UNROLL 3
#endif
constexpr int STEP_UNROLL = DC_STEP_UNROLL;

// warp minimum of each of TPS targets and the lanes holding it; every lane stores the same
// value (no divergent branch); the first lane is taken later
__device__ __forceinline__ void column_merge(const unsigned (&v)[TPS], const unsigned (&m)[TPS],
                                             unsigned* __restrict__ smv,
                                             unsigned* __restrict__ smb) {
#pragma unroll
    for (int t = 0; t < TPS; t += 2) {
        const unsigned q0 = __ballot_sync(0xffffffffu, v[t] == m[t]);
        const unsigned q1 = __ballot_sync(0xffffffffu, v[t + 1] == m[t + 1]);
        *reinterpret_cast<uint2*>(smv + t) = make_uint2(m[t], m[t + 1]);
        *reinterpret_cast<uint2*>(smb + t) = make_uint2(q0, q1);
    }
}

// TPS targets jj..jj+TPS-1 against this thread's rows: row minima into cm (started from
// this step's distances when FIRST, so that no sub-chunk has to fill cm with INFINITY
// first: padded rows and targets carry finite sentinels, so no distance is NaN), per-target
// warp minima and the ballot of the lanes holding them into smv / smb
template <bool BIDIR, bool FIRST, int NP>
__device__ __forceinline__ void step(const float* __restrict__ tx, const float* __restrict__ ty,
                                     const float* __restrict__ tz, int jj,
                                     const float2 (&rx)[PAIRS], const float2 (&ry)[PAIRS],
                                     const float2 (&rz)[PAIRS], float (&cm)[ROWS_PER_THREAD],
                                     unsigned* __restrict__ smv, unsigned* __restrict__ smb) {
    // targets jj..jj+TPS-1 as {-X_j, -X_j} pairs
    float2 X[TPS], Y[TPS], Z[TPS];
#pragma unroll
    for (int t = 0; t < TPS; t += 2) {
        const float4 xq = *reinterpret_cast<const float4*>(tx + 2 * (jj + t));
        const float4 yq = *reinterpret_cast<const float4*>(ty + 2 * (jj + t));
        const float4 zq = *reinterpret_cast<const float4*>(tz + 2 * (jj + t));
        X[t] = make_float2(xq.x, xq.y);
        X[t + 1] = make_float2(xq.z, xq.w);
        Y[t] = make_float2(yq.x, yq.y);
        Y[t + 1] = make_float2(yq.z, yq.w);
        Z[t] = make_float2(zq.x, zq.y);
        Z[t + 1] = make_float2(zq.z, zq.w);
    }
    float c[TPS];
#pragma unroll
    for (int t = 0; t < TPS; ++t) c[t] = INFINITY;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        float2 d[TPS];
#pragma unroll
        for (int t = 0; t < TPS; ++t) {
            // x + (-X) rounds exactly like x - X
            const float2 dx = __fadd2_rn(rx[p], X[t]), dy = __fadd2_rn(ry[p], Y[t]),
                         dz = __fadd2_rn(rz[p], Z[t]);
            d[t] = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
        }
#pragma unroll
        for (int t = 0; t < TPS; t += 2) {
            if (FIRST && t == 0) {
                cm[2 * p] = fminf(d[t].x, d[t + 1].x);
                cm[2 * p + 1] = fminf(d[t].y, d[t + 1].y);
            } else {
                cm[2 * p] = min3(cm[2 * p], d[t].x, d[t + 1].x);
                cm[2 * p + 1] = min3(cm[2 * p + 1], d[t].y, d[t + 1].y);
            }
        }
        if (BIDIR) {
#pragma unroll
            for (int t = 0; t < TPS; ++t) c[t] = min3(c[t], d[t].x, d[t].y);
        }
    }
    if (BIDIR) {
        unsigned v[TPS], m[TPS];
#pragma unroll
        for (int t = 0; t < TPS; ++t) {
            v[t] = __float_as_uint(c[t]);
            m[t] = __reduce_min_sync(0xffffffffu, v[t]);
        }
        column_merge(v, m, smv + jj, smb + jj);
    }
}

// one sub-chunk: SUB targets against this thread's first 2 NP rows; cm[0 .. 2 NP) receives
// the rows' minima over it
template <bool BIDIR, int NP>
__device__ __forceinline__ void sub_chunk(const float* __restrict__ tx, const float* __restrict__ ty,
                                          const float* __restrict__ tz, const float2 (&rx)[PAIRS],
                                          const float2 (&ry)[PAIRS], const float2 (&rz)[PAIRS],
                                          float (&cm)[ROWS_PER_THREAD], unsigned* __restrict__ smv,
                                          unsigned* __restrict__ smb) {
    step<BIDIR, true, NP>(tx, ty, tz, 0, rx, ry, rz, cm, smv, smb);
#pragma unroll(TPS == 2 ? STEP_UNROLL : 1)
    for (int jj = TPS; jj < SUB; jj += TPS)
        step<BIDIR, false, NP>(tx, ty, tz, jj, rx, ry, rz, cm, smv, smb);
}

// Where a row's running minimum over the unit segment (and the sub-chunk holding it) lives:
// in registers for the rows-only pass, which has the registers to spare at 8 warps per SM
// (measured 1.7% faster than shared memory there); in shared memory for the bidirectional
// pass, whose column minima take those registers (registers were 0.6% slower there).
template <bool BIDIR>
struct BestInRegs {
    static constexpr bool value = !BIDIR;
};

// resident CTAs per SM the register budget is sized for, per CTA width: 12 warps per SM with
// 16 rows per thread (8 when the running minima are kept in registers), 16 warps with fewer
// rows (fewer row registers)
template <bool BIDIR, int W>
struct MinBlocks {
#ifdef DC_WARPS_PER_SM
    static constexpr int warps_per_sm = DC_WARPS_PER_SM;
#else
    static constexpr int warps_per_sm =
        ROWS_PER_THREAD >= 16 ? (BestInRegs<BIDIR>::value ? 8 : 12) : 16;
#endif
    static constexpr int value = warps_per_sm / W;
};

template <bool BIDIR, int W>
__global__ void __launch_bounds__(32 * W, (MinBlocks<BIDIR, W>::value))
    k_chamfer(Ws w, int stall) {
    pdl_wait();
    constexpr int THREADS = 32 * W;
    constexpr int WARPS = W;
    constexpr int ROWS_PER_UNIT = ROWS_PER_WARP * W;
    // targets of two chunks, each coordinate negated and twice: [buffer][plane][2 * CHUNK]
    __shared__ __align__(128) float s_t[2][3][2 * CHUNK];
    // per-warp column minima of the chunk and the ballot of the lanes that hold them
    __shared__ __align__(16) unsigned s_cv[BIDIR ? 2 : 1][BIDIR ? WARPS : 1][BIDIR ? CHUNK : 1];
    __shared__ __align__(16) unsigned s_cb[BIDIR ? 2 : 1][BIDIR ? WARPS : 1][BIDIR ? CHUNK : 1];
    // per-row running minimum over the unit and the sub-chunk that holds it, as the key the
    // rows merge with, (distance bits << 32) | sub-chunk (shared-memory copy; one element,
    // unused, when it lives in registers)
    constexpr bool REG_BEST = BestInRegs<BIDIR>::value;
    __shared__ u64 s_key[REG_BEST ? 1 : ROWS_PER_THREAD][REG_BEST ? 1 : THREADS];
    __shared__ UnitState s_u;
    __shared__ __align__(8) u64 s_bar[2];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // the work (units, and their sub-chunks without those of skipped frames) was laid out on
    // the device or by the plan
    const int n_units = w.hdr->n_units, total_sub = w.hdr->total_sub;
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

    uint32_t par = 0;     // bit b: the phase parity to wait for on buffer b
    uint32_t pending = 0; // bit b: a copy into buffer b is in flight (thread 0)
    int seq = 0;          // chunks consumed so far; buffer = seq & 1
    bool abort = false;
    constexpr uint32_t PLANE_BYTES = 2 * CHUNK * sizeof(float);

    while (s < s_end) {
        __syncthreads();  // the previous segment is done with s_u
        if (tid == 0) {
            const FrameDesc* fr = w.frames + w.unit_frame[u];
            const int upre = w.unit_pre[u];
            s_u.N = fr->N;
            s_u.M = fr->M;
            s_u.Mpad = fr->Mpad;
            s_u.row0 = fr->row0;
            s_u.col0 = fr->col0;
            s_u.rb = w.unit_rb[u];
            s_u.sub_lo = s - upre;
            s_u.sub_hi = min(s_end, w.unit_pre[u + 1]) - upre;
            s_u.tx = w.tsoa + 6LL * fr->col0;
            // stage the first two chunks of this segment (both buffers are free here)
            const int c_lo = s_u.sub_lo / SUBS_PER_CHUNK;
            const int c_hi = (s_u.sub_hi - 1) / SUBS_PER_CHUNK;
            for (int c = c_lo; c <= min(c_hi, c_lo + 1); ++c) {
                const int b = (seq + c - c_lo) & 1;
                // test of the bounded waits: the first chunk is never requested, so its
                // barrier never completes and every wait on it gives up (DC_ETIMEOUT)
                if (stall && seq == 0 && c == c_lo) continue;
                mbar_expect_tx(&s_bar[b], 3 * PLANE_BYTES);
                for (int p = 0; p < 3; ++p)
                    bulk_g2s(&s_t[b][p][0], s_u.tx + 2LL * p * s_u.Mpad + 2LL * c * CHUNK,
                             PLANE_BYTES, &s_bar[b]);
                pending |= 1u << b;
            }
        }
        __syncthreads();
        const int N = s_u.N;
        const int wrow0 = s_u.rb * ROWS_PER_UNIT + warp * ROWS_PER_WARP;
        const bool wactive = wrow0 < N;
        // rows per lane: 16, or 12 or 8 for a frame's last warp when that covers its rows, so
        // that the warp does not compute a full tile of padding
        const int rpl = lane_rows(N - wrow0);
        const int trow0 = wrow0 + lane * rpl;

        // this thread's rows as packed pairs {x_2p, x_2p+1}, loaded straight into the pair
        // halves (inactive warps read valid rows of the frame and never use them); building
        // the pairs from whole float4 loads instead costs register moves in the inner loop
        float2 rx[PAIRS], ry[PAIRS], rz[PAIRS];
        {
            const float* xs =
                reinterpret_cast<const float*>(w.x + s_u.row0 + (wactive ? trow0 : 0));
#pragma unroll
            for (int p = 0; p < PAIRS; ++p) {
                rx[p].x = xs[8 * p + 0];
                rx[p].y = xs[8 * p + 4];
                ry[p].x = xs[8 * p + 1];
                ry[p].y = xs[8 * p + 5];
                rz[p].x = xs[8 * p + 2];
                rz[p].y = xs[8 * p + 6];
            }
        }
        float r_best[REG_BEST ? ROWS_PER_THREAD : 1];
        unsigned r_bidx[REG_BEST ? ROWS_PER_THREAD : 1];
#pragma unroll
        for (int r = 0; r < ROWS_PER_THREAD; ++r) {
            if constexpr (REG_BEST) {
                r_best[r] = INFINITY;
                r_bidx[r] = 0u;
            } else {
                s_key[r][tid] = (u64)__float_as_uint(INFINITY) << 32;
            }
        }

        const int c_lo = s_u.sub_lo / SUBS_PER_CHUNK, c_hi = (s_u.sub_hi - 1) / SUBS_PER_CHUNK;
        for (int c = c_lo; c <= c_hi; ++c, ++seq) {
            const int b = seq & 1;
            // every lane of a warp must agree before the warp-wide reductions
            const bool ok = __all_sync(0xffffffffu, mbar_wait(&s_bar[b], (par >> b) & 1u));
            if (ok) par ^= 1u << b;
            const int sc0 = max(s_u.sub_lo, c * SUBS_PER_CHUNK);
            const int sc1 = min(s_u.sub_hi, (c + 1) * SUBS_PER_CHUNK);
            // the sub-chunks of this chunk with the first 2 NP rows of each lane
            auto scan = [&](auto np) {
                constexpr int NP = decltype(np)::value;
                for (int sc = sc0; sc < sc1; ++sc) {
                    const int off = (sc - c * SUBS_PER_CHUNK) * SUB;
                    float cm[ROWS_PER_THREAD];  // set by the sub-chunk's first step
                    sub_chunk<BIDIR, NP>(&s_t[b][0][2 * off], &s_t[b][1][2 * off],
                                         &s_t[b][2][2 * off], rx, ry, rz, cm,
                                         BIDIR ? &s_cv[b][warp][off] : nullptr,
                                         BIDIR ? &s_cb[b][warp][off] : nullptr);
                    // distances are >= 0, so their bits order like the values
#pragma unroll
                    for (int r = 0; r < 2 * NP; ++r) {
                        if constexpr (REG_BEST) {
                            if (cm[r] < r_best[r]) {
                                r_best[r] = cm[r];
                                r_bidx[r] = (unsigned)sc;
                            }
                        } else {
                            const unsigned cb = __float_as_uint(cm[r]);
                            if (cb < (unsigned)(s_key[r][tid] >> 32))
                                s_key[r][tid] = ((u64)cb << 32) | (u64)(unsigned)sc;
                        }
                    }
                }
            };
            if (ok && wactive) {  // rpl is the same for the whole warp
                if (rpl == 16)
                    scan(std::integral_constant<int, 8>());
                else if (rpl == 12)
                    scan(std::integral_constant<int, 6>());
                else
                    scan(std::integral_constant<int, 4>());
            }
            abort = __syncthreads_or(!ok) != 0;
            if (abort) break;
            if (tid == 0) {
                pending &= ~(1u << b);
                // buffer b is free again: stage chunk c + 2 into it
                if (c + 2 <= c_hi) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    mbar_expect_tx(&s_bar[b], 3 * PLANE_BYTES);
                    for (int p = 0; p < 3; ++p)
                        bulk_g2s(&s_t[b][p][0],
                                 s_u.tx + 2LL * p * s_u.Mpad + 2LL * (c + 2) * CHUNK, PLANE_BYTES,
                                 &s_bar[b]);
                    pending |= 1u << b;
                }
            }
            if (BIDIR) {
                // CTA minimum of each target of the chunk over its active warps (the lowest
                // warp and, within it, the lowest lane among equals), merged globally
                const int n_active =
                    min(WARPS, div_up(N - s_u.rb * ROWS_PER_UNIT, ROWS_PER_WARP));
                const int urow0 = s_u.rb * ROWS_PER_UNIT;
                const int j0 = sc0 * SUB - c * CHUNK;
                const int jend = min(sc1 * SUB, s_u.M) - c * CHUNK;
                for (int j = j0 + tid; j < jend; j += THREADS) {
                    unsigned bv = s_cv[b][0][j], bw = 0;
                    for (int q = 1; q < n_active; ++q) {
                        const unsigned v = s_cv[b][q][j];
                        if (v < bv) {
                            bv = v;
                            bw = q;
                        }
                    }
                    // the target's row group: the first row of the lane holding the minimum
                    // (groups are contiguous, so among equal minima the lowest first row
                    // holds the lowest row index)
                    const int lane_first = __ffs(s_cb[b][bw][j]) - 1;
                    const int brow0 = urow0 + (int)bw * ROWS_PER_WARP;
                    const unsigned g0 = (unsigned)(brow0 + lane_first * lane_rows(N - brow0));
                    atomicMin(&w.pba[s_u.col0 + c * CHUNK + j], ((u64)bv << 32) | (u64)g0);
                }
            }
        }
        if (abort) break;
        if (wactive) {
#pragma unroll
            for (int r = 0; r < ROWS_PER_THREAD; ++r) {
                const int row = trow0 + r;
                if (r < rpl && row < N) {
                    u64 key;
                    if constexpr (REG_BEST)
                        key = ((u64)__float_as_uint(r_best[r]) << 32) | (u64)r_bidx[r];
                    else
                        key = s_key[r][tid];
                    atomicMin(&w.pab[s_u.row0 + row], key);
                }
            }
        }
        s = min(s_end, w.unit_pre[u + 1]);
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
    pdl_trigger();
}

int g_chamfer_ctas[64][2][3];  // per device, mode and width: resident CTAs of the grid

template <bool BIDIR, int W>
int occupancy() {
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_chamfer<BIDIR, W>, 32 * W, 0);
    return occ;
}

int width_index(int warps) { return warps == 4 ? 2 : (warps == 2 ? 1 : 0); }

std::atomic<int> g_stall_next{0};  // dc_test_inject_stall: the next launch stalls

int g_tuned_warps = 0;  // process-wide CTA width set by dc_tune_set (0: automatic)

}  // namespace

int chamfer_grid(int mode, int warps) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    const int b = mode == DC_BIDIR_MEAN ? 0 : 1, wi = width_index(warps);
    int& n = g_chamfer_ctas[dev][b][wi];
    if (n == 0) {
        int sms = 0, occ = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (b == 0)
            occ = wi == 2 ? occupancy<true, 4>() : (wi == 1 ? occupancy<true, 2>()
                                                             : occupancy<true, 1>());
        else
            occ = wi == 2 ? occupancy<false, 4>() : (wi == 1 ? occupancy<false, 2>()
                                                              : occupancy<false, 1>());
        n = (sms > 0 ? sms : 1) * (occ > 0 ? occ : 1);
    }
    return n;
}

int choose_warps(int mode, long long sub_w4, long long sub_w2, long long sub_w1) {
    if (g_tuned_warps == 1 || g_tuned_warps == 2 || g_tuned_warps == 4) return g_tuned_warps;
    // Two warps per CTA whenever every resident CTA gets at least 8 sub-chunks (which keeps
    // the per-unit set-up small), else one. Measured on GB300: width 2 is as fast as width 4
    // on uniform trajectories (1.042 against 1.044 ms for 40 frames of 10 000 x 10 000,
    // 24.81 against 24.85 ms for 100 of 32 768 x 32 768) and 2.5% faster on 64 uneven
    // trajectories (271.2 against 278.1 ms), whose last unit per frame leaves fewer warps
    // idle at width 2 (1.4% of the warp slots against 3.8%). Width 1 costs 22% more per-CTA
    // overhead on the 40-frame trajectory. Width 4 stays available through dc_tune_set.
    (void)sub_w4;
    if (sub_w2 >= 8LL * chamfer_grid(mode, 2)) return 2;
    return 1;
}

int take_stall() { return g_stall_next.exchange(0); }

cudaError_t launch_chamfer(const Ws& w, int n_units, int total_sub, int mode, int warps,
                           cudaStream_t s) {
    const int stall = take_stall();
    // total_sub is an upper bound here (frames skipped on the device carry no work); CTAs
    // beyond the work exit at once
    if (n_units <= 0 || total_sub <= 0) return cudaSuccess;
    int grid = chamfer_grid(mode, warps);
    if (grid > total_sub) grid = total_sub;
    prof_before(s);
    const bool bi = mode == DC_BIDIR_MEAN;
    cudaError_t e;
    if (warps == 4)
        e = launch_pdl(bi ? k_chamfer<true, 4> : k_chamfer<false, 4>, grid, 128, 0, s, w,
                       stall);
    else if (warps == 2)
        e = launch_pdl(bi ? k_chamfer<true, 2> : k_chamfer<false, 2>, grid, 64, 0, s, w,
                       stall);
    else
        e = launch_pdl(bi ? k_chamfer<true, 1> : k_chamfer<false, 1>, grid, 32, 0, s, w,
                       stall);
    prof_after(s);
    count_launch();
    return e ? e : cudaGetLastError();
}

void set_tuned_warps(int warps) { g_tuned_warps = warps; }
void inject_stall() { g_stall_next.store(1); }
int tuned_warps() { return g_tuned_warps; }

}  // namespace dc
