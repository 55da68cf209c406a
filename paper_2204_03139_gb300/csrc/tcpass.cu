// Tensor-core filter of the brute-force nearest-neighbour search (Eq. 1, Eq. 2).
//
// Every row point (the sim points, and in Eq. 1 also the targets) is compared with every
// column point of its frame (the targets, respectively the sim points) through the
// expanded form |p - q|^2 = |p|^2 - 2 p.q + |q|^2, evaluated on the tensor cores with the
// split-fp16 forms that the staging kernel wrote (dc_internal.cuh): one m16n8k16 MMA gives
// 16 rows x 8 columns of approximate scaled squared distances (k_tcpass; k_tcpass5 does the
// same with tcgen05 MMAs of 128 x 128). Each of the four lanes that share a row sees a
// quarter of every block's columns (2 of every 8 positions, which tc_form_pos fills with 32
// consecutive points); per row and lane the filter keeps the three smallest block keys
// (approximate minimum over the lane's columns of a block of TC_BLOCK, truncated, with the
// block); it never decides a neighbour. k_tcrecover re-evaluates the candidate block
// quarters those keys admit, and k_tcfallback every column of the
// rows they do not certify, in the exact float32 direct form of the oracle, so neighbours
// and losses are those of the direct form.
//
// Work: units of TC_UNIT_ROWS rows of one side of one frame, times their chunks of
// TC_CHUNK columns. With few units per CTA the flattened list is split evenly over a
// persistent grid (every CTA gets the same number of chunks): a unit covered by one CTA
// writes its rows' keys to their final place; a unit split between CTAs writes each CTA's
// list to that CTA's slot in kpart (slot 0 for the part a CTA started inside the unit, 1 for
// the part that ends the CTA's range), and k_tcmerge merges them. With many units per CTA
// the CTAs take whole units in order from a counter instead.
#include <cuda_fp16.h>

#include <algorithm>

#include "dc_async.cuh"
#include "dc_internal.cuh"

namespace dc {

namespace {

// D = A B for one 16 x 8 x 16 tile (f16 inputs, f32 accumulation, C = 0)
__device__ __forceinline__ void mma_f16(float (&d)[4], const unsigned (&a)[4], unsigned b0,
                                        unsigned b1) {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%10,%10,%10,%10};"
        : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1), "f"(0.0f));
}

// the unit segment a CTA works on (shared memory, written by thread 0)
struct TcSeg {
    long long arow;  // form index of the unit's first row
    long long bcol;  // form index of the frame's first column
    unsigned* kout;  // final keys of the unit's first row
    int rows_live;   // rows of the unit to filter, from its first (k_tcpass: up to the
                     // end of the block of the side's last point; k_tcpass5: every padded row)
    int c_lo, c_hi;  // chunk range of this segment
    int whole, slot;
};

constexpr int TC_THREADS = 32 * TC_WARPS;
constexpr int TC_MT = TC_ROWS_PER_WARP / 16;  // m16 tiles per warp
#ifndef DC_TC_MIN_BLOCKS
#define DC_TC_MIN_BLOCKS 3
#endif
constexpr int TC_MIN_BLOCKS = DC_TC_MIN_BLOCKS;  // 3: 12 warps per SM

// Work split. Stream-K (dyn = 0): CTA b takes the contiguous range [b per, (b + 1) per) of
// the (unit, chunk) list, so every CTA gets the same number of chunks and a unit may be
// split between CTAs (merged by k_tcmerge). With many more units than CTAs (dyn = 1) the
// CTAs instead take whole units in list order from a counter, so that the units in flight at
// any time are neighbours, of a few frames whose target forms stay in L2; a contiguous
// range per CTA would spread the CTAs over the whole list and stream every unit's targets
// from HBM again. The tail costs at most one unit per CTA.
__global__ void __launch_bounds__(TC_THREADS, TC_MIN_BLOCKS) k_tcpass(Ws w, int stall, int dyn) {
    pdl_wait();
    constexpr uint32_t CH_BYTES = TC_CHUNK * 32;  // B forms of one chunk
    __shared__ __align__(128) unsigned s_b[2][CH_BYTES / 4];
    __shared__ __align__(8) u64 s_bar[2];
    __shared__ TcSeg s_u;
    __shared__ int s_next;
    __shared__ int s_done[2];    // warps done with the buffer's current chunk
    __shared__ int s_issued[2];  // copies ever issued into the buffer

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int n_units = w.hdr->tc_units, total = w.hdr->tc_total;
    int s = 0, s_end = 0, u = 0;
    if (!dyn) {
        const int per = (total + gridDim.x - 1) / gridDim.x;
        s = blockIdx.x * per;
        s_end = min(total, s + per);
        if (s >= s_end) return;
        u = last_le(w.tc_upre, n_units, s);
    }
    const long long tot_rows = w.hdr->total_rows;

    if (tid == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        s_done[0] = s_done[1] = 0;
        s_issued[0] = s_issued[1] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    uint32_t par = 0;      // bit b: the phase parity to wait for on buffer b
    int waited0 = 0, waited1 = 0;  // copies into buffers 0 and 1 this thread waited for
    int seq = 0;           // chunks consumed so far; buffer = seq & 1
    bool abort = false;
    const unsigned* A32 = reinterpret_cast<const unsigned*>(w.tca);

    for (;;) {
        __syncthreads();  // the previous segment is done with s_u and the buffers' contents
        if (dyn) {
            if (tid == 0) s_next = atomicAdd(&w.hdr->tc_next, 1);
            __syncthreads();
            u = s_next;
            if (u >= n_units) break;
            s = w.tc_upre[u];
            s_end = w.tc_upre[u + 1];
            if (s >= s_end) continue;  // a skipped frame's unit: no chunks
        } else if (s >= s_end) {
            break;
        }
        if (tid == 0) {
            const FrameDesc* fr = w.frames + w.tc_ufr[u];
            const int urb = w.tc_urb[u];
            const int side = urb >> 30, rb = urb & 0x3fffffff;
            const int upre = w.tc_upre[u], unext = w.tc_upre[u + 1];
            const long long first = (long long)rb * TC_UNIT_ROWS;
            // rows up to the end of the block of the side's last point: the forms spread a
            // block's points over all its positions, and a warp tile beyond has no keys to
            // give (nothing reads them)
            s_u.rows_live = round_up(side ? fr->M : fr->N, TC_BLOCK) - (int)first;
            s_u.arow = (side ? tot_rows + fr->col0 : (long long)fr->row0) + first;
            s_u.bcol = side ? (long long)fr->row0 : tot_rows + fr->col0;
            s_u.kout = side ? w.kba + TC_KEYS * ((long long)fr->col0 + first)
                            : w.kab + TC_KEYS * ((long long)fr->row0 + first);
            s_u.c_lo = s - upre;
            s_u.c_hi = min(s_end, unext) - upre - 1;
            s_u.whole = s == upre && s_end >= unext;
            s_u.slot = s > upre ? 0 : 1;
            // stage the first two chunks of the segment (both buffers are free here)
            for (int c = s_u.c_lo; c <= min(s_u.c_hi, s_u.c_lo + 1); ++c) {
                const int b = (seq + c - s_u.c_lo) & 1;
                // test of the bounded waits: the first chunk is never requested
                if (stall && seq == 0 && c == s_u.c_lo) continue;
                mbar_expect_tx(&s_bar[b], CH_BYTES);
                bulk_g2s(&s_b[b][0], w.tcb + 2 * (s_u.bcol + (long long)c * TC_CHUNK), CH_BYTES,
                         &s_bar[b]);
                ++s_issued[b];
            }
        }
        __syncthreads();
        const int wrow0 = warp * TC_ROWS_PER_WARP;  // within the unit
        // a warp's rows lie in blocks that hold a point of the side, or in none (units of
        // 512 rows may overhang the last point)
        const bool wactive = wrow0 < s_u.rows_live;

        // this warp's m16 tiles of A forms, in registers for the whole segment
        unsigned a[TC_MT][4];
#pragma unroll
        for (int m = 0; m < TC_MT; ++m) {
            const long long p = wactive ? s_u.arow + wrow0 + 16 * m : 0;
            const long long G = p >> 3;  // first of the tile's two groups of 8 rows
            a[m][0] = A32[G * 64 + g * 4 + t];
            a[m][1] = A32[(G + 1) * 64 + g * 4 + t];
            a[m][2] = A32[G * 64 + 32 + g * 4 + t];
            a[m][3] = A32[(G + 1) * 64 + 32 + g * 4 + t];
        }
        // rows 16 m + g (2 m) and 16 m + g + 8 (2 m + 1)
        unsigned k1[2 * TC_MT], k2[2 * TC_MT], k3[2 * TC_MT];
#pragma unroll
        for (int r = 0; r < 2 * TC_MT; ++r) k1[r] = k2[r] = k3[r] = TC_EMPTY;

        const int c_lo = s_u.c_lo, c_hi = s_u.c_hi;
        for (int c = c_lo; c <= c_hi; ++c, ++seq) {
            const int b = seq & 1;
            // every lane of a warp must agree before the warp-wide MMAs
            const bool ok = __all_sync(0xffffffffu, mbar_wait(&s_bar[b], (par >> b) & 1u));
            if (ok) {
                par ^= 1u << b;
                if (b) ++waited1; else ++waited0;
            }
            if (ok && wactive) {
                const unsigned* S = s_b[b];
#pragma unroll
                for (int half = 0; half < TC_CHUNK / TC_BLOCK; ++half) {
                    float bm[2 * TC_MT];
#pragma unroll
                    for (int nt = 0; nt < TC_BLOCK / 8; ++nt) {
                        const int grp = half * (TC_BLOCK / 8) + nt;  // group of 8 columns
                        const unsigned b0 = S[grp * 64 + g * 4 + t];
                        const unsigned b1 = S[grp * 64 + 32 + g * 4 + t];
#pragma unroll
                        for (int m = 0; m < TC_MT; ++m) {
                            float d[4];
                            mma_f16(d, a[m], b0, b1);
                            if (nt == 0) {
                                bm[2 * m] = fminf(d[0], d[1]);
                                bm[2 * m + 1] = fminf(d[2], d[3]);
                            } else {
                                bm[2 * m] = min3(bm[2 * m], d[0], d[1]);
                                bm[2 * m + 1] = min3(bm[2 * m + 1], d[2], d[3]);
                            }
                        }
                    }
                    // the block's keys: value clamped at 0 (the expanded form can dip below
                    // it), truncated, with the block (the lane is implied by the key's slot)
                    const unsigned id = (unsigned)(c * (TC_CHUNK / TC_BLOCK) + half);
#pragma unroll
                    for (int r = 0; r < 2 * TC_MT; ++r)
                        top3_insert(k1[r], k2[r], k3[r],
                                    (__float_as_uint(fmaxf(bm[r], 0.0f)) & TC_VALUE_MASK) | id);
                }
            }
            if (!ok) {  // the chunk never landed: give up the segment
                abort = true;
                break;
            }
            // This warp is done with buffer b. The last of the CTA's warps to get here stages
            // chunk c + 2 into it, so the warps meet at no barrier between chunks and may
            // drift up to a chunk apart (the key inserts of different warps overlap).
            __syncwarp();
            if (lane == 0) {
                __threadfence_block();  // the warp's reads of the buffer before the count
                if (atomicAdd(&s_done[b], 1) == TC_WARPS - 1) {
                    __threadfence_block();  // and every other warp's reads before the copy
                    s_done[b] = 0;
                    if (c + 2 <= c_hi) {
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        mbar_expect_tx(&s_bar[b], CH_BYTES);
                        bulk_g2s(&s_b[b][0],
                                 w.tcb + 2 * (s_u.bcol + (long long)(c + 2) * TC_CHUNK),
                                 CH_BYTES, &s_bar[b]);
                        atomicAdd(&s_issued[b], 1);
                    }
                }
            }
        }
        // a wait that gave up in any warp ends the CTA's work (the other warps' waits for
        // the chunks that are then never staged give up too, so every warp gets here)
        abort = __syncthreads_or(abort) != 0;
        if (abort) break;
        if (wactive) {
            // every lane keeps its own column subset's three smallest keys: [row][lane t][3]
            unsigned* out = s_u.whole
                                ? s_u.kout
                                : w.kpart + TC_KEYS * ((2LL * blockIdx.x + s_u.slot) * TC_UNIT_ROWS);
#pragma unroll
            for (int r = 0; r < 2 * TC_MT; ++r) {
                const int ru = wrow0 + 16 * (r >> 1) + g + 8 * (r & 1);
                unsigned* o = out + TC_KEYS * ru + 3 * t;
                o[0] = k1[r];
                o[1] = k2[r];
                o[2] = k3[r];
            }
        }
        if (!dyn) {
            s = min(s_end, w.tc_upre[u + 1]);
            ++u;
        }
    }

    if (abort) {
        if (tid == 0) {
            set_status(&w.hdr->status, DC_ETIMEOUT);
            // let copies still in flight land before the CTA's shared memory goes away (a
            // buffer holds at most one copy that thread 0 has not waited for)
            if (s_issued[0] > waited0) (void)mbar_wait(&s_bar[0], par & 1u);
            if (s_issued[1] > waited1) (void)mbar_wait(&s_bar[1], (par >> 1) & 1u);
        }
        __syncthreads();
    }
    pdl_trigger();
}

// Units split between CTAs: one CTA per unit merges the lists that its CTAs left in their
// kpart slots (the first CTA wrote slot 1, the later ones slot 0) into the unit's final keys,
// so that every row's keys are in place for the epilogue. Units covered by one CTA exit.
__global__ void __launch_bounds__(TC_THREADS) k_tcmerge(Ws w, int grid) {
    pdl_entry();
    const int u = blockIdx.x;
    if (u >= w.hdr->tc_units) return;
    const int per = max(1, (w.hdr->tc_total + grid - 1) / grid);  // as the pass split it
    const int a = w.tc_upre[u], b = w.tc_upre[u + 1];
    if (a == b) return;  // no work (skipped frame)
    const int clo = a / per, chi = (b - 1) / per;
    if (clo == chi) return;
    const FrameDesc* fr = w.frames + w.tc_ufr[u];
    const int urb = w.tc_urb[u];
    const int side = urb >> 30, rb = urb & 0x3fffffff;
    const long long first = (long long)rb * TC_UNIT_ROWS;
    // the rows whose keys are read: up to the end of the block of the side's last point
    const int rows = min(TC_UNIT_ROWS, round_up(side ? fr->M : fr->N, TC_BLOCK) - (int)first);
    unsigned* out = side ? w.kba + TC_KEYS * ((long long)fr->col0 + first)
                         : w.kab + TC_KEYS * ((long long)fr->row0 + first);
    // one thread per (row, lane) list
    for (int e = threadIdx.x; e < rows * 4; e += blockDim.x) {
        const int ru = e >> 2, lane = e & 3;
        unsigned k1 = TC_EMPTY, k2 = TC_EMPTY, k3 = TC_EMPTY;
        for (int c = clo; c <= chi; ++c) {
            const unsigned* p = w.kpart +
                                TC_KEYS * ((2LL * c + (c == clo ? 1 : 0)) * TC_UNIT_ROWS + ru) +
                                3 * lane;
            top3_insert(k1, k2, k3, p[0]);
            top3_insert(k1, k2, k3, p[1]);
            top3_insert(k1, k2, k3, p[2]);
        }
        unsigned* o = out + TC_KEYS * ru + 3 * lane;
        o[0] = k1;
        o[1] = k2;
        o[2] = k3;
    }
}

// ---------------------------------------------------------------------------------------
// exact recovery of every row's minimum and neighbour from its keys
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ float key_value(unsigned k) {
    return __uint_as_float(k & TC_VALUE_MASK);
}

// Threshold of a row whose scaled point has norm r, given its smallest key kmin (scaled
// units throughout): any block whose minimum exceeds it holds no candidate.
//
// With e(q) the filter's error at column q, the exact float32 minimum j* satisfies
// a(j*) <= d(j*) + e(j*) <= d(k) + e(j*) <= a(k) + e(k) + e(j*) = m + e(k) + e(j*) for the
// column k of the filter's minimum m. Both pairs have d <= D = m + E(D), where
// E(D) = kappa u (2 r + sqrt(D))^2 + 8 u D bounds e for a pair at distance^2 at most D
// (|s_q| <= r + sqrt(d)); so a block whose minimum exceeds tau = m + 2 E(D) holds no
// candidate. The key values are truncated (at most 2^-11 low) and clamped at 0, which the
// bounds below absorb. D is found from an upper bound by two contracting steps.
__device__ __forceinline__ float tc_tau(unsigned kmin, float r) {
    const float u = 0x1p-24f, ku = TC_KAPPA * u, alpha = 2.0f * ku + 8.0f * u;
    const float m = key_value(kmin) * (1.0f + 0x1p-10f);
    auto E = [&](float D) {
        const float q = 2.0f * r + sqrtf(D);
        return ku * q * q + 8.0f * u * D;
    };
    float D = (m + 8.0f * ku * r * r) * (1.0f + 2.0f * alpha);  // >= that / (1 - alpha)
    D = m + E(D);
    D = m + E(D);
    return (m + 2.0f * E(D)) * (1.0f + 0x1p-16f);
}

// dx = a - b, d = fma(dz, dz, fma(dy, dy, dx * dx)): the float32 direct form of the oracle
__device__ __forceinline__ float dist2(float ax, float ay, float az, float bx, float by,
                                       float bz) {
    const float dx = __fsub_rn(ax, bx), dy = __fsub_rn(ay, by), dz = __fsub_rn(az, bz);
    return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
}

__device__ __forceinline__ u64 min64(u64 a, u64 b) { return a < b ? a : b; }

__device__ __forceinline__ u64 pack_d(float d, int j) {
    return ((u64)__float_as_uint(d) << 32) | (u64)(unsigned)j;
}

// The columns of side `side` of frame fr: targets from their compact planes, sim points from
// the sampled rows.
struct Cols {
    const float* X;
    const float* Y;
    const float* Z;
    const float4* P;  // sim points (side 1), else nullptr
    int n;
    __device__ __forceinline__ void get(int j, float& x, float& y, float& z) const {
        if (P) {
            const float4 p = P[j];
            x = p.x, y = p.y, z = p.z;
        } else {
            x = X[j], y = Y[j], z = Z[j];
        }
    }
};

__device__ __forceinline__ Cols frame_cols(const Ws& w, const FrameDesc* fr, int side) {
    Cols c;
    c.X = w.tpl + 3LL * fr->col0;
    c.Y = c.X + fr->Mpad;
    c.Z = c.Y + fr->Mpad;
    c.P = side ? w.x + fr->row0 : nullptr;
    c.n = side ? fr->N : fr->M;
    return c;
}

// the query point of row i of side `side`
__device__ __forceinline__ float3 frame_row(const Ws& w, const FrameDesc* fr, int side, int i) {
    if (side) {
        const float* X = w.tpl + 3LL * fr->col0;
        return make_float3(X[i], X[fr->Mpad + i], X[2 * fr->Mpad + i]);
    }
    const float4 p = w.x[fr->row0 + i];
    return make_float3(p.x, p.y, p.z);
}

constexpr int REC_THREADS = 256;     // one row per thread: 256 rows per CTA step
constexpr int REC_MIN_BLOCKS = 4;    // 64 registers (one small spill): 32 warps per SM
constexpr int REC_MAX_CAND = 2 * 4;  // candidates per row: two blocks per column quarter

// The rows' exact minima from their keys: rows [0, rows) are sim points, rows
// [rows, total) targets (Eq. 1 only). Each CTA takes a contiguous range of rows, 256 at a
// time (frames are padded to multiples of 256 rows, so a step's rows lie in one frame, found
// by walking the frame table forward). Each thread takes one row: it reads the row's 12 keys
// (at the row's form position; loaded during the CTA's previous step), computes the
// threshold once, and lists the candidate block quarters (per quarter, the first two keys
// under the threshold); a warp prefix sum lays the warp's candidates out in shared memory,
// and the warp re-checks them eight at a time, four lanes per candidate (its 32 consecutive
// columns, eight per lane, in loads of 64 contiguous bytes per candidate) in the direct
// form, merging into the row's minimum with a shared atomicMin. A row that the keys do not
// certify (a quarter's third key under the threshold) is queued in its frame's list for
// k_tcfallback. Writes (distance bits << 32 | index) to pab / pba. Measured on 64 uneven
// trajectories (176.8 ms per batch): eight lanes per candidate (a whole line per load, four
// candidates per warp step) took 2.8 to 4.0 ms more, other register budgets (3, 5 or 6 CTAs
// per SM) 2.2 to 3.3 ms more, no key prefetch 1.9 ms more. (Four lanes per row, each with
// one quarter's keys, took 81 warp instructions per row: the threshold was computed four
// times and a warp step covered only 8 rows. With the quarters interleaved in the block, a
// candidate's re-check read 12 lines of targets for 384 bytes.)
__global__ void __launch_bounds__(REC_THREADS, REC_MIN_BLOCKS)
    k_tcrecover(Ws w, int rows, int total) {
    pdl_entry();
    constexpr int NW = REC_THREADS / 32;
    __shared__ float s_q[NW][32][3];                 // per warp: each row's query point
    __shared__ unsigned s_list[NW][32 * REC_MAX_CAND];  // candidates: (cand << 5) | row
    __shared__ u64 s_best[NW][32];                   // per warp: the rows' packed minima
    const int steps = div_up(total, REC_THREADS);
    const int per = div_up(steps, gridDim.x);
    const int st0 = blockIdx.x * per, st1 = min(steps, st0 + per);
    const int n_frames = w.hdr->n_frames;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int k = -1, side = -1;
    // the keys of the CTA's next step are loaded during this step's re-checks (every step's
    // rows lie inside the key arrays: both sides are whole numbers of steps)
    auto key_ptr = [&](int st_) {
        const int b_ = st_ * REC_THREADS;
        const int g_ = (b_ >= rows ? b_ - rows : b_) + (int)threadIdx.x;
        return reinterpret_cast<const uint4*>((b_ >= rows ? w.kba : w.kab) +
                                              (long long)TC_KEYS * tc_form_pos(g_));
    };
    uint4 n0 = make_uint4(0, 0, 0, 0), n1 = n0, n2 = n0;
    if (st0 < st1) {
        const uint4* p = key_ptr(st0);
        n0 = p[0], n1 = p[1], n2 = p[2];
    }
    for (int st = st0; st < st1; ++st) {
        const uint4 v0 = n0, v1 = n1, v2 = n2;  // this step's rows' keys
        if (st + 1 < st1) {
            const uint4* p = key_ptr(st + 1);
            n0 = p[0], n1 = p[1], n2 = p[2];
        }
        const int base = st * REC_THREADS;
        const int sd = base >= rows ? 1 : 0;
        const int g0 = sd ? base - rows : base;  // first row of the step within its side
        if (sd != side) {
            side = sd;
            k = last_le(side ? w.colpre : w.rowpre, n_frames, g0);
        }
        const int* pre = side ? w.colpre : w.rowpre;
        while (k + 1 < n_frames && pre[k + 1] <= g0) ++k;
        const FrameDesc* fr = w.frames + k;
        if (fr->skip) continue;  // uniform over the CTA
        const int g = g0 + threadIdx.x;
        const int i = g - (side ? fr->col0 : fr->row0);
        const bool valid = i < (side ? fr->M : fr->N);
        const Cols C = frame_cols(w, fr, side);

        // candidate j = 2 t + i of the row is quarter t's key i, if bit j of cmask is set
        unsigned kk[TC_KEYS];
        unsigned cmask = 0;
        bool full = false;
        float qx = 0.f, qy = 0.f, qz = 0.f;
        if (valid) {
            // quarter t's keys are kk[3 t], kk[3 t + 1], kk[3 t + 2], smallest first
            kk[0] = v0.x, kk[1] = v0.y, kk[2] = v0.z, kk[3] = v0.w;
            kk[4] = v1.x, kk[5] = v1.y, kk[6] = v1.z, kk[7] = v1.w;
            kk[8] = v2.x, kk[9] = v2.y, kk[10] = v2.z, kk[11] = v2.w;
            const unsigned kmin = min(min(kk[0], kk[3]), min(kk[6], kk[9]));
            const float3 x = frame_row(w, fr, side, i);
            qx = x.x, qy = x.y, qz = x.z;
            if (kmin == TC_EMPTY) {
                full = true;  // no key at all: scan the whole frame
            } else {
                const float4 box = w.fbox[k];
                const float sx = __fmul_rn(__fsub_rn(qx, box.x), box.w);
                const float sy = __fmul_rn(__fsub_rn(qy, box.y), box.w);
                const float sz = __fmul_rn(__fsub_rn(qz, box.z), box.w);
                const float r = sqrtf(__fmaf_rn(sz, sz, __fmaf_rn(sy, sy, __fmul_rn(sx, sx)))) *
                                (1.0f + 0x1p-20f);
                const float tau = tc_tau(kmin, r);
#pragma unroll
                for (int t = 0; t < 4; ++t) {
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        const unsigned key = kk[3 * t + j];
                        if (key != TC_EMPTY && key_value(key) <= tau) cmask |= 1u << (2 * t + j);
                    }
                    // the quarter may hide a candidate beyond its keys
                    if (kk[3 * t + 2] != TC_EMPTY && key_value(kk[3 * t + 2]) <= tau) full = true;
                }
            }
        }
        if (!valid || full) cmask = 0;
        const int nc = __popc(cmask);
        // the warp's candidates, laid out by an exclusive prefix sum of the rows' counts
        int off = nc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, off, o);
            if (lane >= o) off += y;
        }
        const int tot = __shfl_sync(0xffffffffu, off, 31);
        off -= nc;
        s_q[warp][lane][0] = qx;
        s_q[warp][lane][1] = qy;
        s_q[warp][lane][2] = qz;
        s_best[warp][lane] = EMPTY;
        // candidates as (block << 2 | the pass's lane whose columns they name) << 5 | row
#pragma unroll
        for (int j = 0; j < REC_MAX_CAND; ++j)
            if (cmask & (1u << j))
                s_list[warp][off + __popc(cmask & ((1u << j) - 1u))] =
                    ((((kk[(j >> 1) * 3 + (j & 1)] & ~TC_VALUE_MASK) << 2) | (unsigned)(j >> 1))
                     << 5) | (unsigned)lane;
        __syncwarp();
        // each candidate quarter (32 consecutive columns) is scanned by four lanes, eight
        // candidates per warp step, eight columns per lane in contiguous loads (the four
        // lanes of a candidate read 64 contiguous bytes per instruction), and merged into its
        // row's minimum
        const int sub = lane >> 2, l4 = lane & 3;
        for (int e0 = 0; e0 < tot; e0 += 8) {
            const int e = e0 + sub;
            float bd = INFINITY;
            int bj = 0x7fffffff, er = -1;
            if (e < tot) {
                const unsigned ent = s_list[warp][e];
                er = (int)(ent & 31u);
                const unsigned c = ent >> 5;
                // the quarter tq of block blk: points 32 tq .. 32 tq + 31 of the block
                const int q0 = (int)(c >> 2) * TC_BLOCK + (int)(c & 3u) * (TC_BLOCK / 4);
                const float ex = s_q[warp][er][0], ey = s_q[warp][er][1], ez = s_q[warp][er][2];
                if (C.P) {
                    // sim points: this lane takes q0 + l4 + 4 h (a frame's rows are padded to
                    // whole blocks, so every load stays inside it)
                    float4 p[8];
#pragma unroll
                    for (int h = 0; h < 8; ++h) p[h] = C.P[q0 + l4 + 4 * h];
#pragma unroll
                    for (int h = 0; h < 8; ++h) {
                        const int j = q0 + l4 + 4 * h;
                        const float d = dist2(ex, ey, ez, p[h].x, p[h].y, p[h].z);
                        if (j < C.n && d < bd) bd = d, bj = j;
                    }
                } else {
                    // targets: this lane takes q0 + 4 l4 + 16 h .. q0 + 4 l4 + 16 h + 3 (h < 2)
                    // of each plane (16-byte aligned: the planes start at multiples of 256)
                    float4 X[2], Y[2], Z[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int j = q0 + 4 * l4 + 16 * h;
                        X[h] = *reinterpret_cast<const float4*>(C.X + j);
                        Y[h] = *reinterpret_cast<const float4*>(C.Y + j);
                        Z[h] = *reinterpret_cast<const float4*>(C.Z + j);
                    }
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int j = q0 + 4 * l4 + 16 * h;
                        const float d0 = dist2(ex, ey, ez, X[h].x, Y[h].x, Z[h].x);
                        const float d1 = dist2(ex, ey, ez, X[h].y, Y[h].y, Z[h].y);
                        const float d2 = dist2(ex, ey, ez, X[h].z, Y[h].z, Z[h].z);
                        const float d3 = dist2(ex, ey, ez, X[h].w, Y[h].w, Z[h].w);
                        if (j < C.n && d0 < bd) bd = d0, bj = j;
                        if (j + 1 < C.n && d1 < bd) bd = d1, bj = j + 1;
                        if (j + 2 < C.n && d2 < bd) bd = d2, bj = j + 2;
                        if (j + 3 < C.n && d3 < bd) bd = d3, bj = j + 3;
                    }
                }
            }
            // (distance bits << 32 | index): the smallest is the lowest index among equals
            u64 key = bj == 0x7fffffff ? EMPTY : pack_d(bd, bj);
            key = min64(key, __shfl_xor_sync(0xffffffffu, key, 1));
            key = min64(key, __shfl_xor_sync(0xffffffffu, key, 2));
            if (l4 == 0 && er >= 0) atomicMin(&s_best[warp][er], key);
        }
        __syncwarp();
        if (valid) {
            u64* out = side ? w.pba : w.pab;
            if (full) {
                out[g] = EMPTY;
                // the frame's list for this side: entries at its own row range
                const int slot = atomicAdd(&w.tcfn[2 * k + side], 1);
                w.tcfb[(side ? rows + fr->col0 : fr->row0) + slot] = i;
                atomicAdd(&w.hdr->tc_fallback, 1);
            } else {
                out[g] = s_best[warp][lane];
            }
        }
        __syncwarp();  // the next step reuses the warp's shared lists
    }
}

constexpr int FB_THREADS = 256;            // eight warps
constexpr int FB_ROWS_PER_WARP = 8;        // queued rows a warp evaluates at once
constexpr int FB_TILE = 512;               // columns per shared-memory tile
constexpr int FB_SPLIT = 4;                // CTAs per list at least
constexpr int FB_SPLIT_MAX = 64;           // and at most

// The rows that their keys did not certify, `split` CTAs per (frame, side) list, each over
// a contiguous part of the frame's columns: they stream through shared memory in tiles, each
// loaded once for up to 64 queued rows (eight per warp, the lanes splitting the columns); the
// parts' minima merge with atomicMin on (distance bits << 32 | index), so every row ends with
// its minimum and the lowest index attaining it. Few frames get more parts each, so that the
// launch still fills the GPU (one 32 768-point frame: 8 CTAs took 279 us).
__global__ void __launch_bounds__(FB_THREADS) k_tcfallback(Ws w, int rows, int split) {
    pdl_entry();
    __shared__ float s_c[3][FB_TILE];
    const int part = blockIdx.x % split, ks = blockIdx.x / split;
    const int k = ks >> 1, side = ks & 1;
    if (k >= w.hdr->n_frames) return;
    const FrameDesc* fr = w.frames + k;
    if (fr->skip) return;
    const int n = w.tcfn[2 * k + side];
    if (n == 0) return;
    const Cols C = frame_cols(w, fr, side);
    const int* list = w.tcfb + (side ? rows + fr->col0 : fr->row0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int PER_CTA = FB_ROWS_PER_WARP * (FB_THREADS / 32);
    for (int r0 = 0; r0 < n; r0 += PER_CTA) {
        // a warp without a queued row only helps stage the tiles (most lists are short)
        const bool wrows = r0 + warp * FB_ROWS_PER_WARP < n;
        float qx[FB_ROWS_PER_WARP], qy[FB_ROWS_PER_WARP], qz[FB_ROWS_PER_WARP];
        u64 best[FB_ROWS_PER_WARP];
#pragma unroll
        for (int t = 0; t < FB_ROWS_PER_WARP; ++t) {
            const int e = r0 + warp * FB_ROWS_PER_WARP + t;
            const float3 x = frame_row(w, fr, side, e < n ? list[e] : list[0]);
            qx[t] = x.x, qy[t] = x.y, qz[t] = x.z;
            best[t] = EMPTY;
        }
        const int ja = (int)((long long)C.n * part / split);
        const int jb = (int)((long long)C.n * (part + 1) / split);
        for (int j0 = ja; j0 < jb; j0 += FB_TILE) {
            __syncthreads();  // the previous tile is consumed
            for (int j = threadIdx.x; j < FB_TILE; j += FB_THREADS) {
                float x = 0.f, y = 0.f, z = 0.f;
                if (j0 + j < jb) C.get(j0 + j, x, y, z);
                s_c[0][j] = x;
                s_c[1][j] = y;
                s_c[2][j] = z;
            }
            __syncthreads();
            const int jn = wrows ? min(FB_TILE, jb - j0) : 0;
            for (int j = lane; j < jn; j += 32) {
                const float cx = s_c[0][j], cy = s_c[1][j], cz = s_c[2][j];
#pragma unroll
                for (int t = 0; t < FB_ROWS_PER_WARP; ++t)
                    best[t] = min64(best[t], pack_d(dist2(qx[t], qy[t], qz[t], cx, cy, cz),
                                                    j0 + j));
            }
        }
#pragma unroll
        for (int t = 0; t < FB_ROWS_PER_WARP; ++t) {
            u64 b = best[t];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) b = min64(b, __shfl_xor_sync(0xffffffffu, b, o));
            const int e = r0 + warp * FB_ROWS_PER_WARP + t;
            if (lane == 0 && e < n && b != EMPTY) {
                const int i = list[e];
                atomicMin(&(side ? w.pba + fr->col0 : w.pab + fr->row0)[i], b);
            }
        }
    }
}

// ---------------------------------------------------------------------------------------
// The same filter on the fifth-generation tensor cores: tcgen05 MMAs write the distances to
// tensor memory asynchronously. A CTA takes a 512-row unit in two halves of 256 rows, each
// two tiles of M = 128 rows. Each tile has two slots of 128 columns of tensor memory (2 tiles
// x 2 slots x 128 columns fill it), and one MMA (N = 128, K = 16) fills a slot with the
// distances of one key block of TC_BLOCK columns: slot 0 takes the even blocks, slot 1 the
// odd ones. 8 consumer warps hold one row per thread (tile t is read by warps 4t .. 4t+3, one
// lane quarter each) and read their tile's two slots in turn, so a slot's refill with the
// block after next runs while the warp reads the other one. Each warp folds a block into the
// four column subsets (2 of every 8 positions) and their keys exactly as the warp-level kernel
// does, so the keys, their merge across CTAs and the recovery are shared. One MMA warp per slot
// issues its MMAs (a bounded wait for the slot's release and for the chunk, then the MMA and
// its commit), and a producer warp streams the column chunks through four shared-memory
// buffers with bulk copies.
//
// An MMA issues at a fixed cost of about as many cycles as an N = 128, K = 16 product takes,
// whatever N up to 128, and every slot read costs its warp a wait, a vote, fences and an
// arrival; 128-column slots halve that cost per distance against 64-column ones.
// ---------------------------------------------------------------------------------------
constexpr int T5_CWARPS = 8;                           // consumer warps (one row per thread)
constexpr int T5_MWARPS = 4;                           // MMA-issuing warps, one per slot
constexpr int T5_THREADS = 32 * (T5_CWARPS + T5_MWARPS + 1);  // and the producer warp
constexpr int T5_N = TC_BLOCK;                         // columns per MMA: one key block
constexpr int T5_KB = TC_CHUNK / TC_BLOCK;             // key blocks per staged chunk
constexpr int T5_BUFS = 4;                             // staged chunks
constexpr int T5_HALF = 256;                           // rows per half unit (two tiles)
constexpr int T5_SLOTS = 4;                            // (tile, block parity)
constexpr uint32_t T5_TMEM_COLS = T5_SLOTS * T5_N;     // 512: all of an SM's tensor memory
// MMAs that read one staged chunk in a half: each slot once (two tiles x two blocks)
constexpr int T5_CHUNK_READS = T5_SLOTS;
// dynamic shared memory: the staged chunks, padded so that one CTA fills an SM (the CTA
// allocates all of the SM's tensor memory)
constexpr int T5_SMEM_B = T5_BUFS * TC_CHUNK * 32;     // 32 KB of staged chunks
constexpr int T5_SMEM = 100 * 1024;
static_assert(T5_KB == 2 && TC_UNIT_ROWS == 2 * T5_HALF && T5_TMEM_COLS == 512,
              "two key blocks per chunk, two halves per unit, tensor memory full");
static_assert(T5_SMEM_B <= T5_SMEM, "dynamic shared memory");

// shared-memory matrix descriptor of a K-major operand without swizzle, as the staging lays
// it out: core matrices of 8 rows x 16 bytes, 128 bytes between the two halves of K (the
// leading dimension), 256 bytes between groups of 8 rows; descriptor version 1
__device__ __forceinline__ uint64_t t5_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(128 >> 4) << 16) |
           ((uint64_t)(256 >> 4) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor: f16 A and B, f32 D, both K-major, M = 128, N = T5_N
constexpr uint32_t T5_IDESC = (1u << 4) | ((uint32_t)(T5_N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ void t5_mma(uint32_t d_tmem, uint64_t ad, uint64_t bd) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(ad), "l"(bd), "r"(T5_IDESC), "r"(0)
        : "memory");
}
__device__ __forceinline__ void t5_commit(u64* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void t5_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void t5_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(u64* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// 32 consecutive columns of the 32 tensor-memory lanes of this warp, one row per lane
__device__ __forceinline__ void t5_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// fold 32 columns (four groups of 8) into the four column subsets' running minima; subset t
// holds the columns 8 g + 2 t and 8 g + 2 t + 1 of every group g
__device__ __forceinline__ void t5_fold(const float (&v)[32], float (&bm)[4], bool first) {
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        float m = first ? fminf(v[2 * t], v[2 * t + 1]) : min3(bm[t], v[2 * t], v[2 * t + 1]);
#pragma unroll
        for (int g = 1; g < 4; ++g) m = min3(m, v[8 * g + 2 * t], v[8 * g + 2 * t + 1]);
        bm[t] = m;
    }
}

__global__ void __launch_bounds__(T5_THREADS, 1) k_tcpass5(Ws w, int stall, int dyn) {
    pdl_wait();
    __shared__ __align__(1024) uint4 s_a[TC_UNIT_ROWS * 2];  // A forms of the unit, 16 KB
    extern __shared__ __align__(1024) uint4 t5_dyn[];
    uint4* const s_b = t5_dyn;                                // T5_BUFS chunks of B forms
    // s_bar_b: a chunk landed; s_cfree: the MMAs that read a chunk are complete;
    // s_full: a slot's MMA is complete; s_free: a slot's four warps have read it
    __shared__ __align__(8) u64 s_bar_a, s_bar_b[T5_BUFS], s_cfree[T5_BUFS], s_full[T5_SLOTS],
        s_free[T5_SLOTS], s_drain;
    __shared__ uint32_t s_tmem;
    __shared__ TcSeg s_u;
    __shared__ int s_next;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool consumer = warp < T5_CWARPS;
    const bool mwarp = warp >= T5_CWARPS && warp < T5_CWARPS + T5_MWARPS;
    const bool producer = warp == T5_CWARPS + T5_MWARPS;
    const int n_units = w.hdr->tc_units, total = w.hdr->tc_total;
    // the work split of the warp-level kernel: stream-K, or whole units on demand (dyn)
    int s = 0, s_end = 0, u = 0;
    if (!dyn) {
        const int per = (total + gridDim.x - 1) / gridDim.x;
        s = blockIdx.x * per;
        s_end = min(total, s + per);
        if (s >= s_end) return;
        u = last_le(w.tc_upre, n_units, s);
    }
    const long long tot_rows = w.hdr->total_rows;

    if (warp == 0) {
        asm volatile(
            "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                smem_u32(&s_tmem)),
            "r"(T5_TMEM_COLS)
            : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(&s_bar_a, 1);
        mbar_init(&s_drain, T5_MWARPS);  // the four issuing threads
        for (int i = 0; i < T5_BUFS; ++i) {
            mbar_init(&s_bar_b[i], 1);
            mbar_init(&s_cfree[i], T5_CHUNK_READS);
        }
        for (int i = 0; i < T5_SLOTS; ++i) {
            mbar_init(&s_full[i], 1);
            mbar_init(&s_free[i], 4);  // the tile's four warps
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    t5_fence_before();
    __syncthreads();
    t5_fence_after();
    const uint32_t tmem = s_tmem;
    // consumer warp: tile and lane quarter; slot (tile, parity) holds tensor-memory columns
    // 128 (2 tile + parity) ..; MMA warp m issues the MMAs of slot m
    const int quarter = warp & 3, tile = (warp >> 2) & 1;
    const int my_slot = warp - T5_CWARPS;
    const bool issuer = mwarp && lane == 0;
    const bool stager = producer && lane == 0;

    int use0 = 0, use1 = 0;  // consumer: blocks read from its tile's slots 0 and 1
    int nis = 0;             // issuing thread: MMAs issued into its slot
    uint32_t pend_b = 0;     // stager: buffers with a copy in flight
    uint32_t pend_p = 0;     // and the phase that copy completes
    long long chunk0 = 0;    // chunks staged before this pass (buffer of chunk k: k % 4)
    int n_seg = 0;           // segments begun (phase of the A barrier)
    bool abort = false, issued = false;

    while (!abort) {
        __syncthreads();  // the previous segment is done with s_u and s_a
        if (dyn) {
            if (tid == 0) s_next = atomicAdd(&w.hdr->tc_next, 1);
            __syncthreads();
            u = s_next;
            if (u >= n_units) break;
            s = w.tc_upre[u];
            s_end = w.tc_upre[u + 1];
            if (s >= s_end) continue;  // a skipped frame's unit: no chunks
        } else if (s >= s_end) {
            break;
        }
        if (stager) {
            const FrameDesc* fr = w.frames + w.tc_ufr[u];
            const int urb = w.tc_urb[u];
            const int side = urb >> 30, rb = urb & 0x3fffffff;
            const int upre = w.tc_upre[u], unext = w.tc_upre[u + 1];
            const long long first = (long long)rb * TC_UNIT_ROWS;
            s_u.rows_live = (side ? fr->Mpad : fr->Npad) - (int)first;
            s_u.arow = (side ? tot_rows + fr->col0 : (long long)fr->row0) + first;
            s_u.bcol = side ? (long long)fr->row0 : tot_rows + fr->col0;
            s_u.kout = side ? w.kba + TC_KEYS * ((long long)fr->col0 + first)
                            : w.kab + TC_KEYS * ((long long)fr->row0 + first);
            s_u.c_lo = s - upre;
            s_u.c_hi = min(s_end, unext) - upre - 1;
            s_u.whole = s == upre && s_end >= unext;
            s_u.slot = s > upre ? 0 : 1;
            // the unit's A forms (its rows that exist; a multiple of 256 rows)
            const uint32_t abytes = (uint32_t)min(TC_UNIT_ROWS, s_u.rows_live) * 32u;
            mbar_expect_tx(&s_bar_a, abytes);
            bulk_g2s(&s_a[0], w.tca + 2 * s_u.arow, abytes, &s_bar_a);
        }
        __syncthreads();
        const int c_lo = s_u.c_lo, c_hi = s_u.c_hi;
        const int nhalves = s_u.rows_live >= TC_UNIT_ROWS ? 2 : 1;
        const int nkb = (c_hi - c_lo + 1) * T5_KB;

        for (int h = 0; h < nhalves && !abort; ++h) {
            if (stager) {
                // stream the pass's chunks; chunk k reuses the buffer of chunk k - 4 once the
                // MMAs that read that one are complete
                for (int c = c_lo; c <= c_hi; ++c) {
                    const long long k = chunk0 + (c - c_lo);
                    const int b = (int)(k & (T5_BUFS - 1));
                    if (k >= T5_BUFS && !mbar_wait(&s_cfree[b], (uint32_t)(((k >> 2) - 1) & 1))) {
                        abort = true;
                        break;
                    }
                    if (stall && k == 0) continue;  // test of the bounded waits only
                    mbar_expect_tx(&s_bar_b[b], TC_CHUNK * 32);
                    bulk_g2s(s_b + b * (TC_CHUNK * 2),
                             w.tcb + 2 * (s_u.bcol + (long long)c * TC_CHUNK), TC_CHUNK * 32,
                             &s_bar_b[b]);
                    pend_b |= 1u << b;
                    pend_p = (pend_p & ~(1u << b)) | ((uint32_t)((k >> 2) & 1) << b);
                }
            } else if (issuer) {
                // slot my_slot: tile my_slot / 2, key blocks of parity my_slot % 2
                const int mt = my_slot >> 1, par = my_slot & 1;
                const uint64_t a_desc =
                    t5_desc(smem_u32(&s_a[0]) + (uint32_t)((2 * h + mt) * 4096));
                bool ok = h > 0 || mbar_wait(&s_bar_a, (uint32_t)(n_seg & 1));
                int first = 1;
                for (int kb = par; ok && kb < nkb; kb += 2) {
                    if (!first) {
                        // the slot's previous block has been read: its chunk has one reader
                        // fewer, and the slot takes this block
                        ok = mbar_wait(&s_free[my_slot], (uint32_t)((nis - 1) & 1));
                        if (!ok) break;
                        mbar_arrive(&s_cfree[(int)((chunk0 + (kb - 2) / T5_KB) & (T5_BUFS - 1))]);
                    }
                    first = 0;
                    const long long k = chunk0 + kb / T5_KB;
                    const int b = (int)(k & (T5_BUFS - 1));
                    ok = mbar_wait(&s_bar_b[b], (uint32_t)((k >> 2) & 1));
                    if (!ok) break;
                    t5_fence_after();
                    t5_mma(tmem + (uint32_t)(my_slot * T5_N), a_desc,
                           t5_desc(smem_u32(s_b + b * (TC_CHUNK * 2)) +
                                   (uint32_t)((kb % T5_KB) * TC_BLOCK * 32)));
                    t5_commit(&s_full[my_slot]);
                    issued = true;
                    ++nis;
                }
                // the last block of the pass: once read, its chunk has one reader fewer
                if (ok) {
                    const int last = par + ((nkb - 1 - par) / 2) * 2;
                    ok = mbar_wait(&s_free[my_slot], (uint32_t)((nis - 1) & 1));
                    if (ok) mbar_arrive(&s_cfree[(int)((chunk0 + last / T5_KB) & (T5_BUFS - 1))]);
                }
                abort = !ok;
            } else if (consumer) {
                bool ok = true;
                float bm[4];
                unsigned k1[4], k2[4], k3[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) k1[t] = k2[t] = k3[t] = TC_EMPTY;
                const uint32_t taddr = tmem + ((uint32_t)(32 * quarter) << 16);
                for (int kb = 0; kb < nkb; ++kb) {
                    const int sl = 2 * tile + (kb & 1);
                    const int use = (kb & 1) ? use1 : use0;
                    if (!__all_sync(0xffffffffu, mbar_wait(&s_full[sl], (uint32_t)(use & 1)))) {
                        ok = false;
                        break;
                    }
                    t5_fence_after();
                    const uint32_t ta = taddr + (uint32_t)(sl * T5_N);
                    float v[32];
#pragma unroll 1
                    for (int i = 0; i < T5_N / 32 - 1; ++i) {
                        t5_ld32(ta + 32 * i, v);
                        t5_fold(v, bm, i == 0);
                    }
                    t5_ld32(ta + T5_N - 32, v);
                    // the slot is read: release it to its next MMA, then fold
                    t5_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&s_free[sl]);
                    if (kb & 1) ++use1; else ++use0;
                    t5_fold(v, bm, false);
                    // the block's keys: value clamped at 0 and truncated, with the block (the
                    // subset is implied by the key's slot)
                    const unsigned id = (unsigned)(c_lo * T5_KB + kb);
#pragma unroll
                    for (int t = 0; t < 4; ++t)
                        top3_insert(k1[t], k2[t], k3[t],
                                    (__float_as_uint(fmaxf(bm[t], 0.0f)) & TC_VALUE_MASK) | id);
                }
                abort = !ok;
                if (ok) {
                    unsigned* out = s_u.whole
                                        ? s_u.kout
                                        : w.kpart + TC_KEYS * ((2LL * blockIdx.x + s_u.slot) *
                                                               TC_UNIT_ROWS);
                    unsigned* o = out + TC_KEYS * (h * T5_HALF + tile * 128 + quarter * 32 + lane);
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        o[3 * t] = k1[t];
                        o[3 * t + 1] = k2[t];
                        o[3 * t + 2] = k3[t];
                    }
                }
            }
            // a wait that gave up anywhere ends the CTA's work (every other wait then gives
            // up too, since no further MMA is issued or read, so every warp gets here)
            abort = __syncthreads_or(abort) != 0;
            if (abort) break;
            // every copy of the pass has landed: each was waited for before its MMAs
            pend_b = 0;
            chunk0 += c_hi - c_lo + 1;
        }
        if (abort) break;
        ++n_seg;
        if (!dyn) {
            s = min(s_end, w.tc_upre[u + 1]);
            ++u;
        }
    }

    if (abort) {
        if (tid == 0) set_status(&w.hdr->status, DC_ETIMEOUT);
        // let the MMAs and copies still in flight finish before the CTA's tensor memory and
        // shared memory go away
        if (issuer) {
            if (issued)
                t5_commit(&s_drain);
            else
                mbar_arrive(&s_drain);
        }
        if (stager) {
            (void)mbar_wait(&s_drain, 0u);
            for (int b = 0; b < T5_BUFS; ++b)
                if (pend_b & (1u << b)) (void)mbar_wait(&s_bar_b[b], (pend_p >> b) & 1u);
        }
    }
    t5_fence_before();
    __syncthreads();
    t5_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(T5_TMEM_COLS)
                     : "memory");
    pdl_trigger();
}

int g_tc_ctas[64];   // per device: resident CTAs of the persistent grid
int g_rec_ctas[64];  // per device: resident CTAs of the recovery

}  // namespace

int tc_grid(long long total_chunks) {
    int dev = 0, n = TC_MAX_GRID;  // without a device: the largest grid the layout allows
    if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64) {
        int& c = g_tc_ctas[dev];
        if (c == 0) {
            int sms = 0, occ = 0;
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) ==
                    cudaSuccess &&
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_tcpass, TC_THREADS, 0) ==
                    cudaSuccess &&
                sms > 0 && occ > 0)
                c = sms * occ < TC_MAX_GRID ? sms * occ : TC_MAX_GRID;
        }
        if (c > 0) n = c;
    } else {
        cudaGetLastError();  // clear the sticky-free error of a machine without a device
    }
    const long long g = total_chunks < n ? total_chunks : n;
    return (int)(g < 1 ? 1 : g);
}

int g_t5_smem_set[64];

int tc5_grid(long long total_chunks) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms <= 0) {
        cudaGetLastError();
        sms = TC_MAX_GRID;
    }
    const long long g = total_chunks < sms ? total_chunks : sms;
    return (int)(g < 1 ? 1 : g);
}

cudaError_t launch_tcpass(const Ws& w, int engine, int grid, long long total_chunks,
                          int n_units, int rows, int cols, int mode, int n_frames,
                          cudaStream_t s) {
    const int stall = take_stall();
    cudaError_t e = cudaSuccess;
    if (engine == ENGINE_TC5) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (dev >= 0 && dev < 64 && !g_t5_smem_set[dev]) {
            e = cudaFuncSetAttribute(k_tcpass5, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     T5_SMEM);
            if (e) return e;
            g_t5_smem_set[dev] = 1;
        }
    }
    // whole units on demand once there are many more units than CTAs (the tail is then a
    // small part of every CTA's work), else stream-K
    const int dyn = (long long)n_units >= TC_DYN_UNITS_PER_CTA * (long long)grid ? 1 : 0;
    prof_before(s);
    e = engine == ENGINE_TC5
            ? launch_pdl(k_tcpass5, grid, T5_THREADS, T5_SMEM, s, w, stall, dyn)
            : launch_pdl(k_tcpass, grid, TC_THREADS, 0, s, w, stall, dyn);
    prof_after(s);
    count_launch();
    if (e) return e;
    // with stream-K and more than one CTA a unit can be split between CTAs; the merge launch
    // (one CTA per possible unit) finds the split ones on the device, where the live chunk
    // count is known
    (void)total_chunks;
    if (!dyn && grid > 1 && n_units > 0) {
        e = launch_pdl(k_tcmerge, n_units, TC_THREADS, 0, s, w, grid);
        count_launch();
        if (e) return e;
    }
    const int total = rows + (mode == DC_BIDIR_MEAN ? cols : 0);
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // one wave of the recovery: its CTAs take equal ranges of row steps
    if (dev >= 0 && dev < 64 && g_rec_ctas[dev] == 0) {
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_tcrecover, REC_THREADS, 0) !=
                cudaSuccess ||
            occ <= 0)
            occ = 4;
        g_rec_ctas[dev] = occ * (sms > 0 ? sms : 1);
    }
    const int steps = div_up(total, REC_THREADS);
    const int rgrid =
        std::min(steps, dev >= 0 && dev < 64 ? g_rec_ctas[dev] : 4 * std::max(sms, 1));
    e = launch_pdl(k_tcrecover, rgrid, REC_THREADS, 0, s, w, rows, total);
    count_launch();
    if (e) return e;
    const int split = std::max(FB_SPLIT, std::min(FB_SPLIT_MAX, div_up(4 * std::max(sms, 1),
                                                                     2 * n_frames)));
    e = launch_pdl(k_tcfallback, 2 * n_frames * split, FB_THREADS, 0, s, w, rows, split);
    count_launch();
    return e ? e : cudaGetLastError();
}

}  // namespace dc
