// Tensor-core filter of the brute-force nearest-neighbour search (Eq. 1, Eq. 2).
//
// Every row point (the sim points, and in Eq. 1 also the targets) is compared with every
// column point of its frame (the targets, respectively the sim points) through the
// expanded form |p - q|^2 = |p|^2 - 2 p.q + |q|^2, evaluated on the tensor cores with the
// split-fp16 forms that the staging kernel wrote (dc_internal.cuh): one m16n8k16 MMA gives
// 16 rows x 8 columns of approximate scaled squared distances. Each of the four lanes that
// share a row sees a quarter of every block's columns (2 of every 8); per row and lane the
// filter keeps the three smallest block keys (approximate minimum over the lane's columns of
// a block of TC_BLOCK, truncated, with the block); it never decides a neighbour. The
// epilogue
// re-evaluates the candidate blocks those keys admit in the exact float32 direct form of
// the oracle, so neighbours and losses are those of the direct form.
//
// Work: units of TC_UNIT_ROWS rows of one side of one frame, times their chunks of
// TC_CHUNK columns, flattened and split evenly over a persistent grid (every CTA gets the
// same number of chunks). A unit covered by one CTA writes its rows' keys to their final
// place; a unit split between CTAs writes each CTA's list to that CTA's slot in kpart
// (slot 0 for the part a CTA started inside the unit, 1 for the part that ends the CTA's
// range), and the epilogue merges them.
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
    int rows_live;   // rows of the unit that exist (padded rows included), from its first
    int c_lo, c_hi;  // chunk range of this segment
    int whole, slot;
};

constexpr int TC_THREADS = 32 * TC_WARPS;
constexpr int TC_MIN_BLOCKS = 3;  // 12 warps per SM

__global__ void __launch_bounds__(TC_THREADS, TC_MIN_BLOCKS) k_tcpass(Ws w, int stall) {
    pdl_entry();
    constexpr uint32_t CH_BYTES = TC_CHUNK * 32;  // B forms of one chunk
    __shared__ __align__(128) unsigned s_b[2][CH_BYTES / 4];
    __shared__ __align__(8) u64 s_bar[2];
    __shared__ TcSeg s_u;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int n_units = w.hdr->tc_units, total = w.hdr->tc_total;
    const int per = (total + gridDim.x - 1) / gridDim.x;
    int s = blockIdx.x * per;
    const int s_end = min(total, s + per);
    if (s >= s_end) return;
    int u = last_le(w.tc_upre, n_units, s);
    const long long tot_rows = w.hdr->total_rows;

    if (tid == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    uint32_t par = 0;      // bit b: the phase parity to wait for on buffer b
    uint32_t pending = 0;  // bit b: a copy into buffer b is in flight (thread 0)
    int seq = 0;           // chunks consumed so far; buffer = seq & 1
    bool abort = false;
    const unsigned* A32 = reinterpret_cast<const unsigned*>(w.tca);

    while (s < s_end) {
        __syncthreads();  // the previous segment is done with s_u and the buffers' contents
        if (tid == 0) {
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
            // stage the first two chunks of the segment (both buffers are free here)
            for (int c = s_u.c_lo; c <= min(s_u.c_hi, s_u.c_lo + 1); ++c) {
                const int b = (seq + c - s_u.c_lo) & 1;
                // test of the bounded waits: the first chunk is never requested
                if (stall && seq == 0 && c == s_u.c_lo) continue;
                mbar_expect_tx(&s_bar[b], CH_BYTES);
                bulk_g2s(&s_b[b][0], w.tcb + 2 * (s_u.bcol + (long long)c * TC_CHUNK), CH_BYTES,
                         &s_bar[b]);
                pending |= 1u << b;
            }
        }
        __syncthreads();
        const int wrow0 = warp * TC_ROWS_PER_WARP;  // within the unit
        // a frame's padded row count is a multiple of 256, so a warp's 128 rows are all
        // inside it or all beyond it (units of 512 rows may overhang the target side)
        const bool wactive = wrow0 < s_u.rows_live;

        // this warp's eight m16 tiles of A forms, in registers for the whole segment
        unsigned a[8][4];
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const long long p = wactive ? s_u.arow + wrow0 + 16 * m : 0;
            const long long G = p >> 3;  // first of the tile's two groups of 8 rows
            a[m][0] = A32[G * 64 + g * 4 + t];
            a[m][1] = A32[(G + 1) * 64 + g * 4 + t];
            a[m][2] = A32[G * 64 + 32 + g * 4 + t];
            a[m][3] = A32[(G + 1) * 64 + 32 + g * 4 + t];
        }
        unsigned k1[16], k2[16], k3[16];  // rows 16 m + g (2 m) and 16 m + g + 8 (2 m + 1)
#pragma unroll
        for (int r = 0; r < 16; ++r) k1[r] = k2[r] = k3[r] = TC_EMPTY;

        const int c_lo = s_u.c_lo, c_hi = s_u.c_hi;
        for (int c = c_lo; c <= c_hi; ++c, ++seq) {
            const int b = seq & 1;
            // every lane of a warp must agree before the warp-wide MMAs
            const bool ok = __all_sync(0xffffffffu, mbar_wait(&s_bar[b], (par >> b) & 1u));
            if (ok) par ^= 1u << b;
            if (ok && wactive) {
                const unsigned* S = s_b[b];
#pragma unroll 1
                for (int half = 0; half < TC_CHUNK / TC_BLOCK; ++half) {
                    float bm[16];
#pragma unroll
                    for (int nt = 0; nt < TC_BLOCK / 8; ++nt) {
                        const int grp = half * (TC_BLOCK / 8) + nt;  // group of 8 columns
                        const unsigned b0 = S[grp * 64 + g * 4 + t];
                        const unsigned b1 = S[grp * 64 + 32 + g * 4 + t];
#pragma unroll
                        for (int m = 0; m < 8; ++m) {
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
                    for (int r = 0; r < 16; ++r)
                        top3_insert(k1[r], k2[r], k3[r],
                                    (__float_as_uint(fmaxf(bm[r], 0.0f)) & TC_VALUE_MASK) | id);
                }
            }
            abort = __syncthreads_or(!ok) != 0;
            if (abort) break;
            if (tid == 0) {
                pending &= ~(1u << b);
                // buffer b is free again: stage chunk c + 2 into it
                if (c + 2 <= c_hi) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    mbar_expect_tx(&s_bar[b], CH_BYTES);
                    bulk_g2s(&s_b[b][0], w.tcb + 2 * (s_u.bcol + (long long)(c + 2) * TC_CHUNK),
                             CH_BYTES, &s_bar[b]);
                    pending |= 1u << b;
                }
            }
        }
        if (abort) break;
        if (wactive) {
            // every lane keeps its own column subset's three smallest keys: [row][lane t][3]
            unsigned* out = s_u.whole
                                ? s_u.kout
                                : w.kpart + TC_KEYS * ((2LL * blockIdx.x + s_u.slot) * TC_UNIT_ROWS);
#pragma unroll
            for (int r = 0; r < 16; ++r) {
                const int ru = wrow0 + 16 * (r >> 1) + g + 8 * (r & 1);
                unsigned* o = out + TC_KEYS * ru + 3 * t;
                o[0] = k1[r];
                o[1] = k2[r];
                o[2] = k3[r];
            }
        }
        s = min(s_end, w.tc_upre[u + 1]);
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
    const int rows = min(TC_UNIT_ROWS, (side ? fr->Mpad : fr->Npad) - (int)first);
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

constexpr int REC_THREADS = 256;  // 64 rows per CTA step, four lanes per row

// The rows' exact minima from their keys: rows [0, rows) are sim points, rows
// [rows, total) targets (Eq. 1 only). Each CTA takes a contiguous range of rows, 64 at a time
// (frames are padded to multiples of 256 rows, so a step's 64 rows lie in one frame, found
// by walking the frame table forward). The four lanes of a row read the keys of their
// quarter of the columns, agree on the threshold and scan, eight columns each, the candidate
// blocks that any of them admits; the groups of a warp take their candidates in the same
// order (the s-th of each group in step s), so that the warp runs the largest count, not the
// sum. A row that the keys do not certify (a lane's third key under the threshold) is
// queued in its frame's list for k_tcfallback. Writes (distance bits << 32 | index) to
// pab / pba.
__global__ void __launch_bounds__(REC_THREADS) k_tcrecover(Ws w, int rows, int total) {
    pdl_entry();
    constexpr int NW = REC_THREADS / 32;
    __shared__ float s_q[NW][8][4];       // per warp: the query point of each row group
    __shared__ unsigned s_list[NW][64];   // per warp: candidate entries (cand << 3 | group)
    __shared__ u64 s_best[NW][8];         // per warp: the rows' packed minima
    const int steps = div_up(total, REC_THREADS / 4);
    const int per = div_up(steps, gridDim.x);
    const int st0 = blockIdx.x * per, st1 = min(steps, st0 + per);
    const int n_frames = w.hdr->n_frames;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, q = lane & 3, gl = lane & ~3;
    const int grp = lane >> 2, sub = lane >> 3, l8 = lane & 7;
    const unsigned lt = (1u << lane) - 1u;
    int k = -1, side = -1;
    for (int st = st0; st < st1; ++st) {
        const int base = st * (REC_THREADS / 4);
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
        const int g = g0 + (threadIdx.x >> 2);
        const int i = g - (side ? fr->col0 : fr->row0);
        const bool valid = i < (side ? fr->M : fr->N);
        const Cols C = frame_cols(w, fr, side);
        const float4 box = w.fbox[k];

        unsigned kk[3] = {TC_EMPTY, TC_EMPTY, TC_EMPTY};
        float qx = 0.f, qy = 0.f, qz = 0.f, r = 0.f;
        if (valid) {
            const unsigned* p =
                (side ? w.kba + (long long)TC_KEYS * g : w.kab + (long long)TC_KEYS * g) + 3 * q;
            kk[0] = p[0];
            kk[1] = p[1];
            kk[2] = p[2];
            const float3 x = frame_row(w, fr, side, i);
            qx = x.x, qy = x.y, qz = x.z;
            const float sx = __fmul_rn(__fsub_rn(qx, box.x), box.w);
            const float sy = __fmul_rn(__fsub_rn(qy, box.y), box.w);
            const float sz = __fmul_rn(__fsub_rn(qz, box.z), box.w);
            r = sqrtf(__fmaf_rn(sz, sz, __fmaf_rn(sy, sy, __fmul_rn(sx, sx)))) *
                (1.0f + 0x1p-20f);
        }
        unsigned kmin = kk[0];
        kmin = min(kmin, (unsigned)__shfl_xor_sync(0xffffffffu, kmin, 1));
        kmin = min(kmin, (unsigned)__shfl_xor_sync(0xffffffffu, kmin, 2));
        unsigned c0 = TC_EMPTY, c1 = TC_EMPTY;
        bool open = valid;  // this lane's quarter may hide a candidate beyond its keys
        if (valid && kmin != TC_EMPTY) {
            const float tau = tc_tau(kmin, r);
            // candidates as (block << 2 | the pass's lane whose columns they name)
            if (kk[0] != TC_EMPTY && key_value(kk[0]) <= tau)
                c0 = ((kk[0] & ~TC_VALUE_MASK) << 2) | (unsigned)q;
            if (kk[1] != TC_EMPTY && key_value(kk[1]) <= tau)
                c1 = ((kk[1] & ~TC_VALUE_MASK) << 2) | (unsigned)q;
            open = kk[2] != TC_EMPTY && key_value(kk[2]) <= tau;
        }
        const bool full = ((__ballot_sync(0xffffffffu, open) >> gl) & 0xFu) != 0u;
        // the warp's (row, candidate block) entries, in any order: each is scanned by eight
        // lanes and merged into its row's minimum
        const bool use = valid && !full;
        const unsigned b0 = __ballot_sync(0xffffffffu, use && c0 != TC_EMPTY);
        const unsigned b1 = __ballot_sync(0xffffffffu, use && c1 != TC_EMPTY);
        const int n0 = __popc(b0), tot = n0 + __popc(b1);
        if (q == 0) {
            s_q[warp][grp][0] = qx;
            s_q[warp][grp][1] = qy;
            s_q[warp][grp][2] = qz;
            s_best[warp][grp] = EMPTY;
        }
        if (use && c0 != TC_EMPTY) s_list[warp][__popc(b0 & lt)] = (c0 << 3) | (unsigned)grp;
        if (use && c1 != TC_EMPTY)
            s_list[warp][n0 + __popc(b1 & lt)] = (c1 << 3) | (unsigned)grp;
        __syncwarp();
        for (int e0 = 0; e0 < tot; e0 += 4) {
            const int e = e0 + sub;
            float bd = INFINITY;
            int bj = 0x7fffffff, eg = -1;
            if (e < tot) {
                const unsigned ent = s_list[warp][e];
                eg = (int)(ent & 7u);
                const unsigned c = ent >> 3;
                const int blk = (int)(c >> 2), tq = (int)(c & 3u);
                const float ex = s_q[warp][eg][0], ey = s_q[warp][eg][1], ez = s_q[warp][eg][2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    // the block's columns that the pass's lane tq saw: 2 of every group of 8;
                    // this lane takes groups l8 and l8 + 8, in increasing column order
                    const int j0 = blk * TC_BLOCK + 8 * (l8 + 8 * h) + 2 * tq;
                    if (j0 >= C.n) continue;
                    float ax, ay, az, bx, by, bz;
                    if (C.P) {
                        const float4 p0 = C.P[j0], p1 = C.P[j0 + 1];
                        ax = p0.x, ay = p0.y, az = p0.z, bx = p1.x, by = p1.y, bz = p1.z;
                    } else {  // j0 is even and the planes are 8-byte aligned
                        const float2 X = *reinterpret_cast<const float2*>(C.X + j0);
                        const float2 Y = *reinterpret_cast<const float2*>(C.Y + j0);
                        const float2 Z = *reinterpret_cast<const float2*>(C.Z + j0);
                        ax = X.x, ay = Y.x, az = Z.x, bx = X.y, by = Y.y, bz = Z.y;
                    }
                    const float d0 = dist2(ex, ey, ez, ax, ay, az);
                    if (d0 < bd) bd = d0, bj = j0;
                    const float d1 = dist2(ex, ey, ez, bx, by, bz);
                    if (j0 + 1 < C.n && d1 < bd) bd = d1, bj = j0 + 1;
                }
            }
            u64 key = bj == 0x7fffffff ? EMPTY : pack_d(bd, bj);
            key = min64(key, __shfl_xor_sync(0xffffffffu, key, 1));
            key = min64(key, __shfl_xor_sync(0xffffffffu, key, 2));
            key = min64(key, __shfl_xor_sync(0xffffffffu, key, 4));
            if (l8 == 0 && eg >= 0) atomicMin(&s_best[warp][eg], key);
        }
        __syncwarp();
        if (valid && q == 0) {
            u64* out = side ? w.pba : w.pab;
            if (full) {
                out[g] = EMPTY;
                // the frame's list for this side: entries at its own row range
                const int slot = atomicAdd(&w.tcfn[2 * k + side], 1);
                w.tcfb[(side ? rows + fr->col0 : fr->row0) + slot] = i;
                atomicAdd(&w.hdr->tc_fallback, 1);
            } else {
                out[g] = s_best[warp][grp];
            }
        }
        __syncwarp();  // the next step reuses the warp's shared lists
    }
}

constexpr int FB_THREADS = 256;            // eight warps
constexpr int FB_ROWS_PER_WARP = 8;        // queued rows a warp evaluates at once
constexpr int FB_TILE = 512;               // columns per shared-memory tile
constexpr int FB_SPLIT = 4;                // CTAs per list, each over a quarter of the columns

// The rows that their keys did not certify, FB_SPLIT CTAs per (frame, side) list, each over
// a contiguous quarter of the frame's columns: they stream through shared memory in tiles,
// each loaded once for up to 64 queued rows (eight per warp, the lanes splitting the
// columns); the quarters' minima merge with atomicMin on (distance bits << 32 | index), so
// every row ends with its minimum and the lowest index attaining it.
__global__ void __launch_bounds__(FB_THREADS) k_tcfallback(Ws w, int rows) {
    pdl_entry();
    __shared__ float s_c[3][FB_TILE];
    const int part = blockIdx.x % FB_SPLIT, ks = blockIdx.x / FB_SPLIT;
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
        float qx[FB_ROWS_PER_WARP], qy[FB_ROWS_PER_WARP], qz[FB_ROWS_PER_WARP];
        u64 best[FB_ROWS_PER_WARP];
#pragma unroll
        for (int t = 0; t < FB_ROWS_PER_WARP; ++t) {
            const int e = r0 + warp * FB_ROWS_PER_WARP + t;
            const float3 x = frame_row(w, fr, side, e < n ? list[e] : list[0]);
            qx[t] = x.x, qy[t] = x.y, qz[t] = x.z;
            best[t] = EMPTY;
        }
        const int ja = (int)((long long)C.n * part / FB_SPLIT);
        const int jb = (int)((long long)C.n * (part + 1) / FB_SPLIT);
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
            const int jn = min(FB_TILE, jb - j0);
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

int g_tc_ctas[64];  // per device: resident CTAs of the persistent grid

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

cudaError_t launch_tcpass(const Ws& w, int grid, long long total_chunks, int n_units,
                          int rows, int cols, int mode, int n_frames, cudaStream_t s) {
    const int stall = take_stall();
    prof_before(s);
    cudaError_t e = launch_pdl(k_tcpass, grid, TC_THREADS, 0, s, w, stall);
    prof_after(s);
    count_launch();
    if (e) return e;
    // with more than one CTA a unit can be split between CTAs; the merge launch (one CTA per
    // possible unit) finds the split ones on the device, where the live chunk count is known
    (void)total_chunks;
    if (grid > 1 && n_units > 0) {
        e = launch_pdl(k_tcmerge, n_units, TC_THREADS, 0, s, w, grid);
        count_launch();
        if (e) return e;
    }
    const int total = rows + (mode == DC_BIDIR_MEAN ? cols : 0);
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int steps = div_up(total, REC_THREADS / 4);
    const int rgrid = std::min(steps, 8 * (sms > 0 ? sms : 1));
    e = launch_pdl(k_tcrecover, rgrid, REC_THREADS, 0, s, w, rows, total);
    count_launch();
    if (e) return e;
    e = launch_pdl(k_tcfallback, 2 * n_frames * FB_SPLIT, FB_THREADS, 0, s, w, rows);
    count_launch();
    return e ? e : cudaGetLastError();
}

}  // namespace dc
