// Host-side check of the tensor-core forms' layout maps (dc_internal.cuh), compiled and run
// by tests/test_layout.py without a GPU. Exits 0 when every property holds, else prints the
// first violation and exits 1.
//
// The pass, the recovery and the staging kernels rely on these properties:
//  1. tc_form_pos is a bijection of every block of TC_BLOCK form indices onto itself;
//  2. the positions an MMA quad lane t sees in a block (8 g + 2 t + e, g < 16, e < 2) hold
//     the 32 consecutive points 32 t .. 32 t + 31 of the block (the recovery's candidate
//     quarter);
//  3. tc_stage_point is an involution of every block, and the 32 slots of each staging warp
//     write the forms of 32 consecutive positions (whole groups of 8) from four runs of 8
//     consecutive points.
#include <cstdio>
#include <set>

#include "../paper_2204_03139_gb300/csrc/dc_internal.cuh"

using dc::TC_BLOCK;
using dc::tc_form_pos;
using dc::tc_stage_point;

static int fail(const char* what, long long a, long long b) {
    std::printf("FAIL %s (%lld, %lld)\n", what, a, b);
    return 1;
}

int main() {
    static_assert(TC_BLOCK == 128, "the checks below assume blocks of 128");
    // form indices of several blocks, including one far into the array (rows + columns of a
    // large batch)
    const long long bases[] = {0, 128, 256 * 1000, 3LL * 128 * 4096 * 40};
    for (long long base : bases) {
        std::set<long long> seen;
        for (int b = 0; b < TC_BLOCK; ++b) {
            const long long p = tc_form_pos(base + b);
            if (p < base || p >= base + TC_BLOCK)
                return fail("form position leaves the block", base, b);
            seen.insert(p);
        }
        if ((int)seen.size() != TC_BLOCK)
            return fail("form positions collide", base, (long long)seen.size());
        // 2: the quad lane t of the m16n8k16 accumulator sees positions 8 g + 2 t + e
        for (int t = 0; t < 4; ++t) {
            std::set<long long> pts;
            for (int b = 0; b < TC_BLOCK; ++b)
                if (((tc_form_pos(base + b) - base) >> 1 & 3) == t) pts.insert(b);
            if ((int)pts.size() != 32) return fail("quarter size", base, t);
            if (*pts.begin() != 32 * t || *pts.rbegin() != 32 * t + 31)
                return fail("quarter is not 32 consecutive points", base, t);
        }
        // 3: the staging order (slot indices are ints: rows or columns of one call)
        const int b0 = (int)base;
        for (int s = 0; s < TC_BLOCK; ++s) {
            const int sp = tc_stage_point(b0 + s);
            if (tc_stage_point(sp) != b0 + s) return fail("staging order is not an involution", base, s);
            if ((sp & ~(TC_BLOCK - 1)) != b0) return fail("staging order leaves the block", base, s);
        }
        for (int w = 0; w < TC_BLOCK / 32; ++w) {
            std::set<long long> pos;
            std::set<int> runs;
            for (int l = 0; l < 32; ++l) {
                const int pt = tc_stage_point(b0 + 32 * w + l);
                pos.insert(tc_form_pos(pt) - b0);
                runs.insert((pt - b0) >> 3);
                // lanes 8 r .. 8 r + 7 take consecutive points
                if (l % 8 && pt != tc_stage_point(b0 + 32 * w + l - 1) + 1)
                    return fail("a run of 8 is not consecutive", w, l);
            }
            if ((int)pos.size() != 32 || *pos.begin() != 32 * w || *pos.rbegin() != 32 * w + 31)
                return fail("a staging warp's forms are not 32 consecutive positions", base, w);
            if ((int)runs.size() != 4) return fail("a staging warp's points are not 4 runs of 8", base, w);
        }
    }
    std::printf("ok\n");
    return 0;
}
