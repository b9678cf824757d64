// The coverage count of one tile (warp-level), used by the count pass and
// by the fused count-and-fill pass of predicted capacities.
#pragma once
#include "raster_tiles.cuh"

namespace hexfc {

// Per tile: coverage of every chunk of 32 triangles as per-pixel bit masks;
// the masks are kept for the fill pass and their bit counts are the
// per-pixel list lengths. Warp w takes chunks w, w + 8, ... of the tile's list
// on its own: its 32 lanes stage the chunk's triangles, then take the
// triangles' box rows (clipped to the tile) one per lane: a triangle covers
// one run of samples in a row, found from its three edges' crossings of the
// row, and the lane sets bit j of those pixels in the warp's private masks.
// No block barrier until the per-pixel totals are summed at the end.
struct CountWarp {
    CovSoA c;
    // per edge, float data of its crossing with a sample row: (e0f, fb, rfa,
    // eps). The edge value at box column rx of row ry is E = e0f + fb*ry +
    // fa*rx (fa = -256 dy, fb = 256 dx, e0f ~ e0), so it crosses 0 at column
    // t = -(e0f + fb*ry) * rfa, rfa = 1 / fa; eps bounds |t - t_exact|. An
    // edge parallel to the rows (dy = 0) has rfa = 0 and eps = the bound on
    // the float error of its (constant) value.
    float4 ef[3][kChunk];
    // the chunk's rows as one sequence: triangle j's rows start at seq[j].x
    // (seq[j] = start, -, box, -); r2j maps the rank of a non-empty triangle
    // to its index
    uint4 seq[kChunk];
    uint8_t r2j[kChunk];
    uint32_t mask[kTilePix];   // coverage bits of the chunk; after the last chunk, the warp's per-pixel counts
};

// Float crossing data of triangle j's edges in the warp's staging slot. e0f
// is within 0.75 ulp of e0 and fmaf(fb, ry, e0f) adds one rounding, all of
// magnitudes at most M = |e0| + TW |fa| + TH |fb| (tile TW x TH): within
// tol = 8 units of 2^-24 M of the exact value. Dividing by fa (rfa within 0.5
// ulp, one more rounding of t) moves t by at most tol |rfa| + 2^-22 |t|, and
// |t| <= TW + 1 wherever it matters (columns 0..TW-1): eps = tol |rfa|
// (1 + 2^-10) + 2^-17 for TW <= 16 (17 * 2^-22 < 2^-17), + 2^-16 for TW = 32.
__device__ __forceinline__ void stage_rows(const CovSoA& c, float4 (*ef)[kChunk], int j)
{
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float e0 = i64_to_f32(c.e0[k][j]);
        const float fa = -256.f * (float)c.dy[k][j];   // exact: |dy| < 2^24
        const float fb = 256.f * (float)c.dx[k][j];
        const float tol = ldexpf(fabsf(e0) + (float)kTileW * fabsf(fa) + (float)kTileH * fabsf(fb), -21);
        const float rfa = fa != 0.f ? __frcp_rn(fa) : 0.f;
        constexpr float kTabs = kTileW <= 16 ? 0x1p-17f : 0x1p-16f;
        const float eps = fa != 0.f ? fmaf(tol * fabsf(rfa), 1.f + 0x1p-10f, kTabs) : tol;
        ef[k][j] = make_float4(e0, fb, rfa, eps);
    }
}

// Exact: does edge k of triangle j own box column rx of the row whose edge
// value at column 0 is A (edge function > 0, or 0 on an edge the top-left rule
// gives to the triangle)?
__device__ __forceinline__ bool edge_in(const CovSoA& c, int k, int j, int64_t A, int rx)
{
    const int64_t e = A - (int64_t)c.dy[k][j] * (int64_t)(rx << 8);
    return e > 0 || (e == 0 && ((c.meta[j] >> k) & 1u));
}

// The covered box columns [lo, hi] of box row ry of triangle j (empty if lo >
// hi): the intersection of its three edges' half-rows. Each edge's crossing
// is taken from the float data where it is more than eps from an integer
// column; near one (or if eps is not small), the column is decided by exact
// integer tests (a binary search on the monotone edge test).
__device__ __forceinline__ void row_span(const CovSoA& c, const float4 (*ef)[kChunk], int j, int ry, int bw, int& lo,
                                         int& hi)
{
    lo = 0;
    hi = bw - 1;
    const float fry = (float)ry;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float4 f = ef[k][j];
        const float af = fmaf(f.y, fry, f.x);   // edge value at column 0
        if (f.z == 0.f) {   // parallel to the rows: the whole row or nothing
            bool in = af > f.w;
            if (!in && af >= -f.w)
                in = edge_in(c, k, j, c.e0[k][j] + (int64_t)c.dx[k][j] * (int64_t)(ry << 8), 0);
            if (!in) hi = -1;
            continue;
        }
        const float t = -af * f.z;
        const float rt = rintf(t);
        const bool exact = f.w > 0.25f || (fabsf(t - rt) <= f.w && rt >= 0.f && rt <= (float)(bw - 1));
        int b;
        if (!exact) {
            const float ft = floorf(t);
            b = f.z > 0.f ? (int)fminf(fmaxf(ft + 1.f, 0.f), (float)bw)     // first column inside
                          : (int)fminf(fmaxf(ft, -1.f), (float)(bw - 1));   // last column inside
        } else {
            const int64_t A = c.e0[k][j] + (int64_t)c.dx[k][j] * (int64_t)(ry << 8);
            if (f.z > 0.f) {   // inside from the first column that passes: search [0, bw]
                int a = 0, z = bw;
                while (a < z) {
                    const int m = (a + z) >> 1;
                    if (edge_in(c, k, j, A, m)) z = m;
                    else a = m + 1;
                }
                b = a;
            } else {           // inside up to the last column that passes: search [-1, bw - 1]
                int a = -1, z = bw - 1;
                while (a < z) {
                    const int m = (a + z + 1) >> 1;
                    if (edge_in(c, k, j, A, m)) a = m;
                    else z = m - 1;
                }
                b = a;
            }
        }
        if (f.z > 0.f) lo = max(lo, b);
        else hi = min(hi, b);
    }
}

__device__ __forceinline__ void count_chunks(CountWarp* s_w, int warp, int lane, const uint32_t* __restrict__ bins,
                                             const FaceFrame* __restrict__ fframe, uint64_t beg, uint32_t n_chunks,
                                             int px0, int py0, int W, int H, uint32_t* __restrict__ masks)
{
    CountWarp& me = s_w[warp];
    uint32_t count[kTilePix / 32];   // pixels lane + 32 k
#pragma unroll
    for (int k = 0; k < kTilePix / 32; ++k) {
        me.mask[lane + 32 * k] = 0;
        count[k] = 0;
    }
    __syncwarp();
    uint32_t f2t = warp < (int)n_chunks ? bins[beg + (uint64_t)warp * kChunk + lane] : kPadBin;
    for (uint32_t c = warp; c < n_chunks; c += kConsumerWarps) {
        int4 a = make_int4(0, 0, 0, 0), b = a;
        if (f2t != kPadBin) { a = fframe[f2t >> 1].X; b = fframe[f2t >> 1].Y; }
        const uint32_t f2t_next =
            c + kConsumerWarps < n_chunks ? bins[beg + (uint64_t)(c + kConsumerWarps) * kChunk + lane] : kPadBin;
        if (f2t != kPadBin) {
            TriGeom t;
            stage_cov(a, b, f2t, W, H, px0, py0, me.c, lane, t);
            if (me.c.box[lane] != 0) stage_rows(me.c, me.ef, lane);
        } else {
            me.c.box[lane] = 0;
        }
        f2t = f2t_next;
        // the box rows of the chunk's 32 triangles as one sequence, so that
        // every round gives each lane a row whatever the boxes' sizes
        const int bx_l = me.c.box[lane];
        const uint32_t rows_l = (uint32_t)box_bh(bx_l);
        uint32_t incl = rows_l;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const uint32_t start_l = incl - rows_l, total = __shfl_sync(0xffffffffu, incl, 31);
        const unsigned nonempty = __ballot_sync(0xffffffffu, rows_l != 0);
        me.seq[lane] = make_uint4(start_l, 0u, (uint32_t)bx_l, 0u);
        if (rows_l) me.r2j[__popc(nonempty & ((1u << lane) - 1u))] = (uint8_t)lane;
        __syncwarp();
        for (uint32_t g = 0; g < total; g += 32) {
            // triangles starting in [g, g + 32) (bit = offset) and those before g
            const bool starts = rows_l != 0 && start_l >= g && start_l < g + 32;
            const uint32_t smask = __reduce_or_sync(0xffffffffu, starts ? 1u << (start_l - g) : 0u);
            const int before = __popc(__ballot_sync(0xffffffffu, rows_l != 0 && start_l < g));
            const uint32_t idx = g + (uint32_t)lane;
            if (idx < total) {
                const int c = __popc(smask & (0xffffffffu >> (31 - lane)));   // starts in [g, idx]
                const int j = me.r2j[c > 0 ? before + c - 1 : before - 1];
                const uint4 sq = me.seq[j];
                const int bx = (int)sq.z;
                const int ry = (int)(idx - sq.x);
                int lo, hi;
                row_span(me.c, me.ef, j, ry, box_bw(bx), lo, hi);
                uint32_t* mrow = &me.mask[(box_ly0(bx) + ry) * kTileW + box_lx0(bx)];
                for (int rx = lo; rx <= hi; ++rx) atomicOr(mrow + rx, 1u << j);
            }
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k < kTilePix / 32; ++k) {
            const int i = lane + 32 * k;
            const uint32_t m = me.mask[i];
            me.mask[i] = 0;
            masks[(beg / kChunk + c) * kTilePix + i] = m;
            count[k] += __popc(m);
        }
        __syncwarp();
    }
#pragma unroll
    for (int k = 0; k < kTilePix / 32; ++k) me.mask[lane + 32 * k] = count[k];
}

}  // namespace hexfc
