// The coverage count of one tile (warp-level), used by the count pass and
// by the fused count-and-fill pass of predicted capacities.
#pragma once
#include "raster_tiles.cuh"

namespace hexfc {

// Per tile: coverage of every chunk of 32 triangles as per-pixel bit masks;
// the masks are kept for the fill pass and their bit counts are the
// per-pixel list lengths. Warp w takes chunks w, w + 8, ... of the tile's list
// on its own: its 32 lanes stage the chunk's triangles, then walk each
// triangle's box (clipped to the tile) one sample per lane, setting bit j of
// the covered pixels in the warp's private masks. No block barrier until the
// per-pixel totals are summed at the end.
struct CountWarp {
    CovSoA c;
    // float copies of the edge functions, (e0f, fa, fb, tol) per edge: E ~ e0f +
    // fa*rx + fb*ry, and a bound on the float error; outside the bound the
    // float sign is the exact sign (one 16-byte load per edge and sample)
    float4 ef[3][kChunk];
    // the chunk's samples as one sequence: triangle j's box samples start at
    // seq[j].x (seq[j] = start, 1 / box width, box); r2j maps the rank of a
    // non-empty triangle to its index
    uint4 seq[kChunk];
    uint8_t r2j[kChunk];
    uint32_t mask[kTilePix];   // coverage bits of the chunk; after the last chunk, the warp's per-pixel counts
};

// Float version of triangle j's edge functions in the warp's staging slot.
// e0f is within 0.75 ulp of e0 and the float evaluation fmaf(fa, rx,
// fmaf(fb, ry, e0f)) adds two roundings, all of magnitudes at most |e0| +
// 15 (|fa| + |fb|): at most 3.5 units of 2^-24 of that, and tol allows 8.
__device__ __forceinline__ void stage_fast(CountWarp& me, int j)
{
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float e0 = i64_to_f32(me.c.e0[k][j]);
        const float fa = -256.f * (float)me.c.dy[k][j];   // exact: |dy| < 2^24
        const float fb = 256.f * (float)me.c.dx[k][j];
        me.ef[k][j] = make_float4(e0, fa, fb, ldexpf(fabsf(e0) + 16.f * (fabsf(fa) + fabsf(fb)), -21));
    }
}

// Coverage of samples (rx, ry) and, if `second`, (rx + 1, ry) of triangle j
// (bits 0 and 1): decided in float when every edge value is outside its error
// bound (or one is clearly negative), else exactly. The two samples share the
// inner product fmaf(fb, ry, e0f), so each is evaluated as in the bound.
__device__ __forceinline__ uint32_t cover_pair(const CountWarp& me, int j, int rx, int ry, bool second)
{
    const float frx = (float)rx, fry = (float)ry;
    bool pos0 = true, neg0 = false, pos1 = true, neg1 = false;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float4 f = me.ef[k][j];
        const float inner = fmaf(f.z, fry, f.x);
        const float e0 = fmaf(f.y, frx, inner), e1 = fmaf(f.y, frx + 1.f, inner);
        pos0 = pos0 && e0 > f.w;
        neg0 = neg0 || e0 < -f.w;
        pos1 = pos1 && e1 > f.w;
        neg1 = neg1 || e1 < -f.w;
    }
    int64_t l[3];
    uint32_t r = 0;
    if (pos0 || (!neg0 && cover_at(me.c, j, rx, ry, l))) r |= 1u;
    if (second && (pos1 || (!neg1 && cover_at(me.c, j, rx + 1, ry, l)))) r |= 2u;
    return r;
}

// Warp `warp` of a tile block rasterises chunks warp, warp + kConsumerWarps, ...
// of the tile's list into masks (global, per chunk); its per-pixel counts are
// left in s_w[warp].mask.
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
            if (me.c.box[lane] != 0) stage_fast(me, lane);
        } else {
            me.c.box[lane] = 0;
        }
        f2t = f2t_next;
        // the box samples of the chunk's 32 triangles, in horizontal pairs, as
        // one sequence, so that every round gives each lane a pair whatever
        // the boxes' sizes
        const int bx_l = me.c.box[lane];
        const uint32_t pw_l = (uint32_t)(box_bw(bx_l) + 1) >> 1;   // pairs per box row
        const uint32_t area_l = pw_l * (uint32_t)box_bh(bx_l);
        uint32_t incl = area_l;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const uint32_t start_l = incl - area_l, total = __shfl_sync(0xffffffffu, incl, 31);
        const unsigned nonempty = __ballot_sync(0xffffffffu, area_l != 0);
        me.seq[lane] = make_uint4(start_l, __float_as_uint(area_l ? __frcp_rn((float)pw_l) : 0.f), (uint32_t)bx_l,
                                  pw_l);
        if (area_l) me.r2j[__popc(nonempty & ((1u << lane) - 1u))] = (uint8_t)lane;
        __syncwarp();
        for (uint32_t g = 0; g < total; g += 32) {
            // triangles starting in [g, g + 32) (bit = offset) and those before g
            const bool starts = area_l != 0 && start_l >= g && start_l < g + 32;
            const uint32_t smask = __reduce_or_sync(0xffffffffu, starts ? 1u << (start_l - g) : 0u);
            const int before = __popc(__ballot_sync(0xffffffffu, area_l != 0 && start_l < g));
            const uint32_t idx = g + (uint32_t)lane;
            if (idx < total) {
                const int c = __popc(smask & (0xffffffffu >> (31 - lane)));   // starts in [g, idx]
                const int j = me.r2j[c > 0 ? before + c - 1 : before - 1];
                const uint4 sq = me.seq[j];
                const int bx = (int)sq.z;
                const int off = (int)(idx - sq.x);
                // exact for off < 128, pairs per row <= 8: the quotient is never within 1/16 of an integer
                const int ry = (int)(((float)off + 0.5f) * __uint_as_float(sq.y));
                const int rx = 2 * (off - ry * (int)sq.w);
                const uint32_t cov = cover_pair(me, j, rx, ry, rx + 1 < box_bw(bx));
                uint32_t* mrow = &me.mask[(box_ly0(bx) + ry) * kTile + box_lx0(bx) + rx];
                if (cov & 1u) atomicOr(mrow, 1u << j);
                if (cov & 2u) atomicOr(mrow + 1, 1u << j);
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
