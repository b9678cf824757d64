// Per-tile rasterisation shared by the count and fill passes: exact
// coverage data of a chunk of triangles, and the producer/consumer ring of
// the fill pipeline.
#pragma once
#include "pipeline.cuh"
#include "raster_common.cuh"

namespace hexfc {

// ------------------------------------------------------------------ raster per tile

// Coverage data of the kChunk triangles of one chunk (structure of arrays):
// each triangle's three edge functions at the first sample of its box
// (clipped to the tile) and the edge vectors that step them, exact.
struct CovSoA {
    int64_t e0[3][kChunk];          // edge function opposite vertex k at the box origin sample
    int32_t dx[3][kChunk], dy[3][kChunk];  // edge vector (b - a) of that edge, 16.8
    uint32_t meta[kChunk];          // bit k: top-left rule owns edge k
    int32_t box[kChunk];            // lx0 | ly0 << 8 | bw << 16 | bh << 24 (tile-local); bw = bh = 0: misses the tile
};

__device__ __forceinline__ int box_lx0(int b) { return b & 255; }
__device__ __forceinline__ int box_ly0(int b) { return (b >> 8) & 255; }
__device__ __forceinline__ int box_bw(int b) { return (b >> 16) & 255; }
__device__ __forceinline__ int box_bh(int b) { return (b >> 24) & 255; }

__device__ __forceinline__ void stage_cov(int4 a, int4 b, uint32_t f2t, int W, int H, int px0, int py0, CovSoA& c,
                                          int j, TriGeom& t)
{
    int32_t X[4] = {a.x, a.y, a.z, a.w}, Y[4] = {b.x, b.y, b.z, b.w};
    tri_setup(X, Y, (int)(f2t & 1), W, H, t);
    int x0 = max(t.bx0, px0), x1 = min(t.bx1, px0 + kTileW - 1);
    int y0 = max(t.by0, py0), y1 = min(t.by1, py0 + kTileH - 1);
    if (!t.valid || x0 > x1 || y0 > y1) {
        c.box[j] = 0;
        return;
    }
    const int32_t sx = 256 * x0 + 128, sy = 256 * y0 + 128;
    uint32_t meta = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        int ia = (k + 1) % 3, ib = (k + 2) % 3;
        c.e0[k][j] = edge_fn(t.X[ia], t.Y[ia], t.X[ib], t.Y[ib], sx, sy);
        c.dx[k][j] = t.X[ib] - t.X[ia];
        c.dy[k][j] = t.Y[ib] - t.Y[ia];
        meta |= (top_left(t.X[ia], t.Y[ia], t.X[ib], t.Y[ib]) ? 1u : 0u) << k;
    }
    c.meta[j] = meta;
    c.box[j] = (x0 - px0) | ((y0 - py0) << 8) | ((x1 - x0 + 1) << 16) | ((y1 - y0 + 1) << 24);
}

// ------------------------------------------------------------------ tile passes
//
// k_fill runs one block per tile as a pipeline: a producer warp stages each
// chunk of 32 triangles of the tile's (depth-ordered) list into a ring of
// kRing slots in shared memory, while the eight consumer warps shade the
// covered samples of earlier chunks. Slots are handed over with mbarriers
// (full: the 32 producer lanes arrive; empty: lane 0 of each consumer warp
// arrives once no sample in its warp's queue refers to the slot), so the
// producer runs up to kRing chunks ahead. Every wait is bounded; a wait that runs out sets an error bit
// and ends the kernel's loops.

constexpr int kRing = 6;
constexpr int kConsumerWarps = kTilePix / 32;
constexpr int kPipeThreads = kTilePix + 32;
constexpr unsigned long long kErrWait = 4ull;

__device__ __forceinline__ void pipe_init(uint64_t* full, uint64_t* empty)
{
    if (threadIdx.x == 0) {
        for (int s = 0; s < kRing; ++s) {
            mbar_init(&full[s], 32);
            mbar_init(&empty[s], kConsumerWarps);   // lane 0 of each consumer warp
        }
        mbar_init_fence();
    }
    __syncthreads();
}

}  // namespace hexfc
