// Internal declarations of the hexfc CUDA library (not part of the C ABI).
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "hexfc.h"

namespace hexfc {

#ifndef HEXFC_TILE_W
#define HEXFC_TILE_W 16
#endif
constexpr int kTilePix = 256;                  // pixels (= threads) per tile CTA
constexpr int kTileW = HEXFC_TILE_W;           // raster tile width in pixels (a build-time choice)
constexpr int kTileH = kTilePix / kTileW;      // raster tile height
static_assert(kTileW == 8 || kTileW == 16 || kTileW == 32, "tiles of 8x32, 16x16 or 32x8 pixels");
constexpr int kWarpSortMax = 256;         // longest list sorted in registers by one warp
constexpr uint64_t kPadKey = ~0ull;
constexpr int kChunk = 32;                // triangles per raster chunk (one coverage bit each)
constexpr uint32_t kPadBin = 0xFFFFFFFFu; // empty slot: tile lists are padded to whole chunks

// Camera constants of the vertex stage (double, evaluated without FMA).
struct CamParams {
    double eye[3], R[3], U[3], F[3];
    double focal, scale, cx, cy, znear, zfar, zf_over;
    int ortho, W, H;   // W, H: size of the drawn rectangle (the frame's unless a sub-rectangle is drawn)
    int ox, oy;   // drawn rectangle's offset in the frame (pixels): window positions are shifted by it
};

// Focus+context constants of the fragment stage (float).
struct ShadeParams {
    int lens_mode;
    float lens_c[3];
    float lens_inv_r;
    float w_base;
    int lod;
    float delta, s;
    float alpha_min, alpha_span;   // alpha_hat = alpha_min + alpha_span * t
    float tf_lo, tf_inv;           // t = clamp((imp - tf_lo) * tf_inv, 0, 1)
    float bg[3];
    float accent_beta, halo_scale, darken, g_min, g_max;
    float zref;
    int ortho;
    float accent_r2;   // (256 * 2/3 * w_base)^2: accentuation radius squared, 1/256-pixel units
    float desat;       // depth cue strength (0 = off)
    int px_off, py_off;   // drawn rectangle's offset in the frame: pixel (x, y) is frame pixel (x + px_off, ...)
};

// A face as two 64-byte records: the per-frame one (window corners, depths,
// edge flags, eye depths), written by the face stage of every frame into the
// rendering context's buffers, and the static one (corner importance and world
// position), owned by the mesh and rewritten only when importance changes, so
// that contexts can render one resident mesh at the same time.
struct __align__(64) FaceFrame {
    int4 X, Y;            // corner window position, 16.8 fixed point
    uint4 Z;              // bits 0-23: corner window depth (z24); Z.x bits 24-31: edge flags
                          // (bits 0-3 visible in focus, 4-7 visible in context); Z.y bits 24-25:
                          // triangle 0 / 1 drawn, bit 26: a boundary face (of one cell)
    float4 ed;            // corner eye depth
};
struct __align__(64) FaceStatic {
    float4 imp;           // corner importance
    float4 px, py, pz;    // corner world position
};
static_assert(sizeof(FaceFrame) == 64 && sizeof(FaceStatic) == 64, "two sectors each");
constexpr uint32_t kZ24 = 0xFFFFFFu;

// Device scalars of a frame (FrameBufs::scal): 0-2 pixel scan (fragments,
// longest list, lists above the warp sort), 3-4 resolve queue cursors (long,
// out of order), 5 device error bits (kept across frames), 6 tiles above
// their chosen capacity, 8-10 tile scan (bin entries, ...), 11-13 capacity
// scan (regions' total, ...), 14 records taken from the pool, 16-18 count
// pass statistics (fragments, longest list, lists above the warp sort).
constexpr int kScal = 24;
// Copies of the count pass's frame statistics (fragments, longest list, long
// lists, unused), one per tile % kStatCopies, summed on the host: tiles
// adding into one address would queue on it.
constexpr int kStatCopies = 32;
__host__ __device__ inline uint32_t face_edge_flags(const uint4& z) { return z.x >> 24; }
__host__ __device__ inline uint32_t face_tris(const uint4& z) { return (z.y >> 24) & 3u; }
__host__ __device__ inline uint32_t face_boundary(const uint4& z) { return (z.y >> 26) & 1u; }
constexpr uint32_t kNoDepth = 0xFFFFFFFFu;   // no boundary fragment at a pixel

// Resident mesh (device pointers), see hexfc_upload_mesh.
struct DevMesh {
    int64_t n_verts = 0, n_cells = 0, n_faces = 0, n_edges = 0;
    float* verts = nullptr;        // [V*3]
    int32_t* cells = nullptr;      // [C*8]
    int32_t* cell_edges = nullptr; // [C*12] unique edge id per cell edge
    float* cell_imp = nullptr;     // [C]
    int32_t* vkey = nullptr;       // [V] ordered-int max of incident importance
    int32_t* ekey = nullptr;       // [E]
    float* vimp = nullptr;         // [V]
    float* eattr = nullptr;        // [E]
    uint8_t* elevel = nullptr;     // [E]
    int4* fverts = nullptr;        // [F] canonical corners
    int4* fedges = nullptr;        // [F] unique edge id of local edge k = (c_k, c_k+1)
    uint8_t* fbound = nullptr;     // [F] 1: a boundary face (one cell)
    FaceStatic* fstat = nullptr;   // [F] static face records
};

// Tile-capacity network (4 -> 64 -> 64 -> 1): FP32 master weights, the FP16
// copy the kernels use, Adam moments, and per-tile training values.
constexpr int kCapIn = 4, kCapHid = 64;
constexpr int kCapParams = kCapHid * kCapIn + kCapHid + kCapHid * kCapHid + kCapHid + kCapHid + 1;
struct CapNet {
    float* w = nullptr;
    __half* w16 = nullptr;
    float* m = nullptr;
    float* v = nullptr;
    float* grad = nullptr;        // [kCapParams + 1]; the last value is the loss
    float* h1 = nullptr;          // [tiles * kCapHid] layer values and errors of a training pass
    float* h2 = nullptr;
    float* da1 = nullptr;
    float* da2 = nullptr;
    float* dy = nullptr;          // [tiles]
    float* x = nullptr;           // [4 * tiles] features handed in by the caller
    uint32_t* t = nullptr;        // [tiles] counts handed in by the caller
    int64_t tiles = 0;            // capacity of the per-tile arrays
    int64_t step = 0;             // Adam steps taken
    bool ready = false;           // weights set
};

// Per-frame buffers owned by the context.
struct FrameBufs {
    // vertex stage
    int4* vproj = nullptr;   // {X, Y, z24, valid}
    float* ved = nullptr;    // eye depth
    int64_t v_cap = 0;
    // faces
    FaceFrame* fframe = nullptr;    // [F] per-frame face records
    uint32_t* tzsum = nullptr;      // [2F] per triangle (2 face + tri): sum of its window depths
    int64_t f_cap = 0;
    // tiles
    uint32_t* tile_cnt = nullptr;   // [T+1]
    uint64_t* tile_off = nullptr;   // [T+1]
    uint32_t* tile_cur = nullptr;   // [T]
    uint32_t* tile_order = nullptr; // [T] tiles by decreasing chunk count
    uint32_t* tile_frag = nullptr;  // [T] exact fragments per tile (the count's or the fused pass's)
    float* tile_zr = nullptr;       // [T] depth range of the tile's triangles (fraction of the z24 sum range)
    float* cap_x = nullptr;         // [4T] capacity-network features of the frame
    uint32_t* tile_cap = nullptr;   // [T+1] chosen fragment capacity per tile (predicted frames)
    uint64_t* cap_off = nullptr;    // [T+1] its exclusive prefix
    int64_t cap_cap = 0;
    int64_t t_cap = 0;
    uint32_t* bins = nullptr;       // face2tri ids grouped by tile, each tile padded to whole chunks
    uint32_t* bins_tmp = nullptr;   // scratch of the depth order of long tile lists (same layout)
    bool scal_fresh = false;        // scal just allocated (undefined contents)
    int64_t bin_cap = 0;
    uint32_t* masks = nullptr;      // per chunk of a tile list: 256 per-pixel coverage masks
    uint64_t* seg = nullptr;        // per chunk and warp group of 32 pixels: the first fragment of its records
    int64_t seg_cap = 0;
    int64_t mask_cap = 0;
    // pixels (tile-major)
    uint32_t* cnt = nullptr;        // [P]
    uint64_t* off = nullptr;        // [P]
    int64_t p_cap = 0;
    uint64_t* part = nullptr;       // scan partials
    uint32_t* part_max = nullptr;
    int64_t part_cap = 0;
    uint32_t* long_q = nullptr;     // queue of pixels with long lists
    uint32_t* fix_q = nullptr;      // queue of pixels whose list arrived out of order
    uint32_t* zsil = nullptr;       // [P] depth of the nearest boundary fragment (silhouettes), kNoDepth if none
    // fragments
    uint64_t* key = nullptr;
    float4* rgba = nullptr;
    int64_t frag_cap = 0;
    // small device scalars: [0] total fragments, [1] max list, [2] long lists, [3] long queue cursor,
    // [4] out-of-order queue cursor, [5] error bits (kept across frames), [8..10] tile scan totals
    uint64_t* scal = nullptr;       // kScal device scalars (slots: see kScal)
    uint64_t* cstat = nullptr;      // [4 * kStatCopies] count pass statistics (predicted frames)
    uint64_t* h_scal = nullptr;     // pinned mirror
};

// The pixels of the drawn rectangle that go to the output image: [x0, x0 + w) x
// [y0, y0 + h), written at out[(y - y0) w + (x - x0)] (the rest is an apron whose
// depths the silhouettes read).
struct OutWin {
    int x0, y0, w, h;
};

// ---- batched launches: the tiles of up to kBatchLaunchMax frames in one grid ------------
// Each block finds its frame from the frames' first tile (tile_begin, in the
// kernel's parameters) and takes that frame's tile in its tile order.
constexpr int kBatchLaunchMax = 64;
struct CountItem {
    const uint64_t* tile_off;
    const uint32_t* bins;
    const FaceFrame* fframe;
    const uint32_t* order;
    uint32_t* cnt;
    uint32_t* masks;
    uint32_t* tile_frag;
    int tiles_x, W, H;
};
struct CountBatch {
    CountItem it[kBatchLaunchMax];
    uint32_t tile_begin[kBatchLaunchMax + 1];
    int n;
};
struct FillItem {
    const uint64_t* tile_off;
    const uint32_t* bins;
    const uint32_t* masks;
    const FaceFrame* fframe;
    const FaceStatic* fstat;
    const uint32_t* order;
    const uint64_t* off;
    const uint32_t* cnt;
    uint64_t* key;
    float4* rgba;
    uint64_t* seg;
    unsigned long long* err;
    uint32_t* zsil;   // nullptr: no silhouettes
    ShadeParams sp;
    int tiles_x, W, H;
};
struct FillBatch {
    FillItem it[kBatchLaunchMax];
    uint32_t tile_begin[kBatchLaunchMax + 1];
    int n;
};
struct CompositeItem {
    const uint32_t* cnt;
    const uint64_t* seg;
    const uint64_t* tile_off;
    const uint32_t* masks;
    const uint64_t* key;
    const float4* rgba;
    float4* out;
    uint32_t* long_q;
    unsigned long long* long_cursor;
    uint32_t* fix_q;
    unsigned long long* fix_cursor;
    uint64_t frag_cap;
    float bg[3];
    OutWin win;
    int tiles_x, W, H;
};
struct CompositeBatch {
    CompositeItem it[kBatchLaunchMax];
    uint32_t tile_begin[kBatchLaunchMax + 1];
    int n;
};
// The frame of block b in a batched launch: the last with begin[i] <= b.
__device__ __forceinline__ int batch_item(const uint32_t* begin, int n, uint32_t b)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (begin[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}
static_assert(sizeof(FillBatch) < 30000 && sizeof(CompositeBatch) < 30000 && sizeof(CountBatch) < 30000,
              "a batch's parameters fit a kernel's parameter space");

// ---- launches (each returns cudaGetLastError()) -----------------------------------------
cudaError_t launch_cell_quality(const DevMesh& m, int metric, float* out, cudaStream_t s);
// Vertex and edge importance (max over cells) and the faces' static records;
// positions: also the corners' world positions (once, at the upload).
cudaError_t launch_importance(const DevMesh& m, bool positions, cudaStream_t s);

cudaError_t launch_vertex_setup(const DevMesh& m, const CamParams& cam, FrameBufs& fb, cudaStream_t s);
cudaError_t launch_face_setup(const DevMesh& m, const CamParams& cam, int lod, float delta,
                              FrameBufs& fb, int tiles_x, int tiles_y, cudaStream_t s);
cudaError_t launch_bin_fill(const DevMesh& m, FrameBufs& fb, int tiles_x, int W, int H, int reverse,
                            cudaStream_t s);
// Kernel attributes (dynamic shared memory limits), once per device context.
cudaError_t prepare_raster_kernels();
cudaError_t prepare_fill_kernels();
cudaError_t prepare_composite_kernels();

cudaError_t launch_bin_sort(const DevMesh& m, FrameBufs& fb, int tiles_x, int tiles_y, int buckets,
                            cudaStream_t s);
cudaError_t launch_tile_order(FrameBufs& fb, int n_tiles, cudaStream_t s);
cudaError_t launch_count(const DevMesh& m, FrameBufs& fb, int tiles_x, int tiles_y, int W, int H, bool stats,
                         cudaStream_t s);
// The count, fill and main resolve pass of several frames, each one launch.
cudaError_t launch_count_batch(const CountBatch& b, cudaStream_t s);
cudaError_t launch_fill_batch(const FillBatch& b, bool sil, cudaStream_t s);
cudaError_t launch_composite_batch(const CompositeBatch& b, int window, cudaStream_t s);
// The second passes of one frame's resolve (out-of-order and long lists).
cudaError_t launch_composite_tail(FrameBufs& fb, const ShadeParams& sp, int tiles_x, float* out, uint32_t n_long,
                                  OutWin win, cudaStream_t s);
// Tile capacities from the previous frame's exact counts, or `uniform` (> 0) per tile.
cudaError_t launch_capacity_from_previous(FrameBufs& fb, int64_t n_tiles, float margin, uint32_t pad,
                                          uint32_t uniform, cudaStream_t s);
cudaError_t launch_cap_features(FrameBufs& fb, int64_t n_tiles, int tiles_x, float lens_x, float lens_y,
                                float inv_diag, float motion, cudaStream_t s);
cudaError_t launch_cap_forward(const CapNet& net, FrameBufs& fb, int64_t n_tiles, float margin, uint32_t pad,
                               cudaStream_t s);
cudaError_t launch_cap_grad(CapNet& net, const float* X, const uint32_t* counts, int64_t n, cudaStream_t s);
cudaError_t launch_cap_adam(CapNet& net, float lr, cudaStream_t s);
cudaError_t launch_cap_to_half(CapNet& net, cudaStream_t s);
// sil: record each pixel's nearest boundary-fragment depth into fb.zsil.
cudaError_t launch_fill(const DevMesh& m, FrameBufs& fb, const ShadeParams& sp, int tiles_x, int tiles_y, int W,
                        int H, bool regions, bool sil, cudaStream_t s);
cudaError_t launch_composite(FrameBufs& fb, const ShadeParams& sp, int tiles_x, int tiles_y, int W, int H,
                             float* out, uint32_t n_long, int window, OutWin win, cudaStream_t s);
// White silhouettes over the output (Section "Blending Focus and Context"):
// from the boundary surface's depths fb.zsil of the drawn rectangle, which sits
// at (fx0, fy0) of a frame_w x frame_h frame.
cudaError_t launch_silhouette(FrameBufs& fb, int tiles_x, int fx0, int fy0, int frame_w, int frame_h, float alpha,
                              float threshold, float* out, OutWin win, cudaStream_t s);
cudaError_t launch_debug_gather(FrameBufs& fb, const int32_t* d_px, const int32_t* d_py, int64_t n,
                                const uint64_t* d_dst_off, int tiles_x, int W, int H,
                                uint64_t* d_keys, float4* d_rgba, uint32_t* d_counts,
                                cudaStream_t s);

// scans
cudaError_t scan_u32_to_u64(const uint32_t* in, uint64_t* out, int64_t n, uint64_t* part,
                            uint32_t* part_max, uint64_t* total_and_max, uint32_t long_threshold,
                            cudaStream_t s, uint32_t round_to = 0);
int64_t scan_partials_needed(int64_t n);

}  // namespace hexfc
