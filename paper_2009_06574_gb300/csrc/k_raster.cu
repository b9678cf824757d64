// Geometry and fragment stages of the renderer.
//
//   k_vertex_setup  per vertex: camera transform in double (no FMA), window
//                   position snapped to 16.8 fixed point, 24-bit window depth.
//   k_face_setup    per unique face: gather the 4 projected corners, edge
//                   visibility masks of Eq. 1, triangle validity, and the
//                   number of 16x16 tiles each triangle's box touches.
//   k_bin_fill      per face: append 2*face+tri to the list of every touched tile.
//   k_bin_sort      per tile: counting sort of the tile's triangles by depth.
//   k_tile_order    the tiles by decreasing work (for count and fill).
//   k_count         per tile: exact coverage as per-chunk masks and per-pixel
//                   counts.
//   k_fill          per tile: every covered sample (from the masks) gets its
//                   exact depth, is shaded with Eqs. 1-4 and written at its
//                   pixel's offset plus its rank in the pixel's list.
//   k_count_fill    per tile, with capacities chosen before the frame: count
//                   and fill in one pass (no separate count, no global scan).
//
// Each face is drawn as two triangles (Section "Method Overview"; Section "GPU
// Implementation"), all covered samples are kept (per-pixel fragment lists,
// Section "GPU Implementation"), and the fragment shader computes focus from
// the lens, the edge distance to the four face edges ignoring invisible ones,
// and Eqs. 1-4 (Section "Focus+Context").
#include "pipeline.cuh"
#include "shade.cuh"

namespace hexfc {
namespace {

inline unsigned grid_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// ------------------------------------------------------------------ vertex stage

__global__ void k_vertex_setup(const float* __restrict__ verts, int64_t n, CamParams cam,
                               int4* __restrict__ vproj, float* __restrict__ ved)
{
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    double dx = __dsub_rn((double)verts[3 * v], cam.eye[0]);
    double dy = __dsub_rn((double)verts[3 * v + 1], cam.eye[1]);
    double dz = __dsub_rn((double)verts[3 * v + 2], cam.eye[2]);
    double ex = __dadd_rn(__dadd_rn(__dmul_rn(dx, cam.R[0]), __dmul_rn(dy, cam.R[1])), __dmul_rn(dz, cam.R[2]));
    double ey = __dadd_rn(__dadd_rn(__dmul_rn(dx, cam.U[0]), __dmul_rn(dy, cam.U[1])), __dmul_rn(dz, cam.U[2]));
    double ed = __dadd_rn(__dadd_rn(__dmul_rn(dx, cam.F[0]), __dmul_rn(dy, cam.F[1])), __dmul_rn(dz, cam.F[2]));
    double xw, yw, z;
    if (cam.ortho) {
        xw = __dadd_rn(cam.cx, __dmul_rn(ex, cam.scale));
        yw = __dsub_rn(cam.cy, __dmul_rn(ey, cam.scale));
        z = __ddiv_rn(__dsub_rn(ed, cam.znear), __dsub_rn(cam.zfar, cam.znear));
    } else {
        xw = __dadd_rn(cam.cx, __dmul_rn(__ddiv_rn(ex, ed), cam.focal));
        yw = __dsub_rn(cam.cy, __dmul_rn(__ddiv_rn(ey, ed), cam.focal));
        z = __dmul_rn(cam.zf_over, __dsub_rn(1.0, __ddiv_rn(cam.znear, ed)));
    }
    bool valid = (ed > cam.znear) && (ed < cam.zfar) && (fabs(xw) <= 16384.0) && (fabs(yw) <= 16384.0);
    int4 o = make_int4(0, 0, 0, 0);
    if (valid) {
        z = fmin(fmax(z, 0.0), 1.0);
        o.x = (int32_t)rint(__dmul_rn(xw, 256.0));
        o.y = (int32_t)rint(__dmul_rn(yw, 256.0));
        o.z = (int32_t)(uint32_t)rint(__dmul_rn(z, 16777215.0));
        o.w = 1;
    }
    vproj[v] = o;
    ved[v] = (float)ed;
}

// ------------------------------------------------------------------ face stage

__device__ __forceinline__ void tile_range(const TriGeom& t, int& tx0, int& ty0, int& tx1, int& ty1)
{
    tx0 = t.bx0 / kTile; tx1 = t.bx1 / kTile;
    ty0 = t.by0 / kTile; ty1 = t.by1 / kTile;
}

__global__ void k_face_setup(const int4* __restrict__ fverts, const int4* __restrict__ fedges,
                             const uint8_t* __restrict__ elevel, const float* __restrict__ eattr,
                             const int4* __restrict__ vproj, const float* __restrict__ ved, int64_t n_faces,
                             int lod, float delta, int W, int H, int tiles_x, FaceFrame* __restrict__ fframe,
                             uint32_t* __restrict__ tzsum, uint32_t* __restrict__ tile_cnt)
{
    int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n_faces) return;
    int4 c = fverts[f];
    int id[4] = {c.x, c.y, c.z, c.w};
    int32_t X[4], Y[4];
    uint32_t Z[4];
    float E[4];
    bool ok[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        int4 p = vproj[id[k]];
        X[k] = p.x; Y[k] = p.y; Z[k] = (uint32_t)p.z; ok[k] = p.w != 0;
        E[k] = ved[id[k]];
    }
    int4 e = fedges[f];
    int eid[4] = {e.x, e.y, e.z, e.w};
    uint32_t flags = 0, tris = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        bool vis_c = (int)elevel[eid[k]] >= lod;
        bool vis_f = vis_c || eattr[eid[k]] >= delta;
        flags |= (vis_f ? 1u : 0u) << k;
        flags |= (vis_c ? 1u : 0u) << (4 + k);
    }
#pragma unroll
    for (int tri = 0; tri < 2; ++tri) {
        bool vok = ok[0] && (tri == 0 ? (ok[1] && ok[2]) : (ok[2] && ok[3]));
        if (!vok) continue;
        TriGeom t;
        tri_setup(X, Y, tri, W, H, t);
        if (!t.valid) continue;
        tris |= 1u << tri;
        int tx0, ty0, tx1, ty1;
        tile_range(t, tx0, ty0, tx1, ty1);
        for (int ty = ty0; ty <= ty1; ++ty)
            for (int tx = tx0; tx <= tx1; ++tx) atomicAdd(tile_cnt + ty * tiles_x + tx, 1u);
    }
    FaceFrame& r = fframe[f];
    r.X = make_int4(X[0], X[1], X[2], X[3]);
    r.Y = make_int4(Y[0], Y[1], Y[2], Y[3]);
    r.Z = make_uint4((Z[0] & kZ24) | (flags << 24), (Z[1] & kZ24) | (tris << 24), Z[2] & kZ24, Z[3] & kZ24);
    r.ed = make_float4(E[0], E[1], E[2], E[3]);
    const uint32_t z0 = Z[0] & kZ24, z1 = Z[1] & kZ24, z2 = Z[2] & kZ24, z3 = Z[3] & kZ24;
    reinterpret_cast<uint2*>(tzsum)[f] = make_uint2(z0 + z1 + z2, z0 + z2 + z3);   // < 3 * 2^24
}

__global__ void k_bin_fill(const FaceFrame* __restrict__ fframe, int64_t n_faces, int W, int H, int tiles_x,
                           int reverse, const uint64_t* __restrict__ tile_off, uint32_t* __restrict__ tile_cur,
                           uint32_t* __restrict__ bins)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_faces) return;
    int64_t f = reverse ? (n_faces - 1 - i) : i;
    const uint32_t tris = face_tris(fframe[f].Z);
    if (tris == 0) return;
    int4 a = fframe[f].X, b = fframe[f].Y;
    int32_t X[4] = {a.x, a.y, a.z, a.w}, Y[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
    for (int tri = 0; tri < 2; ++tri) {
        if (!(tris & (1u << tri))) continue;
        TriGeom t;
        tri_setup(X, Y, tri, W, H, t);
        int tx0, ty0, tx1, ty1;
        tile_range(t, tx0, ty0, tx1, ty1);
        for (int ty = ty0; ty <= ty1; ++ty)
            for (int tx = tx0; tx <= tx1; ++tx) {
                int tile = ty * tiles_x + tx;
                uint32_t slot = atomicAdd(tile_cur + tile, 1u);
                bins[tile_off[tile] + slot] = (uint32_t)(2 * f + tri);
            }
    }
}

// ------------------------------------------------------------------ bin order

constexpr int kBinSortMax = 4096;   // longer tile lists are sorted through global scratch
constexpr int kDepthBucketsMax = 4096;

// Orders each tile's list front to back by a counting sort of the triangles
// into nb buckets (a power of two, 256..kDepthBucketsMax) of their depth (sum of the three window depths)
// over the tile's depth range; the padding slots stay at the end. Any order
// gives the same fragments; this one makes the fill write every per-pixel list
// sorted or nearly sorted (order within a bucket is arbitrary).
__global__ void __launch_bounds__(256) k_bin_sort(const uint64_t* __restrict__ tile_off,
                                                  const uint32_t* __restrict__ tile_cnt, uint32_t* __restrict__ bins,
                                                  const uint32_t* __restrict__ tzsum, int nb,
                                                  float* __restrict__ tile_zr, uint32_t* __restrict__ tmp)
{
    __shared__ uint32_t s_hist[kDepthBucketsMax];
    __shared__ uint16_t s_b[kBinSortMax];
    __shared__ uint32_t s_out[kBinSortMax];
    __shared__ uint32_t s_red[2][8];
    const int tile = blockIdx.x;
    const uint64_t beg = tile_off[tile];
    const uint32_t n = tile_cnt[tile];   // real entries; the rest of the padded list is kPadBin
    if (n < 2) {   // nothing to order; depth range 0
        if (threadIdx.x == 0) tile_zr[tile] = 0.f;
        return;
    }
    const bool big = n > (uint32_t)kBinSortMax;   // buckets recomputed, scatter through tmp
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    auto zsum = [&](uint32_t f2t) -> uint32_t { return tzsum[f2t]; };   // sum of the triangle's window depths
    // depth range of the tile's triangles
    uint32_t zmin = 0xFFFFFFFFu, zmax = 0;
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
        const uint32_t zs = zsum(bins[beg + i]);
        zmin = min(zmin, zs);
        zmax = max(zmax, zs);
    }
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s_hist[i] = 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        zmin = min(zmin, __shfl_xor_sync(0xffffffffu, zmin, o));
        zmax = max(zmax, __shfl_xor_sync(0xffffffffu, zmax, o));
    }
    if (lane == 0) { s_red[0][warp] = zmin; s_red[1][warp] = zmax; }
    __syncthreads();
    zmin = s_red[0][0];
    zmax = s_red[1][0];
    for (int w = 1; w < 8; ++w) { zmin = min(zmin, s_red[0][w]); zmax = max(zmax, s_red[1][w]); }
    const float scale = (float)nb / (float)(zmax - zmin + 1);
    if (threadIdx.x == 0) tile_zr[tile] = (float)(zmax - zmin) * (1.f / 50331648.f);   // of 3 * 2^24
    auto bucket = [&](uint32_t f2t) -> int { return min((int)((float)(zsum(f2t) - zmin) * scale), nb - 1); };
    // histogram
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
        const int b = bucket(bins[beg + i]);
        if (!big) s_b[i] = (uint16_t)b;
        atomicAdd(&s_hist[b], 1u);
    }
    __syncthreads();
    // exclusive scan of the histogram: nb / 256 buckets per thread
    {
        const int per = nb / 256;
        uint32_t v[kDepthBucketsMax / 256], sum = 0;
#pragma unroll
        for (int k = 0; k < kDepthBucketsMax / 256; ++k) {
            v[k] = k < per ? s_hist[threadIdx.x * per + k] : 0u;
            sum += v[k];
        }
        uint32_t incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        __syncthreads();   // everyone has read s_hist
        if (lane == 31) s_red[0][warp] = incl;
        __syncthreads();
        uint32_t base = incl - sum;
        for (int w = 0; w < warp; ++w) base += s_red[0][w];
#pragma unroll
        for (int k = 0; k < kDepthBucketsMax / 256; ++k) {
            if (k < per) s_hist[threadIdx.x * per + k] = base;
            base += v[k];
        }
    }
    __syncthreads();
    // scatter (arbitrary order inside a bucket), then write back
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
        const uint32_t f2t = bins[beg + i];
        const uint32_t slot = atomicAdd(&s_hist[big ? bucket(f2t) : (int)s_b[i]], 1u);
        if (big) tmp[beg + slot] = f2t;
        else s_out[slot] = f2t;
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) bins[beg + i] = big ? tmp[beg + i] : s_out[i];
}

// ------------------------------------------------------------------ tile order

constexpr int kOrderBuckets = 4096;   // chunk counts above kOrderBuckets - 1 share the first class

// Rank of lane's value among the lanes of the warp holding the same value, and
// how many hold it, so that one lane per value does the shared-memory atomic.
__device__ __forceinline__ uint32_t warp_add_same(uint32_t* s, uint32_t b, bool active)
{
    const unsigned act = __ballot_sync(0xffffffffu, active);
    if (!active) return 0;
    const unsigned peers = __match_any_sync(act, b);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(&s[b], (uint32_t)__popc(peers));
    base = __shfl_sync(peers, base, leader);
    return base + (uint32_t)__popc(peers & ((1u << lane) - 1u));
}

// The tiles in decreasing order of their number of chunks (a counting sort),
// so that the per-tile passes start the longest tiles first and the shortest
// ones fill the tail of the launch. Order inside a class is arbitrary; no
// result depends on it. One block.
__global__ void __launch_bounds__(1024) k_tile_order(const uint64_t* __restrict__ tile_off, int n_tiles,
                                                     uint32_t* __restrict__ order)
{
    __shared__ uint32_t s_hist[kOrderBuckets];
    __shared__ uint32_t s_warp[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    auto cls = [&](int t) -> uint32_t {
        const uint64_t nc = (tile_off[t + 1] - tile_off[t]) / kChunk;
        return (uint32_t)(kOrderBuckets - 1) - (uint32_t)min(nc, (uint64_t)(kOrderBuckets - 1));
    };
    for (int i = threadIdx.x; i < kOrderBuckets; i += blockDim.x) s_hist[i] = 0;
    __syncthreads();
    for (int t0 = 0; t0 < n_tiles; t0 += blockDim.x) {
        const int t = t0 + threadIdx.x;
        warp_add_same(s_hist, t < n_tiles ? cls(t) : 0u, t < n_tiles);
    }
    __syncthreads();
    // exclusive scan of the histogram: kOrderBuckets / 1024 classes per thread
    constexpr int kPer = kOrderBuckets / 1024;
    uint32_t v[kPer], sum = 0;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        v[k] = s_hist[threadIdx.x * kPer + k];
        sum += v[k];
    }
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    uint32_t base = incl - sum;
    for (int w = 0; w < warp; ++w) base += s_warp[w];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        s_hist[threadIdx.x * kPer + k] = base;
        base += v[k];
    }
    __syncthreads();
    for (int t0 = 0; t0 < n_tiles; t0 += blockDim.x) {
        const int t = t0 + threadIdx.x;
        const uint32_t slot = warp_add_same(s_hist, t < n_tiles ? cls(t) : 0u, t < n_tiles);
        if (t < n_tiles) order[slot] = (uint32_t)t;
    }
}

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
    int x0 = max(t.bx0, px0), x1 = min(t.bx1, px0 + kTile - 1);
    int y0 = max(t.by0, py0), y1 = min(t.by1, py0 + kTile - 1);
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

// Exact coverage of the sample (rx, ry) pixels from the box origin of
// triangle j; l[k] = edge function k = weight of vertex k (sum = the area).
__device__ __forceinline__ bool cover_at(const CovSoA& c, int j, int rx, int ry, int64_t l[3])
{
    const int32_t sx = rx << 8, sy = ry << 8;
    const uint32_t meta = c.meta[j];
    bool in = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        int64_t e = c.e0[k][j] + (int64_t)c.dx[k][j] * sy - (int64_t)c.dy[k][j] * sx;
        l[k] = e;
        in = in && (e > 0 || (e == 0 && ((meta >> k) & 1u)));
    }
    return in;
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

constexpr int kRing = 3;
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

// Sum of v over the block's first kTilePix threads (all threads call it).
__device__ __forceinline__ uint32_t tile_sum(uint32_t v, uint32_t* s_tmp)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0 && warp < kConsumerWarps) s_tmp[warp] = v;
    __syncthreads();
    uint32_t t = 0;
#pragma unroll
    for (int w = 0; w < kConsumerWarps; ++w) t += s_tmp[w];
    __syncthreads();
    return t;
}

// Per tile: coverage of every chunk as per-pixel bit masks (kept for the
// fill) and the per-pixel list lengths; the tile's total goes to tile_frag.
__global__ void __launch_bounds__(kTilePix, 5) k_count(const uint64_t* __restrict__ tile_off,
                                                    const uint32_t* __restrict__ bins,
                                                    const FaceFrame* __restrict__ fframe,
                                                    const uint32_t* __restrict__ order, int tiles_x, int W, int H,
                                                    uint32_t* __restrict__ cnt, uint32_t* __restrict__ masks,
                                                    uint32_t* __restrict__ tile_frag)
{
    extern __shared__ __align__(16) unsigned char count_smem[];
    CountWarp* s_w = reinterpret_cast<CountWarp*>(count_smem);   // [kConsumerWarps]
    __shared__ uint32_t s_tmp[kConsumerWarps];
    const int tile = (int)order[blockIdx.x];
    const int px0 = (tile % tiles_x) * kTile, py0 = (tile / tiles_x) * kTile;
    const uint64_t beg = tile_off[tile], end = tile_off[tile + 1];  // multiples of kChunk
    const uint32_t n_chunks = (uint32_t)((end - beg) / kChunk);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    count_chunks(s_w, warp, lane, bins, fframe, beg, n_chunks, px0, py0, W, H, masks);
    __syncthreads();
    uint32_t n = 0;
#pragma unroll
    for (int w = 0; w < kConsumerWarps; ++w) n += s_w[w].mask[threadIdx.x];
    cnt[(int64_t)tile * kTilePix + threadIdx.x] = n;
    const uint32_t total = tile_sum(n, s_tmp);
    if (threadIdx.x == 0) tile_frag[tile] = total;
}

// ------------------------------------------------------------------ fill + shade

// Both records of a face, staged side by side by the producer.
struct __align__(128) RawFace {
    FaceFrame fr;
    FaceStatic st;
};

// Producer lane: fetch the records of face f into shared memory.
__device__ __forceinline__ void rec_fetch(RawFace& r, const FaceFrame* __restrict__ fframe,
                                          const FaceStatic* __restrict__ fstat, uint32_t f)
{
    const int4* a = reinterpret_cast<const int4*>(fframe + f);
    const int4* b = reinterpret_cast<const int4*>(fstat + f);
    int4* dst = reinterpret_cast<int4*>(&r);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        cp_async16(dst + k, a + k);
        cp_async16(dst + 4 + k, b + k);
    }
}

__device__ __forceinline__ void stage_shade(const RawFace& rf, uint32_t f2t, const TriGeom& t, const ShadeParams& sp,
                                            ShadeSoA& S, int j)
{
    const FaceFrame& r = rf.fr;
    const FaceStatic& fs = rf.st;
    const int32_t FX[4] = {r.X.x, r.X.y, r.X.z, r.X.w}, FY[4] = {r.Y.x, r.Y.y, r.Y.z, r.Y.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int k1 = (k + 1) & 3;
        S.FX[k][j] = (float)FX[k];   // |coordinate| <= 2^22: exact
        S.FY[k][j] = (float)FY[k];
        const int32_t ex = FX[k1] - FX[k], ey = FY[k1] - FY[k];
        const float l2 = u64_to_f32((uint64_t)((int64_t)ex * ex + (int64_t)ey * ey));
        S.inv_len2[k][j] = l2 > 0.f ? 1.f / l2 : 0.f;
    }
    const uint32_t zz[4] = {r.Z.x & kZ24, r.Z.y & kZ24, r.Z.z & kZ24, r.Z.w & kZ24};
    const float ee[4] = {r.ed.x, r.ed.y, r.ed.z, r.ed.w}, ii[4] = {fs.imp.x, fs.imp.y, fs.imp.z, fs.imp.w};
    const float xx[4] = {fs.px.x, fs.px.y, fs.px.z, fs.px.w}, yy[4] = {fs.py.x, fs.py.y, fs.py.z, fs.py.w};
    const float ww[4] = {fs.pz.x, fs.pz.y, fs.pz.z, fs.pz.w};
    const bool ortho = sp.ortho != 0;
    float q[3], a[3], P[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int c = t.vi[k];
        // select corner c without dynamic register indexing
        S.z[k][j] = c == 0 ? zz[0] : c == 1 ? zz[1] : c == 2 ? zz[2] : zz[3];
        q[k] = ortho ? 1.f : 1.f / (c == 0 ? ee[0] : c == 1 ? ee[1] : c == 2 ? ee[2] : ee[3]);
        a[k] = (c == 0 ? ii[0] : c == 1 ? ii[1] : c == 2 ? ii[2] : ii[3]) * q[k];
        // offset from the sphere lens centre (unused by the screen lens)
        P[k][0] = ((c == 0 ? xx[0] : c == 1 ? xx[1] : c == 2 ? xx[2] : xx[3]) - sp.lens_c[0]) * q[k];
        P[k][1] = ((c == 0 ? yy[0] : c == 1 ? yy[1] : c == 2 ? yy[2] : yy[3]) - sp.lens_c[1]) * q[k];
        P[k][2] = ((c == 0 ? ww[0] : c == 1 ? ww[1] : c == 2 ? ww[2] : ww[3]) - sp.lens_c[2]) * q[k];
    }
    S.dz[0][j] = (float)(int32_t)(S.z[1][j] - S.z[0][j]);
    S.dz[1][j] = (float)(int32_t)(S.z[2][j] - S.z[0][j]);
    S.q0[j] = q[0];
    S.a0[j] = a[0];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        S.dq[k][j] = q[k + 1] - q[0];
        S.da[k][j] = a[k + 1] - a[0];
#pragma unroll
        for (int d = 0; d < 3; ++d) S.dp[k][d][j] = P[k + 1][d] - P[0][d];
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) S.p0[d][j] = P[0][d];
    S.area[j] = t.area;
    S.inv_area[j] = 1.f / u64_to_f32((uint64_t)t.area);
    S.f2t[j] = f2t;
    S.masks[j] = face_edge_flags(r.Z);
}

struct FillSlot {
    CovSoA c;
    ShadeSoA sh;
};

// Warp queues of covered samples: entry = j | pixel << 5 | ring slot << 13 | counted << 15.
constexpr int kWQ = 256;               // entries per consumer warp (a power of two)
constexpr int kWQWin = kWQ - 32;       // entries queued per window: fewer than 32 leftovers + a window fit
constexpr uint32_t kCounted = 1u << 15;  // the count pass sized the sample's list for it
static_assert(kRing <= 4, "two bits of ring slot");

constexpr size_t kRawOff = (kRing * sizeof(FillSlot) + 127) & ~(size_t)127;   // face records: 128-aligned

__host__ __device__ constexpr size_t fill_smem_bytes()
{
    return kRawOff + 2 * kChunk * sizeof(RawFace) + (size_t)kConsumerWarps * kWQ * sizeof(uint32_t);
}

// The fill pipeline of one tile block: s_base / s_len hold the offsets and
// lengths of the tile's 256 lists, the ring barriers are initialised, and
// `smem` is the dynamic shared memory (fill_smem_bytes()).
__device__ __forceinline__ void fill_tile(unsigned char* smem, const uint64_t* s_base, const uint32_t* s_len,
                                          uint64_t* s_full, uint64_t* s_empty,
                                          const uint32_t* __restrict__ bins, const uint32_t* __restrict__ masks,
                                          const FaceFrame* __restrict__ fframe,
                                          const FaceStatic* __restrict__ fstat, uint64_t beg, uint32_t n_chunks,
                                          int px0, int py0, int W, int H, const ShadeParams& sp,
                                          uint64_t* __restrict__ key, float4* __restrict__ rgba,
                                          unsigned long long* __restrict__ err)
{
    FillSlot* s_ring = reinterpret_cast<FillSlot*>(smem);                                    // [kRing]
    RawFace* s_raw = reinterpret_cast<RawFace*>(smem + kRawOff);                            // [2][kChunk]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == kConsumerWarps) {  // producer
        uint32_t f2t_c = n_chunks > 0 ? bins[beg + lane] : kPadBin;
        uint32_t f2t_n = n_chunks > 1 ? bins[beg + kChunk + lane] : kPadBin;
        if (f2t_c != kPadBin) rec_fetch(s_raw[lane], fframe, fstat, f2t_c >> 1);
        cp_async_commit();
        for (uint32_t c = 0; c < n_chunks; ++c) {
            const int s = c % kRing;
            uint32_t f2t_nn = kPadBin;
            if (c + 1 < n_chunks) {
                if (f2t_n != kPadBin) rec_fetch(s_raw[((c + 1) & 1) * kChunk + lane], fframe, fstat, f2t_n >> 1);
                if (c + 2 < n_chunks) f2t_nn = bins[beg + (uint64_t)(c + 2) * kChunk + lane];
            }
            cp_async_commit();
            cp_async_wait<1>();   // this lane's copies of chunk c have landed
            if (!mbar_wait(&s_empty[s], ((c / kRing) & 1) ^ 1)) {
                if (lane == 0) atomicOr(err, kErrWait);
                break;
            }
            FillSlot& S = s_ring[s];
            if (f2t_c != kPadBin) {
                const RawFace& r = s_raw[(c & 1) * kChunk + lane];
                TriGeom t;
                stage_cov(r.fr.X, r.fr.Y, f2t_c, W, H, px0, py0, S.c, lane, t);
                if (S.c.box[lane] != 0) stage_shade(r, f2t_c, t, sp, S.sh, lane);
            } else {
                S.c.box[lane] = 0;
            }
            mbar_arrive(&s_full[s]);
            f2t_c = f2t_n;
            f2t_n = f2t_nn;
        }
        cp_async_wait<0>();
        return;
    }
    // consumers: warp w owns pixels 32w .. 32w + 31 and a private queue; each
    // warp goes through the chunks on its own (no block barrier), so warps
    // may be up to kRing chunks apart
    const int p = threadIdx.x;
    uint32_t* s_q = reinterpret_cast<uint32_t*>(s_raw + 2 * kChunk) + warp * kWQ;   // [kWQ]
    uint32_t k_run = 0;
    bool bad = false, stalled = false;
    // The warp's 32 lists are one region of the fragment arrays, from the
    // offset of its first pixel; the region holds them chunk-major (fragment
    // e of the warp's queue at region start + e), so every shading round
    // writes 32 consecutive records.
    const uint64_t w_beg = s_base[warp * 32];
    const uint64_t w_end = w_beg + __reduce_add_sync(0xffffffffu, s_len[p]);
    // Queue positions are absolute counts (modulo kWQ): entries [head, tail) are
    // queued. Only whole rounds of 32 entries are shaded; the rest waits for
    // the next chunk unless it would keep an older chunk's slot (then it is
    // shaded as a partial round), so at most the newest chunk's slot is held.
    uint32_t head = 0, tail = 0, released = 0;
    auto shade_entry = [&](uint32_t qe, uint32_t e) {
        const uint64_t o = w_beg + e;
        if (!(qe & kCounted) || o >= w_end) return;
        const int j = (int)(qe & 31u);
        const uint32_t pl = (qe >> 5) & 255u;
        const FillSlot& S = s_ring[(qe >> 13) & 3u];
        const int lx = (int)(pl & (kTile - 1)), ly = (int)(pl / kTile);
        const int bx = S.c.box[j];
        // exact weights of vertices 1 and 2 (edge functions opposite them)
        const int32_t sxr = (lx - box_lx0(bx)) << 8, syr = (ly - box_ly0(bx)) << 8;
        const int64_t l1 = S.c.e0[1][j] + (int64_t)S.c.dx[1][j] * syr - (int64_t)S.c.dy[1][j] * sxr;
        const int64_t l2 = S.c.e0[2][j] + (int64_t)S.c.dx[2][j] * syr - (int64_t)S.c.dy[2][j] * sxr;
        const float ia = S.sh.inv_area[j];
        const float lam1 = u64_to_f32((uint64_t)l1) * ia, lam2 = u64_to_f32((uint64_t)l2) * ia;
        const uint32_t z = sample_depth_lam(S.sh.z[0][j], S.sh.z[1][j], S.sh.z[2][j], l1, l2, S.sh.area[j], lam1,
                                            lam2, S.sh.dz[0][j], S.sh.dz[1][j], bad);
        const float4 col = shade_fragment(S.sh, j, lam1, lam2, px0 + lx, py0 + ly, sp);
        key[o] = ((uint64_t)z << 32) | (uint64_t)S.sh.f2t[j];
        rgba[o] = col;
    };
    // masks of the next two chunks are in flight while this one is shaded
    uint32_t mk_a = n_chunks > 0 ? masks[(beg / kChunk) * kTilePix + p] : 0u;
    uint32_t mk_b = n_chunks > 1 ? masks[(beg / kChunk + 1) * kTilePix + p] : 0u;
    for (uint32_t c = 0; c < n_chunks; ++c) {
        const int s = c % kRing;
        const uint32_t mk = mk_a;
        mk_a = mk_b;
        if (c + 2 < n_chunks) mk_b = masks[(beg / kChunk + c + 2) * kTilePix + p];
        // every entry of the chunks before c - 1 (and of c - 1 if nothing is
        // left over) has been shaded by the whole warp: release their slots
        __syncwarp();
        const uint32_t rel_to = head == tail ? c : c - 1;
        if (lane == 0)
            for (uint32_t r = released; r < rel_to; ++r) mbar_arrive(&s_empty[r % kRing]);
        released = max(released, rel_to);
        if (!__all_sync(0xffffffffu, mbar_wait(&s_full[s], (c / kRing) & 1))) {
            if (lane == 0) atomicOr(err, kErrWait);
            stalled = true;
            break;
        }
        // warp exclusive scan of the hit counts
        const uint32_t h = __popc(mk);
        uint32_t incl = h;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        const bool fits = k_run + h <= s_len[p];   // the count pass sized this list
        bad = bad || !fits;
        const uint32_t chunk_start = tail;
        const uint32_t tag = ((uint32_t)p << 5) | ((uint32_t)s << 13) | (fits ? kCounted : 0u);
        for (uint32_t w0 = 0; w0 < total; w0 += kWQWin) {
            uint32_t m2 = mk, r = incl - h;
            while (m2) {
                const uint32_t j = __ffs(m2) - 1;
                m2 &= m2 - 1;
                if (r >= w0 && r < w0 + kWQWin) s_q[(tail + r - w0) & (kWQ - 1)] = j | tag;
                ++r;
            }
            __syncwarp();   // the window's entries are queued
            tail += min((uint32_t)kWQWin, total - w0);
            const uint32_t rounds = (tail - head) / 32;
            for (uint32_t i = 0; i < rounds; ++i) {
                const uint32_t e = head + i * 32 + lane;
                shade_entry(s_q[e & (kWQ - 1)], e);
            }
            head += rounds * 32;
            __syncwarp();   // shaded entries are read before the next window overwrites them
        }
        if (head < chunk_start) {   // leftovers of an older chunk: shade them all now
            if (lane < tail - head) shade_entry(s_q[(head + lane) & (kWQ - 1)], head + lane);
            head = tail;
        }
        k_run += h;
    }
    // the last leftovers (the producer is done; no slot is released any more)
    if (!stalled && lane < tail - head) shade_entry(s_q[(head + lane) & (kWQ - 1)], head + lane);
    if (bad) atomicOr(err, 1ull);
}

// Per tile: the coverage masks of the count pass give, chunk by chunk, each
// pixel's covered triangles; each consumer warp compacts its 32 pixels'
// covered samples into its queue (pixel-major, in list order) and shades it
// 32 samples at a time, so that every lane has work, writing the fragments in
// queue order into the warp's region (the 32 lists the count pass sized):
// chunk by chunk, pixel by pixel within a chunk. The producer fetches the face
// records of chunk c+1 with cp.async while it sets up chunk c.
__global__ void __launch_bounds__(kPipeThreads, 3) k_fill(const uint64_t* __restrict__ tile_off,
                                                          const uint32_t* __restrict__ bins,
                                                          const uint32_t* __restrict__ masks,
                                                          const FaceFrame* __restrict__ fframe,
                                                          const FaceStatic* __restrict__ fstat,
                                                          const uint32_t* __restrict__ order, int tiles_x, int W,
                                                          int H, ShadeParams sp, const uint64_t* __restrict__ off,
                                                          const uint32_t* __restrict__ cnt,
                                                          uint64_t* __restrict__ key, float4* __restrict__ rgba,
                                                          unsigned long long* __restrict__ err)
{
    extern __shared__ __align__(128) unsigned char fill_smem[];
    __shared__ uint64_t s_base[kTilePix];
    __shared__ uint32_t s_len[kTilePix];
    __shared__ __align__(8) uint64_t s_full[kRing], s_empty[kRing];
    const int tile = (int)order[blockIdx.x];
    const int px0 = (tile % tiles_x) * kTile, py0 = (tile / tiles_x) * kTile;
    const uint64_t beg = tile_off[tile], end = tile_off[tile + 1];  // multiples of kChunk
    const uint32_t n_chunks = (uint32_t)((end - beg) / kChunk);
    if (threadIdx.x < kTilePix) {
        const int64_t q = (int64_t)tile * kTilePix + threadIdx.x;
        s_base[threadIdx.x] = off[q];
        s_len[threadIdx.x] = cnt[q];
    }
    pipe_init(s_full, s_empty);
    fill_tile(fill_smem, s_base, s_len, s_full, s_empty, bins, masks, fframe, fstat, beg, n_chunks, px0, py0,
              W, H, sp, key, rgba, err);
}

// Per tile, with no separate count pass: the consumer warps rasterise the
// tile's chunks into masks and per-pixel counts (as k_count), the block scans
// the counts into offsets inside the tile's region [cap_off[t], cap_off[t+1])
// of the fragment arrays (capacities chosen before the frame), and if the
// tile fits, the fill pipeline draws it. A tile that does not fit draws
// nothing: it appends itself to `over` (scal[6] tiles, scal[14] fragments)
// with its exact counts and masks in place, for k_fill to draw once it has a
// region. tile_frag = the tile's exact total; scal[0] += fragments, scal[1] =
// max list, scal[2] += lists longer than kWarpSortMax.
__global__ void __launch_bounds__(kPipeThreads, 3) k_count_fill(const uint64_t* __restrict__ tile_off,
                                                               const uint32_t* __restrict__ bins,
                                                               uint32_t* __restrict__ masks,
                                                               const FaceFrame* __restrict__ fframe,
                                                               const FaceStatic* __restrict__ fstat,
                                                               const uint32_t* __restrict__ order, int tiles_x,
                                                               int W, int H, ShadeParams sp,
                                                               const uint64_t* __restrict__ cap_off,
                                                               uint64_t frag_cap, uint32_t* __restrict__ cnt,
                                                               uint64_t* __restrict__ off,
                                                               uint32_t* __restrict__ tile_frag,
                                                               uint32_t* __restrict__ over,
                                                               uint64_t* __restrict__ key, float4* __restrict__ rgba,
                                                               unsigned long long* __restrict__ scal)
{
    extern __shared__ __align__(128) unsigned char cf_smem[];
    __shared__ uint64_t s_base[kTilePix];
    __shared__ uint32_t s_len[kTilePix];
    __shared__ uint32_t s_wsum[kConsumerWarps];
    __shared__ uint32_t s_wmax[kConsumerWarps], s_wlong[kConsumerWarps];
    __shared__ __align__(8) uint64_t s_full[kRing], s_empty[kRing];
    const int tile = (int)order[blockIdx.x];
    const int px0 = (tile % tiles_x) * kTile, py0 = (tile / tiles_x) * kTile;
    const uint64_t beg = tile_off[tile], end = tile_off[tile + 1];  // multiples of kChunk
    const uint32_t n_chunks = (uint32_t)((end - beg) / kChunk);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    CountWarp* s_w = reinterpret_cast<CountWarp*>(cf_smem);
    if (warp < kConsumerWarps) count_chunks(s_w, warp, lane, bins, fframe, beg, n_chunks, px0, py0, W, H, masks);
    __syncthreads();
    // the per-pixel counts, their block-wide exclusive scan, maximum and long lists
    uint32_t n = 0;
    if (warp < kConsumerWarps)
#pragma unroll
        for (int w = 0; w < kConsumerWarps; ++w) n += s_w[w].mask[threadIdx.x];
    uint32_t incl = n, mx = n, lg = n > (uint32_t)kWarpSortMax ? 1u : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        lg += __shfl_xor_sync(0xffffffffu, lg, o);
    }
    if (lane == 31 && warp < kConsumerWarps) {
        s_wsum[warp] = incl;
        s_wmax[warp] = mx;
        s_wlong[warp] = lg;
    }
    __syncthreads();
    uint32_t base = 0, total = 0, tmax = 0, tlong = 0;
#pragma unroll
    for (int w = 0; w < kConsumerWarps; ++w) {
        const uint32_t v = s_wsum[w];
        base += w < warp ? v : 0u;
        total += v;
        tmax = max(tmax, s_wmax[w]);
        tlong += s_wlong[w];
    }
    const uint64_t region = cap_off[tile], cap = cap_off[tile + 1] - region;
    const bool fits = total <= cap && region + total <= frag_cap;   // the same on every thread
    if (warp < kConsumerWarps) {
        const int64_t q = (int64_t)tile * kTilePix + threadIdx.x;
        const uint64_t o = region + base + incl - n;
        cnt[q] = n;        // also for a tile that does not fit: its lists are drawn later
        off[q] = o;
        s_base[threadIdx.x] = o;
        s_len[threadIdx.x] = n;
    }
    if (threadIdx.x == 0) {
        tile_frag[tile] = total;
        atomicAdd(&scal[0], (unsigned long long)total);
        atomicMax(&scal[1], (unsigned long long)tmax);
        atomicAdd(&scal[2], (unsigned long long)tlong);
        if (!fits) {
            over[atomicAdd(&scal[6], 1ull)] = (uint32_t)tile;
            atomicAdd(&scal[14], (unsigned long long)total);
        }
    }
    if (!fits) return;
    pipe_init(s_full, s_empty);   // also orders the scan's shared reads before the fill reuses them
    fill_tile(cf_smem, s_base, s_len, s_full, s_empty, bins, masks, fframe, fstat, beg, n_chunks, px0, py0,
              W, H, sp, key, rgba, scal + 5);
}

// Regions for the tiles that did not fit their capacity: after `base`, in
// the order of the list, sized by their exact totals; then the pixels' list
// offsets inside them (one block per listed tile).
__global__ void __launch_bounds__(kTilePix) k_overflow_offsets(const uint32_t* __restrict__ over, uint32_t n_over,
                                                               const uint32_t* __restrict__ tile_frag, uint64_t base,
                                                               const uint32_t* __restrict__ cnt,
                                                               uint64_t* __restrict__ off)
{
    __shared__ uint32_t s_w[kConsumerWarps];
    __shared__ unsigned long long s_region;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t i = blockIdx.x;
    // the tile's region: base + the totals of the tiles listed before it
    unsigned long long acc = 0;
    for (uint32_t k = threadIdx.x; k < i; k += blockDim.x) acc += tile_frag[over[k]];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) s_region = 0;
    __syncthreads();
    if (lane == 0) atomicAdd(&s_region, acc);
    // the pixels' exclusive scan inside the tile
    const uint32_t tile = over[i];
    const int64_t q = (int64_t)tile * kTilePix + threadIdx.x;
    const uint32_t n = cnt[q];
    uint32_t incl = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    uint32_t pre = incl - n;
    for (int w = 0; w < warp; ++w) pre += s_w[w];
    off[q] = base + s_region + pre;
}

// Capacities from the previous frame's exact tile counts: prev * (1 + margin) + pad.
__global__ void k_capacity_from_previous(const uint32_t* __restrict__ prev, int64_t n_tiles, float margin,
                                         uint32_t pad, uint32_t* __restrict__ cap)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tiles) return;
    cap[t] = (uint32_t)fminf((float)prev[t] * (1.f + margin) + (float)pad, 4.0e9f);
}

constexpr size_t count_fill_smem_bytes()
{
    return kConsumerWarps * sizeof(CountWarp) > fill_smem_bytes() ? kConsumerWarps * sizeof(CountWarp)
                                                                     : fill_smem_bytes();
}

}  // namespace

cudaError_t prepare_raster_kernels()
{
    cudaError_t e = cudaFuncSetAttribute(k_count, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(kConsumerWarps * sizeof(CountWarp)));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fill, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fill_smem_bytes());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_count_fill, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)count_fill_smem_bytes());
    return e;
}

cudaError_t launch_capacity_from_previous(FrameBufs& fb, int64_t n_tiles, float margin, uint32_t pad, cudaStream_t s)
{
    k_capacity_from_previous<<<grid_for(n_tiles, 256), 256, 0, s>>>(fb.tile_frag, n_tiles, margin, pad, fb.tile_cap);
    return cudaGetLastError();
}

cudaError_t launch_count_fill(const DevMesh& m, FrameBufs& fb, const ShadeParams& sp, int tiles_x, int tiles_y, int W,
                              int H, cudaStream_t s)
{
    k_count_fill<<<(unsigned)(tiles_x * tiles_y), kPipeThreads, count_fill_smem_bytes(), s>>>(
        fb.tile_off, fb.bins, fb.masks, fb.fframe, m.fstat, fb.tile_order, tiles_x, W, H, sp, fb.cap_off,
        (uint64_t)fb.frag_cap, fb.cnt, fb.off, fb.tile_frag, fb.tile_over, fb.key, fb.rgba,
        reinterpret_cast<unsigned long long*>(fb.scal));
    return cudaGetLastError();
}

cudaError_t launch_overflow_fill(const DevMesh& m, FrameBufs& fb, const ShadeParams& sp, uint32_t n_over,
                                 uint64_t base, int tiles_x, int W, int H, cudaStream_t s)
{
    k_overflow_offsets<<<n_over, kTilePix, 0, s>>>(fb.tile_over, n_over, fb.tile_frag, base, fb.cnt, fb.off);
    k_fill<<<n_over, kPipeThreads, fill_smem_bytes(), s>>>(fb.tile_off, fb.bins, fb.masks, fb.fframe, m.fstat,
                                                            fb.tile_over, tiles_x, W, H, sp, fb.off, fb.cnt, fb.key,
                                                            fb.rgba, reinterpret_cast<unsigned long long*>(fb.scal + 5));
    return cudaGetLastError();
}

cudaError_t launch_vertex_setup(const DevMesh& m, const CamParams& cam, FrameBufs& fb, cudaStream_t s)
{
    k_vertex_setup<<<grid_for(m.n_verts, 256), 256, 0, s>>>(m.verts, m.n_verts, cam, fb.vproj, fb.ved);
    return cudaGetLastError();
}

cudaError_t launch_face_setup(const DevMesh& m, const CamParams& cam, int lod, float delta, FrameBufs& fb,
                              int tiles_x, int tiles_y, cudaStream_t s)
{
    (void)tiles_y;
    k_face_setup<<<grid_for(m.n_faces, 256), 256, 0, s>>>(m.fverts, m.fedges, m.elevel, m.eattr, fb.vproj,
                                                           fb.ved, m.n_faces, lod, delta, cam.W, cam.H, tiles_x,
                                                           fb.fframe, fb.tzsum, fb.tile_cnt);
    return cudaGetLastError();
}

cudaError_t launch_bin_fill(const DevMesh& m, FrameBufs& fb, int tiles_x, int W, int H, int reverse,
                            cudaStream_t s)
{
    k_bin_fill<<<grid_for(m.n_faces, 256), 256, 0, s>>>(fb.fframe, m.n_faces, W, H, tiles_x, reverse,
                                                         fb.tile_off, fb.tile_cur, fb.bins);
    return cudaGetLastError();
}

cudaError_t launch_bin_sort(const DevMesh& m, FrameBufs& fb, int tiles_x, int tiles_y, int buckets, cudaStream_t s)
{
    (void)m;
    if (buckets == 0)   // no depth order (lists keep the faces' arrival order); depth ranges unknown
        return cudaMemsetAsync(fb.tile_zr, 0, sizeof(float) * (size_t)tiles_x * tiles_y, s);
    k_bin_sort<<<(unsigned)(tiles_x * tiles_y), 256, 0, s>>>(fb.tile_off, fb.tile_cnt, fb.bins, fb.tzsum, buckets,
                                                              fb.tile_zr, fb.bins_tmp);
    return cudaGetLastError();
}

cudaError_t launch_tile_order(FrameBufs& fb, int n_tiles, cudaStream_t s)
{
    k_tile_order<<<1, 1024, 0, s>>>(fb.tile_off, n_tiles, fb.tile_order);
    return cudaGetLastError();
}

cudaError_t launch_count(const DevMesh& m, FrameBufs& fb, int tiles_x, int tiles_y, int W, int H, cudaStream_t s)
{
    const size_t smem = kConsumerWarps * sizeof(CountWarp);
    k_count<<<(unsigned)(tiles_x * tiles_y), kTilePix, smem, s>>>(fb.tile_off, fb.bins, fb.fframe, fb.tile_order,
                                                                   tiles_x, W, H, fb.cnt, fb.masks, fb.tile_frag);
    return cudaGetLastError();
}

cudaError_t launch_fill(const DevMesh& m, FrameBufs& fb, const ShadeParams& sp, int tiles_x, int tiles_y, int W,
                        int H, cudaStream_t s)
{
    const size_t smem = fill_smem_bytes();
    k_fill<<<(unsigned)(tiles_x * tiles_y), kPipeThreads, smem, s>>>(
        fb.tile_off, fb.bins, fb.masks, fb.fframe, m.fstat, fb.tile_order, tiles_x, W, H, sp, fb.off, fb.cnt, fb.key,
        fb.rgba, reinterpret_cast<unsigned long long*>(fb.scal + 5));
    return cudaGetLastError();
}

}  // namespace hexfc
