// Geometry and fragment stages of the renderer.
//
//   k_vertex_setup  per vertex: camera transform in double (no FMA), window
//                   position snapped to 16.8 fixed point, 24-bit window depth.
//   k_face_setup    per unique face: gather the 4 projected corners, edge
//                   visibility masks of Eq. 1, triangle validity, and the
//                   number of raster tiles each triangle's box touches.
//   k_bin_fill      per face: append 2*face+tri to the list of every touched tile.
//   k_bin_sort      per tile: counting sort of the tile's triangles by depth.
//   k_tile_order    the tiles by decreasing work (for count and fill).
//   k_count         per tile: exact coverage as per-chunk masks and per-pixel
//                   counts.
//
// The fill pass (k_fill, k_count_fill) is in k_fill.cu.
//
// Each face is drawn as two triangles (Section "Method Overview"; Section "GPU
// Implementation"), all covered samples are kept (per-pixel fragment lists,
// Section "GPU Implementation"), and the fragment shader computes focus from
// the lens, the edge distance to the four face edges ignoring invisible ones,
// and Eqs. 1-4 (Section "Focus+Context").
#include "count_tiles.cuh"

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
        // snapped in frame coordinates, then moved by whole pixels into the drawn
        // rectangle: coverage, depth and edge distances are those of the frame
        o.x = (int32_t)rint(__dmul_rn(xw, 256.0)) - 256 * cam.ox;
        o.y = (int32_t)rint(__dmul_rn(yw, 256.0)) - 256 * cam.oy;
        o.z = (int32_t)(uint32_t)rint(__dmul_rn(z, 16777215.0));
        o.w = 1;
    }
    vproj[v] = o;
    ved[v] = (float)ed;
}

// ------------------------------------------------------------------ face stage

// atomicAdd(ctr + idx, 1) for every calling lane, one atomic per distinct idx
// among the lanes that call together; returns the value this lane's own
// increment would have returned (lanes of one index in lane order).
__device__ __forceinline__ uint32_t agg_inc(uint32_t* ctr, int idx)
{
    const unsigned act = __activemask();
    const unsigned peers = __match_any_sync(act, idx);
    const int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(ctr + idx, (uint32_t)__popc(peers));
    base = __shfl_sync(peers, base, leader);
    return base + (uint32_t)__popc(peers & ((1u << lane) - 1u));
}

__device__ __forceinline__ void tile_range(const TriGeom& t, int& tx0, int& ty0, int& tx1, int& ty1)
{
    tx0 = t.bx0 / kTileW; tx1 = t.bx1 / kTileW;
    ty0 = t.by0 / kTileH; ty1 = t.by1 / kTileH;
}

__global__ void k_face_setup(const int4* __restrict__ fverts, const int4* __restrict__ fedges,
                             const uint8_t* __restrict__ fbound,
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
            for (int tx = tx0; tx <= tx1; ++tx) agg_inc(tile_cnt, ty * tiles_x + tx);
    }
    FaceFrame& r = fframe[f];
    r.X = make_int4(X[0], X[1], X[2], X[3]);
    r.Y = make_int4(Y[0], Y[1], Y[2], Y[3]);
    const uint32_t bnd = fbound[f] ? 1u : 0u;
    r.Z = make_uint4((Z[0] & kZ24) | (flags << 24), (Z[1] & kZ24) | (tris << 24) | (bnd << 26), Z[2] & kZ24,
                     Z[3] & kZ24);
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
                const uint32_t slot = agg_inc(tile_cur, tile);
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
    constexpr int kItems = kBinSortMax / 256;   // entries per thread of a list held in registers
    __shared__ uint32_t s_hist[kDepthBucketsMax];
    __shared__ uint32_t s_out[kBinSortMax];
    __shared__ uint32_t s_red[2][8];
    const int tile = blockIdx.x;
    const uint64_t beg = tile_off[tile];
    const uint32_t n = tile_cnt[tile];   // real entries; the rest of the padded list is kPadBin
    if (n < 2) {   // nothing to order; depth range 0
        if (threadIdx.x == 0) tile_zr[tile] = 0.f;
        return;
    }
    const bool big = n > (uint32_t)kBinSortMax;   // entries re-read, scatter through tmp
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // a list of up to kBinSortMax entries is read once: entry tid + 256 k of
    // the list and its triangle's depth sum (sum of the three window depths)
    // stay in this thread's registers
    uint32_t f2t[kItems], zs[kItems];
    uint32_t zmin = 0xFFFFFFFFu, zmax = 0;
    if (!big) {
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            const uint32_t i = threadIdx.x + 256u * k;
            f2t[k] = i < n ? bins[beg + i] : 0u;
        }
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            const uint32_t i = threadIdx.x + 256u * k;
            zs[k] = i < n ? tzsum[f2t[k]] : 0u;
            if (i < n) {
                zmin = min(zmin, zs[k]);
                zmax = max(zmax, zs[k]);
            }
        }
    } else {
        for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
            const uint32_t z = tzsum[bins[beg + i]];
            zmin = min(zmin, z);
            zmax = max(zmax, z);
        }
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
    auto bucket = [&](uint32_t z) -> int { return min((int)((float)(z - zmin) * scale), nb - 1); };
    // histogram
    if (!big) {
#pragma unroll
        for (int k = 0; k < kItems; ++k)
            if (threadIdx.x + 256u * k < n) atomicAdd(&s_hist[bucket(zs[k])], 1u);
    } else {
        for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) atomicAdd(&s_hist[bucket(tzsum[bins[beg + i]])], 1u);
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
    if (!big) {
#pragma unroll
        for (int k = 0; k < kItems; ++k)
            if (threadIdx.x + 256u * k < n) s_out[atomicAdd(&s_hist[bucket(zs[k])], 1u)] = f2t[k];
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) bins[beg + i] = s_out[i];
    } else {
        for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
            const uint32_t f = bins[beg + i];
            tmp[beg + atomicAdd(&s_hist[bucket(tzsum[f])], 1u)] = f;
        }
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) bins[beg + i] = tmp[beg + i];
    }
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
    // the classes of tiles threadIdx.x + 1024 k, k < kReg, are read once, all
    // loads in flight together, and kept in registers for both passes
    constexpr int kReg = 16;
    uint32_t cl[kReg];
#pragma unroll
    for (int k = 0; k < kReg; ++k) {
        const int t = k * 1024 + threadIdx.x;
        cl[k] = t < n_tiles ? cls(t) : 0u;
    }
    for (int i = threadIdx.x; i < kOrderBuckets; i += blockDim.x) s_hist[i] = 0;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kReg; ++k)
        if (k * 1024 < n_tiles) warp_add_same(s_hist, cl[k], k * 1024 + (int)threadIdx.x < n_tiles);
    for (int t0 = kReg * 1024; t0 < n_tiles; t0 += blockDim.x) {
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
#pragma unroll
    for (int k = 0; k < kReg; ++k) {
        const int t = k * 1024 + threadIdx.x;
        if (k * 1024 < n_tiles) {
            const uint32_t slot = warp_add_same(s_hist, cl[k], t < n_tiles);
            if (t < n_tiles) order[slot] = (uint32_t)t;
        }
    }
    for (int t0 = kReg * 1024; t0 < n_tiles; t0 += blockDim.x) {
        const int t = t0 + threadIdx.x;
        const uint32_t slot = warp_add_same(s_hist, t < n_tiles ? cls(t) : 0u, t < n_tiles);
        if (t < n_tiles) order[slot] = (uint32_t)t;
    }
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
// fill) and the per-pixel list lengths; the tile's total goes to tile_frag,
// and, if stats is given, into copy tile % kStatCopies of the counters
// (stats + 4 copy): [0] += fragments, [1] = longest list, [2] += lists longer
// than kWarpSortMax (the frame's statistics without
// the pixel scan).
// The count of one tile (the body of k_count and k_count_batch).
__device__ __forceinline__ void count_tile(int tile, const uint64_t* __restrict__ tile_off,
                                           const uint32_t* __restrict__ bins, const FaceFrame* __restrict__ fframe,
                                           int tiles_x, int W, int H, uint32_t* __restrict__ cnt,
                                           uint32_t* __restrict__ masks, uint32_t* __restrict__ tile_frag,
                                           unsigned long long* __restrict__ stats)
{
    extern __shared__ __align__(16) unsigned char count_smem[];
    CountWarp* s_w = reinterpret_cast<CountWarp*>(count_smem);   // [kConsumerWarps]
    __shared__ uint32_t s_tmp[kConsumerWarps];
    const int px0 = (tile % tiles_x) * kTileW, py0 = (tile / tiles_x) * kTileH;
    const uint64_t beg = tile_off[tile], end = tile_off[tile + 1];  // multiples of kChunk
    const uint32_t n_chunks = (uint32_t)((end - beg) / kChunk);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    count_chunks(s_w, warp, lane, bins, fframe, beg, n_chunks, px0, py0, W, H, masks);
    __syncthreads();
    uint32_t n = 0;
#pragma unroll
    for (int w = 0; w < kConsumerWarps; ++w) n += s_w[w].mask[threadIdx.x];
    cnt[(int64_t)tile * kTilePix + threadIdx.x] = n;
    __shared__ uint32_t s_mx[kConsumerWarps], s_lg[kConsumerWarps];
    if (stats) {   // (the pixel scan gives them otherwise)
        const uint32_t mx = __reduce_max_sync(0xffffffffu, n);
        const uint32_t lg = __reduce_add_sync(0xffffffffu, n > (uint32_t)kWarpSortMax ? 1u : 0u);
        if (lane == 0) {
            s_mx[warp] = mx;
            s_lg[warp] = lg;
        }
    }
    const uint32_t total = tile_sum(n, s_tmp);   // (its block barrier also publishes s_mx, s_lg)
    if (threadIdx.x == 0) {
        tile_frag[tile] = total;
        if (stats) {   // one copy of the counters per tile % kStatCopies: no queue on one address
            uint32_t mx = 0, lg = 0;
#pragma unroll
            for (int w = 0; w < kConsumerWarps; ++w) {
                mx = max(mx, s_mx[w]);
                lg += s_lg[w];
            }
            unsigned long long* st = stats + (tile % kStatCopies) * 4;
            if (total) atomicAdd(&st[0], (unsigned long long)total);
            if (mx) atomicMax(&st[1], (unsigned long long)mx);
            if (lg) atomicAdd(&st[2], (unsigned long long)lg);
        }
    }
}

__global__ void __launch_bounds__(kTilePix, 5) k_count(const uint64_t* __restrict__ tile_off,
                                                    const uint32_t* __restrict__ bins,
                                                    const FaceFrame* __restrict__ fframe,
                                                    const uint32_t* __restrict__ order, int tiles_x, int W, int H,
                                                    uint32_t* __restrict__ cnt, uint32_t* __restrict__ masks,
                                                    uint32_t* __restrict__ tile_frag,
                                                    unsigned long long* __restrict__ stats)
{
    count_tile((int)order[blockIdx.x], tile_off, bins, fframe, tiles_x, W, H, cnt, masks, tile_frag, stats);
}

// The count of several frames in one grid (a batch).
__global__ void __launch_bounds__(kTilePix, 5) k_count_batch(const __grid_constant__ CountBatch b)
{
    const int i = batch_item(b.tile_begin, b.n, blockIdx.x);
    const CountItem& it = b.it[i];
    const int tile = (int)it.order[blockIdx.x - b.tile_begin[i]];
    count_tile(tile, it.tile_off, it.bins, it.fframe, it.tiles_x, it.W, it.H, it.cnt, it.masks, it.tile_frag,
               nullptr);
}

}  // namespace

cudaError_t prepare_raster_kernels()
{
    cudaError_t e = cudaFuncSetAttribute(k_count, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(kConsumerWarps * sizeof(CountWarp)));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_count_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(kConsumerWarps * sizeof(CountWarp)));
    return e;
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
    k_face_setup<<<grid_for(m.n_faces, 256), 256, 0, s>>>(m.fverts, m.fedges, m.fbound, m.elevel, m.eattr, fb.vproj,
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

cudaError_t launch_count(const DevMesh& m, FrameBufs& fb, int tiles_x, int tiles_y, int W, int H, bool stats,
                         cudaStream_t s)
{
    const size_t smem = kConsumerWarps * sizeof(CountWarp);
    k_count<<<(unsigned)(tiles_x * tiles_y), kTilePix, smem, s>>>(fb.tile_off, fb.bins, fb.fframe, fb.tile_order,
                                                                   tiles_x, W, H, fb.cnt, fb.masks, fb.tile_frag,
                                                                   stats ? reinterpret_cast<unsigned long long*>(fb.cstat)
                                                                         : nullptr);
    return cudaGetLastError();
}

cudaError_t launch_count_batch(const CountBatch& b, cudaStream_t s)
{
    const size_t smem = kConsumerWarps * sizeof(CountWarp);
    if (b.n == 0 || b.tile_begin[b.n] == 0) return cudaSuccess;
    k_count_batch<<<b.tile_begin[b.n], kTilePix, smem, s>>>(b);
    return cudaGetLastError();
}

}  // namespace hexfc
