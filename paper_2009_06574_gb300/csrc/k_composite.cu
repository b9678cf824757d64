// Per-pixel depth sort and front-to-back compositing (Section "Method
// Overview": fragments sorted by increasing distance to the camera and
// alpha-blended in visibility order; Section "GPU Implementation": per-pixel
// fragment lists resolved by a sorting pass).
//
// The paper sorts with a per-pixel priority queue. Here the fill pass visits
// each tile's triangles in depth order, so every list arrives sorted or nearly
// sorted. Layout: for each chunk of 32 triangles of a tile's list and each
// group of 32 pixels of the tile (a warp, tile-major pixel order), the
// group's fragments of that chunk are one run of records, pixel by pixel,
// each pixel's in list order; seg gives the run's first record. A pixel finds
// its fragments of a chunk from the chunk's coverage masks: its own bit
// count, after those of the lower pixels of its group. One thread per pixel walks the chunks and streams its list
// front to back through a small sorted window in registers, checking the
// order of what it blends; a list the window cannot sort is gathered and
// resolved by a whole warp: a bitonic network over (key, index) in registers.
// Lists longer than 256 (up to HEXFC_MAX_LIST) are sorted by a whole block in
// shared memory. Keys are unique within a pixel (depth, face, triangle), so
// the order is unique.
// Every path blends a list front to back one element after the other (the
// warp-wide paths pass the running colour from lane to lane), so the image
// does not depend on which path resolved a list, bit for bit.
#include "hexfc_internal.cuh"
#include "pipeline.cuh"

namespace hexfc {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kGroups = kTilePix / 32;   // warp groups of 32 pixels per tile
constexpr int kWarpList = kWarpSortMax;   // longest list a warp resolves

struct CT { float r, g, b, t; };  // premultiplied colour and transmittance

__device__ __forceinline__ CT ct_over(CT a, CT b)  // a in front of b
{
    return CT{a.r + a.t * b.r, a.g + a.t * b.g, a.b + a.t * b.b, a.t * b.t};
}

// Front-to-back blend of a sorted list whose ranks are held by the lanes in
// runs, lane 0's first: each lane in turn blends its run onto the running
// colour, run(c) returning c after its elements. This is the same sequence of
// ct_over steps as one thread blending the whole list, so every resolve path
// gives the same image bit for bit, whichever path a list takes.
template <class F>
__device__ __forceinline__ CT warp_chain_blend(int lane, F&& run)
{
    CT c{0.f, 0.f, 0.f, 1.f};
    for (int l = 0; l < 32; ++l) {
        if (lane == l) c = run(c);
        c.r = __shfl_sync(kFull, c.r, l);
        c.g = __shfl_sync(kFull, c.g, l);
        c.b = __shfl_sync(kFull, c.b, l);
        c.t = __shfl_sync(kFull, c.t, l);
    }
    return c;
}

// ---------------------------------------------------------------- resolve

__device__ __forceinline__ uint64_t shfl_xor_u64(uint64_t v, int m)
{
    uint32_t lo = (uint32_t)v, hi = (uint32_t)(v >> 32);
    lo = __shfl_xor_sync(kFull, lo, m);
    hi = __shfl_xor_sync(kFull, hi, m);
    return ((uint64_t)hi << 32) | lo;
}

// Bitonic sort of 32*M (key, idx) pairs across a warp, blocked layout: after
// the call lane L holds ranks L*M .. L*M+M-1 in k[0..M-1].
template <int M>
__device__ __forceinline__ void warp_bitonic(uint64_t (&k)[M], uint32_t (&v)[M], int lane)
{
#pragma unroll
    for (int size = 2; size <= 32 * M; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride >= M) {
                const int ls = stride / M;
#pragma unroll
                for (int j = 0; j < M; ++j) {
                    int i = lane * M + j;
                    uint64_t ok = shfl_xor_u64(k[j], ls);
                    uint32_t ov = __shfl_xor_sync(kFull, v[j], ls);
                    bool up = (i & size) == 0;
                    bool lower = (i & stride) == 0;
                    bool take = (lower == up) ? (ok < k[j]) : (ok > k[j]);
                    if (take) { k[j] = ok; v[j] = ov; }
                }
            } else {
#pragma unroll
                for (int j = 0; j < M; ++j) {
                    if ((j & stride) == 0) {
                        const int jj = j | stride;
                        int i = lane * M + j;
                        bool up = (i & size) == 0;
                        bool sw = up ? (k[j] > k[jj]) : (k[j] < k[jj]);
                        if (sw) {
                            uint64_t tk = k[j]; k[j] = k[jj]; k[jj] = tk;
                            uint32_t tv = v[j]; v[j] = v[jj]; v[jj] = tv;
                        }
                    }
                }
            }
        }
    }
}

// Out-of-order list: sort (key, index) in registers, composite by index.
template <int M>
__device__ __noinline__ CT warp_sort_resolve(const uint64_t* key, const float4* rgba, uint32_t n, int lane,
                                             uint64_t* out_key, float4* out_rgba)
{
    uint64_t k[M];
    uint32_t v[M];
#pragma unroll
    for (int j = 0; j < M; ++j) {
        uint32_t i = j * 32 + lane;
        k[j] = i < n ? key[i] : kPadKey;
        v[j] = i;
    }
    warp_bitonic<M>(k, v, lane);
    return warp_chain_blend(lane, [&](CT c) {
#pragma unroll
        for (int j = 0; j < M; ++j) {
            const uint32_t r = lane * M + j;
            if (r < n) {
                const float4 f = rgba[v[j]];
                c = ct_over(c, CT{f.x, f.y, f.z, 1.f - f.w});
                if (out_key) {
                    out_key[r] = k[j];
                    out_rgba[r] = f;
                }
            }
        }
        return c;
    });
}

// Resolve one list of n <= kWarpList fragments held in shared memory (key[i],
// rgba[i], read only) with one warp: check the order, sort if needed, and
// composite front to back. If out_key is given, the sorted list is written.
__device__ CT warp_resolve(const uint64_t* key, const float4* rgba, uint32_t n, int lane, uint64_t* out_key,
                           float4* out_rgba)
{
    if (n == 0) return CT{0.f, 0.f, 0.f, 1.f};
    const uint32_t M = (n + 31) / 32;
    const uint32_t i0 = lane * M;
    bool inv = false;
    for (uint32_t j = 0; j < M; ++j) {
        uint32_t i = i0 + j;
        if (i + 1 < n && key[i + 1] < key[i]) inv = true;
    }
    if (__any_sync(kFull, inv)) {
        if (M == 1) return warp_sort_resolve<1>(key, rgba, n, lane, out_key, out_rgba);
        if (M == 2) return warp_sort_resolve<2>(key, rgba, n, lane, out_key, out_rgba);
        if (M <= 4) return warp_sort_resolve<4>(key, rgba, n, lane, out_key, out_rgba);
        return warp_sort_resolve<8>(key, rgba, n, lane, out_key, out_rgba);
    }
    return warp_chain_blend(lane, [&](CT c) {
        for (uint32_t j = 0; j < M; ++j) {
            const uint32_t r = i0 + j;
            if (r < n) {
                const float4 f = rgba[r];
                c = ct_over(c, CT{f.x, f.y, f.z, 1.f - f.w});
                if (out_key) {
                    out_key[r] = key[r];
                    out_rgba[r] = f;
                }
            }
        }
        return c;
    });
}

__device__ __forceinline__ void tile_pixel(int64_t q, int tiles_x, int& x, int& y)
{
    int64_t tile = q / kTilePix;
    int local = (int)(q % kTilePix);
    x = (int)(tile % tiles_x) * kTileW + local % kTileW;
    y = (int)(tile / tiles_x) * kTileH + local / kTileW;
}

// The fragments of pixel q, in list order, found by one whole warp (lane i
// reads the masks of pixel i of q's group): f(i, e) for list element i at
// fragment index e. Elements past `limit`, or at an index past frag_cap
// (inconsistent runs), are skipped.
template <class F>
__device__ __forceinline__ void list_walk(const uint64_t* __restrict__ tile_off, const uint32_t* __restrict__ masks,
                                          const uint64_t* __restrict__ seg, uint64_t frag_cap, uint32_t q, int lane,
                                          uint32_t limit, F&& f)
{
    const uint32_t tile = q / kTilePix, l = q & 31u, g0 = q - l, grp = (g0 % kTilePix) / 32;
    const uint64_t cb = tile_off[tile] / kChunk, ce = tile_off[tile + 1] / kChunk;
    const uint32_t* mp = masks + cb * kTilePix + (g0 % kTilePix) + lane;
    uint32_t k = 0;
    // eight chunks at a time: their masks and run starts are loaded together
    for (uint64_t c0 = cb; c0 < ce; c0 += 8, mp += 8 * kTilePix) {
        uint32_t mm[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) mm[i] = c0 + i < ce ? mp[i * kTilePix] : 0u;
        const uint64_t cl = c0 + (uint64_t)(lane & 7);
        const unsigned long long sgl = cl < ce ? seg[cl * kGroups + grp] : 0ull;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const uint32_t h = __popc(mm[i]);
            const uint32_t before = __reduce_add_sync(kFull, (uint32_t)lane < l ? h : 0u);
            const uint32_t hl = __shfl_sync(kFull, h, l);
            const uint64_t sg = __shfl_sync(kFull, sgl, i);
            if (hl == 0) continue;
            const uint64_t e = sg + before;
            for (uint32_t t = lane; t < hl; t += 32)
                if (k + t < limit && e + t < frag_cap) f(k + t, e + t);   // (records beyond the arrays: skipped)
            k += hl;
        }
    }
}

struct WarpList {  // staging of one list per warp (out-of-order lists, debug gather)
    uint64_t key[kWarpList];
    float4 rgba[kWarpList];
};

__device__ __forceinline__ float4 finish(CT c, float bg0, float bg1, float bg2)
{
    return make_float4(c.r + c.t * bg0, c.g + c.t * bg1, c.b + c.t * bg2, 1.f - c.t);
}

// One block per tile, one thread per pixel: the thread walks the tile's
// chunks (its fragments of a chunk start at the group's run of that chunk,
// after those of the lower pixels of the group) and streams its list through
// a sorted window of KW (key, colour) pairs in registers, blending the
// smallest pair each time the window overflows, so a list whose elements sit
// at most KW - 1 places from their sorted position comes out sorted. The blend checks that the keys it consumes increase; a
// list that breaks that is queued for the warp-wide resolve of
// k_composite_fix, or, if longer than 256, for the block-wide sort of
// k_composite_long. KW (2, 4 or 8) trades registers and moves for fewer
// queued lists; the result does not depend on it.
struct KC {
    uint64_t k;
    float4 c;
};

__device__ __forceinline__ void kc_sort2(KC& a, KC& b)  // (a, b) -> (min, max)
{
    const bool sw = b.k < a.k;
    const KC lo = sw ? b : a, hi = sw ? a : b;
    a = lo;
    b = hi;
}

__device__ __forceinline__ void blend_checked(CT& c, uint64_t& last, bool& ok, const KC& e)
{
    ok = ok && e.k > last;
    last = e.k;
    c = ct_over(c, CT{e.c.x, e.c.y, e.c.z, 1.f - e.c.w});
}

// Output index of drawn pixel (x, y), if it belongs to the output window.
__device__ __forceinline__ bool out_index(const OutWin& w, int x, int y, int64_t& o)
{
    const int u = x - w.x0, v = y - w.y0;
    if (u < 0 || v < 0 || u >= w.w || v >= w.h) return false;
    o = (int64_t)v * w.w + u;
    return true;
}

// The main resolve pass of one tile (the body of k_composite and k_composite_batch).
template <int KW>
__device__ __forceinline__ void composite_tile(int tile, const uint32_t* __restrict__ cnt,
                                               const uint64_t* __restrict__ seg,
                                               const uint64_t* __restrict__ tile_off,
                                               const uint32_t* __restrict__ masks,
                                               const uint64_t* __restrict__ key,
                                               const float4* __restrict__ rgba, uint64_t frag_cap, int tiles_x,
                                               int W, int H, float bg0, float bg1, float bg2,
                                               float4* __restrict__ out, const OutWin& win,
                                               uint32_t* __restrict__ long_q,
                                               unsigned long long* __restrict__ long_cursor,
                                               uint32_t* __restrict__ fix_q,
                                               unsigned long long* __restrict__ fix_cursor)
{
    const int lane = threadIdx.x & 31;
    const int64_t q = (int64_t)tile * kTilePix + threadIdx.x;
    const uint64_t cb = tile_off[tile] / kChunk;
    const uint32_t n_chunks = (uint32_t)(tile_off[tile + 1] / kChunk - cb);
    const uint64_t* sp = seg + cb * kGroups + (threadIdx.x >> 5);   // the group's record of each chunk
    const uint32_t n = cnt[q];
    CT c{0.f, 0.f, 0.f, 1.f};
    bool ok = true;
    uint64_t last = 0;   // keys are > 0 unless depth and face id are both 0, which the check then flags
    // the window w[0] <= ... <= w[KW-1]; empty places hold the largest key
    const uint64_t kPad = ~0ull;
    KC w[KW];
#pragma unroll
    for (int k = 0; k < KW; ++k) w[k] = KC{kPad, {}};
    uint32_t seen = 0;
    const uint32_t* mp = masks + cb * kTilePix + threadIdx.x;
    uint32_t mk_next = n_chunks > 0 ? mp[0] : 0u;   // the next chunk's mask and record are in flight
    uint64_t sg_next = n_chunks > 0 ? sp[0] : 0u;
    for (uint32_t ch = 0; ch < n_chunks; ++ch) {
        const uint32_t m = mk_next;
        const uint64_t sg = sg_next;
        if (ch + 1 < n_chunks) {
            mk_next = mp[(uint64_t)(ch + 1) * kTilePix];
            sg_next = sp[(uint64_t)(ch + 1) * kGroups];
        }
        const uint32_t h = __popc(m);
        uint32_t incl = h;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        // The group reads its region chunk after chunk, each run right after
        // the last: the 128 records from 24 past the end of this chunk's run
        // are brought into L2 while the chunk is placed (lanes 0-7 a key line
        // each, 8-23 a colour line each). Placing the span by the run start
        // of the next chunk waits for that load; wider spans measured slower.
        {
            const uint64_t nb = sg + __shfl_sync(kFull, incl, 31) + 24;
            if (lane < 24) {
                const uint64_t r = lane < 8 ? nb + 16 * (uint64_t)lane : nb + 8 * (uint64_t)(lane - 8);
                if (r < frag_cap) {
                    const void* a = lane < 8 ? (const void*)(key + r) : (const void*)(rgba + r);
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
                }
            }
        }
        if (h == 0) continue;
        const uint64_t e = sg + incl - h;
        if (e + h > frag_cap) {   // inconsistent run: not read (the list is sent to the checked resolve)
            ok = false;
            continue;
        }
        KC nx{};   // the next element is loaded while this one is placed
        if (h > 0) nx = KC{key[e], rgba[e]};
        for (uint32_t t = 0; t < h; ++t) {
            const KC f = nx;
            if (t + 1 < h) nx = KC{key[e + t + 1], rgba[e + t + 1]};
            const bool full = seen >= (uint32_t)KW;
            ++seen;
            if (full && f.k < w[0].k) {   // smaller than the whole window: blend it at once
                blend_checked(c, last, ok, f);
            } else if (full && f.k > w[KW - 1].k) {   // in order (the common case): append
                blend_checked(c, last, ok, w[0]);
#pragma unroll
                for (int k = 0; k + 1 < KW; ++k) w[k] = w[k + 1];
                w[KW - 1] = f;
            } else {                      // blend the window's minimum (once full), insert f
                if (full) {
                    blend_checked(c, last, ok, w[0]);
#pragma unroll
                    for (int k = 0; k + 1 < KW; ++k) w[k] = w[k + 1];
                }
                w[KW - 1] = f;
#pragma unroll
                for (int k = KW - 1; k > 0; --k) kc_sort2(w[k - 1], w[k]);
            }
        }
    }
    const uint32_t pre = seen < (uint32_t)KW ? seen : (uint32_t)KW;
#pragma unroll
    for (int k = 0; k < KW; ++k)
        if ((uint32_t)k < pre) blend_checked(c, last, ok, w[k]);
    ok = ok && seen == n;
    int x, y;
    tile_pixel(q, tiles_x, x, y);
    if (x >= W || y >= H) return;
    int64_t o;
    if (!out_index(win, x, y, o)) return;   // an apron pixel: only its depth is used
    if (ok) out[o] = finish(c, bg0, bg1, bg2);
    else if (n > (uint32_t)kWarpList) long_q[atomicAdd(long_cursor, 1ull)] = (uint32_t)q;
    else fix_q[atomicAdd(fix_cursor, 1ull)] = (uint32_t)q;
}

template <int KW>
__global__ void __launch_bounds__(256) k_composite(const uint32_t* __restrict__ cnt,
                                                   const uint64_t* __restrict__ seg,
                                                   const uint64_t* __restrict__ tile_off,
                                                   const uint32_t* __restrict__ masks,
                                                   const uint64_t* __restrict__ key,
                                                   const float4* __restrict__ rgba, uint64_t frag_cap, int tiles_x,
                                                   int W, int H, float bg0, float bg1, float bg2,
                                                   float4* __restrict__ out, OutWin win,
                                                   uint32_t* __restrict__ long_q,
                                                   unsigned long long* __restrict__ long_cursor,
                                                   uint32_t* __restrict__ fix_q,
                                                   unsigned long long* __restrict__ fix_cursor)
{
    composite_tile<KW>(blockIdx.x, cnt, seg, tile_off, masks, key, rgba, frag_cap, tiles_x, W, H, bg0, bg1, bg2, out,
                       win, long_q, long_cursor, fix_q, fix_cursor);
}

// The main resolve pass of several frames in one grid (a batch); tiles in
// index order within a frame, as k_composite takes them.
template <int KW>
__global__ void __launch_bounds__(256, KW == 2 ? 4 : (KW == 4 ? 3 : 2))
k_composite_batch(const __grid_constant__ CompositeBatch b)
{
    __shared__ CompositeItem s_it;   // the frame's pointers and constants, read from shared memory
    const int i = batch_item(b.tile_begin, b.n, blockIdx.x);
    if (threadIdx.x == 0) s_it = b.it[i];
    __syncthreads();
    const CompositeItem& it = s_it;
    composite_tile<KW>((int)(blockIdx.x - b.tile_begin[i]), it.cnt, it.seg, it.tile_off, it.masks, it.key, it.rgba,
                       it.frag_cap, it.tiles_x, it.W, it.H, it.bg[0], it.bg[1], it.bg[2], it.out, it.win, it.long_q,
                       it.long_cursor, it.fix_q, it.fix_cursor);
}

// Out-of-order lists (n <= 256): one warp each, gathered into shared memory
// and sorted in registers.
__global__ void __launch_bounds__(256) k_composite_fix(const uint32_t* __restrict__ cnt,
                                                       const uint64_t* __restrict__ seg,
                                                       const uint64_t* __restrict__ tile_off,
                                                       const uint32_t* __restrict__ masks,
                                                       const uint64_t* __restrict__ key,
                                                       const float4* __restrict__ rgba, uint64_t frag_cap,
                                                       int tiles_x, float bg0, float bg1, float bg2,
                                                       float4* __restrict__ out, OutWin win,
                                                       const uint32_t* __restrict__ fix_q,
                                                       const unsigned long long* __restrict__ fix_cursor)
{
    extern __shared__ __align__(16) unsigned char smem[];
    WarpList& b = reinterpret_cast<WarpList*>(smem)[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const uint64_t n_fix = *fix_cursor;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x / 32);
    for (uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; w < n_fix; w += warps) {
        const uint32_t q = fix_q[w];
        const uint32_t n = min(cnt[q], (uint32_t)kWarpList);
        list_walk(tile_off, masks, seg, frag_cap, q, lane, n, [&](uint32_t i, uint64_t e) {
            b.key[i] = key[e];
            b.rgba[i] = rgba[e];
        });
        __syncwarp();
        int x, y;
        tile_pixel(q, tiles_x, x, y);
        CT c = warp_resolve(b.key, b.rgba, n, lane, nullptr, nullptr);
        int64_t o;
        if (lane == 0 && out_index(win, x, y, o)) out[o] = finish(c, bg0, bg1, bg2);
        __syncwarp();   // the staging is reused by the warp's next list
    }
}

// ---------------------------------------------------------------- long lists

// Block-wide bitonic sort of a long list in shared memory (n <= HEXFC_MAX_LIST).
__device__ void block_sort(uint64_t* s_k, uint32_t* s_v, uint32_t n, uint32_t np2)
{
    for (uint32_t i = threadIdx.x; i < np2; i += blockDim.x)
        if (i >= n) { s_k[i] = kPadKey; s_v[i] = i; }
    __syncthreads();
    for (uint32_t size = 2; size <= np2; size <<= 1)
        for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
            for (uint32_t i = threadIdx.x; i < np2; i += blockDim.x) {
                uint32_t p = i ^ stride;
                if (p > i) {
                    bool up = (i & size) == 0;
                    uint64_t a = s_k[i], b = s_k[p];
                    if (up ? (a > b) : (a < b)) {
                        s_k[i] = b; s_k[p] = a;
                        uint32_t t = s_v[i]; s_v[i] = s_v[p]; s_v[p] = t;
                    }
                }
            }
            __syncthreads();
        }
}

// List of pixel q (n <= HEXFC_MAX_LIST elements): the first warp finds the
// elements' fragment indices (relative to the group's region) in s_e, then the
// block sorts (key, element) pairs and the first warp composites.
__device__ CT block_composite(const uint64_t* __restrict__ tile_off, const uint32_t* __restrict__ masks,
                              const uint64_t* __restrict__ seg, uint64_t frag_cap, const uint64_t* __restrict__ key,
                              const float4* __restrict__ rgba, uint32_t q, uint32_t n, uint64_t* s_k, uint32_t* s_v,
                              uint64_t* s_e, uint64_t* out_key, float4* out_rgba)
{
    uint32_t np2 = 32;
    while (np2 < n) np2 <<= 1;
    if (threadIdx.x < 32) {
        for (uint32_t i = threadIdx.x; i < n; i += 32) s_e[i] = 0;   // elements a walk may skip
        __syncwarp();
        list_walk(tile_off, masks, seg, frag_cap, q, (int)threadIdx.x, n,
                  [&](uint32_t i, uint64_t e) { s_e[i] = e; });
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) { s_k[i] = key[s_e[i]]; s_v[i] = i; }
    __syncthreads();
    block_sort(s_k, s_v, n, np2);
    // first warp: the lanes blend contiguous runs of ranks in turn
    CT c{0.f, 0.f, 0.f, 1.f};
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const uint32_t per = np2 / 32;
        c = warp_chain_blend(lane, [&](CT a) {
            for (uint32_t j = 0; j < per; ++j) {
                const uint32_t rank = lane * per + j;
                if (rank < n) {
                    const float4 f = rgba[s_e[s_v[rank]]];
                    a = ct_over(a, CT{f.x, f.y, f.z, 1.f - f.w});
                    if (out_key) { out_key[rank] = s_k[rank]; out_rgba[rank] = f; }
                }
            }
            return a;
        });
    }
    return c;
}

// Lists longer than 256: one block each, queued by k_composite (the queue
// length is read on the device, so the grid need not match it). A list above
// HEXFC_MAX_LIST is never drawn; the frame reports it as an overflow.
__global__ void __launch_bounds__(1024) k_composite_long(const uint32_t* __restrict__ cnt,
                                                         const uint64_t* __restrict__ seg,
                                                         const uint64_t* __restrict__ tile_off,
                                                         const uint32_t* __restrict__ masks,
                                                         const uint64_t* __restrict__ key,
                                                         const float4* __restrict__ rgba, uint64_t frag_cap,
                                                         const uint32_t* __restrict__ long_q,
                                                         const unsigned long long* __restrict__ n_long,
                                                         int tiles_x, float bg0, float bg1, float bg2,
                                                         float4* __restrict__ out, OutWin win)
{
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* s_k = reinterpret_cast<uint64_t*>(smem);
    uint64_t* s_e = s_k + HEXFC_MAX_LIST;
    uint32_t* s_v = reinterpret_cast<uint32_t*>(s_e + HEXFC_MAX_LIST);
    const unsigned long long total = *n_long;
    for (unsigned long long i = blockIdx.x; i < total; i += gridDim.x) {
        const uint32_t q = long_q[i];
        const uint32_t n = cnt[q];
        if (n > (uint32_t)HEXFC_MAX_LIST) continue;
        int x, y;
        tile_pixel(q, tiles_x, x, y);
        CT c = block_composite(tile_off, masks, seg, frag_cap, key, rgba, q, n, s_k, s_v, s_e, nullptr, nullptr);
        int64_t o;
        if (threadIdx.x == 0 && out_index(win, x, y, o)) out[o] = finish(c, bg0, bg1, bg2);
        __syncthreads();   // the shared arrays are reused by the next list
    }
}

// ---------------------------------------------------------------- silhouettes

// White silhouettes of the boundary surface (Section "Blending Focus and
// Context": the boundary surface is rendered and fragments along sharp edges
// of its depth buffer are emphasised). zsil holds, per drawn pixel (tile-major),
// the 24-bit depth of its nearest boundary-face fragment (kNoDepth: none). An
// output pixel p with a depth is a silhouette pixel if a 4-neighbour inside the
// frame has none (exterior), or if for a neighbour q and the opposite q' (both
// with depths) D(q) - D(p) > T and |D(q) - 2 D(p) + D(q')| > T (interior: the
// near side of a depth jump; a plane, however steep, has no second
// difference); its colour and opacity move towards white by alpha. The drawn
// rectangle starts at frame pixel (fx0, fy0) and holds every in-frame
// neighbour of the output window (an apron around a sub-rectangle).
__device__ __forceinline__ uint32_t zsil_at(const uint32_t* __restrict__ zsil, int tiles_x, int x, int y)
{
    const int64_t t = (int64_t)(y / kTileH) * tiles_x + x / kTileW;
    return zsil[t * kTilePix + (y % kTileH) * kTileW + (x % kTileW)];
}

__global__ void __launch_bounds__(256) k_silhouette(const uint32_t* __restrict__ zsil, int tiles_x, int fx0, int fy0,
                                                    int frame_w, int frame_h, float alpha, int64_t T,
                                                    float4* __restrict__ out, OutWin win)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)win.w * win.h) return;
    const int x = win.x0 + (int)(i % win.w), y = win.y0 + (int)(i / win.w);
    const uint32_t zp = zsil_at(zsil, tiles_x, x, y);
    if (zp == kNoDepth) return;
    const int dx[4] = {1, -1, 0, 0}, dy[4] = {0, 0, 1, -1};   // k ^ 1: the opposite side
    int64_t zq[4];
    bool has[4];
    bool sil = false;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int qx = x + dx[k], qy = y + dy[k];
        const bool inside = qx + fx0 >= 0 && qy + fy0 >= 0 && qx + fx0 < frame_w && qy + fy0 < frame_h;
        const uint32_t z = inside ? zsil_at(zsil, tiles_x, qx, qy) : kNoDepth;
        has[k] = z != kNoDepth;
        zq[k] = (int64_t)z;
        sil = sil || (inside && !has[k]);   // exterior: the surface ends here
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int o = k ^ 1;
        if (has[k] && has[o]) {
            const int64_t d1 = zq[k] - (int64_t)zp, d2 = zq[k] - 2 * (int64_t)zp + zq[o];
            sil = sil || (d1 > T && (d2 > T || -d2 > T));   // interior: the near side of a jump
        }
    }
    if (!sil) return;
    float4 c = out[i];
    c.x = fmaf(alpha, 1.f - c.x, c.x);
    c.y = fmaf(alpha, 1.f - c.y, c.y);
    c.z = fmaf(alpha, 1.f - c.z, c.z);
    c.w = fmaf(alpha, 1.f - c.w, c.w);
    out[i] = c;
}

// ---------------------------------------------------------------- debug gather

// Sorted lists of requested pixels written at dst_off[i], by the same resolve
// routines as the composite (one warp per pixel for n <= 256).
__global__ void __launch_bounds__(256) k_debug_short(const uint32_t* __restrict__ cnt, const uint64_t* __restrict__ seg,
                                                     const uint64_t* __restrict__ tile_off,
                                                     const uint32_t* __restrict__ masks,
                                                     const uint64_t* __restrict__ key,
                                                     const float4* __restrict__ rgba, uint64_t frag_cap,
                                                     const int32_t* __restrict__ px,
                                                     const int32_t* __restrict__ py, int64_t n_req,
                                                     const uint64_t* __restrict__ dst_off, int tiles_x,
                                                     uint64_t* __restrict__ out_key, float4* __restrict__ out_rgba)
{
    extern __shared__ __align__(16) unsigned char smem[];
    WarpList& b = reinterpret_cast<WarpList*>(smem)[threadIdx.x >> 5];
    int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (i >= n_req) return;
    int x = px[i], y = py[i];
    int64_t q = ((int64_t)(y / kTileH) * tiles_x + x / kTileW) * kTilePix + (y % kTileH) * kTileW + (x % kTileW);
    uint32_t n = cnt[q];
    if (n == 0 || n > (uint32_t)kWarpList) return;
    list_walk(tile_off, masks, seg, frag_cap, (uint32_t)q, lane, n, [&](uint32_t k, uint64_t e) {
        b.key[k] = key[e];
        b.rgba[k] = rgba[e];
    });
    __syncwarp();
    (void)warp_resolve(b.key, b.rgba, n, lane, out_key + dst_off[i], out_rgba + dst_off[i]);
}

__global__ void __launch_bounds__(1024) k_debug_long(const uint32_t* __restrict__ cnt, const uint64_t* __restrict__ seg,
                                                     const uint64_t* __restrict__ tile_off,
                                                     const uint32_t* __restrict__ masks,
                                                     const uint64_t* __restrict__ key, const float4* __restrict__ rgba,
                                                     uint64_t frag_cap, const int32_t* __restrict__ px,
                                                     const int32_t* __restrict__ py,
                                                     const uint64_t* __restrict__ dst_off, int tiles_x,
                                                     uint64_t* __restrict__ out_key, float4* __restrict__ out_rgba)
{
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* s_k = reinterpret_cast<uint64_t*>(smem);
    uint64_t* s_e = s_k + HEXFC_MAX_LIST;
    uint32_t* s_v = reinterpret_cast<uint32_t*>(s_e + HEXFC_MAX_LIST);
    int64_t i = blockIdx.x;
    int x = px[i], y = py[i];
    int64_t q = ((int64_t)(y / kTileH) * tiles_x + x / kTileW) * kTilePix + (y % kTileH) * kTileW + (x % kTileW);
    uint32_t n = cnt[q];
    if (n <= (uint32_t)kWarpList || n > (uint32_t)HEXFC_MAX_LIST) return;
    (void)block_composite(tile_off, masks, seg, frag_cap, key, rgba, (uint32_t)q, n, s_k, s_v, s_e,
                          out_key + dst_off[i], out_rgba + dst_off[i]);
}

__global__ void k_debug_counts(const uint32_t* __restrict__ cnt, const int32_t* __restrict__ px,
                               const int32_t* __restrict__ py, int64_t n_req, int tiles_x,
                               uint32_t* __restrict__ out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_req) return;
    int x = px[i], y = py[i];
    int64_t q = ((int64_t)(y / kTileH) * tiles_x + x / kTileW) * kTilePix + (y % kTileH) * kTileW + (x % kTileW);
    out[i] = cnt[q];
}

constexpr size_t kLongSmem = (size_t)HEXFC_MAX_LIST * (2 * sizeof(uint64_t) + sizeof(uint32_t));
constexpr size_t kFixSmem = 8 * sizeof(WarpList);
constexpr unsigned kFixBlocks = 4 * 152;   // persistent: warps stride over the queue of out-of-order lists
constexpr unsigned kLongGridMax = 2 * 152;  // persistent: blocks stride over the queue of long lists

}  // namespace

cudaError_t launch_composite_tail(FrameBufs& fb, const ShadeParams& sp, int tiles_x, float* out, uint32_t n_long,
                                  OutWin win, cudaStream_t s)
{
    float4* o4 = reinterpret_cast<float4*>(out);
    unsigned long long* long_cursor = reinterpret_cast<unsigned long long*>(fb.scal + 3);
    unsigned long long* fix_cursor = reinterpret_cast<unsigned long long*>(fb.scal + 4);
    k_composite_fix<<<kFixBlocks, 256, kFixSmem, s>>>(fb.cnt, fb.seg, fb.tile_off, fb.masks, fb.key, fb.rgba,
                                                      (uint64_t)fb.frag_cap, tiles_x, sp.bg[0], sp.bg[1],
                                                      sp.bg[2], o4, win, fb.fix_q, fix_cursor);
    if (n_long > 0) {   // n_long: the number of long lists if known, else an upper bound on the useful grid
        const unsigned grid = n_long < kLongGridMax ? n_long : kLongGridMax;
        k_composite_long<<<grid, 1024, kLongSmem, s>>>(fb.cnt, fb.seg, fb.tile_off, fb.masks, fb.key, fb.rgba,
                                                       (uint64_t)fb.frag_cap, fb.long_q, long_cursor, tiles_x,
                                                       sp.bg[0], sp.bg[1], sp.bg[2], o4, win);
    }
    return cudaGetLastError();
}

cudaError_t launch_composite(FrameBufs& fb, const ShadeParams& sp, int tiles_x, int tiles_y, int W, int H, float* out,
                             uint32_t n_long, int window, OutWin win, cudaStream_t s)
{
    float4* o4 = reinterpret_cast<float4*>(out);
    const int64_t n_pix = (int64_t)tiles_x * tiles_y * kTilePix;
    unsigned long long* long_cursor = reinterpret_cast<unsigned long long*>(fb.scal + 3);
    unsigned long long* fix_cursor = reinterpret_cast<unsigned long long*>(fb.scal + 4);
    const unsigned grid = (unsigned)(n_pix / kTilePix);
    auto resolve = [&](auto kernel) {
        kernel<<<grid, 256, 0, s>>>(fb.cnt, fb.seg, fb.tile_off, fb.masks, fb.key, fb.rgba, (uint64_t)fb.frag_cap,
                                    tiles_x, W, H, sp.bg[0], sp.bg[1], sp.bg[2], o4, win, fb.long_q, long_cursor,
                                    fb.fix_q, fix_cursor);
    };
    if (window == 8) resolve(k_composite<8>);
    else if (window == 4) resolve(k_composite<4>);
    else resolve(k_composite<2>);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_composite_tail(fb, sp, tiles_x, out, n_long, win, s);
}

cudaError_t launch_composite_batch(const CompositeBatch& b, int window, cudaStream_t s)
{
    if (b.n == 0 || b.tile_begin[b.n] == 0) return cudaSuccess;
    const unsigned grid = b.tile_begin[b.n];
    if (window == 8) k_composite_batch<8><<<grid, 256, 0, s>>>(b);
    else if (window == 4) k_composite_batch<4><<<grid, 256, 0, s>>>(b);
    else k_composite_batch<2><<<grid, 256, 0, s>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_silhouette(FrameBufs& fb, int tiles_x, int fx0, int fy0, int frame_w, int frame_h, float alpha,
                              float threshold, float* out, OutWin win, cudaStream_t s)
{
    const int64_t n = (int64_t)win.w * win.h;
    if (n == 0) return cudaSuccess;
    k_silhouette<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(fb.zsil, tiles_x, fx0, fy0, frame_w, frame_h, alpha,
                                                             (int64_t)threshold, reinterpret_cast<float4*>(out), win);
    return cudaGetLastError();
}

cudaError_t prepare_composite_kernels()
{
    cudaError_t e = cudaFuncSetAttribute(k_composite_long, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLongSmem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_composite_fix, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFixSmem);
}

cudaError_t launch_debug_gather(FrameBufs& fb, const int32_t* d_px, const int32_t* d_py, int64_t n,
                                const uint64_t* d_dst_off, int tiles_x, int W, int H, uint64_t* d_keys,
                                float4* d_rgba, uint32_t* d_counts, cudaStream_t s)
{
    (void)W;
    (void)H;
    if (n <= 0) return cudaSuccess;
    if (d_counts) {
        k_debug_counts<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(fb.cnt, d_px, d_py, n, tiles_x, d_counts);
        return cudaGetLastError();
    }
    const size_t dsm = 8 * sizeof(WarpList);
    cudaFuncSetAttribute(k_debug_short, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm);
    k_debug_short<<<(unsigned)((n * 32 + 255) / 256), 256, dsm, s>>>(fb.cnt, fb.seg, fb.tile_off, fb.masks, fb.key,
                                                                    fb.rgba, (uint64_t)fb.frag_cap, d_px, d_py, n,
                                                                    d_dst_off, tiles_x, d_keys, d_rgba);
    cudaFuncSetAttribute(k_debug_long, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLongSmem);
    k_debug_long<<<(unsigned)n, 1024, kLongSmem, s>>>(fb.cnt, fb.seg, fb.tile_off, fb.masks, fb.key, fb.rgba,
                                                      (uint64_t)fb.frag_cap, d_px,
                                                      d_py, d_dst_off, tiles_x, d_keys, d_rgba);
    return cudaGetLastError();
}

}  // namespace hexfc
