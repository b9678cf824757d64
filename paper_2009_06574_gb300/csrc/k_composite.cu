// Per-pixel depth sort and front-to-back compositing (Section "Method
// Overview": fragments sorted by increasing distance to the camera and
// alpha-blended in visibility order; Section "GPU Implementation": per-pixel
// fragment lists resolved by a sorting pass).
//
// The paper sorts with a per-pixel priority queue. Here the fill pass visits
// each tile's triangles in depth order, so nearly every list arrives sorted:
// one warp stages a list (<= 256 fragments) in shared memory with cp.async
// while it resolves the previous one, checks the order with one comparison
// per element and a vote, and only an out-of-order list is sorted, by a
// warp-wide bitonic network over (key, index) in shared memory. Lists longer
// than 256 (up to HEXFC_MAX_LIST) are sorted by a whole block. Keys are
// unique within a pixel (depth, face, triangle), so the order is unique.
// Compositing is an ordered reduction of (colour, transmittance) pairs,
// (C1,T1)(C2,T2) = (C1 + T1 C2, T1 T2), equal to the sequential
// front-to-back blend.
#include "hexfc_internal.cuh"

namespace hexfc {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarpList = kWarpSortMax;   // per-warp staging capacity (fragments)
constexpr int kWarps = kTilePix / 32;     // warps per composite block

struct CT { float r, g, b, t; };  // premultiplied colour and transmittance

__device__ __forceinline__ CT ct_over(CT a, CT b)  // a in front of b
{
    return CT{a.r + a.t * b.r, a.g + a.t * b.g, a.b + a.t * b.b, a.t * b.t};
}

__device__ __forceinline__ CT warp_ordered_reduce(CT c, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        CT r;
        r.r = __shfl_down_sync(kFull, c.r, o);
        r.g = __shfl_down_sync(kFull, c.g, o);
        r.b = __shfl_down_sync(kFull, c.b, o);
        r.t = __shfl_down_sync(kFull, c.t, o);
        if ((lane & (2 * o - 1)) == 0) c = ct_over(c, r);
    }
    return c;
}

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Per-warp staging buffer of one list.
struct WarpBuf {
    uint64_t key[kWarpList];
    float4 rgba[kWarpList];
    uint16_t idx[kWarpList];
};

__device__ __forceinline__ void stage_list(WarpBuf& b, const uint64_t* __restrict__ key,
                                           const float4* __restrict__ rgba, uint64_t base, uint32_t n, int lane)
{
    for (uint32_t i = lane; i < n; i += 32) {
        cp_async8(&b.key[i], key + base + i);
        cp_async16(&b.rgba[i], rgba + base + i);
    }
}

// Resolve one staged list (n <= kWarpList) with one warp: sort if needed and
// composite front to back. If out_key is given, the sorted list is written.
__device__ CT warp_resolve(WarpBuf& b, uint32_t n, int lane, uint64_t* out_key, float4* out_rgba)
{
    if (n == 0) return CT{0.f, 0.f, 0.f, 1.f};
    const uint32_t M = (n + 31) / 32;
    const uint32_t i0 = lane * M;
    bool inv = false;
    for (uint32_t j = 0; j < M; ++j) {
        uint32_t i = i0 + j;
        if (i + 1 < n && b.key[i + 1] < b.key[i]) inv = true;
    }
    const bool sorted = !__any_sync(kFull, inv);
    if (!sorted) {
        // bitonic network over (key, idx), padded to a power of two >= 32
        uint32_t np2 = 32;
        while (np2 < n) np2 <<= 1;
        for (uint32_t i = lane; i < np2; i += 32) {
            if (i >= n) b.key[i] = kPadKey;
            b.idx[i] = (uint16_t)i;
        }
        __syncwarp();
        for (uint32_t size = 2; size <= np2; size <<= 1)
            for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
                for (uint32_t t = lane; t < np2 / 2; t += 32) {
                    uint32_t i = 2 * stride * (t / stride) + (t % stride);
                    uint32_t p = i + stride;
                    bool up = (i & size) == 0;
                    uint64_t a = b.key[i], c = b.key[p];
                    if (up ? (a > c) : (a < c)) {
                        b.key[i] = c;
                        b.key[p] = a;
                        uint16_t ti = b.idx[i];
                        b.idx[i] = b.idx[p];
                        b.idx[p] = ti;
                    }
                }
                __syncwarp();
            }
    }
    CT c{0.f, 0.f, 0.f, 1.f};
    for (uint32_t j = 0; j < M; ++j) {
        uint32_t r = i0 + j;
        if (r < n) {
            float4 f = b.rgba[sorted ? r : b.idx[r]];
            c = ct_over(c, CT{f.x, f.y, f.z, 1.f - f.w});
            if (out_key) {
                out_key[r] = b.key[r];
                out_rgba[r] = f;
            }
        }
    }
    return warp_ordered_reduce(c, lane);
}

__device__ __forceinline__ void tile_pixel(int64_t q, int tiles_x, int& x, int& y)
{
    int64_t tile = q / kTilePix;
    int local = (int)(q % kTilePix);
    x = (int)(tile % tiles_x) * kTile + (local & (kTile - 1));
    y = (int)(tile / tiles_x) * kTile + local / kTile;
}

// One block per tile; warp w resolves pixels 32w .. 32w+31 of the tile, staging
// the next list while it resolves the current one.
__global__ void __launch_bounds__(kTilePix) k_composite(const uint32_t* __restrict__ cnt,
                                                        const uint64_t* __restrict__ off,
                                                        const uint64_t* __restrict__ key,
                                                        const float4* __restrict__ rgba, int tiles_x, int W, int H,
                                                        float bg0, float bg1, float bg2, float4* __restrict__ out,
                                                        uint32_t* __restrict__ long_q,
                                                        unsigned long long* __restrict__ long_cursor)
{
    extern __shared__ __align__(16) unsigned char smem[];
    WarpBuf* bufs = reinterpret_cast<WarpBuf*>(smem);
    __shared__ uint32_t s_cnt[kTilePix];
    __shared__ uint64_t s_off[kTilePix];
    const int tile = blockIdx.x;
    const int64_t q0 = (int64_t)tile * kTilePix;
    s_cnt[threadIdx.x] = cnt[q0 + threadIdx.x];
    s_off[threadIdx.x] = off[q0 + threadIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WarpBuf* wb = bufs + 2 * warp;
    const int px0 = (tile % tiles_x) * kTile, py0 = (tile / tiles_x) * kTile;
    auto len_of = [&](int p) -> uint32_t {
        uint32_t n = s_cnt[p];
        return n <= (uint32_t)kWarpList ? n : 0u;
    };
    int p = warp * 32;
    stage_list(wb[0], key, rgba, s_off[p], len_of(p), lane);
    cp_async_commit();
    for (int i = 0; i < 32; ++i, ++p) {
        if (i + 1 < 32) {
            stage_list(wb[(i + 1) & 1], key, rgba, s_off[p + 1], len_of(p + 1), lane);
            cp_async_commit();
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncwarp();
        const int x = px0 + (p & (kTile - 1)), y = py0 + p / kTile;
        const uint32_t n = s_cnt[p];
        if (n > (uint32_t)kWarpList) {
            if (lane == 0) long_q[atomicAdd(long_cursor, 1ull)] = (uint32_t)(q0 + p);
        } else if (x < W && y < H) {
            CT c = warp_resolve(wb[i & 1], n, lane, nullptr, nullptr);
            if (lane == 0)
                out[(int64_t)y * W + x] = make_float4(c.r + c.t * bg0, c.g + c.t * bg1, c.b + c.t * bg2, 1.f - c.t);
        }
        __syncwarp();
    }
}

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

__device__ CT block_composite(const uint64_t* __restrict__ key, const float4* __restrict__ rgba, uint64_t base,
                              uint32_t n, uint64_t* s_k, uint32_t* s_v, uint64_t* out_key, float4* out_rgba)
{
    uint32_t np2 = 32;
    while (np2 < n) np2 <<= 1;
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) { s_k[i] = key[base + i]; s_v[i] = i; }
    __syncthreads();
    block_sort(s_k, s_v, n, np2);
    // first warp: each lane composites a contiguous run of ranks, then an ordered reduction
    CT c{0.f, 0.f, 0.f, 1.f};
    if (threadIdx.x < 32) {
        int lane = threadIdx.x;
        uint32_t per = np2 / 32;
        for (uint32_t j = 0; j < per; ++j) {
            uint32_t rank = lane * per + j;
            if (rank < n) {
                float4 f = rgba[base + s_v[rank]];
                c = ct_over(c, CT{f.x, f.y, f.z, 1.f - f.w});
                if (out_key) { out_key[rank] = s_k[rank]; out_rgba[rank] = f; }
            }
        }
        c = warp_ordered_reduce(c, lane);
    }
    return c;
}

__global__ void __launch_bounds__(1024) k_composite_long(const uint32_t* __restrict__ cnt,
                                                         const uint64_t* __restrict__ off,
                                                         const uint64_t* __restrict__ key,
                                                         const float4* __restrict__ rgba,
                                                         const uint32_t* __restrict__ long_q, int tiles_x, int W,
                                                         float bg0, float bg1, float bg2, float4* __restrict__ out)
{
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* s_k = reinterpret_cast<uint64_t*>(smem);
    uint32_t* s_v = reinterpret_cast<uint32_t*>(s_k + HEXFC_MAX_LIST);
    uint32_t q = long_q[blockIdx.x];
    int x, y;
    tile_pixel(q, tiles_x, x, y);
    uint32_t n = cnt[q];
    CT c = block_composite(key, rgba, off[q], n, s_k, s_v, nullptr, nullptr);
    if (threadIdx.x == 0)
        out[(int64_t)y * W + x] = make_float4(c.r + c.t * bg0, c.g + c.t * bg1, c.b + c.t * bg2, 1.f - c.t);
}

// Debug: sorted lists of requested pixels written at dst_off[i], by the same
// resolve routines as the composite (one warp per pixel for n <= 256).
__global__ void __launch_bounds__(256) k_debug_short(const uint32_t* __restrict__ cnt, const uint64_t* __restrict__ off,
                                                     const uint64_t* __restrict__ key,
                                                     const float4* __restrict__ rgba, const int32_t* __restrict__ px,
                                                     const int32_t* __restrict__ py, int64_t n_req,
                                                     const uint64_t* __restrict__ dst_off, int tiles_x,
                                                     uint64_t* __restrict__ out_key, float4* __restrict__ out_rgba)
{
    extern __shared__ __align__(16) unsigned char smem[];
    WarpBuf& b = reinterpret_cast<WarpBuf*>(smem)[threadIdx.x >> 5];
    int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (i >= n_req) return;
    int x = px[i], y = py[i];
    int64_t q = ((int64_t)(y / kTile) * tiles_x + x / kTile) * kTilePix + (y % kTile) * kTile + (x % kTile);
    uint32_t n = cnt[q];
    if (n == 0 || n > (uint32_t)kWarpList) return;
    stage_list(b, key, rgba, off[q], n, lane);
    cp_async_commit();
    cp_async_wait<0>();
    __syncwarp();
    (void)warp_resolve(b, n, lane, out_key + dst_off[i], out_rgba + dst_off[i]);
}

__global__ void __launch_bounds__(1024) k_debug_long(const uint32_t* __restrict__ cnt, const uint64_t* __restrict__ off,
                                                     const uint64_t* __restrict__ key, const float4* __restrict__ rgba,
                                                     const int32_t* __restrict__ px, const int32_t* __restrict__ py,
                                                     const uint64_t* __restrict__ dst_off, int tiles_x,
                                                     uint64_t* __restrict__ out_key, float4* __restrict__ out_rgba)
{
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* s_k = reinterpret_cast<uint64_t*>(smem);
    uint32_t* s_v = reinterpret_cast<uint32_t*>(s_k + HEXFC_MAX_LIST);
    int64_t i = blockIdx.x;
    int x = px[i], y = py[i];
    int64_t q = ((int64_t)(y / kTile) * tiles_x + x / kTile) * kTilePix + (y % kTile) * kTile + (x % kTile);
    uint32_t n = cnt[q];
    if (n <= (uint32_t)kWarpList) return;
    (void)block_composite(key, rgba, off[q], n, s_k, s_v, out_key + dst_off[i], out_rgba + dst_off[i]);
}

__global__ void k_debug_counts(const uint32_t* __restrict__ cnt, const int32_t* __restrict__ px,
                               const int32_t* __restrict__ py, int64_t n_req, int tiles_x,
                               uint32_t* __restrict__ out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_req) return;
    int x = px[i], y = py[i];
    int64_t q = ((int64_t)(y / kTile) * tiles_x + x / kTile) * kTilePix + (y % kTile) * kTile + (x % kTile);
    out[i] = cnt[q];
}

constexpr size_t kLongSmem = (size_t)HEXFC_MAX_LIST * (sizeof(uint64_t) + sizeof(uint32_t));
constexpr size_t kCompositeSmem = 2 * kWarps * sizeof(WarpBuf);

}  // namespace

cudaError_t launch_composite(FrameBufs& fb, const ShadeParams& sp, int tiles_x, int tiles_y, int W, int H, float* out,
                             uint32_t n_long, cudaStream_t s)
{
    float4* o4 = reinterpret_cast<float4*>(out);
    cudaFuncSetAttribute(k_composite, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCompositeSmem);
    k_composite<<<(unsigned)(tiles_x * tiles_y), kTilePix, kCompositeSmem, s>>>(
        fb.cnt, fb.off, fb.key, fb.rgba, tiles_x, W, H, sp.bg[0], sp.bg[1], sp.bg[2], o4, fb.long_q,
        reinterpret_cast<unsigned long long*>(fb.scal + 3));
    if (n_long > 0) {
        cudaFuncSetAttribute(k_composite_long, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLongSmem);
        k_composite_long<<<n_long, 1024, kLongSmem, s>>>(fb.cnt, fb.off, fb.key, fb.rgba, fb.long_q, tiles_x, W,
                                                         sp.bg[0], sp.bg[1], sp.bg[2], o4);
    }
    return cudaGetLastError();
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
    const size_t dsm = 8 * sizeof(WarpBuf);
    cudaFuncSetAttribute(k_debug_short, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm);
    k_debug_short<<<(unsigned)((n * 32 + 255) / 256), 256, dsm, s>>>(fb.cnt, fb.off, fb.key, fb.rgba, d_px, d_py, n,
                                                                    d_dst_off, tiles_x, d_keys, d_rgba);
    cudaFuncSetAttribute(k_debug_long, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLongSmem);
    k_debug_long<<<(unsigned)n, 1024, kLongSmem, s>>>(fb.cnt, fb.off, fb.key, fb.rgba, d_px, d_py, d_dst_off,
                                                      tiles_x, d_keys, d_rgba);
    return cudaGetLastError();
}

}  // namespace hexfc
