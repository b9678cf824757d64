// Per-pixel depth sort and front-to-back compositing (Section "Method
// Overview": fragments sorted by increasing distance to the camera and
// alpha-blended in visibility order; Section "GPU Implementation": per-pixel
// fragment lists resolved by a sorting pass).
//
// A tile's lists are one contiguous range of the fragment buffers (pixels in
// tile-major order). The composite streams that range through shared memory
// with bulk asynchronous copies (cp.async.bulk, completion on an mbarrier) in
// segments of consecutive pixels, two segments in flight, while the warps
// resolve the pixels of the segment that has landed. The paper sorts with a
// per-pixel priority queue; here the fill pass visits each tile's triangles in
// depth order, so nearly every list arrives sorted: one comparison per element
// and a vote confirm it, and only an out-of-order list is sorted, by a
// warp-wide bitonic network over (key, index) in registers. Lists longer
// than 256 (up to HEXFC_MAX_LIST) are sorted by a whole block. Keys are unique
// within a pixel (depth, face, triangle), so the order is unique. Compositing
// is an ordered reduction of (colour, transmittance) pairs,
// (C1,T1)(C2,T2) = (C1 + T1 C2, T1 T2), equal to the sequential blend.
#include "hexfc_internal.cuh"

namespace hexfc {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarpList = kWarpSortMax;   // longest list a warp resolves
constexpr int kWarps = kTilePix / 32;     // warps per composite block
constexpr int kSegCap = 1024;             // segment target (fragments); a segment spans < kSegCap + kWarpList
constexpr int kStageFrags = kSegCap + kWarpList + 2;   // +2: key copies are widened to 16-byte boundaries
constexpr uint32_t kWaitLimit = 1u << 26; // bounded mbarrier waits

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

// ---------------------------------------------------------------- async copies

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_addr(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
// Waits for phase `parity` of the barrier to complete; false if the bound
// (about half a second of SM clock, or kWaitLimit polls) ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity)
{
    const unsigned a = smem_addr(bar);
    const long long t0 = clock64();
    for (uint32_t it = 0; it < kWaitLimit && clock64() - t0 < (1ll << 30); ++it) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}
__device__ __forceinline__ void bulk_g2s(void* smem, const void* gmem, unsigned bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_addr(smem)),
        "l"(gmem), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

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
    CT c{0.f, 0.f, 0.f, 1.f};
#pragma unroll
    for (int j = 0; j < M; ++j) {
        uint32_t r = lane * M + j;
        if (r < n) {
            float4 f = rgba[v[j]];
            c = ct_over(c, CT{f.x, f.y, f.z, 1.f - f.w});
            if (out_key) {
                out_key[r] = k[j];
                out_rgba[r] = f;
            }
        }
    }
    return warp_ordered_reduce(c, lane);
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
    CT c{0.f, 0.f, 0.f, 1.f};
    for (uint32_t j = 0; j < M; ++j) {
        uint32_t r = i0 + j;
        if (r < n) {
            float4 f = rgba[r];
            c = ct_over(c, CT{f.x, f.y, f.z, 1.f - f.w});
            if (out_key) {
                out_key[r] = key[r];
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

// Shared memory of the composite block.
struct StageBuf {
    uint64_t key[kStageFrags];
    float4 rgba[kStageFrags];
};
struct WarpList {  // fallback staging of one list per warp
    uint64_t key[kWarpList];
    float4 rgba[kWarpList];
};
union CompositeSmem {
    StageBuf stage[2];
    WarpList warp[kWarps];
};

__device__ __forceinline__ float4 finish(CT c, float bg0, float bg1, float bg2)
{
    return make_float4(c.r + c.t * bg0, c.g + c.t * bg1, c.b + c.t * bg2, 1.f - c.t);
}

// One block per tile. Segment k of the tile holds the pixels whose lists end
// in ((k-1) kSegCap, k kSegCap] fragments from the tile's start; it is copied
// whole into stage k % 2 and resolved by the 8 warps, pixel by pixel.
__global__ void __launch_bounds__(kTilePix) k_composite(const uint32_t* __restrict__ cnt,
                                                        const uint64_t* __restrict__ off,
                                                        const uint64_t* __restrict__ key,
                                                        const float4* __restrict__ rgba, int tiles_x, int W, int H,
                                                        float bg0, float bg1, float bg2, float4* __restrict__ out,
                                                        uint32_t* __restrict__ long_q,
                                                        unsigned long long* __restrict__ long_cursor,
                                                        unsigned long long* __restrict__ err)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    CompositeSmem& sm = *reinterpret_cast<CompositeSmem*>(smem_raw);
    __shared__ uint32_t s_cnt[kTilePix];
    __shared__ uint64_t s_off[kTilePix + 1];
    __shared__ uint16_t s_first[kTilePix * kWarpList / kSegCap + 2];   // first pixel of each segment (+ end)
    __shared__ __align__(8) uint64_t s_bar[2];
    const int tile = blockIdx.x;
    const int64_t q0 = (int64_t)tile * kTilePix;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int px0 = (tile % tiles_x) * kTile, py0 = (tile / tiles_x) * kTile;
    const uint32_t n_me = cnt[q0 + threadIdx.x];
    s_cnt[threadIdx.x] = n_me;
    s_off[threadIdx.x] = off[q0 + threadIdx.x];
    if (threadIdx.x == 0) s_off[kTilePix] = off[q0 + kTilePix];
    const int has_long = __syncthreads_or(n_me > (uint32_t)kWarpList);

    if (has_long) {
        // rare: a list longer than 256 in this tile; warp by warp, one list at a time
        for (int p = warp; p < kTilePix; p += kWarps) {
            const uint32_t n = s_cnt[p];
            const int x = px0 + (p & (kTile - 1)), y = py0 + p / kTile;
            if (n > (uint32_t)kWarpList) {
                if (lane == 0) long_q[atomicAdd(long_cursor, 1ull)] = (uint32_t)(q0 + p);
                continue;
            }
            WarpList& b = sm.warp[warp];
            for (uint32_t i = lane; i < n; i += 32) {
                cp_async8(&b.key[i], key + s_off[p] + i);
                cp_async16(&b.rgba[i], rgba + s_off[p] + i);
            }
            cp_async_commit();
            cp_async_wait_all();
            __syncwarp();
            CT c = warp_resolve(b.key, b.rgba, n, lane, nullptr, nullptr);
            if (lane == 0 && x < W && y < H) out[(int64_t)y * W + x] = finish(c, bg0, bg1, bg2);
            __syncwarp();
        }
        return;
    }

    // segments: pixel p belongs to segment (rel_end(p) - 1) / kSegCap
    const uint64_t base = s_off[0];
    const uint64_t total = s_off[kTilePix] - base;
    const uint32_t n_seg = total == 0 ? 1u : (uint32_t)((total - 1) / kSegCap) + 1u;
    {
        const int p = threadIdx.x;
        const uint64_t re = s_off[p + 1] - base;
        const uint32_t sg = re > 0 ? (uint32_t)((re - 1) / kSegCap) : 0u;
        uint32_t sp = 0;
        if (p > 0) {
            const uint64_t rp = s_off[p] - base;
            sp = rp > 0 ? (uint32_t)((rp - 1) / kSegCap) : 0u;
        }
        if (p == 0) s_first[0] = 0;
        else if (sg != sp) s_first[sg] = (uint16_t)p;
        if (p == 0) s_first[n_seg] = kTilePix;
        if (p == 0) {
            mbar_init(&s_bar[0], 1);
            mbar_init(&s_bar[1], 1);
            asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        }
    }
    __syncthreads();

    // producer: thread 0 copies segment k into stage k % 2
    auto issue = [&](uint32_t k) {
        const uint32_t p_a = s_first[k], p_b = s_first[k + 1];
        const uint64_t f0 = s_off[p_a], f1 = s_off[p_b];
        StageBuf& st = sm.stage[k & 1];
        if (f1 == f0) {  // nothing to copy: complete the phase by a plain arrive
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_addr(&s_bar[k & 1])) : "memory");
            return;
        }
        const uint64_t k0 = f0 & ~1ull, k1 = (f1 + 1) & ~1ull;   // 16-byte aligned key range
        const unsigned kb = (unsigned)((k1 - k0) * sizeof(uint64_t));
        const unsigned rb = (unsigned)((f1 - f0) * sizeof(float4));
        mbar_expect_tx(&s_bar[k & 1], kb + rb);
        bulk_g2s(st.key, key + k0, kb, &s_bar[k & 1]);
        bulk_g2s(st.rgba, rgba + f0, rb, &s_bar[k & 1]);
    };
    if (threadIdx.x == 0) {
        issue(0);
        if (n_seg > 1) issue(1);
    }
    bool timed_out = false;
    for (uint32_t k = 0; k < n_seg; ++k) {
        const uint32_t sidx = k & 1;
        if (!mbar_wait(&s_bar[sidx], (k >> 1) & 1)) timed_out = true;
        StageBuf& st = sm.stage[sidx];
        const uint32_t p_a = s_first[k], p_b = s_first[k + 1];
        const uint64_t kbase = s_off[p_a] & ~1ull, rbase = s_off[p_a];
        for (uint32_t p = p_a + warp; p < p_b; p += kWarps) {
            const uint32_t n = s_cnt[p];
            const int x = px0 + (int)(p & (kTile - 1)), y = py0 + (int)(p / kTile);
            CT c{0.f, 0.f, 0.f, 1.f};
            if (n > 0 && !timed_out)
                c = warp_resolve(st.key + (s_off[p] - kbase), st.rgba + (s_off[p] - rbase), n, lane, nullptr,
                                 nullptr);
            if (lane == 0 && x < W && y < H) out[(int64_t)y * W + x] = finish(c, bg0, bg1, bg2);
        }
        __syncthreads();  // stage sidx is free again
        if (threadIdx.x == 0 && k + 2 < n_seg) {
            fence_proxy_async();  // order the warps' shared-memory accesses before the async overwrite
            issue(k + 2);
        }
    }
    if (timed_out && threadIdx.x == 0) atomicOr(err, 2ull);
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
    if (threadIdx.x == 0) out[(int64_t)y * W + x] = finish(c, bg0, bg1, bg2);
}

// ---------------------------------------------------------------- debug gather

// Sorted lists of requested pixels written at dst_off[i], by the same resolve
// routines as the composite (one warp per pixel for n <= 256).
__global__ void __launch_bounds__(256) k_debug_short(const uint32_t* __restrict__ cnt, const uint64_t* __restrict__ off,
                                                     const uint64_t* __restrict__ key,
                                                     const float4* __restrict__ rgba, const int32_t* __restrict__ px,
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
    int64_t q = ((int64_t)(y / kTile) * tiles_x + x / kTile) * kTilePix + (y % kTile) * kTile + (x % kTile);
    uint32_t n = cnt[q];
    if (n == 0 || n > (uint32_t)kWarpList) return;
    for (uint32_t e = lane; e < n; e += 32) {
        cp_async8(&b.key[e], key + off[q] + e);
        cp_async16(&b.rgba[e], rgba + off[q] + e);
    }
    cp_async_commit();
    cp_async_wait_all();
    __syncwarp();
    (void)warp_resolve(b.key, b.rgba, n, lane, out_key + dst_off[i], out_rgba + dst_off[i]);
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
constexpr size_t kCompositeSmem = sizeof(CompositeSmem);

}  // namespace

cudaError_t launch_composite(FrameBufs& fb, const ShadeParams& sp, int tiles_x, int tiles_y, int W, int H, float* out,
                             uint32_t n_long, cudaStream_t s)
{
    float4* o4 = reinterpret_cast<float4*>(out);
    cudaFuncSetAttribute(k_composite, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCompositeSmem);
    k_composite<<<(unsigned)(tiles_x * tiles_y), kTilePix, kCompositeSmem, s>>>(
        fb.cnt, fb.off, fb.key, fb.rgba, tiles_x, W, H, sp.bg[0], sp.bg[1], sp.bg[2], o4, fb.long_q,
        reinterpret_cast<unsigned long long*>(fb.scal + 3), reinterpret_cast<unsigned long long*>(fb.scal + 5));
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
    const size_t dsm = 8 * sizeof(WarpList);
    cudaFuncSetAttribute(k_debug_short, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm);
    k_debug_short<<<(unsigned)((n * 32 + 255) / 256), 256, dsm, s>>>(fb.cnt, fb.off, fb.key, fb.rgba, d_px, d_py, n,
                                                                    d_dst_off, tiles_x, d_keys, d_rgba);
    cudaFuncSetAttribute(k_debug_long, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLongSmem);
    k_debug_long<<<(unsigned)n, 1024, kLongSmem, s>>>(fb.cnt, fb.off, fb.key, fb.rgba, d_px, d_py, d_dst_off,
                                                      tiles_x, d_keys, d_rgba);
    return cudaGetLastError();
}

}  // namespace hexfc
