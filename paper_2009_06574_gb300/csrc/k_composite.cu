// Per-pixel depth sort and front-to-back compositing (Section "Method
// Overview": fragments sorted by increasing distance to the camera and
// alpha-blended in visibility order; Section "GPU Implementation": per-pixel
// fragment lists resolved by a sorting pass).
//
// The paper sorts with a per-pixel priority queue; here a list of n <= 256
// fragments is sorted by one warp with a bitonic network held in registers
// (32*M slots, M = 1, 2, 4 or 8 per lane), carrying the fragment's index in
// its list; longer lists (up to HEXFC_MAX_LIST) go to a block-wide bitonic
// sort in shared memory. Keys are unique within a pixel (depth, face,
// triangle), so the order is unique. Compositing is an ordered reduction of
// (colour, transmittance) pairs, (C1,T1)(C2,T2) = (C1 + T1 C2, T1 T2), which
// equals the sequential front-to-back blend.
#include "hexfc_internal.cuh"

namespace hexfc {
namespace {

constexpr unsigned kFull = 0xffffffffu;

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

// Load, sort and (optionally) composite one pixel list with one warp.
template <int M>
__device__ __forceinline__ CT warp_pixel(const uint64_t* __restrict__ key, const float4* __restrict__ rgba,
                                         uint64_t base, uint32_t n, int lane, uint64_t* out_key, float4* out_rgba)
{
    uint64_t k[M];
    uint32_t v[M];
#pragma unroll
    for (int j = 0; j < M; ++j) {  // striped, coalesced load; the network does not care where keys start
        uint32_t i = j * 32 + lane;
        k[j] = i < n ? key[base + i] : kPadKey;
        v[j] = i;
    }
    warp_bitonic<M>(k, v, lane);
    CT c{0.f, 0.f, 0.f, 1.f};
#pragma unroll
    for (int j = 0; j < M; ++j) {
        uint32_t rank = lane * M + j;
        if (rank < n) {
            float4 f = rgba[base + v[j]];
            c = ct_over(c, CT{f.x, f.y, f.z, 1.f - f.w});
            if (out_key) {
                out_key[rank] = k[j];
                out_rgba[rank] = f;
            }
        }
    }
    return warp_ordered_reduce(c, lane);
}

__device__ __forceinline__ CT warp_pixel_any(const uint64_t* __restrict__ key, const float4* __restrict__ rgba,
                                             uint64_t base, uint32_t n, int lane, uint64_t* ok, float4* orgba)
{
    if (n <= 32) return warp_pixel<1>(key, rgba, base, n, lane, ok, orgba);
    if (n <= 64) return warp_pixel<2>(key, rgba, base, n, lane, ok, orgba);
    if (n <= 128) return warp_pixel<4>(key, rgba, base, n, lane, ok, orgba);
    return warp_pixel<8>(key, rgba, base, n, lane, ok, orgba);
}

__device__ __forceinline__ void tile_pixel(int64_t q, int tiles_x, int& x, int& y)
{
    int64_t tile = q / kTilePix;
    int local = (int)(q % kTilePix);
    x = (int)(tile % tiles_x) * kTile + (local & (kTile - 1));
    y = (int)(tile / tiles_x) * kTile + local / kTile;
}

__global__ void __launch_bounds__(256) k_composite(const uint32_t* __restrict__ cnt, const uint64_t* __restrict__ off,
                                                   const uint64_t* __restrict__ key, const float4* __restrict__ rgba,
                                                   int64_t n_pix, int tiles_x, int W, int H, float bg0, float bg1,
                                                   float bg2, float4* __restrict__ out, uint32_t* __restrict__ long_q,
                                                   unsigned long long* __restrict__ long_cursor)
{
    int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (q >= n_pix) return;
    int x, y;
    tile_pixel(q, tiles_x, x, y);
    if (x >= W || y >= H) return;
    uint32_t n = cnt[q];
    if (n > (uint32_t)kWarpSortMax) {
        if (lane == 0) long_q[atomicAdd(long_cursor, 1ull)] = (uint32_t)q;
        return;
    }
    CT c{0.f, 0.f, 0.f, 1.f};
    if (n > 0) c = warp_pixel_any(key, rgba, off[q], n, lane, nullptr, nullptr);
    if (lane == 0)
        out[(int64_t)y * W + x] = make_float4(c.r + c.t * bg0, c.g + c.t * bg1, c.b + c.t * bg2, 1.f - c.t);
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

// Debug: sorted lists of requested pixels, written at d_dst_off[i] (warp per pixel).
__global__ void k_debug_short(const uint32_t* __restrict__ cnt, const uint64_t* __restrict__ off,
                              const uint64_t* __restrict__ key, const float4* __restrict__ rgba,
                              const int32_t* __restrict__ px, const int32_t* __restrict__ py, int64_t n_req,
                              const uint64_t* __restrict__ dst_off, int tiles_x, int W, int H,
                              uint64_t* __restrict__ out_key, float4* __restrict__ out_rgba)
{
    int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (i >= n_req) return;
    int x = px[i], y = py[i];
    int64_t q = ((int64_t)(y / kTile) * tiles_x + x / kTile) * kTilePix + (y % kTile) * kTile + (x % kTile);
    uint32_t n = cnt[q];
    if (n == 0 || n > (uint32_t)kWarpSortMax) return;
    (void)warp_pixel_any(key, rgba, off[q], n, lane, out_key + dst_off[i], out_rgba + dst_off[i]);
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
    if (n <= (uint32_t)kWarpSortMax) return;
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

}  // namespace

cudaError_t launch_composite(FrameBufs& fb, const ShadeParams& sp, int tiles_x, int tiles_y, int W, int H, float* out,
                             uint32_t n_long, cudaStream_t s)
{
    int64_t n_pix = (int64_t)tiles_x * tiles_y * kTilePix;
    unsigned blocks = (unsigned)((n_pix * 32 + 255) / 256);
    float4* o4 = reinterpret_cast<float4*>(out);
    k_composite<<<blocks, 256, 0, s>>>(fb.cnt, fb.off, fb.key, fb.rgba, n_pix, tiles_x, W, H, sp.bg[0], sp.bg[1],
                                       sp.bg[2], o4, fb.long_q, reinterpret_cast<unsigned long long*>(fb.scal + 3));
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
    if (n <= 0) return cudaSuccess;
    if (d_counts) {
        k_debug_counts<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(fb.cnt, d_px, d_py, n, tiles_x, d_counts);
        return cudaGetLastError();
    }
    k_debug_short<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(fb.cnt, fb.off, fb.key, fb.rgba, d_px, d_py, n,
                                                                 d_dst_off, tiles_x, W, H, d_keys, d_rgba);
    cudaFuncSetAttribute(k_debug_long, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLongSmem);
    k_debug_long<<<(unsigned)n, 1024, kLongSmem, s>>>(fb.cnt, fb.off, fb.key, fb.rgba, d_px, d_py, d_dst_off,
                                                      tiles_x, d_keys, d_rgba);
    return cudaGetLastError();
}

}  // namespace hexfc
