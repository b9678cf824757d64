// Exclusive prefix scan of uint32 counts into uint64 offsets, with the total,
// the maximum and the number of entries above a threshold (each count can be
// rounded up to a power of two first). Three phases:
// per-block reduce, scan of the block partials in one block, per-block
// down-sweep. It replaces the global append counter of per-pixel linked lists
// (Section "GPU Implementation") by exact offsets, so that every pixel's
// fragments are contiguous.
#include "hexfc_internal.cuh"

namespace hexfc {
namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanChunk = kScanThreads * kScanItems;   // elements per block

__device__ __forceinline__ uint64_t warp_incl_scan(uint64_t v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Block-wide exclusive scan of one value per thread; returns the block total in *total.
__device__ uint64_t block_excl_scan(uint64_t v, uint64_t* total)
{
    __shared__ uint64_t warp_sums[32];
    __shared__ uint64_t block_total;
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint64_t incl = warp_incl_scan(v, lane);
    if (lane == 31) warp_sums[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int nw = blockDim.x >> 5;
        uint64_t s = lane < nw ? warp_sums[lane] : 0;
        uint64_t si = warp_incl_scan(s, lane);
        if (lane < nw) warp_sums[lane] = si - s;   // exclusive prefix of each warp
        if (lane == nw - 1) block_total = si;
    }
    __syncthreads();
    uint64_t res = incl - v + warp_sums[wid];
    *total = block_total;
    __syncthreads();
    return res;
}

__device__ __forceinline__ uint32_t warp_max(uint32_t v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ uint64_t warp_sum(uint64_t v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t* __restrict__ in, int64_t n,
                                                              uint64_t* __restrict__ part,
                                                              uint32_t* __restrict__ part_max,
                                                              uint32_t long_thr, uint32_t round_mask)
{
    __shared__ uint64_t s_sum[32], s_long[32];
    __shared__ uint32_t s_max[32];
    int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * kScanItems;
    uint64_t sum = 0, nlong = 0;
    uint32_t mx = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        uint32_t v = i < n ? ((in[i] + round_mask) & ~round_mask) : 0u;
        sum += v;
        mx = max(mx, v);
        nlong += v > long_thr ? 1u : 0u;
    }
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    sum = warp_sum(sum);
    nlong = warp_sum(nlong);
    mx = warp_max(mx);
    if (lane == 0) { s_sum[wid] = sum; s_max[wid] = mx; s_long[wid] = nlong; }
    __syncthreads();
    if (wid == 0) {
        int nw = blockDim.x >> 5;
        sum = lane < nw ? s_sum[lane] : 0;
        mx = lane < nw ? s_max[lane] : 0;
        nlong = lane < nw ? s_long[lane] : 0;
        sum = warp_sum(sum);
        mx = warp_max(mx);
        nlong = warp_sum(nlong);
        if (lane == 0) {
            part[2 * blockIdx.x] = sum;
            part[2 * blockIdx.x + 1] = nlong;
            part_max[blockIdx.x] = mx;
        }
    }
}

// One block: exclusive scan of the nb block sums (in place, even slots), totals into scal.
__global__ void __launch_bounds__(kScanThreads) k_scan_partials(uint64_t* __restrict__ part,
                                                                const uint32_t* __restrict__ part_max,
                                                                int64_t nb, uint64_t* __restrict__ scal)
{
    uint64_t carry = 0, nlong = 0;
    uint32_t mx = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += kScanThreads) {
        int64_t b = b0 + threadIdx.x;
        uint64_t v = b < nb ? part[2 * b] : 0;
        uint64_t tot;
        uint64_t ex = block_excl_scan(v, &tot);
        if (b < nb) part[2 * b] = carry + ex;
        carry += tot;
        uint64_t l = b < nb ? part[2 * b + 1] : 0;
        uint64_t ltot;
        (void)block_excl_scan(l, &ltot);
        nlong += ltot;
        uint32_t m = b < nb ? part_max[b] : 0;
        m = warp_max(m);
        __shared__ uint32_t s_m[32];
        if ((threadIdx.x & 31) == 0) s_m[threadIdx.x >> 5] = m;
        __syncthreads();
        if (threadIdx.x < 32) {
            uint32_t mm = threadIdx.x < (blockDim.x >> 5) ? s_m[threadIdx.x] : 0;
            mm = warp_max(mm);
            if (threadIdx.x == 0) mx = max(mx, mm);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        scal[0] = carry;
        scal[1] = mx;
        scal[2] = nlong;
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(const uint32_t* __restrict__ in, int64_t n,
                                                            const uint64_t* __restrict__ part,
                                                            uint64_t* __restrict__ out,
                                                            const uint64_t* __restrict__ scal, uint32_t round_mask)
{
    int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint64_t local = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        v[k] = i < n ? ((in[i] + round_mask) & ~round_mask) : 0u;
        local += v[k];
    }
    uint64_t tot;
    uint64_t ex = block_excl_scan(local, &tot) + part[2 * blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        if (i < n) out[i] = ex;
        ex += v[k];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = scal[0];
}

}  // namespace

int64_t scan_partials_needed(int64_t n) { return (n + kScanChunk - 1) / kScanChunk; }

cudaError_t scan_u32_to_u64(const uint32_t* in, uint64_t* out, int64_t n, uint64_t* part,
                            uint32_t* part_max, uint64_t* scal, uint32_t long_thr, cudaStream_t s,
                            uint32_t round_to)
{
    int64_t nb = scan_partials_needed(n);
    if (nb < 1) nb = 1;
    const uint32_t rm = round_to > 1 ? round_to - 1 : 0u;   // round_to: 0/1 or a power of two
    k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, part, part_max, long_thr, rm);
    k_scan_partials<<<1, kScanThreads, 0, s>>>(part, part_max, nb, scal);
    k_scan_down<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, part, out, scal, rm);
    return cudaGetLastError();
}

}  // namespace hexfc
