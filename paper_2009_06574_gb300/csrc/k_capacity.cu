// Tile-capacity network: per raster tile, a 4 -> 64 -> 64 -> 1 ReLU network
// predicts y ~ log(1 + fragments of the tile) from four features, so that
// fragment storage can be divided among the tiles before a frame is counted.
// Weights are used in FP16 (staged in shared memory), sums in FP32; training
// keeps an FP32 master copy and Adam moments. No counterpart in the paper.
//
//   k_cap_features  per tile: log1p(previous frame's count) / 12, the depth
//                   range of its triangles, the distance from the tile to the
//                   lens on screen / screen diagonal, the camera's motion
//                   since the previous frame
//   k_cap_forward   per tile: y and the capacity expm1(y) (1 + margin) + pad
//   k_cap_backward  per tile: mean-squared loss on log1p(exact count); stores
//                   the layer values and the back-propagated errors
//   k_cap_reduce    per parameter: gradient = sum over tiles (tile slices,
//                   atomics between slices)
//   k_cap_adam      per parameter: Adam step on the master copy, FP16 copy
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>

#include "hexfc_internal.cuh"

namespace hexfc {
namespace {

constexpr int kIn = kCapIn, kHid = kCapHid;
constexpr int oW1 = 0, oB1 = oW1 + kHid * kIn, oW2 = oB1 + kHid, oB2 = oW2 + kHid * kHid, oW3 = oB2 + kHid,
              oB3 = oW3 + kHid;
static_assert(oB3 + 1 == kCapParams, "parameter layout");

inline unsigned grid_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

__device__ __forceinline__ void load_weights(const __half* __restrict__ w16, float* s_w)
{
    for (int i = threadIdx.x; i < kCapParams; i += blockDim.x) s_w[i] = __half2float(w16[i]);
    __syncthreads();
}

__global__ void k_cap_features(int64_t n_tiles, int tiles_x, const uint32_t* __restrict__ prev,
                               const float* __restrict__ zr, float lens_x, float lens_y, float inv_diag,
                               float motion, float* __restrict__ X)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tiles) return;
    const float cx = (float)((t % tiles_x) * kTileW) + 0.5f * kTileW;
    const float cy = (float)((t / tiles_x) * kTileH) + 0.5f * kTileH;
    const float dx = cx - lens_x, dy = cy - lens_y;
    X[4 * t + 0] = log1pf((float)prev[t]) * (1.f / 12.f);
    X[4 * t + 1] = zr[t];
    X[4 * t + 2] = fminf(sqrtf(dx * dx + dy * dy) * inv_diag, 2.f);
    X[4 * t + 3] = motion;
}

__global__ void __launch_bounds__(256) k_cap_forward(const float* __restrict__ X, int64_t n,
                                                     const __half* __restrict__ w16, float margin, uint32_t pad,
                                                     uint32_t* __restrict__ cap)
{
    __shared__ float s_w[kCapParams];
    load_weights(w16, s_w);
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const float x0 = X[4 * t], x1 = X[4 * t + 1], x2 = X[4 * t + 2], x3 = X[4 * t + 3];
    float h1[kHid];
#pragma unroll
    for (int i = 0; i < kHid; ++i) {
        const float* w = s_w + oW1 + i * kIn;
        h1[i] = fmaxf(fmaf(w[3], x3, fmaf(w[2], x2, fmaf(w[1], x1, fmaf(w[0], x0, s_w[oB1 + i])))), 0.f);
    }
    float y = s_w[oB3];
    for (int j = 0; j < kHid; ++j) {
        const float* w = s_w + oW2 + j * kHid;
        float a = s_w[oB2 + j];
#pragma unroll
        for (int i = 0; i < kHid; ++i) a = fmaf(w[i], h1[i], a);
        y = fmaf(s_w[oW3 + j], fmaxf(a, 0.f), y);
    }
    const float c = expm1f(fminf(y, 20.f)) * (1.f + margin) + (float)pad;
    cap[t] = (uint32_t)fminf(fmaxf(c, 0.f), 4.0e9f);
}

// Forward and backward of one tile; loss = mean over the n tiles of (y - t)^2.
__global__ void __launch_bounds__(256) k_cap_backward(const float* __restrict__ X,
                                                      const uint32_t* __restrict__ counts, int64_t n,
                                                      const __half* __restrict__ w16, float* __restrict__ H1,
                                                      float* __restrict__ H2, float* __restrict__ DA1,
                                                      float* __restrict__ DA2, float* __restrict__ DY,
                                                      float* __restrict__ loss)
{
    __shared__ float s_w[kCapParams];
    __shared__ float s_loss[8];
    load_weights(w16, s_w);
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.f;
    if (t < n) {
        const float x0 = X[4 * t], x1 = X[4 * t + 1], x2 = X[4 * t + 2], x3 = X[4 * t + 3];
        float h1[kHid];
        uint64_t m1 = 0, m2 = 0;
#pragma unroll
        for (int i = 0; i < kHid; ++i) {
            const float* w = s_w + oW1 + i * kIn;
            const float a = fmaf(w[3], x3, fmaf(w[2], x2, fmaf(w[1], x1, fmaf(w[0], x0, s_w[oB1 + i]))));
            h1[i] = fmaxf(a, 0.f);
            m1 |= (uint64_t)(a > 0.f) << i;
            H1[t * kHid + i] = h1[i];
        }
        float y = s_w[oB3];
        for (int j = 0; j < kHid; ++j) {
            const float* w = s_w + oW2 + j * kHid;
            float a = s_w[oB2 + j];
#pragma unroll
            for (int i = 0; i < kHid; ++i) a = fmaf(w[i], h1[i], a);
            const float h2 = fmaxf(a, 0.f);
            m2 |= (uint64_t)(a > 0.f) << j;
            H2[t * kHid + j] = h2;
            y = fmaf(s_w[oW3 + j], h2, y);
        }
        const float e = y - log1pf((float)counts[t]);
        l = e * e / (float)n;
        const float dy = 2.f * e / (float)n;
        DY[t] = dy;
        float dh1[kHid];
#pragma unroll
        for (int i = 0; i < kHid; ++i) dh1[i] = 0.f;
        for (int j = 0; j < kHid; ++j) {
            const float da2 = ((m2 >> j) & 1ull) ? dy * s_w[oW3 + j] : 0.f;
            DA2[t * kHid + j] = da2;
            const float* w = s_w + oW2 + j * kHid;
#pragma unroll
            for (int i = 0; i < kHid; ++i) dh1[i] = fmaf(w[i], da2, dh1[i]);
        }
#pragma unroll
        for (int i = 0; i < kHid; ++i) DA1[t * kHid + i] = ((m1 >> i) & 1ull) ? dh1[i] : 0.f;
    }
    // the block's share of the loss
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) s_loss[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
        float b = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += s_loss[w];
        atomicAdd(loss, b);
    }
}

// Parameter p's gradient over tiles [s0, s1): a sum of products of the stored
// layer values and errors.
__global__ void __launch_bounds__(256) k_cap_reduce(const float* __restrict__ X, int64_t n,
                                                    const float* __restrict__ H1, const float* __restrict__ H2,
                                                    const float* __restrict__ DA1, const float* __restrict__ DA2,
                                                    const float* __restrict__ DY, int slices,
                                                    float* __restrict__ grad)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kCapParams) return;
    const int64_t per = (n + slices - 1) / slices;
    const int64_t s0 = (int64_t)blockIdx.y * per, s1 = min(n, s0 + per);
    float g = 0.f;
    if (p < oB1) {                 // W1[i][k]
        const int i = p / kIn, k = p % kIn;
        for (int64_t t = s0; t < s1; ++t) g = fmaf(DA1[t * kHid + i], X[4 * t + k], g);
    } else if (p < oW2) {          // b1[i]
        const int i = p - oB1;
        for (int64_t t = s0; t < s1; ++t) g += DA1[t * kHid + i];
    } else if (p < oB2) {          // W2[j][i]
        const int j = (p - oW2) / kHid, i = (p - oW2) % kHid;
        for (int64_t t = s0; t < s1; ++t) g = fmaf(DA2[t * kHid + j], H1[t * kHid + i], g);
    } else if (p < oW3) {          // b2[j]
        const int j = p - oB2;
        for (int64_t t = s0; t < s1; ++t) g += DA2[t * kHid + j];
    } else if (p < oB3) {          // w3[j]
        const int j = p - oW3;
        for (int64_t t = s0; t < s1; ++t) g = fmaf(DY[t], H2[t * kHid + j], g);
    } else {                       // b3
        for (int64_t t = s0; t < s1; ++t) g += DY[t];
    }
    atomicAdd(&grad[p], g);
}

__global__ void k_cap_adam(float* __restrict__ w, __half* __restrict__ w16, const float* __restrict__ grad,
                           float* __restrict__ m, float* __restrict__ v, float lr, float b1, float b2, float eps,
                           float c1, float c2)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kCapParams) return;
    const float g = grad[p];
    const float mm = fmaf(b1, m[p], (1.f - b1) * g);
    const float vv = fmaf(b2, v[p], (1.f - b2) * g * g);
    m[p] = mm;
    v[p] = vv;
    const float wn = w[p] - lr * (mm * c1) / (sqrtf(vv * c2) + eps);
    w[p] = wn;
    w16[p] = __float2half_rn(wn);
}

__global__ void k_cap_to_half(const float* __restrict__ w, __half* __restrict__ w16)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < kCapParams) w16[p] = __float2half_rn(w[p]);
}

}  // namespace

cudaError_t launch_cap_features(FrameBufs& fb, int64_t n_tiles, int tiles_x, float lens_x, float lens_y,
                                float inv_diag, float motion, cudaStream_t s)
{
    k_cap_features<<<grid_for(n_tiles, 256), 256, 0, s>>>(n_tiles, tiles_x, fb.tile_frag, fb.tile_zr, lens_x, lens_y,
                                                          inv_diag, motion, fb.cap_x);
    return cudaGetLastError();
}

cudaError_t launch_cap_forward(const CapNet& net, FrameBufs& fb, int64_t n_tiles, float margin, uint32_t pad,
                               cudaStream_t s)
{
    k_cap_forward<<<grid_for(n_tiles, 256), 256, 0, s>>>(fb.cap_x, n_tiles, net.w16, margin, pad, fb.tile_cap);
    return cudaGetLastError();
}

cudaError_t launch_cap_grad(CapNet& net, const float* X, const uint32_t* counts, int64_t n, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(net.grad, 0, sizeof(float) * (kCapParams + 1), s);   // grad[kCapParams] = loss
    if (e != cudaSuccess) return e;
    k_cap_backward<<<grid_for(n, 256), 256, 0, s>>>(X, counts, n, net.w16, net.h1, net.h2, net.da1, net.da2, net.dy,
                                                    net.grad + kCapParams);
    const int slices = (int)std::min<int64_t>(64, std::max<int64_t>(1, n / 256));
    k_cap_reduce<<<dim3(grid_for(kCapParams, 256), (unsigned)slices), 256, 0, s>>>(X, n, net.h1, net.h2, net.da1,
                                                                                   net.da2, net.dy, slices, net.grad);
    return cudaGetLastError();
}

cudaError_t launch_cap_adam(CapNet& net, float lr, cudaStream_t s)
{
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    net.step += 1;
    const float c1 = 1.f / (1.f - std::pow(b1, (float)net.step)), c2 = 1.f / (1.f - std::pow(b2, (float)net.step));
    k_cap_adam<<<grid_for(kCapParams, 256), 256, 0, s>>>(net.w, net.w16, net.grad, net.m, net.v, lr, b1, b2, eps, c1,
                                                         c2);
    return cudaGetLastError();
}

cudaError_t launch_cap_to_half(CapNet& net, cudaStream_t s)
{
    k_cap_to_half<<<grid_for(kCapParams, 256), 256, 0, s>>>(net.w, net.w16);
    return cudaGetLastError();
}

}  // namespace hexfc
