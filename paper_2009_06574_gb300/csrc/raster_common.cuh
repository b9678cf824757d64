// Device helpers shared by the raster kernels of this library: triangle setup
// in 16.8 fixed point, exact edge functions with the top-left rule, exact
// per-sample depth.
#pragma once
#include "hexfc_internal.cuh"

namespace hexfc {

// 2x the signed area of (a, b, p): (b - a) x (p - a), exact in int64.
__device__ __forceinline__ int64_t edge_fn(int32_t xa, int32_t ya, int32_t xb, int32_t yb, int32_t px,
                                           int32_t py)
{
    return (int64_t)(xb - xa) * (int64_t)(py - ya) - (int64_t)(yb - ya) * (int64_t)(px - xa);
}

// Tie rule for samples exactly on an edge a->b of a positively wound triangle:
// the edge owns them iff it goes up (dy < 0) or is horizontal going right.
// Exactly one of the two triangles sharing an edge owns its samples.
__device__ __forceinline__ bool top_left(int32_t xa, int32_t ya, int32_t xb, int32_t yb)
{
    int32_t dx = xb - xa, dy = yb - ya;
    return (dy < 0) || (dy == 0 && dx > 0);
}

__device__ __forceinline__ int64_t floor_div_i64(int64_t a, int64_t b)  // b > 0
{
    int64_t q = a / b;
    if ((a % b != 0) && (a < 0)) --q;
    return q;
}

// Triangle of a face: tri 0 = corners (0,1,2), tri 1 = (0,2,3), wound to positive area.
struct TriGeom {
    int32_t X[3], Y[3];
    int vi[3];          // face corner of each vertex
    int64_t area;       // 2x area, > 0 when valid
    int32_t bx0, by0, bx1, by1;  // pixel box of covered centres, clamped to the screen
    bool valid;
};

__device__ __forceinline__ void tri_setup(const int32_t FX[4], const int32_t FY[4], int tri, int W, int H,
                                          TriGeom& t)
{
    int i1 = tri == 0 ? 1 : 2, i2 = tri == 0 ? 2 : 3;
    t.vi[0] = 0; t.vi[1] = i1; t.vi[2] = i2;
    // selects instead of FX[i1]: no dynamic register indexing
    t.X[0] = FX[0]; t.Y[0] = FY[0];
    t.X[1] = tri == 0 ? FX[1] : FX[2]; t.Y[1] = tri == 0 ? FY[1] : FY[2];
    t.X[2] = tri == 0 ? FX[2] : FX[3]; t.Y[2] = tri == 0 ? FY[2] : FY[3];
    int64_t a = edge_fn(t.X[0], t.Y[0], t.X[1], t.Y[1], t.X[2], t.Y[2]);
    if (a < 0) {
        int32_t tx = t.X[1], ty = t.Y[1];
        t.X[1] = t.X[2]; t.Y[1] = t.Y[2];
        t.X[2] = tx; t.Y[2] = ty;
        t.vi[1] = i2; t.vi[2] = i1;
        a = -a;
    }
    t.area = a;
    int32_t xmin = min(t.X[0], min(t.X[1], t.X[2])), xmax = max(t.X[0], max(t.X[1], t.X[2]));
    int32_t ymin = min(t.Y[0], min(t.Y[1], t.Y[2])), ymax = max(t.Y[0], max(t.Y[1], t.Y[2]));
    // pixel p has its centre at 256 p + 128
    int64_t bx0 = -floor_div_i64(-((int64_t)xmin - 128), 256);
    int64_t by0 = -floor_div_i64(-((int64_t)ymin - 128), 256);
    int64_t bx1 = floor_div_i64((int64_t)xmax - 128, 256);
    int64_t by1 = floor_div_i64((int64_t)ymax - 128, 256);
    bx0 = max(bx0, (int64_t)0);
    by0 = max(by0, (int64_t)0);
    bx1 = min(bx1, (int64_t)W - 1);
    by1 = min(by1, (int64_t)H - 1);
    t.bx0 = (int32_t)bx0; t.by0 = (int32_t)by0; t.bx1 = (int32_t)bx1; t.by1 = (int32_t)by1;
    t.valid = (a != 0) && bx0 <= bx1 && by0 <= by1;
}

// Exact floor(n / a) for a > 0 and |n / a| < 2^25, with |n| < 2^63:
// float estimate, then integer correction (at most a few steps).
__device__ __forceinline__ int64_t floor_div_est(int64_t n, int64_t a, bool& bad)
{
    float qf = floorf(__fdiv_rn((float)n, (float)a));
    int64_t q = (int64_t)qf;
    int64_t r = n - q * a;
#pragma unroll 1
    for (int it = 0; it < 16 && r < 0; ++it) { --q; r += a; }
#pragma unroll 1
    for (int it = 0; it < 16 && r >= a; ++it) { ++q; r -= a; }
    if (r < 0 || r >= a) bad = true;
    return q;
}

// 0 <= v < 2^55 to float through 32-bit conversions (the 64-bit conversion
// instructions run on the FP64 unit, which is narrow on this part): correctly
// rounded below 2^32, else within 0.75 ulp (one rounding of hi * 2^32 + lo,
// lo rounded first).
__device__ __forceinline__ float u64_to_f32(uint64_t v)
{
    return fmaf((float)(uint32_t)(v >> 32), 4294967296.f, (float)(uint32_t)v);
}

// |v| < 2^55 to float by sign and magnitude (u64_to_f32): within 0.75 ulp.
__device__ __forceinline__ float i64_to_f32(int64_t v)
{
    const float m = u64_to_f32((uint64_t)(v < 0 ? -v : v));
    return v < 0 ? -m : m;
}

// Per-sample depth: z0 + floor((l1 (z1 - z0) + l2 (z2 - z0)) / area), exact.
__device__ __forceinline__ uint32_t sample_depth(uint32_t z0, uint32_t z1, uint32_t z2, int64_t l1, int64_t l2,
                                                 int64_t area, bool& bad)
{
    int64_t d1 = (int64_t)z1 - (int64_t)z0, d2 = (int64_t)z2 - (int64_t)z0;
    int64_t q;
    if (area < (1ll << 38)) {
        // |l| <= area < 2^38 and |d| < 2^24: the numerator fits in int64
        q = floor_div_est(l1 * d1 + l2 * d2, area, bad);
    } else {
        __int128 n = (__int128)l1 * d1 + (__int128)l2 * d2;
        double qd = floor((double)n / (double)area);
        __int128 qq = (__int128)qd;
        __int128 r = n - qq * area;
#pragma unroll 1
        for (int it = 0; it < 64 && r < 0; ++it) { --qq; r += area; }
#pragma unroll 1
        for (int it = 0; it < 64 && r >= area; ++it) { ++qq; r -= area; }
        if (r < 0 || r >= area) bad = true;
        q = (int64_t)qq;
    }
    return (uint32_t)((int64_t)z0 + q);
}

// sample_depth for a covered sample (l0, l1, l2 >= 0), from the float
// barycentric weights lam1 ~ l1 / area, lam2 ~ l2 / area and the float depth
// deltas dz1, dz2 (same result). With lam within 5 ulp and 0 <= lam <= 1,
// |d| < 2^24, the float estimate is within 8 of the quotient; the integer
// remainder then corrects it.
__device__ __forceinline__ uint32_t sample_depth_lam(uint32_t z0, uint32_t z1, uint32_t z2, int64_t l1, int64_t l2,
                                                     int64_t area, float lam1, float lam2, float dz1, float dz2,
                                                     bool& bad)
{
    if (area >= (1ll << 38)) return sample_depth(z0, z1, z2, l1, l2, area, bad);
    const int32_t d1 = (int32_t)(z1 - z0), d2 = (int32_t)(z2 - z0);
    int64_t q = __float2int_rd(fmaf(lam1, dz1, lam2 * dz2));
    // |l| <= area < 2^38 and |d| < 2^24: the numerator fits in int64
    int64_t r = l1 * d1 + l2 * d2 - q * area;
#pragma unroll 1
    for (int it = 0; it < 16 && r < 0; ++it) { --q; r += area; }
#pragma unroll 1
    for (int it = 0; it < 16 && r >= area; ++it) { ++q; r -= area; }
    if (r < 0 || r >= area) bad = true;
    return (uint32_t)((int64_t)z0 + q);
}

// sample_depth_lam for a triangle with area < 2^26 (16.8 units squared: below
// 512 square pixels), in 32-bit arithmetic: its weights satisfy 0 <= l <=
// area < 2^26, the float estimate is within 8 of the quotient, so the exact
// remainder l1 d1 + l2 d2 - q area lies within (-9, 9) areas, below 2^30 in
// magnitude, and its value modulo 2^32 read as a signed integer is exact.
__device__ __forceinline__ uint32_t sample_depth_small(uint32_t z0, uint32_t z1, uint32_t z2, uint32_t l1,
                                                       uint32_t l2, uint32_t area, float lam1, float lam2, float dz1,
                                                       float dz2, bool& bad)
{
    int32_t q = __float2int_rd(fmaf(lam1, dz1, lam2 * dz2));
    int32_t r = (int32_t)(l1 * (z1 - z0) + l2 * (z2 - z0) - (uint32_t)q * area);
#pragma unroll 1
    for (int it = 0; it < 16 && r < 0; ++it) { --q; r += (int32_t)area; }
#pragma unroll 1
    for (int it = 0; it < 16 && r >= (int32_t)area; ++it) { ++q; r -= (int32_t)area; }
    if (r < 0 || r >= (int32_t)area) bad = true;
    return z0 + (uint32_t)q;
}

}  // namespace hexfc
