// Fragment shading of the focus+context renderer (Section "Focus+Context",
// Eqs. 1-4), used by the fill kernel of this library.
#pragma once
#include "raster_common.cuh"

namespace hexfc {

// Shading inputs of the kChunk triangles of one chunk, structure of arrays
// (element j = triangle j, vertices in wound order), so that lanes reading
// different triangles touch different shared-memory banks. Coordinates are in
// 1/256-pixel units; integers below 2^24 are exact in float.
//
// Perspective-correct interpolation of an attribute a with vertex weights
// lam_k (lam_0 = 1 - lam_1 - lam_2) is sum lam_k a_k / w_k over
// sum lam_k / w_k (w = eye depth). Both sums are affine in (lam_1, lam_2), so
// each is kept as its value at vertex 0 and two differences: with q_k = 1/w_k,
// Q = q0 + lam_1 dq1 + lam_2 dq2 and sum lam_k a_k q_k = A0 + lam_1 dA1 + lam_2 dA2.
// Orthographic views use q_k = 1.
struct ShadeSoA {
    float FX[4][kChunk], FY[4][kChunk];     // face corners
    float inv_len2[4][kChunk];              // 1 / squared length of face edge k -> k+1 (0: degenerate)
    uint32_t z[3][kChunk];                  // window depth of the triangle's vertices
    float dz[2][kChunk];                    // z[1] - z[0], z[2] - z[0] (exact: |d| < 2^24)
    float q0[kChunk], dq[2][kChunk];        // 1 / eye depth
    float a0[kChunk], da[2][kChunk];        // importance / eye depth
    float p0[3][kChunk], dp[2][3][kChunk];  // (world position - sphere lens centre) / eye depth
    int64_t area[kChunk];                   // twice the area (16.8 squared)
    uint32_t area32[kChunk];                // the area below 2^26, else 0
    uint32_t l0[2][kChunk];                 // low words of the edge functions of vertices 1, 2 at the box origin
    float inv_area[kChunk];
    uint32_t f2t[kChunk];
    uint32_t masks[kChunk];                 // bits 0-3 focus-visible, 4-7 context-visible face edges
};

// Square root of x >= 0 (0 at 0), the hardware approximation (a few units in
// the last place).
__device__ __forceinline__ float sqrt_approx(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Eqs. 1-4 for one fragment of triangle j at pixel (px, py); lam1, lam2 are
// the screen-space barycentric weights of vertices 1 and 2. Returns the
// premultiplied RGBA of Eq. 4.
__device__ __forceinline__ float4 shade_fragment(const ShadeSoA& t, int j, float lam1, float lam2, int px, int py,
                                                 const ShadeParams& sp)
{
    const float Q = fmaf(lam2, t.dq[1][j], fmaf(lam1, t.dq[0][j], t.q0[j]));   // 1 / eye depth of the fragment
    const float iQ = __fdividef(1.f, Q);
    const float g = sp.ortho ? 1.f : fminf(fmaxf(sp.zref * Q, sp.g_min), sp.g_max);   // z_ref / z_eye
    const float t_imp = fmaf(lam2, t.da[1][j], fmaf(lam1, t.da[0][j], t.a0[j])) * iQ;
    // lens distance, normalised to 1 at the lens border
    float dist;
    if (sp.lens_mode == HEXFC_LENS_SCREEN) {
        const float dx = ((float)px + 0.5f) - sp.lens_c[0], dy = ((float)py + 0.5f) - sp.lens_c[1];
        dist = sqrt_approx(dx * dx + dy * dy) * sp.lens_inv_r;
    } else {
        // the interpolated offset from the centre, P - C = D / Q (D affine in lam)
        const float Dx = fmaf(lam2, t.dp[1][0][j], fmaf(lam1, t.dp[0][0][j], t.p0[0][j]));
        const float Dy = fmaf(lam2, t.dp[1][1][j], fmaf(lam1, t.dp[0][1][j], t.p0[1][j]));
        const float Dz = fmaf(lam2, t.dp[1][2][j], fmaf(lam1, t.dp[0][2][j], t.p0[2][j]));
        dist = sqrt_approx(fmaf(Dx, Dx, fmaf(Dy, Dy, Dz * Dz))) * (iQ * sp.lens_inv_r);
    }
    // focus = 1 - smoothstep(0.7, 1, dist)
    const float st = __saturatef((dist - 0.7f) * (1.f / 0.3f));
    const float focus = 1.f - st * st * (3.f - 2.f * st);
    // squared distances to the face edge segments: the closest point of edge k
    // is corner k + t e_k, t = clamp(v_k . e_k / |e_k|^2, 0, 1), with
    // v_k = sample - corner k and e_k = corner k+1 - corner k (both exact)
    const float sx = (float)(256 * px + 128), sy = (float)(256 * py + 128);
    const float vx0 = sx - t.FX[0][j], vy0 = sy - t.FY[0][j];
    float vx = vx0, vy = vy0;   // corner k of the loop
    const uint32_t masks = t.masks[j];
    float a2 = INFINITY, f2 = INFINITY, c2 = INFINITY;   // all edges, visible in focus, visible in context
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int k1 = (k + 1) & 3;
        const float nx = k1 == 0 ? vx0 : sx - t.FX[k1][j], ny = k1 == 0 ? vy0 : sy - t.FY[k1][j];
        const float ex = vx - nx, ey = vy - ny;
        const float tp = __saturatef(fmaf(vx, ex, vy * ey) * t.inv_len2[k][j]);
        const float dx = fmaf(-tp, ex, vx), dy = fmaf(-tp, ey, vy);
        const float d2 = fmaf(dx, dx, dy * dy);
        a2 = fminf(a2, d2);
        f2 = ((masks >> k) & 1u) ? fminf(f2, d2) : f2;
        c2 = ((masks >> (4 + k)) & 1u) ? fminf(c2, d2) : c2;
        vx = nx;
        vy = ny;
    }
    // Eq. 1 with the depth-dependent width w, halo band h (focus edges); the
    // tests compare squared distances in 1/256-pixel units. Edges visible in
    // context are visible in focus too (c2 >= f2), so an edge in context
    // (alpha 1) is one in focus, and an edge in focus or in the halo band has
    // alpha = focus (in the band with focus 0 that is 0 as well).
    const float wg = 256.f * sp.w_base * g;                      // >= 0: w_base, g_min, halo_scale >= 0
    const float w256 = fmaf(0.3f * focus, wg, wg);
    const float wh256 = fmaf((0.3f + sp.halo_scale) * focus, wg, wg);
    const float w2 = w256 * w256;
    const bool band = f2 <= wh256 * wh256;
    const bool halo = band && f2 > w2 && focus > 0.f;
    const float alpha_e = c2 <= w2 ? 1.f : (band ? focus : 0.f);
    // colour table ctf = (t, 0, 1 - t); Eq. 2: accentuated faces (s_e = s > 1)
    // move the face colour towards white by beta
    const float tt = __saturatef((t_imp - sp.tf_lo) * sp.tf_inv);
    const bool accent = a2 <= sp.accent_r2;
    const float s_e = accent ? sp.s : 1.f;
    const float beta = s_e > 1.f ? sp.accent_beta : 0.f;
    const float dk = fmaf(-sp.darken, focus, 1.f);
    const float er = halo ? 1.f : tt * dk, eg = halo ? 1.f : 0.f, eb = halo ? 1.f : (1.f - tt) * dk;
    // Eq. 3 and Eq. 4
    const float ahat = fmaf(sp.alpha_span, tt, sp.alpha_min);
    const float dc = fminf(dist, 1.f);
    const float dc2 = dc * dc;
    const float af = fminf(s_e * (ahat * (dc2 * dc2)), 1.f);
    const float wf = (1.f - alpha_e) * af;
    float4 c = make_float4(fmaf(alpha_e, er, wf * fmaf(beta, 1.f - tt, tt)), fmaf(alpha_e, eg, wf * beta),
                           fmaf(alpha_e, eb, wf * fmaf(beta, tt, 1.f - tt)), alpha_e + wf);
    // depth cue (Section "Evaluation"): in focus and beyond the reference
    // depth, the colour moves towards its luma; opacity unchanged
    if (sp.desat > 0.f) {
        const float k = sp.desat * focus * fminf(fmaxf(1.f - g, 0.f), 1.f);
        const float y = 0.299f * c.x + 0.587f * c.y + 0.114f * c.z;
        c.x = fmaf(k, y - c.x, c.x);
        c.y = fmaf(k, y - c.y, c.y);
        c.z = fmaf(k, y - c.z, c.z);
    }
    return c;
}

}  // namespace hexfc
