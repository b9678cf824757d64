// Fragment shading of the focus+context renderer (Section "Focus+Context",
// Eqs. 1-4), used by the fill kernel of this library.
#pragma once
#include "raster_common.cuh"

namespace hexfc {

// Shading inputs of the kChunk triangles of one chunk, structure of arrays
// (element j = triangle j, vertices in wound order), so that lanes reading
// different triangles touch different shared-memory banks. Coordinates are in
// 1/256-pixel units; integers below 2^24 are exact in float.
struct ShadeSoA {
    float FX[4][kChunk], FY[4][kChunk];     // face corners
    float ex[4][kChunk], ey[4][kChunk];     // face edge vectors corner k -> k+1
    float len2[4][kChunk];                  // their squared lengths
    float inv_len[4][kChunk];               // 1 / length
    uint32_t z[3][kChunk];                  // window depth of the triangle's vertices
    float dz[2][kChunk];                    // z[1] - z[0], z[2] - z[0] (exact: |d| < 2^24)
    float inv_ed[3][kChunk];                // 1 / eye depth
    float imp[3][kChunk];                   // vertex importance
    float P[3][3][kChunk];                  // world position P[vertex][axis]
    int64_t area[kChunk];                   // twice the area (16.8 squared)
    float inv_area[kChunk];
    uint32_t f2t[kChunk];
    uint32_t masks[kChunk];                 // bits 0-3 focus-visible, 4-7 context-visible face edges
};

// Squared distance (1/256-pixel units squared) from sample (sx, sy) to face
// edge k of triangle j: the closest point of the segment (an end point or the
// foot of the perpendicular), chosen without branches.
__device__ __forceinline__ float seg_dist2(const ShadeSoA& S, int j, int k, float sx, float sy)
{
    const float px = sx - S.FX[k][j], py = sy - S.FY[k][j];   // exact: both are integers < 2^24
    const float ex = S.ex[k][j], ey = S.ey[k][j];
    const float dot = fmaf(px, ex, py * ey);
    const float da = fmaf(px, px, py * py);
    const float qx = px - ex, qy = py - ey;
    const float db = fmaf(qx, qx, qy * qy);
    const float cr = fmaf(px, ey, -py * ex) * S.inv_len[k][j];
    const float dp = cr * cr;
    return dot <= 0.f ? da : (dot >= S.len2[k][j] ? db : dp);
}

__device__ __forceinline__ float fast_sqrt(float x) { return x > 0.f ? x * rsqrtf(x) : 0.f; }

// Eqs. 1-4 for one fragment of triangle j at pixel (px, py); lam1, lam2 are
// the screen-space barycentric weights of vertices 1 and 2. Returns the
// premultiplied RGBA of Eq. 4.
__device__ __forceinline__ float4 shade_fragment(const ShadeSoA& t, int j, float lam1, float lam2, int px, int py,
                                                 const ShadeParams& sp)
{
    const float lam0 = 1.f - lam1 - lam2;
    float b0, b1, b2, g = 1.f;
    if (sp.ortho) {
        b0 = lam0; b1 = lam1; b2 = lam2;
    } else {  // perspective-correct interpolation: weights lam_k / w_k, renormalised
        const float q0 = lam0 * t.inv_ed[0][j], q1 = lam1 * t.inv_ed[1][j], q2 = lam2 * t.inv_ed[2][j];
        const float Q = q0 + q1 + q2;   // 1 / eye depth of the fragment
        const float iQ = __frcp_rn(Q);
        b0 = q0 * iQ; b1 = q1 * iQ; b2 = q2 * iQ;
        g = fminf(fmaxf(sp.zref * Q, sp.g_min), sp.g_max);   // depth factor z_ref / z_eye
    }
    const float t_imp = b0 * t.imp[0][j] + b1 * t.imp[1][j] + b2 * t.imp[2][j];
    // lens distance, normalised to 1 at the lens border
    float dist;
    if (sp.lens_mode == HEXFC_LENS_SCREEN) {
        const float dx = ((float)px + 0.5f) - sp.lens_c[0], dy = ((float)py + 0.5f) - sp.lens_c[1];
        dist = fast_sqrt(dx * dx + dy * dy) * sp.lens_inv_r;
    } else {
        const float Px = b0 * t.P[0][0][j] + b1 * t.P[1][0][j] + b2 * t.P[2][0][j];
        const float Py = b0 * t.P[0][1][j] + b1 * t.P[1][1][j] + b2 * t.P[2][1][j];
        const float Pz = b0 * t.P[0][2][j] + b1 * t.P[1][2][j] + b2 * t.P[2][2][j];
        const float dx = Px - sp.lens_c[0], dy = Py - sp.lens_c[1], dz = Pz - sp.lens_c[2];
        dist = fast_sqrt(dx * dx + dy * dy + dz * dz) * sp.lens_inv_r;
    }
    // focus = 1 - smoothstep(0.7, 1, dist)
    const float st = fminf(fmaxf((dist - 0.7f) * (1.f / 0.3f), 0.f), 1.f);
    const float focus = 1.f - st * st * (3.f - 2.f * st);
    // distances to the face edges: all, visible in focus, visible in context
    const uint32_t masks = t.masks[j];
    const float sx = (float)(256 * px + 128), sy = (float)(256 * py + 128);
    float a2 = INFINITY, f2 = INFINITY, c2 = INFINITY;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float d2 = seg_dist2(t, j, k, sx, sy);
        a2 = fminf(a2, d2);
        f2 = ((masks >> k) & 1u) ? fminf(f2, d2) : f2;
        c2 = ((masks >> (4 + k)) & 1u) ? fminf(c2, d2) : c2;
    }
    const float d_a = fast_sqrt(a2) * (1.f / 256.f);
    const float d_f = f2 < INFINITY ? fast_sqrt(f2) * (1.f / 256.f) : INFINITY;
    const float d_c = c2 < INFINITY ? fast_sqrt(c2) * (1.f / 256.f) : INFINITY;
    // Eq. 1 with the depth-dependent width, halo band of the focus edges
    const float w = (1.f + 0.3f * focus) * sp.w_base * g;
    const bool e_focus = d_f <= w, e_context = d_c <= w;
    const float h = sp.halo_scale * sp.w_base * focus * g;
    float alpha_e = (float)e_context + focus * ((float)e_focus - (float)e_context);
    const bool halo = !e_focus && (d_f <= w + h) && focus > 0.f;
    if (halo) alpha_e = focus;
    // colour table and Eq. 2
    const float tt = fminf(fmaxf((t_imp - sp.tf_lo) * sp.tf_inv, 0.f), 1.f);
    const float ctf[3] = {tt, 0.f, 1.f - tt};
    const float dk = 1.f - sp.darken * focus;
    const bool accent = d_a <= (2.f / 3.f) * sp.w_base;
    const float s_e = accent ? sp.s : 1.f;
    float cf[3], ce[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        ce[k] = halo ? 1.f : ctf[k] * dk;
        cf[k] = s_e > 1.f ? ctf[k] + sp.accent_beta * (1.f - ctf[k]) : ctf[k];
    }
    // Eq. 3 and Eq. 4
    const float ahat = sp.alpha_min + sp.alpha_span * tt;
    const float dc = fminf(dist, 1.f);
    const float dc2 = dc * dc;
    const float af = fminf(s_e * (ahat * (dc2 * dc2)), 1.f);
    const float wf = (1.f - alpha_e) * af;
    return make_float4(alpha_e * ce[0] + wf * cf[0], alpha_e * ce[1] + wf * cf[1], alpha_e * ce[2] + wf * cf[2],
                       alpha_e + wf);
}

}  // namespace hexfc
