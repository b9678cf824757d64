// Fragment shading of the focus+context renderer (Section "Focus+Context",
// Eqs. 1-4), used by the fill kernel of this library.
#pragma once
#include "raster_common.cuh"

namespace hexfc {

// Shading and depth inputs of one triangle of a chunk (vertices in wound
// order), read by the consumer lanes 16 bytes at a time: eleven vectors, an
// odd stride in 16-byte units, so the lanes of a quarter warp that read
// different triangles of the chunk share banks only when the triangles'
// indices agree modulo 8. Coordinates are in 1/256-pixel units; integers
// below 2^24 are exact in float.
//
// Perspective-correct interpolation of an attribute a with vertex weights
// lam_k (lam_0 = 1 - lam_1 - lam_2) is sum lam_k a_k / w_k over
// sum lam_k / w_k (w = eye depth). Both sums are affine in (lam_1, lam_2), so
// each is kept as its value at vertex 0 and two differences: with q_k = 1/w_k,
// Q = q0 + lam_1 dq1 + lam_2 dq2 and sum lam_k a_k q_k = A0 + lam_1 dA1 + lam_2 dA2.
// Orthographic views use q_k = 1.
struct ShadeRec {
    float4 fx, fy;   // face corners
    float4 il;       // 1 / squared length of face edge k -> k+1 (0: degenerate)
    float4 qa;       // q0, dq1, dq2 (1 / eye depth); a0 (importance / eye depth)
    float4 ap;       // da1, da2; p0.x, p0.y  (p = (world position - sphere lens centre) / eye depth)
    float4 pp;       // p0.z; dp1.x, dp1.y, dp1.z
    float4 pq;       // dp2.x, dp2.y, dp2.z; unused
    uint4 zm;        // window depth of the three vertices; face edge flags (bits 0-3 focus, 4-7 context)
    uint4 wd;        // low words of the edge functions of vertices 1, 2 at the tile's first sample; dz1, dz2 (float bits)
    int4 ev;         // dx, dy of the edges opposite vertices 1 and 2 (16.8)
    uint4 hd;        // box (as CovSoA::box), f2t, twice the area if below 2^26 else 0, 1 / twice the area (float bits)
};
static_assert(sizeof(ShadeRec) == 11 * 16, "eleven 16-byte vectors");

// Square root of x >= 0 (0 at 0), the hardware approximation (a few units in
// the last place).
__device__ __forceinline__ float sqrt_approx(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Eqs. 1-4 for one fragment of triangle t at pixel (px, py); lam1, lam2 are
// the screen-space barycentric weights of vertices 1 and 2, masks the face
// edge flags (t.zm.w). Returns the premultiplied RGBA of Eq. 4.
__device__ __forceinline__ float4 shade_fragment(const ShadeRec& t, uint32_t masks, float lam1, float lam2, int px,
                                                 int py, const ShadeParams& sp)
{
    const float4 qa = t.qa, ap = t.ap;
    const float Q = fmaf(lam2, qa.z, fmaf(lam1, qa.y, qa.x));   // 1 / eye depth of the fragment
    const float iQ = __fdividef(1.f, Q);
    const float g = sp.ortho ? 1.f : fminf(fmaxf(sp.zref * Q, sp.g_min), sp.g_max);   // z_ref / z_eye
    const float t_imp = fmaf(lam2, ap.y, fmaf(lam1, ap.x, qa.w)) * iQ;
    // lens distance, normalised to 1 at the lens border
    float dist;
    if (sp.lens_mode == HEXFC_LENS_SCREEN) {
        // (frame pixel coordinates, so that a drawn rectangle shades as the frame does)
        const float dx = ((float)(px + sp.px_off) + 0.5f) - sp.lens_c[0];
        const float dy = ((float)(py + sp.py_off) + 0.5f) - sp.lens_c[1];
        dist = sqrt_approx(dx * dx + dy * dy) * sp.lens_inv_r;
    } else {
        // the interpolated offset from the centre, P - C = D / Q (D affine in lam)
        const float4 pp = t.pp, pq = t.pq;
        const float Dx = fmaf(lam2, pq.x, fmaf(lam1, pp.y, ap.z));
        const float Dy = fmaf(lam2, pq.y, fmaf(lam1, pp.z, ap.w));
        const float Dz = fmaf(lam2, pq.z, fmaf(lam1, pp.w, pp.x));
        dist = sqrt_approx(fmaf(Dx, Dx, fmaf(Dy, Dy, Dz * Dz))) * (iQ * sp.lens_inv_r);
    }
    // focus = 1 - smoothstep(0.7, 1, dist)
    const float st = __saturatef((dist - 0.7f) * (1.f / 0.3f));
    const float focus = 1.f - st * st * (3.f - 2.f * st);
    // squared distances to the face edge segments: the closest point of edge k
    // is corner k + t e_k, t = clamp(v_k . e_k / |e_k|^2, 0, 1), with
    // v_k = sample - corner k and e_k = corner k+1 - corner k (both exact)
    const float sx = (float)(256 * px + 128), sy = (float)(256 * py + 128);
    const float4 fx = t.fx, fy = t.fy, il = t.il;
    const float FX[4] = {fx.x, fx.y, fx.z, fx.w}, FY[4] = {fy.x, fy.y, fy.z, fy.w};
    const float IL[4] = {il.x, il.y, il.z, il.w};
    const float vx0 = sx - FX[0], vy0 = sy - FY[0];
    float vx = vx0, vy = vy0;   // corner k of the loop
    float a2 = INFINITY, f2 = INFINITY, c2 = INFINITY;   // all edges, visible in focus, visible in context
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int k1 = (k + 1) & 3;
        const float nx = k1 == 0 ? vx0 : sx - FX[k1], ny = k1 == 0 ? vy0 : sy - FY[k1];
        const float ex = vx - nx, ey = vy - ny;
        const float tp = __saturatef(fmaf(vx, ex, vy * ey) * IL[k]);
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
