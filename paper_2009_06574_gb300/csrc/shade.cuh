// Fragment shading of the focus+context renderer (Section "Focus+Context",
// Eqs. 1-4), shared by the fill kernels of this library.
#pragma once
#include "raster_common.cuh"

namespace hexfc {

struct TriShade {
    int32_t FX[4], FY[4];   // face corners (16.8)
    uint32_t z[3];          // window depth of the triangle's vertices (wound order)
    float ed[3], imp[3], P[3][3];
    int64_t area;
    uint32_t f2t;
    uint32_t masks;         // bits 0-3 focus-visible, 4-7 context-visible face edges
};

__device__ __forceinline__ float smoothstepf(float e0, float e1, float x)
{
    float t = fminf(fmaxf((x - e0) / (e1 - e0), 0.f), 1.f);
    return t * t * (3.f - 2.f * t);
}

// Distance in pixels from sample (sx, sy) to segment a-b; exact integer
// deltas (16.8), one float rounding at the end of each branch.
__device__ __forceinline__ float seg_dist(int32_t sx, int32_t sy, int32_t ax, int32_t ay, int32_t bx, int32_t by)
{
    int64_t px = sx - ax, py = sy - ay;
    int64_t ex = (int64_t)bx - ax, ey = (int64_t)by - ay;
    int64_t len2 = ex * ex + ey * ey;
    int64_t dot = px * ex + py * ey;
    float d;
    if (len2 == 0 || dot <= 0) {
        d = sqrtf((float)(px * px + py * py));
    } else if (dot >= len2) {
        int64_t qx = sx - bx, qy = sy - by;
        d = sqrtf((float)(qx * qx + qy * qy));
    } else {
        float cr = (float)(px * ey - py * ex);
        d = fabsf(cr) / sqrtf((float)len2);
    }
    return d * (1.f / 256.f);
}

// Eqs. 1-4 for one fragment (Section "Focus+Context"); returns premultiplied RGBA.
__device__ __forceinline__ float4 shade_fragment(const TriShade& t, const int64_t l[3], int px, int py, int32_t sx, int32_t sy,
                                 const ShadeParams& sp)
{
    float inv_a = 1.f / (float)t.area;
    float lam[3] = {(float)l[0] * inv_a, (float)l[1] * inv_a, (float)l[2] * inv_a};
    float b[3], z_eye;
    if (sp.ortho) {
        b[0] = lam[0]; b[1] = lam[1]; b[2] = lam[2];
        z_eye = lam[0] * t.ed[0] + lam[1] * t.ed[1] + lam[2] * t.ed[2];
    } else {  // perspective-correct interpolation
        float q0 = lam[0] / t.ed[0], q1 = lam[1] / t.ed[1], q2 = lam[2] / t.ed[2];
        float Q = q0 + q1 + q2;
        float iQ = 1.f / Q;
        b[0] = q0 * iQ; b[1] = q1 * iQ; b[2] = q2 * iQ;
        z_eye = iQ;
    }
    float t_imp = b[0] * t.imp[0] + b[1] * t.imp[1] + b[2] * t.imp[2];
    // lens distance, normalised to 1 at the lens border
    float dist;
    if (sp.lens_mode == HEXFC_LENS_SCREEN) {
        float dx = ((float)px + 0.5f) - sp.lens_c[0], dy = ((float)py + 0.5f) - sp.lens_c[1];
        dist = sqrtf(dx * dx + dy * dy) * sp.lens_inv_r;
    } else {
        float Px = b[0] * t.P[0][0] + b[1] * t.P[1][0] + b[2] * t.P[2][0];
        float Py = b[0] * t.P[0][1] + b[1] * t.P[1][1] + b[2] * t.P[2][1];
        float Pz = b[0] * t.P[0][2] + b[1] * t.P[1][2] + b[2] * t.P[2][2];
        float dx = Px - sp.lens_c[0], dy = Py - sp.lens_c[1], dz = Pz - sp.lens_c[2];
        dist = sqrtf(dx * dx + dy * dy + dz * dz) * sp.lens_inv_r;
    }
    float focus = 1.f - smoothstepf(0.7f, 1.f, dist);
    // distances to the face edges: all, visible in focus, visible in context
    float d_a = INFINITY, d_f = INFINITY, d_c = INFINITY;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        int k1 = (k + 1) & 3;
        float d = seg_dist(sx, sy, t.FX[k], t.FY[k], t.FX[k1], t.FY[k1]);
        d_a = fminf(d_a, d);
        if ((t.masks >> k) & 1u) d_f = fminf(d_f, d);
        if ((t.masks >> (4 + k)) & 1u) d_c = fminf(d_c, d);
    }
    float g = 1.f;
    if (!sp.ortho) g = fminf(fmaxf(sp.zref / z_eye, sp.g_min), sp.g_max);
    // Eq. 1 with the depth-dependent width, halo band of the focus edges
    float w = (1.f + 0.3f * focus) * sp.w_base * g;
    bool e_focus = d_f <= w, e_context = d_c <= w;
    float h = sp.halo_scale * sp.w_base * focus * g;
    float alpha_e = (float)e_context + focus * ((float)e_focus - (float)e_context);
    bool halo = !e_focus && (d_f <= w + h) && focus > 0.f;
    if (halo) alpha_e = focus;
    // colour table and Eq. 2
    float tt = fminf(fmaxf((t_imp - sp.tf_lo) * sp.tf_inv, 0.f), 1.f);
    float ctf[3] = {tt, 0.f, 1.f - tt};
    float dk = 1.f - sp.darken * focus;
    bool accent = d_a <= (2.f / 3.f) * sp.w_base;
    float s_e = accent ? sp.s : 1.f;
    float cf[3], ce[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        ce[k] = halo ? 1.f : ctf[k] * dk;
        cf[k] = s_e > 1.f ? ctf[k] + sp.accent_beta * (1.f - ctf[k]) : ctf[k];
    }
    // Eq. 3 and Eq. 4
    float ahat = sp.alpha_min + sp.alpha_span * tt;
    float dc = fminf(dist, 1.f);
    float dc2 = dc * dc;
    float af = fminf(s_e * (ahat * (dc2 * dc2)), 1.f);
    float wf = (1.f - alpha_e) * af;
    return make_float4(alpha_e * ce[0] + wf * cf[0], alpha_e * ce[1] + wf * cf[1], alpha_e * ce[2] + wf * cf[2],
                       alpha_e + wf);
}

}  // namespace hexfc
