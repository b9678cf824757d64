// Geometry and fragment stages of the renderer.
//
//   k_vertex_setup  per vertex: camera transform in double (no FMA), window
//                   position snapped to 16.8 fixed point, 24-bit window depth.
//   k_face_setup    per unique face: gather the 4 projected corners, edge
//                   visibility masks of Eq. 1, triangle validity, and the
//                   number of 16x16 tiles each triangle's box touches.
//   k_bin_fill      per face: append 2*face+tri to the list of every touched tile.
//   k_count         per tile (one thread per pixel): exact coverage count.
//   k_fill          per tile: exact coverage again; every covered sample is
//                   shaded with Eqs. 1-4 and written at its pixel's offset.
//
// Each face is drawn as two triangles (Section "Method Overview"; Section "GPU
// Implementation"), all covered samples are kept (per-pixel fragment lists,
// Section "GPU Implementation"), and the fragment shader computes focus from
// the lens, the edge distance to the four face edges ignoring invisible ones,
// and Eqs. 1-4 (Section "Focus+Context").
#include "raster_common.cuh"

namespace hexfc {
namespace {

inline unsigned grid_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// ------------------------------------------------------------------ vertex stage

__global__ void k_vertex_setup(const float* __restrict__ verts, int64_t n, CamParams cam,
                               int4* __restrict__ vproj, float* __restrict__ ved)
{
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    double dx = __dsub_rn((double)verts[3 * v], cam.eye[0]);
    double dy = __dsub_rn((double)verts[3 * v + 1], cam.eye[1]);
    double dz = __dsub_rn((double)verts[3 * v + 2], cam.eye[2]);
    double ex = __dadd_rn(__dadd_rn(__dmul_rn(dx, cam.R[0]), __dmul_rn(dy, cam.R[1])), __dmul_rn(dz, cam.R[2]));
    double ey = __dadd_rn(__dadd_rn(__dmul_rn(dx, cam.U[0]), __dmul_rn(dy, cam.U[1])), __dmul_rn(dz, cam.U[2]));
    double ed = __dadd_rn(__dadd_rn(__dmul_rn(dx, cam.F[0]), __dmul_rn(dy, cam.F[1])), __dmul_rn(dz, cam.F[2]));
    double xw, yw, z;
    if (cam.ortho) {
        xw = __dadd_rn(cam.cx, __dmul_rn(ex, cam.scale));
        yw = __dsub_rn(cam.cy, __dmul_rn(ey, cam.scale));
        z = __ddiv_rn(__dsub_rn(ed, cam.znear), __dsub_rn(cam.zfar, cam.znear));
    } else {
        xw = __dadd_rn(cam.cx, __dmul_rn(__ddiv_rn(ex, ed), cam.focal));
        yw = __dsub_rn(cam.cy, __dmul_rn(__ddiv_rn(ey, ed), cam.focal));
        z = __dmul_rn(cam.zf_over, __dsub_rn(1.0, __ddiv_rn(cam.znear, ed)));
    }
    bool valid = (ed > cam.znear) && (ed < cam.zfar) && (fabs(xw) <= 16384.0) && (fabs(yw) <= 16384.0);
    int4 o = make_int4(0, 0, 0, 0);
    if (valid) {
        z = fmin(fmax(z, 0.0), 1.0);
        o.x = (int32_t)rint(__dmul_rn(xw, 256.0));
        o.y = (int32_t)rint(__dmul_rn(yw, 256.0));
        o.z = (int32_t)(uint32_t)rint(__dmul_rn(z, 16777215.0));
        o.w = 1;
    }
    vproj[v] = o;
    ved[v] = (float)ed;
}

// ------------------------------------------------------------------ face stage

__device__ __forceinline__ void tile_range(const TriGeom& t, int& tx0, int& ty0, int& tx1, int& ty1)
{
    tx0 = t.bx0 / kTile; tx1 = t.bx1 / kTile;
    ty0 = t.by0 / kTile; ty1 = t.by1 / kTile;
}

__global__ void k_face_setup(const int4* __restrict__ fverts, const int4* __restrict__ fedges,
                             const uint8_t* __restrict__ elevel, const float* __restrict__ eattr,
                             const int4* __restrict__ vproj, const float* __restrict__ ved, int64_t n_faces,
                             int lod, float delta, int W, int H, int tiles_x,
                             int4* __restrict__ fx, int4* __restrict__ fy, uint4* __restrict__ fz,
                             float4* __restrict__ fed, uint32_t* __restrict__ fflags,
                             uint32_t* __restrict__ tile_cnt)
{
    int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n_faces) return;
    int4 c = fverts[f];
    int id[4] = {c.x, c.y, c.z, c.w};
    int32_t X[4], Y[4];
    uint32_t Z[4];
    float E[4];
    bool ok[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        int4 p = vproj[id[k]];
        X[k] = p.x; Y[k] = p.y; Z[k] = (uint32_t)p.z; ok[k] = p.w != 0;
        E[k] = ved[id[k]];
    }
    int4 e = fedges[f];
    int eid[4] = {e.x, e.y, e.z, e.w};
    uint32_t flags = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        bool vis_c = (int)elevel[eid[k]] >= lod;
        bool vis_f = vis_c || eattr[eid[k]] >= delta;
        flags |= (vis_f ? 1u : 0u) << k;
        flags |= (vis_c ? 1u : 0u) << (4 + k);
    }
#pragma unroll
    for (int tri = 0; tri < 2; ++tri) {
        bool vok = ok[0] && (tri == 0 ? (ok[1] && ok[2]) : (ok[2] && ok[3]));
        if (!vok) continue;
        TriGeom t;
        tri_setup(X, Y, tri, W, H, t);
        if (!t.valid) continue;
        flags |= 1u << (8 + tri);
        int tx0, ty0, tx1, ty1;
        tile_range(t, tx0, ty0, tx1, ty1);
        for (int ty = ty0; ty <= ty1; ++ty)
            for (int tx = tx0; tx <= tx1; ++tx) atomicAdd(tile_cnt + ty * tiles_x + tx, 1u);
    }
    fx[f] = make_int4(X[0], X[1], X[2], X[3]);
    fy[f] = make_int4(Y[0], Y[1], Y[2], Y[3]);
    fz[f] = make_uint4(Z[0], Z[1], Z[2], Z[3]);
    fed[f] = make_float4(E[0], E[1], E[2], E[3]);
    fflags[f] = flags;
}

__global__ void k_bin_fill(const int4* __restrict__ fx, const int4* __restrict__ fy,
                           const uint32_t* __restrict__ fflags, int64_t n_faces, int W, int H, int tiles_x,
                           int reverse, const uint64_t* __restrict__ tile_off, uint32_t* __restrict__ tile_cur,
                           uint32_t* __restrict__ bins)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_faces) return;
    int64_t f = reverse ? (n_faces - 1 - i) : i;
    uint32_t flags = fflags[f];
    if ((flags & (3u << 8)) == 0) return;
    int4 a = fx[f], b = fy[f];
    int32_t X[4] = {a.x, a.y, a.z, a.w}, Y[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
    for (int tri = 0; tri < 2; ++tri) {
        if (!(flags & (1u << (8 + tri)))) continue;
        TriGeom t;
        tri_setup(X, Y, tri, W, H, t);
        int tx0, ty0, tx1, ty1;
        tile_range(t, tx0, ty0, tx1, ty1);
        for (int ty = ty0; ty <= ty1; ++ty)
            for (int tx = tx0; tx <= tx1; ++tx) {
                int tile = ty * tiles_x + tx;
                uint32_t slot = atomicAdd(tile_cur + tile, 1u);
                bins[tile_off[tile] + slot] = (uint32_t)(2 * f + tri);
            }
    }
}

// ------------------------------------------------------------------ raster per tile

// Triangle data staged in shared memory for one chunk of a tile's list.
struct TriS {
    int32_t X[3], Y[3];
    int16_t bx0, by0, bx1, by1;
    uint32_t meta;   // bits 0-2 top-left of the edge opposite vertex k
};

__device__ __forceinline__ void stage_tri(const int4* __restrict__ fx, const int4* __restrict__ fy,
                                          uint32_t f2t, int W, int H, TriS& s, TriGeom& t)
{
    uint32_t f = f2t >> 1, tri = f2t & 1;
    int4 a = fx[f], b = fy[f];
    int32_t X[4] = {a.x, a.y, a.z, a.w}, Y[4] = {b.x, b.y, b.z, b.w};
    tri_setup(X, Y, (int)tri, W, H, t);
    uint32_t meta = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        s.X[k] = t.X[k];
        s.Y[k] = t.Y[k];
        int a0 = (k + 1) % 3, b0 = (k + 2) % 3;
        meta |= (top_left(t.X[a0], t.Y[a0], t.X[b0], t.Y[b0]) ? 1u : 0u) << k;
    }
    s.bx0 = (int16_t)t.bx0; s.by0 = (int16_t)t.by0; s.bx1 = (int16_t)t.bx1; s.by1 = (int16_t)t.by1;
    s.meta = meta;
}

// Exact coverage of sample (sx, sy) (16.8) by a staged triangle; barycentric weights out.
__device__ __forceinline__ bool covers(const TriS& s, int px, int py, int32_t sx, int32_t sy, int64_t l[3])
{
    if (px < s.bx0 || px > s.bx1 || py < s.by0 || py > s.by1) return false;
    bool in = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        int a = (k + 1) % 3, b = (k + 2) % 3;
        int64_t e = edge_fn(s.X[a], s.Y[a], s.X[b], s.Y[b], sx, sy);
        l[k] = e;
        in = in && (e > 0 || (e == 0 && ((s.meta >> k) & 1u)));
    }
    return in;
}

__global__ void __launch_bounds__(kTilePix) k_count(const uint64_t* __restrict__ tile_off,
                                                    const uint32_t* __restrict__ bins,
                                                    const int4* __restrict__ fx, const int4* __restrict__ fy,
                                                    int tiles_x, int W, int H, uint32_t* __restrict__ cnt)
{
    __shared__ TriS s_tri[kTilePix];
    int tile = blockIdx.x;
    int tx = tile % tiles_x, ty = tile / tiles_x;
    int px = tx * kTile + (threadIdx.x & (kTile - 1));
    int py = ty * kTile + (threadIdx.x / kTile);
    int32_t sx = 256 * px + 128, sy = 256 * py + 128;
    uint64_t beg = tile_off[tile], end = tile_off[tile + 1];
    uint32_t n = 0;
    for (uint64_t base = beg; base < end; base += kTilePix) {
        uint64_t i = base + threadIdx.x;
        if (i < end) {
            TriGeom t;
            stage_tri(fx, fy, bins[i], W, H, s_tri[threadIdx.x], t);
        }
        __syncthreads();
        int m = (int)min((uint64_t)kTilePix, end - base);
        for (int j = 0; j < m; ++j) {
            int64_t l[3];
            n += covers(s_tri[j], px, py, sx, sy, l) ? 1u : 0u;
        }
        __syncthreads();
    }
    cnt[(int64_t)tile * kTilePix + threadIdx.x] = n;
}

// ------------------------------------------------------------------ fill + shade

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
__device__ float4 shade_fragment(const TriShade& t, const int64_t l[3], int px, int py, int32_t sx, int32_t sy,
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

__global__ void __launch_bounds__(kTilePix) k_fill(const uint64_t* __restrict__ tile_off,
                                                   const uint32_t* __restrict__ bins,
                                                   const int4* __restrict__ fx, const int4* __restrict__ fy,
                                                   const uint4* __restrict__ fz, const float4* __restrict__ fed,
                                                   const uint32_t* __restrict__ fflags,
                                                   const float4* __restrict__ fimp, const float4* __restrict__ fpx,
                                                   const float4* __restrict__ fpy, const float4* __restrict__ fpz,
                                                   int tiles_x, int W, int H, ShadeParams sp,
                                                   const uint64_t* __restrict__ off, uint64_t* __restrict__ key,
                                                   float4* __restrict__ rgba, uint64_t* __restrict__ err)
{
    __shared__ TriS s_tri[kTilePix];
    __shared__ TriShade s_sh[kTilePix];
    int tile = blockIdx.x;
    int tx = tile % tiles_x, ty = tile / tiles_x;
    int px = tx * kTile + (threadIdx.x & (kTile - 1));
    int py = ty * kTile + (threadIdx.x / kTile);
    int32_t sx = 256 * px + 128, sy = 256 * py + 128;
    uint64_t beg = tile_off[tile], end = tile_off[tile + 1];
    uint64_t o = off[(int64_t)tile * kTilePix + threadIdx.x];
    const uint64_t o_end = off[(int64_t)tile * kTilePix + threadIdx.x + 1];
    bool bad = false;
    for (uint64_t base = beg; base < end; base += kTilePix) {
        uint64_t i = base + threadIdx.x;
        if (i < end) {
            uint32_t f2t = bins[i];
            TriGeom t;
            stage_tri(fx, fy, f2t, W, H, s_tri[threadIdx.x], t);
            uint32_t f = f2t >> 1;
            TriShade& S = s_sh[threadIdx.x];
            int4 a = fx[f], b = fy[f];
            S.FX[0] = a.x; S.FX[1] = a.y; S.FX[2] = a.z; S.FX[3] = a.w;
            S.FY[0] = b.x; S.FY[1] = b.y; S.FY[2] = b.z; S.FY[3] = b.w;
            uint4 z4 = fz[f];
            float4 e4 = fed[f], i4 = fimp[f], x4 = fpx[f], y4 = fpy[f], w4 = fpz[f];
            uint32_t zz[4] = {z4.x, z4.y, z4.z, z4.w};
            float ee[4] = {e4.x, e4.y, e4.z, e4.w}, ii[4] = {i4.x, i4.y, i4.z, i4.w};
            float xx[4] = {x4.x, x4.y, x4.z, x4.w}, yy[4] = {y4.x, y4.y, y4.z, y4.w}, ww[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                int c = t.vi[k];
                // select corner c without dynamic register indexing
                uint32_t zc = c == 0 ? zz[0] : c == 1 ? zz[1] : c == 2 ? zz[2] : zz[3];
                float ec = c == 0 ? ee[0] : c == 1 ? ee[1] : c == 2 ? ee[2] : ee[3];
                float ic = c == 0 ? ii[0] : c == 1 ? ii[1] : c == 2 ? ii[2] : ii[3];
                float xc = c == 0 ? xx[0] : c == 1 ? xx[1] : c == 2 ? xx[2] : xx[3];
                float yc = c == 0 ? yy[0] : c == 1 ? yy[1] : c == 2 ? yy[2] : yy[3];
                float wc = c == 0 ? ww[0] : c == 1 ? ww[1] : c == 2 ? ww[2] : ww[3];
                S.z[k] = zc; S.ed[k] = ec; S.imp[k] = ic;
                S.P[k][0] = xc; S.P[k][1] = yc; S.P[k][2] = wc;
            }
            S.area = t.area;
            S.f2t = f2t;
            S.masks = fflags[f] & 0xFFu;
        }
        __syncthreads();
        int m = (int)min((uint64_t)kTilePix, end - base);
        for (int j = 0; j < m; ++j) {
            int64_t l[3];
            if (!covers(s_tri[j], px, py, sx, sy, l)) continue;
            const TriShade& S = s_sh[j];
            uint32_t z = sample_depth(S.z[0], S.z[1], S.z[2], l[1], l[2], S.area, bad);
            float4 c = shade_fragment(S, l, px, py, sx, sy, sp);
            if (o < o_end) {  // the count pass sized this list; never write past it
                key[o] = ((uint64_t)z << 32) | (uint64_t)S.f2t;
                rgba[o] = c;
            } else {
                bad = true;
            }
            ++o;
        }
        __syncthreads();
    }
    if (bad) atomicOr(reinterpret_cast<unsigned long long*>(err), 1ull);
}

}  // namespace

cudaError_t launch_vertex_setup(const DevMesh& m, const CamParams& cam, FrameBufs& fb, cudaStream_t s)
{
    k_vertex_setup<<<grid_for(m.n_verts, 256), 256, 0, s>>>(m.verts, m.n_verts, cam, fb.vproj, fb.ved);
    return cudaGetLastError();
}

cudaError_t launch_face_setup(const DevMesh& m, const CamParams& cam, int lod, float delta, FrameBufs& fb,
                              int tiles_x, int tiles_y, cudaStream_t s)
{
    (void)tiles_y;
    k_face_setup<<<grid_for(m.n_faces, 256), 256, 0, s>>>(m.fverts, m.fedges, m.elevel, m.eattr, fb.vproj,
                                                           fb.ved, m.n_faces, lod, delta, cam.W, cam.H, tiles_x,
                                                           fb.fx, fb.fy, fb.fz, fb.fed, fb.fflags, fb.tile_cnt);
    return cudaGetLastError();
}

cudaError_t launch_bin_fill(const DevMesh& m, FrameBufs& fb, int tiles_x, int W, int H, int reverse,
                            cudaStream_t s)
{
    k_bin_fill<<<grid_for(m.n_faces, 256), 256, 0, s>>>(fb.fx, fb.fy, fb.fflags, m.n_faces, W, H, tiles_x, reverse,
                                                         fb.tile_off, fb.tile_cur, fb.bins);
    return cudaGetLastError();
}

cudaError_t launch_count(FrameBufs& fb, int tiles_x, int tiles_y, int W, int H, cudaStream_t s)
{
    k_count<<<(unsigned)(tiles_x * tiles_y), kTilePix, 0, s>>>(fb.tile_off, fb.bins, fb.fx, fb.fy, tiles_x, W, H,
                                                                fb.cnt);
    return cudaGetLastError();
}

cudaError_t launch_fill(const DevMesh& m, FrameBufs& fb, const ShadeParams& sp, int tiles_x, int tiles_y, int W,
                        int H, cudaStream_t s)
{
    k_fill<<<(unsigned)(tiles_x * tiles_y), kTilePix, 0, s>>>(fb.tile_off, fb.bins, fb.fx, fb.fy, fb.fz, fb.fed,
                                                               fb.fflags, m.fimp, m.fpx, m.fpy, m.fpz, tiles_x, W, H,
                                                               sp, fb.off, fb.key, fb.rgba, fb.scal + 5);
    return cudaGetLastError();
}

}  // namespace hexfc
