// Per-cell quality (Jacobian of the cube-to-cell map) and importance max-reduce.
//
// Quality: the paper names the Jacobian-based deformation measures (Section
// "Introduction"; Section "Results and Analysis": per-cell scaled Jacobian
// ratio) without printing a formula. Evaluated here: the Jacobian at the 8
// corners (three edge vectors to the corner's neighbours) and at the cell
// centre (the three principal axes, sums of the four parallel edges):
//   scaled Jacobian = min det of the unit-length vectors,
//   Jacobian ratio  = min det / max det (centre axes scaled by 1/4),
//   importance      = clamp(1 - scaled Jacobian, 0, 1).
// Importance: every vertex and every edge takes the maximum importance of the
// cells sharing it (Section "Method Overview").
#include "hexfc_internal.cuh"

namespace hexfc {
namespace {

// neighbours of corner k of a VTK hexahedron, right-handed
__constant__ int8_t c_corner_nb[8][3] = {{1, 3, 4}, {2, 0, 5}, {3, 1, 6}, {0, 2, 7},
                                         {7, 5, 0}, {4, 6, 1}, {5, 7, 2}, {6, 4, 3}};

__device__ __forceinline__ float det3f(float3 a, float3 b, float3 c)
{
    return a.x * (b.y * c.z - b.z * c.y) + a.y * (b.z * c.x - b.x * c.z) + a.z * (b.x * c.y - b.y * c.x);
}
__device__ __forceinline__ float3 sub3(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 add3(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float len3(float3 a) { return sqrtf(a.x * a.x + a.y * a.y + a.z * a.z); }

__global__ void k_cell_quality(const float* __restrict__ verts, const int32_t* __restrict__ cells,
                               int64_t n_cells, int metric, float* __restrict__ out)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cells) return;
    const int4* cc = reinterpret_cast<const int4*>(cells + 8 * c);
    int4 a = __ldg(cc), b = __ldg(cc + 1);
    int id[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    float3 p[8];
#pragma unroll
    for (int k = 0; k < 8; ++k)
        p[k] = make_float3(__ldg(verts + 3 * (int64_t)id[k]), __ldg(verts + 3 * (int64_t)id[k] + 1),
                           __ldg(verts + 3 * (int64_t)id[k] + 2));
    float sj = 3.0e38f, dmin = 3.0e38f, dmax = -3.0e38f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        float3 e0 = sub3(p[c_corner_nb[k][0]], p[k]);
        float3 e1 = sub3(p[c_corner_nb[k][1]], p[k]);
        float3 e2 = sub3(p[c_corner_nb[k][2]], p[k]);
        float d = det3f(e0, e1, e2);
        float l = len3(e0) * len3(e1) * len3(e2);
        float nd = l > 0.f ? d / l : 0.f;
        sj = fminf(sj, nd);
        dmin = fminf(dmin, d);
        dmax = fmaxf(dmax, d);
    }
    {
        float3 X0 = add3(add3(sub3(p[1], p[0]), sub3(p[2], p[3])), add3(sub3(p[5], p[4]), sub3(p[6], p[7])));
        float3 X1 = add3(add3(sub3(p[3], p[0]), sub3(p[2], p[1])), add3(sub3(p[7], p[4]), sub3(p[6], p[5])));
        float3 X2 = add3(add3(sub3(p[4], p[0]), sub3(p[5], p[1])), add3(sub3(p[6], p[2]), sub3(p[7], p[3])));
        float d = det3f(X0, X1, X2);
        float l = len3(X0) * len3(X1) * len3(X2);
        float nd = l > 0.f ? d / l : 0.f;
        sj = fminf(sj, nd);
        float dc = d * (1.0f / 64.0f);
        dmin = fminf(dmin, dc);
        dmax = fmaxf(dmax, dc);
    }
    float v;
    if (metric == HEXFC_METRIC_SCALED_JACOBIAN) v = sj;
    else if (metric == HEXFC_METRIC_JACOBIAN_RATIO) v = dmax > 0.f ? dmin / dmax : -1.f;
    else v = fminf(fmaxf(1.f - sj, 0.f), 1.f);
    out[c] = v;
}

// float <-> int order-preserving map, so that atomicMax on int is a float max
__device__ __forceinline__ int32_t f2key(float f)
{
    int32_t i = __float_as_int(f);
    return i >= 0 ? i : (i ^ 0x7FFFFFFF);
}
__device__ __forceinline__ float key2f(int32_t k) { return __int_as_float(k >= 0 ? k : (k ^ 0x7FFFFFFF)); }

// Both key arrays (vertices, then edges) to v in one launch.
__global__ void k_init_keys(int32_t* __restrict__ a, int64_t na, int32_t* __restrict__ b, int64_t nb, int32_t v)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < na) a[i] = v;
    else if (i - na < nb) b[i - na] = v;
}

__global__ void k_importance_scatter(const int32_t* __restrict__ cells, const int32_t* __restrict__ cell_edges,
                                     const float* __restrict__ cell_imp, int64_t n_cells,
                                     int32_t* __restrict__ vkey, int32_t* __restrict__ ekey)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cells) return;
    int32_t k = f2key(cell_imp[c]);
#pragma unroll
    for (int j = 0; j < 8; ++j) atomicMax(vkey + cells[8 * c + j], k);
#pragma unroll
    for (int j = 0; j < 12; ++j) atomicMax(ekey + cell_edges[12 * c + j], k);
}

// Both key arrays back to floats in one launch (vertices, then edges); an
// unreferenced vertex or edge gets 0.
__global__ void k_key_to_float(const int32_t* __restrict__ ka, float* __restrict__ oa, int64_t na,
                               const int32_t* __restrict__ kb, float* __restrict__ ob, int64_t nb)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < na) {
        const int32_t k = ka[i];
        oa[i] = (k == INT32_MIN) ? 0.f : key2f(k);
    } else if (i - na < nb) {
        const int32_t k = kb[i - na];
        ob[i - na] = (k == INT32_MIN) ? 0.f : key2f(k);
    }
}

// Static face records: importance and world position of the 4 corners. The
// positions do not change after the upload: with positions false only the
// importances are written.
__global__ void k_face_static(const int4* __restrict__ fverts, const float* __restrict__ vimp,
                              const float* __restrict__ verts, int64_t n_faces, bool positions,
                              FaceStatic* __restrict__ fstat)
{
    int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n_faces) return;
    int4 c = fverts[f];
    int id[4] = {c.x, c.y, c.z, c.w};
    FaceStatic& r = fstat[f];
    r.imp = make_float4(vimp[id[0]], vimp[id[1]], vimp[id[2]], vimp[id[3]]);
    if (!positions) return;
    float x[4], y[4], z[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        x[k] = verts[3 * (int64_t)id[k]];
        y[k] = verts[3 * (int64_t)id[k] + 1];
        z[k] = verts[3 * (int64_t)id[k] + 2];
    }
    r.px = make_float4(x[0], x[1], x[2], x[3]);
    r.py = make_float4(y[0], y[1], y[2], y[3]);
    r.pz = make_float4(z[0], z[1], z[2], z[3]);
}

inline unsigned grid_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

cudaError_t launch_cell_quality(const DevMesh& m, int metric, float* out, cudaStream_t s)
{
    if (m.n_cells > 0)
        k_cell_quality<<<grid_for(m.n_cells, 256), 256, 0, s>>>(m.verts, m.cells, m.n_cells, metric, out);
    return cudaGetLastError();
}

cudaError_t launch_importance(const DevMesh& m, bool positions, cudaStream_t s)
{
    const int64_t nk = m.n_verts + m.n_edges;
    k_init_keys<<<grid_for(nk, 256), 256, 0, s>>>(m.vkey, m.n_verts, m.ekey, m.n_edges, INT32_MIN);
    k_importance_scatter<<<grid_for(m.n_cells, 256), 256, 0, s>>>(m.cells, m.cell_edges, m.cell_imp,
                                                                   m.n_cells, m.vkey, m.ekey);
    k_key_to_float<<<grid_for(nk, 256), 256, 0, s>>>(m.vkey, m.vimp, m.n_verts, m.ekey, m.eattr, m.n_edges);
    k_face_static<<<grid_for(m.n_faces, 256), 256, 0, s>>>(m.fverts, m.vimp, m.verts, m.n_faces, positions,
                                                           m.fstat);
    return cudaGetLastError();
}

}  // namespace hexfc
