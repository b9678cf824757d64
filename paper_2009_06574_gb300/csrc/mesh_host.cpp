// Unique faces and edges of a hexahedral mesh (host precomputation).
//
// Every geometric face is drawn once as a quad of two triangles (Section
// "Method Overview"; Section "GPU Implementation"). A face is identified by
// its sorted vertex ids; its id is the rank of that tuple, its corner 0 is
// the smallest vertex id and corner 1 the smaller of corner 0's two
// neighbours on the quad, so both cells sharing a face produce the same quad
// and the same diagonal (corner 0 to corner 2). Edges are unique vertex pairs;
// an edge's LoD level is the largest of the levels given for it by its cells
// (Section "Level of Detail Structure": an edge carries the highest level at
// which it still exists). A face of one cell is on the boundary surface, whose
// depth image gives the silhouettes (Section "Blending Focus and Context").
#include "mesh_host.h"

#include <algorithm>
#include <cmath>
#include <numeric>

namespace hexfc {
namespace {

// cyclic corner order of the six faces of a VTK hexahedron
const int kHexFace[6][4] = {{0, 1, 2, 3}, {4, 5, 6, 7}, {0, 1, 5, 4}, {1, 2, 6, 5}, {2, 3, 7, 6}, {3, 0, 4, 7}};
// the twelve cell edges in the order of the per-cell-edge level input
const int kHexEdge[12][2] = {{0, 1}, {1, 2}, {2, 3}, {3, 0}, {4, 5}, {5, 6},
                             {6, 7}, {7, 4}, {0, 4}, {1, 5}, {2, 6}, {3, 7}};

struct FaceRec {
    uint64_t k0, k1;   // sorted ids packed: (s0, s1), (s2, s3)
    int32_t c[4];      // canonical cyclic corners
};

inline uint64_t pack(int32_t a, int32_t b) { return ((uint64_t)(uint32_t)a << 32) | (uint32_t)b; }

}  // namespace

int build_host_tables(const float* verts, int64_t n_verts, const int32_t* cells, int64_t n_cells,
                      const uint8_t* cell_edge_level, HostTables& out)
{
    for (int64_t i = 0; i < 3 * n_verts; ++i)
        if (!std::isfinite(verts[i])) return -1;
    for (int64_t i = 0; i < 8 * n_cells; ++i)
        if (cells[i] < 0 || cells[i] >= n_verts) return -1;

    // ---- faces
    std::vector<FaceRec> fr((size_t)(6 * n_cells));
    for (int64_t c = 0; c < n_cells; ++c) {
        const int32_t* cv = cells + 8 * c;
        for (int f = 0; f < 6; ++f) {
            int32_t q[4];
            for (int k = 0; k < 4; ++k) q[k] = cv[kHexFace[f][k]];
            int m = 0;
            for (int k = 1; k < 4; ++k)
                if (q[k] < q[m]) m = k;
            bool fwd = q[(m + 1) & 3] < q[(m + 3) & 3];
            FaceRec& r = fr[(size_t)(6 * c + f)];
            for (int k = 0; k < 4; ++k) r.c[k] = fwd ? q[(m + k) & 3] : q[(m - k + 4) & 3];
            int32_t s[4] = {q[0], q[1], q[2], q[3]};
            std::sort(s, s + 4);
            r.k0 = pack(s[0], s[1]);
            r.k1 = pack(s[2], s[3]);
        }
    }
    std::sort(fr.begin(), fr.end(), [](const FaceRec& a, const FaceRec& b) {
        return a.k0 != b.k0 ? a.k0 < b.k0 : a.k1 < b.k1;
    });
    size_t nf = 0;
    std::vector<uint32_t> ncell;   // cells sharing each unique face
    ncell.reserve(fr.size());
    for (size_t i = 0; i < fr.size(); ++i) {
        if (nf == 0 || fr[i].k0 != fr[nf - 1].k0 || fr[i].k1 != fr[nf - 1].k1) {
            fr[nf++] = fr[i];
            ncell.push_back(1);
        } else {
            ++ncell.back();
        }
    }
    fr.resize(nf);
    out.fbound.resize(nf);
    for (size_t f = 0; f < nf; ++f) out.fbound[f] = ncell[f] == 1 ? 1 : 0;

    // ---- edges
    size_t ne_all = (size_t)(12 * n_cells);
    std::vector<uint64_t> ekey(ne_all);
    for (int64_t c = 0; c < n_cells; ++c)
        for (int k = 0; k < 12; ++k) {
            int32_t a = cells[8 * c + kHexEdge[k][0]], b = cells[8 * c + kHexEdge[k][1]];
            ekey[(size_t)(12 * c + k)] = a < b ? pack(a, b) : pack(b, a);
        }
    std::vector<uint32_t> order(ne_all);
    std::iota(order.begin(), order.end(), 0u);
    std::sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) { return ekey[x] < ekey[y]; });
    std::vector<uint64_t> ukey;
    ukey.reserve(ne_all / 3 + 16);
    out.cell_edges.assign(ne_all, 0);
    out.elevel.clear();
    for (size_t i = 0; i < ne_all; ++i) {
        uint32_t e = order[i];
        if (ukey.empty() || ukey.back() != ekey[e]) {
            ukey.push_back(ekey[e]);
            out.elevel.push_back(0);
        }
        int32_t id = (int32_t)(ukey.size() - 1);
        out.cell_edges[e] = id;
        uint8_t lv = cell_edge_level ? cell_edge_level[e] : 0;
        if (lv > out.elevel[(size_t)id]) out.elevel[(size_t)id] = lv;
    }

    out.n_faces = (int64_t)nf;
    out.n_edges = (int64_t)ukey.size();
    out.fverts.resize(4 * nf);
    out.fedges.resize(4 * nf);
    for (size_t f = 0; f < nf; ++f)
        for (int k = 0; k < 4; ++k) {
            int32_t a = fr[f].c[k], b = fr[f].c[(k + 1) & 3];
            out.fverts[4 * f + k] = a;
            uint64_t key = a < b ? pack(a, b) : pack(b, a);
            auto it = std::lower_bound(ukey.begin(), ukey.end(), key);
            out.fedges[4 * f + k] = (it != ukey.end() && *it == key) ? (int32_t)(it - ukey.begin()) : -1;
            if (out.fedges[4 * f + k] < 0) return -1;  // a face edge that is no cell edge
        }
    return 0;
}

}  // namespace hexfc
