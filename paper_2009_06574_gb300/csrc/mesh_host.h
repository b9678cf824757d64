// Host-side mesh tables of the hexfc library (C++ only).
#pragma once
#include <stdint.h>

#include <vector>

namespace hexfc {

struct HostTables {
    std::vector<int32_t> fverts;     // [F*4] canonical corners of each unique face
    std::vector<int32_t> fedges;     // [F*4] unique edge id of local edge k = (c_k, c_k+1)
    std::vector<int32_t> cell_edges; // [C*12] unique edge id of each cell edge
    std::vector<uint8_t> elevel;     // [E] LoD level of each unique edge
    std::vector<uint8_t> fbound;     // [F] 1: the face belongs to one cell (the boundary surface)
    int64_t n_faces = 0, n_edges = 0;
};

// Returns 0 on success, -1 on an invalid mesh (index out of range, non-finite vertex).
int build_host_tables(const float* verts, int64_t n_verts, const int32_t* cells, int64_t n_cells,
                      const uint8_t* cell_edge_level, HostTables& out);

}  // namespace hexfc
