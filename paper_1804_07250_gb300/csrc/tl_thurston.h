// Extreme height functions of a simply-connected lattice region (Sec. 1.1:
// the maximal and minimal tilings T_max, T_min and tileability by
// Thurston's algorithm).  Host code, used to build domains from a boundary
// path and the top / bottom configurations for coupling from the past.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace tl {

// One lattice edge of the region, directed from vertex u to vertex v.  The
// height changes by `a_free` along it when no tile crosses it and by
// `a_cross` when one does (a_free != a_cross).  `interior` edges border two
// region cells and may be crossed; boundary edges border one and never are.
// `slot` is the edge's index in the canonical configuration array.
struct HEdge {
    int u, v;
    int8_t a_free, a_cross;
    uint8_t interior;
    int64_t slot;
};

// Height function of the tiling with the largest (top = true) or smallest
// heights, on vertices 0..nv-1 (`active[v]` marks the region's vertices).
// The boundary heights are fixed by walking the boundary edges from the
// lowest-numbered active vertex (height 0).  Errors: TL_ENOTSIMPLY if the
// boundary edges do not form one connected cycle through every boundary
// vertex or the region is not connected, TL_ENOTTILEABLE if the boundary
// heights are inconsistent or the extreme function violates them.
int thurston_heights(int nv, const std::vector<uint8_t>& active, const std::vector<HEdge>& edges, bool top,
                     std::vector<int>& h, std::string& why);

// Configuration from a height function: bit `slot` = 1 for every interior
// edge whose height step equals its a_cross.
void tiling_from_heights(const std::vector<HEdge>& edges, const std::vector<int>& h, uint8_t* canon);

}  // namespace tl
