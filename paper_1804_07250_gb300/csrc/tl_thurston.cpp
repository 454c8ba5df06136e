// Thurston's algorithm for the extreme height functions of a region
// (Sec. 1.1; Thurston, "Conway's tiling groups", 1990).
//
// Along every edge u -> v the height step lies between lo = min(a_free,
// a_cross) and hi = max(a_free, a_cross); along a boundary edge it is
// exactly a_free.  The boundary heights are therefore fixed by the boundary
// itself.  The largest function obeying the interior bounds and the
// boundary values is h_top(v) = min over boundary vertices b of
// (h(b) + d(b, v)), d the shortest-path distance with cost hi for a step
// u -> v and -lo for a step v -> u; the smallest is the same construction
// applied to -h.  The region is tileable iff h_top agrees with the boundary
// values.  Costs are small non-negative integers, so the shortest paths use
// a bucket queue (Dial's algorithm): time proportional to the region size.
#include "tl_thurston.h"

#include "tiling.h"

#include <algorithm>
#include <climits>

namespace tl {

int thurston_heights(int nv, const std::vector<uint8_t>& active, const std::vector<HEdge>& edges, bool top,
                     std::vector<int>& h, std::string& why)
{
    // adjacency (CSR) over both directions of every edge
    std::vector<int> deg(nv + 1, 0);
    for (const HEdge& e : edges) {
        ++deg[e.u + 1];
        ++deg[e.v + 1];
    }
    for (int i = 0; i < nv; ++i) deg[i + 1] += deg[i];
    struct Step {
        int to, edge;
        bool fwd;
    };
    std::vector<Step> adj(deg[nv]);
    {
        std::vector<int> pos(deg.begin(), deg.end() - 1);
        for (int i = 0; i < (int)edges.size(); ++i) {
            adj[pos[edges[i].u]++] = Step{edges[i].v, i, true};
            adj[pos[edges[i].v]++] = Step{edges[i].u, i, false};
        }
    }
    int base = -1;
    for (int v = 0; v < nv; ++v)
        if (active[v]) {
            base = v;
            break;
        }
    if (base < 0) {
        why = "empty region";
        return TL_EINVAL;
    }
    // boundary heights: walk the boundary edges from the base vertex
    const int NONE = INT_MIN;
    std::vector<int> hb(nv, NONE);
    std::vector<uint8_t> on_boundary(nv, 0);
    for (const HEdge& e : edges)
        if (!e.interior) on_boundary[e.u] = on_boundary[e.v] = 1;
    if (!on_boundary[base]) {
        why = "lowest vertex is not on the boundary";
        return TL_ENOTSIMPLY;
    }
    std::vector<int> queue;
    queue.reserve(nv);
    hb[base] = 0;
    queue.push_back(base);
    for (size_t qi = 0; qi < queue.size(); ++qi) {
        const int u = queue[qi];
        for (int s = deg[u]; s < deg[u + 1]; ++s) {
            const HEdge& e = edges[adj[s].edge];
            if (e.interior) continue;
            const int w = adj[s].to;
            const int hw = hb[u] + (adj[s].fwd ? e.a_free : -e.a_free);
            if (hb[w] == NONE) {
                hb[w] = hw;
                queue.push_back(w);
            } else if (hb[w] != hw) {
                why = "boundary heights do not close up";
                return TL_ENOTTILEABLE;
            }
        }
    }
    for (int v = 0; v < nv; ++v)
        if (on_boundary[v] && hb[v] == NONE) {
            why = "boundary is not one closed path (region with a hole or in pieces)";
            return TL_ENOTSIMPLY;
        }
    // shortest paths from all boundary vertices at once (labels g = +-h)
    const int sgn = top ? 1 : -1;
    int lmin = INT_MAX;
    for (int v = 0; v < nv; ++v)
        if (on_boundary[v]) lmin = std::min(lmin, sgn * hb[v]);
    std::vector<int> dist(nv, INT_MAX);
    std::vector<std::vector<int>> bucket;
    auto push = [&](int v, int lab) {
        const size_t b = (size_t)(lab - lmin);
        if (b >= bucket.size()) bucket.resize(b + 1);
        bucket[b].push_back(v);
    };
    for (int v = 0; v < nv; ++v)
        if (on_boundary[v]) {
            dist[v] = sgn * hb[v];
            push(v, dist[v]);
        }
    for (size_t b = 0; b < bucket.size(); ++b) {
        for (size_t i = 0; i < bucket[b].size(); ++i) {
            const int u = bucket[b][i];
            const int lab = (int)b + lmin;
            if (dist[u] != lab) continue;   // stale entry
            for (int s = deg[u]; s < deg[u + 1]; ++s) {
                const HEdge& e = edges[adj[s].edge];
                if (!e.interior) continue;
                const int lo = std::min(e.a_free, e.a_cross), hi = std::max(e.a_free, e.a_cross);
                // bound on g(to) - g(u): top: h steps <= hi forward, <= -lo backward;
                // bottom (g = -h): <= -lo forward, <= hi backward
                const int cost = adj[s].fwd ? (top ? hi : -lo) : (top ? -lo : hi);
                const int w = adj[s].to;
                if (lab + cost < dist[w]) {
                    dist[w] = lab + cost;
                    push(w, dist[w]);
                }
            }
        }
        std::vector<int>().swap(bucket[b]);
    }
    h.assign(nv, 0);
    for (int v = 0; v < nv; ++v) {
        if (!active[v]) continue;
        if (dist[v] == INT_MAX) {
            why = "region is not connected";
            return TL_ENOTSIMPLY;
        }
        h[v] = sgn * dist[v];
        if (on_boundary[v] && h[v] != hb[v]) {
            why = "no tiling agrees with the boundary heights";
            return TL_ENOTTILEABLE;
        }
    }
    for (const HEdge& e : edges) {
        const int d = h[e.v] - h[e.u];
        if (d != e.a_free && !(e.interior && d == e.a_cross)) {
            why = "extreme heights do not define a tiling";
            return TL_ENOTTILEABLE;
        }
    }
    return TL_OK;
}

void tiling_from_heights(const std::vector<HEdge>& edges, const std::vector<int>& h, uint8_t* canon)
{
    for (const HEdge& e : edges)
        if (e.interior) canon[e.slot] = (h[e.v] - h[e.u] == e.a_cross) ? 1 : 0;
}

}  // namespace tl
