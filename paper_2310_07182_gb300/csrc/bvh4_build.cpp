// bvh4_build.cpp -- BVH4: the BVH2 collapsed into 4-wide nodes with FP32 child boxes.
// The paper names a BVH as its acceleration structure (Sec. 1, Sec. 2.3) without detailing
// it; this layout keeps the BVH2's boxes and leaves exactly (every child box is a BVH2 node
// box, every leaf a BVH2 leaf over the same triangle records), so a traversal that is
// conservative against these boxes finds the BVH2 traversal's closest hits, while a ray
// visits about half as many nodes.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "cr_internal.h"

namespace cr {
namespace {

struct Kid {
    float lo[3], hi[3];
    int32_t link; // BVH2 link: >= 0 inner node, < 0 leaf code
};

Kid kid_of(const HostBVH2& b, uint32_t node, int which) {
    const float* o = &b.nodes[16 * (size_t)node];
    Kid c;
    if (which == 0) {
        c.lo[0] = o[0]; c.hi[0] = o[1]; c.lo[1] = o[2]; c.hi[1] = o[3]; c.lo[2] = o[8]; c.hi[2] = o[9];
        std::memcpy(&c.link, &o[12], 4);
    } else {
        c.lo[0] = o[4]; c.hi[0] = o[5]; c.lo[1] = o[6]; c.hi[1] = o[7]; c.lo[2] = o[10]; c.hi[2] = o[11];
        std::memcpy(&c.link, &o[13], 4);
    }
    return c;
}

double area(const Kid& c) {
    const double dx = (double)c.hi[0] - c.lo[0], dy = (double)c.hi[1] - c.lo[1], dz = (double)c.hi[2] - c.lo[2];
    return 2.0 * (dx * dy + dy * dz + dz * dx);
}

struct B4 {
    const HostBVH2& b2;
    std::vector<float> nodes;
    uint32_t depth = 0;
    explicit B4(const HostBVH2& b) : b2(b) {}

    // The 4-wide node for BVH2 inner node `n2`: its two children, then the inner child of
    // largest surface area opened into its own two, until there are four (or only leaves).
    uint32_t build(uint32_t n2, uint32_t level) {
        depth = std::max(depth, level + 1);
        std::vector<Kid> kids = {kid_of(b2, n2, 0), kid_of(b2, n2, 1)};
        while (kids.size() < 4) {
            int best = -1;
            double ba = -1.0;
            for (size_t i = 0; i < kids.size(); ++i)
                if (kids[i].link >= 0 && area(kids[i]) > ba) {
                    ba = area(kids[i]);
                    best = (int)i;
                }
            if (best < 0) break;
            const uint32_t open = (uint32_t)kids[best].link;
            kids[best] = kid_of(b2, open, 0);
            kids.insert(kids.begin() + best + 1, kid_of(b2, open, 1));
        }
        const uint32_t idx = (uint32_t)(nodes.size() / kBvh4NodeFloats);
        nodes.resize(nodes.size() + kBvh4NodeFloats, 0.0f);
        int32_t code[4] = {kBvh4Empty, kBvh4Empty, kBvh4Empty, kBvh4Empty};
        for (size_t k = 0; k < kids.size(); ++k)
            code[k] = kids[k].link < 0 ? kids[k].link : (int32_t)build((uint32_t)kids[k].link, level + 1);
        float* o = &nodes[(size_t)idx * kBvh4NodeFloats]; // after the recursion: nodes may have moved
        for (size_t k = kids.size(); k < 4; ++k) // unused slots: NaN planes, which no slab test enters
            for (int a = 0; a < 3; ++a) {
                o[8 * a + k] = NAN;
                o[8 * a + 4 + k] = NAN;
            }
        for (size_t k = 0; k < kids.size(); ++k)
            for (int a = 0; a < 3; ++a) {
                o[8 * a + k] = kids[k].lo[a];
                o[8 * a + 4 + k] = kids[k].hi[a];
            }
        std::memcpy(&o[24], code, sizeof(code));
        return idx;
    }
};

bool inside(const float* lo, const float* hi, const float* tri) {
    for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k)
            if (!(tri[3 * j + k] >= lo[k] && tri[3 * j + k] <= hi[k])) return false;
    return true;
}

} // namespace

// Walk every root-to-leaf path of the BVH4: each triangle must be reached (covered counts
// the triangles reached at least once) and every box on its path must contain its three
// vertices (violations counts the (triangle, box) pairs that do not); an unused slot must
// carry kBvh4Empty and NaN planes, a used one finite planes (also counted as violations).
void check_bvh4(const HostBVH4& b4, const HostBVH2& b2, const float* v, uint32_t n_tri, uint32_t& covered,
                uint32_t& violations) {
    std::vector<uint32_t> seen(n_tri, 0);
    violations = 0;
    std::vector<std::pair<uint32_t, std::vector<float>>> st;
    if (b4.n_nodes) st.push_back({0u, {}});
    while (!st.empty()) {
        auto it = std::move(st.back());
        st.pop_back();
        const float* o = &b4.nodes[(size_t)it.first * kBvh4NodeFloats];
        int32_t link[4];
        std::memcpy(link, &o[24], sizeof(link));
        for (int k = 0; k < 4; ++k) {
            float lo[3], hi[3];
            for (int a = 0; a < 3; ++a) {
                lo[a] = o[8 * a + k];
                hi[a] = o[8 * a + 4 + k];
            }
            const bool planes_nan = std::isnan(lo[0]) && std::isnan(lo[1]) && std::isnan(lo[2]) && std::isnan(hi[0]) &&
                                    std::isnan(hi[1]) && std::isnan(hi[2]);
            if (link[k] == kBvh4Empty) {
                if (!planes_nan) ++violations;
                continue;
            }
            if (!(std::isfinite(lo[0]) && std::isfinite(lo[1]) && std::isfinite(lo[2]) && std::isfinite(hi[0]) &&
                  std::isfinite(hi[1]) && std::isfinite(hi[2]))) {
                ++violations;
                continue;
            }
            std::vector<float> p = it.second;
            p.insert(p.end(), lo, lo + 3);
            p.insert(p.end(), hi, hi + 3);
            if (link[k] >= 0) {
                if ((uint32_t)link[k] >= b4.n_nodes) {
                    ++violations;
                    continue;
                }
                st.push_back({(uint32_t)link[k], std::move(p)});
            } else {
                const uint32_t code = (uint32_t)(~link[k]);
                const uint32_t first = code >> 2, count = (code & 3u) + 1u;
                for (uint32_t i = first; i < first + count && i < b2.leaf_order.size(); ++i) {
                    const uint32_t t = b2.leaf_order[i];
                    seen[t]++;
                    for (size_t q = 0; q < p.size(); q += 6)
                        if (!inside(&p[q], &p[q + 3], &v[9 * (size_t)t])) ++violations;
                }
            }
        }
    }
    covered = 0;
    for (uint32_t t = 0; t < n_tri; ++t) covered += seen[t] >= 1 ? 1u : 0u;
}

HostBVH4 build_bvh4(const HostBVH2& b2) {
    B4 b(b2);
    if (b2.n_nodes > 0) b.build(0, 0);
    HostBVH4 out;
    out.nodes = std::move(b.nodes);
    out.n_nodes = (uint32_t)(out.nodes.size() / kBvh4NodeFloats);
    out.depth = b.depth;
    out.stack_bound = 3 * b.depth; // a visit pushes at most three children
    return out;
}

} // namespace cr
