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

} // namespace

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
