// bvh8_build.cpp -- BVH8-Q: the BVH2 collapsed into 8-wide nodes whose child boxes are
// quantised to 8 bits per plane (after Ylitie, Karras and Laine 2017), and its host check.
// The paper names a BVH as its acceleration structure (Sec. 1, Sec. 2.3) without detailing
// it; this wide layout is the alternative to the BVH2 traversal.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "cr_internal.h"

// ------------------------------------------------------------------------------------
// BVH8-Q: collapse the BVH2 into 8-wide nodes and quantise the child boxes.
namespace cr {
namespace {

struct Child {
    float lo[3], hi[3];
    int32_t link;             // BVH2 link: >= 0 inner node, < 0 leaf
    uint32_t first, count;    // leaf: BVH2 leaf-order range of its triangles
};

Child child_of(const HostBVH2& b, uint32_t node, int which) {
    const float* o = &b.nodes[16 * (size_t)node];
    Child c;
    if (which == 0) {
        c.lo[0] = o[0]; c.hi[0] = o[1]; c.lo[1] = o[2]; c.hi[1] = o[3]; c.lo[2] = o[8]; c.hi[2] = o[9];
        std::memcpy(&c.link, &o[12], 4);
    } else {
        c.lo[0] = o[4]; c.hi[0] = o[5]; c.lo[1] = o[6]; c.hi[1] = o[7]; c.lo[2] = o[10]; c.hi[2] = o[11];
        std::memcpy(&c.link, &o[13], 4);
    }
    const uint32_t code = (uint32_t)(~c.link);
    c.first = c.link < 0 ? code >> 2 : 0;
    c.count = c.link < 0 ? (code & 3u) + 1u : 0;
    return c;
}

double child_area(const Child& c) {
    double dx = c.hi[0] - c.lo[0], dy = c.hi[1] - c.lo[1], dz = c.hi[2] - c.lo[2];
    return 2.0 * (dx * dy + dy * dz + dz * dx);
}

// The quantised box a code stands for: origin + q * step in float (q * step is exact, the sum
// rounds once).  The quantiser chooses codes so that this box contains the child.  The
// traversal kernel does not decode planes: it tests fma(q, step / d, (origin - o) / d) with an
// error bias (trace_bvh8.cu) that makes its slab test conservative against this box.
float decode(float origin, uint32_t q, float step) {
    volatile float prod = (float)q * step; // exact: 8-bit integer times a power of two
    volatile float sum = origin + prod;
    return sum;
}

#ifndef CR_BVH8_SPLIT_LEAVES
#define CR_BVH8_SPLIT_LEAVES 1
#endif
// Fill a node's free child slots by splitting its multi-triangle leaves (0: leaves stay as
// the BVH2 made them, the layout before this option existed).
constexpr bool kSplitLeaves = CR_BVH8_SPLIT_LEAVES != 0;

struct B8 {
    const HostBVH2& b2;
    std::vector<uint32_t> nodes;
    std::vector<uint32_t> tri_order;
    uint32_t max_depth = 0, stack_bound = 0;
    const float* v; // triangle vertices, 9 floats per original triangle
    B8(const HostBVH2& b, const float* tri_xyz) : b2(b), v(tri_xyz) {}

    // exact box of the triangles at BVH2 leaf-order positions [first, first + count)
    Child leaf_box(uint32_t first, uint32_t count) const {
        Child c;
        for (int k = 0; k < 3; ++k) {
            c.lo[k] = INFINITY;
            c.hi[k] = -INFINITY;
        }
        for (uint32_t i = first; i < first + count; ++i) {
            const float* t = &v[9 * (size_t)b2.leaf_order[i]];
            for (int j = 0; j < 3; ++j)
                for (int k = 0; k < 3; ++k) {
                    c.lo[k] = std::min(c.lo[k], t[3 * j + k]);
                    c.hi[k] = std::max(c.hi[k], t[3 * j + k]);
                }
        }
        c.link = -1;
        c.first = first;
        c.count = count;
        return c;
    }

    // Children of the BVH8 node made from BVH2 inner node n: expand the inner child of
    // largest surface area until there are 8 children or none left to expand, then fill
    // the free slots by splitting leaves.
    std::vector<Child> gather(uint32_t n) {
        std::vector<Child> ch = {child_of(b2, n, 0), child_of(b2, n, 1)};
        while (ch.size() < 8) {
            int best = -1;
            double ba = -1.0;
            for (size_t i = 0; i < ch.size(); ++i)
                if (ch[i].link >= 0 && child_area(ch[i]) > ba) {
                    ba = child_area(ch[i]);
                    best = (int)i;
                }
            if (best < 0) break;
            const uint32_t m = (uint32_t)ch[best].link;
            ch[best] = child_of(b2, m, 0);
            ch.push_back(child_of(b2, m, 1));
        }
        // Slots still free: split the leaf of largest area that holds several triangles,
        // one triangle off at a time.  All 8 slots of a node are tested together, so a free
        // slot costs nothing, and a ray that misses a single triangle's box skips its test.
        while (kSplitLeaves && ch.size() < 8) {
            int best = -1;
            double ba = -1.0;
            for (size_t i = 0; i < ch.size(); ++i)
                if (ch[i].link < 0 && ch[i].count > 1 && child_area(ch[i]) > ba) {
                    ba = child_area(ch[i]);
                    best = (int)i;
                }
            if (best < 0) break;
            const uint32_t first = ch[best].first, count = ch[best].count;
            ch[best] = leaf_box(first, 1);
            ch.push_back(leaf_box(first + 1, count - 1));
        }
        return ch;
    }

    // Emit the node at index `self` (already reserved) for BVH2 node n.
    void emit(uint32_t self, uint32_t n, uint32_t depth) {
        max_depth = std::max(max_depth, depth);
        std::vector<Child> ch = gather(n);
        // node box and octant slot assignment by the child centroids
        float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (auto& c : ch)
            for (int k = 0; k < 3; ++k) {
                lo[k] = std::min(lo[k], c.lo[k]);
                hi[k] = std::max(hi[k], c.hi[k]);
            }
        double mid[3];
        for (int k = 0; k < 3; ++k) mid[k] = 0.5 * ((double)lo[k] + (double)hi[k]);
        int slot_of[8];
        bool used[8] = {false, false, false, false, false, false, false, false};
        // greedy: repeatedly take the (child, slot) pair whose centroid lies farthest toward
        // the slot's corner (slot bit k set = high side of axis k)
        std::vector<bool> done(ch.size(), false);
        for (size_t it = 0; it < ch.size(); ++it) {
            double best = -INFINITY;
            int bc = -1, bs = -1;
            for (size_t c = 0; c < ch.size(); ++c) {
                if (done[c]) continue;
                double cc[3];
                for (int k = 0; k < 3; ++k) cc[k] = 0.5 * ((double)ch[c].lo[k] + (double)ch[c].hi[k]) - mid[k];
                for (int sl = 0; sl < 8; ++sl) {
                    if (used[sl]) continue;
                    double sc = 0.0;
                    for (int k = 0; k < 3; ++k) sc += ((sl >> k) & 1 ? 1.0 : -1.0) * cc[k];
                    if (sc > best) {
                        best = sc;
                        bc = (int)c;
                        bs = sl;
                    }
                }
            }
            done[bc] = true;
            used[bs] = true;
            slot_of[bc] = bs;
        }
        // quantisation grid per axis
        uint32_t ebias[3];
        float step[3];
        for (int k = 0; k < 3; ++k) {
            const double ext = (double)hi[k] - (double)lo[k];
            int e = -126;
            while (e < 127 && std::ldexp(255.0, e) < ext) ++e;
            while (e < 127 && decode(lo[k], 255, std::ldexp(1.0f, e)) < hi[k]) ++e;
            ebias[k] = (uint32_t)(e + 127);
            step[k] = std::ldexp(1.0f, e);
        }
        uint32_t* w = &nodes[20 * (size_t)self];
        std::memset(w, 0, 80);
        std::memcpy(&w[0], &lo[0], 4);
        std::memcpy(&w[1], &lo[1], 4);
        std::memcpy(&w[2], &lo[2], 4);
        uint8_t* meta = reinterpret_cast<uint8_t*>(&w[6]);
        uint8_t* q = reinterpret_cast<uint8_t*>(&w[8]); // qlo_x, qlo_y, qlo_z, qhi_x, qhi_y, qhi_z
        uint32_t imask = 0;
        // inner children are numbered in slot order; leaf triangles are laid out in slot order
        std::vector<std::pair<int, uint32_t>> inner; // (slot, BVH2 node)
        const uint32_t tri_base = (uint32_t)tri_order.size();
        for (int sl = 0; sl < 8; ++sl) {
            int c = -1;
            for (size_t i = 0; i < ch.size(); ++i)
                if (slot_of[i] == sl) c = (int)i;
            if (c < 0) continue;
            const Child& C = ch[c];
            for (int k = 0; k < 3; ++k) {
                double fl = std::floor(((double)C.lo[k] - (double)lo[k]) / (double)step[k]);
                uint32_t ql = (uint32_t)std::min(255.0, std::max(0.0, fl));
                while (ql > 0 && decode(lo[k], ql, step[k]) > C.lo[k]) --ql;
                double ce = std::ceil(((double)C.hi[k] - (double)lo[k]) / (double)step[k]);
                uint32_t qh = (uint32_t)std::min(255.0, std::max(0.0, ce));
                while (qh < 255 && decode(lo[k], qh, step[k]) < C.hi[k]) ++qh;
                q[8 * k + sl] = (uint8_t)ql;
                q[24 + 8 * k + sl] = (uint8_t)qh;
            }
            if (C.link >= 0) {
                meta[sl] = (uint8_t)inner.size();
                imask |= 1u << sl;
                inner.emplace_back(sl, (uint32_t)C.link);
            } else {
                const uint32_t off = (uint32_t)tri_order.size() - tri_base;
                for (uint32_t i = 0; i < C.count; ++i) tri_order.push_back(C.first + i); // BVH2 leaf positions
                meta[sl] = (uint8_t)((C.count << 5) | off);
            }
        }
        w[3] = ebias[0] | (ebias[1] << 8) | (ebias[2] << 16) | (imask << 24);
        w[5] = tri_base;
        const uint32_t child_base = (uint32_t)(nodes.size() / 20);
        w[4] = child_base;
        nodes.resize(nodes.size() + 20 * inner.size());
        // the traversal keeps at most one (first child, hit mask) entry per tree level
        stack_bound = std::max(stack_bound, depth);
        for (size_t i = 0; i < inner.size(); ++i) emit(child_base + (uint32_t)i, inner[i].second, depth + 1);
    }
};

} // namespace

HostBVH8 build_bvh8q(const HostBVH2& b2, const float* tri_xyz) {
    B8 b(b2, tri_xyz);
    b.nodes.resize(20);
    b.emit(0, 0, 1);
    HostBVH8 out;
    out.n_nodes = (uint32_t)(b.nodes.size() / 20);
    out.nodes.swap(b.nodes);
    // BVH8 triangle positions refer to BVH2 leaf-order positions; map to original indices
    out.leaf_order.resize(b.tri_order.size());
    for (size_t i = 0; i < b.tri_order.size(); ++i) out.leaf_order[i] = b2.leaf_order[b.tri_order[i]];
    out.depth = b.max_depth;
    out.stack_bound = b.stack_bound;
    return out;
}

} // namespace cr

// ------------------------------------------------------------------------------------
// Host verification of the BVH8-Q (used by cr_debug_bvh_check).
namespace cr {
namespace {

bool contains(const float* lo, const float* hi, const float* v) {
    for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k)
            if (v[3 * j + k] < lo[k] || v[3 * j + k] > hi[k]) return false;
    return true;
}

} // namespace

void check_bvh8(const HostBVH8& b, const float* v, uint32_t n_tri, uint32_t& covered, uint32_t& violations) {
    std::vector<uint32_t> seen(n_tri, 0);
    violations = 0;
    std::vector<std::pair<uint32_t, std::vector<float>>> st;
    st.push_back({0u, {}});
    while (!st.empty()) {
        auto it = std::move(st.back());
        st.pop_back();
        const uint32_t* w = &b.nodes[20 * (size_t)it.first];
        float org[3], step[3];
        std::memcpy(org, w, 12);
        for (int k = 0; k < 3; ++k) {
            const uint32_t bits = ((w[3] >> (8 * k)) & 0xffu) << 23;
            std::memcpy(&step[k], &bits, 4);
        }
        const uint32_t imask = w[3] >> 24;
        const uint8_t* meta = reinterpret_cast<const uint8_t*>(&w[6]);
        const uint8_t* q = reinterpret_cast<const uint8_t*>(&w[8]);
        for (int sl = 0; sl < 8; ++sl) {
            const bool inner = (imask >> sl) & 1u;
            if (!inner && meta[sl] < 32) continue;
            std::vector<float> p = it.second;
            for (int k = 0; k < 3; ++k) p.push_back(decode(org[k], q[8 * k + sl], step[k]));
            for (int k = 0; k < 3; ++k) p.push_back(decode(org[k], q[24 + 8 * k + sl], step[k]));
            if (inner) {
                st.push_back({w[4] + meta[sl], std::move(p)});
            } else {
                const uint32_t first = w[5] + (meta[sl] & 31u), count = meta[sl] >> 5;
                for (uint32_t i = first; i < first + count; ++i) {
                    const uint32_t t = b.leaf_order[i];
                    seen[t]++;
                    for (size_t qq = 0; qq < p.size(); qq += 6)
                        if (!contains(&p[qq], &p[qq + 3], &v[9 * (size_t)t])) ++violations;
                }
            }
        }
    }
    covered = 0;
    for (uint32_t t = 0; t < n_tri; ++t) covered += seen[t] >= 1 ? 1u : 0u;
}

} // namespace cr
