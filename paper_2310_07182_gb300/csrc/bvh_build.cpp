// bvh_build.cpp -- host binned-SAH BVH2 builder (the paper names a BVH as its acceleration
// structure, Sec. 1 and Sec. 2.3, without detailing it).
//
// Top-down build over triangle centroids: the split minimising A_L N_L + A_R N_R is taken,
// from an exact sweep over the centroids sorted along each axis for nodes of <= 1024
// triangles and from 32 bins per axis above.  A node of <= 4 triangles becomes a leaf when
// testing its triangles costs no more than the best split (surface area heuristic with an
// inner-node visit at 1.2 triangle tests: on the GB300 trace kernel this gives ~2% more
// rays/s than leaves of up to 4 triangles everywhere, and lower costs 0.6-1.6 do no better).
// Below depth 40, when depth + log2(n) reaches 60, or when all centroids coincide, the node
// is split at the median along its widest centroid axis, so the depth stays below 62.
// The top levels run on several threads (independent subtrees).
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstring>
#include <functional>
#include <mutex>
#include <thread>

#include "cr_internal.h"

namespace cr {
namespace {

struct Box {
    float lo[3], hi[3];
    void reset() {
        for (int k = 0; k < 3; ++k) {
            lo[k] = INFINITY;
            hi[k] = -INFINITY;
        }
    }
    void grow(const Box& b) {
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], b.lo[k]);
            hi[k] = std::max(hi[k], b.hi[k]);
        }
    }
    double area() const {
        double dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
        if (dx < 0 || dy < 0 || dz < 0) return 0.0;
        return 2.0 * (dx * dy + dy * dz + dz * dx);
    }
};

struct TNode { // temporary tree node
    Box box;
    int32_t left = -1, right = -1;
    uint32_t first = 0, count = 0; // leaf range
};

constexpr int kBins = 32;
constexpr uint32_t kLeafMax = 4;
constexpr uint32_t kSweepMax = 1024; // exact SAH sweep over sorted centroids at or below this size
constexpr double kCt = 1.2;          // cost of an inner-node visit (two box tests) per triangle test
constexpr uint32_t kSahDepth = 40;

struct Builder {
    const float* v;
    std::vector<Box> pbox;
    std::vector<float> cen; // 3 per prim
    std::vector<uint32_t> idx;
    std::vector<TNode> nodes;
    std::mutex mu;
    std::atomic<uint32_t> max_depth{0};

    int32_t alloc_node() {
        std::lock_guard<std::mutex> g(mu);
        nodes.emplace_back();
        return (int32_t)nodes.size() - 1;
    }

    // Returns the split position in idx[begin, end).
    uint32_t split(uint32_t begin, uint32_t end, uint32_t depth, double* out_cost) {
        *out_cost = INFINITY;
        float clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (uint32_t i = begin; i < end; ++i) {
            const float* c = &cen[3 * idx[i]];
            for (int k = 0; k < 3; ++k) {
                clo[k] = std::min(clo[k], c[k]);
                chi[k] = std::max(chi[k], c[k]);
            }
        }
        int wide = 0;
        for (int k = 1; k < 3; ++k)
            if (chi[k] - clo[k] > chi[wide] - clo[wide]) wide = k;
        const uint32_t n = end - begin;
        auto median = [&](int axis) {
            uint32_t mid = begin + n / 2;
            std::nth_element(idx.begin() + begin, idx.begin() + mid, idx.begin() + end, [&](uint32_t a, uint32_t b) {
                float ca = cen[3 * a + axis], cb = cen[3 * b + axis];
                return ca < cb || (ca == cb && a < b);
            });
            return mid;
        };
        uint32_t log2n = 0;
        while ((1u << log2n) < n) ++log2n;
        // median splits from here on keep the total depth below 62
        if (depth >= kSahDepth || depth + log2n >= 60 || !(chi[wide] > clo[wide])) return median(wide);

        double best_cost = INFINITY;
        int best_axis = -1, best_bin = -1;
        if (n <= kSweepMax) {
            std::vector<uint32_t> ord[3];
            std::vector<double> right(n);
            uint32_t best_pos = 0;
            for (int axis = 0; axis < 3; ++axis) {
                ord[axis].assign(idx.begin() + begin, idx.begin() + end);
                std::sort(ord[axis].begin(), ord[axis].end(), [&](uint32_t a, uint32_t b) {
                    float ca = cen[3 * a + axis], cb = cen[3 * b + axis];
                    return ca < cb || (ca == cb && a < b);
                });
                Box acc;
                acc.reset();
                for (uint32_t i = n - 1; i > 0; --i) {
                    acc.grow(pbox[ord[axis][i]]);
                    right[i] = acc.area();
                }
                acc.reset();
                for (uint32_t i = 0; i + 1 < n; ++i) {
                    acc.grow(pbox[ord[axis][i]]);
                    const double cost = acc.area() * (i + 1) + right[i + 1] * (n - i - 1);
                    if (cost < best_cost) {
                        best_cost = cost;
                        best_axis = axis;
                        best_pos = i + 1;
                    }
                }
            }
            std::copy(ord[best_axis].begin(), ord[best_axis].end(), idx.begin() + begin);
            *out_cost = best_cost;
            return begin + best_pos;
        }
        for (int axis = 0; axis < 3; ++axis) {
            float ext = chi[axis] - clo[axis];
            if (!(ext > 0.0f)) continue;
            float scale = (float)kBins / ext * (1.0f - 1e-6f);
            Box bb[kBins];
            uint32_t cnt[kBins] = {0};
            for (int b = 0; b < kBins; ++b) bb[b].reset();
            for (uint32_t i = begin; i < end; ++i) {
                uint32_t p = idx[i];
                int b = std::min(kBins - 1, std::max(0, (int)((cen[3 * p + axis] - clo[axis]) * scale)));
                cnt[b]++;
                bb[b].grow(pbox[p]);
            }
            double right_area[kBins];
            uint32_t right_cnt[kBins];
            Box acc;
            acc.reset();
            uint32_t c = 0;
            for (int b = kBins - 1; b > 0; --b) {
                acc.grow(bb[b]);
                c += cnt[b];
                right_area[b] = acc.area();
                right_cnt[b] = c;
            }
            acc.reset();
            c = 0;
            for (int b = 0; b < kBins - 1; ++b) {
                acc.grow(bb[b]);
                c += cnt[b];
                if (c == 0 || right_cnt[b + 1] == 0) continue;
                double cost = acc.area() * c + right_area[b + 1] * right_cnt[b + 1];
                if (cost < best_cost) {
                    best_cost = cost;
                    best_axis = axis;
                    best_bin = b;
                }
            }
        }
        if (best_axis < 0) return median(wide);
        *out_cost = best_cost;
        const int axis = best_axis;
        const float scale = (float)kBins / (chi[axis] - clo[axis]) * (1.0f - 1e-6f);
        auto mid_it = std::stable_partition(idx.begin() + begin, idx.begin() + end, [&](uint32_t p) {
            int b = std::min(kBins - 1, std::max(0, (int)((cen[3 * p + axis] - clo[axis]) * scale)));
            return b <= best_bin;
        });
        uint32_t mid = (uint32_t)(mid_it - idx.begin());
        if (mid == begin || mid == end) return median(wide);
        return mid;
    }

    void build(int32_t node, uint32_t begin, uint32_t end, uint32_t depth, int spawn_levels) {
        Box b;
        b.reset();
        for (uint32_t i = begin; i < end; ++i) b.grow(pbox[idx[i]]);
        {
            std::lock_guard<std::mutex> g(mu);
            nodes[node].box = b;
        }
        const uint32_t n = end - begin;
        bool leaf = n <= kLeafMax;
        uint32_t mid = 0;
        if (n > 1) {
            double split_cost;
            mid = split(begin, end, depth, &split_cost);
            if (leaf) leaf = n * b.area() <= kCt * b.area() + split_cost;
        }
        if (leaf) {
            std::lock_guard<std::mutex> g(mu);
            nodes[node].first = begin;
            nodes[node].count = end - begin;
            uint32_t d = max_depth.load();
            while (depth > d && !max_depth.compare_exchange_weak(d, depth)) {
            }
            return;
        }
        int32_t l = alloc_node(), r = alloc_node();
        {
            std::lock_guard<std::mutex> g(mu);
            nodes[node].left = l;
            nodes[node].right = r;
        }
        if (spawn_levels > 0) {
            std::thread th([&, l, begin, mid, depth, spawn_levels] { build(l, begin, mid, depth + 1, spawn_levels - 1); });
            build(r, mid, end, depth + 1, spawn_levels - 1);
            th.join();
        } else {
            build(l, begin, mid, depth + 1, 0);
            build(r, mid, end, depth + 1, 0);
        }
    }
};

} // namespace

HostBVH2 build_bvh2(const float* v, uint32_t n_tri, int n_threads) {
    Builder B;
    B.v = v;
    B.pbox.resize(n_tri);
    B.cen.resize(3 * (size_t)n_tri);
    B.idx.resize(n_tri);
    for (uint32_t t = 0; t < n_tri; ++t) {
        Box& b = B.pbox[t];
        b.reset();
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) {
                float x = v[9 * (size_t)t + 3 * j + k];
                b.lo[k] = std::min(b.lo[k], x);
                b.hi[k] = std::max(b.hi[k], x);
            }
        for (int k = 0; k < 3; ++k) B.cen[3 * (size_t)t + k] = 0.5f * (b.lo[k] + b.hi[k]);
        B.idx[t] = t;
    }
    B.nodes.reserve(2 * (size_t)n_tri + 2);
    int32_t root = B.alloc_node();
    int levels = 0;
    while ((1 << levels) < n_threads && levels < 6) ++levels;
    B.build(root, 0, n_tri, 0, n_tri > 65536 ? levels : 0);

    HostBVH2 out;
    const Box& rb = B.nodes[root].box;
    for (int k = 0; k < 3; ++k) {
        out.lo[k] = rb.lo[k];
        out.hi[k] = rb.hi[k];
    }
    out.leaf_order = B.idx;
    out.depth = B.max_depth.load();

    // Flatten: inner nodes in depth-first order; the root is always an inner node (a leaf
    // root is split into two leaves over the same triangles, which is harmless).
    auto link_of = [&](int32_t tn, std::vector<int32_t>& stack_children, uint32_t& next) -> int32_t {
        const TNode& t = B.nodes[tn];
        if (t.count > 0) return ~(int32_t)((t.first << 2) | (t.count - 1));
        stack_children.push_back(tn);
        return (int32_t)(next++);
    };
    std::vector<float>& nd = out.nodes;
    std::vector<int32_t> order; // temporary-node index of each emitted inner node
    int32_t c0 = B.nodes[root].left, c1 = B.nodes[root].right;
    if (B.nodes[root].count > 0) {
        // root leaf: emit two leaf children splitting the range
        const TNode& t = B.nodes[root];
        TNode a = t, b = t;
        a.count = std::max<uint32_t>(1, t.count / 2);
        b.first = t.first + (t.count > 1 ? a.count : 0);
        b.count = t.count > 1 ? t.count - a.count : 1;
        B.nodes.push_back(a);
        B.nodes.push_back(b);
        c0 = (int32_t)B.nodes.size() - 2;
        c1 = (int32_t)B.nodes.size() - 1;
        // box of each half
        for (int32_t ci : {c0, c1}) {
            TNode& tn = B.nodes[ci];
            tn.box.reset();
            for (uint32_t i = tn.first; i < tn.first + tn.count; ++i) tn.box.grow(B.pbox[B.idx[i]]);
        }
    }
    // iterative emission: each emitted node needs slot index before its children are emitted
    struct Item {
        int32_t c0, c1;
        uint32_t slot;
    };
    std::vector<Item> work;
    uint32_t next = 1;
    work.push_back({c0, c1, 0});
    nd.resize(16);
    while (!work.empty()) {
        Item it = work.back();
        work.pop_back();
        std::vector<int32_t> kids;
        int32_t l0 = link_of(it.c0, kids, next);
        int32_t l1 = link_of(it.c1, kids, next);
        if (nd.size() < 16 * (size_t)next) nd.resize(16 * (size_t)next);
        const Box& b0 = B.nodes[it.c0].box;
        const Box& b1 = B.nodes[it.c1].box;
        float* o = &nd[16 * (size_t)it.slot];
        o[0] = b0.lo[0]; o[1] = b0.hi[0]; o[2] = b0.lo[1]; o[3] = b0.hi[1];
        o[4] = b1.lo[0]; o[5] = b1.hi[0]; o[6] = b1.lo[1]; o[7] = b1.hi[1];
        o[8] = b0.lo[2]; o[9] = b0.hi[2]; o[10] = b1.lo[2]; o[11] = b1.hi[2];
        std::memcpy(&o[12], &l0, 4);
        std::memcpy(&o[13], &l1, 4);
        o[14] = 0.0f;
        o[15] = 0.0f;
        // siblings get adjacent slots; the left subtree is emitted first
        uint32_t slot_l = l0 >= 0 ? (uint32_t)l0 : 0, slot_r = l1 >= 0 ? (uint32_t)l1 : 0;
        if (l1 >= 0) work.push_back({B.nodes[it.c1].left, B.nodes[it.c1].right, slot_r});
        if (l0 >= 0) work.push_back({B.nodes[it.c0].left, B.nodes[it.c0].right, slot_l});
    }
    out.n_nodes = next;
    nd.resize(16 * (size_t)next);
    return out;
}

} // namespace cr

// ------------------------------------------------------------------------------------
// Host verification of the BVH2 (used by cr_debug_bvh_check).
namespace cr {
namespace {

struct Child2 {
    float lo[3], hi[3];
    int32_t link; // >= 0 inner node, < 0 leaf code
};

Child2 child2_of(const HostBVH2& b, uint32_t node, int which) {
    const float* o = &b.nodes[16 * (size_t)node];
    Child2 c;
    const int x = which == 0 ? 0 : 4, z = which == 0 ? 8 : 10;
    c.lo[0] = o[x]; c.hi[0] = o[x + 1]; c.lo[1] = o[x + 2]; c.hi[1] = o[x + 3]; c.lo[2] = o[z]; c.hi[2] = o[z + 1];
    std::memcpy(&c.link, &o[12 + which], 4);
    return c;
}

bool contains(const float* lo, const float* hi, const float* v) {
    for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k)
            if (v[3 * j + k] < lo[k] || v[3 * j + k] > hi[k]) return false;
    return true;
}

} // namespace

void check_bvh2(const HostBVH2& b, const float* v, uint32_t n_tri, uint32_t& covered, uint32_t& violations) {
    std::vector<uint32_t> seen(n_tri, 0);
    violations = 0;
    // iterative DFS carrying the boxes on the path
    std::vector<std::pair<int32_t, std::vector<float>>> st; // link, path boxes (6 floats each)
    st.push_back({0, {}});
    while (!st.empty()) {
        auto it = std::move(st.back());
        st.pop_back();
        const int32_t link = it.first;
        if (link >= 0) {
            for (int w = 0; w < 2; ++w) {
                const Child2 c = child2_of(b, (uint32_t)link, w);
                std::vector<float> p = it.second;
                p.insert(p.end(), {c.lo[0], c.lo[1], c.lo[2], c.hi[0], c.hi[1], c.hi[2]});
                st.push_back({c.link, std::move(p)});
            }
        } else {
            const uint32_t code = (uint32_t)(~link);
            const uint32_t first = code >> 2, count = (code & 3u) + 1u;
            for (uint32_t i = first; i < first + count; ++i) {
                const uint32_t t = b.leaf_order[i];
                seen[t]++;
                for (size_t q = 0; q < it.second.size(); q += 6)
                    if (!contains(&it.second[q], &it.second[q + 3], &v[9 * (size_t)t])) ++violations;
            }
        }
    }
    covered = 0;
    for (uint32_t t = 0; t < n_tri; ++t) covered += seen[t] >= 1 ? 1u : 0u;
    // the root-leaf case emits the same triangles twice on purpose; count distinct coverage
}

} // namespace cr
