// Drives the host BVH builders (BVH2 and the BVH8-Q collapse) under AddressSanitizer and
// UndefinedBehaviorSanitizer on a random soup, a heightfield patch and degenerate inputs
// (one triangle, identical triangles, zero-area triangles, coincident centroids), and checks
// with the library's own host verification that every triangle is covered by the boxes on
// its path and that the leaf orders are permutations.  Exits 0 when all hold.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "cr_internal.h"

static uint32_t rng = 777u;
static float urand() {
    rng = rng * 1664525u + 1013904223u;
    return (float)(rng >> 8) * (1.0f / 16777216.0f);
}

static int check(const std::vector<float>& v, const char* what) {
    const uint32_t n = (uint32_t)(v.size() / 9);
    cr::HostBVH2 b2 = cr::build_bvh2(v.data(), n, 4);
    uint32_t cov = 0, bad = 0;
    cr::check_bvh2(b2, v.data(), n, cov, bad);
    if (bad || cov != n) {
        std::printf("%s: BVH2 covered %u of %u, %u violations\n", what, cov, n, bad);
        return 1;
    }
    std::vector<char> seen(n, 0);
    for (uint32_t t : b2.leaf_order) {
        if (t >= n || seen[t]) return 1;
        seen[t] = 1;
    }
    if (b2.depth >= cr::kBvh2StackCapacity) return 1;
    cr::HostBVH8 b8 = cr::build_bvh8q(b2, v.data());
    cr::check_bvh8(b8, v.data(), n, cov, bad);
    if (bad || cov != n) {
        std::printf("%s: BVH8-Q covered %u of %u, %u violations\n", what, cov, n, bad);
        return 1;
    }
    return 0;
}

int main() {
    int fails = 0;
    std::vector<float> soup(9 * 5000);
    for (size_t i = 0; i < soup.size() / 9; ++i) {
        const float c[3] = {2 * urand() - 1, 2 * urand() - 1, 2 * urand() - 1};
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) soup[9 * i + 3 * j + k] = c[k] + 0.1f * urand() - 0.05f;
    }
    fails += check(soup, "soup");
    std::vector<float> grid;
    const int G = 40;
    auto h = [](int x, int z) { return 0.3f * (float)((x * 7 + z * 13) % 11); };
    for (int x = 0; x < G; ++x)
        for (int z = 0; z < G; ++z) {
            const float p[4][3] = {{(float)x, h(x, z), (float)z}, {(float)x + 1, h(x + 1, z), (float)z},
                                   {(float)x + 1, h(x + 1, z + 1), (float)z + 1}, {(float)x, h(x, z + 1), (float)z + 1}};
            const int tri[2][3] = {{0, 1, 2}, {0, 2, 3}};
            for (auto& t : tri)
                for (int j : t)
                    for (int k = 0; k < 3; ++k) grid.push_back(p[j][k]);
        }
    fails += check(grid, "heightfield");
    fails += check(std::vector<float>{0, 0, 0, 1, 0, 0, 0, 1, 0}, "one triangle");
    std::vector<float> same;
    for (int i = 0; i < 100; ++i)
        for (float x : {0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 1.f, 0.f}) same.push_back(x);
    fails += check(same, "identical triangles");
    std::vector<float> flat;
    for (int i = 0; i < 200; ++i)
        for (int j = 0; j < 9; ++j) flat.push_back(0.25f * (float)(i % 5)); // zero area, coincident
    fails += check(flat, "zero-area triangles");
    if (fails) return 1;
    std::printf("bvh sanitize run ok\n");
    return 0;
}
