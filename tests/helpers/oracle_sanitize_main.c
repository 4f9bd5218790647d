/* Drives the oracle under AddressSanitizer and UndefinedBehaviorSanitizer: a small scene
 * with every material type (Lambert, GGX, mirror, emitter, dielectric, translucent), every
 * mode with and without next-event estimation and with the per-bounce debug outputs, plus
 * closest-hit and shadow queries by BVH and by brute force, which must agree.  Exits 0
 * when everything ran and agreed; a sanitizer report aborts with a nonzero status. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

static uint32_t rng = 12345u;
static float urand(void) {
    rng = rng * 1664525u + 1013904223u;
    return (float)(rng >> 8) * (1.0f / 16777216.0f);
}

int main(void) {
    enum { N_SOUP = 300, N_TRI = N_SOUP + 4 };
    float* v = (float*)calloc(9 * N_TRI, sizeof(float));
    uint32_t* tm = (uint32_t*)calloc(N_TRI, sizeof(uint32_t));
    /* ground quad (2 triangles) and a ceiling emitter (2 triangles) */
    const float g[18] = {-5, -1, -5, 5, -1, -5, 5, -1, 5, -5, -1, -5, 5, -1, 5, -5, -1, 5};
    const float e[18] = {-1, 2, -1, -1, 2, 1, 1, 2, 1, -1, 2, -1, 1, 2, 1, 1, 2, -1};
    memcpy(v, g, sizeof g);
    memcpy(v + 18, e, sizeof e);
    tm[0] = tm[1] = 0;
    tm[2] = tm[3] = 3;
    for (int i = 4; i < N_TRI; ++i) {
        const float c[3] = {1.8f * urand() - 0.9f, 1.8f * urand() - 0.9f, 1.8f * urand() - 0.9f};
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) v[9 * i + 3 * j + k] = c[k] + 0.2f * urand() - 0.1f;
        tm[i] = (uint32_t)(i % 6);
    }
    const uint32_t mt[6] = {0, 1, 2, 3, 4, 5}; /* Lambert, GGX, mirror, emitter, dielectric, translucent */
    float mp[6 * 7];
    memset(mp, 0, sizeof mp);
    for (int m = 0; m < 6; ++m) {
        mp[7 * m + 0] = 0.6f;
        mp[7 * m + 1] = 0.5f;
        mp[7 * m + 2] = 0.4f;
        mp[7 * m + 3] = m == 1 ? 0.3f : (m == 4 ? 1.5f : 0.0f);
    }
    mp[7 * 3 + 4] = mp[7 * 3 + 5] = mp[7 * 3 + 6] = 4.0f;
    const float env[3] = {0.3f, 0.3f, 0.3f};
    orc_scene* s = orc_scene_new(v, N_TRI, tm, mt, mp, 6, env);
    if (!s) return 2;

    orc_camera cam = {{0.1f, 0.2f, -3.0f}, {0.0f, 0.0f, 0.0f}, {0.0f, 1.0f, 0.0f}, 50.0f, 20, 12};
    const uint32_t npx = cam.width * cam.height, B = 3;
    const uint32_t tiles = ((cam.width + 3) / 4) * ((cam.height + 3) / 4);
    double* accum = (double*)calloc(3 * npx, sizeof(double));
    uint8_t* taint = (uint8_t*)calloc(npx, 1);
    int32_t* dprim = (int32_t*)calloc((B + 1) * npx, sizeof(int32_t));
    uint8_t* dcat = (uint8_t*)calloc(B * npx, 1);
    uint8_t* dcls = (uint8_t*)calloc(B * npx, 1);
    uint8_t* dflags = (uint8_t*)calloc(B * npx, 1);
    float* dlocal = (float*)calloc(3 * B * npx, sizeof(float));
    float* dworld = (float*)calloc(3 * B * npx, sizeof(float));
    uint64_t counters[5];
    for (uint32_t mode = 0; mode < 4; ++mode)
        for (uint32_t opts = 0; opts < 8; ++opts) {
            if ((opts & ORC_OPT_NEE_SHARED) && !(opts & ORC_OPT_NEE)) continue;
            orc_params p = {1, B, mode, 4, 4, 8, 1, 0, 0, opts, 7};
            orc_outputs o = {accum, taint, dprim, dcat, dcls, dflags, dlocal, dworld, counters};
            memset(counters, 0, sizeof counters);
            orc_render_tiles(s, &cam, &p, 0, tiles, &o);
            for (uint32_t i = 0; i < 3 * npx; ++i)
                if (!isfinite(accum[i])) return 3;
        }

    /* closest hit and shadow rays: BVH against brute force */
    enum { NR = 500 };
    float rays[8 * NR];
    int32_t skip[NR], p0[NR], p1[NR];
    double t0[NR], t1[NR];
    uint8_t f0[NR], f1[NR], o0[NR], o1[NR];
    for (int i = 0; i < NR; ++i) {
        for (int k = 0; k < 3; ++k) rays[8 * i + k] = 3.0f * urand() - 1.5f;
        for (int k = 0; k < 3; ++k) rays[8 * i + 4 + k] = 2.0f * urand() - 1.0f;
        rays[8 * i + 3] = 0.0f;
        rays[8 * i + 7] = 0.5f + urand();
        skip[i] = i % 7 == 0 ? (int32_t)(i % N_TRI) : -1;
    }
    orc_trace(s, rays, skip, NR, 1, p0, t0, f0);
    orc_trace(s, rays, skip, NR, 0, p1, t1, f1);
    for (int i = 0; i < NR; ++i)
        if (!f0[i] && !f1[i] && p0[i] != p1[i]) return 4;
    orc_shadow(s, rays, skip, NR, 1, o0, f0);
    orc_shadow(s, rays, skip, NR, 0, o1, f1);
    for (int i = 0; i < NR; ++i)
        if (!f0[i] && !f1[i] && o0[i] != o1[i]) return 5;

    float total = 0.0f, pt[3];
    if (orc_scene_lights(s, &total) < 2 || !(total > 0.0f)) return 6;
    if (orc_light_sample(s, 0.3f, 0.2f, 0.7f, pt) < 0) return 7;

    orc_scene_free(s);
    free(v);
    free(tm);
    free(accum);
    free(taint);
    free(dprim);
    free(dcat);
    free(dcls);
    free(dflags);
    free(dlocal);
    free(dworld);
    printf("oracle sanitize run ok\n");
    return 0;
}
