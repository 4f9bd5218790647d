/*
 * oracle.h -- plain, slow CPU oracle for the direction-reuse path tracer of
 * "Generate Coherent Rays Directly" (Liu et al., arXiv 2310.07182).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU
 * baseline may load this library.  It shares no code, header, table or constant
 * generator with the CUDA library under paper_2310_07182_gb300/csrc; the two only meet
 * on the seeded input arrays produced by paper_2310_07182_gb300/scenes.py.
 *
 * Precision: closest-hit intersection and radiance accumulation are FP64.  Direction
 * sampling, tangent frames, reuse and throughput are computed in IEEE FP32 with a fixed
 * operation order (no FMA contraction, correctly rounded division and square root, own
 * polynomial sine/cosine), because ray directions must agree bit for bit with the GPU;
 * the paper does not state a precision (Sec. 4-5).
 *
 * Parity pins for each function are listed in oracle/README.md.  The hybrid-group weight
 * (Sec. 3.2, "Hybrid Tile") has no formula in the paper: parity unpinned beyond the
 * invariants the tests check.
 */
#ifndef ORC_ORACLE_H
#define ORC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): out = bijection_key(ctr). */
void orc_philox4x32_10(uint32_t k0, uint32_t k1, const uint32_t ctr[4], uint32_t out[4]);

/* Full-period LCG sequence x_{k+1} = (a x_k + c) mod m, x_0 given (Sec. 3.3). */
void orc_lcg_sequence(uint32_t m, uint32_t a, uint32_t c, uint32_t x0, uint32_t* out);

/* Interleaved grouping of one W*H tile (Sec. 3.3): sigma[i] = shuffled number of the
 * tile's i-th pixel (row-major); group = sigma / K.  abc_x0 receives (a, c, x0). */
void orc_tile_sigma(uint32_t tile_w, uint32_t tile_h, uint32_t tile, uint32_t frame,
                    uint64_t seed, int lcg, uint32_t* sigma, uint32_t* abc_x0);

/* FP32 sine/cosine for |x| <= pi/4 by Taylor polynomials (1/n! coefficients). */
void orc_sincos(float x, float* s, float* c);

/* Cosine-weighted hemisphere sample (Shirley-Chiu concentric map). */
void orc_sample_cosine(float u1, float u2, float* w);

/* GGX visible-normal-free sampling of D(m)(m.n) (Walter et al. 2007); returns 1 if the
 * sample is valid.  weight = f cos / pdf per channel. */
int orc_sample_ggx(const float* wo, float alpha, const float* f0, float u1, float u2,
                   float* wi, float* weight);

/* Tangent frame (t, b) of a unit normal n (Duff et al., JCGT 2017). */
void orc_frame(const float* n, float* t, float* b);

/* Smooth dielectric scattering (IOR eta, front = entering through the front face): writes
 * the reflected (returns 0) or refracted (returns 1) tangent-space direction. */
int orc_sample_dielectric(const float* wo, float eta, int front, float u, float* wi);

typedef struct orc_scene orc_scene;

orc_scene* orc_scene_new(const float* tri_xyz, uint32_t n_tri, const uint32_t* tri_mat,
                         const uint32_t* mat_type, const float* mat_params, uint32_t n_mat,
                         const float* env);
void orc_scene_free(orc_scene* s);
uint32_t orc_scene_nodes(const orc_scene* s);

/* Closest hit of n rays (rays: n x 8 fp32: o.xyz, unused, d.xyz, unused).
 * prim = original triangle index or -1, t in units of |d|; fragile bit 0 = decision too
 * close to call in FP32 (near-tie, near an edge, near the origin), bit 1 = t too
 * ill-conditioned in FP32 to agree to 1e-5 relative.  use_bvh=0: brute force. */
void orc_trace(const orc_scene* s, const float* rays, const int32_t* skip_prim, uint32_t n,
               int use_bvh, int32_t* prim, double* t, uint8_t* fragile);

/* orc_trace plus terr[i], the error scale an FP32 intersector's t can have for the winning
 * hit: 4 * 2^-24 * (coordinate magnitude) / |d| / |cos| of the ray against the triangle's
 * plane (0 on a miss). */
void orc_trace_bound(const orc_scene* s, const float* rays, const int32_t* skip_prim, uint32_t n,
                     int use_bvh, int32_t* prim, double* t, uint8_t* fragile, double* terr);

/* Shadow rays (n x 8 floats: origin, unused, direction, tmax): occluded if a triangle other
 * than skip_prim[i] is hit at 0 < t < tmax; fragile if FP32 could decide otherwise. */
void orc_shadow(const orc_scene* s, const float* rays, const int32_t* skip_prim, uint32_t n,
                int use_bvh, uint8_t* occluded, uint8_t* fragile);

/* Area of the triangle given by 9 floats (double arithmetic). */
double orc_triangle_area(const float* v);

/* Emitter triangles of the scene and their total area (float running sum). */
uint32_t orc_scene_lights(const orc_scene* s, float* total);

/* Light sample from uniforms (u0: emitter by area, u1 u2: point); returns the emitter's
 * original triangle index (-1: no emitter) and the point in p[3]. */
int32_t orc_light_sample(const orc_scene* s, float u0, float u1, float u2, float* p);

/* Solid-angle density of orc_sample_ggx's direction wi (double). */
double orc_pdf_ggx(const float* wo, const float* wi, float alpha);

/* GGX BSDF value f(wo, wi) in the tangent frame (double). */
void orc_eval_ggx(const float* wo, const float* wi, float alpha, const float* f0, double* f);

typedef struct {
    float pos[3], look_at[3], up[3];
    float vfov_deg;
    uint32_t width, height;
} orc_camera;

enum { ORC_INDEPENDENT = 0, ORC_MORTON_SORT = 1, ORC_DIRECTION_REUSE = 2, ORC_WORLD_REUSE = 3 };
/* ORC_OPT_NEE: next-event estimation at non-specular points.  ORC_OPT_HYBRID_DONOR: in hybrid
 * groups the diffuse members reuse the first diffuse member's own sample (the diffuse-group
 * rule restricted to them) instead of the average glossy direction. */
enum { ORC_OPT_NEE = 1, ORC_OPT_HYBRID_DONOR = 2, ORC_OPT_NEE_SHARED = 4 };
/* ORC_OPT_NEE_SHARED (with ORC_OPT_NEE): the members of a group join one light point, drawn
 * from the stream of the group's first alive member. */

typedef struct {
    uint32_t spp, max_bounces, mode;
    uint32_t tile_w, tile_h, k, interleave;
    uint32_t frame_base, reuse_depth; /* reuse at bounces b <= reuse_depth; 0 = all */
    uint32_t opts;                    /* ORC_OPT_* bits */
    uint64_t seed;
    /* Roughness threshold of the reuse classes (a knob the paper leaves open, Sec. 3.2): with
     * diffuse_roughness > 0 a GGX point of roughness >= it joins the diffuse class where
     * directions are reused; it then draws a cosine sample and weighs any direction it takes
     * by f cos / p_cos = pi f.  0: classes by material type only. */
    float diffuse_roughness;
} orc_params;

typedef struct {
    double* accum;      /* npx*3: += sum over samples of path radiance */
    uint8_t* taint;     /* npx: 1 if the pixel's result depends on a fragile decision */
    /* optional per-bounce debug (spp == 1), NULL to skip */
    int32_t* dbg_prim;  /* (B+1)*npx: original id of the hit of trace b; -1 miss, -2 none */
    uint8_t* dbg_cat;   /* B*npx: category of the pixel's group at reuse step b (1..B) */
    uint8_t* dbg_cls;   /* B*npx: material class of the pixel at step b */
    uint8_t* dbg_flags; /* B*npx: bit0 alive at step b, bit1 spawned a ray, bit2 tainted */
    float* dbg_local;   /* B*npx*3: tangent-space exit direction */
    float* dbg_world;   /* B*npx*3: world-space exit direction */
    uint64_t* counters; /* [0] primary rays, [1] secondary rays, [2] fragile decisions,
                           [3] shadow rays, [4] fragile shadow decisions */
    /* optional replay capture (spp == 1), NULL to skip: what trace b received and returned */
    float* dbg_ray;     /* (B+1)*npx*8: origin (rounded to float), skip id (int32 bits), direction, inf */
    float* dbg_t;       /* (B+1)*npx: hit distance rounded to float (inf on a miss) */
    float* dbg_beta;    /* (B+1)*npx*4: throughput rgb and the direction's density (rounded to float) */
} orc_outputs;

/* Render tiles [tile_begin, tile_end) of the image (Sec. 3, whole method). */
void orc_render_tiles(const orc_scene* s, const orc_camera* cam, const orc_params* p,
                      uint32_t tile_begin, uint32_t tile_end, orc_outputs* out);

/* Replay mode: one shading step recomputed from another renderer's captured state, so that
 * each stage is checked on that renderer's own inputs (one fragile closest-hit decision then
 * changes nothing downstream of it in the comparison).  Inputs, per pixel of the image (npx):
 * what trace b-1 received and returned. */
typedef struct {
    const float* ray;     /* npx*8: o.xyz, (unused), d.xyz, (unused) of trace b-1 */
    const int32_t* prim;  /* npx: its hit (original index), -1 miss, -2 not traced (path over) */
    const float* t;       /* npx: its hit distance */
    const float* beta;    /* npx*4: throughput rgb carried by the ray, w = its direction's density */
} orc_replay_in;

/* Outputs (each may be NULL), per pixel: what step b computes from those inputs. */
typedef struct {
    double* dL;           /* npx*3: radiance added at this step (environment, emission, light samples) */
    double* next_o;       /* npx*3: origin of the spawned ray of trace b (FP64; NaN if none) */
    float* next_beta;     /* npx*3: throughput it carries (NaN if none) */
    double* next_pdf;     /* npx: density of its direction (MIS under next-event estimation) */
    uint8_t* next_alive;  /* npx: 1 if the path spawned a ray */
    uint8_t* staint;      /* npx: a fragile shadow-ray decision at this step */
    uint8_t* cat, *cls, *flags; /* npx: as orc_outputs' per-bounce arrays, for step b */
    float* local, *world; /* npx*3 */
} orc_replay_out;

/* Step `bounce` (1..B: shade, classify, reuse, spawn; B + 1: the environment or emission at
 * the end of the last ray) of frame `frame` over tiles [tile_begin, tile_end). */
void orc_replay_step(const orc_scene* s, const orc_camera* cam, const orc_params* p, uint32_t frame,
                     uint32_t bounce, uint32_t tile_begin, uint32_t tile_end, const orc_replay_in* in,
                     orc_replay_out* out);

/* Primary ray direction through pixel (px, py) jittered by (u, v) in [0,1)^2 (pinhole camera,
 * vertical field of view, row 0 at the top). */
void orc_camera_ray(const orc_camera* cam, uint32_t px, uint32_t py, float u, float v, float* d);

/* Spawn point of a ray leaving a surface: p = o + t d in FP64, then p + side eps n with
 * eps = 2^-18 max(1, |p|_inf) (side +1: the incoming side of the surface, -1: through it). */
void orc_spawn_point(const double* o, const float* d, double t, const float* n, double side, double* out);

#ifdef __cplusplus
}
#endif
#endif
