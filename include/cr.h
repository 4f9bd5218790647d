/*
 * cr.h -- C ABI of libcr.so: a GB300 (sm_103a) direction-reuse path tracer after
 * "Generate Coherent Rays Directly" (Liu et al., arXiv 2310.07182).
 *
 * The library renders triangle scenes by wavefront path tracing on one GPU.  Its
 * secondary rays are generated in coherent form by the paper's method: pixels are
 * gathered into interleaved reuse groups (Sec. 3.3), each group is classed as diffuse,
 * glossy or hybrid from its shading points' materials, and shares a tangent-space exit
 * direction accordingly (Sec. 3.2).  Two comparators run on the same kernels:
 * independent sampling ("NoOpt", Table 1) and Morton-code ray sorting ("TwoPoint",
 * Table 1 and Sec. 4).
 *
 * Conventions for every entry point:
 *   - Every call returns a cr_status; CR_OK (0) on success.  On failure nothing the call
 *     owns is leaked, output buffers may be partly written, and cr_last_error() returns a
 *     message for the calling thread.  No call aborts, throws across the ABI or traps the
 *     GPU.
 *   - Pointers documented "host or device" may be either; the kind is found with
 *     cudaPointerGetAttributes.  Host buffers are copied through library-owned device
 *     memory; device buffers are used in place on the call's stream.
 *   - Buffers passed in are owned by the caller and are not retained after the call
 *     returns (device work on the call's stream may still read or write them until that
 *     stream is synchronised; every call below synchronises its stream before returning
 *     unless the description says otherwise).
 *   - A cr_scene is not thread-safe: calls on one scene must be serialised by the caller.
 */
#ifndef CR_H
#define CR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CR_OK = 0,
    CR_ERR_INVALID_ARG = 1,    /* an argument is out of range; message says which */
    CR_ERR_OOM = 2,            /* device or host allocation failed */
    CR_ERR_CUDA = 3,           /* a CUDA runtime call failed; message has its text */
    CR_ERR_TIMEOUT = 4,        /* a bounded device-side wait ran out */
    CR_ERR_STACK_OVERFLOW = 5, /* BVH deeper than the traversal stack (never for built scenes) */
    CR_ERR_BUSY = 6,           /* result not ready yet (server polling) */
    CR_ERR_NOT_FOUND = 7       /* unknown handle or id */
} cr_status;

/* Message of the last failed call on this thread ("" if none).  Owned by the library. */
const char* cr_last_error(void);
/* Library version string, e.g. "cr 0.1 sm_103a". */
const char* cr_version(void);

/* ---------------------------------------------------------------------------------- */
/* Scenes.  Material classes follow Sec. 3.2: Lambert is diffuse, GGX and mirror are glossy
 * or specular; emitters end a path and take no part in grouping.
 * Transmission (the paper's future work, Sec. 6): a translucent material (Lambertian
 * transmission) is diffuse with its lobe in the lower hemisphere; direction reuse gives it
 * the shared tangent-space direction mirrored through the tangent plane (z -> -|z|), so
 * the direction stays cosine-distributed in its own lobe.  A dielectric (smooth glass:
 * Fresnel reflection or Snell refraction, chosen by the reflectance) is specular.  Its
 * inside lies behind the triangles' front faces, the side cross(v1 - v0, v2 - v0) points
 * away from. */
typedef enum {
    CR_MAT_LAMBERT = 0,
    CR_MAT_GGX = 1,
    CR_MAT_MIRROR = 2,
    CR_MAT_EMITTER = 3,
    CR_MAT_DIELECTRIC = 4,
    CR_MAT_TRANSLUCENT = 5
} cr_mat_type;

typedef struct {
    uint32_t type;     /* cr_mat_type */
    float albedo[3];   /* Lambert/translucent albedo, GGX/mirror F0 (Schlick), dielectric tint; in [0, 1] */
    float roughness;   /* GGX alpha in (0, 1]; dielectric index of refraction in (0, 10]; else ignored */
    float emission[3]; /* emitter radiance; ignored by other types */
} cr_material;         /* 32 bytes */

typedef struct {
    float radiance[3]; /* constant environment radiance seen by rays that miss */
} cr_env;

enum { CR_BVH2 = 1u, CR_BVH8Q = 2u, CR_BVH4 = 4u };

typedef struct cr_scene cr_scene;

/* Build a device-resident scene: an SAH BVH2 (exact sweep up to 1024 triangles, 32 bins
 * above, SAH-chosen leaves of <= 4 triangles, depth <= 64) on the host, optionally collapsed into 8-wide nodes with 8-bit
 * conservatively quantised child boxes (bvh_flags & CR_BVH8Q; Ylitie et al. 2017, cited
 * in Sec. 2.3) and/or into 4-wide nodes that keep the BVH2's FP32 boxes (bvh_flags &
 * CR_BVH4; both give the BVH2's closest hits), then uploaded once.
 *   tri_xyz  host, n_tri * 9 floats: v0.xyz v1.xyz v2.xyz per triangle; all finite.
 *   tri_mat  host, n_tri material indices < n_mat.
 *   mats     host, n_mat materials.
 *   env      host, may be NULL (black).
 *   bvh_flags CR_BVH2 (always built) | CR_BVH8Q | CR_BVH4.
 *   out      receives the handle; destroy it with cr_scene_destroy.
 * The inputs are copied; the caller may free them when the call returns.
 * Errors: CR_ERR_INVALID_ARG (n_tri == 0 or > 2^28, NaN/Inf vertex, material index or
 * type out of range, NULL pointer), CR_ERR_OOM, CR_ERR_CUDA. */
cr_status cr_scene_create(const float* tri_xyz, uint32_t n_tri, const uint32_t* tri_mat,
                          const cr_material* mats, uint32_t n_mat, const cr_env* env,
                          uint32_t bvh_flags, cr_scene** out);

/* Free the scene's device and host memory (waits for the device).  NULL is a no-op. */
cr_status cr_scene_destroy(cr_scene* scene);

typedef struct {
    uint32_t n_tri, n_mat;
    uint32_t n_nodes2, depth2; /* BVH2 inner nodes, maximum leaf depth */
    uint32_t n_nodes8;         /* BVH8-Q nodes (0 if not built) */
    uint32_t n_lights;         /* emitter triangles (light samples of next-event estimation) */
    uint64_t device_bytes;     /* scene bytes resident on the device */
    double build_ms;           /* host build time */
    float bounds_lo[3], bounds_hi[3];
    float light_area;          /* total emitter area: float running sum of the areas (below) */
    uint32_t n_nodes4, depth4; /* BVH4 nodes and depth (0 if not built) */
} cr_scene_info;

cr_status cr_scene_get_info(const cr_scene* scene, cr_scene_info* info);

/* ---------------------------------------------------------------------------------- */
/* Rendering. */
typedef struct {
    float pos[3], look_at[3], up[3];
    float vfov_deg;          /* vertical field of view, in (0, 180) */
    uint32_t width, height;  /* >= 1, width * height <= 2^26 */
} cr_camera;

/* CR_WORLD_REUSE is the paper's Sec. 3.1 direct direction reusing, kept as an ablation: the
 * first alive member of a group shares its world-space exit direction and each diffuse
 * member weighs it with its own material (directions below its surface end the path). */
typedef enum { CR_INDEPENDENT = 0, CR_MORTON_SORT = 1, CR_DIRECTION_REUSE = 2, CR_WORLD_REUSE = 3 } cr_reuse_mode;

/* Per-call statistics (filled when cr_render_opts.stats != NULL).  Stage times are CUDA
 * event times on the call's stream summed over samples and bounces.  The queue compaction
 * runs inside the shade kernels (ms_compact reads 0) unless CR_OPT_ORDERED_QUEUES. */
typedef struct {
    double ms_total;           /* first launch to last (events) */
    double ms_raygen, ms_trace_primary, ms_trace_secondary, ms_shade, ms_compact, ms_sort, ms_accum;
    uint64_t primary_rays;     /* rays of the primary trace (valid pixels x spp) */
    uint64_t secondary_rays;   /* rays traced at bounces 1..B */
    uint64_t secondary_rays_b1;/* rays traced at bounce 1 */
    uint64_t kernel_launches;  /* library kernels launched by the call */
    uint64_t node_visits, tri_tests; /* counting pass only (CR_OPT_COUNT) */
    uint64_t shadow_rays;      /* shadow rays of next-event estimation (CR_OPT_NEE) */
    double ms_trace_shadow;    /* their any-hit trace */
    uint64_t h2d_bytes;        /* bytes the call copied host to device (job and scene tables) */
    uint64_t d2h_bytes;        /* bytes it copied device to host (a host out_rgb) */
} cr_stats;

/* Optional per-bounce capture (device pointers, spp must be 1).  npx = width * height.
 * Entries of rays that were not traced / pixels not alive are left untouched, so fill the
 * buffers beforehand (e.g. prim with -2). */
typedef struct {
    int32_t* prim;   /* (B+1) * npx: original triangle index hit by trace b (0 = primary), -1 miss */
    uint8_t* cat;    /* B * npx: category of the pixel's group at step b: 0 empty, 1 diffuse, 2 glossy, 3 hybrid */
    uint8_t* cls;    /* B * npx: class of the pixel's shading point: 0 none, 1 diffuse, 2 glossy/specular,
                        3 diffuse transmission (translucent, grouped with the diffuse class) */
    uint8_t* flags;  /* B * npx: bit0 alive at step b, bit1 spawned a secondary ray */
    float* local;    /* B * npx * 3: tangent-space exit direction */
    float* world;    /* B * npx * 3: world-space exit direction */
    /* Optional replay capture (all three or none; NULL = off).  What trace b received and
     * returned, so that a checker can recompute each later stage from the GPU's own inputs
     * (a stage-by-stage comparison that one fragile decision cannot derail). */
    float* ray;      /* (B+1) * npx * 8: the ray of trace b: origin.xyz, the skipped triangle's
                        original index (int32 bits, -1 none), direction.xyz, tmax */
    float* t;        /* (B+1) * npx: its hit distance in units of |d| (inf on a miss) */
    float* beta;     /* (B+1) * npx * 4: the path throughput the ray carried (rgb) and, in w,
                        the density of its direction (next-event estimation; 0 otherwise) */
} cr_debug;

enum {
    CR_OPT_STATS = 1u,      /* record per-stage CUDA events (adds event records between launches) */
    CR_OPT_COUNT = 2u,      /* counting pass: count node visits / triangle tests (slower) */
    CR_OPT_NO_SYNC = 4u,    /* return without synchronising the stream (device out_rgb only) */
    CR_OPT_PERSISTENT = 8u, /* persistent trace kernel with dynamic ray fetch (BVH2) */
    CR_OPT_SPECULATIVE = 16u, /* speculative traversal with a parked leaf per lane (BVH2) */
    CR_OPT_PACKET_PRIMARY = 32u,  /* warp-packet traversal of primary rays (BVH2) */
    CR_OPT_PACKET_SECONDARY = 64u, /* warp-packet traversal of secondary rays (BVH2) */
    CR_OPT_TWO_PHASE = 128u, /* secondary rays: 32-visit budget, compact the unfinished, resume (BVH2) */
    CR_OPT_NEE = 256u,     /* cr_render: next-event estimation (the job flag CR_JOB_NEE) */
    CR_OPT_ANY_HIT = 512u, /* cr_trace_rays: visibility only (any hit before tmax, see there) */
    CR_OPT_HYBRID_DONOR = 1024u, /* cr_render: the job flag CR_JOB_HYBRID_DONOR */
    CR_OPT_NEE_SHARED = 2048u,   /* cr_render: the job flag CR_JOB_NEE_SHARED */
    CR_OPT_STATS_TRACES = 4096u, /* like CR_OPT_STATS but events only around the trace launches
                                    (less event traffic in the step; other stage times read 0) */
    CR_OPT_ORDERED_QUEUES = 8192u /* build the ray and group queues in position order with a
                                     separate three-launch compaction (count, scan, scatter)
                                     instead of appending them in the shade; same images */
};

/* Reordering keys of CR_MORTON_SORT (Table 1 comparators; 30-bit keys, layouts in path.cu):
 * TwoPoint interleaves origin and an estimated end point 0.25 x the largest scene extent
 * away; Origin is the origin's Morton code; Reis puts origin bits above direction bits,
 * Costa the reverse; AilaCompact interleaves origin and direction.  HierarchyCut is a key
 * from the BVH2 (a reading of MLHCC, of which the paper gives only the name, the code length
 * and lambda = 0.125): the 15-level descent paths of the origin and of the point 0.125 x the
 * largest scene extent along the ray, interleaved. */
typedef enum {
    CR_SORT_TWO_POINT = 0, CR_SORT_ORIGIN = 1, CR_SORT_REIS = 2, CR_SORT_COSTA = 3, CR_SORT_AILA_COMPACT = 4,
    CR_SORT_HIERARCHY_CUT = 5
} cr_sort_key;

typedef struct {
    uint32_t k;            /* pixels per reuse group K; 0 = W*H.  Power of two dividing W*H, <= 256 */
    uint32_t interleave;   /* 1: LCG-shuffled groups (Sec. 3.3, default); 0: contiguous groups */
    uint64_t seed;         /* Philox key */
    uint32_t frame_base;   /* frame index of the first sample (progressive rendering) */
    uint32_t reuse_depth;  /* reuse at bounces b <= reuse_depth; 0 = every bounce */
    uint32_t bvh;          /* CR_BVH2 (default), CR_BVH8Q or CR_BVH4 (scene must have it; with
                              CR_BVH4 shadow rays stay on the BVH2, and the BVH2 traversal
                              variants of flags -- persistent, packet, speculative, two-phase --
                              do not apply) */
    uint32_t block;        /* trace block size, multiple of 32 in [32, 512]; 0 = 128 for
                            * primary rays and 64 for secondary rays */
    uint32_t flags;        /* CR_OPT_* */
    uint32_t sort_key;     /* cr_sort_key of CR_MORTON_SORT (default TwoPoint) */
    uint32_t stack;        /* BVH2 traversal stack entries per thread in shared memory: 8, 16 or 32 (0 = 16) */
    float diffuse_roughness; /* > 0: GGX of at least this roughness joins the diffuse class
                              * of the reuse groups (cosine samples weighted pi f while
                              * directions are reused; independent sampling is unchanged);
                              * 0: classes by material type (Sec. 3.2).  Finite, >= 0. */
    void* stream;          /* cudaStream_t to run on; NULL = legacy default stream */
    cr_stats* stats;       /* optional, host */
    cr_debug* debug;       /* optional, host struct of device pointers */
    /* Render only tiles [tile_begin, tile_end) of the image's group_w x group_h tiling
     * (row-major tile order; 0, 0 = every tile).  Pixels outside the range are left as they
     * are in out_rgb.  Every reuse group lies inside one tile (Sec. 3.3) and random numbers
     * are keyed by pixel, so tile-aligned parts of an image rendered separately (on one or
     * several devices) equal the whole render bit for bit. */
    uint32_t tile_begin, tile_end;
} cr_render_opts;

/* Fill opts with the defaults: k = 0, interleave = 1, seed = 0, frame_base = 0,
 * reuse_depth = 0, bvh = CR_BVH2, block = 0, flags = 0, stream = NULL, stats = debug = NULL. */
cr_status cr_render_opts_default(cr_render_opts* opts);

/* Render spp samples per pixel with paths of up to max_bounces secondary rays and write
 * the mean radiance (linear fp32 RGB, row-major, top row first) to out_rgb.
 *   scene        from cr_scene_create.
 *   camera       host struct.
 *   spp          >= 1 (Sec. 3.1: several samples = one sample in each of several finer pixels).
 *   max_bounces  1..16: number of secondary rays per path (no Russian roulette).
 *   mode         CR_INDEPENDENT (each path samples its own BSDF), CR_MORTON_SORT (the same
 *                paths, secondary rays sorted by a 30-bit TwoPoint Morton key before each
 *                trace), CR_DIRECTION_REUSE (Sec. 3.2-3.3).
 *   group_w, group_h  tile W x H of the reuse-domain partition (Sec. 3.3); W*H a power of
 *                two <= 1024.  Rays of every mode are laid out tile by tile.
 *   out_rgb      host or device, width*height*3 floats, written once at the end.  Host
 *                memory gets a staging buffer and one device-to-host copy (a DMA copy from
 *                page-locked memory; on GB300 it beats the output kernel writing
 *                page-locked memory over the chip-to-chip link: 0.13 ms against 0.15-0.48
 *                ms for a 1920x1080 image).
 * With opts == NULL (cr_render) K = W*H.  The result depends only on (scene, camera, spp,
 * bounces, mode, W, H, K, interleave, seed, frame_base, reuse_depth): random numbers are
 * keyed by (pixel, frame, bounce), never by ray order, so CR_MORTON_SORT gives the same
 * image as CR_INDEPENDENT bit for bit.
 * Errors: CR_ERR_INVALID_ARG, CR_ERR_OOM, CR_ERR_CUDA. */
cr_status cr_render(cr_scene* scene, const cr_camera* camera, uint32_t spp, uint32_t max_bounces,
                    cr_reuse_mode mode, uint32_t group_w, uint32_t group_h, float* out_rgb);

cr_status cr_render_ex(cr_scene* scene, const cr_camera* camera, uint32_t spp, uint32_t max_bounces,
                       cr_reuse_mode mode, uint32_t group_w, uint32_t group_h, float* out_rgb,
                       const cr_render_opts* opts);

/* ---------------------------------------------------------------------------------- */
/* Batched rendering: many jobs (scenes, cameras, spp, bounces, modes) merged into one
 * wavefront, one launch per stage per bounce over the slots of all jobs, optionally replayed
 * from a CUDA graph.  Jobs of one batch share the tile shape, K, interleave and BVH layout. */
typedef struct {
    cr_scene* scene;     /* must outlive the batch */
    cr_camera camera;
    uint32_t spp;        /* >= 1 */
    uint32_t max_bounces;/* 1..16 */
    uint32_t mode;       /* cr_reuse_mode */
    uint32_t reuse_depth;/* 0 = every bounce */
    uint64_t seed;
    uint32_t frame_base;
    uint32_t flags;      /* CR_JOB_* */
    float* out_rgb;      /* DEVICE buffer of width*height*3 floats */
    float diffuse_roughness; /* as in cr_render_opts (0: classes by material type) */
} cr_job;                /* 104 bytes */

/* Next-event estimation (a standard path-tracing estimator the paper does not discuss; it
 * leaves the reuse of exit directions unchanged).  At every shading point that is not a
 * mirror, one emitter point is drawn and joined by a shadow ray:
 *   emitter  x = u0 * A (float), A = the float running sum of the emitter triangles' areas
 *            in triangle-index order, each area 0.5 |(v1 - v0) x (v2 - v0)| in double; the
 *            first emitter whose running sum exceeds x (the last if none), i.e. by area;
 *   point    s = sqrt(u1), p = (1 - s) v0 + s (1 - u2) v1 + s u2 v2 (float);
 *   (u0, u1, u2) from Philox(seed; pixel, frame, bounce, "LITE").
 * The shadow ray leaves from the spawn point of the path's next ray toward p and ends at
 * 1 - 2^-10 of the way; if nothing blocks it, L += w_l beta f Le cos_i cos_l A / r^2 (cos_l
 * at the two-sided emitter).  Emission that the path's next BSDF-sampled ray meets is
 * weighed by 1 - w_l of that direction: multiple importance sampling with the power
 * heuristic, w_l = p_l^2 / (p_l^2 + p_b^2), p_l = r^2 / (cos_l A) the light sample's
 * solid-angle density and p_b the shading point's own BSDF density (cos / pi, or the GGX
 * reflection density; mirrors and camera rays keep full emission).  Where the continuation
 * direction has density p_b (independent sampling, diffuse and glossy groups) the mean
 * equals plain path tracing's. */
/* CR_JOB_HYBRID_DONOR: an unbiased alternative to the paper's hybrid-group rule (Sec. 3.2
 * gives diffuse members the average glossy direction, which is not cosine-distributed, so
 * the image is biased).  With the flag, the diffuse members of a hybrid group reuse the
 * first diffuse member's own cosine sample (the diffuse-group rule among them) and the
 * glossy / specular members keep their own samples: every direction keeps its density. */
/* CR_JOB_NEE_SHARED (with CR_JOB_NEE): the members of a reuse group join one light point,
 * drawn from the "LITE" stream of the group's first alive member, so the group's shadow rays
 * converge (coherent traversal); each pixel's light point is still distributed by area, so
 * the estimate keeps its mean (an extension in the spirit of Sec. 3.2, not in the paper). */
enum { CR_JOB_NEE = 1u, CR_JOB_HYBRID_DONOR = 2u, CR_JOB_NEE_SHARED = 4u };

enum { CR_BATCH_GRAPH = 1u /* capture the launch sequence once, replay it on every run */ };

typedef struct {
    uint32_t group_w, group_h; /* tile W x H */
    uint32_t k;                /* 0 = W*H */
    uint32_t interleave;       /* 1 LCG (Sec. 3.3), 0 contiguous */
    uint32_t bvh;              /* CR_BVH2 or CR_BVH8Q (every scene must have it) */
    uint32_t block;            /* trace block size; 0 = 128 */
    uint32_t flags;            /* CR_BATCH_GRAPH | CR_OPT_PERSISTENT */
    uint32_t sort_key;         /* cr_sort_key of CR_MORTON_SORT jobs */
    uint32_t stack;            /* shared-memory traversal stack entries: 8, 16, 32 (0 = 16) */
    void* stream;              /* cudaStream_t used by cr_batch_run (NULL = a stream the batch owns) */
} cr_batch_opts;

typedef struct cr_batch cr_batch;

/* Plan a batch: checks every job, builds the per-sample-pass job tables, allocates the path
 * state for the largest pass (see cr_batch_device_bytes) and, with CR_BATCH_GRAPH, captures
 * the whole launch sequence into a CUDA graph.  jobs is copied; scenes and outputs are not.
 * Errors: CR_ERR_INVALID_ARG, CR_ERR_OOM, CR_ERR_CUDA. */
cr_status cr_batch_create(const cr_job* jobs, uint32_t n_jobs, const cr_batch_opts* opts, cr_batch** out);
/* Render every job of the batch once (each job's spp samples) into its out_rgb and wait.
 * stats (may be NULL): ms_total (CUDA events around the run), secondary rays, launches. */
cr_status cr_batch_run(cr_batch* batch, cr_stats* stats);
cr_status cr_batch_destroy(cr_batch* batch);
/* Path-state bytes a batch of these jobs would allocate (admission by device footprint). */
cr_status cr_batch_device_bytes(const cr_job* jobs, uint32_t n_jobs, const cr_batch_opts* opts, uint64_t* bytes);

/* Autotuner: times candidate (W,H) in {4x4, 8x8, 16x16}, K <= W*H/4 (larger K loses image
 * quality, Sec. 5.3), interleave {LCG, contiguous} if allowed, and trace block {64, 128,
 * 256} on the given jobs (renders them), then the traversal stack depth in shared memory
 * {8, 16, 32} for the fastest of those, and writes the winner into *opts (its bvh and
 * flags are kept).  allow_contiguous = 0 keeps the LCG interleave of Sec. 3.3.
 * Quality guard: grouping changes which directions are shared, so speed alone could pick a
 * grouping that shows the method's correlation artifacts (Sec. 3.3, 5.3).  When some job
 * reuses directions, the largest such job of at most 512 x 512 pixels (the probe) is
 * rendered once at 64 spp with independent sampling as a reference, and once per distinct
 * (W, H, K, interleave) at its own spp, seed and frames.  The error measure is the MSE of
 * 4x4-pixel block means: at a fixed spp, pixel-wise MSE is blind to how errors of
 * neighbouring pixels correlate, and the block means are not.  A grouping whose error
 * exceeds the default grouping's (8x8, K=8, LCG) by more than 10% is not chosen. */
typedef struct {
    uint32_t n_candidates;
    uint32_t best_group_w, best_group_h, best_k, best_interleave, best_block, best_stack;
    double best_ms;   /* device ms of one run of the best candidate */
    double worst_ms;  /* slowest candidate */
    double default_ms;/* 8x8, K=8, LCG, block 128 */
    /* Quality guard (when a job reuses directions): error of the probe job against its 64-spp
     * independent reference (MSE of 4x4-pixel block means) for the chosen grouping and for
     * the default one, the candidates rejected for an error more than 10% above the
     * default's (not timed), and the probe job's index (all 0 when the guard is off). */
    double best_mse, default_mse;
    uint32_t n_rejected, probe_job;
} cr_tune_report;

cr_status cr_batch_autotune(const cr_job* jobs, uint32_t n_jobs, uint32_t allow_contiguous, cr_batch_opts* opts,
                            cr_tune_report* report);

/* ---------------------------------------------------------------------------------- */
/* Serving: a request loop with continuous batching at bounce granularity.  A server thread
 * runs a rolling wavefront: each iteration is one launch per stage (shade, light samples,
 * sample sums, ray generation, trace) over the slots of every admitted job, whatever bounce
 * each job is at, so a request joins at the next bounce launch after it is admitted and its
 * buffers are free for others as soon as its last sample is summed.  Queued jobs are
 * admitted first-come (later ones may backfill) while their device footprint fits the budget:
 * path-state slots (whole tiles, ~170 B per slot), accumulation (16 B/px) and, for host
 * outputs, staging (12 B/px), each a first-fit range of an arena allocated at creation (the
 * loop allocates nothing).  Results equal stand-alone renders with the same tile shape, K and
 * interleave. */
typedef struct {
    uint64_t hbm_budget;       /* bytes of device memory the server may use (>= 64 MiB) */
    uint32_t group_w, group_h, k, interleave, bvh, block; /* as cr_batch_opts */
    /* Express lane (0 = none): jobs of at most express_rays ray steps (pixels x spp x
     * (max_bounces + 1)) run in a second rolling wavefront with its own path state (1/8 of
     * the slots) on a stream of the device's highest priority, so their bounce launches do
     * not wait for the large jobs' launches.  An express job that does not fit its lane goes
     * to the main one.  Results are the same in either lane. */
    uint32_t express_rays, pad;
} cr_server_opts;

typedef struct {
    double t_submit_ms, t_admit_ms, t_done_ms; /* server clock (ms since cr_server_create) */
    double latency_ms;                         /* t_done - t_submit: result available on the host */
    uint32_t samples, pad;
    uint64_t footprint_bytes;
} cr_job_stats;

typedef struct {
    uint64_t jobs_submitted, jobs_done;
    uint64_t passes;           /* iterations of the rolling wavefronts (one bounce step of every active job of a lane) */
    uint64_t secondary_rays, kernel_launches, used_bytes;
    double busy_ms;            /* host time spent enqueueing iterations (up to four run ahead of the GPU) */
    uint32_t queued, active;
} cr_server_stats;

typedef struct cr_server cr_server;

cr_status cr_server_create(const cr_server_opts* opts, cr_server** out);
/* Queue a job (copied).  out_rgb may be host or device memory and must stay valid until the
 * job completes.  Errors: CR_ERR_INVALID_ARG, CR_ERR_OOM (larger than the whole budget). */
cr_status cr_server_submit(cr_server* server, const cr_job* job, uint64_t* job_id);
/* CR_OK once the job's output is written (then the id is forgotten), CR_ERR_BUSY while it is
 * queued or rendering, CR_ERR_NOT_FOUND for unknown ids, or the job's error. */
cr_status cr_server_poll(cr_server* server, uint64_t job_id, cr_job_stats* stats);
/* As poll, but waits up to timeout_ms; CR_ERR_TIMEOUT if the job is still running. */
cr_status cr_server_wait(cr_server* server, uint64_t job_id, uint32_t timeout_ms, cr_job_stats* stats);
cr_status cr_server_get_stats(cr_server* server, cr_server_stats* stats);
/* Stop the loop (jobs not yet completed are dropped: their outputs are undefined) and free
 * the server's memory. */
cr_status cr_server_destroy(cr_server* server);

/* ---------------------------------------------------------------------------------- */
/* Parity / debug entry points (the same kernels as the render path). */

/* Closest hit of n rays (Sec. 1: the intersection step).
 *   rays      host or device, n * 8 floats: o.xyz, (unused), d.xyz, tmax (inf = unbounded).
 *   skip_prim host or device or NULL: n original triangle indices the ray must ignore (-1 none).
 *   prim      host or device, n int32: original index of the closest hit, -1 if none.
 *   t         host or device, n floats: hit distance in units of |d| (inf if none).
 * Hit rule: watertight test (Woop et al. 2013), t > 0, edges inclusive; equal t goes to the
 * smaller original index.  opts may be NULL (bvh, block, stream, flags are read).
 * With CR_OPT_ANY_HIT in opts->flags the traversal stops at the first triangle hit before
 * tmax (the shadow-ray kernel's traversal): prim is then some occluder (not necessarily the
 * closest) and t its distance, or -1 and inf if the ray reaches tmax unblocked. */
cr_status cr_trace_rays(cr_scene* scene, const float* rays, const int32_t* skip_prim, uint32_t n,
                        int32_t* prim, float* t, const cr_render_opts* opts);

/* Interleaved grouping (Sec. 3.3) of one frame: slot_of_pixel[p] = tile * W*H + sigma(i),
 * where i is the pixel's row-major index within its tile; its group is slot / K.
 * slot_of_pixel: host or device, width*height uint32. */
cr_status cr_debug_groups(uint32_t width, uint32_t height, uint32_t group_w, uint32_t group_h,
                          uint32_t interleave, uint64_t seed, uint32_t frame, uint32_t* slot_of_pixel);

/* Philox4x32-10 of n counters under key = seed: out[4i..4i+3] = philox(seed, ctr[4i..4i+3]).
 * ctr, out: host or device, n*4 uint32. */
cr_status cr_debug_philox(uint64_t seed, const uint32_t* ctr, uint32_t n, uint32_t* out);

/* The ray sort of CR_MORTON_SORT (a stable LSD radix sort: three passes of 10-bit digits in
 * one cooperative launch, grid barriers between the phases of a pass) on caller keys:
 * keys_out, vals_out = (keys & (2^30 - 1), vals) in ascending key order, equal keys in input
 * order.  The sort runs reps times on the same input and *ms (may be NULL) receives the mean
 * device time of one sort (CUDA events; the key kernel and the three passes).
 * keys, vals, keys_out, vals_out: host or device, n elements.  n <= 2^28.
 * Errors: CR_ERR_INVALID_ARG, CR_ERR_OOM, CR_ERR_CUDA, CR_ERR_TIMEOUT (a bounded grid-barrier
 * wait ran out; the order may then be wrong). */
cr_status cr_debug_sort(const uint32_t* keys, const int32_t* vals, uint32_t n, uint32_t reps, uint32_t* keys_out,
                        int32_t* vals_out, double* ms);

/* The device BSDF samplers, one call per row (fp32, same code as the render path):
 *   kind 0: cosine hemisphere from (u1, u2); kind 1: GGX with alpha = param[4i+0] and
 *   F0 = param[4i+1..3] about wo; kind 2: mirror.  wo: n*3, u: n*2, param: n*4,
 *   wi/weight: n*3, valid: n.  All host or device.  Also sincos: kind 3 writes
 *   (sin x, cos x, 0) of x = u[2i] to wi. */
cr_status cr_debug_sample(uint32_t kind, uint32_t n, const float* wo, const float* u, const float* param,
                          float* wi, float* weight, uint8_t* valid);

/* Host-only check of the BVH builders (no GPU needed): builds the BVH2 (and the BVH8-Q if
 * flags & CR_BVH8Q, the BVH4 if flags & CR_BVH4) for the triangles and verifies them by
 * walking every root-to-leaf path: each triangle must sit in a leaf, and every box on its
 * path (BVH8-Q boxes as the kernel decodes them from 8-bit codes) must contain all three of
 * its vertices; BVH4 slots must be used with finite planes or unused with NaN planes. */
typedef struct {
    uint32_t n_nodes2, depth2, n_nodes8, depth8, stack_bound8;
    uint32_t covered2, covered8;       /* triangles found in a leaf */
    uint32_t violations2, violations8; /* (triangle, ancestor box) pairs not containing it */
    uint32_t pad;
    double build_ms2, build_ms8;
    uint32_t n_nodes4, depth4, stack_bound4, covered4, violations4, pad4;
} cr_bvh_report;

cr_status cr_debug_bvh_check(const float* tri_xyz, uint32_t n_tri, uint32_t flags, cr_bvh_report* report);

/* ---------------------------------------------------------------------------------- */
/* Tracing without allocation.  The paper has no counterpart: this is a library service.
 *
 * cr_trace_rays allocates device staging buffers on every call.  Some callers cannot allow
 * that: a host framework that owns all device memory through its own pool allocator and
 * forbids raw cudaMalloc, a latency-critical loop that cannot afford the device-wide
 * synchronisation of cudaMalloc/cudaFree, or a process that has reserved nearly all device
 * memory, so an allocation could fail mid-frame.  cr_trace_rays_static computes exactly
 * what cr_trace_rays computes (same kernels, BVH2, block 128) but keeps its scratch (ray and
 * hit records, 40 bytes per ray) in one file-scope device array sized for
 * CR_TRACE_STATIC_MAX_RAYS rays (2.5 MiB), which every GPU that loads the library holds
 * until the process exits.  It calls no cudaMalloc, cudaFree or allocating library routine.
 *   rays, skip_prim (or NULL), prim, t: DEVICE pointers of the current device with the
 *   layouts of cr_trace_rays; host pointers (staging them would need an allocation) and
 *   other devices' memory are rejected, and so is a scene created on another device.
 *   n: 0..CR_TRACE_STATIC_MAX_RAYS; larger n returns CR_ERR_INVALID_ARG (trace in chunks).
 *   stream: cudaStream_t to run on (NULL = legacy default stream).  The call synchronises
 *   this stream before it returns.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress,
 * with that device current); make that first call before any stream capture.  All calls
 * share the one array and it keeps the last call's contents: calls that overlap on the GPU
 * (other host threads, or other streams) race on it, so serialise them.
 * Errors: CR_ERR_INVALID_ARG, CR_ERR_CUDA. */
#define CR_TRACE_STATIC_MAX_RAYS 65536u
cr_status cr_trace_rays_static(cr_scene* scene, const float* rays, const int32_t* skip_prim, uint32_t n,
                               int32_t* prim, float* t, void* stream);

/* ---------------------------------------------------------------------------------- */
/* Measurement utility (no counterpart in the paper): the L2 read roof of the roofline.
 * Allocates a device buffer of `bytes` (rounded down to 16 B), fills it, reads it once to
 * warm the L2, then times `reps` passes of a read-only kernel (16-byte read-only loads, a
 * grid of 8 blocks of 256 threads per SM, a grid-stride loop) with CUDA events and writes the
 * bytes read per second (GB/s, 1e9) to *gbs.  Choose `bytes` well below the L2 size so the
 * passes hit in L2.  Frees the buffer before returning.
 * Errors: CR_ERR_INVALID_ARG (bytes < 1 MiB, reps 0, NULL gbs), CR_ERR_OOM, CR_ERR_CUDA. */
cr_status cr_measure_l2_read(uint64_t bytes, uint32_t reps, double* gbs);

#ifdef __cplusplus
}
#endif
#endif
