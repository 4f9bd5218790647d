// cr_internal.h -- host-side declarations shared by the library's translation units
// (scene build, kernel launchers, C ABI).  Not installed; the public ABI is include/cr.h.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "cr.h"

namespace cr {

// ------------------------------------------------------------------------------------
// BVH2 in the device layout: 4 x 16 B per inner node, holding both children:
//   n0 = (c0.lo.x, c0.hi.x, c0.lo.y, c0.hi.y)
//   n1 = (c1.lo.x, c1.hi.x, c1.lo.y, c1.hi.y)
//   n2 = (c0.lo.z, c0.hi.z, c1.lo.z, c1.hi.z)
//   n3 = (link0, link1, 0, 0) as int bits
// link >= 0: inner node index; link < 0: leaf ~((first << 2) | (count - 1)), count 1..4,
// first = index of the leaf's first triangle in leaf order.
struct HostBVH2 {
    std::vector<float> nodes;         // 16 floats per inner node
    std::vector<uint32_t> leaf_order; // leaf-order position -> original triangle index
    uint32_t n_nodes = 0;
    uint32_t depth = 0;
    float lo[3], hi[3];
};

// SAH build (exact sweep up to 1024 triangles, 32 bins per axis above; SAH-chosen leaves
// of <= 4 triangles; median splits below depth 40 so the depth stays <= 64).
HostBVH2 build_bvh2(const float* tri_xyz, uint32_t n_tri, int n_threads);

// BVH8-Q: 8-wide nodes of 80 B (five 16-byte words) with 8-bit child boxes, after the
// compressed wide BVH of Ylitie et al. 2017 (the node format; collapse, slot order and
// traversal here are our own):
//   words 0-2  origin.xyz (float)                 word 3  ex | ey << 8 | ez << 16 | imask << 24
//   word 4     first inner child node             word 5  first triangle (BVH8 leaf order)
//   words 6-7  meta[8]: inner child: its rank among the inner children; leaf child:
//              (count << 5) | offset from the first triangle; empty: 0 with imask bit clear
//   words 8-19 qlo_x[8] qlo_y[8] qlo_z[8] qhi_x[8] qhi_y[8] qhi_z[8]
// ex/ey/ez are biased float exponents: the grid step of axis a is 2^(e_a - 127).  A child box
// decodes as origin + q * step in float (one exact product, one rounded add); the builder
// rounds lower bounds down and upper bounds up and checks the float decode, so every
// decoded box contains the exact child box.  Children sit in slots by the octant of their
// centroid, and a ray visits slots in the order k ^ octant(ray direction).
struct HostBVH8 {
    std::vector<uint32_t> nodes;      // 20 words per node
    std::vector<uint32_t> leaf_order; // BVH8 triangle position -> original triangle index
    uint32_t n_nodes = 0;
    uint32_t depth = 0;
    uint32_t stack_bound = 0;         // largest traversal stack a ray can need (the depth)
};
HostBVH8 build_bvh8q(const HostBVH2& b2, const float* tri_xyz);
// BVH4: the BVH2 collapsed into 4-wide nodes with FP32 child boxes, 32 floats (128 B) per node:
//   floats 0-3 lo.x of children 0-3, 4-7 hi.x, 8-11 lo.y, 12-15 hi.y, 16-19 lo.z, 20-23 hi.z,
//   24-27 child links as int bits (>= 0 BVH4 node, < 0 BVH2 leaf code, kBvh4Empty unused), 28-31 0.
// Boxes and leaves are the BVH2's (same triangle records); the root is node 0.  An unused
// slot's planes are NaN: the slab test's far distance is then NaN and the box is never entered.
constexpr uint32_t kBvh4NodeFloats = 32;
constexpr int32_t kBvh4Empty = 0x7fffffff;
struct HostBVH4 {
    std::vector<float> nodes;
    uint32_t n_nodes = 0;
    uint32_t depth = 0;
    uint32_t stack_bound = 0; // largest traversal stack a ray can need (three per level)
};
HostBVH4 build_bvh4(const HostBVH2& b2);
void check_bvh4(const HostBVH4& b4, const HostBVH2& b2, const float* v, uint32_t n_tri, uint32_t& covered,
                uint32_t& violations);
constexpr uint32_t kBvh4StackCapacity = 96; // traversal stack entries of the BVH4 kernel
constexpr uint32_t kBvh2StackCapacity = 64; // traversal stack entries of the BVH2 kernels (> tree depth)
constexpr uint32_t kBvh8StackCapacity = 48; // traversal stack entries of the BVH8-Q kernel (one per level)
void check_bvh2(const HostBVH2& b, const float* v, uint32_t n_tri, uint32_t& covered, uint32_t& violations);
void check_bvh8(const HostBVH8& b, const float* v, uint32_t n_tri, uint32_t& covered, uint32_t& violations);

// ------------------------------------------------------------------------------------
// Device-side scene description (host copy kept in the scene handle).
struct DevScene {
    const float4* nodes2 = nullptr; // 4 per node
    const uint4* nodes8 = nullptr;  // 5 per node
    const float4* nodes4 = nullptr; // 8 per node (BVH4, if built)
    const float4* tris = nullptr;   // 3 per triangle in leaf order: v0|orig, v1|mat, v2|0
    const float4* tris8 = nullptr;  // the same records in BVH8-Q leaf order (if built)
    const float4* mats = nullptr;   // 2 per material: (type bits, albedo), (roughness, emission)
    float env[3] = {0, 0, 0};
    float lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    uint32_t n_tri = 0, n_mat = 0;
    // emitter triangles for next-event estimation
    const float* light_cdf = nullptr; // float running sum of the areas, triangle-index order
    const float4* lights = nullptr;   // 4 per emitter: v0|orig, v1|0, v2|0, emission|0
    uint32_t n_lights = 0;
    float light_total = 0.0f;
    uint32_t n_nodes2 = 0, n_nodes8 = 0, n_nodes4 = 0;
    uint32_t* err = nullptr; // device word: index checks that failed (debug builds)
};

// One entry of the device scene table a pass reads (tris in the order of the BVH traversed).
struct SceneDev {
    const float4* nodes2;
    const uint4* nodes8;
    const float4* nodes4; // BVH4 (with the BVH2's triangle records), or NULL
    const float4* tris;
    const float4* mats;
    float env[4];
    float lo[4], hi[4];
    const float* light_cdf;
    const float4* lights;
    uint32_t n_lights;
    float light_total;
    // sizes of this entry's arrays and the scene's error word (bounds checks of a debug build)
    uint32_t n_nodes, n_tris, n_mats;
    uint32_t* err;
    uint32_t n_nodes4 = 0; // BVH4 nodes (set where render and trace entries are made)
};
SceneDev scene_entry(const DevScene& s, bool bvh8);

// Camera basis rounded to float once (computed in double on the host).
struct CamBasis {
    float pos[3], fwd[3], right[3], up[3];
    float tx, ty; // tan(vfov/2) * aspect, tan(vfov/2)
    uint32_t width, height;
};
CamBasis make_camera(const cr_camera& c);

// One render job of one sample pass: a device table entry.  Jobs of a pass occupy
// consecutive tile ranges; every reuse group lies inside one tile, hence inside one job.
struct JobDev {
    CamBasis cam;
    uint32_t tiles_x;
    uint32_t tile_base;   // first tile of the job in the pass
    uint32_t px_base;     // first pixel of the job in the accumulation buffer
    uint32_t scene;       // index into the scene table
    uint32_t frame;       // frame index of this pass (frame_base + sample)
    uint32_t max_bounces; // B of the job
    uint32_t reuse_mask;  // bit b: direction reuse at bounce b
    uint32_t interleave;
    uint64_t seed;
    float* out;           // device output (w*h*3 floats) of the job
    float inv_spp;
    uint32_t world_mask;  // bit b: world-space direct reuse (Sec. 3.1 ablation) at bounce b
    uint32_t nee;         // 1: next-event estimation, 2: with light points shared per group
    uint32_t hybrid_donor; // 1: hybrid groups reuse the first diffuse member's sample
    uint32_t sample_flags; // bit 0: this pass is the job's first sample, bit 1: its last
    float diffuse_rough;   // GGX of at least this roughness is in the diffuse class (0: off)
    uint32_t tile_first;   // the job's first rendered tile of its image tiling (a tile range)
    // rolling wavefront (the server): each job advances on its own.  step = the job's bounce
    // at this iteration (0: ray generation, 1..B: shade + spawn, B + 1: last shade + sum);
    // slot_tile = first tile of the job's slot range (slot = (slot_tile + t) m + i)
    uint32_t step;
    uint32_t slot_tile;
};

// Launch-uniform description of a pass.
struct PassArgs {
    const JobDev* jobs = nullptr;
    uint32_t n_jobs = 0;
    const SceneDev* scenes = nullptr;
    uint32_t tile_w = 0, tile_h = 0, m = 0, k = 0;
    uint32_t n_tiles = 0;  // tiles of all jobs of the pass
    uint32_t bounce = 0;   // shade: 1..B (B + 1 = final)
    uint32_t npx = 0;      // pixels of the debug capture (single-job renders)
    bool nee = false;      // some job of the plan uses next-event estimation
    // bit 0: a job's first sample writes its pixel sums without reading them (the buffer is
    // not cleared first); bit 1: its last sample writes the output instead of the sums
    uint32_t accum_mode = 0;
    // rolling wavefront: every kernel takes a slot's bounce from its job (JobDev::step), and
    // ray generation / the final sum run over launch lists: entry e covers job launch_job[e]
    // from unit launch_prefix[e] (tiles for ray generation, slots for the sum) on
    bool rolling = false;
    const uint32_t* launch_job = nullptr;
    const uint32_t* launch_prefix = nullptr;
    uint32_t n_launch = 0;
    uint32_t* queue_counts = nullptr;   // rolling ray generation: appends (rays, groups) here
    int32_t* ray_queue = nullptr;       //   ... its slots to this queue
    int32_t* group_queue_out = nullptr; //   ... and its groups to this one
};

// Per-call launch statistics.
struct LaunchCount {
    uint64_t n = 0;
};

// Saved traversal of a ray suspended by the two-phase trace (128 bytes).
struct TraceState {
    int node, sp, leaf, orig;
    float t;
    int pad[3];
    int stack[24];
};
// Buffers of the two-phase trace (per slot: state, flag; per queue entry: second queue).
struct PhaseBuffers {
    TraceState* state = nullptr;
    uint8_t* susp = nullptr;
    int32_t* queue2 = nullptr;
    uint32_t* count2 = nullptr;       // device count of queue2 (+ scratch words)
    uint32_t* block_counts = nullptr; // compaction scratch
    uint32_t budget = 32;
};
// Exclusive scan of per-block counts (column 0 of 2) into offsets; total -> *total.
void launch_scan_counts(uint32_t* block_counts, uint32_t n_blocks, uint32_t* total, cudaStream_t st);

// Arguments of one trace launch over a queue of slots.
struct TraceArgs {
    const float4* ray_o = nullptr; // slot-indexed (o.xyz, skip original index as int bits)
    const float4* ray_d = nullptr; // slot-indexed (d.xyz, tmax); tmax < 0: no ray
    const int32_t* queue = nullptr;     // slots to trace; NULL = slots [0, n_max)
    const uint32_t* queue_count = nullptr; // device count of queue entries (NULL: n_max)
    uint32_t n_max = 0;            // upper bound on the number of rays
    int2* hit = nullptr;           // slot-indexed (leaf triangle index or -1, t bits)
    const SceneDev* scenes = nullptr;  // scene table
    const uint16_t* slot_scene = nullptr; // per-slot scene index (NULL: scene 0)
    unsigned long long* counters = nullptr; // [0] node visits, [1] triangle tests (counting pass)
    uint32_t* work_counter = nullptr;       // persistent mode: atomic ray counter (zeroed)
    int block = 128;
    uint32_t refill = 0; // persistent mode: refill a warp's idle lanes when at least this many (0 = 8)
    bool persistent = false;
    bool speculative = false; // parked-leaf speculative traversal (BVH2)
    bool packet = false;      // warp-packet traversal (BVH2)
    bool any_hit = false;     // stop at the first hit before tmax (visibility)
    uint32_t stack = 16;      // BVH2 stack entries per thread in shared memory (8, 16, 32)
    bool two_phase = false;   // budgeted traversal, compaction of unfinished rays, resume (BVH2)
    PhaseBuffers phase;
    bool bvh8 = false;
    bool bvh4 = false; // closest hits through the BVH4 (any-hit queries stay on the BVH2)
};
void launch_trace(const TraceArgs& a, cudaStream_t st, LaunchCount& lc);
void launch_trace_bvh4(const TraceArgs& a, cudaStream_t st, LaunchCount& lc);
// Map leaf-order triangle indices of hits to original indices and split (prim, t).
void launch_hits_to_user(const float4* tris, const int2* hit, uint32_t n, int32_t* prim, float* t,
                         cudaStream_t st, LaunchCount& lc);

// ------------------------------------------------------------------------------------
// Wavefront path state, slot-indexed.  Slot = (tile of the pass) * m + sigma(i) (Sec. 3.3),
// so a reuse group's K members occupy K consecutive slots.
struct PathBuffers {
    uint32_t n_slots = 0, n_groups = 0;
    int32_t* pixel = nullptr;   // slot -> pixel of its job (-1: none)
    uint16_t* slot_job = nullptr;   // slot -> job of the pass
    uint16_t* slot_scene = nullptr; // slot -> scene table index
    float4* ray_o = nullptr;
    float4* ray_d = nullptr;
    int2* hit = nullptr;
    float4* beta = nullptr;     // throughput rgb, w unused
    float4* radiance = nullptr; // path radiance rgb
    uint8_t* alive = nullptr;   // 1 while the path continues
    int32_t* ray_queue = nullptr;   // alive slots in slot order
    int32_t* group_queue = nullptr; // groups with an alive member (2 x n_groups, double-buffered)
    // counts (kCountsWords words): [2] persistent work counter; [kQueueErrWord] queue
    // overflow flag; [8 + 2b], [8 + 2b + 1] ray and group queue lengths after the compaction
    // of bounce b (kQueueCountWords words, zeroed by raygen each pass); from word kStatWord, 64-bit
    // running totals of rays traced per bounce (index b); from kCounterWord, 64-bit node
    // visits and triangle tests of the counting pass.
    uint32_t* counts = nullptr;
    uint32_t* block_counts = nullptr; // compaction scratch (2 per block) + offsets
    // next-event estimation (allocated on first use): shadow ray origin|skip, direction|tmax
    // (w < 0: no shadow ray), unoccluded contribution rgb
    float4* shadow_o = nullptr;
    float4* shadow_d = nullptr;
    float4* shadow_c = nullptr;
    uint32_t n_blocks_cap = 0;
    // Morton sort
    uint32_t* keys = nullptr;   // 2 x n_slots
    int32_t* vals = nullptr;    // 2 x n_slots
    uint32_t* sort_hist = nullptr;
    uint32_t sort_hist_cap = 0;
    float4* accum = nullptr;    // per pixel of all jobs
    uint32_t n_px_cap = 0;
    unsigned long long* counters = nullptr; // counting pass
};

constexpr uint32_t kCountsWords = 256, kStatWord = 64, kCounterWord = 128, kShadowWord = 200;
constexpr uint32_t kQueueErrWord = 5, kQueueCountWords = kStatWord - 8;
// Shadow rays of the last shade (positions of its group queue): any-hit traversal, and the
// contribution of each unblocked one added to the path radiance.
void launch_shadow(const PassArgs& p, PathBuffers& b, bool first, bool bvh8, cudaStream_t st, LaunchCount& lc);
void launch_trace_bvh8(const TraceArgs& a, cudaStream_t st, LaunchCount& lc);
void launch_shadow_rays_bvh8(const SceneDev* scenes, const uint16_t* slot_scene, const float4* sh_o,
                             const float4* sh_d, const float4* sh_c, const int32_t* group_queue,
                             const uint32_t* group_count, uint32_t n_groups_max, uint32_t K, float4* radiance,
                             unsigned long long* n_traced, cudaStream_t st, LaunchCount& lc);
void launch_shadow_rays(const SceneDev* scenes, const uint16_t* slot_scene, const float4* sh_o, const float4* sh_d,
                        const float4* sh_c, const int32_t* group_queue, const uint32_t* group_count,
                        uint32_t n_groups_max, uint32_t K, float4* radiance, unsigned long long* n_traced, bool bvh8,
                        cudaStream_t st, LaunchCount& lc);

void launch_raygen(const PassArgs& p, PathBuffers& b, cudaStream_t st, LaunchCount& lc);
// raygen leaves the primary trace's visiting order (row-major pixels per tile) in the ray queue
bool primary_pixel_order();
// Shade the slots of the current group queue.  With `compact` the same launch appends the
// continuing slots and groups to the next ray and group queues (block ranges in completion
// order); without it launch_compact builds them in position order.
void launch_shade(const PassArgs& p, PathBuffers& b, bool first, bool compact, const cr_debug* dbg,
                  cudaStream_t st, LaunchCount& lc);
// Group-granular, order-preserving compaction (three launches) of the slots processed by the
// last shade into ray and group queues.
void launch_compact(const PassArgs& p, PathBuffers& b, bool first, cudaStream_t st, LaunchCount& lc);
const int32_t* launch_morton_sort(const PassArgs& p, PathBuffers& b, uint32_t bounce, uint32_t key_kind,
                                  cudaStream_t st, LaunchCount& lc);
uint32_t sort_hist_len(uint32_t n_slots);
int32_t* launch_sort_only(const uint32_t* key_in, const int32_t* val_in, uint32_t n, uint32_t* keys, int32_t* vals,
                          uint32_t* ws, uint32_t* count, uint32_t* err, cudaStream_t st, LaunchCount& lc);
uint32_t compact_blocks(uint32_t n_pos);
void launch_rays_from_user(const float* rays, const int32_t* skip, uint32_t n, float4* ray_o, float4* ray_d,
                           cudaStream_t st, LaunchCount& lc);
// End of a pass (bounce B + 1): the environment or emission where each live path's last ray
// ended, then every slot's radiance added to its pixel.
// Rolling wavefront (the server): the stages over jobs at different bounces.  parity selects
// the double-buffered group queue read at this iteration (the other one is appended to).
void launch_raygen_rolling(const PassArgs& p, PathBuffers& b, uint32_t n_tiles, cudaStream_t st, LaunchCount& lc);
void launch_shade_rolling(const PassArgs& p, PathBuffers& b, uint32_t parity, uint32_t n_groups_max,
                          cudaStream_t st, LaunchCount& lc);
void launch_shadow_rolling(const PassArgs& p, PathBuffers& b, uint32_t parity, uint32_t n_groups_max, bool bvh8,
                           cudaStream_t st, LaunchCount& lc);
void launch_finish_rolling(const PassArgs& p, PathBuffers& b, uint32_t n_slots, cudaStream_t st, LaunchCount& lc);
void launch_finish_accumulate(const PassArgs& p, PathBuffers& b, const cr_debug* dbg, cudaStream_t st,
                              LaunchCount& lc);
// out[job] = accum / spp for every job of the table (all pixels of all jobs, one launch).
void launch_output(const JobDev* jobs, uint32_t n_jobs, const float4* accum, uint32_t npx_total, cudaStream_t st,
                   LaunchCount& lc);
// out = accum[0, npx) * inv_spp for one job (accum already offset to the job's pixels).
void launch_output_one(const float4* accum, uint32_t npx, float inv_spp, float* out, cudaStream_t st, LaunchCount& lc);
void launch_groups(const CamBasis& cam, uint32_t tile_w, uint32_t tile_h, uint32_t interleave, uint64_t seed,
                   uint32_t frame, uint32_t* slot_of_pixel, cudaStream_t st, LaunchCount& lc);
void launch_philox(uint64_t seed, const uint32_t* ctr, uint32_t n, uint32_t* out, cudaStream_t st, LaunchCount& lc);
void launch_sample(uint32_t kind, uint32_t n, const float* wo, const float* u, const float* param, float* wi,
                   float* weight, uint8_t* valid, cudaStream_t st, LaunchCount& lc);

// Path-state allocation of a scene (single renders) or a batch.
struct Workspace {
    PathBuffers pb;
    void* base = nullptr;
    size_t bytes = 0;
    // shadow-ray buffers of next-event estimation, allocated on first use
    void* nee_base = nullptr;
    uint32_t nee_slots = 0;
    cr_status ensure_nee(uint32_t n_slots);
    // two-phase trace buffers, allocated on first use
    void* phase_base = nullptr;
    uint32_t phase_slots = 0;
    PhaseBuffers phase;
    cr_status ensure(uint32_t n_slots, uint32_t npx);
    cr_status ensure_phase(uint32_t n_slots);
    void release();
    ~Workspace() { release(); }
};
size_t workspace_bytes(uint32_t n_slots, uint32_t npx);

// A set of jobs sharing the tile shape, K, interleave and BVH layout, cut into sample
// passes: pass p renders sample p of every job with spp > p, all jobs in one wavefront.
struct PlanOpts {
    uint32_t tile_w = 8, tile_h = 8, k = 0, interleave = 1;
    bool bvh8 = false;
    bool bvh4 = false; // closest-hit traces through the BVH4 (single renders; shadow rays stay on the BVH2)
    uint32_t tile_begin = 0, tile_end = 0; // single-job plans: render only these tiles (0, 0 = all)
};
struct Pass {
    uint32_t job_offset = 0, n_jobs = 0, n_tiles = 0;
};
struct RenderPlan {
    uint32_t tile_w = 0, tile_h = 0, m = 0, k = 0;
    bool bvh8 = false, sort = false;
    bool bvh4 = false;
    bool nee = false; // some job uses next-event estimation
    uint32_t max_bounces = 0, max_slots = 0, npx_total = 0;
    std::vector<JobDev> jobs;     // all passes' tables, pass by pass
    std::vector<SceneDev> scenes; // scene table
    std::vector<Pass> passes;
};
// Device copies of a plan's tables.
struct Plan {
    JobDev* d_jobs = nullptr;
    SceneDev* d_scenes = nullptr;
    size_t cap_jobs = 0, cap_scenes = 0;
    cr_status upload(const RenderPlan& p, cudaStream_t st);
    void release();
    ~Plan() { release(); }
};
// Default trace block sizes (cr_render_opts.block = 0): 128 threads for the coherent primary
// rays, 64 for secondary rays (1.4% less secondary trace time on the landscape, 0.8% on the
// interior; primary rays are 0.5-1% faster in blocks of 128).
constexpr int kSecondaryBlock = 64;
struct ExecOpts {
    int block = 128;           // trace block size of the primary rays
    int block_secondary = 0;   // of the secondary rays (0: block)
    uint32_t stack = 16; // BVH2 traversal stack entries per thread in shared memory
    bool persistent = false, count = false, speculative = false;
    bool packet_primary = false, packet_secondary = false; // warp-packet traversal per ray kind
    uint32_t sort_key = 0; // reordering key of CR_MORTON_SORT (cr_sort_key)
    uint32_t phase_budget = 0; // two-phase secondary trace: node visits before suspension (0 = off)
    bool clear_accum = true; // zero the accumulation buffer first
    bool stats_traces_only = false; // stage events only around the trace launches
    bool write_output = true; // write every job's output after the last pass
    bool ordered_queues = false; // three-launch order-preserving compaction instead of appends
    const cr_debug* debug = nullptr;
    uint32_t debug_npx = 0;
};
struct StageTimes {
    double raygen = 0, trace_primary = 0, trace_secondary = 0, shade = 0, compact = 0, sort = 0, accum = 0;
    double trace_shadow = 0;
};
cr_status build_plan(const cr_job* jobs, uint32_t n_jobs, const PlanOpts& po, RenderPlan& plan);
JobDev job_dev(const cr_job& j, const PlanOpts& po, uint32_t scene_idx, uint32_t sample);
// CR_OK unless the queues of the run whose counts words these are overflowed (never expected)
cr_status queue_status(const uint64_t* host_counts);
cr_status check_job(const cr_job& j, uint32_t tile_w, uint32_t tile_h);
bool scene_has_bvh8(const cr_scene* s);
cr_status enqueue_plan(const RenderPlan& p, const Plan& dev, Workspace& ws, const ExecOpts& eo, cudaStream_t stream,
                       LaunchCount& lc, StageTimes* times);

// Thread-local message returned by cr_last_error(); handle -> device scene.
void set_last_error(const char* msg);
const DevScene* dev_scene_of(const cr_scene* s);
const SceneDev* dev_scene_entry(const cr_scene* s, bool bvh8); // device pointer
int scene_device(const cr_scene* s);                            // CUDA device of the scene's memory

} // namespace cr
