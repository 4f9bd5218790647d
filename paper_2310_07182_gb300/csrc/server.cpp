// server.cpp -- render request loop with continuous batching at bounce granularity.
//
// One host thread owns the device work and runs a rolling wavefront: every iteration is one
// launch per stage over the slots of all admitted jobs, whatever bounce each job is at.
// An iteration shades (each job's own step; the step after a job's last bounce only adds
// the end radiance), sums the samples of jobs that end one, generates the rays of jobs that
// start one, and traces every queued ray.  A job therefore joins at the next bounce launch
// after it is admitted, and leaves (its buffers free for others) right after its last sum.
// Each sample of a job in flight is a "run" with its own entry in the device job table
// (stable index, so slots keep pointing at it), which is how a job can end sample s and
// start sample s + 1 in the same iteration.  Admission is by device footprint: path-state
// slots (whole tiles), accumulation pixels and, for host outputs, staging pixels, each from
// a first-fit arena allocated once, so the loop allocates nothing.  The host enqueues up to
// kDepth iterations ahead of the GPU; events mark the iterations in which jobs complete.
//
// With an express lane (cr_server_opts.express_rays), small jobs run in a second wavefront
// with its own path state, job tables and queues, on a stream of the highest priority: a
// small job then takes one bounce step per iteration of its own lane, whose launches the
// GPU schedules ahead of the main lane's waiting blocks, instead of one step per iteration
// of the main lane (as long as the largest jobs' bounce).  Accumulation, staging and the
// scene table are shared; each lane has its own slots.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "cr_internal.h"

namespace cr {
namespace {

// path state per slot, with the 48 bytes of shadow-ray records (jobs may use CR_JOB_NEE)
constexpr uint64_t kSlotBytes = 4 + 2 + 2 + 16 + 16 + 8 + 16 + 16 + 1 + 4 + 8 + 8 + 8 + 48;
constexpr uint32_t kMaxRuns = 16384;   // device job-table entries (runs in flight)
constexpr uint32_t kMaxScenes = 256;   // distinct scenes the server may hold in its table
constexpr uint32_t kListWords = 4 * kMaxRuns; // launch lists: finish (job, prefix), raygen (job, prefix)
constexpr uint32_t kDepth = 4;        // iterations the host may enqueue ahead of the GPU (buffer sets)

struct SJob {
    uint64_t id = 0;
    cr_job job;
    bool host_out = false;
    float* d_out = nullptr;   // output on the device (user buffer or staging)
    uint32_t npx = 0, tiles = 0, slots = 0;
    uint64_t footprint = 0;
    uint32_t px_base = 0;     // in the accumulation arena
    uint32_t slot_tile = 0;   // first tile of its slot range
    uint32_t stg_at = 0;      // first pixel of its staging range (host outputs)
    uint32_t scene_idx = 0;
    uint32_t done = 0;        // samples summed
    uint32_t step = 0;        // bounce step of the current sample at the next iteration
    uint32_t run = 0;         // job-table entry of the current sample
    uint32_t lane = 0;        // 0 main, 1 express
    bool shared_freed = false; // its accumulation and staging ranges are back in the arenas
    uint64_t ray_steps = 0;   // pixels x spp x (max_bounces + 1)
    double t_submit = 0, t_admit = -1, t_done = -1;
    int state = 0;            // 0 queued, 1 active, 2 done, 3 failed, 4 waiting for its output
    cr_status status = CR_OK;
};

struct Arena { // first-fit ranges of units
    std::vector<std::pair<uint32_t, uint32_t>> free_; // (start, length), sorted by start
    void init(uint32_t n) { free_.assign(1, {0u, n}); }
    bool alloc(uint32_t n, uint32_t& at) {
        if (n == 0) {
            at = 0;
            return true;
        }
        for (size_t i = 0; i < free_.size(); ++i)
            if (free_[i].second >= n) {
                at = free_[i].first;
                free_[i].first += n;
                free_[i].second -= n;
                if (free_[i].second == 0) free_.erase(free_.begin() + i);
                return true;
            }
        return false;
    }
    void release(uint32_t at, uint32_t n) {
        if (n == 0) return;
        auto it = std::lower_bound(free_.begin(), free_.end(), std::make_pair(at, 0u));
        it = free_.insert(it, {at, n});
        size_t i = it - free_.begin();
        if (i + 1 < free_.size() && free_[i].first + free_[i].second == free_[i + 1].first) {
            free_[i].second += free_[i + 1].second;
            free_.erase(free_.begin() + i + 1);
        }
        if (i > 0 && free_[i - 1].first + free_[i - 1].second == free_[i].first) {
            free_[i - 1].second += free_[i].second;
            free_.erase(free_.begin() + i);
        }
    }
};

// One rolling wavefront: its stream, path state, device job tables and launch lists (kDepth
// sets used round robin by the iterations in flight) with their pinned host sources, and
// the jobs it runs.
struct Lane {
    cudaStream_t stream = nullptr;
    cudaStream_t copy_stream = nullptr; // job-table uploads, off the render stream
    Workspace ws;
    JobDev* d_table[kDepth] = {};
    uint32_t* d_lists[kDepth] = {};
    JobDev* h_table[kDepth] = {};
    uint32_t* h_lists[kDepth] = {};
    uint64_t* h_counts = nullptr; // pinned: (rays traced at bounces >= 1, queue error word)
    cudaEvent_t ev_iter[kDepth] = {};
    cudaEvent_t ev_copied[kDepth] = {};
    bool ev_used[kDepth] = {};
    std::deque<std::pair<cudaEvent_t, std::vector<uint64_t>>> pending; // completion events
    Arena tile_alloc;
    uint32_t tiles_cap = 0;
    std::vector<uint32_t> free_runs;
    std::vector<uint64_t> active;
    uint64_t iter = 0;
    uint64_t rays = 0; // last read of the lane's ray counter

    // streams (of the given priority), tables, lists and events; the path state for `tiles`
    // whole tiles of m slots is allocated separately (Workspace, a cr_status)
    cudaError_t create(uint32_t tiles, int priority) {
        tiles_cap = tiles;
        tile_alloc.init(tiles);
        for (uint32_t i = kMaxRuns; i-- > 0;) free_runs.push_back(i);
        cudaError_t e = cudaStreamCreateWithPriority(&stream, cudaStreamNonBlocking, priority);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&copy_stream, cudaStreamNonBlocking, priority);
        for (uint32_t p = 0; p < kDepth && e == cudaSuccess; ++p) {
            e = cudaMalloc(&d_table[p], sizeof(JobDev) * kMaxRuns);
            if (e == cudaSuccess) e = cudaMalloc(&d_lists[p], 4ull * kListWords);
            if (e == cudaSuccess) e = cudaMallocHost(&h_table[p], sizeof(JobDev) * kMaxRuns);
            if (e == cudaSuccess) e = cudaMallocHost(&h_lists[p], 4ull * kListWords);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_iter[p], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_copied[p], cudaEventDisableTiming);
        }
        if (e == cudaSuccess) e = cudaMallocHost(&h_counts, 2 * sizeof(uint64_t));
        if (e == cudaSuccess) std::memset(h_counts, 0, 2 * sizeof(uint64_t));
        return e;
    }
    // after the streams are drained; frees whatever create allocated
    void destroy() {
        for (auto& pe : pending) cudaEventDestroy(pe.first);
        pending.clear();
        for (uint32_t p = 0; p < kDepth; ++p) {
            if (d_table[p]) cudaFree(d_table[p]);
            if (d_lists[p]) cudaFree(d_lists[p]);
            if (h_table[p]) cudaFreeHost(h_table[p]);
            if (h_lists[p]) cudaFreeHost(h_lists[p]);
            if (ev_iter[p]) cudaEventDestroy(ev_iter[p]);
            if (ev_copied[p]) cudaEventDestroy(ev_copied[p]);
        }
        if (h_counts) cudaFreeHost(h_counts);
        ws.release();
        if (stream) cudaStreamDestroy(stream);
        if (copy_stream) cudaStreamDestroy(copy_stream);
    }
    // the next iteration's buffer set is free (the iteration kDepth before it has completed)
    bool ready() const {
        const uint32_t set = (uint32_t)(iter % kDepth);
        return !ev_used[set] || cudaEventQuery(ev_iter[set]) != cudaErrorNotReady;
    }
};

} // namespace
} // namespace cr

using namespace cr;

struct cr_server {
    cr_server_opts opts;
    PlanOpts po;
    ExecOpts eo;
    int device = 0;
    Lane lanes[2];            // 0 main, 1 express (used when opts.express_rays != 0)
    uint32_t n_lanes = 1;
    SceneDev* d_scenes = nullptr;
    std::vector<cudaEvent_t> event_pool;
    float4* arena = nullptr;  // accumulation (16 B per pixel)
    uint32_t arena_px = 0;
    float* staging = nullptr; // host-output staging (12 B per pixel)
    uint32_t staging_px = 0;
    Arena alloc, stg_alloc;
    std::vector<const cr_scene*> scene_list;
    bool scenes_dirty = false;
    uint64_t budget = 0, used = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> queue;
    std::map<uint64_t, SJob> jobs;
    uint64_t next_id = 1;
    bool stop = false;
    cr_status fatal = CR_OK;
    std::string fatal_msg;
    std::thread th;
    std::chrono::steady_clock::time_point t0;
    cr_server_stats stats;

    double now_ms() const {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    void loop();
    void admit_locked();
    bool admit_to_locked(SJob& j, uint32_t lane);
    bool poll_completions(Lane& L, bool wait_oldest);
    void release_job_locked(SJob& j);
    bool iterate(Lane& L, LaunchCount& lc);
    size_t active_count() const { return lanes[0].active.size() + lanes[1].active.size(); }
};

// Admit queued jobs (in arrival order, later ones may backfill) while their slots,
// accumulation and staging ranges and a job-table entry fit.  A job of at most express_rays
// ray steps tries the express lane first, then the main one.  Called with the lock held.
void cr_server::admit_locked() {
    for (auto it = queue.begin(); it != queue.end();) {
        SJob& j = jobs[*it];
        uint32_t scene_idx = 0;
        while (scene_idx < scene_list.size() && scene_list[scene_idx] != j.job.scene) ++scene_idx;
        if (scene_idx == scene_list.size() && scene_list.size() >= kMaxScenes) {
            ++it; // the scene table is full: wait until it can be rebuilt
            continue;
        }
        const bool express = n_lanes > 1 && j.ray_steps <= opts.express_rays;
        if (!(express && admit_to_locked(j, 1)) && !admit_to_locked(j, 0)) {
            ++it;
            continue;
        }
        if (scene_idx == scene_list.size()) {
            scene_list.push_back(j.job.scene);
            scenes_dirty = true;
        }
        j.scene_idx = scene_idx;
        j.step = 0;
        j.done = 0;
        j.state = 1;
        j.t_admit = now_ms();
        used += j.footprint;
        lanes[j.lane].active.push_back(j.id);
        it = queue.erase(it);
    }
}

// Take the job's slot tiles in `lane`, its accumulation and staging ranges and a job-table
// entry, or nothing.
bool cr_server::admit_to_locked(SJob& j, uint32_t lane) {
    Lane& L = lanes[lane];
    uint32_t st = 0, px = 0, sg = 0;
    // at most half the job table is held by active jobs: a job that ends a sample takes a
    // second entry for its next one in the same iteration
    if (L.active.size() >= kMaxRuns / 2 || !L.tile_alloc.alloc(j.tiles, st)) return false;
    if (!alloc.alloc(j.npx, px)) {
        L.tile_alloc.release(st, j.tiles);
        return false;
    }
    if (j.host_out && !stg_alloc.alloc(j.npx, sg)) {
        L.tile_alloc.release(st, j.tiles);
        alloc.release(px, j.npx);
        return false;
    }
    j.lane = lane;
    j.slot_tile = st;
    j.px_base = px;
    j.stg_at = sg;
    if (j.host_out) j.d_out = staging + 3ull * sg;
    j.run = L.free_runs.back();
    L.free_runs.pop_back();
    return true;
}

// Free a job's slots and job-table entry once its last sum is enqueued: later iterations on
// its lane's stream run after that sum (and its output copy), so they can go to other jobs
// of the lane at once.  The accumulation and staging ranges are shared by the lanes; with
// one lane they are freed here too, with two only when the job's completion event has
// passed (release_shared_locked), since the other lane's stream is not ordered after it.
void cr_server::release_job_locked(SJob& j) {
    Lane& L = lanes[j.lane];
    L.tile_alloc.release(j.slot_tile, j.tiles);
    L.free_runs.push_back(j.run);
    if (n_lanes == 1) { // one stream: every later launch is ordered after the job's last sum
        alloc.release(j.px_base, j.npx);
        if (j.host_out) stg_alloc.release(j.stg_at, j.npx);
        used -= j.footprint;
        j.shared_freed = true;
    }
}

// Ranges of the shared arenas a completed job still holds (two lanes: freed on completion).
static void release_shared_locked(cr_server& s, SJob& j) {
    if (j.shared_freed) return;
    s.alloc.release(j.px_base, j.npx);
    if (j.host_out) s.stg_alloc.release(j.stg_at, j.npx);
    s.used -= j.footprint;
    j.shared_freed = true;
}

// Mark the jobs of the lane's completed iterations done (their outputs are where the caller
// asked).  Returns true if an event was retired.
bool cr_server::poll_completions(Lane& L, bool wait_oldest) {
    bool any = false;
    while (true) {
        cudaEvent_t ev = nullptr;
        {
            std::lock_guard<std::mutex> lk(mu);
            if (L.pending.empty()) return any;
            ev = L.pending.front().first;
        }
        cudaError_t e = wait_oldest ? cudaEventSynchronize(ev) : cudaEventQuery(ev);
        wait_oldest = false;
        if (e == cudaErrorNotReady) return any;
        any = true;
        std::vector<uint64_t> ids;
        {
            std::lock_guard<std::mutex> lk(mu);
            ids = std::move(L.pending.front().second);
            L.pending.pop_front();
            event_pool.push_back(ev);
            const double t = now_ms();
            for (uint64_t id : ids) {
                auto it = jobs.find(id);
                if (it == jobs.end()) continue;
                release_shared_locked(*this, it->second);
                if (e == cudaSuccess) {
                    it->second.state = 2;
                } else {
                    it->second.state = 3;
                    it->second.status = CR_ERR_CUDA;
                }
                it->second.t_done = t;
                stats.jobs_done++;
            }
            if (e != cudaSuccess && fatal == CR_OK) {
                cudaGetLastError();
                fatal = CR_ERR_CUDA;
                fatal_msg = cudaGetErrorString(e);
            }
        }
        cv_done.notify_all();
    }
}

// One iteration of the rolling wavefront: shade (every job at its own step), sum the samples
// that end, generate the rays of the samples that start, trace every queued ray.  Returns
// false when no job is active.
bool cr_server::iterate(Lane& L, LaunchCount& lc) {
    const uint32_t par = (uint32_t)(L.iter & 1u);            // group queue read at this iteration
    const uint32_t set = (uint32_t)(L.iter % kDepth);        // table, lists and counters of this iteration
    if (L.ev_used[set]) cudaEventSynchronize(L.ev_iter[set]); // iteration iter - kDepth freed this set
    const uint32_t m = po.tile_w * po.tile_h, K = po.k ? po.k : m;
    JobDev* tab = L.h_table[set];
    uint32_t* fin_job = L.h_lists[set];
    uint32_t* fin_pre = fin_job + kMaxRuns;
    uint32_t* st_job = fin_job + 2 * kMaxRuns;
    uint32_t* st_pre = fin_job + 3 * kMaxRuns;
    uint32_t n_fin = 0, n_start = 0, fin_slots = 0, start_tiles = 0, n_groups = 0, trace_max = 0, max_run = 0;
    bool nee = false, sort = false, upload_scenes = false;
    std::vector<SceneDev> scene_tab;
    std::vector<uint64_t> completing, host_copies;
    std::map<uint64_t, uint32_t> next_run;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (L.ev_used[set] && set == 0) { // what iteration iter - kDepth read back
            L.rays = std::max<uint64_t>(L.rays, L.h_counts[0]);
            stats.secondary_rays = lanes[0].rays + lanes[1].rays;
            const uint32_t err = (uint32_t)L.h_counts[1];
            if (err != 0u && fatal == CR_OK) {
                fatal = (err & 2u) ? CR_ERR_TIMEOUT : CR_ERR_CUDA;
                fatal_msg = (err & 2u) ? "a ray-sort wait ran out" : "a ray or group queue overflowed";
            }
        }
        if (fatal != CR_OK) { // fail what is left
            for (uint64_t id : L.active) {
                SJob& j = jobs[id];
                j.state = 3;
                j.status = fatal;
                j.t_done = now_ms();
                release_job_locked(j);
            }
            L.active.clear();
            cv_done.notify_all();
            return false;
        }
        if (L.active.empty()) return false;
        if (scenes_dirty) {
            for (const cr_scene* sc : scene_list) scene_tab.push_back(scene_entry(*dev_scene_of(sc), po.bvh8));
            scenes_dirty = false;
            upload_scenes = true;
        }
        for (uint64_t id : L.active) {
            SJob& j = jobs[id];
            const uint32_t B = j.job.max_bounces;
            JobDev d = job_dev(j.job, po, j.scene_idx, j.done);
            d.out = j.d_out;
            d.px_base = j.px_base;
            d.slot_tile = j.slot_tile;
            d.step = j.step;
            tab[j.run] = d;
            max_run = std::max(max_run, j.run);
            nee = nee || d.nee;
            sort = sort || j.job.mode == CR_MORTON_SORT;
            if (j.step >= 1) n_groups += j.slots / K; // its groups may be in the queue read now
            if (j.step == 0) {
                st_job[n_start] = j.run;
                st_pre[n_start++] = start_tiles;
                start_tiles += j.tiles;
                trace_max += j.slots;
            } else if (j.step <= B) {
                trace_max += j.slots;
            } else { // the sample ends here: its sum, and the next sample starts at once
                fin_job[n_fin] = j.run;
                fin_pre[n_fin++] = fin_slots;
                fin_slots += j.slots;
                if (j.done + 1 < j.job.spp) {
                    const uint32_t nr = L.free_runs.back();
                    L.free_runs.pop_back();
                    JobDev d2 = job_dev(j.job, po, j.scene_idx, j.done + 1);
                    d2.out = j.d_out;
                    d2.px_base = j.px_base;
                    d2.slot_tile = j.slot_tile;
                    d2.step = 0;
                    tab[nr] = d2;
                    max_run = std::max(max_run, nr);
                    st_job[n_start] = nr;
                    st_pre[n_start++] = start_tiles;
                    start_tiles += j.tiles;
                    trace_max += j.slots;
                    next_run[id] = nr;
                } else {
                    completing.push_back(id);
                    if (j.host_out) host_copies.push_back(id);
                }
            }
        }
    }
    PathBuffers& b = L.ws.pb;
    b.n_groups = b.n_slots / K;
    b.accum = arena;
    // the uploads run on the lane's copy stream (this set's device buffers were last read by
    // iteration iter - kDepth, which has completed), overlapping the iterations in flight;
    // the render stream waits for them before this iteration's first launch
    cudaMemcpyAsync(L.d_table[set], tab, sizeof(JobDev) * (max_run + 1), cudaMemcpyHostToDevice, L.copy_stream);
    if (n_fin) {
        cudaMemcpyAsync(L.d_lists[set], fin_job, 4ull * n_fin, cudaMemcpyHostToDevice, L.copy_stream);
        cudaMemcpyAsync(L.d_lists[set] + kMaxRuns, fin_pre, 4ull * n_fin, cudaMemcpyHostToDevice, L.copy_stream);
    }
    if (n_start) {
        cudaMemcpyAsync(L.d_lists[set] + 2 * kMaxRuns, st_job, 4ull * n_start, cudaMemcpyHostToDevice, L.copy_stream);
        cudaMemcpyAsync(L.d_lists[set] + 3 * kMaxRuns, st_pre, 4ull * n_start, cudaMemcpyHostToDevice, L.copy_stream);
    }
    cudaEventRecord(L.ev_copied[set], L.copy_stream);
    cudaStreamWaitEvent(L.stream, L.ev_copied[set], 0);
    if (upload_scenes) // append-only: entries in-flight iterations read do not change
        cudaMemcpy(d_scenes, scene_tab.data(), sizeof(SceneDev) * scene_tab.size(), cudaMemcpyHostToDevice);
    PassArgs P;
    P.jobs = L.d_table[set];
    P.n_jobs = max_run + 1;
    P.scenes = d_scenes;
    P.tile_w = po.tile_w;
    P.tile_h = po.tile_h;
    P.m = m;
    P.k = K;
    P.nee = nee;
    P.rolling = true;
    P.accum_mode = 3u;
    uint32_t* qn = b.counts + 8 + 2 * (par ^ 1u); // (rays, groups) appended for the next iteration
    cudaMemsetAsync(qn, 0, 8, L.stream);
    launch_shade_rolling(P, b, par, n_groups, L.stream, lc);
    launch_shadow_rolling(P, b, par, n_groups, po.bvh8, L.stream, lc);
    if (n_fin) {
        P.launch_job = L.d_lists[set];
        P.launch_prefix = L.d_lists[set] + kMaxRuns;
        P.n_launch = n_fin;
        launch_finish_rolling(P, b, fin_slots, L.stream, lc);
    }
    {
        std::lock_guard<std::mutex> lk(mu);
        for (uint64_t id : host_copies) {
            SJob& j = jobs[id];
            cudaMemcpyAsync(j.job.out_rgb, j.d_out, 12ull * j.npx, cudaMemcpyDeviceToHost, L.stream);
        }
    }
    if (n_start) {
        P.launch_job = L.d_lists[set] + 2 * kMaxRuns;
        P.launch_prefix = L.d_lists[set] + 3 * kMaxRuns;
        P.n_launch = n_start;
        P.queue_counts = qn;
        P.ray_queue = b.ray_queue;
        P.group_queue_out = b.group_queue + (size_t)(par ^ 1u) * b.n_groups;
        launch_raygen_rolling(P, b, start_tiles, L.stream, lc);
    }
    if (trace_max) {
        TraceArgs ta;
        ta.ray_o = b.ray_o;
        ta.ray_d = b.ray_d;
        ta.hit = b.hit;
        ta.block = eo.block_secondary ? eo.block_secondary : eo.block;
        ta.stack = eo.stack;
        ta.bvh8 = po.bvh8;
        ta.scenes = d_scenes;
        ta.slot_scene = b.slot_scene;
        ta.queue = b.ray_queue;
        ta.queue_count = qn;
        ta.n_max = trace_max;
        if (sort) ta.queue = launch_morton_sort(P, b, par ^ 1u, eo.sort_key, L.stream, lc);
        launch_trace(ta, L.stream, lc);
    }
    // the ray total and the error word, read back every kDepth-th iteration (the copies
    // would otherwise sit between the kernels of consecutive iterations)
    if (set == 0) {
        cudaMemcpyAsync(&L.h_counts[0], reinterpret_cast<unsigned long long*>(b.counts + kStatWord) + 1, 8,
                        cudaMemcpyDeviceToHost, L.stream);
        cudaMemcpyAsync(&L.h_counts[1], b.counts + kQueueErrWord, 4, cudaMemcpyDeviceToHost, L.stream);
    }
    cudaEventRecord(L.ev_iter[set], L.stream);
    L.ev_used[set] = true;
    cudaError_t e = cudaGetLastError();
    std::lock_guard<std::mutex> lk(mu);
    if (e != cudaSuccess && fatal == CR_OK) {
        fatal = CR_ERR_CUDA;
        fatal_msg = cudaGetErrorString(e);
    }
    if (!completing.empty()) {
        cudaEvent_t ev = nullptr;
        if (!event_pool.empty()) {
            ev = event_pool.back();
            event_pool.pop_back();
        } else {
            cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        }
        cudaEventRecord(ev, L.stream);
        L.pending.push_back({ev, completing});
    }
    // advance every job by one bounce step
    std::vector<uint64_t> keep;
    for (uint64_t id : L.active) {
        SJob& j = jobs[id];
        if (j.step <= j.job.max_bounces) {
            j.step++;
            keep.push_back(id);
            continue;
        }
        j.done++;
        auto nr = next_run.find(id);
        if (nr != next_run.end()) {
            L.free_runs.push_back(j.run);
            j.run = nr->second;
            j.step = 1;
            keep.push_back(id);
        } else {
            j.state = 4; // done on the device once its completion event has passed
            release_job_locked(j);
        }
    }
    L.active.swap(keep);
    stats.passes++;
    stats.kernel_launches = lc.n;
    L.iter++;
    return true;
}

// The host thread: admit, then enqueue one iteration of every lane whose next buffer set is
// free (the express lane first); when no lane can take one, wait briefly (or, with nothing
// active, for the oldest completion).
void cr_server::loop() {
    cudaSetDevice(device);
    LaunchCount lc;
    while (true) {
        for (uint32_t l = 0; l < n_lanes; ++l) poll_completions(lanes[l], false);
        bool any_active = false, any_pending = false;
        {
            std::unique_lock<std::mutex> lk(mu);
            if (stop) break;
            if (fatal == CR_OK) admit_locked();
            for (uint32_t l = 0; l < n_lanes; ++l) {
                any_active = any_active || !lanes[l].active.empty();
                any_pending = any_pending || !lanes[l].pending.empty();
            }
            if (!any_active && !any_pending) {
                cv_work.wait_for(lk, std::chrono::milliseconds(5));
                continue;
            }
        }
        if (!any_active) { // nothing to launch: wait for the oldest completion of a lane
            for (uint32_t l = n_lanes; l-- > 0;)
                if (poll_completions(lanes[l], true)) break;
            continue;
        }
        bool launched = false;
        for (uint32_t l = n_lanes; l-- > 0;) { // express lane (1) first
            Lane& L = lanes[l];
            bool has;
            {
                std::lock_guard<std::mutex> lk(mu);
                has = !L.active.empty();
            }
            if (!has || (n_lanes > 1 && !L.ready())) continue;
            const double tb = now_ms();
            launched = iterate(L, lc) || launched;
            std::lock_guard<std::mutex> lk(mu);
            stats.busy_ms += now_ms() - tb;
        }
        if (!launched) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

extern "C" cr_status cr_server_create(const cr_server_opts* o, cr_server** out) {
    set_last_error("");
    if (!o || !out) {
        set_last_error("cr_server_create: NULL argument");
        return CR_ERR_INVALID_ARG;
    }
    *out = nullptr;
    const uint32_t m = o->group_w * o->group_h;
    const uint32_t K = o->k ? o->k : m;
    if (!o->group_w || !o->group_h || (m & (m - 1)) || m > 1024 || o->hbm_budget < (64ull << 20) || (K & (K - 1)) ||
        m % K != 0 || K > 256) {
        set_last_error("cr_server_create: bad tile shape or K, or budget below 64 MiB");
        return CR_ERR_INVALID_ARG;
    }
    std::unique_ptr<cr_server> s(new (std::nothrow) cr_server());
    if (!s) return CR_ERR_OOM;
    s->opts = *o;
    s->po.tile_w = o->group_w;
    s->po.tile_h = o->group_h;
    s->po.k = o->k;
    s->po.interleave = o->interleave;
    s->po.bvh8 = o->bvh == CR_BVH8Q;
    s->eo.block = o->block ? (int)o->block : 128;
    s->eo.block_secondary = o->block ? (int)o->block : kSecondaryBlock;
    s->budget = o->hbm_budget;
    s->n_lanes = o->express_rays ? 2u : 1u;
    // the budget is split once: 60% path state (whole tiles of slots; an express lane takes
    // 1/8 of them), 25% the accumulation arena (16 B per pixel of every admitted job), 15%
    // output staging for jobs with host outputs (12 B per pixel)
    const uint64_t slots = std::min<uint64_t>(o->hbm_budget * 6 / 10 / kSlotBytes, 1ull << 27);
    const uint32_t tiles = (uint32_t)(slots / m);
    const uint32_t tiles_express = s->n_lanes > 1 ? tiles / 8 : 0u;
    if (tiles_express == 0) s->n_lanes = 1; // a budget too small to split
    s->arena_px = (uint32_t)std::min<uint64_t>(o->hbm_budget / 4 / 16, 1ull << 28);
    s->staging_px = (uint32_t)std::min<uint64_t>(o->hbm_budget * 15 / 100 / 12, 1ull << 28);
    cudaGetDevice(&s->device);
    cr_server* r = s.get();
    auto cleanup = [r]() { // releases whatever was allocated before a failure
        for (Lane& L : r->lanes) L.destroy();
        if (r->d_scenes) cudaFree(r->d_scenes);
        if (r->arena) cudaFree(r->arena);
        if (r->staging) cudaFree(r->staging);
    };
    int lo_pri = 0, hi_pri = 0; // numerically lower is the higher priority
    cudaDeviceGetStreamPriorityRange(&lo_pri, &hi_pri);
    cudaError_t e = r->lanes[0].create(tiles - tiles_express, lo_pri);
    if (e == cudaSuccess && r->n_lanes > 1) e = r->lanes[1].create(tiles_express, hi_pri);
    if (e == cudaSuccess) e = cudaMalloc(&r->arena, 16ull * r->arena_px);
    if (e == cudaSuccess) e = cudaMalloc(&r->staging, 12ull * r->staging_px);
    if (e == cudaSuccess) e = cudaMalloc(&r->d_scenes, sizeof(SceneDev) * kMaxScenes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_last_error("cr_server_create: device allocation failed");
        cleanup();
        return e == cudaErrorMemoryAllocation ? CR_ERR_OOM : CR_ERR_CUDA;
    }
    cr_status st = CR_OK;
    for (uint32_t l = 0; l < r->n_lanes && st == CR_OK; ++l) {
        Workspace& ws = r->lanes[l].ws;
        st = ws.ensure(r->lanes[l].tiles_cap * m, 1);
        if (st == CR_OK) st = ws.ensure_nee(r->lanes[l].tiles_cap * m);
        if (st == CR_OK && cudaMemset(ws.pb.counts, 0, 4 * kCountsWords) != cudaSuccess) {
            cudaGetLastError();
            set_last_error("cr_server_create: clearing the counters failed");
            st = CR_ERR_CUDA;
        }
    }
    if (st != CR_OK) {
        cleanup();
        return st;
    }
    r->alloc.init(r->arena_px);
    r->stg_alloc.init(r->staging_px);
    std::memset(&r->stats, 0, sizeof(r->stats));
    r->t0 = std::chrono::steady_clock::now();
    r->th = std::thread([r] { r->loop(); });
    *out = s.release();
    return CR_OK;
}

extern "C" cr_status cr_server_submit(cr_server* s, const cr_job* job, uint64_t* id) {
    set_last_error("");
    if (!s || !job || !id) {
        set_last_error("cr_server_submit: NULL argument");
        return CR_ERR_INVALID_ARG;
    }
    if (!job->out_rgb) {
        set_last_error("cr_server_submit: out_rgb is NULL");
        return CR_ERR_INVALID_ARG;
    }
    cr_status cst = check_job(*job, s->po.tile_w, s->po.tile_h);
    if (cst != CR_OK) return cst;
    if (s->po.bvh8 && !scene_has_bvh8(job->scene)) {
        set_last_error("cr_server_submit: the server traverses BVH8-Q but the job's scene has none");
        return CR_ERR_INVALID_ARG;
    }
    SJob j;
    j.job = *job;
    cudaPointerAttributes a;
    j.host_out = !(cudaPointerGetAttributes(&a, job->out_rgb) == cudaSuccess &&
                   (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged));
    cudaGetLastError();
    if (!j.host_out) j.d_out = job->out_rgb;
    j.npx = job->camera.width * job->camera.height;
    const uint32_t m = s->po.tile_w * s->po.tile_h;
    const uint32_t tx = (job->camera.width + s->po.tile_w - 1) / s->po.tile_w;
    const uint32_t ty = (job->camera.height + s->po.tile_h - 1) / s->po.tile_h;
    j.tiles = tx * ty;
    j.slots = j.tiles * m;
    j.footprint = 16ull * j.npx + (j.host_out ? 12ull * j.npx : 0) + kSlotBytes * j.slots;
    j.ray_steps = (uint64_t)j.npx * job->spp * (job->max_bounces + 1ull);
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->fatal != CR_OK) {
        set_last_error("cr_server_submit: the server stopped after a device error");
        return s->fatal;
    }
    if (j.tiles > s->lanes[0].tiles_cap || j.npx > s->arena_px || (j.host_out && j.npx > s->staging_px)) {
        set_last_error("cr_server_submit: job larger than the server's device budget");
        return CR_ERR_OOM;
    }
    j.id = s->next_id++;
    j.t_submit = s->now_ms();
    *id = j.id;
    s->jobs[j.id] = j;
    s->queue.push_back(j.id);
    s->stats.jobs_submitted++;
    s->cv_work.notify_one();
    return CR_OK;
}

static cr_status fill_job_stats(const SJob& j, cr_job_stats* js) {
    if (js) {
        js->t_submit_ms = j.t_submit;
        js->t_admit_ms = j.t_admit;
        js->t_done_ms = j.t_done;
        js->latency_ms = j.t_done - j.t_submit;
        js->samples = j.done;
        js->footprint_bytes = j.footprint;
    }
    return j.state == 2 ? CR_OK : j.status;
}

static bool finished(const SJob& j) { return j.state == 2 || j.state == 3; }

extern "C" cr_status cr_server_poll(cr_server* s, uint64_t id, cr_job_stats* js) {
    set_last_error("");
    if (!s) return CR_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(id);
    if (it == s->jobs.end()) return CR_ERR_NOT_FOUND;
    if (!finished(it->second)) return CR_ERR_BUSY;
    cr_status st = fill_job_stats(it->second, js);
    s->jobs.erase(it);
    return st;
}

extern "C" cr_status cr_server_wait(cr_server* s, uint64_t id, uint32_t timeout_ms, cr_job_stats* js) {
    set_last_error("");
    if (!s) return CR_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto done = [&] {
        auto it = s->jobs.find(id);
        return it == s->jobs.end() || finished(it->second);
    };
    if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) return CR_ERR_TIMEOUT;
    auto it = s->jobs.find(id);
    if (it == s->jobs.end()) return CR_ERR_NOT_FOUND;
    cr_status st = fill_job_stats(it->second, js);
    s->jobs.erase(it);
    return st;
}

extern "C" cr_status cr_server_get_stats(cr_server* s, cr_server_stats* out) {
    if (!s || !out) return CR_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    out->queued = (uint32_t)s->queue.size();
    out->active = (uint32_t)s->active_count();
    out->used_bytes = s->used;
    return CR_OK;
}

extern "C" cr_status cr_server_destroy(cr_server* s) {
    if (!s) return CR_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->th.joinable()) s->th.join();
    for (Lane& L : s->lanes) {
        if (L.stream) cudaStreamSynchronize(L.stream);
        if (L.copy_stream) cudaStreamSynchronize(L.copy_stream);
    }
    for (Lane& L : s->lanes) L.destroy();
    for (cudaEvent_t ev : s->event_pool) cudaEventDestroy(ev);
    cudaFree(s->d_scenes);
    cudaFree(s->arena);
    cudaFree(s->staging);
    delete s;
    return CR_OK;
}
