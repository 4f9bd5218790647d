// server.cpp -- render request loop with continuous batching.
//
// One host thread owns the device work.  Each iteration renders ONE sample pass of every
// active job as a single merged wavefront (one launch per stage per bounce over the slots
// of all jobs).  Between passes it retires jobs whose last sample is done (output, copy to
// the host if needed, completion time) and admits queued jobs while their device
// footprint fits the budget, so requests that arrive while others are on the GPU join the
// next pass.  Accumulations live in one arena with a first-fit allocator, so jobs keep
// their partial sums while others come and go.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "cr_internal.h"

namespace cr {
namespace {

// path state per slot, with the 48 bytes of shadow-ray records (jobs may use CR_JOB_NEE)
constexpr uint64_t kSlotBytes = 4 + 2 + 2 + 16 + 16 + 8 + 16 + 16 + 1 + 4 + 8 + 8 + 8 + 48;

struct SJob {
    uint64_t id = 0;
    cr_job job;
    bool host_out = false;
    float* d_out = nullptr;   // output on the device (user buffer or staging)
    uint32_t npx = 0, slots = 0;
    uint64_t footprint = 0;
    uint32_t px_base = 0;     // in the accumulation arena
    uint32_t done = 0;        // samples accumulated
    double t_submit = 0, t_admit = -1, t_done = -1;
    int state = 0;            // 0 queued, 1 active, 2 done, 3 failed
    cr_status status = CR_OK;
};

struct Arena { // first-fit ranges of float4 pixels
    std::vector<std::pair<uint32_t, uint32_t>> free_; // (start, length), sorted by start
    void init(uint32_t n) { free_.assign(1, {0u, n}); }
    bool alloc(uint32_t n, uint32_t& at) {
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

} // namespace
} // namespace cr

using namespace cr;

struct cr_server {
    cr_server_opts opts;
    PlanOpts po;
    ExecOpts eo;
    int device = 0;
    cudaStream_t stream = nullptr;
    Workspace ws;
    Plan dev;
    float4* arena = nullptr;
    uint32_t arena_px = 0;
    Arena alloc;
    uint32_t slots_cap = 0, slots_used = 0;
    uint64_t budget = 0, used = 0;
    uint64_t staging_cap = 0, staging_used = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> queue;
    std::map<uint64_t, SJob> jobs;
    std::vector<uint64_t> active;
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
    bool admit_locked();
};

// Admit queued jobs (in arrival order, later ones may backfill) while they fit.  Returns
// true if anything is active.  Called with the lock held.
bool cr_server::admit_locked() {
    for (auto it = queue.begin(); it != queue.end();) {
        SJob& j = jobs[*it];
        const uint64_t stg = j.host_out ? 12ull * j.npx : 0;
        const bool fits = slots_used + j.slots <= slots_cap && staging_used + stg <= staging_cap;
        uint32_t at = 0;
        if (fits && alloc.alloc(j.npx, at)) {
            if (j.host_out) {
                if (cudaMalloc(&j.d_out, 12ull * j.npx) != cudaSuccess) {
                    cudaGetLastError();
                    alloc.release(at, j.npx);
                    ++it;
                    continue; // retry when memory frees up
                }
            }
            j.px_base = at;
            j.state = 1;
            j.t_admit = now_ms();
            used += j.footprint;
            slots_used += j.slots;
            staging_used += stg;
            cudaMemsetAsync(arena + at, 0, 16ull * j.npx, stream);
            active.push_back(j.id);
            it = queue.erase(it);
        } else {
            ++it;
        }
    }
    return !active.empty();
}

void cr_server::loop() {
    cudaSetDevice(device);
    LaunchCount lc;
    while (true) {
        std::vector<uint64_t> act;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_work.wait(lk, [&] { return stop || !queue.empty() || !active.empty(); });
            if (stop) break;
            admit_locked();
            act = active;
            if (act.empty()) { // nothing fits yet: wait for a completion or a new request
                cv_work.wait_for(lk, std::chrono::milliseconds(5));
                continue;
            }
        }
        // one sample pass of every active job
        std::vector<cr_job> pj;
        std::vector<uint32_t> bases;
        {
            std::lock_guard<std::mutex> lk(mu);
            for (uint64_t id : act) {
                SJob& j = jobs[id];
                cr_job c = j.job;
                c.spp = 1;
                c.frame_base = j.job.frame_base + j.done;
                c.out_rgb = j.d_out;
                pj.push_back(c);
                bases.push_back(j.px_base);
            }
        }
        RenderPlan plan;
        cr_status st = build_plan(pj.data(), (uint32_t)pj.size(), po, plan);
        if (st == CR_OK) {
            for (size_t i = 0; i < plan.jobs.size(); ++i) plan.jobs[i].px_base = bases[i];
            plan.npx_total = arena_px;
            st = dev.upload(plan, stream);
        }
        if (st == CR_OK) {
            ws.pb.accum = arena;
            const double tb = now_ms();
            st = enqueue_plan(plan, dev, ws, eo, stream, lc, nullptr);
            uint64_t counts[kCountsWords / 2];
            if (st == CR_OK) {
                std::lock_guard<std::mutex> lk(mu);
                for (uint64_t id : act) {
                    SJob& j = jobs[id];
                    if (j.done + 1 == j.job.spp) {
                        launch_output_one(arena + j.px_base, j.npx, 1.0f / (float)j.job.spp, j.d_out, stream, lc);
                        if (j.host_out)
                            cudaMemcpyAsync(j.job.out_rgb, j.d_out, 12ull * j.npx, cudaMemcpyDeviceToHost, stream);
                    }
                }
            }
            cudaMemcpyAsync(counts, ws.pb.counts, 4 * kCountsWords, cudaMemcpyDeviceToHost, stream);
            cudaError_t e = cudaStreamSynchronize(stream);
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e != cudaSuccess && st == CR_OK) {
                st = CR_ERR_CUDA;
                std::lock_guard<std::mutex> lk(mu);
                fatal_msg = cudaGetErrorString(e);
            }
            if (e == cudaSuccess && st == CR_OK && queue_status(counts) != CR_OK) {
                st = CR_ERR_CUDA;
                std::lock_guard<std::mutex> lk(mu);
                fatal_msg = "queue compaction overflowed";
            }
            if (st == CR_OK) {
                std::lock_guard<std::mutex> lk(mu);
                stats.passes++;
                stats.busy_ms += now_ms() - tb;
                const uint64_t* stat = counts + kStatWord / 2;
                for (uint32_t b = 1; b <= 16; ++b) stats.secondary_rays += stat[b];
                stats.kernel_launches = lc.n;
            }
        }
        {
            std::lock_guard<std::mutex> lk(mu);
            const double t = now_ms();
            std::vector<uint64_t> keep;
            for (uint64_t id : act) {
                SJob& j = jobs[id];
                if (st != CR_OK) {
                    j.state = 3;
                    j.status = st;
                } else if (++j.done < j.job.spp) {
                    keep.push_back(id);
                    continue;
                } else {
                    j.state = 2;
                }
                j.t_done = t;
                alloc.release(j.px_base, j.npx);
                used -= j.footprint;
                slots_used -= j.slots;
                if (j.host_out) staging_used -= 12ull * j.npx;
                if (j.host_out && j.d_out) {
                    cudaFree(j.d_out);
                    j.d_out = nullptr;
                }
                stats.jobs_done++;
            }
            active = keep;
            if (st != CR_OK) fatal = st;
        }
        cv_done.notify_all();
    }
}

extern "C" cr_status cr_server_create(const cr_server_opts* o, cr_server** out) {
    set_last_error("");
    if (!o || !out) {
        set_last_error("cr_server_create: NULL argument");
        return CR_ERR_INVALID_ARG;
    }
    *out = nullptr;
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
    s->eo.clear_accum = false;
    s->eo.write_output = false;
    const uint32_t m = o->group_w * o->group_h;
    if (!o->group_w || !o->group_h || (m & (m - 1)) || m > 1024 || o->hbm_budget < (64ull << 20)) {
        set_last_error("cr_server_create: bad tile shape or budget below 64 MiB");
        return CR_ERR_INVALID_ARG;
    }
    s->budget = o->hbm_budget;
    // the budget is split once: 60% path state (slots of the merged wavefront), 25% the
    // accumulation arena (16 B per pixel of every admitted job), 15% output staging for
    // jobs with host outputs (12 B per pixel)
    s->slots_cap = (uint32_t)std::min<uint64_t>(o->hbm_budget * 6 / 10 / kSlotBytes, 1ull << 27);
    s->arena_px = (uint32_t)std::min<uint64_t>(o->hbm_budget / 4 / 16, 1ull << 28);
    s->staging_cap = o->hbm_budget * 15 / 100;
    cudaGetDevice(&s->device);
    cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&s->arena, 16ull * s->arena_px);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_last_error("cr_server_create: device allocation failed");
        if (s->stream) cudaStreamDestroy(s->stream);
        return e == cudaErrorMemoryAllocation ? CR_ERR_OOM : CR_ERR_CUDA;
    }
    cr_status st = s->ws.ensure(s->slots_cap, 1);
    if (st == CR_OK) st = s->ws.ensure_nee(s->slots_cap);
    if (st != CR_OK) {
        cudaFree(s->arena);
        cudaStreamDestroy(s->stream);
        return st;
    }
    s->alloc.init(s->arena_px);
    std::memset(&s->stats, 0, sizeof(s->stats));
    s->t0 = std::chrono::steady_clock::now();
    cr_server* raw = s.get();
    raw->th = std::thread([raw] { raw->loop(); });
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
    const uint32_t tx = (job->camera.width + s->po.tile_w - 1) / s->po.tile_w;
    const uint32_t ty = (job->camera.height + s->po.tile_h - 1) / s->po.tile_h;
    j.slots = tx * ty * s->po.tile_w * s->po.tile_h;
    j.footprint = 16ull * j.npx + (j.host_out ? 12ull * j.npx : 0) + kSlotBytes * j.slots;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->fatal != CR_OK) {
        set_last_error("cr_server_submit: the server stopped after a device error");
        return s->fatal;
    }
    if (j.slots > s->slots_cap || j.npx > s->arena_px || (j.host_out && 12ull * j.npx > s->staging_cap)) {
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

extern "C" cr_status cr_server_poll(cr_server* s, uint64_t id, cr_job_stats* js) {
    set_last_error("");
    if (!s) return CR_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(id);
    if (it == s->jobs.end()) return CR_ERR_NOT_FOUND;
    if (it->second.state < 2) return CR_ERR_BUSY;
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
        return it == s->jobs.end() || it->second.state >= 2;
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
    out->active = (uint32_t)s->active.size();
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
    cudaStreamSynchronize(s->stream);
    for (auto& kv : s->jobs)
        if (kv.second.host_out && kv.second.d_out) cudaFree(kv.second.d_out);
    s->ws.release();
    s->dev.release();
    cudaFree(s->arena);
    cudaStreamDestroy(s->stream);
    delete s;
    return CR_OK;
}
