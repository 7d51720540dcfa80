// Slot-driven serving loop with continuous batching (mmgap_server_*).
//
// Callers submit uplink detection jobs and downlink VPP precoding jobs
// (inputs already resident on the device, e.g. channel state kept there
// across slots) from any host thread.  A
// dispatcher thread admits queued jobs in arrival order into launch groups:
// a group goes to a free lane (a CUDA stream with its own batch runner and
// coupling scratch) and takes jobs while they fit that lane's scratch
// (admission by memory).  Each group runs as one batched launch (replayed
// from a CUDA graph); groups on different lanes overlap on the device, so
// jobs that arrive while others are running start as soon as a lane frees
// up.  A host callback at the end of each group timestamps its jobs and frees
// the lane.  Results do not depend on grouping: each job is computed exactly
// as mmgap_detect or mmgap_precode computes it.  A precoding job's channel
// inverse and VPP build run just before its group's batched launch, its
// problems go through the same batched solver, and its output kernel runs
// right after.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/mmgap.h"
#include "batch.h"

using namespace mmgap;

namespace {

double now_us() {
    using namespace std::chrono;
    return duration<double, std::micro>(steady_clock::now().time_since_epoch()).count();
}

struct JobRec {
    bool precode = false;
    mmgap_detect_job job{};
    mmgap_precode_job pjob{};
    mmgap_job_info info;
    bool done = false;
    int n_problems() const { return precode ? pjob.n_problems : job.n_problems; }
    size_t scratch() const {
        return precode ? BatchRunner::precode_scratch_bytes(pjob) : BatchRunner::scratch_bytes(job.n_t, job.n_problems);
    }
    GroupJob group_job() const {
        GroupJob g;
        if (precode) g.pre = &pjob;
        else g.det = &job;
        return g;
    }
};

struct Lane {
    cudaStream_t stream = nullptr;
    BatchRunner runner;
    bool busy = false;
    std::vector<uint64_t> tickets;  // jobs of the group in flight
    double start_us = 0.0;
};

}  // namespace

struct mmgap_server {
    int device = 0;
    mmgap_params params{};
    size_t lane_scratch = 0;
    int lane_jobs = 0;
    int max_n_t = 16, max_n_r = 16;
    long long lane_problems = 0;
    double deadline_us = 0.0;
    double inject_delay_us = 0.0;
    bool use_graph = true;
    int* err_word = nullptr;

    std::vector<Lane> lanes;
    std::mutex mu;
    std::condition_variable cv_dispatch;  // dispatcher wake-up
    std::condition_variable cv_done;      // waiters
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, JobRec> jobs;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread dispatcher;
    mmgap_status fault = MMGAP_OK;
    // statistics
    std::vector<double> latencies_us;
    long long completed = 0, problems_done = 0, deadline_misses = 0, groups = 0, max_group_jobs = 0;
    double first_submit_us = -1.0, last_done_us = 0.0;
};

namespace {

struct Callback {
    mmgap_server* s;
    int lane;
};

void CUDART_CB on_group_done(void* p) {
    auto* cb = static_cast<Callback*>(p);
    mmgap_server* s = cb->s;
    const double t = now_us();
    {
        std::lock_guard<std::mutex> lock(s->mu);
        Lane& L = s->lanes[cb->lane];
        for (uint64_t tk : L.tickets) {
            JobRec& r = s->jobs[tk];
            r.info.done_us = t;
            r.info.status = MMGAP_OK;
            r.done = true;
            const double lat = t - r.info.submit_us;
            s->latencies_us.push_back(lat);
            s->completed++;
            s->problems_done += r.n_problems();
            if (s->deadline_us > 0.0 && lat > s->deadline_us) s->deadline_misses++;
        }
        s->last_done_us = t;
        L.tickets.clear();
        L.busy = false;
    }
    s->cv_done.notify_all();
    s->cv_dispatch.notify_one();
    delete cb;
}

void dispatch_loop(mmgap_server* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lock(s->mu);
    for (;;) {
        s->cv_dispatch.wait(lock, [&] {
            if (s->stop) return true;
            if (s->queue.empty()) return false;
            for (const Lane& L : s->lanes)
                if (!L.busy) return true;
            return false;
        });
        if (s->stop) break;
        int li = -1;
        for (int i = 0; i < (int)s->lanes.size(); ++i)
            if (!s->lanes[i].busy) {
                li = i;
                break;
            }
        Lane& L = s->lanes[li];
        // admit queued jobs in arrival order while they fit this lane
        // (records stay in the map, whose nodes do not move, until their tickets are waited for)
        std::vector<GroupJob> group;
        size_t scratch = 0;
        long long probs = 0;
        while (!s->queue.empty() && (int)group.size() < s->lane_jobs) {
            const uint64_t tk = s->queue.front();
            const JobRec& r = s->jobs[tk];
            const size_t need = r.scratch();
            if (scratch + need > s->lane_scratch || probs + r.n_problems() > s->lane_problems) break;
            scratch += need;
            probs += r.n_problems();
            group.push_back(r.group_job());
            L.tickets.push_back(tk);
            s->queue.pop_front();
        }
        if (group.empty()) continue;  // cannot happen: submit rejects jobs larger than a lane
        L.busy = true;
        const double t0 = now_us();
        for (uint64_t tk : L.tickets) s->jobs[tk].info.start_us = t0;
        s->groups++;
        s->max_group_jobs = std::max<long long>(s->max_group_jobs, (long long)group.size());
        L.start_us = t0;
        const double delay = s->inject_delay_us;
        lock.unlock();
        if (delay > 0.0) std::this_thread::sleep_for(std::chrono::microseconds((long long)delay));
        // largest users first inside the group
        std::vector<int> order(group.size());
        for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return group[a].n_t() > group[b].n_t(); });
        cudaError_t e = cudaSuccess;
        {
            NvtxRange nvtx_range("mmgap_server_group");
            if (L.runner.stage(group.data(), order.data(), (int)group.size()) != 0) e = cudaErrorInvalidValue;
            if (e == cudaSuccess) e = L.runner.run(s->params, L.stream, s->use_graph);
            if (e == cudaSuccess) e = cudaLaunchHostFunc(L.stream, on_group_done, new Callback{s, li});
        }
        lock.lock();
        if (e != cudaSuccess) {
            fprintf(stderr, "mmgap_server: launch failed: %s\n", cudaGetErrorString(e));
            s->fault = MMGAP_ECUDA;
            for (uint64_t tk : L.tickets) {
                s->jobs[tk].info.status = MMGAP_ECUDA;
                s->jobs[tk].done = true;
            }
            L.tickets.clear();
            L.busy = false;
            s->cv_done.notify_all();
        }
    }
}

}  // namespace

extern "C" {

mmgap_status mmgap_server_create(mmgap_server** out, int device, const mmgap_params* params,
                                 const mmgap_server_config* cfg) {
    if (!out || !params || !cfg) return MMGAP_EINVAL;
    *out = nullptr;
    if (BatchRunner::check_params(*params)) {
        fprintf(stderr, "mmgap_server_create: %s\n", BatchRunner::check_params(*params));
        return MMGAP_EUNSUPPORTED;
    }
    if (const char* why = BatchRunner::check_early_exit(*params, nullptr, 0, cfg->tensor_core != 0)) {
        fprintf(stderr, "mmgap_server_create: %s\n", why);
        return MMGAP_EUNSUPPORTED;
    }
    if (cfg->n_lanes < 1 || cfg->n_lanes > 16 || cfg->scratch_bytes == 0 || cfg->max_jobs_per_group < 1 ||
        cfg->max_problems_per_group < 1 || cfg->max_n_r < 1 || cfg->max_n_r > 64 ||
        !(cfg->max_n_t == 4 || cfg->max_n_t == 8 || cfg->max_n_t == 16 || cfg->max_n_t == 32))
        return MMGAP_EINVAL;
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) return MMGAP_EINVAL;
    auto* s = new (std::nothrow) mmgap_server();
    if (!s) return MMGAP_ENOMEM;
    s->device = device;
    s->params = *params;
    s->lane_scratch = cfg->scratch_bytes / (size_t)cfg->n_lanes;
    s->lane_jobs = cfg->max_jobs_per_group;
    s->lane_problems = cfg->max_problems_per_group;
    s->max_n_t = cfg->max_n_t;
    s->max_n_r = cfg->max_n_r;
    s->deadline_us = cfg->deadline_us;
    s->inject_delay_us = cfg->inject_delay_us;
    s->use_graph = cfg->use_graph != 0;
    mmgap_status st = MMGAP_OK;
    if (cudaMalloc(&s->err_word, sizeof(int)) != cudaSuccess || cudaMemset(s->err_word, 0, sizeof(int)) != cudaSuccess)
        st = MMGAP_ENOMEM;
    s->lanes.resize(cfg->n_lanes);
    for (Lane& L : s->lanes) {
        if (st != MMGAP_OK) break;
        if (cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking) != cudaSuccess) st = MMGAP_ECUDA;
        else if (L.runner.init(device, s->lane_jobs, s->lane_problems, s->lane_scratch, cfg->max_n_r, cfg->max_n_t,
                               s->err_word, cfg->tensor_core != 0) != cudaSuccess)
            st = MMGAP_ENOMEM;
    }
    if (st != MMGAP_OK) {
        cudaGetLastError();
        for (Lane& L : s->lanes) {
            L.runner.release();
            if (L.stream) cudaStreamDestroy(L.stream);
        }
        if (s->err_word) cudaFree(s->err_word);
        delete s;
        if (prev >= 0) cudaSetDevice(prev);
        return st;
    }
    s->dispatcher = std::thread(dispatch_loop, s);
    if (prev >= 0) cudaSetDevice(prev);
    *out = s;
    return MMGAP_OK;
}

mmgap_status mmgap_server_submit(mmgap_server* s, const mmgap_detect_job* job, uint64_t* ticket) {
    if (!s || !job || !ticket) return MMGAP_EINVAL;
    if (const char* why = BatchRunner::check_job(*job)) {
        fprintf(stderr, "mmgap_server_submit: %s\n", why);
        return MMGAP_EUNSUPPORTED;
    }
    if (const char* why = BatchRunner::check_early_exit(s->params, job, 1, false)) {
        fprintf(stderr, "mmgap_server_submit: %s\n", why);
        return MMGAP_EUNSUPPORTED;
    }
    if (job->n_t > s->max_n_t || job->n_r > s->max_n_r) return MMGAP_EUNSUPPORTED;
    if (BatchRunner::scratch_bytes(job->n_t, job->n_problems) > s->lane_scratch ||
        job->n_problems > s->lane_problems)
        return MMGAP_ENOMEM;  // can never be admitted
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->stop) return MMGAP_EBUSY;
        const uint64_t tk = s->next_ticket++;
        JobRec& r = s->jobs[tk];
        r.job = *job;
        r.info = mmgap_job_info{};
        r.info.ticket = tk;
        r.info.status = -1;
        r.info.submit_us = now_us();
        if (s->first_submit_us < 0.0) s->first_submit_us = r.info.submit_us;
        s->queue.push_back(tk);
        *ticket = tk;
    }
    s->cv_dispatch.notify_one();
    return MMGAP_OK;
}

mmgap_status mmgap_server_submit_precode(mmgap_server* s, const mmgap_precode_job* job, uint64_t* ticket) {
    if (!s || !job || !ticket) return MMGAP_EINVAL;
    if (const char* why = BatchRunner::check_precode(*job)) {
        fprintf(stderr, "mmgap_server_submit_precode: %s\n", why);
        return MMGAP_EUNSUPPORTED;
    }
    if (job->n_u > s->max_n_t) return MMGAP_EUNSUPPORTED;
    if (BatchRunner::precode_scratch_bytes(*job) > s->lane_scratch || job->n_problems > s->lane_problems)
        return MMGAP_ENOMEM;  // can never be admitted
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->stop) return MMGAP_EBUSY;
        const uint64_t tk = s->next_ticket++;
        JobRec& r = s->jobs[tk];
        r.precode = true;
        r.pjob = *job;
        r.info = mmgap_job_info{};
        r.info.ticket = tk;
        r.info.status = -1;
        r.info.submit_us = now_us();
        if (s->first_submit_us < 0.0) s->first_submit_us = r.info.submit_us;
        s->queue.push_back(tk);
        *ticket = tk;
    }
    s->cv_dispatch.notify_one();
    return MMGAP_OK;
}

mmgap_status mmgap_server_wait(mmgap_server* s, uint64_t ticket, int64_t timeout_us, mmgap_job_info* info) {
    if (!s) return MMGAP_EINVAL;
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return MMGAP_EINVAL;
    auto ready = [&] { return it->second.done; };
    if (timeout_us < 0) s->cv_done.wait(lock, ready);
    else if (!s->cv_done.wait_for(lock, std::chrono::microseconds(timeout_us), ready)) return MMGAP_ETIMEOUT;
    if (info) *info = it->second.info;
    const int st = it->second.info.status;
    s->jobs.erase(it);
    return st == MMGAP_OK ? MMGAP_OK : (mmgap_status)st;
}

mmgap_status mmgap_server_stats(mmgap_server* s, mmgap_serve_stats* out, int reset) {
    if (!s || !out) return MMGAP_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    *out = mmgap_serve_stats{};
    out->completed = s->completed;
    out->problems = s->problems_done;
    out->deadline_misses = s->deadline_misses;
    out->groups = s->groups;
    out->max_group_jobs = s->max_group_jobs;
    out->queued = (long long)s->queue.size();
    if (!s->latencies_us.empty()) {
        std::vector<double> v = s->latencies_us;
        std::sort(v.begin(), v.end());
        auto pct = [&](double q) {
            size_t i = (size_t)std::ceil(q * v.size());
            return v[std::min(v.size() - 1, i == 0 ? 0 : i - 1)];
        };
        out->p50_us = pct(0.50);
        out->p99_us = pct(0.99);
        out->max_us = v.back();
        double sum = 0.0;
        for (double x : v) sum += x;
        out->mean_us = sum / v.size();
    }
    if (s->first_submit_us >= 0.0 && s->last_done_us > s->first_submit_us)
        out->span_us = s->last_done_us - s->first_submit_us;
    if (reset) {
        s->latencies_us.clear();
        s->completed = s->problems_done = s->deadline_misses = s->groups = s->max_group_jobs = 0;
        s->first_submit_us = -1.0;
        s->last_done_us = 0.0;
    }
    return s->fault;
}

mmgap_status mmgap_server_destroy(mmgap_server* s) {
    if (!s) return MMGAP_OK;
    {
        std::unique_lock<std::mutex> lock(s->mu);
        // let queued and running groups finish
        s->cv_done.wait(lock, [&] {
            if (!s->queue.empty()) return false;
            for (const Lane& L : s->lanes)
                if (L.busy) return false;
            return true;
        });
        s->stop = true;
    }
    s->cv_dispatch.notify_all();
    if (s->dispatcher.joinable()) s->dispatcher.join();
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    for (Lane& L : s->lanes) {
        cudaStreamSynchronize(L.stream);
        L.runner.release();
        cudaStreamDestroy(L.stream);
    }
    cudaFree(s->err_word);
    delete s;
    if (prev >= 0) cudaSetDevice(prev);
    return MMGAP_OK;
}

}  // extern "C"
