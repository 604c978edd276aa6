// Serving loop of the KCM library (declared in include/kcm.h, kcm_server_*): folding jobs of
// different chain lengths are admitted by a device-memory budget, stepped in batches that stay
// resident on the device, and retired when they converge or reach their iteration cap.
//
// Continuous batching. A batch is a kcm_create_batch handle on a stream of its own; it advances in
// chunks of `chunk` iterations launched without waiting. A tick that finds a chunk finished (CUDA
// event) reads every chain's state, retires the jobs that are done (their theta copied out), caps the
// others at their remaining iterations (kcm_set_chain_max_iters: a retired chain takes no more steps
// and costs no pair or solvation work) and launches the next chunk. Work admitted at different times
// runs on the device at once.
//
// Slots are refilled by compaction: the next batch takes the waiting jobs (in arrival order, as the
// budget allows) together with the running jobs of the batch with the most retired slots, which move
// over at that batch's next chunk boundary with the theta they reached; the old batch is then freed,
// so the memory of its retired jobs returns to the budget and its free slots are taken by the new
// jobs. A batch whose jobs have all retired is freed at once.
//
// The host work of making a batch (topologies, bond classes, uploads: milliseconds for large chains)
// runs on worker threads, up to four admission waves and one compaction at a time; ticks go on collecting and
// launching meanwhile and pick a batch up when it is ready. Device memory comes from the library's
// stream-ordered pool, so making and freeing batches does not wait on the other batches' work. The
// tick thread never waits on the device except to read the state of a batch whose chunk has already
// finished.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <deque>
#include <future>
#include <memory>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "kcm.h"
#include "kcm_internal.h"

namespace {

// device bytes per atom and per joint of a batch (neighbour lists dominate: kMaxNbr entries of 20 B
// per atom), used to admit jobs before their batch exists; the true size is read back after creation
constexpr int64_t kBytesPerAtom = 20 * kcm::kMaxNbr + 700;
constexpr int64_t kBytesPerJoint = 400;
constexpr int64_t kBytesPerBatch = 8 << 20;
// finished job records kept for kcm_server_job after they were polled (the oldest go first)
constexpr size_t kRetainedJobs = 1 << 16;
// batches made at once: admission waves on kWaveWorkers threads, and one compaction (the last slot)
constexpr int kWaveWorkers = 4;
constexpr int kMakeSlots = kWaveWorkers + 1;
constexpr int kCompactSlot = kWaveWorkers;

struct Job {
    int64_t id = 0;
    std::vector<int32_t> res;       // topology: released when the job retires
    std::vector<kcm_restype> types;
    kcm_geometry geom{};
    bool has_geom = false;
    std::vector<double> theta;  // start, then the angles reached (updated at migration and retirement)
    std::vector<double> chi;    // side-chain joints (params.side_joints): empty until the job first moves
                                // (they start at 0), then the angles reached
    int32_t max_iters = 0;
    int64_t natoms = 0;
    int32_t iters = 0;          // taken so far
    int32_t converged = 0;
    double last_dtheta = 0.0;
    int32_t state = 0;          // KCM_JOB_*
    bool cancel = false;        // kcm_server_cancel on a job that has a slot: retire at its next chunk boundary
    double t_submit = 0, t_admit = 0, t_done = 0;
    int error = KCM_OK;
};

struct Batch {
    kcm_handle h = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    std::vector<Job*> jobs;
    std::vector<int64_t> joff;
    int64_t bytes = 0;
    bool chunk_pending = false;
    bool moving = false;  // its running jobs move to the batch being made: no chunk after the current one
    bool handed = false;  // moving, its last chunk collected: the jobs' theta is in Job::theta
};

// the result of making a batch on the worker thread
struct Made {
    kcm_handle h = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    int rc = KCM_OK;
};

}  // namespace

struct kcm_server {
    kcm_params prm{};
    int device = 0;
    int64_t budget = 0;
    int64_t used = 0;      // device bytes held by the batches, and reserved by the one being made
    int32_t max_chains = 0;
    int32_t chunk = 0;
    int32_t min_wave = 1;     // admission: wait for this many jobs ...
    double max_wait = 0.0;    // ... or until the oldest waiting job has waited this long (s)
    int64_t next_id = 1;
    std::deque<Job*> pending;
    std::vector<std::unique_ptr<Batch>> active;
    // batches being made, each on a worker thread: admission waves, then one compaction (kCompactSlot)
    struct Making {
        bool busy = false;
        std::vector<Job*> jobs;   // the new jobs, then the movers
        Batch* from = nullptr;    // the batch the movers come from (compaction)
        int64_t reserved = 0;     // bytes reserved for it in the budget
        std::future<Made> fut;
    } mk[kMakeSlots];
    std::unordered_map<int64_t, std::unique_ptr<Job>> jobs;  // live and retained job records
    std::deque<int64_t> retained;             // polled finished jobs, oldest first
    std::vector<int64_t> finished;            // ids not yet reported by kcm_server_poll
    std::chrono::steady_clock::time_point t0;
    std::string err;
};

namespace {

double now(const kcm_server* s) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

int64_t estimate_bytes(const Job& j) {
    return kBytesPerAtom * j.natoms + kBytesPerJoint * static_cast<int64_t>(j.theta.size());
}

void retire(kcm_server* s, Job* j, int error) {
    j->state = KCM_JOB_DONE;
    j->error = error;
    j->t_done = now(s);
    std::vector<int32_t>().swap(j->res);  // the topology is no longer needed
    std::vector<kcm_restype>().swap(j->types);
    s->finished.push_back(j->id);
}

void destroy_batch(kcm_server* s, Batch* b) {
    if (b->h) kcm_destroy(b->h);
    if (b->ev) cudaEventDestroy(b->ev);
    if (b->stream) cudaStreamDestroy(b->stream);
    s->used -= b->bytes;
    b->bytes = 0;
    b->h = nullptr;
    b->ev = nullptr;
    b->stream = nullptr;
}

// launch the next chunk of a batch: every running job capped at its remaining iterations
int launch_chunk(kcm_server* s, Batch* b) {
    std::vector<int32_t> cap(b->jobs.size());
    for (size_t c = 0; c < b->jobs.size(); ++c) {
        const Job* j = b->jobs[c];
        cap[c] = j->state == KCM_JOB_RUNNING ? std::min(s->chunk, j->max_iters - j->iters) : 0;
    }
    int rc = kcm_set_chain_max_iters(b->h, cap.data());
    if (rc == KCM_OK) rc = kcm_step_async(b->h, s->chunk);
    if (rc == KCM_OK && cudaEventRecord(b->ev, b->stream) != cudaSuccess) rc = KCM_E_CUDA;
    b->chunk_pending = rc == KCM_OK;
    return rc;
}

// A finished chunk: account every chain, retire the jobs that are done (and those cancelled), then
// launch the next chunk; a moving batch instead hands its running jobs' theta over and stops.
int collect(kcm_server* s, Batch* b) {
    const size_t C = b->jobs.size();
    std::vector<int32_t> it(C), cv(C), er(C);
    std::vector<double> dm(C);
    int32_t dummy = 0;
    double dmax = 0.0;
    int rc = kcm_step_status(b->h, &dummy, &dmax);  // chain failures are read per chain below
    if (rc != KCM_OK && rc != KCM_E_NONFINITE && rc != KCM_E_OVERFLOW) return rc;
    rc = kcm_chain_state(b->h, it.data(), cv.data(), dm.data(), er.data());
    if (rc != KCM_OK) return rc;
    bool any_out = b->moving;
    for (size_t c = 0; c < C; ++c) {
        Job* j = b->jobs[c];
        if (j->state != KCM_JOB_RUNNING) continue;
        j->iters += it[c];
        if (it[c] > 0) j->last_dtheta = dm[c];
        const bool conv = cv[c] && j->last_dtheta < s->prm.conv_tol && it[c] > 0;
        if (er[c] != KCM_OK || conv || j->iters >= j->max_iters || j->cancel) any_out = true;
    }
    std::vector<double> theta;
    if (any_out) {
        const int64_t l = b->joff.back();
        theta.resize(static_cast<size_t>(l));
        rc = kcm_get_theta(b->h, theta.data(), l);
        if (rc != KCM_OK) return rc;
    }
    // a moving batch hands its side-chain angles over too
    std::vector<double> chi;
    std::vector<int64_t> soff;
    if (b->moving && s->prm.side_joints) {
        const int64_t ls = kcm_nside_joints(b->h);
        chi.resize(static_cast<size_t>(ls));
        soff.resize(C + 1);
        rc = kcm_get_side_theta(b->h, chi.data(), ls);
        if (rc == KCM_OK) rc = kcm_side_offsets(b->h, soff.data());
        if (rc != KCM_OK) return rc;
    }
    int running = 0;
    for (size_t c = 0; c < C; ++c) {
        Job* j = b->jobs[c];
        if (j->state != KCM_JOB_RUNNING) continue;
        const bool conv = cv[c] && j->last_dtheta < s->prm.conv_tol && it[c] > 0 && er[c] == KCM_OK;
        const bool out = er[c] != KCM_OK || conv || j->iters >= j->max_iters || j->cancel;
        if (out || b->moving) std::copy(theta.begin() + b->joff[c], theta.begin() + b->joff[c + 1], j->theta.begin());
        if (b->moving && !chi.empty()) j->chi.assign(chi.begin() + soff[c], chi.begin() + soff[c + 1]);
        if (out) {
            j->converged = conv;
            retire(s, j, er[c] != KCM_OK ? er[c] : (j->cancel && !conv && j->iters < j->max_iters ? KCM_E_CANCELLED : KCM_OK));
        } else {
            ++running;
        }
    }
    b->chunk_pending = false;
    if (b->moving || (running == 0 && b == s->mk[kCompactSlot].from)) {
        b->moving = true;
        b->handed = true;  // the batch being made picks the running jobs up (and then frees this one)
        return KCM_OK;
    }
    if (running == 0) {
        destroy_batch(s, b);
        return KCM_OK;
    }
    return launch_chunk(s, b);
}

// the worker: a batch of the given chains on a stream of its own (on the server's device)
Made make_batch(int device, std::vector<kcm_topology> tops, kcm_params prm) {
    Made m;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&m.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&m.ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        m.rc = KCM_E_CUDA;
        return m;
    }
    m.rc = kcm_create_batch(tops.data(), static_cast<int32_t>(tops.size()), &prm, m.stream, &m.h);
    // batches run beside each other on their own streams: no launch overlap (kcm_set_graph_overlap)
    if (m.rc == KCM_OK) m.rc = kcm_set_graph_overlap(m.h, 0);
    return m;
}

void free_made(Made& m) {
    if (m.h) kcm_destroy(m.h);
    if (m.ev) cudaEventDestroy(m.ev);
    if (m.stream) cudaStreamDestroy(m.stream);
    m = Made{};
}

// Start making the next batches when there is work for them. A ready admission wave (min_wave jobs
// wait, the oldest has waited max_wait, or nothing runs) that fits the budget becomes a batch of its own
// on a free admission worker (up to four run at once), so admission never waits on a chunk boundary.
// Independently, the batch with the most retired slots is compacted on the compaction worker: its running jobs move to a new batch,
// together with the waiting jobs that the admission policy or the budget holds back (as many as fit its
// free slots), when at least half of its slots are free (its memory comes back) or when such jobs wait
// and it holds no more than four running jobs per free slot (so that moving them costs a bounded
// multiple of the new jobs' set-up).
int launch_make(kcm_server* s, int slot, std::vector<Job*>& take, Batch* from, int64_t bytes);

int start_making(kcm_server* s) {
    const bool wave_ready = !s->pending.empty() &&
        (static_cast<int32_t>(s->pending.size()) >= s->min_wave || s->active.empty() ||
         now(s) - s->pending.front()->t_submit >= s->max_wait);
    std::vector<Job*> take;
    int64_t bytes = kBytesPerBatch;
    // the waiting jobs, in arrival order, that fit the budget (at most `room`)
    auto take_pending = [&](int room) {
        while (!s->pending.empty() && static_cast<int32_t>(take.size()) < room) {
            Job* j = s->pending.front();
            const int64_t need = estimate_bytes(*j);
            if (s->used + bytes + need > s->budget) {
                if (take.empty() && s->active.empty()) {  // can never fit: refuse it
                    s->pending.pop_front();
                    retire(s, j, KCM_E_NOMEM);
                    continue;
                }
                break;
            }
            bytes += need;
            take.push_back(j);
            s->pending.pop_front();
        }
    };
    bool wave_blocked = false;  // a ready wave that the budget holds back
    int wslot = 0;
    while (wslot < kWaveWorkers && s->mk[wslot].busy) ++wslot;
    if (wave_ready && wslot < kWaveWorkers) {
        take_pending(s->max_chains);
        if (!take.empty()) {
            const int rc = launch_make(s, wslot, take, nullptr, bytes);
            if (rc != KCM_OK) return rc;
        } else {
            wave_blocked = !s->pending.empty();
        }
    }
    // waiting jobs join a compaction only when the admission policy or the budget holds them back (a
    // ready wave waits for the admission worker instead of a compacted batch's chunk boundary)
    const bool absorb = !s->pending.empty() && (!wave_ready || wave_blocked);
    take.clear();
    bytes = kBytesPerBatch;
    Batch* from = nullptr;
    if (!s->mk[kCompactSlot].busy) {
        int from_running = 0, best_free = 0;
        for (auto& b : s->active) {
            if (!b->h || b->moving || !b->chunk_pending) continue;
            int run = 0;
            for (Job* j : b->jobs) run += j->state == KCM_JOB_RUNNING;
            const int free = static_cast<int>(b->jobs.size()) - run;
            const bool worth = 2 * free >= static_cast<int>(b->jobs.size()) || (absorb && run <= 4 * free);
            if (run > 0 && free > 0 && run < s->max_chains && worth && free > best_free) {
                from = b.get();
                from_running = run;
                best_free = free;
            }
        }
        if (from) {  // the movers' memory is held twice until their old batch is freed
            int64_t need = 0;
            for (Job* j : from->jobs)
                if (j->state == KCM_JOB_RUNNING) need += estimate_bytes(*j);
            if (s->used + bytes + need > s->budget) {
                from = nullptr;
            } else {
                bytes += need;
                if (absorb) take_pending(s->max_chains - from_running);
                for (Job* j : from->jobs)
                    if (j->state == KCM_JOB_RUNNING) take.push_back(j);
            }
        }
    }
    if (take.empty()) return KCM_OK;
    return launch_make(s, kCompactSlot, take, from, bytes);
}

// hands the jobs to a worker thread that makes their batch (a wave, or the compaction slot)
int launch_make(kcm_server* s, int slot, std::vector<Job*>& take, Batch* from, int64_t bytes) {
    std::vector<kcm_topology> tops(take.size());
    for (size_t c = 0; c < take.size(); ++c) {
        Job* j = take[c];
        tops[c].n_res = static_cast<int32_t>(j->res.size());
        tops[c].res_type = j->res.data();
        tops[c].n_types = static_cast<int32_t>(j->types.size());
        tops[c].types = j->types.data();
        tops[c].geometry = j->has_geom ? &j->geom : nullptr;
    }
    try {
        s->mk[slot].fut = std::async(std::launch::async, make_batch, s->device, std::move(tops), s->prm);
    } catch (...) {  // no thread: put the new jobs back in arrival order
        for (auto it = take.rbegin(); it != take.rend(); ++it)
            if ((*it)->state == KCM_JOB_WAITING) s->pending.push_front(*it);
        return KCM_E_NOMEM;
    }
    kcm_server::Making& k = s->mk[slot];
    k.busy = true;
    k.jobs = take;
    k.from = from;  // it runs on until the new batch is ready, then stops at its next chunk boundary
    k.reserved = bytes;
    s->used += bytes;
    return KCM_OK;
}

// The batch being made, once the worker is done and its movers (if any) have been handed over: set its
// theta (the new jobs' starts, the movers' angles reached), start it, free the batch the movers left.
int finish_making(kcm_server* s, int slot) {
    kcm_server::Making& k = s->mk[slot];
    if (!k.busy) return KCM_OK;
    if (k.fut.wait_for(std::chrono::seconds(0)) != std::future_status::ready) return KCM_OK;
    Batch* from = k.from;
    if (from && !from->handed) {  // stop the movers' batch at the end of its current chunk
        from->moving = true;
        return KCM_OK;
    }
    Made m = k.fut.get();
    k.busy = false;
    s->used -= k.reserved;
    std::vector<Job*> take;
    take.swap(k.jobs);
    k.from = nullptr;
    if (m.rc != KCM_OK) {  // the new jobs fail; the movers go on in their batch
        free_made(m);
        for (Job* j : take)
            if (j->state == KCM_JOB_WAITING) retire(s, j, m.rc);
        if (from) {
            from->moving = false;
            from->handed = false;
            int run = 0;
            for (Job* j : from->jobs) run += j->state == KCM_JOB_RUNNING;
            if (run == 0) destroy_batch(s, from);
            else return launch_chunk(s, from);
        }
        return KCM_OK;
    }
    if (from) {
        from->jobs.clear();  // its jobs live on in the new batch (or have retired)
        destroy_batch(s, from);
    }
    // a job cancelled, or a mover that retired at the hand-over, has no slot to take: keep the others
    auto has_slot = [](const Job* j) { return j->state != KCM_JOB_DONE; };
    std::unique_ptr<Batch> b(new Batch());
    b->h = m.h;
    b->stream = m.stream;
    b->ev = m.ev;
    b->bytes = kcm_device_bytes(m.h);
    s->used += b->bytes;
    b->joff.resize(take.size() + 1);
    int rc = kcm_chain_offsets(b->h, nullptr, b->joff.data());
    std::vector<double> theta;
    for (Job* j : take) theta.insert(theta.end(), j->theta.begin(), j->theta.end());
    if (rc == KCM_OK) rc = kcm_set_theta(b->h, theta.data(), static_cast<int64_t>(theta.size()));
    if (rc == KCM_OK && s->prm.side_joints) {  // the movers' side-chain angles; new jobs start at 0
        const int64_t ls = kcm_nside_joints(b->h);
        std::vector<int64_t> soff(take.size() + 1);
        std::vector<double> chi(static_cast<size_t>(ls), 0.0);
        rc = kcm_side_offsets(b->h, soff.data());
        for (size_t c = 0; rc == KCM_OK && c < take.size(); ++c) {
            const Job* j = take[c];
            if (!j->chi.empty() && static_cast<int64_t>(j->chi.size()) == soff[c + 1] - soff[c])
                std::copy(j->chi.begin(), j->chi.end(), chi.begin() + soff[c]);
        }
        if (rc == KCM_OK && ls > 0) rc = kcm_set_side_theta(b->h, chi.data(), ls);
    }
    if (rc != KCM_OK) {
        for (Job* j : take)
            if (has_slot(j)) retire(s, j, rc);
        destroy_batch(s, b.get());
        return KCM_OK;
    }
    const double t = now(s);
    for (Job* j : take) {
        if (j->state == KCM_JOB_WAITING) {
            if (j->cancel) {  // cancelled while its batch was made
                retire(s, j, KCM_E_CANCELLED);
                continue;
            }
            j->state = KCM_JOB_RUNNING;
            j->t_admit = t;
        }
    }
    b->jobs = take;
    bool any = false;
    for (Job* j : take) any = any || j->state == KCM_JOB_RUNNING;
    if (!any) {
        destroy_batch(s, b.get());
        return KCM_OK;
    }
    rc = launch_chunk(s, b.get());
    s->active.push_back(std::move(b));
    return rc;
}

int fail(kcm_server* s, int code, const std::string& msg) {
    if (s) s->err = msg;
    return code;
}

}  // namespace

extern "C" {

int kcm_server_create(const kcm_params* prm, int64_t hbm_budget_bytes, int32_t max_chains_per_batch,
                      int32_t chunk_iters, kcm_server** out) {
    if (!out) return KCM_E_INVAL;
    *out = nullptr;
    std::string err;
    int rc = kcm::validate_params(prm, &err);
    if (rc != KCM_OK) return rc;
    if (hbm_budget_bytes <= 0 || max_chains_per_batch < 1 || chunk_iters < 1) return KCM_E_INVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return KCM_E_NODEVICE;
    }
    kcm_server* s = new (std::nothrow) kcm_server();
    if (!s) return KCM_E_NOMEM;
    s->prm = *prm;
    s->device = dev;
    s->budget = hbm_budget_bytes;
    s->max_chains = max_chains_per_batch;
    s->chunk = chunk_iters;
    s->t0 = std::chrono::steady_clock::now();
    *out = s;
    return KCM_OK;
}

void kcm_server_destroy(kcm_server* s) {
    if (!s) return;
    for (auto& k : s->mk) {
        if (!k.busy) continue;
        Made m = k.fut.get();  // wait for the worker, then drop what it made
        free_made(m);
    }
    for (auto& b : s->active) destroy_batch(s, b.get());
    delete s;
}

int kcm_server_submit(kcm_server* s, const kcm_topology* top, const double* theta0, int64_t l, int32_t max_iters,
                      int64_t* job_id) {
    if (!s || !top || !job_id) return KCM_E_INVAL;
    *job_id = 0;
    if (max_iters < 1) return fail(s, KCM_E_INVAL, "max_iters < 1");
    if (!top->res_type || !top->types || top->n_res < 1 || top->n_types < 1)
        return fail(s, KCM_E_INVAL, "incomplete topology");
    const int64_t natoms = kcm_topology_natoms(top);
    if (natoms < 0) return fail(s, static_cast<int>(natoms), "invalid topology");
    if (l != 2 * static_cast<int64_t>(top->n_res) || (l > 0 && !theta0))
        return fail(s, KCM_E_INVAL, "theta length must be 2 n_res");
    std::unique_ptr<Job> j(new (std::nothrow) Job());
    if (!j) return KCM_E_NOMEM;
    j->id = s->next_id++;
    j->res.assign(top->res_type, top->res_type + top->n_res);
    j->types.assign(top->types, top->types + top->n_types);
    if (top->geometry) { j->geom = *top->geometry; j->has_geom = true; }
    j->theta.assign(theta0, theta0 + l);
    j->max_iters = max_iters;
    j->natoms = natoms;
    j->state = KCM_JOB_WAITING;
    j->t_submit = now(s);
    *job_id = j->id;
    s->pending.push_back(j.get());
    s->jobs.emplace(j->id, std::move(j));
    return KCM_OK;
}

int kcm_server_tick(kcm_server* s, int32_t* n_waiting, int32_t* n_running) {
    if (!s) return KCM_E_INVAL;
    int rc = KCM_OK;
    for (auto& b : s->active) {  // collect the batches whose chunk has finished
        if (!b->h || !b->chunk_pending) continue;
        const cudaError_t q = cudaEventQuery(b->ev);
        if (q == cudaErrorNotReady) continue;
        if (q != cudaSuccess) { cudaGetLastError(); return fail(s, KCM_E_CUDA, cudaGetErrorString(q)); }
        rc = collect(s, b.get());
        if (rc != KCM_OK) return fail(s, rc, "collecting a batch failed");
    }
    for (int slot = 0; slot < kMakeSlots; ++slot) {
        rc = finish_making(s, slot);
        if (rc != KCM_OK) return fail(s, rc, "starting a batch failed");
    }
    s->active.erase(std::remove_if(s->active.begin(), s->active.end(), [](const std::unique_ptr<Batch>& b) { return !b->h; }),
                    s->active.end());
    rc = start_making(s);
    if (rc != KCM_OK) return fail(s, rc, "making a batch failed");
    int32_t running = 0;
    for (auto& b : s->active)
        for (Job* j : b->jobs) running += j->state == KCM_JOB_RUNNING;
    int32_t waiting = static_cast<int32_t>(s->pending.size());
    for (auto& k : s->mk)
        if (k.busy)
            for (Job* j : k.jobs) waiting += j->state == KCM_JOB_WAITING;
    if (running == 0 && waiting == 0) {
        // every job of a batch being made retired meanwhile: nothing else runs, so wait for the worker and
        // drop what it made, with the batch its movers came from
        for (auto& k : s->mk) {
            if (!k.busy) continue;
            Made m = k.fut.get();
            free_made(m);
            k.busy = false;
            s->used -= k.reserved;
            k.jobs.clear();
            if (k.from) {
                k.from->jobs.clear();
                destroy_batch(s, k.from);
                k.from = nullptr;
            }
        }
        s->active.erase(std::remove_if(s->active.begin(), s->active.end(), [](const std::unique_ptr<Batch>& b) { return !b->h; }),
                        s->active.end());
    }
    if (n_waiting) *n_waiting = waiting;
    if (n_running) *n_running = running;
    return KCM_OK;
}

int kcm_server_cancel(kcm_server* s, int64_t job_id) {
    if (!s) return KCM_E_INVAL;
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return fail(s, KCM_E_INVAL, "unknown job");
    Job* j = it->second.get();
    if (j->state == KCM_JOB_DONE) return fail(s, KCM_E_INVAL, "the job has finished");
    if (j->cancel) return KCM_OK;
    j->cancel = true;
    auto p = std::find(s->pending.begin(), s->pending.end(), j);
    if (p != s->pending.end()) {  // still queued: retire it now
        s->pending.erase(p);
        retire(s, j, KCM_E_CANCELLED);
    }
    return KCM_OK;
}

int kcm_server_set_admission(kcm_server* s, int32_t min_jobs, double max_wait_s) {
    if (!s || min_jobs < 1 || !(max_wait_s >= 0.0) || !std::isfinite(max_wait_s)) return KCM_E_INVAL;
    s->min_wave = min_jobs;
    s->max_wait = max_wait_s;
    return KCM_OK;
}

int kcm_server_poll(kcm_server* s, int64_t* ids, int32_t capacity, int32_t* n) {
    if (!s || !n || (capacity > 0 && !ids)) return KCM_E_INVAL;
    const int32_t k = std::min<int32_t>(capacity, static_cast<int32_t>(s->finished.size()));
    for (int32_t i = 0; i < k; ++i) {
        ids[i] = s->finished[i];
        s->retained.push_back(ids[i]);
    }
    s->finished.erase(s->finished.begin(), s->finished.begin() + k);
    while (s->retained.size() > kRetainedJobs) {  // the oldest polled records go
        s->jobs.erase(s->retained.front());
        s->retained.pop_front();
    }
    *n = k;
    return KCM_OK;
}

int kcm_server_job(kcm_server* s, int64_t job_id, kcm_job_info* info, double* theta, int64_t l) {
    if (!s) return KCM_E_INVAL;
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return fail(s, KCM_E_INVAL, "unknown job, or its record was dropped");
    const Job* j = it->second.get();
    if (info) {
        info->state = j->state;
        info->error = j->error;
        info->iters = j->iters;
        info->converged = j->converged;
        info->max_dtheta = j->last_dtheta;
        info->natoms = j->natoms;
        info->t_submit = j->t_submit;
        info->t_admit = j->t_admit;
        info->t_done = j->t_done;
    }
    if (theta) {
        if (l != static_cast<int64_t>(j->theta.size())) return KCM_E_INVAL;
        std::memcpy(theta, j->theta.data(), sizeof(double) * j->theta.size());
    }
    return KCM_OK;
}

int64_t kcm_server_device_bytes(kcm_server* s) { return s ? s->used : -1; }

}  // extern "C"
