// Serving loop of the KCM library (declared in include/kcm.h, kcm_server_*): folding jobs of
// different chain lengths are admitted by a device-memory budget, stepped in batches that stay
// resident on the device, and retired when they converge or reach their iteration cap.
//
// Continuous batching: every kcm_server_tick admits the jobs that are waiting, as far as the budget
// allows, into a new batch (kcm_create_batch on a stream of its own), so work admitted at different
// times runs on the device at once. A batch advances in chunks of `chunk` iterations launched
// without waiting; a tick that finds a chunk finished (CUDA event) reads every chain's state,
// retires the jobs that are done (their theta copied out), caps the others at their remaining
// iterations (kcm_set_chain_max_iters: a retired chain takes no more steps and costs no pair or
// solvation work) and launches the next chunk. A batch whose jobs have all retired is destroyed and
// its memory returned to the budget. The host thread never blocks on the device inside a tick except
// to read the state of a batch whose chunk has already finished.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <chrono>
#include <cstdint>
#include <cstring>
#include <deque>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "kcm.h"
#include "kcm_internal.h"

namespace {

// device bytes per atom and per joint of a batch (neighbour lists dominate: kMaxNbr entries of 20 B
// per atom), used to admit jobs before their batch exists; the true size is read back after creation
constexpr int64_t kBytesPerAtom = 20 * kcm::kMaxNbr + 700;
constexpr int64_t kBytesPerJoint = 400;
constexpr int64_t kBytesPerBatch = 8 << 20;

struct Job {
    int64_t id = 0;
    std::vector<int32_t> res;
    std::vector<kcm_restype> types;
    kcm_geometry geom{};
    bool has_geom = false;
    std::vector<double> theta;  // start, then the result
    int32_t max_iters = 0;
    int64_t natoms = 0;
    int32_t iters = 0;          // taken so far
    int32_t converged = 0;
    double last_dtheta = 0.0;
    int32_t state = 0;          // KCM_JOB_*
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
};

}  // namespace

struct kcm_server {
    kcm_params prm{};
    int64_t budget = 0;
    int64_t used = 0;
    int32_t max_chains = 0;
    int32_t chunk = 0;
    int32_t min_wave = 1;     // admission: wait for this many jobs ...
    double max_wait = 0.0;    // ... or until the oldest waiting job has waited this long (s)
    int64_t next_id = 1;
    std::deque<Job*> pending;
    std::vector<std::unique_ptr<Batch>> active;
    std::vector<std::unique_ptr<Job>> jobs;   // every job ever submitted, by id - 1
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
    s->finished.push_back(j->id);
}

void destroy_batch(kcm_server* s, Batch* b) {
    if (b->h) kcm_destroy(b->h);
    if (b->ev) cudaEventDestroy(b->ev);
    if (b->stream) cudaStreamDestroy(b->stream);
    s->used -= b->bytes;
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

// a finished chunk: account every chain, retire the jobs that are done, launch the next chunk
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
    std::vector<double> theta;
    bool any_done = false;
    for (size_t c = 0; c < C; ++c) {
        Job* j = b->jobs[c];
        if (j->state != KCM_JOB_RUNNING) continue;
        j->iters += it[c];
        if (it[c] > 0) j->last_dtheta = dm[c];
        const bool conv = cv[c] && j->last_dtheta < s->prm.conv_tol && it[c] > 0;
        if (er[c] != KCM_OK || conv || j->iters >= j->max_iters) any_done = true;
    }
    if (any_done) {
        const int64_t l = b->joff.back();
        theta.resize(static_cast<size_t>(l));
        rc = kcm_get_theta(b->h, theta.data(), l);
        if (rc != KCM_OK) return rc;
    }
    int running = 0;
    for (size_t c = 0; c < C; ++c) {
        Job* j = b->jobs[c];
        if (j->state != KCM_JOB_RUNNING) continue;
        const bool conv = cv[c] && j->last_dtheta < s->prm.conv_tol && it[c] > 0 && er[c] == KCM_OK;
        if (er[c] != KCM_OK || conv || j->iters >= j->max_iters) {
            j->converged = conv;
            std::copy(theta.begin() + b->joff[c], theta.begin() + b->joff[c + 1], j->theta.begin());
            retire(s, j, er[c]);
        } else {
            ++running;
        }
    }
    b->chunk_pending = false;
    if (running == 0) {
        destroy_batch(s, b);
        return KCM_OK;
    }
    return launch_chunk(s, b);
}

// admit waiting jobs (in arrival order) that fit the budget into one new batch: once min_wave jobs
// wait, once the oldest has waited max_wait, or at once when nothing runs
int admit(kcm_server* s) {
    if (s->pending.empty()) return KCM_OK;
    if (static_cast<int32_t>(s->pending.size()) < s->min_wave && !s->active.empty() &&
        now(s) - s->pending.front()->t_submit < s->max_wait)
        return KCM_OK;
    std::vector<Job*> take;
    int64_t bytes = kBytesPerBatch;
    while (!s->pending.empty() && static_cast<int32_t>(take.size()) < s->max_chains) {
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
    if (take.empty()) return KCM_OK;
    std::unique_ptr<Batch> b(new Batch());
    std::vector<kcm_topology> tops(take.size());
    for (size_t c = 0; c < take.size(); ++c) {
        Job* j = take[c];
        tops[c].n_res = static_cast<int32_t>(j->res.size());
        tops[c].res_type = j->res.data();
        tops[c].n_types = static_cast<int32_t>(j->types.size());
        tops[c].types = j->types.data();
        tops[c].geometry = j->has_geom ? &j->geom : nullptr;
    }
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        destroy_batch(s, b.get());
        s->pending.insert(s->pending.begin(), take.begin(), take.end());  // back in arrival order
        return KCM_E_CUDA;
    }
    int rc = kcm_create_batch(tops.data(), static_cast<int32_t>(tops.size()), &s->prm, b->stream, &b->h);
    if (rc != KCM_OK) {
        destroy_batch(s, b.get());
        for (Job* j : take) retire(s, j, rc);
        return KCM_OK;  // these jobs fail; the server goes on
    }
    b->bytes = kcm_device_bytes(b->h);
    s->used += b->bytes;
    b->joff.resize(take.size() + 1);
    kcm_chain_offsets(b->h, nullptr, b->joff.data());
    std::vector<double> theta;
    for (Job* j : take) theta.insert(theta.end(), j->theta.begin(), j->theta.end());
    rc = kcm_set_theta(b->h, theta.data(), static_cast<int64_t>(theta.size()));
    if (rc != KCM_OK) {
        for (Job* j : take) retire(s, j, rc);
        destroy_batch(s, b.get());
        return KCM_OK;
    }
    const double t = now(s);
    for (Job* j : take) {
        j->state = KCM_JOB_RUNNING;
        j->t_admit = t;
    }
    b->jobs = take;
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
    kcm_server* s = new (std::nothrow) kcm_server();
    if (!s) return KCM_E_NOMEM;
    s->prm = *prm;
    s->budget = hbm_budget_bytes;
    s->max_chains = max_chains_per_batch;
    s->chunk = chunk_iters;
    s->t0 = std::chrono::steady_clock::now();
    *out = s;
    return KCM_OK;
}

void kcm_server_destroy(kcm_server* s) {
    if (!s) return;
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
    std::unique_ptr<Job> j(new Job());
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
    s->jobs.push_back(std::move(j));
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
    s->active.erase(std::remove_if(s->active.begin(), s->active.end(), [](const std::unique_ptr<Batch>& b) { return !b->h; }),
                    s->active.end());
    rc = admit(s);
    if (rc != KCM_OK) return fail(s, rc, "admitting jobs failed");
    int32_t running = 0;
    for (auto& b : s->active)
        for (Job* j : b->jobs) running += j->state == KCM_JOB_RUNNING;
    if (n_waiting) *n_waiting = static_cast<int32_t>(s->pending.size());
    if (n_running) *n_running = running;
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
    for (int32_t i = 0; i < k; ++i) ids[i] = s->finished[i];
    s->finished.erase(s->finished.begin(), s->finished.begin() + k);
    *n = k;
    return KCM_OK;
}

int kcm_server_job(kcm_server* s, int64_t job_id, kcm_job_info* info, double* theta, int64_t l) {
    if (!s || job_id < 1 || job_id >= s->next_id) return KCM_E_INVAL;
    const Job* j = s->jobs[static_cast<size_t>(job_id - 1)].get();
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
