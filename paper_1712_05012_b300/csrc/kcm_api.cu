// C ABI of the KCM library (declared in include/kcm.h): handle life cycle, uploads, the captured
// per-iteration CUDA graph and host/device copies of results.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "kcm_device.h"
#include "nvtx3/nvToolsExt.h"

struct kcm_ctx {
    kcm::DevChain d;
    kcm::HostChain hc;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t side = nullptr;       // the long-list solvation kernel beside the main one
    cudaEvent_t fork = nullptr, join = nullptr;
    cudaGraphExec_t graph = nullptr;        // one iteration
    cudaGraphExec_t graph_first = nullptr;  // the loop-state reset and one iteration (a step call's first)
    cudaGraphExec_t graph_timed = nullptr;
    cudaGraphExec_t graph_io_first = nullptr;  // kcm_step_host: graph_first and graph with the host exchange
    cudaGraphExec_t graph_io = nullptr;
    kcm::Status* st_host = nullptr;          // page-locked copy of the status record (read back by the calls)
    double* theta_io = nullptr;              // kcm_step_host's page-locked angles [l] (made at its first call)
    double* theta_io_dev = nullptr;          // the device addresses of theta_io and st_host
    kcm::Status* st_io_dev = nullptr;
    cudaEvent_t ev[KCM_NUM_STAGES + 2] = {};
    int sm_count = 148;
    bool bin_cluster = true;         // the cluster binning kernel where the chain qualifies (kcm_set_binning_kernel)
    bool pdl = true;                 // captured graphs use programmatic dependent launch (dropped if a capture fails)
    std::vector<void*> allocs;       // every allocation of the handle from the pool (arena chunks included)
    char* arena = nullptr;           // small arrays are carved from chunks of kArenaChunk bytes
    size_t arena_left = 0;
    size_t bytes = 0;  // device memory held
    std::string err;
};

namespace {

thread_local std::string g_last_error;
constexpr double kPi = 3.14159265358979323846;

int set_err(kcm_ctx* h, int code, const std::string& msg) {
    if (h) h->err = msg;
    g_last_error = msg;
    return code;
}

int cuda_fail(kcm_ctx* h, cudaError_t e, const char* what) {
    std::string msg = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();
    return set_err(h, KCM_E_CUDA, msg);
}

// Device memory of the handles comes from one stream-ordered memory pool per device that the library
// owns (cudaMallocFromPoolAsync and cudaFreeAsync on the handle's stream). Freed blocks stay in the pool
// for the next handle, so making and freeing a handle never calls cudaMalloc or cudaFree, which wait for
// or serialise with the work of every other stream on the device (the serving loop makes and frees
// batches while others run). The pool lives until the process exits.
constexpr int kPoolDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kPoolDevices] = {};

cudaError_t device_pool(cudaMemPool_t* out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kPoolDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        e = cudaMemPoolCreate(&pool, &props);
        if (e != cudaSuccess) return e;
        uint64_t keep = UINT64_MAX;  // keep freed memory in the pool
        e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(pool);
            return e;
        }
        g_pool[dev] = pool;
    }
    *out = g_pool[dev];
    return cudaSuccess;
}

cudaError_t pool_alloc(kcm_ctx* h, void** p, size_t bytes) {
    cudaMemPool_t pool = nullptr;
    cudaError_t e = device_pool(&pool);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync(p, bytes, pool, h->stream);
    return e;
}

// Page-locked status records (one per handle), carved from chunks that live until the process exits: a
// cudaMallocHost / cudaFreeHost per handle would synchronise the device.
std::mutex g_pin_mu;
std::vector<kcm::Status*> g_pin_free;

kcm::Status* pinned_status() {
    std::lock_guard<std::mutex> lock(g_pin_mu);
    if (g_pin_free.empty()) {
        constexpr int kPerChunk = 64;
        void* c = nullptr;
        if (cudaMallocHost(&c, kPerChunk * sizeof(kcm::Status)) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        for (int i = kPerChunk - 1; i >= 0; --i) g_pin_free.push_back(static_cast<kcm::Status*>(c) + i);
    }
    kcm::Status* r = g_pin_free.back();
    g_pin_free.pop_back();
    return r;
}

void release_status(kcm::Status* p) {
    if (!p) return;
    std::lock_guard<std::mutex> lock(g_pin_mu);
    g_pin_free.push_back(p);
}

// Device arrays of a handle: arrays up to kArenaMax bytes are carved (256-byte aligned) from shared
// chunks, so a handle makes a few allocations instead of one per array (creation time matters to the
// serving loop); larger arrays, and those that are freed and reallocated (own = true), get their own.
constexpr size_t kArenaChunk = 8u << 20;
constexpr size_t kArenaMax = 1u << 20;

template <typename T>
int dalloc(kcm_ctx* h, T** p, size_t count, bool own = false) {
    size_t bytes = sizeof(T) * std::max<size_t>(count, 1);
    if (!own && bytes <= kArenaMax) {
        const size_t need = (bytes + 255) & ~static_cast<size_t>(255);
        if (need > h->arena_left) {
            void* c = nullptr;
            cudaError_t e = pool_alloc(h, &c, kArenaChunk);
            if (e != cudaSuccess) {
                *p = nullptr;
                cudaGetLastError();
                return set_err(h, KCM_E_NOMEM, "device allocation of " + std::to_string(kArenaChunk) + " bytes failed");
            }
            h->allocs.push_back(c);
            h->bytes += kArenaChunk;
            h->arena = static_cast<char*>(c);
            h->arena_left = kArenaChunk;
        }
        *p = reinterpret_cast<T*>(h->arena);
        h->arena += need;
        h->arena_left -= need;
        return KCM_OK;
    }
    void* q = nullptr;
    cudaError_t e = pool_alloc(h, &q, bytes);
    *p = static_cast<T*>(q);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return set_err(h, KCM_E_NOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    }
    h->allocs.push_back(*p);
    h->bytes += bytes;
    return KCM_OK;
}

template <typename T>
int upload(kcm_ctx* h, T* dst, const T* src, size_t count) {
    cudaError_t e = cudaMemcpyAsync(dst, src, sizeof(T) * count, cudaMemcpyHostToDevice, h->stream);
    return e == cudaSuccess ? KCM_OK : cuda_fail(h, e, "upload");
}

int sync(kcm_ctx* h) {
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "stream synchronize");
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "kernel launch");
    return KCM_OK;
}

// Algorithm 1: the atoms with long neighbour lists are taken by a second kernel on a side stream,
// forked after the pair kernel and joined before the wrenches (a parallel branch of the captured graph)
void enqueue_sasa(kcm_ctx* h, cudaStream_t s) {
    if (h->side && h->d.prm.solvation == 1) {
        cudaEventRecord(h->fork, s);
        cudaStreamWaitEvent(h->side, h->fork, 0);
        kcm::launch_sasa_long(h->d, h->side);
        cudaEventRecord(h->join, h->side);
        kcm::launch_sasa(h->d, s);
        cudaStreamWaitEvent(s, h->join, 0);
    } else {
        kcm::launch_sasa(h->d, s);
    }
}

// An NVTX range around the host-side enqueue of one stage (named by the KCM_STAGE_* order), so that a
// profiler's timeline groups each stage's kernels, in the captured graphs too (their nodes are made
// inside the ranges). Without a profiler attached the calls return at once.
struct StageRange {
    explicit StageRange(int stage) {
        static const char* kNames[KCM_NUM_STAGES] = {"kcm:kinematics", "kcm:binning", "kcm:pairs", "kcm:solvation",
                                                     "kcm:torques_step"};
        nvtxRangePushA(kNames[stage]);
    }
    ~StageRange() { nvtxRangePop(); }
    StageRange(const StageRange&) = delete;
    StageRange& operator=(const StageRange&) = delete;
};

void enqueue_stages(kcm_ctx* h, bool step) {
    kcm::DevChain d = h->d;  // the cluster binning kernel, where it bins, forms the grid
    d.grid_in_bin = d.bin_c ? 1 : 0;
    { StageRange r(KCM_STAGE_KINEMATICS); kcm::launch_fk(d, h->stream); }
    { StageRange r(KCM_STAGE_BINNING); kcm::launch_binning(d, h->stream); }
    { StageRange r(KCM_STAGE_PAIRS); kcm::launch_pairs(h->d, h->stream); }
    { StageRange r(KCM_STAGE_SOLVATION); enqueue_sasa(h, h->stream); }
    {
        StageRange r(KCM_STAGE_TORQUES);
        if (step) kcm::launch_torques_step(h->d, h->stream);
        else kcm::launch_torques(h->d, h->stream);
    }
}

void enqueue_evaluation(kcm_ctx* h) { enqueue_stages(h, false); }

void enqueue_iteration(kcm_ctx* h) { enqueue_stages(h, true); }

int read_status(kcm_ctx* h, kcm::Status* st) {
    kcm::Status* dst = h->st_host ? h->st_host : st;  // page-locked: an asynchronous copy, one wait
    cudaError_t e = cudaMemcpyAsync(dst, h->d.status, sizeof(kcm::Status), cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "status copy");
    int rc = sync(h);
    if (rc == KCM_OK && dst != st) *st = *dst;
    return rc;
}

int status_code(kcm_ctx* h, const kcm::Status& st) {
    if (st.error & kcm::kErrNonfinite) return set_err(h, KCM_E_NONFINITE, "a torque or coordinate is not finite");
    if (st.error & kcm::kErrTimeout) return set_err(h, KCM_E_TIMEOUT, "a bounded device wait gave up");
    if (st.error & kcm::kErrOverflow)
        return set_err(h, KCM_E_OVERFLOW, "an atom has more than " + std::to_string(kcm::kMaxNbr) + " solvation neighbours");
    return KCM_OK;
}

// evaluate at the current theta (no step), synchronise and check the device status
int evaluate(kcm_ctx* h) {
    kcm::launch_reset_loop(h->d, h->stream);
    enqueue_evaluation(h);
    kcm::Status st;
    int rc = read_status(h, &st);
    if (rc != KCM_OK) return rc;
    return status_code(h, st);
}

// Captures what `enqueue` launches on the handle's stream into an executable graph. Its kernels allow
// programmatic dependent launch (each waits for the previous grid of the stream at its start, so only
// launch latency overlaps); should a capture or instantiation fail that way, it is taken again without
// and the handle stops asking for it.
template <class F>
cudaError_t capture_graph(kcm_ctx* h, F enqueue, cudaGraphExec_t* out) {
    cudaError_t e = cudaSuccess;
    for (int attempt = 0; attempt < 2; ++attempt) {
        h->d.pdl = h->pdl ? 1 : 0;
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            enqueue();
            e = cudaStreamEndCapture(h->stream, &g);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
        if (g) cudaGraphDestroy(g);
        h->d.pdl = 0;
        if (e == cudaSuccess) return e;
        *out = nullptr;
        if (!h->pdl) return e;
        (void)cudaGetLastError();
        h->pdl = false;
    }
    return e;
}

// the iteration graph, and the same preceded by the loop-state reset (the first launch of a step call)
int build_graph(kcm_ctx* h) {
    if (h->graph && h->graph_first) return KCM_OK;
    for (int first = 0; first < 2; ++first) {
        cudaGraphExec_t* out = first ? &h->graph_first : &h->graph;
        if (*out) continue;
        const cudaError_t e = capture_graph(
            h,
            [&] {
                if (first) kcm::launch_reset_loop(h->d, h->stream);
                enqueue_iteration(h);
            },
            out);
        if (e != cudaSuccess) return cuda_fail(h, e, "graph capture");
    }
    return KCM_OK;
}

// kcm_step_host's graphs: graph_first and graph again, with the host exchange of DevChain (theta_io,
// status_io, io_import) set during their capture only. Returns false (and the call copies instead) where
// the page-locked buffers are not to be had.
int build_io_graphs(kcm_ctx* h, bool* ok) {
    *ok = false;
    if (!h->st_host) return KCM_OK;
    if (!h->theta_io) {
        void* p = nullptr;
        cudaError_t e = cudaHostAlloc(&p, sizeof(double) * std::max(h->d.l, 1), cudaHostAllocMapped);
        if (e == cudaSuccess) {
            h->theta_io = static_cast<double*>(p);
            void* dp = nullptr;
            e = cudaHostGetDevicePointer(&dp, p, 0);
            h->theta_io_dev = static_cast<double*>(dp);
        }
        if (e == cudaSuccess) {
            void* dp = nullptr;
            e = cudaHostGetDevicePointer(&dp, h->st_host, 0);
            h->st_io_dev = static_cast<kcm::Status*>(dp);
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            if (h->theta_io) cudaFreeHost(h->theta_io);
            h->theta_io = nullptr;
            return KCM_OK;
        }
    }
    for (int first = 0; first < 2; ++first) {
        cudaGraphExec_t* out = first ? &h->graph_io_first : &h->graph_io;
        if (*out) continue;
        h->d.theta_io = h->theta_io_dev;
        h->d.status_io = h->st_io_dev;
        h->d.io_import = first;
        const cudaError_t e = capture_graph(
            h,
            [&] {
                if (first) kcm::launch_reset_loop(h->d, h->stream);
                enqueue_iteration(h);
            },
            out);
        h->d.theta_io = nullptr;
        h->d.status_io = nullptr;
        h->d.io_import = 0;
        if (e != cudaSuccess) return cuda_fail(h, e, "graph capture");
    }
    *ok = true;
    return KCM_OK;
}

// the loop-state reset and n_iters iterations: the first with the reset in one graph launch
int launch_steps(kcm_ctx* h, int32_t n_iters) {
    if (n_iters == 0) {
        kcm::launch_reset_loop(h->d, h->stream);
        return KCM_OK;
    }
    for (int32_t i = 0; i < n_iters; ++i) {
        cudaError_t e = cudaGraphLaunch(i == 0 ? h->graph_first : h->graph, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "graph launch");
    }
    return KCM_OK;
}

// the same iteration with an event recorded before each stage and after the last
int build_timed_graph(kcm_ctx* h) {
    if (h->graph_timed) return KCM_OK;
    for (int i = 0; i < KCM_NUM_STAGES + 2; ++i) {
        if (!h->ev[i]) {
            cudaError_t e = cudaEventCreate(&h->ev[i]);
            if (e != cudaSuccess) return cuda_fail(h, e, "event create");
        }
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(h, e, "begin capture");
    cudaStream_t s = h->stream;
    cudaEventRecordWithFlags(h->ev[1], s, cudaEventRecordExternal);
    kcm::DevChain d = h->d;  // as in enqueue_stages
    d.grid_in_bin = d.bin_c ? 1 : 0;
    { StageRange r(KCM_STAGE_KINEMATICS); kcm::launch_fk(d, s); }
    cudaEventRecordWithFlags(h->ev[2], s, cudaEventRecordExternal);
    { StageRange r(KCM_STAGE_BINNING); kcm::launch_binning(d, s); }
    cudaEventRecordWithFlags(h->ev[3], s, cudaEventRecordExternal);
    { StageRange r(KCM_STAGE_PAIRS); kcm::launch_pairs(h->d, s); }
    cudaEventRecordWithFlags(h->ev[4], s, cudaEventRecordExternal);
    { StageRange r(KCM_STAGE_SOLVATION); enqueue_sasa(h, s); }
    cudaEventRecordWithFlags(h->ev[5], s, cudaEventRecordExternal);
    { StageRange r(KCM_STAGE_TORQUES); kcm::launch_torques_step(h->d, s); }
    cudaEventRecordWithFlags(h->ev[6], s, cudaEventRecordExternal);
    e = cudaStreamEndCapture(s, &g);
    if (e != cudaSuccess) return cuda_fail(h, e, "end capture");
    e = cudaGraphInstantiate(&h->graph_timed, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        h->graph_timed = nullptr;
        return cuda_fail(h, e, "graph instantiate");
    }
    return KCM_OK;
}

int check_handle(kcm_ctx* h) { return h ? KCM_OK : set_err(nullptr, KCM_E_INVAL, "NULL handle"); }

// each double as the float pair (hi, lo), hi = nearest float, lo = nearest float to the rest, stored
// in the 8 bytes of a double slot (the mixed kernels' double-float format)
std::vector<double> pack_df(const std::vector<double>& v) {
    std::vector<double> out(v.size());
    for (size_t i = 0; i < v.size(); ++i) {
        float pr[2];
        pr[0] = static_cast<float>(v[i]);
        pr[1] = static_cast<float>(v[i] - static_cast<double>(pr[0]));
        std::memcpy(&out[i], pr, sizeof(pr));
    }
    return out;
}

void dfree(kcm_ctx* h, void* p, size_t bytes) {
    if (!p) return;
    cudaFreeAsync(p, h->stream);  // back to the pool after the stream's earlier work
    h->allocs.erase(std::remove(h->allocs.begin(), h->allocs.end(), p), h->allocs.end());
    h->bytes -= bytes;
}

void drop_graphs(kcm_ctx* h) {
    if (h->graph) cudaGraphExecDestroy(h->graph);
    if (h->graph_first) cudaGraphExecDestroy(h->graph_first);
    if (h->graph_timed) cudaGraphExecDestroy(h->graph_timed);
    if (h->graph_io_first) cudaGraphExecDestroy(h->graph_io_first);
    if (h->graph_io) cudaGraphExecDestroy(h->graph_io);
    h->graph = nullptr;
    h->graph_first = nullptr;
    h->graph_timed = nullptr;
    h->graph_io_first = nullptr;
    h->graph_io = nullptr;
}

// the pair kernel's grid: one block per W atoms, or with pair_persistent one block per resident slot
// (SMs x resident blocks per SM of the kernel's current form)
int set_pair_grid(kcm_ctx* h) {
    kcm::DevChain& d = h->d;
    d.pair_grid_cap = 0;
    if (!d.pair_persistent) return KCM_OK;
    const int b = kcm::pair_resident_blocks(d);
    if (b <= 0) return cuda_fail(h, cudaGetLastError(), "occupancy query");
    d.pair_grid_cap = b * h->sm_count;
    return KCM_OK;
}

// Applies a requested cell edge: the stencil (one cell on either side when the edge reaches the
// largest interaction range, two when it is smaller; the device raises the edge to the smallest
// legal one for that stencil), each chain's cell cap (a chain's grid is coarsened to fit it; half
// the edge needs eight times the cells), the cell arrays (grown when the caps outgrow them), and
// drops the captured graphs, which hold the old launch parameters.
int set_cell_size(kcm_ctx* h, double cell_size) {
    kcm::DevChain& d = h->d;
    const kcm::HostChain& hc = h->hc;
    const int stencil = (cell_size > 0.0 && cell_size < d.rmax) ? 2 : 1;
    std::vector<int> ccap(hc.nchains);
    long long tot = 0;
    for (int ch = 0; ch < hc.nchains; ++ch) {
        const long long nc = hc.atom_off[ch + 1] - hc.atom_off[ch];
        long long cap = hc.nchains == 1 ? std::max(8 * nc, 65536LL) : std::max(8 * nc, 4096LL);
        if (stencil == 2) cap *= 8;
        if (cap > (1LL << 30)) cap = 1LL << 30;
        ccap[ch] = static_cast<int>(cap);
        tot += cap;
    }
    if (tot > (1LL << 30)) return set_err(h, KCM_E_INVAL, "the batch needs more than 2^30 cells");
    if (h->stream) {  // nothing of the old configuration in flight
        int rc = sync(h);
        if (rc) return rc;
    }
    drop_graphs(h);
    if (tot > d.cell_alloc) {  // grow the cell arrays (counts start at zero; the scan keeps them so)
        dfree(h, d.cell_count, sizeof(int) * std::max<size_t>(d.cell_alloc, 1));
        dfree(h, d.cell_start, sizeof(int) * (d.cell_alloc + 1));
        dfree(h, d.scan_part, sizeof(int) * std::max<size_t>((d.cell_alloc + kcm::kScanCells - 1) / kcm::kScanCells, 1));
        d.cell_count = d.cell_start = d.scan_part = nullptr;
        d.cell_alloc = 0;
        const size_t nb = (static_cast<size_t>(tot) + kcm::kScanCells - 1) / kcm::kScanCells;
        int rc;
        if ((rc = dalloc(h, &d.cell_count, static_cast<size_t>(tot), true)) ||
            (rc = dalloc(h, &d.cell_start, static_cast<size_t>(tot) + 1, true)) || (rc = dalloc(h, &d.scan_part, nb, true)))
            return rc;
        cudaError_t e = cudaMemsetAsync(d.cell_count, 0, sizeof(int) * static_cast<size_t>(tot), h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "memset");
        d.cell_alloc = tot;
    }
    d.cell_cap = static_cast<int>(tot);
    d.scan_blocks = (d.cell_cap + kcm::kScanCells - 1) / kcm::kScanCells;
    d.scan_fused = d.cell_cap <= kcm::kScanFusedMaxCells;
    d.stencil = stencil;
    d.prm.cell_size = cell_size;
    if (int prc = set_pair_grid(h)) return prc;  // the stencil picks the pair kernel's form
    cudaError_t fe = kcm::plan_bin_cluster(d, h->bin_cluster);  // the cell cap sizes its cell ranges
    if (fe != cudaSuccess) return cuda_fail(h, fe, "binning kernel attributes");
    int rc = upload(h, d.ccap, ccap.data(), hc.nchains);
    return rc ? rc : sync(h);
}

}  // namespace

extern "C" {

int kcm_params_default(kcm_params* p) {
    if (!p) return KCM_E_INVAL;
    p->cutoff = 10.0;
    p->vdw_cutoff = 0.0;
    p->kappa = 1e-3;
    p->dtheta_max = 0.02;
    p->w14_elec = 0.5;
    p->w14_vdw = 0.5;
    p->r_probe = 1.4;
    p->delta_r = 0.02;
    p->coulomb_k = 332.0636;
    p->conv_tol = 1e-4;
    p->cell_size = 0.0;
    p->n_sample = 256;
    p->solvation = 1;
    p->precision = KCM_FP64;
    p->step_mode = KCM_STEP_CLAMP;
    p->side_joints = 0;
    return KCM_OK;
}

static int create_impl(const kcm_topology* tops, int32_t n_chains, const kcm_params* prm, void* cuda_stream, kcm_handle* out) {
    if (!out) return set_err(nullptr, KCM_E_INVAL, "out is NULL");
    *out = nullptr;
    if (!tops || n_chains < 1) return set_err(nullptr, KCM_E_INVAL, "need at least one topology");
    std::string err;
    int rc = kcm::validate_params(prm, &err);
    if (rc != KCM_OK) return set_err(nullptr, rc, err);
    kcm_ctx* h = new (std::nothrow) kcm_ctx();
    if (!h) return set_err(nullptr, KCM_E_NOMEM, "host allocation failed");
    auto bail = [&](int code) {
        std::string msg = h->err;
        kcm_destroy(h);
        g_last_error = msg;
        return code;
    };
    {
        std::vector<kcm::HostChain> parts(n_chains);
        for (int32_t c = 0; c < n_chains; ++c) {
            rc = kcm::build_host_chain(&tops[c], &parts[c], &err);
            if (rc != KCM_OK) {
                set_err(h, rc, n_chains > 1 ? "chain " + std::to_string(c) + ": " + err : err);
                return bail(rc);
            }
        }
        kcm::concat_chains(parts, &h->hc);
    }

    int dev = 0, major = 0, minor = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_err(h, KCM_E_NODEVICE, std::string("no usable CUDA device: ") + cudaGetErrorString(e));
        return bail(KCM_E_NODEVICE);
    }
    if (cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        h->sm_count = 148;
    }
    if (major != 10 || minor != 3) {
        set_err(h, KCM_E_NODEVICE, "this library is built for sm_103 (B300); device is sm_" + std::to_string(major) +
                                       std::to_string(minor));
        return bail(KCM_E_NODEVICE);
    }
    if (cuda_stream) {
        h->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { cuda_fail(h, e, "stream create"); return bail(KCM_E_CUDA); }
        h->own_stream = true;
    }

    h->st_host = pinned_status();  // NULL: status reads then go through pageable memory
    if (prm->solvation == 1) {  // the long solvation lists run beside the main solvation kernel
        e = cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->join, cudaEventDisableTiming);
        if (e != cudaSuccess) { cuda_fail(h, e, "side stream create"); return bail(KCM_E_CUDA); }
    }
    const kcm::HostChain& hc = h->hc;
    kcm::DevChain& d = h->d;
    d.prm = *prm;
    d.pair_tile = prm->precision == KCM_MIXED && hc.n >= kcm::kPairTileDefaultAtoms ? KCM_PAIR_CELL_TILES
                                                                                 : KCM_PAIR_WARP_PER_ATOM;
    d.m = hc.m; d.n = hc.n; d.l = hc.l; d.L = hc.L; d.N = prm->n_sample;
    d.ls = prm->side_joints ? hc.ls : 0;
    d.nmv = prm->side_joints ? static_cast<int>(hc.mv_atom.size()) : 0;
    for (int h0 = 0; h0 < hc.L; h0 += 32) {  // the wrench kernel stages one 32-link tile in shared memory
        const int h1 = std::min(h0 + 32, hc.L);
        if (hc.link_start[h1] - hc.link_start[h0] > kcm::kWrenchTileAtoms)
            return bail(set_err(h, KCM_E_INVAL, "32 consecutive links hold more atoms than the wrench tile"));
    }
    const int fkq = kcm::fk_block_joints();
    // scan blocks spanned by the longest chain with J joints per lane
    auto chain_span = [&](int J) {
        int span = 0;
        for (int c = 0; c < hc.nchains; ++c) {
            const int j0 = hc.joint_off[c], j1 = hc.joint_off[c + 1];
            if (j1 > j0) span = std::max(span, (j1 - 1) / (fkq * J) - j0 / (fkq * J) + 1);
        }
        return span;
    };
    // Batches take two joints per lane wherever every chain then lies within kcm::kFkTreeTiles scan blocks
    // (measured on the 512-chain batch: kinematics 213, 185, 191 and 216 us with 1, 2, 4 and 8 joints per
    // lane); otherwise as few as keep the scan blocks within what k_fk_tiles scans, and at least two for a
    // single chain beyond the tree (8,000-residue chain: 366.7 -> 363.0 us per iteration with two; the
    // 1,000-residue chain, within the tree, 94.1 us with one against 99.9 us with two).
    if (hc.nchains > 1 && chain_span(2) <= kcm::fk_tree_tiles()) {
        d.fk_j = 2;
    } else {
        d.fk_j = kcm::fk_joints_per_lane(d.l);
        if (d.fk_j == 1 && chain_span(1) > kcm::fk_tree_tiles()) d.fk_j = 2;
    }
    d.ntiles = (d.l + fkq * d.fk_j - 1) / (fkq * d.fk_j);
    // every chain within kcm::kFkTreeTiles scan blocks: the apply kernel reduces its chain's earlier block
    // products itself, and no kernel scans all of them
    d.fk_chain_tree = chain_span(d.fk_j) <= kcm::fk_tree_tiles() ? 1 : 0;
    d.ltiles = (d.L + 31) / 32;
    {
        const int rb = kcm::wrench_resident_blocks(d);
        if (rb < 0) cudaGetLastError();
        d.wrench_static = rb > 0 && (long long)rb * h->sm_count >= d.ltiles ? 1 : 0;
    }
    d.nchains = hc.nchains;
    d.rcut2 = prm->cutoff * prm->cutoff;
    double rv = prm->vdw_cutoff > 0.0 ? prm->vdw_cutoff : prm->cutoff;
    d.rvdw2 = rv * rv;
    double rmaxR = 0.0;
    for (double r : hc.R) rmaxR = std::max(rmaxR, r);
    d.roff_max = rmaxR + prm->r_probe;
    d.rmax = std::max(prm->cutoff, rv);
    if (prm->solvation) d.rmax = std::max(d.rmax, 2.0 * d.roff_max + prm->delta_r + 0.02);
    d.s_base = d.rmax * (1.0 + 1e-5) + 0.01;
    d.f_K = (float)prm->coulomb_k;
    d.f_w14e = (float)prm->w14_elec;
    d.f_w14v = (float)prm->w14_vdw;
    d.f_rc2 = (float)d.rcut2;
    d.f_rv2 = (float)d.rvdw2;
    d.f_rall2 = (float)(d.rmax * d.rmax) + 0.01f;  // FP32 candidate range, padded for rounding
    d.f_dr = (float)prm->delta_r;
    d.f_invN = 1.0f / (float)d.N;

    const int n = d.n, l = d.l, L = d.L, N = d.N;
    const size_t nn = static_cast<size_t>(n);
    if ((rc = dalloc(h, &d.r0, 3 * nn)) || (rc = dalloc(h, &d.link, nn)) || (rc = dalloc(h, &d.link_start, L + 1)) ||
        (rc = dalloc(h, &d.u0, 3 * l)) || (rc = dalloc(h, &d.step0, 3 * l)) || (rc = dalloc(h, &d.aprm64, nn)) ||
        (rc = dalloc(h, &d.aprm32, nn)) || (rc = dalloc(h, &d.G0, nn)) || (rc = dalloc(h, &d.qfx, nn)) ||
        (rc = dalloc(h, &d.exm, nn)) || (rc = dalloc(h, &d.m14m, nn)) || (rc = dalloc(h, &d.Q64, 3 * N)) ||
        (rc = dalloc(h, &d.Q32, 3 * N)) || (rc = dalloc(h, &d.Q4, N)) || (rc = dalloc(h, &d.theta, l + d.ls)) || (rc = dalloc(h, &d.dtheta, l + d.ls)) ||
        (rc = dalloc(h, &d.tau, l + d.ls)) || (rc = dalloc(h, &d.G, 12 * (size_t)l)) ||
        (rc = dalloc(h, &d.tileP, 12 * (size_t)d.ntiles)) || (rc = dalloc(h, &d.tileE, 12 * (size_t)d.ntiles)) || (rc = dalloc(h, &d.u0df, 3 * l)) ||
        (rc = dalloc(h, &d.step0df, 3 * l)) || (rc = dalloc(h, &d.r0df, 3 * nn)) || (rc = dalloc(h, &d.rdf, 3 * nn)) ||
        (rc = dalloc(h, &d.ucurdf, 3 * l)) || (rc = dalloc(h, &d.pcurdf, 3 * l)) || (rc = dalloc(h, &d.G0f, nn)) ||
        (rc = dalloc(h, &d.M, 12 * (size_t)L)) || (rc = dalloc(h, &d.ucur, 3 * l)) || (rc = dalloc(h, &d.pcur, 3 * l)) ||
        (rc = dalloc(h, &d.r, 3 * nn)) || (rc = dalloc(h, &d.key, nn)) || (rc = dalloc(h, &d.rank, nn)) ||
        (rc = dalloc(h, &d.sorted, nn)) || (hc.nchains > 1 && (rc = dalloc(h, &d.slot_chain, nn))) || (rc = dalloc(h, &d.sorted_tmp, nn)) || (rc = dalloc(h, &d.slot_cell, nn)) || (rc = dalloc(h, &d.smask, nn)) || (rc = dalloc(h, &d.spos64, nn)) ||
        (rc = dalloc(h, &d.spos32, nn)) || (rc = dalloc(h, &d.sprm32, nn)) || (rc = dalloc(h, &d.sprm64, nn)) ||
        (rc = dalloc(h, &d.Fpair, 3 * nn)) || (rc = dalloc(h, &d.Fpx, 3 * nn)) || (rc = dalloc(h, &d.Fov, 3 * nn)) || (rc = dalloc(h, &d.Fox, 3 * nn)) ||
        (rc = dalloc(h, &d.gflag, nn)) || (rc = dalloc(h, &d.Fcav, 3 * nn)) || (rc = dalloc(h, &d.nbr_cnt, nn)) ||
        (rc = dalloc(h, &d.nbr, nn * kcm::kMaxNbr)) || (rc = dalloc(h, &d.nbr_off, nn * kcm::kMaxNbr)) ||
        (rc = dalloc(h, &d.covered, nn)) || (rc = dalloc(h, &d.long_atoms, nn)) || (rc = dalloc(h, &d.epair, 2 * nn)) || (rc = dalloc(h, &d.pstat, nn)) ||
        (rc = dalloc(h, &d.sstat, nn)) || (rc = dalloc(h, &d.esolv, nn)) ||
        (rc = dalloc(h, &d.tileS, 6 * (size_t)d.ltiles)) || (rc = dalloc(h, &d.tileStat, d.ltiles)) ||
        (rc = dalloc(h, &d.lb_epoch, 1)) ||
        (rc = dalloc(h, &d.Ftot, 3 * nn)) || (rc = dalloc(h, &d.Fcav64, 3 * nn)) ||
        (rc = dalloc(h, &d.grid, hc.nchains)) || (rc = dalloc(h, &d.status, 1)) ||
        (rc = dalloc(h, &d.atom_chain, nn)) || (rc = dalloc(h, &d.joint_chain, l)) || (rc = dalloc(h, &d.link_chain, L)) ||
        (rc = dalloc(h, &d.joint_off, hc.nchains + 1)) || (rc = dalloc(h, &d.ccap, hc.nchains)) ||
        (rc = dalloc(h, &d.cbox, 6 * (size_t)hc.nchains)) || (rc = dalloc(h, &d.chain_done, hc.nchains)) ||
        (rc = dalloc(h, &d.chain_iters, hc.nchains)) || (rc = dalloc(h, &d.chain_maxit, hc.nchains)) ||
        (rc = dalloc(h, &d.chain_err, hc.nchains)) || (rc = dalloc(h, &d.chain_maxdt, hc.nchains)) ||
        (rc = dalloc(h, &d.chain_maxtau, hc.nchains)) || (rc = dalloc(h, &d.chain_lastdt, hc.nchains)) ||
        (rc = dalloc(h, &d.chain_E, 3 * (size_t)hc.nchains)) || (rc = dalloc(h, &d.gseg, l)) ||
        (rc = dalloc(h, &d.jhead, l)) || (rc = dalloc(h, &d.jfixed, l + d.ls)) || (rc = dalloc(h, &d.lflag, L)) ||
        (rc = dalloc(h, &d.tileF, d.ntiles)) || (rc = dalloc(h, &d.tileT, d.ltiles)))
        return bail(rc);

    // per-atom constants
    std::vector<kcm::dbl4> ap64(n);
    std::vector<float4> ap32(n);
    std::vector<double> G0(n);
    std::vector<long long> qfx(n);
    std::vector<int> gflag(n);
    std::vector<float> G0f(n);
    for (int a = 0; a < n; ++a) {
        double roff = hc.R[a] + prm->r_probe;
        ap64[a] = kcm::make_dbl4(hc.q[a], std::sqrt(hc.eps[a]), hc.R[a], roff);
        ap32[a] = make_float4((float)hc.q[a], (float)std::sqrt(hc.eps[a]), (float)hc.R[a], (float)roff);
        G0[a] = 4.0 * kPi * kcm::gamma_of_class(hc.cls[a]) * roff * roff;  // G^cav_{i,0} of Algorithm 1
        qfx[a] = std::llrint(G0[a] / (static_cast<double>(N) * prm->delta_r) * kcm::kFxScale);
        gflag[a] = G0[a] != 0.0;
        G0f[a] = static_cast<float>(G0[a]);
    }
    std::vector<double> Q64(3 * (size_t)N);
    kcm::sample_points(N, Q64.data());
    std::vector<float> Q32(Q64.begin(), Q64.end());
    std::vector<float4> Q4(N);
    for (int k = 0; k < N; ++k) Q4[k] = make_float4(Q32[3 * k], Q32[3 * k + 1], Q32[3 * k + 2], 0.0f);
    std::vector<double> ident = {1, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0};
    if (prm->precision == KCM_MIXED) ident = pack_df(ident);  // base-link poses in the mixed kernels' format
    std::vector<int> atom_chain(n), joint_chain(l), link_chain(L);
    std::vector<unsigned char> jhead(l, 0), lflag(L, 0);
    for (int ch = 0; ch < hc.nchains; ++ch) {
        for (int a = hc.atom_off[ch]; a < hc.atom_off[ch + 1]; ++a) atom_chain[a] = ch;
        for (int j = hc.joint_off[ch]; j < hc.joint_off[ch + 1]; ++j) joint_chain[j] = ch;
        for (int k = hc.link_off[ch]; k < hc.link_off[ch + 1]; ++k) link_chain[k] = ch;
        jhead[hc.joint_off[ch]] = 1;
        lflag[hc.link_off[ch]] |= 1;
        lflag[hc.link_off[ch + 1] - 1] |= 2;
    }
    std::vector<double> u0df = pack_df(hc.u0), step0df = pack_df(hc.step0), r0df = pack_df(hc.zp_rel);
    if ((rc = upload(h, d.r0, hc.zp_rel.data(), 3 * nn)) || (rc = upload(h, d.link, hc.link.data(), nn)) ||
        (rc = upload(h, d.link_start, hc.link_start.data(), L + 1)) || (rc = upload(h, d.u0, hc.u0.data(), 3 * l)) ||
        (rc = upload(h, d.step0, hc.step0.data(), 3 * l)) || (rc = upload(h, d.aprm64, ap64.data(), nn)) ||
        (rc = upload(h, d.aprm32, ap32.data(), nn)) || (rc = upload(h, d.G0, G0.data(), nn)) ||
        (rc = upload(h, d.qfx, qfx.data(), nn)) || (rc = upload(h, d.gflag, gflag.data(), nn)) || (rc = upload(h, d.G0f, G0f.data(), nn)) ||
        (rc = upload(h, d.exm, reinterpret_cast<const unsigned long long*>(hc.ex_mask.data()), nn)) ||
        (rc = upload(h, d.m14m, reinterpret_cast<const unsigned long long*>(hc.m14_mask.data()), nn)) ||
        (rc = upload(h, d.Q64, Q64.data(), 3 * (size_t)N)) || (rc = upload(h, d.Q32, Q32.data(), 3 * (size_t)N)) || (rc = upload(h, d.Q4, Q4.data(), N)) ||
        (rc = upload(h, d.atom_chain, atom_chain.data(), nn)) || (rc = upload(h, d.joint_chain, joint_chain.data(), l)) ||
        (rc = upload(h, d.link_chain, link_chain.data(), L)) || (rc = upload(h, d.joint_off, hc.joint_off.data(), hc.nchains + 1)) ||
        (rc = upload(h, d.jhead, jhead.data(), l)) ||
        (rc = upload(h, d.lflag, lflag.data(), L)) || (rc = upload(h, d.u0df, u0df.data(), 3 * l)) ||
        (rc = upload(h, d.step0df, step0df.data(), 3 * l)) || (rc = upload(h, d.r0df, r0df.data(), 3 * nn)))
        return bail(rc);
    if (hc.nchains > 1 && prm->precision == KCM_MIXED &&  // the per-chain binning kernel's chain ranges
        ((rc = dalloc(h, &d.atom_off, hc.nchains + 1)) || (rc = upload(h, d.atom_off, hc.atom_off.data(), hc.nchains + 1))))
        return bail(rc);
    if ((rc = set_cell_size(h, prm->cell_size))) return bail(rc);  // cell caps and arrays
    // the offsets the FK reads: the static ones, or with side-chain joints a copy that k_side_fk
    // rewrites for the side atoms they move
    double* r0mode = prm->precision == KCM_MIXED ? d.r0df : d.r0;
    if (d.ls > 0) {
        std::vector<int2> mv(d.nmv);
        for (int k = 0; k < d.nmv; ++k) mv[k] = make_int2(hc.mv_chi0[k], hc.mv_nk[k]);
        const size_t ls = static_cast<size_t>(d.ls);
        std::vector<int> chi_tile(d.ltiles + 1, d.ls);  // side-chain joints by the wrench tile of their link
        for (int c = d.ls - 1; c >= 0; --c) chi_tile[hc.link[hc.chi_b[c]] / 32] = c;
        for (int t = d.ltiles - 1; t >= 0; --t) chi_tile[t] = std::min(chi_tile[t], chi_tile[t + 1]);
        for (int t = 0; t < d.ltiles; ++t)  // one thread of the wrench kernel per side-chain joint of a tile
            if (chi_tile[t + 1] - chi_tile[t] > kcm::kWrenchWarps * 32)
                return bail(set_err(h, KCM_E_INVAL, "internal: a wrench tile holds too many side-chain joints"));
        const bool mixed = prm->precision == KCM_MIXED;  // the bond tables in the kernels' number format
        const std::vector<double> p0 = mixed ? pack_df(hc.chi_p0) : hc.chi_p0, u0 = mixed ? pack_df(hc.chi_u0) : hc.chi_u0,
                                  inv = mixed ? pack_df(hc.chi_inv) : hc.chi_inv;
        if ((rc = dalloc(h, &d.r0fk, 3 * nn)) || (rc = dalloc(h, &d.chi_a, ls)) || (rc = dalloc(h, &d.chi_b, ls)) ||
            (rc = dalloc(h, &d.chi_end, ls)) || (rc = dalloc(h, &d.chi_p0, 3 * ls)) || (rc = dalloc(h, &d.chi_u0, 3 * ls)) ||
            (rc = dalloc(h, &d.chi_inv, ls)) || (rc = dalloc(h, &d.mv_atom, d.nmv)) || (rc = dalloc(h, &d.mv_chi, d.nmv)) ||
            (rc = upload(h, d.chi_a, hc.chi_a.data(), ls)) || (rc = upload(h, d.chi_b, hc.chi_b.data(), ls)) ||
            (rc = upload(h, d.chi_end, hc.chi_end.data(), ls)) || (rc = upload(h, d.chi_p0, p0.data(), 3 * ls)) ||
            (rc = upload(h, d.chi_u0, u0.data(), 3 * ls)) || (rc = upload(h, d.chi_inv, inv.data(), ls)) ||
            (rc = upload(h, d.mv_atom, hc.mv_atom.data(), d.nmv)) || (rc = upload(h, d.mv_chi, mv.data(), d.nmv)) ||
            (rc = dalloc(h, &d.chi_tile, d.ltiles + 1)) || (rc = upload(h, d.chi_tile, chi_tile.data(), d.ltiles + 1)))
            return bail(rc);
        e = cudaMemcpyAsync(d.r0fk, r0mode, sizeof(double) * 3 * nn, cudaMemcpyDeviceToDevice, h->stream);
        if (e != cudaSuccess) { cuda_fail(h, e, "offset copy"); return bail(KCM_E_CUDA); }
    } else {
        d.r0fk = r0mode;
    }
    e = cudaMemsetAsync(d.theta, 0, sizeof(double) * (l + d.ls), h->stream);
    // no tile total published yet, launch number 0 (the torque kernel's flags are launch numbers)
    if (e == cudaSuccess) e = cudaMemsetAsync(d.tileStat, 0, sizeof(unsigned int) * d.ltiles, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.lb_epoch, 0, sizeof(unsigned int), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.jfixed, 0, l + d.ls, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.Fcav, 0, sizeof(long long) * 3 * nn, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.covered, 0, sizeof(int) * nn, h->stream);
    if (e != cudaSuccess) { cuda_fail(h, e, "memset"); return bail(KCM_E_CUDA); }
    {
        std::vector<int> maxit(hc.nchains, INT32_MAX);  // no cap until kcm_set_chain_max_iters
        rc = upload(h, d.chain_maxit, maxit.data(), hc.nchains);
        if (rc) return bail(rc);
    }
    for (int ch = 0; ch < hc.nchains && rc == KCM_OK; ++ch)  // the base link of every chain stays at the origin
        rc = upload(h, d.M + 12 * (size_t)hc.link_off[ch], ident.data(), 12);
    if (rc) return bail(rc);
    kcm::launch_init_status(d, h->stream);
    rc = sync(h);
    if (rc != KCM_OK) return bail(rc);
    *out = h;
    return KCM_OK;
}

int kcm_create(const kcm_topology* top, const kcm_params* prm, void* cuda_stream, kcm_handle* out) {
    return create_impl(top, 1, prm, cuda_stream, out);
}

int kcm_create_batch(const kcm_topology* tops, int32_t n_chains, const kcm_params* prm, void* cuda_stream,
                     kcm_handle* out) {
    return create_impl(tops, n_chains, prm, cuda_stream, out);
}

int32_t kcm_nchains(kcm_handle h) { return h ? h->d.nchains : -1; }

int kcm_chain_offsets(kcm_handle h, int64_t* atom_off, int64_t* joint_off) {
    if (check_handle(h)) return KCM_E_INVAL;
    for (int c = 0; c <= h->hc.nchains; ++c) {
        if (atom_off) atom_off[c] = h->hc.atom_off[c];
        if (joint_off) joint_off[c] = h->hc.joint_off[c];
    }
    return KCM_OK;
}

int kcm_chain_energies(kcm_handle h, double* E) {
    if (check_handle(h)) return KCM_E_INVAL;
    if (!E) return set_err(h, KCM_E_INVAL, "E is NULL");
    int rc = evaluate(h);
    if (rc) return rc;
    cudaError_t e = cudaMemcpyAsync(E, h->d.chain_E, sizeof(double) * 3 * h->d.nchains, cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "energy copy");
    return sync(h);
}

int kcm_set_chain_max_iters(kcm_handle h, const int32_t* max_iters) {
    if (check_handle(h)) return KCM_E_INVAL;
    std::vector<int> m(h->d.nchains, INT32_MAX);
    if (max_iters)
        for (int c = 0; c < h->d.nchains; ++c) m[c] = max_iters[c];
    int rc = upload(h, h->d.chain_maxit, m.data(), m.size());
    return rc ? rc : sync(h);
}

int64_t kcm_device_bytes(kcm_handle h) { return h ? static_cast<int64_t>(h->bytes) : -1; }

int kcm_set_fixed_joints(kcm_handle h, const uint8_t* fixed, int64_t l) {
    if (check_handle(h)) return KCM_E_INVAL;
    if (fixed && l != h->d.l) return set_err(h, KCM_E_INVAL, "fixed must hold one flag per joint");
    std::vector<unsigned char> m(h->d.l, 0);
    if (fixed)
        for (int j = 0; j < h->d.l; ++j) m[j] = fixed[j] ? 1 : 0;
    int rc = upload(h, h->d.jfixed, m.data(), m.size());
    return rc ? rc : sync(h);
}

int64_t kcm_nside_joints(kcm_handle h) { return h ? h->d.ls : -1; }

int kcm_side_offsets(kcm_handle h, int64_t* side_off) {
    if (check_handle(h)) return KCM_E_INVAL;
    if (!side_off) return set_err(h, KCM_E_INVAL, "side_off is NULL");
    for (int c = 0; c <= h->hc.nchains; ++c) side_off[c] = h->d.ls ? h->hc.side_off[c] : 0;
    return KCM_OK;
}

int kcm_set_side_theta(kcm_handle h, const double* chi, int64_t ls) {
    if (check_handle(h)) return KCM_E_INVAL;
    if (ls != h->d.ls || (ls > 0 && !chi)) return set_err(h, KCM_E_INVAL, "chi length must equal the side-chain joint count");
    for (int64_t k = 0; k < ls; ++k)
        if (!std::isfinite(chi[k])) return set_err(h, KCM_E_INVAL, "chi is not finite");
    if (ls == 0) return KCM_OK;
    int rc = upload(h, h->d.theta + h->d.l, chi, static_cast<size_t>(ls));
    return rc ? rc : sync(h);
}

int kcm_get_side_theta(kcm_handle h, double* chi, int64_t ls) {
    if (check_handle(h)) return KCM_E_INVAL;
    if (ls != h->d.ls || (ls > 0 && !chi)) return set_err(h, KCM_E_INVAL, "chi length must equal the side-chain joint count");
    if (ls == 0) return KCM_OK;
    cudaError_t e = cudaMemcpyAsync(chi, h->d.theta + h->d.l, sizeof(double) * ls, cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "chi copy");
    return sync(h);
}

int kcm_set_side_theta_dev(kcm_handle h, const double* chi_dev, int64_t ls) {
    if (check_handle(h)) return KCM_E_INVAL;
    if (ls != h->d.ls || (ls > 0 && !chi_dev)) return set_err(h, KCM_E_INVAL, "chi length must equal the side-chain joint count");
    if (ls == 0) return KCM_OK;
    cudaError_t e = cudaMemcpyAsync(h->d.theta + h->d.l, chi_dev, sizeof(double) * ls, cudaMemcpyDeviceToDevice, h->stream);
    return e == cudaSuccess ? KCM_OK : cuda_fail(h, e, "chi copy");
}

int kcm_get_side_theta_dev(kcm_handle h, double* chi_dev, int64_t ls) {
    if (check_handle(h)) return KCM_E_INVAL;
    if (ls != h->d.ls || (ls > 0 && !chi_dev)) return set_err(h, KCM_E_INVAL, "chi length must equal the side-chain joint count");
    if (ls == 0) return KCM_OK;
    cudaError_t e = cudaMemcpyAsync(chi_dev, h->d.theta + h->d.l, sizeof(double) * ls, cudaMemcpyDeviceToDevice, h->stream);
    return e == cudaSuccess ? KCM_OK : cuda_fail(h, e, "chi copy");
}

int kcm_side_torques(kcm_handle h, double* tau, int64_t ls) {
    if (check_handle(h)) return KCM_E_INVAL;
    if (ls != h->d.ls || (ls > 0 && !tau)) return set_err(h, KCM_E_INVAL, "ls must equal the side-chain joint count");
    int rc = evaluate(h);
    if (rc || ls == 0) return rc;
    cudaError_t e = cudaMemcpyAsync(tau, h->d.tau + h->d.l, sizeof(double) * ls, cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "torque copy");
    return sync(h);
}

int kcm_chain_state(kcm_handle h, int32_t* iters, int32_t* converged, double* max_dtheta, int32_t* errors) {
    if (check_handle(h)) return KCM_E_INVAL;
    const int C = h->d.nchains;
    cudaError_t e = cudaSuccess;
    std::vector<int32_t> bits(errors ? C : 0);
    if (errors) e = cudaMemcpyAsync(bits.data(), h->d.chain_err, sizeof(int32_t) * C, cudaMemcpyDeviceToHost, h->stream);
    if (iters) e = cudaMemcpyAsync(iters, h->d.chain_iters, sizeof(int32_t) * C, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && converged)
        e = cudaMemcpyAsync(converged, h->d.chain_done, sizeof(int32_t) * C, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && max_dtheta)
        e = cudaMemcpyAsync(max_dtheta, h->d.chain_lastdt, sizeof(double) * C, cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "chain state copy");
    int rc = sync(h);
    if (rc) return rc;
    for (int c = 0; errors && c < C; ++c)
        errors[c] = (bits[c] & kcm::kErrNonfinite) ? KCM_E_NONFINITE : (bits[c] & kcm::kErrOverflow) ? KCM_E_OVERFLOW : KCM_OK;
    return KCM_OK;
}

void kcm_destroy(kcm_handle h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->side) cudaStreamSynchronize(h->side);
    drop_graphs(h);
    for (cudaEvent_t ev : h->ev)
        if (ev) cudaEventDestroy(ev);
    for (void* p : h->allocs) cudaFreeAsync(p, h->stream);  // back to the pool; the stream has no work left
    if (h->side) cudaStreamDestroy(h->side);
    if (h->fork) cudaEventDestroy(h->fork);
    if (h->join) cudaEventDestroy(h->join);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    release_status(h->st_host);
    if (h->theta_io) cudaFreeHost(h->theta_io);
    cudaGetLastError();
    delete h;
}

int64_t kcm_natoms(kcm_handle h) { return h ? h->d.n : -1; }
int64_t kcm_njoints(kcm_handle h) { return h ? h->d.l : -1; }
void* kcm_stream(kcm_handle h) { return h ? static_cast<void*>(h->stream) : nullptr; }

int kcm_set_theta(kcm_handle h, const double* theta, int64_t l) {
    if (check_handle(h)) return KCM_E_INVAL;
    if (!theta || l != h->d.l) return set_err(h, KCM_E_INVAL, "theta length must equal the joint count");
    for (int64_t k = 0; k < l; ++k)
        if (!std::isfinite(theta[k])) return set_err(h, KCM_E_INVAL, "theta is not finite");
    int rc = upload(h, h->d.theta, theta, static_cast<size_t>(l));
    return rc ? rc : sync(h);
}

int kcm_get_theta(kcm_handle h, double* theta, int64_t l) {
    if (check_handle(h)) return KCM_E_INVAL;
    if (!theta || l != h->d.l) return set_err(h, KCM_E_INVAL, "theta length must equal the joint count");
    cudaError_t e = cudaMemcpyAsync(theta, h->d.theta, sizeof(double) * l, cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "theta copy");
    return sync(h);
}

int kcm_set_theta_dev(kcm_handle h, const double* theta_dev, int64_t l) {
    if (check_handle(h)) return KCM_E_INVAL;
    if (!theta_dev || l != h->d.l) return set_err(h, KCM_E_INVAL, "theta length must equal the joint count");
    cudaError_t e = cudaMemcpyAsync(h->d.theta, theta_dev, sizeof(double) * l, cudaMemcpyDeviceToDevice, h->stream);
    return e == cudaSuccess ? KCM_OK : cuda_fail(h, e, "theta copy");
}

int kcm_get_theta_dev(kcm_handle h, double* theta_dev, int64_t l) {
    if (check_handle(h)) return KCM_E_INVAL;
    if (!theta_dev || l != h->d.l) return set_err(h, KCM_E_INVAL, "theta length must equal the joint count");
    cudaError_t e = cudaMemcpyAsync(theta_dev, h->d.theta, sizeof(double) * l, cudaMemcpyDeviceToDevice, h->stream);
    return e == cudaSuccess ? KCM_OK : cuda_fail(h, e, "theta copy");
}

int kcm_positions(kcm_handle h, double* xyz, int64_t n) {
    if (check_handle(h)) return KCM_E_INVAL;
    if (!xyz || n != h->d.n) return set_err(h, KCM_E_INVAL, "n must equal the atom count");
    kcm::launch_reset_loop(h->d, h->stream);
    kcm::launch_fk(h->d, h->stream);
    kcm::launch_centres64(h->d, h->stream);
    cudaError_t e = cudaMemcpyAsync(xyz, h->d.r, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "positions copy");
    return sync(h);
}

int kcm_force_terms(kcm_handle h, double* F_pair, double* F_cav, int64_t n) {
    if (check_handle(h)) return KCM_E_INVAL;
    if (n != h->d.n) return set_err(h, KCM_E_INVAL, "n must equal the atom count");
    int rc = evaluate(h);
    if (rc) return rc;
    kcm::launch_force_out(h->d, h->stream);
    cudaError_t e = cudaSuccess;
    if (F_pair) e = cudaMemcpyAsync(F_pair, h->d.Fpair, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && F_cav)
        e = cudaMemcpyAsync(F_cav, h->d.Fcav64, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "force copy");
    return sync(h);
}

int kcm_forces(kcm_handle h, double* F, int64_t n) {
    if (check_handle(h)) return KCM_E_INVAL;
    if (!F || n != h->d.n) return set_err(h, KCM_E_INVAL, "n must equal the atom count");
    int rc = evaluate(h);
    if (rc) return rc;
    kcm::launch_force_out(h->d, h->stream);
    cudaError_t e = cudaMemcpyAsync(F, h->d.Ftot, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "force copy");
    return sync(h);
}

int kcm_torques(kcm_handle h, double* tau, int64_t l) {
    if (check_handle(h)) return KCM_E_INVAL;
    if (!tau || l != h->d.l) return set_err(h, KCM_E_INVAL, "l must equal the joint count");
    int rc = evaluate(h);
    if (rc) return rc;
    cudaError_t e = cudaMemcpyAsync(tau, h->d.tau, sizeof(double) * l, cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "torque copy");
    return sync(h);
}

int kcm_torques_dev(kcm_handle h, double* tau_dev, int64_t l) {
    if (check_handle(h)) return KCM_E_INVAL;
    if (!tau_dev || l != h->d.l) return set_err(h, KCM_E_INVAL, "l must equal the joint count");
    kcm::launch_reset_loop(h->d, h->stream);
    enqueue_evaluation(h);
    cudaError_t e = cudaMemcpyAsync(tau_dev, h->d.tau, sizeof(double) * l, cudaMemcpyDeviceToDevice, h->stream);
    return e == cudaSuccess ? KCM_OK : cuda_fail(h, e, "torque copy");
}

int kcm_energy(kcm_handle h, double E[3]) {
    if (check_handle(h)) return KCM_E_INVAL;
    if (!E) return set_err(h, KCM_E_INVAL, "E is NULL");
    kcm::launch_reset_loop(h->d, h->stream);
    enqueue_evaluation(h);
    kcm::Status st;
    int rc = read_status(h, &st);
    if (rc != KCM_OK) return rc;
    rc = status_code(h, st);
    if (rc != KCM_OK) return rc;
    std::vector<double> ce(3 * (size_t)h->d.nchains);
    cudaError_t e = cudaMemcpyAsync(ce.data(), h->d.chain_E, sizeof(double) * ce.size(), cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "energy copy");
    rc = sync(h);
    if (rc) return rc;
    E[0] = E[1] = E[2] = 0.0;  // the sum over the chains of a batch
    for (int c = 0; c < h->d.nchains; ++c)
        for (int k = 0; k < 3; ++k) E[k] += ce[3 * c + k];
    return KCM_OK;
}

int kcm_sasa_counts(kcm_handle h, int32_t* covered, int64_t n) {
    if (check_handle(h)) return KCM_E_INVAL;
    if (!covered || n != h->d.n) return set_err(h, KCM_E_INVAL, "n must equal the atom count");
    int rc = evaluate(h);
    if (rc) return rc;
    cudaError_t e = cudaMemcpyAsync(covered, h->d.covered, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "count copy");
    return sync(h);
}

int kcm_step_async(kcm_handle h, int32_t n_iters) {
    if (check_handle(h)) return KCM_E_INVAL;
    if (n_iters < 0) return set_err(h, KCM_E_INVAL, "n_iters < 0");
    int rc = build_graph(h);
    if (rc) return rc;
    return launch_steps(h, n_iters);
}

int kcm_step_status(kcm_handle h, int32_t* iters_done, double* max_dtheta) {
    if (check_handle(h)) return KCM_E_INVAL;
    kcm::Status st;
    int rc = read_status(h, &st);
    if (rc) return rc;
    if (iters_done) *iters_done = st.iters;
    if (max_dtheta) *max_dtheta = st.last_max_dtheta;
    return status_code(h, st);
}

int kcm_step(kcm_handle h, int32_t n_iters, int32_t* iters_done, double* max_dtheta) {
    int rc = kcm_step_async(h, n_iters);
    if (rc) return rc;
    return kcm_step_status(h, iters_done, max_dtheta);
}

int kcm_step_host(kcm_handle h, const double* theta_in, double* theta_out, int64_t l, int32_t n_iters,
                  int32_t* iters_done, double* max_dtheta) {
    if (check_handle(h)) return KCM_E_INVAL;
    if (n_iters < 0) return set_err(h, KCM_E_INVAL, "n_iters < 0");
    if ((theta_in || theta_out) && l != h->d.l) return set_err(h, KCM_E_INVAL, "theta length must equal the joint count");
    bool io = false;
    if (theta_in && theta_out && n_iters >= 1) {
        const int rc = build_io_graphs(h, &io);
        if (rc) return rc;
    }
    if (io) {
        // the angles go through the page-locked buffer that the graphs read and write: no copies on the
        // stream, and the status record arrives with the last iteration (an iters of -1 left in it means
        // that nothing exported it, and the record is then read from the device)
        for (int64_t k = 0; k < l; ++k) {
            const double v = theta_in[k];
            if (!std::isfinite(v)) return set_err(h, KCM_E_INVAL, "theta is not finite");
            h->theta_io[k] = v;
        }
        h->st_host->iters = -1;
        for (int32_t i = 0; i < n_iters; ++i) {
            const cudaError_t e = cudaGraphLaunch(i == 0 ? h->graph_io_first : h->graph_io, h->stream);
            if (e != cudaSuccess) {
                cudaStreamSynchronize(h->stream);  // nothing may still read theta_io when the call returns
                return cuda_fail(h, e, "graph launch");
            }
        }
        int rc = sync(h);
        if (rc) return rc;
        kcm::Status st = *h->st_host;
        if (st.iters < 0) {
            rc = read_status(h, &st);
            if (rc) return rc;
        }
        std::memcpy(theta_out, h->theta_io, sizeof(double) * l);
        if (iters_done) *iters_done = st.iters;
        if (max_dtheta) *max_dtheta = st.last_max_dtheta;
        return status_code(h, st);
    }
    for (int64_t k = 0; theta_in && k < l; ++k)
        if (!std::isfinite(theta_in[k])) return set_err(h, KCM_E_INVAL, "theta is not finite");
    int rc = build_graph(h);
    if (rc) return rc;
    cudaError_t e = cudaSuccess;
    if (theta_in) e = cudaMemcpyAsync(h->d.theta, theta_in, sizeof(double) * l, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "theta copy");
    rc = launch_steps(h, n_iters);
    if (rc) return rc;
    if (theta_out) e = cudaMemcpyAsync(theta_out, h->d.theta, sizeof(double) * l, cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "theta copy");
    kcm::Status st;
    rc = read_status(h, &st);  // the one wait of the call
    if (rc) return rc;
    if (iters_done) *iters_done = st.iters;
    if (max_dtheta) *max_dtheta = st.last_max_dtheta;
    return status_code(h, st);
}

int kcm_autotune_cell(kcm_handle h, const double* candidates, int32_t n_candidates, int32_t reps, double* times_ms,
                      double* chosen) {
    if (check_handle(h)) return KCM_E_INVAL;
    if (!candidates || n_candidates < 1 || n_candidates > KCM_AUTOTUNE_MAX)
        return set_err(h, KCM_E_INVAL, "need 1 to KCM_AUTOTUNE_MAX candidate cell edges");
    if (reps < 1 || reps > 1000) return set_err(h, KCM_E_INVAL, "reps must be in [1, 1000]");
    for (int i = 0; i < n_candidates; ++i)
        if (!(candidates[i] >= 0.0) || !std::isfinite(candidates[i]))
            return set_err(h, KCM_E_INVAL, "a candidate cell edge is negative or not finite");
    const double old = h->d.prm.cell_size;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_fail(h, e, "event create");
    }
    std::vector<double> t(n_candidates, 0.0);
    int rc = KCM_OK;
    for (int i = 0; i < n_candidates && rc == KCM_OK; ++i) {
        // one evaluation at the current theta (no step) per launch of a graph captured for this edge
        rc = set_cell_size(h, candidates[i]);
        if (rc) break;
        cudaGraphExec_t ge = nullptr;
        e = capture_graph(
            h,
            [&] {
                kcm::launch_reset_loop(h->d, h->stream);
                enqueue_evaluation(h);
            },
            &ge);
        if (e == cudaSuccess) e = cudaGraphLaunch(ge, h->stream);  // warm-up
        if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
        for (int r = 0; r < reps && e == cudaSuccess; ++r) e = cudaGraphLaunch(ge, h->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (ge) cudaGraphExecDestroy(ge);
        if (e != cudaSuccess) { rc = cuda_fail(h, e, "autotune run"); break; }
        kcm::Status st;
        rc = read_status(h, &st);
        if (rc == KCM_OK) rc = status_code(h, st);
        t[i] = static_cast<double>(ms) / reps;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) {
        set_cell_size(h, old);
        return rc;
    }
    int best = 0;
    for (int i = 1; i < n_candidates; ++i)
        if (t[i] < t[best]) best = i;
    if (times_ms)
        for (int i = 0; i < n_candidates; ++i) times_ms[i] = t[i];
    if (chosen) *chosen = candidates[best];
    return set_cell_size(h, candidates[best]);
}

static bool tile_ok(int32_t w) {
    for (int t : kcm::kTileWarps)
        if (w == t) return true;
    return false;
}

int kcm_set_tiles(kcm_handle h, int32_t pair_warps, int32_t sasa_warps, int32_t pair_persistent) {
    if (check_handle(h)) return KCM_E_INVAL;
    if (!tile_ok(pair_warps) || !tile_ok(sasa_warps)) return set_err(h, KCM_E_INVAL, "atoms per block must be 1, 2 or 4");
    if (pair_persistent != 0 && pair_persistent != 1) return set_err(h, KCM_E_INVAL, "pair_persistent must be 0 or 1");
    int rc = sync(h);  // no launch of the old shape is pending when the graphs go
    if (rc) return rc;
    drop_graphs(h);
    h->d.pair_warps = pair_warps;
    h->d.sasa_warps = sasa_warps;
    h->d.pair_persistent = pair_persistent;
    return set_pair_grid(h);
}

int kcm_get_tiles(kcm_handle h, int32_t* pair_warps, int32_t* sasa_warps, int32_t* pair_persistent) {
    if (check_handle(h)) return KCM_E_INVAL;
    if (pair_warps) *pair_warps = h->d.pair_warps;
    if (sasa_warps) *sasa_warps = h->d.sasa_warps;
    if (pair_persistent) *pair_persistent = h->d.pair_persistent;
    return KCM_OK;
}

int kcm_set_pair_kernel(kcm_handle h, int32_t kind) {
    if (check_handle(h)) return KCM_E_INVAL;
    if (kind != KCM_PAIR_WARP_PER_ATOM && kind != KCM_PAIR_CELL_TILES)
        return set_err(h, KCM_E_INVAL, "pair kernel must be KCM_PAIR_WARP_PER_ATOM or KCM_PAIR_CELL_TILES");
    if (kind == KCM_PAIR_CELL_TILES && h->d.prm.precision != KCM_MIXED)
        return set_err(h, KCM_E_INVAL, "the cell-pair tile kernel is the mixed-precision pair kernel");
    int rc = sync(h);  // no launch of the old kernel is pending when the graphs go
    if (rc) return rc;
    drop_graphs(h);
    h->d.pair_tile = kind;
    return KCM_OK;
}

int kcm_set_test_withhold(kcm_handle h, int32_t tile) {
    if (check_handle(h)) return KCM_E_INVAL;
    if (tile < -1 || tile >= h->d.ltiles) return set_err(h, KCM_E_INVAL, "tile out of range");
    int rc = sync(h);  // the captured graphs hold the old setting
    if (rc) return rc;
    drop_graphs(h);
    h->d.lb_withhold = tile;
    return KCM_OK;
}

int kcm_set_graph_overlap(kcm_handle h, int32_t on) {
    if (check_handle(h)) return KCM_E_INVAL;
    if (on != 0 && on != 1) return set_err(h, KCM_E_INVAL, "on must be 0 or 1");
    int rc = sync(h);  // no launch of the old graphs is pending when they go
    if (rc) return rc;
    drop_graphs(h);
    h->pdl = on != 0;
    return KCM_OK;
}

int kcm_set_binning_kernel(kcm_handle h, int32_t kind) {
    if (check_handle(h)) return KCM_E_INVAL;
    if (kind != KCM_BIN_BLOCKS && kind != KCM_BIN_CLUSTER)
        return set_err(h, KCM_E_INVAL, "binning kernel must be KCM_BIN_BLOCKS or KCM_BIN_CLUSTER");
    int rc = sync(h);  // no launch of the old kernels is pending when the graphs go
    if (rc) return rc;
    drop_graphs(h);
    h->bin_cluster = kind == KCM_BIN_CLUSTER;
    cudaError_t e = kcm::plan_bin_cluster(h->d, h->bin_cluster);
    return e == cudaSuccess ? KCM_OK : cuda_fail(h, e, "binning kernel attributes");
}

int kcm_get_binning_kernel(kcm_handle h, int32_t* kind, int32_t* ctas) {
    if (check_handle(h)) return KCM_E_INVAL;
    if (!kind) return set_err(h, KCM_E_INVAL, "kind is NULL");
    *kind = h->d.bin_c ? KCM_BIN_CLUSTER : KCM_BIN_BLOCKS;
    if (ctas) *ctas = h->d.bin_c;
    return KCM_OK;
}

int kcm_get_pair_kernel(kcm_handle h, int32_t* kind) {
    if (check_handle(h)) return KCM_E_INVAL;
    if (!kind) return set_err(h, KCM_E_INVAL, "kind is NULL");
    *kind = h->d.pair_tile;
    return KCM_OK;
}

int kcm_autotune_tiles(kcm_handle h, int32_t reps, double* times_ms, int32_t* pair_warps, int32_t* sasa_warps,
                       int32_t* pair_persistent) {
    if (check_handle(h)) return KCM_E_INVAL;
    if (reps < 1 || reps > 1000) return set_err(h, KCM_E_INVAL, "reps must be in [1, 1000]");
    const int old_p = h->d.pair_warps, old_s = h->d.sasa_warps, old_pp = h->d.pair_persistent;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_fail(h, e, "event create");
    }
    constexpr int nt = sizeof(kcm::kTileWarps) / sizeof(kcm::kTileWarps[0]);
    constexpr int ncomb = 2 * nt * nt;  // (persistent, pair shape, solvation shape)
    auto shape = [&](int i, int* pp, int* pw, int* sw) {
        *pp = i / (nt * nt);
        *pw = kcm::kTileWarps[(i / nt) % nt];
        *sw = kcm::kTileWarps[i % nt];
    };
    auto shape_pp = [&](int i) { return i / (nt * nt); };
    std::vector<double> t(ncomb, 0.0);
    // the cell-pair tile kernel takes the pair shape as its split (warps per window and stencil row) and has
    // no persistent grid: the combinations of the other grid take the time of the same shapes on this one
    const bool pair_fixed = h->d.pair_tile && h->d.prm.precision == KCM_MIXED;
    int rc = KCM_OK;
    for (int i = 0; i < ncomb && rc == KCM_OK; ++i) {
        // one evaluation at the current theta (no step) per launch of a graph captured for this shape
        int pp, pw, sw;
        shape(i, &pp, &pw, &sw);
        if (pair_fixed && pp != old_pp) continue;
        rc = kcm_set_tiles(h, pw, sw, pp);
        if (rc) break;
        cudaGraphExec_t ge = nullptr;
        e = capture_graph(
            h,
            [&] {
                kcm::launch_reset_loop(h->d, h->stream);
                enqueue_evaluation(h);
            },
            &ge);
        if (e == cudaSuccess) e = cudaGraphLaunch(ge, h->stream);  // warm-up
        if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
        for (int r = 0; r < reps && e == cudaSuccess; ++r) e = cudaGraphLaunch(ge, h->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (ge) cudaGraphExecDestroy(ge);
        if (e != cudaSuccess) { rc = cuda_fail(h, e, "autotune run"); break; }
        kcm::Status st;
        rc = read_status(h, &st);
        if (rc == KCM_OK) rc = status_code(h, st);
        t[i] = static_cast<double>(ms) / reps;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) {
        kcm_set_tiles(h, old_p, old_s, old_pp);
        return rc;
    }
    if (pair_fixed) {
        for (int i = 0; i < ncomb; ++i) {
            int pp, pw, sw;
            shape(i, &pp, &pw, &sw);
            if (pp == old_pp) continue;
            for (int k = 0; k < ncomb; ++k) {
                int pp2, pw2, sw2;
                shape(k, &pp2, &pw2, &sw2);
                if (pp2 == old_pp && pw2 == pw && sw2 == sw) t[i] = t[k];
            }
        }
    }
    int best = 0;
    for (int i = 1; i < ncomb; ++i)
        if (t[i] < t[best] || (pair_fixed && t[i] == t[best] && shape_pp(i) == old_pp && shape_pp(best) != old_pp)) best = i;
    if (times_ms)
        for (int i = 0; i < ncomb; ++i) times_ms[i] = t[i];
    int pp, pw, sw;
    shape(best, &pp, &pw, &sw);
    if (pair_warps) *pair_warps = pw;
    if (sasa_warps) *sasa_warps = sw;
    if (pair_persistent) *pair_persistent = pp;
    return kcm_set_tiles(h, pw, sw, pp);
}

int kcm_autotune_pair_kernel(kcm_handle h, int32_t reps, double* times_ms, int32_t* kind) {
    if (check_handle(h)) return KCM_E_INVAL;
    if (reps < 1 || reps > 1000) return set_err(h, KCM_E_INVAL, "reps must be in [1, 1000]");
    const int old_kind = h->d.pair_tile;
    const int nkind = h->d.prm.precision == KCM_MIXED ? 2 : 1;
    double best_t[2] = {0.0, 0.0};
    int32_t shapes[2][3] = {{1, 1, 0}, {1, 1, 0}};
    for (int k = 0; k < nkind; ++k) {
        // the warp-per-atom kernel first, then the cell-pair tile kernel, each with its best tile shapes
        const int kk = nkind == 1 ? KCM_PAIR_WARP_PER_ATOM : k;
        int rc = kcm_set_pair_kernel(h, kk);
        double t[18];
        if (rc == KCM_OK) rc = kcm_autotune_tiles(h, reps, t, &shapes[k][0], &shapes[k][1], &shapes[k][2]);
        if (rc) {
            kcm_set_pair_kernel(h, old_kind);
            return rc;
        }
        best_t[k] = *std::min_element(t, t + 18);
    }
    const int win = nkind == 2 && best_t[1] < best_t[0] ? 1 : 0;
    if (times_ms)
        for (int k = 0; k < 2; ++k) times_ms[k] = k < nkind ? best_t[k] : 0.0;
    if (kind) *kind = nkind == 1 ? KCM_PAIR_WARP_PER_ATOM : win;
    int rc = kcm_set_pair_kernel(h, nkind == 1 ? KCM_PAIR_WARP_PER_ATOM : win);
    if (rc) return rc;
    return kcm_set_tiles(h, shapes[win][0], shapes[win][1], shapes[win][2]);
}

int kcm_get_stats(kcm_handle h, kcm_stats* out) {
    if (check_handle(h)) return KCM_E_INVAL;
    if (!out) return set_err(h, KCM_E_INVAL, "stats is NULL");
    kcm::Status st;
    kcm::GridInfo g;
    cudaError_t e = cudaMemcpyAsync(&g, h->d.grid, sizeof g, cudaMemcpyDeviceToHost, h->stream);  // chain 0
    if (e != cudaSuccess) return cuda_fail(h, e, "grid copy");
    int rc = read_status(h, &st);
    if (rc) return rc;
    out->pairs = static_cast<int64_t>(st.pairs);
    out->sasa_neighbors = static_cast<int64_t>(st.nbr_total);
    out->max_neighbors = st.max_nbr;
    out->guard_rechecks = static_cast<int64_t>(st.guard);
    out->cells = st.ncells;
    out->cell_size = g.s;
    out->iterations = st.iters;
    out->sasa_tests = static_cast<int64_t>(st.sasa_tests);
    return KCM_OK;
}

int kcm_step_timed(kcm_handle h, float* stage_ms, int32_t n_stages, float* total_ms) {
    if (check_handle(h)) return KCM_E_INVAL;
    if (n_stages < 0 || n_stages > KCM_NUM_STAGES || (n_stages > 0 && !stage_ms))
        return set_err(h, KCM_E_INVAL, "n_stages must be in [0, KCM_NUM_STAGES]");
    int rc = build_timed_graph(h);
    if (rc) return rc;
    cudaError_t e = cudaEventRecord(h->ev[0], h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "event record");
    kcm::launch_reset_loop(h->d, h->stream);
    e = cudaGraphLaunch(h->graph_timed, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "graph launch");
    kcm::Status st;
    rc = read_status(h, &st);
    if (rc) return rc;
    for (int i = 0; i < n_stages; ++i) {
        e = cudaEventElapsedTime(&stage_ms[i], h->ev[1 + i], h->ev[2 + i]);
        if (e != cudaSuccess) return cuda_fail(h, e, "event elapsed");
    }
    if (total_ms) {
        e = cudaEventElapsedTime(total_ms, h->ev[0], h->ev[KCM_NUM_STAGES + 1]);
        if (e != cudaSuccess) return cuda_fail(h, e, "event elapsed");
    }
    return status_code(h, st);
}

int kcm_sample_points(int32_t N, double* Q) {
    if (!Q || N < 1) return set_err(nullptr, KCM_E_INVAL, "N must be >= 1 and Q non-NULL");
    return kcm::sample_points(N, Q);
}

int64_t kcm_topology_natoms(const kcm_topology* top) {
    kcm::HostChain hc;
    std::string err;
    int rc = kcm::build_host_chain(top, &hc, &err);
    if (rc) { set_err(nullptr, rc, err); return rc; }
    return hc.n;
}

int kcm_build_zp(const kcm_topology* top, double* xyz0, int32_t* link, int64_t n) {
    kcm::HostChain hc;
    std::string err;
    int rc = kcm::build_host_chain(top, &hc, &err);
    if (rc) return set_err(nullptr, rc, err);
    if (n != hc.n) return set_err(nullptr, KCM_E_INVAL, "n must equal the atom count");
    if (xyz0) std::memcpy(xyz0, hc.zp.data(), sizeof(double) * 3 * n);
    if (link)
        for (int64_t a = 0; a < n; ++a) link[a] = hc.link[a];
    return KCM_OK;
}

int kcm_pair_class(const kcm_topology* top, const int32_t* a, const int32_t* b, int64_t n_pairs, int32_t* cls) {
    kcm::HostChain hc;
    std::string err;
    int rc = kcm::build_host_chain(top, &hc, &err);
    if (rc) return set_err(nullptr, rc, err);
    if (n_pairs < 0 || (n_pairs > 0 && (!a || !b || !cls))) return set_err(nullptr, KCM_E_INVAL, "bad pair arrays");
    for (int64_t k = 0; k < n_pairs; ++k) {
        int x = a[k], y = b[k];
        if (x < 0 || y < 0 || x >= hc.n || y >= hc.n || x == y) return set_err(nullptr, KCM_E_INVAL, "pair index out of range");
        int lo = std::min(x, y), off = std::max(x, y) - lo;
        int c = 0;
        if (off <= kcm::kMaskWindow) {
            if ((hc.ex_mask[lo] >> off) & 1ULL) c = 1;
            else if ((hc.m14_mask[lo] >> off) & 1ULL) c = 2;
        }
        cls[k] = c;
    }
    return KCM_OK;
}

const char* kcm_strerror(int code) {
    switch (code) {
        case KCM_OK: return "ok";
        case KCM_E_INVAL: return "invalid argument";
        case KCM_E_NOMEM: return "out of memory";
        case KCM_E_CUDA: return "CUDA error";
        case KCM_E_NONFINITE: return "non-finite torque";
        case KCM_E_OVERFLOW: return "solvation neighbour list overflow";
        case KCM_E_NODEVICE: return "no sm_103 CUDA device";
        case KCM_E_CANCELLED: return "cancelled";
        case KCM_E_TIMEOUT: return "a bounded device wait gave up";
        default: return "unknown status";
    }
}

const char* kcm_last_error(kcm_handle h) { return h ? h->err.c_str() : g_last_error.c_str(); }

}  // extern "C"
