// kcm_torques_noalloc: joint torques from per-atom forces with no device allocation.
//
// Some callers cannot allocate device memory when they need torques: a serving process that has
// reserved all of the GPU's memory up front for its own pool allocator (a cudaMalloc would fail
// or fragment that pool), or a latency-critical host loop that must never wait on the driver's
// allocator. For them this entry point keeps its working memory (the link wrenches and the
// per-chunk sums of the suffix scan) in one fixed array that is part of the library image, so a
// call only launches kernels on the caller's stream.
//
// The array is a file-scope __device__ variable: every GPU that loads the library holds it
// (about 2 MB) until the process exits, and all calls on that GPU share it.
#include <cuda_runtime.h>

#include <mutex>

#include "kcm.h"

namespace {

constexpr int kNaMaxLinks = KCM_NOALLOC_MAX_LINKS;
constexpr int kNaChunk = 8;  // links per thread
constexpr int kNaMaxChunks = (kNaMaxLinks + kNaChunk - 1) / kNaChunk;
constexpr size_t kNaWrench = 6 * static_cast<size_t>(kNaMaxLinks);  // P_h = [T_h ; F_h]
constexpr size_t kNaChunkSums = 6 * static_cast<size_t>(kNaMaxChunks);
constexpr size_t kNaDoubles = kNaWrench + 2 * kNaChunkSums;

// The scratch. In host code this name is only a stand-in for the symbol, never a device address:
// host code obtains the address with cudaGetSymbolAddress and passes that to the kernels.
static __device__ __align__(256) double g_torque_scratch[kNaDoubles];

constexpr int kNaMaxDevices = 64;
std::mutex g_na_mutex;
double* g_na_ptr[kNaMaxDevices] = {};

// wrench of every link (moments about the origin, eq. KCM_01/02) and the chunk sums of links >= 1;
// every word of the scratch that is read later is written here first
__global__ void na_wrench(int L, const int* __restrict__ link_start, const double* __restrict__ xyz,
                          const double* __restrict__ F, double* __restrict__ P, double* __restrict__ S) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    int nc = (L + kNaChunk - 1) / kNaChunk;
    if (c >= nc) return;
    int h0 = c * kNaChunk, h1 = min(L, h0 + kNaChunk);
    double s[6] = {0, 0, 0, 0, 0, 0};
    for (int h = h0; h < h1; ++h) {
        double w[6] = {0, 0, 0, 0, 0, 0};
        for (int a = link_start[h]; a < link_start[h + 1]; ++a) {
            double x = xyz[3 * a], y = xyz[3 * a + 1], z = xyz[3 * a + 2];
            double fx = F[3 * a], fy = F[3 * a + 1], fz = F[3 * a + 2];
            w[0] += y * fz - z * fy;
            w[1] += z * fx - x * fz;
            w[2] += x * fy - y * fx;
            w[3] += fx;
            w[4] += fy;
            w[5] += fz;
        }
        for (int k = 0; k < 6; ++k) {
            P[6 * h + k] = w[k];
            if (h >= 1) s[k] += w[k];
        }
    }
    for (int k = 0; k < 6; ++k) S[6 * c + k] = s[k];
}

// exclusive suffix sums of the chunk sums (one block)
__global__ void na_scan(int nc, const double* __restrict__ S, double* __restrict__ Suf) {
    __shared__ double part[64][6];
    int t = threadIdx.x;
    int per = (nc + 63) / 64;
    int c0 = min(nc, t * per), c1 = min(nc, c0 + per);
    double a[6] = {0, 0, 0, 0, 0, 0};
    for (int c = c1 - 1; c >= c0; --c)
        for (int k = 0; k < 6; ++k) a[k] += S[6 * c + k];
    for (int k = 0; k < 6; ++k) part[t][k] = a[k];
    __syncthreads();
    if (t == 0) {
        double run[6] = {0, 0, 0, 0, 0, 0};
        for (int u = 63; u >= 0; --u)
            for (int k = 0; k < 6; ++k) {
                double v = part[u][k];
                part[u][k] = run[k];
                run[k] += v;
            }
    }
    __syncthreads();
    for (int k = 0; k < 6; ++k) a[k] = part[t][k];
    for (int c = c1 - 1; c >= c0; --c)
        for (int k = 0; k < 6; ++k) {
            Suf[6 * c + k] = a[k];
            a[k] += S[6 * c + k];
        }
}

// P^agg_k = P_k + P^agg_{k+1} and tau_k = u_k . T^agg_k + (p_k x u_k) . F^agg_k (Sec. 3.5)
__global__ void na_torque(int L, const double* __restrict__ P, const double* __restrict__ Suf,
                          const double* __restrict__ axis, const double* __restrict__ point, double* __restrict__ tau) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    int nc = (L + kNaChunk - 1) / kNaChunk;
    if (c >= nc) return;
    int h0 = c * kNaChunk, h1 = min(L, h0 + kNaChunk);
    double a[6];
    for (int k = 0; k < 6; ++k) a[k] = Suf[6 * c + k];
    for (int h = h1 - 1; h >= h0 && h >= 1; --h) {
        for (int k = 0; k < 6; ++k) a[k] += P[6 * h + k];
        const double* u = &axis[3 * (h - 1)];
        const double* p = &point[3 * (h - 1)];
        double px = p[1] * u[2] - p[2] * u[1], py = p[2] * u[0] - p[0] * u[2], pz = p[0] * u[1] - p[1] * u[0];
        tau[h - 1] = u[0] * a[0] + u[1] * a[1] + u[2] * a[2] + px * a[3] + py * a[4] + pz * a[5];
    }
}

// device address of the scratch on the current device, looked up once per device
int scratch_address(double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return KCM_E_NODEVICE;
    }
    if (dev < 0 || dev >= kNaMaxDevices) return KCM_E_NODEVICE;
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_torque_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return KCM_E_CUDA;
        }
        g_na_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_na_ptr[dev];
    return KCM_OK;
}

}  // namespace

extern "C" int kcm_torques_noalloc(int32_t n_links, const int32_t* link_start_dev, const double* xyz_dev,
                                   const double* F_dev, const double* axis_dev, const double* point_dev,
                                   double* tau_dev, void* cuda_stream) {
    if (n_links < 2 || n_links > kNaMaxLinks) return KCM_E_INVAL;
    if (!link_start_dev || !xyz_dev || !F_dev || !axis_dev || !point_dev || !tau_dev) return KCM_E_INVAL;
    double* base = nullptr;
    int rc = scratch_address(&base);
    if (rc != KCM_OK) return rc;
    double* P = base;
    double* S = base + kNaWrench;
    double* Suf = S + kNaChunkSums;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int nc = (n_links + kNaChunk - 1) / kNaChunk;
    int tpb = 32;
    int blocks = (nc + tpb - 1) / tpb;
    na_wrench<<<blocks, tpb, 0, s>>>(n_links, link_start_dev, xyz_dev, F_dev, P, S);
    na_scan<<<1, 64, 0, s>>>(nc, S, Suf);
    na_torque<<<blocks, tpb, 0, s>>>(n_links, P, Suf, axis_dev, point_dev, tau_dev);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? KCM_OK : KCM_E_CUDA;
}
