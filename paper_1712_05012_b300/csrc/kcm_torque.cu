// A7-A9: link wrenches, suffix sums over links, joint torques and the kinetostatic step (FP64).
// The wrench kernel, which visits every atom once with one thread each, also converts the
// mixed-mode fixed-point forces to FP64 and adds the cavity energy G0_i f_i of its atoms.
//
// Wrench of link h about the origin, P_h = [sum r x F ; sum F] (eq. KCM_01/02), and
// P^agg_k = sum_{h >= k} P_h (Sec. 3.5) as a reverse scan: k_wrench_tile forms P_h from the atoms of
// a 32-link tile and scans the tile, its last block scans the tile totals, and k_torque takes
// tau_k = u_k . T^agg_k + (p_k x u_k) . F^agg_k (eq. KCM_05/06).
// In the clamped step mode the same thread applies dtheta_k = clamp(kappa tau_k, +-dtheta_max)
// (eq. KCM_07); the last block to finish closes the iteration.
#include <cuda_runtime.h>

#include "kcm_common.cuh"
#include "kcm_device.h"

namespace kcm {

namespace {
using namespace dev;

// One block per tile of 32 links h in [32 t, 32 t + 32). The block's warps take the tile's atoms in
// chunks of 32 (one thread per atom: r x F and F, and the conversion of the mixed-mode fixed-point
// forces); a shuffle sum segmented by link adds each link's atoms within the chunk. A link (at most
// 11 atoms) meets at most two chunks, so its wrench P_h is part 0 + part 1 in shared memory, in a
// fixed order. Warp q then scans component q of the tile's P_h from the end (Kogge-Stone), and the
// last block to finish (ticket, no waiting) forms the exclusive suffix sums of the tile totals.
__global__ void __launch_bounds__(kWrenchWarps * 32) k_wrench_tile(const DevChain d) {
    __shared__ double sP[32][2][6];
    __shared__ bool last;
    Status* st = d.status;
    if (st->done) return;
    const int t = blockIdx.x, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int h0 = 32 * t, h1 = min(h0 + 32, d.L);
    for (int x = threadIdx.x; x < 32 * 2 * 6; x += blockDim.x) (&sP[0][0][0])[x] = 0.0;
    __syncthreads();
    const int a0 = d.link_start[h0], a1 = d.link_start[h1];
    double Ecav = 0.0;
    for (int c = a0 + 32 * w; c < a1; c += 32 * kWrenchWarps) {
        const int a = c + lane;
        double v[6] = {0, 0, 0, 0, 0, 0};
        int h = -1 - lane;  // distinct keys for lanes past the tile's last atom
        if (a < a1) {
            double fx, fy, fz;
            if (d.prm.precision == KCM_MIXED) {  // pair forces in fixed point plus oversized terms
                fx = (double)d.Fpx[3 * a] * kPairFxInv + (double)d.Fov[3 * a];
                fy = (double)d.Fpx[3 * a + 1] * kPairFxInv + (double)d.Fov[3 * a + 1];
                fz = (double)d.Fpx[3 * a + 2] * kPairFxInv + (double)d.Fov[3 * a + 2];
            } else {
                fx = d.Fpair[3 * a]; fy = d.Fpair[3 * a + 1]; fz = d.Fpair[3 * a + 2];
            }
            if (d.prm.solvation) {
                fx += (double)d.Fcav[3 * a] * kFxInv;
                fy += (double)d.Fcav[3 * a + 1] * kFxInv;
                fz += (double)d.Fcav[3 * a + 2] * kFxInv;
                const double G0a = d.G0[a];  // G^cav_i = G0_i f_i, f_i = 1 - covered_i / N (Sec. 3.4)
                if (G0a != 0.0) Ecav += G0a - G0a * (double)d.covered[a] / (double)d.N;
            }
            const double x = d.r[3 * a], y = d.r[3 * a + 1], z = d.r[3 * a + 2];
            v[0] = y * fz - z * fy;
            v[1] = z * fx - x * fz;
            v[2] = x * fy - y * fx;
            v[3] = fx; v[4] = fy; v[5] = fz;
            h = d.link[a];
        }
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int hp = __shfl_up_sync(0xffffffffu, h, off);
            const bool take = lane >= off && hp == h;
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                const double y = __shfl_up_sync(0xffffffffu, v[k], off);
                if (take) v[k] += y;
            }
        }
        const int hn = __shfl_down_sync(0xffffffffu, h, 1);
        if (a < a1 && (lane == 31 || hn != h)) {  // last lane of a segment: its sum is one part of P_h
            const int part = d.link_start[h] < c ? 1 : 0;  // the link began in the previous chunk
#pragma unroll
            for (int k = 0; k < 6; ++k) sP[h - h0][part][k] = v[k];
        }
    }
    if (d.prm.solvation) {  // cavity energy of the block's atoms
        Ecav = warp_sum(Ecav);
        if (lane == 0 && Ecav != 0.0) atomicAdd(&st->E[2], Ecav);
    }
    __syncthreads();
    if (w < 6) {  // reverse inclusive scan of component w over the tile (links 1..l; link 0 has no joint)
        const int h = h0 + lane;
        double x = (h >= 1 && h < h1) ? sP[lane][0][w] + sP[lane][1][w] : 0.0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const double y = __shfl_down_sync(0xffffffffu, x, off);
            if (lane + off < 32) x += y;
        }
        if (h < d.L) d.lane_suf[6 * (size_t)h + w] = x;
        if (lane == 0) d.tileS[6 * (size_t)t + w] = x;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&st->ticket_w, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (w < 6) {  // exclusive suffix sums of the tile totals, 32 tiles per round from the end
        double carry = 0.0;
        for (int top = d.ltiles; top > 0; top -= 32) {
            const int tt = top - 32 + lane;
            double x = tt >= 0 ? __ldcg(&d.tileS[6 * (size_t)tt + w]) : 0.0;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const double y = __shfl_down_sync(0xffffffffu, x, off);
                if (lane + off < 32) x += y;
            }
            double e = __shfl_down_sync(0xffffffffu, x, 1);
            if (lane == 31) e = 0.0;
            if (tt >= 0) d.tileSuf[6 * (size_t)tt + w] = e + carry;
            carry += __shfl_sync(0xffffffffu, x, 0);
        }
    }
    if (threadIdx.x == 0) st->ticket_w = 0u;
}

// tau_k from P^agg; with STEP the clamped step and the end of the iteration
template <bool STEP>
__global__ void __launch_bounds__(128) k_torque(const DevChain d) {
    __shared__ unsigned long long smax[4];
    __shared__ bool last;
    Status* st = d.status;
    if (st->done) return;
    const int jj = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long adt = 0ULL, atau = 0ULL;  // bit patterns of non-negative doubles
    bool bad = false;
    if (jj < d.l) {
        const int h = jj + 1, tile = h >> 5;  // joint jj moves links jj+1 .. l
        double A[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) A[k] = d.lane_suf[6 * (size_t)h + k] + d.tileSuf[6 * (size_t)tile + k];
        const double* u = &d.ucur[3 * jj];
        const double* p = &d.pcur[3 * jj];
        const double px = p[1] * u[2] - p[2] * u[1], py = p[2] * u[0] - p[0] * u[2], pz = p[0] * u[1] - p[1] * u[0];
        const double t = u[0] * A[0] + u[1] * A[1] + u[2] * A[2] + px * A[3] + py * A[4] + pz * A[5];
        d.tau[jj] = t;
        bad = !isfinite(t);
        atau = (unsigned long long)__double_as_longlong(fabs(t));
        if (STEP && !bad) {
            const double dt = fmin(fmax(d.prm.kappa * t, -d.prm.dtheta_max), d.prm.dtheta_max);
            d.theta[jj] += dt;
            d.dtheta[jj] = dt;
            adt = (unsigned long long)__double_as_longlong(fabs(dt));
        }
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&st->error, kErrNonfinite);
    for (int o = 16; o > 0; o >>= 1) {
        adt = max(adt, __shfl_down_sync(0xffffffffu, adt, o));
        atau = max(atau, __shfl_down_sync(0xffffffffu, atau, o));
    }
    if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = adt;
    if ((threadIdx.x & 31) == 0 && atau) atomicMax(&st->max_abs_tau, atau);
    if (!STEP) return;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long m = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) m = max(m, smax[k]);
        atomicMax(&st->max_dtheta, m);
        __threadfence();
        last = atomicAdd(&st->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {  // the last block closes the iteration
        __threadfence();
        const double mall = __longlong_as_double((long long)atomicAdd(&st->max_dtheta, 0ULL));
        if (st->error) {
            st->done = 1;  // a failed iteration leaves theta as the kernels found it at the first error
        } else {
            st->last_max_dtheta = mall;
            st->iters += 1;
            if (mall < d.prm.conv_tol) st->done = 1;
        }
        st->max_dtheta = 0ULL;
        st->max_abs_tau = 0ULL;
        st->ticket = 0u;
    }
}

// the paper's normalised step (eq. KCM_07): dtheta_k = kappa tau_k / max |tau|
__global__ void __launch_bounds__(128) k_step_normalized(const DevChain d) {
    __shared__ unsigned long long smax[4];
    __shared__ bool last;
    Status* st = d.status;
    if (st->done) return;
    if (st->error) {
        if (blockIdx.x == 0 && threadIdx.x == 0) st->done = 1;
        return;
    }
    const int jj = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long adt = 0ULL;
    if (jj < d.l) {
        const double tm = __longlong_as_double((long long)st->max_abs_tau);
        const double dt = tm > 0.0 ? d.prm.kappa * d.tau[jj] / tm : 0.0;
        d.theta[jj] += dt;
        d.dtheta[jj] = dt;
        adt = (unsigned long long)__double_as_longlong(fabs(dt));
    }
    for (int o = 16; o > 0; o >>= 1) adt = max(adt, __shfl_down_sync(0xffffffffu, adt, o));
    if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = adt;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long m = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) m = max(m, smax[k]);
        atomicMax(&st->max_dtheta, m);
        __threadfence();
        last = atomicAdd(&st->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        const double mall = __longlong_as_double((long long)atomicAdd(&st->max_dtheta, 0ULL));
        st->last_max_dtheta = mall;
        st->iters += 1;
        if (mall < d.prm.conv_tol) st->done = 1;
        st->max_dtheta = 0ULL;
        st->max_abs_tau = 0ULL;
        st->ticket = 0u;
    }
}

}  // namespace

void launch_torques(DevChain& d, cudaStream_t s) {
    k_wrench_tile<<<d.ltiles, kWrenchWarps * 32, 0, s>>>(d);
    k_torque<false><<<(d.l + 127) / 128, 128, 0, s>>>(d);
}

// torques plus the step of one iteration (the evaluation kernels must already be enqueued)
void launch_torques_step(DevChain& d, cudaStream_t s) {
    k_wrench_tile<<<d.ltiles, kWrenchWarps * 32, 0, s>>>(d);
    if (d.prm.step_mode == KCM_STEP_CLAMP) {
        k_torque<true><<<(d.l + 127) / 128, 128, 0, s>>>(d);
    } else {
        k_torque<false><<<(d.l + 127) / 128, 128, 0, s>>>(d);
        k_step_normalized<<<(d.l + 127) / 128, 128, 0, s>>>(d);
    }
}

}  // namespace kcm
