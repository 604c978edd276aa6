// A1: forward kinematics as a prefix product of local link-frame transforms (FP64).
//
// Link frame poses T_j = L_1 o ... o L_j with L_j = Tr(step_j) o Rot(u0_j, theta_j) (eq. kin_04 in
// local frames; App. B prefix computation). Atom centres are T_link(r0 - frame origin) (eq. r1, r2).
//
// On B300 an FP64 instruction costs the SM's FP64 pipe about as much for one active lane as for 32,
// and a dependent FP64 operation takes ~70 cycles, so the scan is done by full warps: each lane
// composes J consecutive joints, a warp composes its 32 lane products with a Kogge-Stone shuffle scan
// (the extra compositions of that scan are free), one warp scans the tile products, and each lane
// then applies its tile and lane prefix. Tiles are one warp per block, which spreads them over SMs.
#include <cuda_runtime.h>

#include "kcm_common.cuh"
#include "kcm_device.h"

namespace kcm {

namespace {
using namespace dev;

__device__ __forceinline__ void shfl_up12(const double* X, double* Y, int off) {
#pragma unroll
    for (int k = 0; k < 12; ++k) Y[k] = __shfl_up_sync(0xffffffffu, X[k], off);
}

// inclusive Kogge-Stone scan of affine transforms over the 32 lanes (composition on the left)
__device__ __forceinline__ void warp_scan_aff(double* X, int lane) {
    double Y[12];
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        shfl_up12(X, Y, off);
        if (lane >= off) aff_compose(Y, X, X);
    }
}

// per lane: product of its J joints (each joint's lane-local inclusive prefix kept in G); per warp:
// exclusive lane prefixes and the tile product
template <int J>
__global__ void __launch_bounds__(32) k_fk_tile(const DevChain d) {
    if (d.status->done) return;
    const int tile = blockIdx.x, lane = threadIdx.x;
    const int j0 = (tile * 32 + lane) * J;
    double A[12], Gj[12];
    aff_identity(A);
#pragma unroll
    for (int q = 0; q < J; ++q) {
        const int jj = j0 + q;
        if (jj < d.l) {
            joint_tf(&d.u0[3 * jj], &d.step0[3 * jj], d.theta[jj], Gj);
            aff_compose(A, Gj, A);
            aff_store(&d.G[12 * (size_t)jj], A);
        }
    }
    double X[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) X[k] = A[k];
    warp_scan_aff(X, lane);
    double E[12];
    shfl_up12(X, E, 1);
    if (lane == 0) aff_identity(E);
    aff_store(&d.lane_ex[12 * ((size_t)tile * 32 + lane)], E);
    if (lane == 31) aff_store(&d.tileP[12 * (size_t)tile], X);
}

// exclusive prefix of the tile products, 32 tiles per round with a carried product (one warp)
__global__ void __launch_bounds__(32) k_fk_tilescan(const DevChain d) {
    if (d.status->done) return;
    const int lane = threadIdx.x;
    double carry[12];
    aff_identity(carry);
    for (int base = 0; base < d.ntiles; base += 32) {
        const int t = base + lane;
        double X[12], E[12], T[12];
        if (t < d.ntiles) aff_load(&d.tileP[12 * (size_t)t], X);
        else aff_identity(X);
        warp_scan_aff(X, lane);
        shfl_up12(X, E, 1);
        if (lane == 0) aff_identity(E);
        aff_compose(carry, E, E);
        if (t < d.ntiles) aff_store(&d.tileE[12 * (size_t)t], E);
#pragma unroll
        for (int k = 0; k < 12; ++k) T[k] = __shfl_sync(0xffffffffu, X[k], 31);
        aff_compose(carry, T, carry);
    }
}

// link poses M_{j+1} = (tile prefix o lane prefix) o lane-local prefix_j; current axis
// u_j = R(M_j) u0_j through p_j = origin of frame j+1
template <int J>
__global__ void __launch_bounds__(32) k_fk_apply(const DevChain d) {
    if (d.status->done) return;
    const int tile = blockIdx.x, lane = threadIdx.x;
    const int j0 = (tile * 32 + lane) * J;
    if (j0 >= d.l) return;
    double B[12], T[12], Mb[12], Ma[12], Gj[12];
    aff_load(&d.tileE[12 * (size_t)tile], T);
    aff_load(&d.lane_ex[12 * ((size_t)tile * 32 + lane)], B);
    aff_compose(T, B, B);
#pragma unroll
    for (int k = 0; k < 12; ++k) Mb[k] = B[k];
#pragma unroll
    for (int q = 0; q < J; ++q) {
        const int jj = j0 + q;
        if (jj < d.l) {
            const double* u = &d.u0[3 * jj];
#pragma unroll
            for (int i = 0; i < 3; ++i) d.ucur[3 * jj + i] = Mb[3 * i] * u[0] + Mb[3 * i + 1] * u[1] + Mb[3 * i + 2] * u[2];
            aff_load(&d.G[12 * (size_t)jj], Gj);
            aff_compose(B, Gj, Ma);
            aff_store(&d.M[12 * ((size_t)jj + 1)], Ma);
#pragma unroll
            for (int i = 0; i < 3; ++i) d.pcur[3 * jj + i] = Ma[9 + i];
#pragma unroll
            for (int k = 0; k < 12; ++k) Mb[k] = Ma[k];
        }
    }
}

__global__ void k_fk_atoms(const DevChain d) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= d.n || d.status->done) return;
    const double* M = &d.M[12 * (size_t)d.link[a]];
    const double x = d.r0[3 * a], y = d.r0[3 * a + 1], z = d.r0[3 * a + 2];
#pragma unroll
    for (int i = 0; i < 3; ++i) d.r[3 * a + i] = M[3 * i] * x + M[3 * i + 1] * y + M[3 * i + 2] * z + M[9 + i];
}

template <int J>
void launch_fk_j(DevChain& d, cudaStream_t s) {
    k_fk_tile<J><<<d.ntiles, 32, 0, s>>>(d);
    k_fk_tilescan<<<1, 32, 0, s>>>(d);
    k_fk_apply<J><<<d.ntiles, 32, 0, s>>>(d);
    k_fk_atoms<<<(d.n + 127) / 128, 128, 0, s>>>(d);
}

}  // namespace

// joints per lane: the J minimising the dependent compositions, J in the tile pass plus 6 per
// 32-tile round of the tile scan plus J in the apply pass
int fk_joints_per_lane(int l) {
    int best = 1;
    long long best_cost = -1;
    for (int J = 1; J <= 32; J *= 2) {
        long long ntiles = (l + 32LL * J - 1) / (32LL * J);
        long long cost = 2LL * J + 6 * ((ntiles + 31) / 32);
        if (best_cost < 0 || cost < best_cost) {
            best = J;
            best_cost = cost;
        }
    }
    return best;
}

void launch_fk(DevChain& d, cudaStream_t s) {
    switch (d.fk_j) {
        case 1: launch_fk_j<1>(d, s); break;
        case 2: launch_fk_j<2>(d, s); break;
        case 4: launch_fk_j<4>(d, s); break;
        case 8: launch_fk_j<8>(d, s); break;
        case 16: launch_fk_j<16>(d, s); break;
        default: launch_fk_j<32>(d, s); break;
    }
}

}  // namespace kcm
