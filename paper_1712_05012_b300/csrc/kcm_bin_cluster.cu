// A2 binning of a single chain in one launch: the counting sort of Sec. 3.2 (cell counts, their
// exclusive scan, the atoms in slot order) run by one thread-block cluster of C CTAs (C <= 16), where
// the multi-block path takes a count kernel whose last block scans the counts and a placement kernel.
// The double-float centres and the box keys come from the kinematics (k_fk_apply); mixed mode only.
// In the step and evaluation graphs the cluster also forms the grid from the box (every CTA, one thread
// each), which the kinematics' last block does for the other binning kernels: the kinematics then end
// without that block's tail, and the grid code, run once on a dummy box before the wait for the
// kinematics (programmatic dependent launch), is already fetched when the real box arrives.
//
// CTA b holds atoms [b n / C, (b + 1) n / C) and the cells [b P, (b + 1) P) of the grid
// (P = ceil(cells / C)), whose counts, then starts within the range, live in its shared memory:
// - every atom's cell is counted by an atomic in the shared memory of the CTA that holds the cell
//   (distributed shared memory), its rank within the cell returned by that atomic;
// - each CTA scans its cells (a run of consecutive cells per thread, one block scan of the run sums)
//   and publishes its total; every CTA forms the offsets of all ranges from the totals;
// - each atom's slot is (offset of its cell's range) + (start within the range, read from the owner's
//   shared memory) + its rank; the slot-ordered copies are those of k_bin_place.
// The stages meet at cluster barriers; no global memory passes between them (a thread keeps the
// centres, cells and ranks of its atoms, at most kBcAtoms, in registers). Chains of up to 32,768 atoms:
// on longer ones (the 83,746-atom chain measured 36.6 us against 19 us for the multi-block kernels) the
// 16 SMs of a cluster are too few, and the multi-block kernels bin them.
//
// The cell of an atom and its offset from the cell corner are formed in double-float from the
// double-float centre (the grid origin, the box minimum, is an exact double-float: it is one of the
// centres) and rounded once to float, as the multi-block kernels do in mixed mode (mixed_cell,
// mixed_offset): the two give the same cells and offsets.
#include <cuda_runtime.h>

#include <cooperative_groups.h>

#include <algorithm>

#include "kcm_cells.cuh"
#include "kcm_common.cuh"
#include "kcm_df.cuh"
#include "kcm_device.h"

namespace kcm {

namespace cg = cooperative_groups;

namespace {
using namespace dev;

// the grid of the chain from its six box keys (lowest x, y, z, then highest; keys of double-float
// values), the arithmetic of the kinematics' last block (grid_from_bounds_df); not inlined, so that the
// run on a dummy box executes the very instructions of the real one
__device__ __noinline__ bool cluster_grid(unsigned long long k0, unsigned long long k1, unsigned long long k2,
                                          unsigned long long k3, unsigned long long k4, unsigned long long k5,
                                          double s_base, int stencil, double cell, long long cap, GridInfo* out) {
    df lo[3] = {dfkey_inv(k0), dfkey_inv(k1), dfkey_inv(k2)};
    const df hi[3] = {dfkey_inv(k3), dfkey_inv(k4), dfkey_inv(k5)};
    return grid_from_bounds_df(s_base, stencil, cell, lo, hi, cap, out);
}

constexpr int kBcThreads = 1024;
constexpr int kBcWarps = kBcThreads / 32;
constexpr int kBcAtoms = 2;                       // most atoms per thread
constexpr int kBcMaxCtas = 16;
constexpr int kBcMaxCells = 52 * 1024;            // most cells of a CTA's range (208 KB of shared memory)
constexpr int kBcAtomsPerCta = 512;               // atoms per CTA the plan aims at (half the threads: the
                                                  // shorter ranges of cells and atoms per CTA end sooner;
                                                  // 1,000-residue chain with 16 CTAs instead of 11: binning
                                                  // 16.1 -> 14.4 us, 95.0 -> 93.9 us per iteration)

__global__ void __launch_bounds__(kBcThreads) k_bin_cluster(const DevChain d) {
    extern __shared__ int4 sCell4[];  // the CTA's cell counts, then their starts within the range
    int* sCell = reinterpret_cast<int*>(sCell4);
    __shared__ int sWs[kBcWarps];
    __shared__ int sRange;  // atoms in the CTA's cells (read by every CTA)
    __shared__ int sOff[kBcMaxCtas + 1];
    __shared__ GridInfo sG;
    __shared__ bool sFinite;
    // the dummy box (1 A wide), before the wait for the kinematics (only with programmatic dependent
    // launch: otherwise the kernel starts after them and the run would only add its time); sG is rewritten
    if (d.grid_in_bin && d.pdl && threadIdx.x == 0) {
        const unsigned long long z = dfkey(df{0.0f, 0.0f}), o = dfkey(df{1.0f, 0.0f});
        sFinite = cluster_grid(z, z, z, o, o, o, d.s_base, d.stencil, d.prm.cell_size, 1 << 16, &sG);
    }
    grid_dep_sync();

    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks(), b = (int)cl.block_rank();
    if (d.status->done) return;  // the same for every CTA: nothing writes it while the kernel runs
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    Status* st = d.status;
    if (!d.grid_in_bin) {
        if (threadIdx.x == 0) { sG = d.grid[0]; sFinite = true; }
    } else if (threadIdx.x == 0) {
        unsigned long long k[6];  // every CTA reads the box before the cluster barrier; CTA 0 resets it after
#pragma unroll
        for (int i = 0; i < 6; ++i) k[i] = __ldcg(&d.cbox[i]);
        GridInfo gg;
        const bool fin = cluster_grid(k[0], k[1], k[2], k[3], k[4], k[5], d.s_base, d.stencil, d.prm.cell_size,
                                      d.ccap[0], &gg);
        sG = gg;
        sFinite = fin;
    }
    for (int i = threadIdx.x; i < d.bin_capc / 4; i += blockDim.x) sCell4[i] = make_int4(0, 0, 0, 0);
    const int a0 = (int)((long long)d.n * b / C), a1 = (int)((long long)d.n * (b + 1) / C);  // <= kBcAtoms each
    const df* rdf = reinterpret_cast<const df*>(d.rdf);
    // the thread's centres, loaded now so that they arrive while the grid is formed
    df p0[kBcAtoms][3];
#pragma unroll
    for (int k = 0; k < kBcAtoms; ++k) {
        const int at = a0 + k * kBcThreads + (int)threadIdx.x;
        if (at < a1) {
            p0[k][0] = rdf[3 * at]; p0[k][1] = rdf[3 * at + 1]; p0[k][2] = rdf[3 * at + 2];
        }
    }
    cl.sync();  // (1) every CTA's counts are zero, and every CTA has the grid
    const GridInfo g = sG;
    if (d.grid_in_bin && b == 0) {
        // after the barrier (every CTA has read the box): the box reset for the next evaluation, and what
        // the kinematics' last block records for the other binning kernels
        if (threadIdx.x < 6) d.cbox[threadIdx.x] = threadIdx.x < 3 ? ~0ULL : 0ULL;
        if (threadIdx.x == 32) d.grid[0] = g;
        if (threadIdx.x == 64) {
            d.chain_E[0] = 0.0; d.chain_E[1] = 0.0; d.chain_E[2] = 0.0;
            st->ncells = g.ncells;
            st->pairs = 0;
            st->nbr_total = 0;
            st->guard = 0;
            st->sasa_tests = 0;
            st->max_nbr = 0;
            st->nlong = 0;
            if (!sFinite) {  // non-finite centres: the chain fails and the loop ends
                d.chain_err[0] |= kErrNonfinite;
                d.chain_done[0] = 1;
                atomicOr(&st->error, kErrNonfinite);
                st->done = 1;
                export_status(d);
            }
        }
    }
    if (!sFinite) return;  // the same in every CTA (one box)
    const int nc = g.ncells, per = (nc + C - 1) / C;

    // ---- cell counts
    int key0[kBcAtoms], rank0[kBcAtoms];
    {
#pragma unroll
        for (int k = 0; k < kBcAtoms; ++k) {
            const int at = a0 + k * kBcThreads + (int)threadIdx.x;
            if (at >= a1) continue;
            const df px = p0[k][0], py = p0[k][1], pz = p0[k][2];
            const int cx = mixed_cell_axis(px, g.of[0], g.inv_sf, g.nx);
            const int cy = mixed_cell_axis(py, g.of[1], g.inv_sf, g.ny);
            const int cz = mixed_cell_axis(pz, g.of[2], g.inv_sf, g.nz);
            const int key = (cz * g.ny + cy) * g.nx + cx;
            const int owner = key / per;
            const unsigned peers = __match_any_sync(__activemask(), key);
            const int leader = __ffs(peers) - 1;
            int rk = 0;
            if (lane == leader) rk = atomicAdd(cl.map_shared_rank(sCell, owner) + (key - owner * per), __popc(peers));
            rk = __shfl_sync(peers, rk, leader) + __popc(peers & ((1u << lane) - 1u));
            key0[k] = key;
            rank0[k] = rk;
        }
    }
    cl.sync();  // (2) every count

    // ---- starts within the CTA's cells: each thread sums a run of consecutive cells, then one scan of
    // the run sums
    const int c0 = b * per, cn = max(0, min(nc, c0 + per) - c0);
    {
        const int K = (cn + (int)blockDim.x - 1) / (int)blockDim.x;
        const int i0 = min((int)threadIdx.x * K, cn), i1 = min(i0 + K, cn);
        int sum = 0;
        for (int i = i0; i < i1; ++i) sum += sCell[i];
        int v = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        if (lane == 31) sWs[w] = v;
        __syncthreads();
        int x = sWs[lane];  // kBcWarps == 32: every warp scans the warp sums (one int per lane)
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        const int before = __shfl_sync(0xffffffffu, x, max(w - 1, 0));
        int run = v - sum + (w > 0 ? before : 0);
        for (int i = i0; i < i1; ++i) {
            const int c = sCell[i];
            sCell[i] = run;
            run += c;
        }
        if (threadIdx.x == blockDim.x - 1) sRange = run;
    }
    cl.sync();  // (3) every CTA's starts and total
    if (w == 0) {  // the offsets of the CTAs' ranges
        int v = lane < C ? *cl.map_shared_rank(&sRange, lane) : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        if (lane < C) sOff[lane + 1] = v;
        if (lane == 0) sOff[0] = 0;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < cn; i += blockDim.x) d.cell_start[c0 + i] = sOff[b] + sCell[i];
    if (b == C - 1 && threadIdx.x == 0) d.cell_start[nc] = sOff[C];

    // ---- the atoms in slot order (as k_bin_place; the offsets from the cell corner in double-float, the
    // corner's multiple of the edge exact as a product of two floats)
    {
#pragma unroll
        for (int k = 0; k < kBcAtoms; ++k) {
            const int at = a0 + k * kBcThreads + (int)threadIdx.x;
            if (at >= a1) continue;
            const int key = key0[k], rk = rank0[k];
            const df px = p0[k][0], py = p0[k][1], pz = p0[k][2];
            const int owner = key / per;
            const int sl = sOff[owner] + cl.map_shared_rank(sCell, owner)[key - owner * per] + rk;
            if (d.prm.solvation) { d.Fcav[3 * at] = 0; d.Fcav[3 * at + 1] = 0; d.Fcav[3 * at + 2] = 0; }
            d.sorted[sl] = at;
            d.slot_cell[sl] = key;
            d.smask[sl] = make_ulonglong2(d.exm[at], d.m14m[at]);
            d.Fpx[3 * at] = 0; d.Fpx[3 * at + 1] = 0; d.Fpx[3 * at + 2] = 0;
            d.Fov[3 * at] = 0.0f; d.Fov[3 * at + 1] = 0.0f; d.Fov[3 * at + 2] = 0.0f;
            d.Fox[3 * at] = 0; d.Fox[3 * at + 1] = 0; d.Fox[3 * at + 2] = 0;
            d.nbr_cnt[at] = 0;
            const int cx = key % g.nx, cy = (key / g.nx) % g.ny, cz = key / (g.nx * g.ny);
            const float fx = mixed_offset(px, g.of[0], cx, g.sf);
            const float fy = mixed_offset(py, g.of[1], cy, g.sf);
            const float fz = mixed_offset(pz, g.of[2], cz, g.sf);
            d.spos32[sl] = make_float4(fx, fy, fz, (float)cx);
            d.sprm32[sl] = d.aprm32[at];
        }
    }
    // (4) no CTA leaves while another may still read its shared memory: every read above has returned
    // its value, so the arrival needs no release (no wait for this CTA's stores)
    asm volatile("barrier.cluster.arrive.relaxed.aligned;\n\tbarrier.cluster.wait.aligned;" ::: "memory");
}

size_t bin_cluster_smem(int capc) { return sizeof(int) * (size_t)capc; }

cudaLaunchConfig_t bin_cluster_config(const DevChain& d, cudaStream_t s, cudaLaunchAttribute* at) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(d.bin_c, 1, 1);
    cfg.blockDim = dim3(kBcThreads, 1, 1);
    cfg.dynamicSmemBytes = bin_cluster_smem(d.bin_capc);
    cfg.stream = s;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = d.bin_c;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;  // as launch_k
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = d.pdl ? 2 : 1;
    return cfg;
}

}  // namespace

// k_bin_cluster for single chains in mixed mode of up to kBcMaxCtas * kBcThreads * kBcAtoms atoms: about
// kBcAtomsPerCta atoms per CTA, at least as many CTAs as split the cell cap into ranges of at most
// kBcMaxCells, at most 16; the cluster must fit the device
cudaError_t plan_bin_cluster(DevChain& d, bool want) {
    d.bin_c = 0;
    if (!want || d.prm.precision != KCM_MIXED || d.nchains != 1 || d.n < 1 ||
        d.n > kBcMaxCtas * kBcThreads * kBcAtoms)
        return cudaSuccess;
    const long long cap = d.cell_cap;
    const long long c_atoms = (d.n + kBcAtomsPerCta - 1) / kBcAtomsPerCta;
    const long long c_cells = (cap + kBcMaxCells - 1) / kBcMaxCells;
    const int C = (int)std::max<long long>(1, std::min<long long>(kBcMaxCtas, std::max(c_atoms, c_cells)));
    const long long capc = ((cap + C - 1) / C + 3) / 4 * 4;
    if (capc > kBcMaxCells || (d.n + C - 1) / C > kBcThreads * kBcAtoms) return cudaSuccess;  // does not fit
    static bool attrs = false;  // function attributes: once per process
    if (!attrs) {
        cudaError_t e = cudaFuncSetAttribute(k_bin_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_bin_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bin_cluster_smem(kBcMaxCells));
        if (e != cudaSuccess) return e;
        attrs = true;
    }
    DevChain t = d;
    t.bin_c = C;
    t.bin_capc = (int)capc;
    cudaLaunchAttribute at[2];
    cudaLaunchConfig_t cfg = bin_cluster_config(t, nullptr, at);
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, k_bin_cluster, &cfg) != cudaSuccess || clusters < 1) {
        (void)cudaGetLastError();  // no such cluster on this device: the multi-block kernels
        return cudaSuccess;
    }
    d.bin_c = C;
    d.bin_capc = (int)capc;
    return cudaSuccess;
}

void launch_bin_cluster(DevChain& d, cudaStream_t s) {
    cudaLaunchAttribute at[2];
    const cudaLaunchConfig_t cfg = bin_cluster_config(d, s, at);
    cudaLaunchKernelEx(&cfg, k_bin_cluster, d);
}

}  // namespace kcm
