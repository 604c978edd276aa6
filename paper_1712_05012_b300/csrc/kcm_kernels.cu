// CUDA kernels of one KCM iteration for sm_103a (B300).
//
// Stages (Sec. 4.1 steps 4-8):
//   A1 forward kinematics: prefix product of per-joint affine transforms (FP64), Sec. 2.1 and
//      App. B; atom centres r = M_link(r^0)
//   A2 binning: bounding box, uniform grid (Sec. 3.2), counting sort by cell with warp-aggregated
//      atomics, cells ordered by atom index for determinism
//   A3-A5 pair forces over the 27- or 125-cell neighbourhood (eq. 02_2, 03_2, 03_8, 03_9) and the
//      solvation neighbour lists A'_i (Sec. 3.2 "neighbourhood matrix")
//   A6 surface enumeration, Algorithm 1 (Sec. 3.4), one warp per atom
//   A7-A8 link wrenches (eq. KCM_01/02) and the suffix sum of Sec. 3.5, tau_k = J_k^T P^agg_k
//   A9 clamped step (eq. KCM_07), A10 energies (eq. 01, G_cav_patch)
//
// B300 has about one FP64 FMA per 64 FP32 FMAs, so every FP64 stage is cut into many small blocks
// (a few threads each) that the scheduler spreads over all SMs; FP32 work uses full warps.
// Every reduction has a fixed order or is integer, so an iteration is bitwise reproducible.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <type_traits>

#include "kcm_cells.cuh"
#include "kcm_common.cuh"
#include "kcm_device.h"
#include "kcm_launch.h"

namespace kcm {

namespace {
using namespace dev;

// ================================================================ A2: binning
// (the bounding box and the grid are formed by the last block of the FK apply kernel)

// Cell of each atom (FP32 from the FP64 offset to the grid origin; the cell-edge margin makes
// the one-cell neighbourhood exact) and its rank within the cell, from one atomic per group of
// lanes that share a cell. Ranks depend on timing; nothing downstream depends on the order.
static_assert(kBinThreads == 1024, "the fused scan of k_bin_count scans 32 warp totals in one warp");
__global__ void __launch_bounds__(kBinThreads) k_bin_count(const DevChain d) {
    grid_dep_sync();
    __shared__ int ws[kBinThreads / 32];
    __shared__ bool last;
    if (d.status->done) return;
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (a < d.n) {
        const GridInfo g = d.grid[atom_chain(d, a)];
        int cx, cy, cz;
        if (d.prm.precision == KCM_MIXED) {  // from the double-float centres, no FP64 (kcm_cells.cuh)
            const df* p = reinterpret_cast<const df*>(d.rdf) + 3 * a;
            cx = mixed_cell_axis(p[0], g.of[0], g.inv_sf, g.nx);
            cy = mixed_cell_axis(p[1], g.of[1], g.inv_sf, g.ny);
            cz = mixed_cell_axis(p[2], g.of[2], g.inv_sf, g.nz);
        } else {
            cx = min(max((int)floorf((float)(d.r[3 * a] - g.ox) * g.inv_sf), 0), g.nx - 1);
            cy = min(max((int)floorf((float)(d.r[3 * a + 1] - g.oy) * g.inv_sf), 0), g.ny - 1);
            cz = min(max((int)floorf((float)(d.r[3 * a + 2] - g.oz) * g.inv_sf), 0), g.nz - 1);
        }
        int key = g.cbase + (cz * g.ny + cy) * g.nx + cx;
        d.key[a] = key;
        unsigned peers = __match_any_sync(__activemask(), key);
        int leader = __ffs(peers) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(&d.cell_count[key], __popc(peers));
        base = __shfl_sync(peers, base, leader);
        d.rank[a] = base + __popc(peers & ((1u << lane) - 1u));
    }
    if (!d.scan_fused) return;
    // small grids: the last block scans the cell counts, 4 * kBinThreads cells per pass with coalesced
    // int4 accesses (the loads of eight passes in flight together) and a carry between passes, and
    // zeroes them for the next evaluation
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&d.status->ticket_bin, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int nc = d.status->ncells;
    constexpr int kPass = 4 * kBinThreads;  // cells per pass
    constexpr int kPre = 8;                 // passes whose loads are in flight together
    int carry = 0;
    for (int g0 = 0; g0 < nc; g0 += kPre * kPass) {
        int k[kPre][4];
#pragma unroll
        for (int p = 0; p < kPre; ++p) {
            const int c = g0 + p * kPass + 4 * threadIdx.x;
            if (c + 3 < nc) {
                const int4 v4 = __ldcg(reinterpret_cast<const int4*>(&d.cell_count[c]));
                k[p][0] = v4.x; k[p][1] = v4.y; k[p][2] = v4.z; k[p][3] = v4.w;
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) k[p][q] = c + q < nc ? __ldcg(&d.cell_count[c + q]) : 0;
            }
        }
#pragma unroll
        for (int p = 0; p < kPre; ++p) {
            if (g0 + p * kPass >= nc) break;  // uniform
            const int c = g0 + p * kPass + 4 * threadIdx.x;
            const int local = k[p][0] + k[p][1] + k[p][2] + k[p][3];
            int v = local;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += y;
            }
            if (lane == 31) ws[w] = v;
            __syncthreads();
            if (w == 0) {
                int x = ws[lane];
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, x, o);
                    if (lane >= o) x += y;
                }
                ws[lane] = x;
            }
            __syncthreads();
            const int s0 = carry + v - local + (w > 0 ? ws[w - 1] : 0);
            const int st[4] = {s0, s0 + k[p][0], s0 + k[p][0] + k[p][1], s0 + k[p][0] + k[p][1] + k[p][2]};
            if (c + 3 < nc) {
                *reinterpret_cast<int4*>(&d.cell_start[c]) = make_int4(st[0], st[1], st[2], st[3]);
                *reinterpret_cast<int4*>(&d.cell_count[c]) = make_int4(0, 0, 0, 0);
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (c + q < nc) { d.cell_start[c + q] = st[q]; d.cell_count[c + q] = 0; }
            }
            carry += ws[kBinThreads / 32 - 1];
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) d.cell_start[nc] = carry;
    if (threadIdx.x == 0) d.status->ticket_bin = 0u;
}

// exclusive scan of the cell counts in two passes over blocks of kScanCells cells: block sums,
// then each block adds the sums of the blocks before it and scans its own cells (and zeroes the
// counts for the next iteration)
__global__ void k_scan_sums(const DevChain d) {
    grid_dep_sync();
    __shared__ int ws[32];
    if (d.status->done) return;
    int nc = d.status->ncells;
    int c0 = blockIdx.x * kScanCells;
    if (c0 >= nc) return;
    int s = 0;
    for (int c = c0 + threadIdx.x; c < min(nc, c0 + kScanCells); c += blockDim.x) s += d.cell_count[c];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int k2 = 0; k2 < (int)(blockDim.x >> 5); ++k2) t += ws[k2];
        d.scan_part[blockIdx.x] = t;
    }
}

__global__ void k_scan_cells(const DevChain d) {
    grid_dep_sync();
    __shared__ int ws[32];
    __shared__ int base_s;
    if (d.status->done) return;
    int nc = d.status->ncells;
    int c0 = blockIdx.x * kScanCells;
    if (c0 >= nc) return;
    // sum of the previous blocks' counts
    int s = 0;
    for (int b = threadIdx.x; b < (int)blockIdx.x; b += blockDim.x) s += d.scan_part[b];
    s = warp_sum(s);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) ws[w] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int k2 = 0; k2 < nw; ++k2) t += ws[k2];
        base_s = t;
    }
    __syncthreads();
    int base = base_s;
    // each thread owns kScanCells / blockDim.x consecutive cells
    const int per = kScanCells / kScanThreadsBig;
    int cb = c0 + threadIdx.x * per;
    int cnt[kScanCells / kScanThreadsBig];
    int local = 0;
#pragma unroll
    for (int q = 0; q < per; ++q) {
        int c = cb + q;
        cnt[q] = c < nc ? d.cell_count[c] : 0;
        local += cnt[q];
    }
    int v = local;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    __syncthreads();
    if (lane == 31) ws[w] = v;
    __syncthreads();
    if (w == 0) {
        int x = lane < nw ? ws[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        ws[lane] = x;
    }
    __syncthreads();
    int run = base + v - local + (w > 0 ? ws[w - 1] : 0);
#pragma unroll
    for (int q = 0; q < per; ++q) {
        int c = cb + q;
        if (c < nc) {
            d.cell_start[c] = run;
            d.cell_count[c] = 0;
            run += cnt[q];
            if (c == nc - 1) d.cell_start[nc] = run;
        }
    }
}

// sorted slot = start of the cell + rank; sorted copies: FP64 centres, or FP32 offsets from the
// cell corner (|offset| <= s plus the assignment margin, rounding below s 2^-24). The ranks come from
// atomics, so the order within a cell depends on timing: mixed mode sums its pair terms in exact fixed
// point and does not depend on it; FP64 mode only records the slot here and k_bin_stable puts each
// cell's atoms in atom order, so that its floating-point sums, and with them the torques, are the same
// from run to run.
template <bool MIXED>
__global__ void k_bin_place(const DevChain d) {
    grid_dep_sync();
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= d.n || d.status->done) return;
    int key = d.key[a];
    int sl = d.cell_start[key] + d.rank[a];
    if (d.prm.solvation) {  // Algorithm 1 adds its exchanges to both atoms of a pair: zero the sums (no memset node)
        d.Fcav[3 * a] = 0; d.Fcav[3 * a + 1] = 0; d.Fcav[3 * a + 2] = 0;
    }
    if (!MIXED) {
        d.sorted_tmp[sl] = a;
        return;
    }
    const int ca = atom_chain(d, a);
    const GridInfo g = d.grid[ca];
    d.sorted[sl] = a;
    if (d.nchains > 1) d.slot_chain[sl] = ca;
    d.slot_cell[sl] = key;
    d.smask[sl] = make_ulonglong2(d.exm[a], d.m14m[a]);  // bond classes in slot order (no dependent load later)
    if (MIXED) {
        // the pair kernel adds each pair's share to both atoms: zero the sums and the list counters
        d.Fpx[3 * a] = 0; d.Fpx[3 * a + 1] = 0; d.Fpx[3 * a + 2] = 0;
        d.Fov[3 * a] = 0.0f; d.Fov[3 * a + 1] = 0.0f; d.Fov[3 * a + 2] = 0.0f;
        d.Fox[3 * a] = 0; d.Fox[3 * a + 1] = 0; d.Fox[3 * a + 2] = 0;
        d.nbr_cnt[a] = 0;
        const int lk = key - g.cbase;
        int cx = lk % g.nx, cy = (lk / g.nx) % g.ny, cz = lk / (g.nx * g.ny);
        const df* pc = reinterpret_cast<const df*>(d.rdf) + 3 * a;  // no FP64 (kcm_cells.cuh)
        const float ox = mixed_offset(pc[0], g.of[0], cx, g.sf);
        const float oy = mixed_offset(pc[1], g.of[1], cy, g.sf);
        const float oz = mixed_offset(pc[2], g.of[2], cz, g.sf);
        float4 p = d.aprm32[a];
        d.spos32[sl] = make_float4(ox, oy, oz, (float)cx);  // w: the cell's x index (exact), for the pair shifts
        d.sprm32[sl] = p;
    }
}

// Mixed-mode batches: the cells, ranks and cell starts of every chain in one launch, one block per
// chain (in place of the count kernel and the two scan kernels). A chain's cells are consecutive in
// the global cell numbering and hold exactly its atoms, so its slots are [atom_off[c], atom_off[c + 1])
// and a block sorts its chain alone: the cell and rank of each atom from atomics on counts in shared
// memory (in the chain's part of the global counts when its grid has more than kBinChainCells cells,
// which the scan leaves at zero again), then a block scan of the counts into the cell starts.
// k_bin_place<true> then places the atoms, one thread each. The cell arithmetic is that of
// k_bin_count; only the order of the atoms within a cell (from atomics, as there) can differ, and no
// mixed-mode result depends on it.
constexpr int kBinChainThreads = 1024;
constexpr int kBinChainCells = 8192;
constexpr int kBinChainBatch = 1;  // atoms per thread whose centres are loaded together (two loaded together spill at the
                                   // 32 registers of two blocks per SM, and measured 1-2 us slower on the batch)

__global__ void __launch_bounds__(kBinChainThreads, 2) k_bin_chains(const DevChain d) {
    grid_dep_sync();
    __shared__ int scnt[kBinChainCells];
    __shared__ int ws[kBinChainThreads / 32];
    if (d.status->done) return;
    const int c = blockIdx.x, t = threadIdx.x, lane = t & 31, w = t >> 5;
    const GridInfo g = d.grid[c];
    const int a0 = d.atom_off[c], a1 = d.atom_off[c + 1];
    const int nc = g.ncells;
    const bool sm = nc <= kBinChainCells;
    int* cnt = sm ? scnt : d.cell_count + g.cbase;
    if (sm)
        for (int k = t; k < nc; k += kBinChainThreads) scnt[k] = 0;
    __syncthreads();
    const df* rdf = reinterpret_cast<const df*>(d.rdf);
    for (int ab = a0; ab < a1; ab += kBinChainBatch * kBinChainThreads) {  // uniform
        df p[kBinChainBatch][3];
#pragma unroll
        for (int i = 0; i < kBinChainBatch; ++i) {
            const int a = ab + i * kBinChainThreads + t;
#pragma unroll
            for (int k = 0; k < 3; ++k) p[i][k] = a < a1 ? rdf[3 * a + k] : df{0.0f, 0.0f};
        }
#pragma unroll
        for (int i = 0; i < kBinChainBatch; ++i) {
            const int a = ab + i * kBinChainThreads + t;
            if (a < a1) {
                const int cx = mixed_cell_axis(p[i][0], g.of[0], g.inv_sf, g.nx);
                const int cy = mixed_cell_axis(p[i][1], g.of[1], g.inv_sf, g.ny);
                const int cz = mixed_cell_axis(p[i][2], g.of[2], g.inv_sf, g.nz);
                const int lk = (cz * g.ny + cy) * g.nx + cx;
                d.key[a] = g.cbase + lk;
                const unsigned peers = __match_any_sync(__activemask(), lk);
                const int leader = __ffs(peers) - 1;
                int base = 0;
                if (lane == leader) base = atomicAdd(&cnt[lk], __popc(peers));
                base = __shfl_sync(peers, base, leader);
                d.rank[a] = base + __popc(peers & ((1u << lane) - 1u));
            }
        }
    }
    __syncthreads();
    // exclusive scan of the counts, four consecutive cells per thread and pass; cell_start holds slots
    int carry = 0;
    for (int c0 = 0; c0 < nc; c0 += 4 * kBinChainThreads) {  // uniform
        const int cb = c0 + 4 * t;
        int k[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)  // global counts from L2: a line may be in L1 from a neighbouring chain's block
            k[q] = cb + q >= nc ? 0 : (sm ? scnt[cb + q] : __ldcg(&cnt[cb + q]));
        const int local = k[0] + k[1] + k[2] + k[3];
        int v = local;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        if (lane == 31) ws[w] = v;
        __syncthreads();
        if (w == 0) {
            int x = ws[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            ws[lane] = x;
        }
        __syncthreads();
        int run = carry + v - local + (w > 0 ? ws[w - 1] : 0);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (cb + q < nc) {
                d.cell_start[g.cbase + cb + q] = a0 + run;
                if (!sm) cnt[cb + q] = 0;  // global counts are left at zero for the next evaluation
                run += k[q];
            }
        }
        carry += ws[kBinChainThreads / 32 - 1];
        __syncthreads();
    }
    if (t == 0) d.cell_start[g.cbase + nc] = a0 + carry;  // = a1: the next chain's first cell start
}

// FP64 mode: the atoms of each cell in atom order (a stable counting sort): the atom at slot s of the
// placement by atomic ranks takes slot (cell start) + (atoms of its cell with a smaller index)
__global__ void k_bin_stable(const DevChain d) {
    grid_dep_sync();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= d.n || d.status->done) return;
    const int a = d.sorted_tmp[s];
    const int key = d.key[a];
    const int cs = d.cell_start[key], ce = d.cell_start[key + 1];
    int r = 0;
    for (int t = cs; t < ce; ++t) r += d.sorted_tmp[t] < a;
    const int sl = cs + r;
    d.sorted[sl] = a;
    if (d.nchains > 1) d.slot_chain[sl] = atom_chain(d, a);
    d.slot_cell[sl] = key;
    d.smask[sl] = make_ulonglong2(d.exm[a], d.m14m[a]);
    const dbl4 p = d.aprm64[a];
    d.spos64[sl] = make_dbl4(d.r[3 * a], d.r[3 * a + 1], d.r[3 * a + 2], p.x);
    d.sprm64[sl] = p;
}

// ================================================================ A3-A5: pair forces + lists
// One warp per home atom i (sorted slot). The neighbourhood is the (2 KR + 1)^3 cells around the home
// cell (KR = 1 for cells at least as wide as the largest interaction range, KR = 2 for cells down to
// half of it). Cells adjacent in x are adjacent in slot order, so the stencil is walked as x-rows,
// lane t taking row t: each row is one slot range, trimmed at both ends to the cells that lie within
// reach of the home atom. The candidates of the rows are then taken in strides of 32 over their
// concatenation, so every lane has the same trip count.
//
// FP64 mode walks the whole stencil and evaluates every ordered pair (i, j) in i's warp, so each
// atom's force is one warp's sum in a fixed order. Mixed mode evaluates each unordered pair once
// (Newton's third law): the home row from the atom after i up to +KR cells, the rows (dy > 0, dz = 0)
// and the rows with dz > 0, i.e. half the stencil. Its FP32 terms are summed in fixed point (units of
// 2^-23, see fx_add): the pair term is computed symmetrically and its fixed-point pieces are rounded
// symmetrically, so i keeps the pieces and j receives their exact negative by one 64-bit integer
// atomic add per component. The sums are exact and order-free, hence bitwise what the full-stencil
// evaluation gives, and the forces of a pair cancel exactly, so no net force or moment builds up over
// the chain. Terms of 2^22 kcal/mol/A or more (near-overlapping atoms) go to float side sums. The
// solvation neighbour lists take both directions of each pair, at slots drawn by atomic counters;
// Algorithm 1's mixed kernel does not depend on the order of a list. The per-atom results stay
// integers here; the thread-per-atom consumers convert them to FP64 (a warp-per-atom kernel would
// spend a whole FP64 warp instruction on each atom's lane 0).
template <bool MIXED, int KR, int W>
__global__ void __launch_bounds__(W * 32, (MIXED ? 32 : 24) / W) k_pair(const DevChain d) {
    grid_dep_sync();
    typedef typename std::conditional<MIXED, float, double>::type R;
    typedef typename std::conditional<MIXED, float4, dbl4>::type QV;
    constexpr int kW = 2 * KR + 1;  // cells per row
    constexpr bool HALF = MIXED;    // half stencil, each unordered pair once
    constexpr int kRows = HALF ? 1 + KR + KR * kW : kW * kW;
    static_assert(kRows <= 32, "one lane per row");
    __shared__ int s_beg[W][32];
    __shared__ int s_off[W][32];
    __shared__ float2 s_sh[W][32];
    __shared__ QV s_qv[W][kPairQueue];   // queued pairs: r_i - r_j, d^2
    __shared__ int s_qts[W][kPairQueue];  // queued pairs: sorted slot of j
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // a block takes atoms sl, sl + (blocks) W, ...: one round with the full grid, several with the
    // persistent grid (one block per resident slot); the loop form also compiles better for one round
    for (int sl = blockIdx.x * W + w; sl < d.n; sl += gridDim.x * W) {
    R Eel = 0, Evdw = 0;
    unsigned npairs = 0, nguard = 0;
    int ncount = 0;
    int ca = -1;  // chain of the home atom
    if (sl < d.n && !d.status->done) {
        const int a = d.sorted[sl];
        const int scell = d.slot_cell[sl];  // loaded beside the atom (independent of it)
        float4 hpos = make_float4(0.0f, 0.0f, 0.0f, 0.0f);  // mixed: the home atom's offset, likewise
        if constexpr (MIXED) hpos = d.spos32[sl];
        ca = slot_chain(d, sl);
        const GridInfo g = d.grid[ca];  // the home atom's chain: its candidates are that chain's atoms
        if (!d.chain_done[ca]) {  // a converged chain takes no more steps: no forces needed
        const int cell = scell - g.cbase;
        const int cx = cell % g.nx, cy = (cell / g.nx) % g.ny, cz = cell / (g.nx * g.ny);
        // The non-empty rows, compacted in stencil order: first slot, offset of their candidates in
        // the concatenation, and (mixed) the row's shift ((cy_j - cy_i) s, (cz_j - cz_i) s). A cell
        // whose box lies farther from the home atom than the largest interaction range (less a margin
        // over the FP32 cell assignment) holds no candidate: whole rows, and the cells at either end
        // of a row, are dropped that way.
        int beg = 0, len = 0;
        // row of this lane: (dy, dz) and the lowest x offset it takes
        int dyc, dzc, dxlo = -KR;
        if constexpr (HALF) {
            if (lane == 0) { dyc = 0; dzc = 0; dxlo = 0; }                  // home row: i's cell onwards
            else if (lane <= KR) { dyc = lane; dzc = 0; }                    // dy > 0, dz = 0
            else { const int r = lane - 1 - KR; dyc = r % kW - KR; dzc = 1 + r / kW; }  // dz > 0
        } else {
            dyc = lane % kW - KR;
            dzc = lane / kW - KR;
        }
        if (lane < kRows) {
            const int ncy = cy + dyc, ncz = cz + dzc;
            if (ncy >= 0 && ncy < g.ny && ncz >= 0 && ncz < g.nz) {
                R hx, hy, hz, es, reach2;
                if constexpr (MIXED) {
                    const float4 hp = hpos;  // offset from the home cell's corner
                    hx = hp.x; hy = hp.y; hz = hp.z; es = g.sf; reach2 = d.f_rall2;
                } else {
                    const dbl4 hp = d.spos64[sl];
                    hx = hp.x - (g.ox + cx * g.s); hy = hp.y - (g.oy + cy * g.s); hz = hp.z - (g.oz + cz * g.s);
                    es = g.s; reach2 = d.rmax * d.rmax;
                }
                const R mg = (R)0.02;
                // gap between the home atom and the cell at offset k along one axis (0 inside)
                auto gap = [&](int k, R h) -> R {
                    return k > 0 ? fmax((R)k * es - h - mg, (R)0) : (k < 0 ? fmax(h - (R)(k + 1) * es - mg, (R)0) : (R)0);
                };
                const R gy = gap(dyc, hy), gz = gap(dzc, hz);
                const R rem = reach2 - (gy * gy + gz * gz);
                if (rem >= (R)0) {
                    // the gap grows with |dx|: the cells within reach are one run around the home cell
                    int xlo = max(cx + dxlo, 0), xhi = min(cx + KR, g.nx - 1);
#pragma unroll
                    for (int k = 1; k <= KR; ++k) {
                        const R gl = gap(-k, hx), gr = gap(k, hx);
                        if (gl * gl > rem) xlo = max(xlo, cx - k + 1);
                        if (gr * gr > rem) xhi = min(xhi, cx + k - 1);
                    }
                    const int rb = g.cbase + (ncz * g.ny + ncy) * g.nx;
                    // the home row of the half stencil starts after i itself
                    beg = (HALF && lane == 0) ? sl + 1 : d.cell_start[rb + xlo];
                    len = d.cell_start[rb + xhi + 1] - beg;
                }
            }
        }
        int incl = len;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        const unsigned nem = __ballot_sync(0xffffffffu, len > 0);
        const int nne = __popc(nem);
        if (len > 0) {
            const int cslot = __popc(nem & ((1u << lane) - 1u));
            s_beg[w][cslot] = beg;
            s_off[w][cslot] = incl - len;
            s_sh[w][cslot] = make_float2((float)dyc * g.sf, (float)dzc * g.sf);
        }
        __syncwarp();
        R K, w14e, w14v, rc2, rv2, rall2, gp, dr, pad;
        if constexpr (MIXED) {
            K = d.f_K; w14e = d.f_w14e; w14v = d.f_w14v; rc2 = d.f_rc2; rv2 = d.f_rv2; rall2 = d.f_rall2;
            gp = g.gpf; dr = d.f_dr; pad = 0.01f;
        } else {
            K = d.prm.coulomb_k; w14e = d.prm.w14_elec; w14v = d.prm.w14_vdw; rc2 = d.rcut2; rv2 = d.rvdw2;
            rall2 = d.rmax * d.rmax; gp = 0.0; dr = d.prm.delta_r; pad = 0.0;
        }
        const bool solv = d.prm.solvation != 0;
        const R sf = (R)g.sf;
        R px, py, pz, qi, sei, Ri, Roi;
        float fcx = 0.0f;  // mixed: the home cell's x index
        if constexpr (MIXED) {
            float4 p = hpos, q = d.sprm32[sl];
            px = p.x; py = p.y; pz = p.z; fcx = p.w; qi = q.x; sei = q.y; Ri = q.z; Roi = q.w;
        } else {
            dbl4 p = d.spos64[sl], q = d.sprm64[sl];
            px = p.x; py = p.y; pz = p.z; qi = p.w; sei = q.y; Ri = q.z; Roi = q.w;
        }
        const unsigned long long exa = d.exm[a], m14a = d.m14m[a];
        int hix = 0, hiy = 0, hiz = 0;                           // mixed: integer parts (kcal/mol/A)
        int lox = 0, loy = 0, loz = 0;                           // mixed: fractions in units of 2^-23
        float ove = 0, ovv = 0;                                  // mixed: energies
        double dfx = 0, dfy = 0, dfz = 0;                        // FP64 mode
        int t = 0;
        const unsigned lt = (1u << lane) - 1u;
        // Phase A filters the candidates by distance and queues the in-range ones, in candidate order,
        // in a ring of kPairQueue; phase B evaluates 32 queued pairs at a time, so the pair terms run
        // with every lane busy instead of the ~30 % of candidates that are in range.
        int qhead = 0, qtail = 0, nround = 0;
        bool ovf = false;     // half stencil: a list slot beyond kMaxNbr
        // mixed: the home atom's lane sums, reduced exactly (int32 pieces |.| <= 2^30 by 32-bit warp
        // reductions of their biased 16-bit halves) and added to its fixed-point force, at the end and
        // after every kPairFoldRounds pair rounds (so that the int32 lane sums cannot overflow)
        auto flush_sums = [&]() {
            const long long Hx = warp_sum_i32(hix), Hy = warp_sum_i32(hiy), Hz = warp_sum_i32(hiz);
            const long long Lx = warp_sum_i32(lox), Ly = warp_sum_i32(loy), Lz = warp_sum_i32(loz);
            if (lane == 0) {
                unsigned long long* Fi = reinterpret_cast<unsigned long long*>(&d.Fpx[3 * a]);
                atomicAdd(Fi, (unsigned long long)(Hx * 8388608LL + Lx));
                atomicAdd(Fi + 1, (unsigned long long)(Hy * 8388608LL + Ly));
                atomicAdd(Fi + 2, (unsigned long long)(Hz * 8388608LL + Lz));
            }
            hix = hiy = hiz = lox = loy = loz = 0;
        };
        auto phase_b = [&](int nvalid) {
            const int e = (qhead + lane) & (kPairQueue - 1);
            const bool act = lane < nvalid;
            bool isn = false;
            int b = -1, ts = 0;
            R ddx = 0, ddy = 0, ddz = 0, d2 = 0, qj = 0, sej = 0, Rj = 0, Roj = 0;
            ulonglong2 mk = make_ulonglong2(0ULL, 0ULL);
            if (act) {
                ts = s_qts[w][e];
                const QV v = s_qv[w][e];
                ddx = v.x; ddy = v.y; ddz = v.z; d2 = v.w;
                b = d.sorted[ts];
                mk = d.smask[ts];  // j's bond-class masks, loaded beside its index
                if constexpr (MIXED) {
                    float4 q = d.sprm32[ts];
                    qj = q.x; sej = q.y; Rj = q.z; Roj = q.w;
                } else {
                    dbl4 q = d.sprm64[ts];
                    qj = q.x; sej = q.y; Rj = q.z; Roj = q.w;
                }
                if (solv) {  // solvation neighbour A'_i: d_ij <= Roff_i + Roff_j + dr
                    if constexpr (MIXED) {
                        isn = solv_near_f32(d2, Roi, Roj, dr, pad);
                    } else {
                        R lim = Roi + Roj + dr + pad;
                        isn = d2 <= lim * lim;
                    }
                }
            }
            const unsigned bm = __ballot_sync(0xffffffffu, isn);
            // half stencil: list slots of both directions, requested before the pair term so that the
            // atomics' latency overlaps it
            int base_slot = 0, rslot = 0;
            if constexpr (HALF) {
                if (bm) {  // uniform
                    if (lane == 0) base_slot = atomicAdd(&d.nbr_cnt[a], __popc(bm));
                    if (isn) rslot = atomicAdd(&d.nbr_cnt[b], 1);
                }
            }
            if (act) {
                int lo = min(a, b), off = max(a, b) - lo;
                bool excl = false, is14 = false;
                if (off <= kMaskWindow) {
                    unsigned long long em = (lo == a) ? exa : mk.x;
                    unsigned long long mm = (lo == a) ? m14a : mk.y;
                    excl = (em >> off) & 1ULL;
                    is14 = (mm >> off) & 1ULL;
                }
                bool inE = !excl && d2 <= rc2, inV = !excl && d2 <= rv2;
                if (MIXED && !excl && (fabs(d2 - rc2) <= gp || fabs(d2 - rv2) <= gp)) {
                    // guard band: decide the cutoff in FP64 exactly as the FP64 path does
                    double ex = __dsub_rn(centre64(d, a, 0), centre64(d, b, 0)),
                           ey = __dsub_rn(centre64(d, a, 1), centre64(d, b, 1)),
                           ez = __dsub_rn(centre64(d, a, 2), centre64(d, b, 2));
                    double d64 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
                    inE = d64 <= d.rcut2;
                    inV = d64 <= d.rvdw2;
                    ++nguard;
                }
                if (inE || inV) {
                    // symmetric in (i, j): products of the two atoms' constants are formed first
                    const R we = is14 ? w14e : (R)1, wv = is14 ? w14v : (R)1;
                    R coef = 0, e_el = 0, e_vd = 0;
                    if constexpr (MIXED) {
                        const PairTermF pt = pair_term_f32(d2, qi, qj, sei, sej, Ri, Rj, K, we, wv, inE, inV);
                        coef = pt.coef; e_el = pt.e_el; e_vd = pt.e_vd;
                    } else {
                    const R inv2 = 1.0 / d2;
                    if (inE) {
                        const R qq = (we * K) * (qi * qj);
                        coef += (R)0.5 * qq * (inv2 * inv2);
                        e_el = (R)0.25 * qq * inv2;
                    }
                    if (inV) {
                        const R D = Ri + Rj;
                        const R D2 = D * D;
                        const R x2 = D2 * inv2;
                        const R t6 = x2 * x2 * x2;
                        const R t12 = t6 * t6;
                        const R eij = wv * (sei * sej);
                        coef += (R)12 * eij * (t12 - t6) * inv2;
                        e_vd = eij * (t12 - (R)2 * t6);
                    }
                    }
                    // mixed: a near-coincident pair (d of a few thousandths of an A) would overflow the FP32
                    // term; pair_term_f32 holds it at a large finite repulsion, so the torques stay finite
                    // and the clamped step goes ahead as on the FP64 path
                    const bool count_e = HALF || a < b;  // each unordered pair's energy once
                    if (count_e && (we != (R)0 || wv != (R)0)) ++npairs;
                    if constexpr (MIXED) {
                        const float fx1 = __fmul_rn(coef, ddx), fy1 = __fmul_rn(coef, ddy), fz1 = __fmul_rn(coef, ddz);
                        unsigned long long* Fj = reinterpret_cast<unsigned long long*>(&d.Fpx[3 * b]);
                        if (fabsf(fx1) < kPairFxMax && fabsf(fy1) < kPairFxMax && fabsf(fz1) < kPairFxMax) {
                            int n0, f0, n1, f1, n2, f2;
                            fx_pieces(fx1, n0, f0);
                            fx_pieces(fy1, n1, f1);
                            fx_pieces(fz1, n2, f2);
                            hix += n0; lox += f0; hiy += n1; loy += f1; hiz += n2; loz += f2;
                            // j's term is exactly the negative (two's complement adds)
                            atomicAdd(Fj, (unsigned long long)(-fx_units(n0, f0)));
                            atomicAdd(Fj + 1, (unsigned long long)(-fx_units(n1, f1)));
                            atomicAdd(Fj + 2, (unsigned long long)(-fx_units(n2, f2)));
                        } else {  // clash-sized (or non-finite) term
                            add_oversized(d, a, b, fx1, fy1, fz1);
                        }
                        if (count_e) { ove += e_el; ovv += e_vd; }
                    } else {
                        dfx += coef * ddx; dfy += coef * ddy; dfz += coef * ddz;
                        if (count_e) { Eel += e_el; Evdw += e_vd; }
                    }
                }
            }
            if constexpr (HALF) {
                if (bm) {  // uniform
                    base_slot = __shfl_sync(0xffffffffu, base_slot, 0);
                    if (isn) {
                        const int slot = base_slot + __popc(bm & lt);
                        if (slot < kMaxNbr) {  // j in i's list: r_j - r_i, Roff_j^2
                            d.nbr[(size_t)a * kMaxNbr + slot] = b;
                            d.nbr_off[(size_t)a * kMaxNbr + slot] = make_float4(-(float)ddx, -(float)ddy, -(float)ddz, __fmul_rn((float)Roj, (float)Roj));
                        }
                        if (rslot < kMaxNbr) {  // i in j's list: r_i - r_j, Roff_i^2
                            d.nbr[(size_t)b * kMaxNbr + rslot] = a;
                            d.nbr_off[(size_t)b * kMaxNbr + rslot] = make_float4((float)ddx, (float)ddy, (float)ddz, __fmul_rn((float)Roi, (float)Roi));
                        }
                        ovf |= slot >= kMaxNbr || rslot >= kMaxNbr;
                        // an atom whose list passes kSasaStage entries goes to the long-list kernels
                        // (the append that draws slot kSasaStage is unique)
                        if (slot == kSasaStage) d.long_atoms[atomicAdd(&d.status->nlong, 1)] = a;
                        if (rslot == kSasaStage) d.long_atoms[atomicAdd(&d.status->nlong, 1)] = b;
                    }
                    ncount += 2 * __popc(bm);
                }
            } else {
                if (isn) {
                    const int slot = ncount + __popc(bm & lt);
                    if (slot < kMaxNbr) {
                        d.nbr[(size_t)a * kMaxNbr + slot] = b;
                        if (MIXED) d.nbr_off[(size_t)a * kMaxNbr + slot] = make_float4(-(float)ddx, -(float)ddy, -(float)ddz, (float)(Roj * Roj));
                    }
                }
                ncount += __popc(bm);
            }
            qhead += 32;
            if constexpr (MIXED) {
                // at most one term per lane and round: kPairFoldRounds terms of |piece| <= 2^22 fit in int32
                if (++nround == kPairFoldRounds) {
                    flush_sums();
                    nround = 0;
                }
            }
        };
        for (int base = 0; base < total; base += 32) {
            const int k2 = base + lane;
            bool inr = false;
            QV v;
            int ts = 0;
            if (k2 < total) {
                while (t < nne - 1 && s_off[w][t + 1] <= k2) ++t;
                ts = s_beg[w][t] + (k2 - s_off[w][t]);
                if (ts != sl) {
                    R ddx, ddy, ddz;
                    if constexpr (MIXED) {
                        const float4 p = d.spos32[ts];
                        const float2 sh = s_sh[w][t];
                        // r_i - r_j = (o_i - o_j) - (c_j - c_i) s; (cx_j - cx_i) s is exact
                        ddx = pair_delta_f32(px, p.x, __fmul_rn(__fsub_rn(p.w, fcx), sf));
                        ddy = pair_delta_f32(py, p.y, sh.x);
                        ddz = pair_delta_f32(pz, p.z, sh.y);
                    } else {
                        dbl4 p = d.spos64[ts];
                        ddx = __dsub_rn(px, p.x); ddy = __dsub_rn(py, p.y); ddz = __dsub_rn(pz, p.z);
                    }
                    R d2;
                    if constexpr (MIXED) d2 = pair_d2_f32(ddx, ddy, ddz);
                    else d2 = __dadd_rn(__dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy)), __dmul_rn(ddz, ddz));
                    inr = d2 <= rall2;
                    v.x = ddx; v.y = ddy; v.z = ddz; v.w = d2;
                }
            }
            const unsigned bm = __ballot_sync(0xffffffffu, inr);
            if (inr) {
                const int e = (qtail + __popc(bm & lt)) & (kPairQueue - 1);
                s_qv[w][e] = v;
                s_qts[w][e] = ts;
            }
            qtail += __popc(bm);
            __syncwarp();
            if (qtail - qhead >= 32) phase_b(32);
            __syncwarp();
        }
        if (qtail > qhead) phase_b(qtail - qhead);
        if constexpr (MIXED) {
            flush_sums();  // added to the partners' shares; converted to FP64 by the thread-per-atom consumers
            ove = warp_sum(ove); ovv = warp_sum(ovv);
            Eel = ove;
            Evdw = ovv;
        } else {
            dfx = warp_sum(dfx); dfy = warp_sum(dfy); dfz = warp_sum(dfz);
            Eel = warp_sum(Eel); Evdw = warp_sum(Evdw);
            if (lane == 0) { d.Fpair[3 * a] = dfx; d.Fpair[3 * a + 1] = dfy; d.Fpair[3 * a + 2] = dfz; }
        }
        npairs = __reduce_add_sync(0xffffffffu, npairs);
        nguard = __reduce_add_sync(0xffffffffu, nguard);
        if constexpr (HALF) {
            ovf = __any_sync(0xffffffffu, ovf);
        } else {
            ovf = ncount > kMaxNbr;
        }
        if (lane == 0) {
            if (!HALF) {
                d.nbr_cnt[a] = ncount;
                if (ncount > kSasaStage) d.long_atoms[atomicAdd(&d.status->nlong, 1)] = a;
            }
            if (ovf) {
                atomicOr(&d.status->error, kErrOverflow);
                atomicOr(&d.chain_err[ca], kErrOverflow);
            }
        }
        }
        // the atom's pair energies and counters (zero for a converged chain), summed per chain by the
        // wrench kernel: no atomics on shared totals here
        if (lane == 0) {
            if constexpr (MIXED) reinterpret_cast<float2*>(d.epair)[a] = make_float2(Eel, Evdw);
            else reinterpret_cast<double2*>(d.epair)[a] = make_double2(Eel, Evdw);
            d.pstat[a] = make_int2((int)npairs, (int)nguard);
        }
    }
    __syncwarp();  // the warp's shared rows and queue are reused by its next atom
    }
}

// ================================================================ A6: Algorithm 1
// One warp per atom i; lane L takes the sample points k = L, L + 32, ... Step 1 counts the
// overlapping neighbours of each point up to two and keeps the critical one; step 2 re-tests
// exposed points (C = 0) against every neighbour displaced by dr e_s and critically overlapped
// points (C = 1) against their critical neighbour only. Net exchange counts per (j, s) go to
// shared memory; the force quantum G0_i / (N dr) is applied in fixed point, so
// F_j += q c_js and F_i -= q c_js are exact integer additions.
__global__ void __launch_bounds__(kSasaWarps * 32) k_sasa(const DevChain d) {
    grid_dep_sync();
    __shared__ int s_idx[kSasaWarps][kSasaStage];
    __shared__ int s_cnt[kSasaWarps][3 * kSasaStage];
    __shared__ dbl4 s_pos[kSasaWarps][kSasaStage];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int a = blockIdx.x * kSasaWarps + w;
    if (a < d.n && !d.status->done) {
        if (d.chain_done[atom_chain(d, a)]) {  // a converged chain takes no more steps
            if (lane == 0) d.sstat[a] = make_int2(0, 0);
        } else if (!d.gflag[a]) {
            if (lane == 0) { d.covered[a] = 0; d.sstat[a] = make_int2(0, 0); }
        } else {
            // a list longer than kSasaStage is k_sasa_long's: nothing to do here, nothing written
            const bool mine = d.nbr_cnt[a] <= kSasaStage;
            const int cnt = mine ? d.nbr_cnt[a] : 0;
            for (int k = lane; k < cnt; k += 32) {
                int b = d.nbr[(size_t)a * kMaxNbr + k];
                s_idx[w][k] = b;
                s_cnt[w][3 * k] = 0; s_cnt[w][3 * k + 1] = 0; s_cnt[w][3 * k + 2] = 0;
                double ro = d.aprm64[b].w;
                s_pos[w][k] = make_dbl4(d.r[3 * b], d.r[3 * b + 1], d.r[3 * b + 2], __dmul_rn(ro, ro));
            }
            __syncwarp();
            const double Roa = d.aprm64[a].w;
            const double rax = d.r[3 * a], ray = d.r[3 * a + 1], raz = d.r[3 * a + 2];
            const double dr = d.prm.delta_r;
            int ncov = 0;
            unsigned long long ntest = 0;
            for (int k = lane; k < d.N; k += 32) {
                // T_i(q_k) = r_i + Roff_i q_k (Sec. 3.4)
                const double qx = __dadd_rn(rax, __dmul_rn(Roa, d.Q64[3 * k]));
                const double qy = __dadd_rn(ray, __dmul_rn(Roa, d.Q64[3 * k + 1]));
                const double qz = __dadd_rn(raz, __dmul_rn(Roa, d.Q64[3 * k + 2]));
                auto test = [&](int j, int s) -> bool {
                    ++ntest;
                    dbl4 p = s_pos[w][j];
                    return covers64(qx, qy, qz, p.x, p.y, p.z, p.w, s, dr);
                };
                int C = 0, crit = -1;
                for (int j = 0; j < cnt; ++j) {
                    if (test(j, -1)) {
                        if (++C == 1) crit = j;
                        else break;
                    }
                }
                if (C >= 1) ++ncov;
                if (C == 0) {
                    for (int j = 0; j < cnt; ++j)
                        for (int s = 0; s < 3; ++s)
                            if (test(j, s)) atomicAdd(&s_cnt[w][3 * j + s], 1);
                } else if (C == 1) {
                    for (int s = 0; s < 3; ++s)
                        if (!test(crit, s)) atomicAdd(&s_cnt[w][3 * crit + s], -1);
                }
            }
            ncov = warp_sum(ncov);
            ntest = warp_sum(ntest);
            __syncwarp();
            const long long qa = d.qfx[a];
            long long f0 = 0, f1 = 0, f2 = 0;
            for (int j = lane; j < cnt; j += 32) {
                int b = s_idx[w][j];
                int c0 = s_cnt[w][3 * j], c1 = s_cnt[w][3 * j + 1], c2 = s_cnt[w][3 * j + 2];
                if (c0) { atomicAdd((unsigned long long*)&d.Fcav[3 * b], (unsigned long long)(qa * c0)); f0 -= qa * c0; }
                if (c1) { atomicAdd((unsigned long long*)&d.Fcav[3 * b + 1], (unsigned long long)(qa * c1)); f1 -= qa * c1; }
                if (c2) { atomicAdd((unsigned long long*)&d.Fcav[3 * b + 2], (unsigned long long)(qa * c2)); f2 -= qa * c2; }
            }
            f0 = warp_sum(f0); f1 = warp_sum(f1); f2 = warp_sum(f2);
            if (lane == 0 && mine) {
                if (f0) atomicAdd((unsigned long long*)&d.Fcav[3 * a], (unsigned long long)f0);
                if (f1) atomicAdd((unsigned long long*)&d.Fcav[3 * a + 1], (unsigned long long)f1);
                if (f2) atomicAdd((unsigned long long*)&d.Fcav[3 * a + 2], (unsigned long long)f2);
                d.covered[a] = ncov;
                d.sstat[a] = make_int2((int)ntest, 0);
            }
        }
    }
}


// Algorithm 1 for the atoms with more than kSasaStage solvation neighbours: the steps of k_sasa with
// the neighbours read from global memory and each exchange added to the partner's fixed-point sum at
// once. It runs beside k_sasa (a second stream), which skips these atoms; a warp per atom of the list
// the pair kernel recorded (none, mostly: the kernel then returns at once).
__global__ void __launch_bounds__(kSasaWarps * 32) k_sasa_long(const DevChain d) {
    grid_dep_sync();
    const int lane = threadIdx.x & 31;
    if (d.status->done) return;
    const int nlong = d.status->nlong;
    for (int e = blockIdx.x * kSasaWarps + (threadIdx.x >> 5); e < nlong; e += gridDim.x * kSasaWarps) {  // uniform
        const int a = d.long_atoms[e];
        {
            if (!d.gflag[a] || d.chain_done[atom_chain(d, a)]) continue;  // written by k_sasa
            const int cnt = min(d.nbr_cnt[a], kMaxNbr);
            const int* nl = &d.nbr[(size_t)a * kMaxNbr];
            const long long qa = d.qfx[a];
            long long f0 = 0, f1 = 0, f2 = 0;  // atom i's share of the exchanges
            auto exchange = [&](int j, int s, int delta) {
                atomicAdd((unsigned long long*)&d.Fcav[3 * nl[j] + s], (unsigned long long)(qa * delta));
                if (s == 0) f0 -= qa * delta;
                else if (s == 1) f1 -= qa * delta;
                else f2 -= qa * delta;
            };
            const double Roa = d.aprm64[a].w;
            const double rax = d.r[3 * a], ray = d.r[3 * a + 1], raz = d.r[3 * a + 2];
            const double dr = d.prm.delta_r;
            int ncov = 0;
            unsigned long long ntest = 0;
            for (int k = lane; k < d.N; k += 32) {
                // T_i(q_k) = r_i + Roff_i q_k (Sec. 3.4)
                const double qx = __dadd_rn(rax, __dmul_rn(Roa, d.Q64[3 * k]));
                const double qy = __dadd_rn(ray, __dmul_rn(Roa, d.Q64[3 * k + 1]));
                const double qz = __dadd_rn(raz, __dmul_rn(Roa, d.Q64[3 * k + 2]));
                auto test = [&](int j, int s) -> bool {
                    ++ntest;
                    const int b = nl[j];
                    const double ro = d.aprm64[b].w;
                    const dbl4 p = make_dbl4(d.r[3 * b], d.r[3 * b + 1], d.r[3 * b + 2], __dmul_rn(ro, ro));
                    return covers64(qx, qy, qz, p.x, p.y, p.z, p.w, s, dr);
                };
                int C = 0, crit = -1;
                for (int j = 0; j < cnt; ++j) {
                    if (test(j, -1)) {
                        if (++C == 1) crit = j;
                        else break;
                    }
                }
                if (C >= 1) ++ncov;
                if (C == 0) {
                    for (int j = 0; j < cnt; ++j)
                        for (int s = 0; s < 3; ++s)
                            if (test(j, s)) exchange(j, s, 1);
                } else if (C == 1) {
                    for (int s = 0; s < 3; ++s)
                        if (!test(crit, s)) exchange(crit, s, -1);
                }
            }
            ncov = warp_sum(ncov);
            ntest = warp_sum(ntest);
            __syncwarp();
            f0 = warp_sum(f0); f1 = warp_sum(f1); f2 = warp_sum(f2);
            if (lane == 0) {
                if (f0) atomicAdd((unsigned long long*)&d.Fcav[3 * a], (unsigned long long)f0);
                if (f1) atomicAdd((unsigned long long*)&d.Fcav[3 * a + 1], (unsigned long long)f1);
                if (f2) atomicAdd((unsigned long long*)&d.Fcav[3 * a + 2], (unsigned long long)f2);
                d.covered[a] = ncov;
                d.sstat[a] = make_int2((int)ntest, 0);
            }
        }
    }
}

// Mixed-precision Algorithm 1. The test of sample point k of atom i against neighbour j,
// |Roff_i Q_k - o_j|^2 <= Roff_j^2 with o_j = r_j - r_i, is for a unit Q_k the same as
// m_kj = Q_k . o_j - h_j >= 0,  h_j = (Roff_i^2 + |o_j|^2 - Roff_j^2) / (2 Roff_i),
// and with j displaced by dr e_s it is Q_k . o_j + dr Q_k,s >= h_js, h_js = h_j + (2 dr o_j,s + dr^2)
// / (2 Roff_i). A displacement can change a point's state only where the two squared distances
// straddle Roff_j^2, i.e. within |m_kj| <= (2 dr Roff_j + 3 dr^2) / (2 Roff_i) of the cap boundary.
//
// Step 1 keeps, per point, only M_k = max_j m_kj (three FFMA and one FMNMX per test). The band is
// wider than the FP32 error of m (the guard gd), so:
//  * M_k > band: some neighbour covers the point robustly. It is covered, and it takes no part in
//    step 2: with C >= 2 no single displacement uncovers it, and with C = 1 the critical neighbour
//    is the robust one, which no displacement by dr moves off the point;
//  * M_k <= -band: every neighbour misses it robustly, even displaced: exposed, no exchange;
//  * otherwise the point is re-scanned, one at a time with the neighbours spread over the lanes:
//    exact C, the critical neighbour, FP64 re-decisions of guard-band tests (covers64, as in the
//    FP64 kernel), and step 2 on the near-boundary neighbours.
// The exchanges are exactly Algorithm 1's: an exposed point gains coverage only from a near
// neighbour, and a critically overlapped point loses it only if its critical neighbour is near.
constexpr int kPtsPerLane = 8;                  // sample points each lane holds in registers
constexpr int kBatch = 32 * kPtsPerLane;         // points per batch (256)

static_assert(kSasaStage % 2 == 0, "an odd staged list has room for the pad entry of step 1");
// max(a, b, c) in one instruction (the three-input form of max.f32, sm_100 and later); exact, like fmaxf
__device__ __forceinline__ float fmax3f(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

template <int W>
__global__ void __launch_bounds__(W * 32) k_sasa_mixed(const DevChain d) {
    grid_dep_sync();
    __shared__ float4 s_o[W][kSasaStage];   // o_j, h_j
    __shared__ int s_idx[W][kSasaStage];
    __shared__ int s_cnt[W][3 * kSasaStage];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int a = blockIdx.x * W + w;
    if (a < d.n && !d.status->done) {
        const int ca = atom_chain(d, a);
        const int cnt0 = d.nbr_cnt[a];  // loaded beside the flags below (independent of them)
        const float Ra = d.aprm32[a].w;
        const bool gam = d.gflag[a] != 0;
        const float gsf = d.grid[ca].sf;
        if (d.chain_done[ca]) {  // a converged chain takes no more steps
            if (lane == 0) d.sstat[a] = make_int2(0, 0);
        } else if (!gam) {
            if (lane == 0) { d.covered[a] = 0; d.sstat[a] = make_int2(0, 0); }
        } else {
            // a list longer than kSasaStage is k_sasa_mixed_long's: nothing to do here, nothing written
            const bool mine = cnt0 <= kSasaStage;
            const int cnt = min(mine ? cnt0 : 0, kSasaStage);
            const float inv2R = 0.5f / Ra;
            const float drf = d.f_dr;
            const float gd = 1e-4f + 1.2e-5f * gsf;  // guard band in Q.o units (A)
            float rmax2 = 0.0f;
            for (int j = lane; j < cnt; j += 32) {
                const float4 o = d.nbr_off[(size_t)a * kMaxNbr + j];  // r_j - r_i, Roff_j^2
                const float oo = o.x * o.x + o.y * o.y + o.z * o.z;
                s_o[w][j] = make_float4(o.x, o.y, o.z, (Ra * Ra + oo - o.w) * inv2R);
                s_idx[w][j] = d.nbr[(size_t)a * kMaxNbr + j];
                s_cnt[w][3 * j] = 0; s_cnt[w][3 * j + 1] = 0; s_cnt[w][3 * j + 2] = 0;
                rmax2 = fmaxf(rmax2, o.w);
            }
            for (int q = 16; q > 0; q >>= 1) rmax2 = fmaxf(rmax2, __shfl_xor_sync(0xffffffffu, rmax2, q));
            // band of m around 0 where a displacement by dr can change a point's state, widened to the
            // largest neighbour radius so that it is one number per atom
            const float band = (2.0f * drf * sqrtf(rmax2) + 3.0f * drf * drf) * inv2R + gd;
            // an odd list is padded with a neighbour no point touches (m = -inf) for the paired step 1
            if (lane == 0 && (cnt & 1)) s_o[w][cnt] = make_float4(0.0f, 0.0f, 0.0f, INFINITY);
            __syncwarp();
            int ncov = 0, nguard = 0;
            unsigned long long ntest = 0;
            auto recheck = [&](int j, int k, int s) -> bool {  // FP64, identical to the FP64 kernel
                ++nguard;
                const double Roa = d.aprm64[a].w, dr = d.prm.delta_r;
                const double rax = centre64(d, a, 0), ray = centre64(d, a, 1), raz = centre64(d, a, 2);
                const int b = s_idx[w][j];
                const double ro = d.aprm64[b].w;
                const double qx = __dadd_rn(rax, __dmul_rn(Roa, d.Q64[3 * k]));
                const double qy = __dadd_rn(ray, __dmul_rn(Roa, d.Q64[3 * k + 1]));
                const double qz = __dadd_rn(raz, __dmul_rn(Roa, d.Q64[3 * k + 2]));
                return covers64(qx, qy, qz, centre64(d, b, 0), centre64(d, b, 1), centre64(d, b, 2), __dmul_rn(ro, ro),
                                s, dr);
            };
            bool exch = false;  // this lane added an exchange count
            for (int kb = 0; kb < d.N; kb += kBatch) {
                float qx[kPtsPerLane], qy[kPtsPerLane], qz[kPtsPerLane], mx[kPtsPerLane];
                unsigned valid = 0;
                if (kb + kBatch <= d.N) {  // a whole batch (N a multiple of 256, the default among them)
                    valid = (1u << kPtsPerLane) - 1u;
                    const float4* Qb = d.Q4 + kb + lane;
#pragma unroll
                    for (int p = 0; p < kPtsPerLane; ++p) {
                        const float4 qk = Qb[32 * p];
                        qx[p] = qk.x;
                        qy[p] = qk.y;
                        qz[p] = qk.z;
                        mx[p] = -INFINITY;
                    }
                } else {
#pragma unroll
                    for (int p = 0; p < kPtsPerLane; ++p) {
                        const int k = kb + lane + 32 * p;
                        const bool v = k < d.N;
                        const float4 qk = v ? d.Q4[k] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                        qx[p] = qk.x;
                        qy[p] = qk.y;
                        qz[p] = qk.z;
                        valid |= v ? (1u << p) : 0u;
                        mx[p] = -INFINITY;  // a missing point stays at -inf: neither covered nor near
                    }
                }
                // step 1: the largest m of each point over all neighbours
#pragma unroll 2
                for (int j = 0; j < cnt; j += 2) {  // two neighbours per round, one max over both
                    const float4 o = s_o[w][j], o2 = s_o[w][j + 1];
#pragma unroll
                    for (int p = 0; p < kPtsPerLane; ++p) {
                        const float m = fmaf(qz[p], o.z, fmaf(qy[p], o.y, fmaf(qx[p], o.x, -o.w)));
                        const float m2 = fmaf(qz[p], o2.z, fmaf(qy[p], o2.y, fmaf(qx[p], o2.x, -o2.w)));
                        mx[p] = fmax3f(mx[p], m, m2);
                    }
                }
                ntest += (unsigned long long)__popc(valid) * cnt;
                // decided points are counted; the rest (bits p of each lane) are re-scanned
                unsigned cov = 0, res = 0;
#pragma unroll
                for (int p = 0; p < kPtsPerLane; ++p) {
                    cov |= mx[p] > band ? (1u << p) : 0u;
                    res |= (mx[p] > -band && mx[p] <= band) ? (1u << p) : 0u;
                }
                ncov += __popc(cov);
                // re-scan, one point at a time (lane by lane, then by p); lane t takes neighbours t, t + 32,
                // ... (at most 4)
                for (unsigned rl = __ballot_sync(0xffffffffu, res != 0u); rl; rl &= rl - 1u)
                for (unsigned pb = __shfl_sync(0xffffffffu, res, __ffs(rl) - 1); pb; pb &= pb - 1u) {
                    const int k = kb + (__ffs(rl) - 1) + 32 * (__ffs(pb) - 1);
                    const float4 qk = d.Q4[k];
                    const float Qx = qk.x, Qy = qk.y, Qz = qk.z;
                    unsigned inb = 0, nrb = 0;
                    for (int r = 0; 32 * r < cnt; ++r) {
                        const int j = 32 * r + lane;
                        if (j < cnt) {
                            const float4 o = s_o[w][j];
                            const float m = fmaf(Qz, o.z, fmaf(Qy, o.y, fmaf(Qx, o.x, -o.w)));
                            bool in = m > 0.0f;
                            if (fabsf(m) <= gd) in = recheck(j, k, -1);
                            inb |= in ? (1u << r) : 0u;
                            nrb |= fabsf(m) <= band ? (1u << r) : 0u;
                        }
                    }
                    const int C = (int)__reduce_add_sync(0xffffffffu, (unsigned)__popc(inb));
                    if (lane == 0) ncov += C >= 1;
                    // step 2 against neighbour j displaced along each axis s: m_s = m + dr Q_s - (2 dr o_s +
                    // dr^2) / (2 R_i), the test at rest with j moved by dr e_s (FP64 inside the guard band)
                    auto covers3 = [&](int j, bool want, int delta) {
                        const float4 o = s_o[w][j];
                        const float m = fmaf(Qz, o.z, fmaf(Qy, o.y, fmaf(Qx, o.x, -o.w)));
#pragma unroll
                        for (int s = 0; s < 3; ++s) {
                            const float os = s == 0 ? o.x : (s == 1 ? o.y : o.z);
                            const float Qs = s == 0 ? Qx : (s == 1 ? Qy : Qz);
                            const float ms = fmaf(drf, Qs, m) - (2.0f * drf * os + drf * drf) * inv2R;
                            ++ntest;
                            const bool cv = fabsf(ms) > gd ? ms >= 0.0f : recheck(j, k, s);
                            if (cv == want) {
                                atomicAdd(&s_cnt[w][3 * j + s], delta);
                                exch = true;
                            }
                        }
                    };
                    if (C == 0) {  // exposed: every near neighbour may cover it once displaced
                        for (unsigned b = nrb; b; b &= b - 1) covers3(32 * (__ffs(b) - 1) + lane, true, 1);
                    } else if (C == 1 && (inb & nrb)) {  // critically overlapped by a near neighbour
                        covers3(32 * (__ffs(inb) - 1) + lane, false, -1);
                    }
                }
                __syncwarp();
            }
            // counts of the warp by 32-bit reductions (each below 2^31: at most 4096 points x kMaxNbr
            // neighbours x 3 axes); atom i's force is minus the quantum times its net exchanges
            ncov = (int)__reduce_add_sync(0xffffffffu, (unsigned)ncov);
            nguard = (int)__reduce_add_sync(0xffffffffu, (unsigned)nguard);
            const unsigned nt = __reduce_add_sync(0xffffffffu, (unsigned)ntest);
            __syncwarp();
            const long long qa = d.qfx[a];
            int s0 = 0, s1 = 0, s2 = 0;
            const bool any_exch = __any_sync(0xffffffffu, exch);  // most atoms have none
            for (int j = lane; any_exch && j < cnt; j += 32) {
                const int b = s_idx[w][j];
                const int c0 = s_cnt[w][3 * j], c1 = s_cnt[w][3 * j + 1], c2 = s_cnt[w][3 * j + 2];
                if (c0) atomicAdd((unsigned long long*)&d.Fcav[3 * b], (unsigned long long)(qa * c0));
                if (c1) atomicAdd((unsigned long long*)&d.Fcav[3 * b + 1], (unsigned long long)(qa * c1));
                if (c2) atomicAdd((unsigned long long*)&d.Fcav[3 * b + 2], (unsigned long long)(qa * c2));
                s0 += c0; s1 += c1; s2 += c2;
            }
            s0 = __reduce_add_sync(0xffffffffu, s0);
            s1 = __reduce_add_sync(0xffffffffu, s1);
            s2 = __reduce_add_sync(0xffffffffu, s2);
            if (lane == 0 && mine) {
                if (s0) atomicAdd((unsigned long long*)&d.Fcav[3 * a], (unsigned long long)(-qa * s0));
                if (s1) atomicAdd((unsigned long long*)&d.Fcav[3 * a + 1], (unsigned long long)(-qa * s1));
                if (s2) atomicAdd((unsigned long long*)&d.Fcav[3 * a + 2], (unsigned long long)(-qa * s2));
                d.covered[a] = ncov;
                d.sstat[a] = make_int2((int)nt, nguard);  // summed by the wrench kernel
            }
        }
    }
}

// Algorithm 1 in mixed precision for the atoms with more than kSasaStage solvation neighbours (compact
// regions): the steps of k_sasa_mixed, with the list read from global memory (rewritten in place as
// (o_j, h_j)) and each exchange added to the partner's fixed-point sum at once. It runs beside
// k_sasa_mixed (a second stream), which skips these atoms; a warp per atom of the list the pair
// kernel recorded (none, mostly: the kernel then returns at once).
__global__ void __launch_bounds__(kSasaWarps * 32) k_sasa_mixed_long(const DevChain d) {
    grid_dep_sync();
    __shared__ unsigned short s_near[kSasaWarps][kBatch];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (d.status->done) return;
    const int nlong = d.status->nlong;
    for (int e = blockIdx.x * kSasaWarps + w; e < nlong; e += gridDim.x * kSasaWarps) {  // uniform in the warp
        const int a = d.long_atoms[e];
        {
            if (!d.gflag[a] || d.chain_done[atom_chain(d, a)]) continue;  // written by k_sasa_mixed
            const int cnt = min(d.nbr_cnt[a], kMaxNbr);
            float4* ol = &d.nbr_off[(size_t)a * kMaxNbr];  // rewritten in place as (o_j, h_j)
            const int* nl = &d.nbr[(size_t)a * kMaxNbr];
            const float Ra = d.aprm32[a].w;
            const float inv2R = 0.5f / Ra;
            const float drf = d.f_dr;
            const float gd = 1e-4f + 1.2e-5f * d.grid[atom_chain(d, a)].sf;  // guard band in Q.o units (A)
            float rmax2 = 0.0f;
            for (int j = lane; j < cnt; j += 32) {
                const float4 o = ol[j];  // r_j - r_i, Roff_j^2
                const float oo = o.x * o.x + o.y * o.y + o.z * o.z;
                ol[j] = make_float4(o.x, o.y, o.z, (Ra * Ra + oo - o.w) * inv2R);
                rmax2 = fmaxf(rmax2, o.w);
            }
            for (int q = 16; q > 0; q >>= 1) rmax2 = fmaxf(rmax2, __shfl_xor_sync(0xffffffffu, rmax2, q));
            // band of m around 0 where a displacement by dr can change a point's state, widened to the
            // largest neighbour radius so that it is one number per atom
            const float band = (2.0f * drf * sqrtf(rmax2) + 3.0f * drf * drf) * inv2R + gd;
            __syncwarp();
            const long long qa = d.qfx[a];
            int ncov = 0, nguard = 0, s0 = 0, s1 = 0, s2 = 0;
            unsigned long long ntest = 0;
            // an exchange goes to the partner's fixed-point sum at once; atom i keeps the net count
            auto exchange = [&](int j, int s, int delta) {
                atomicAdd((unsigned long long*)&d.Fcav[3 * nl[j] + s], (unsigned long long)(qa * delta));
                if (s == 0) s0 += delta;
                else if (s == 1) s1 += delta;
                else s2 += delta;
            };
            auto recheck = [&](int j, int k, int s) -> bool {  // FP64, identical to the FP64 kernel
                ++nguard;
                const double Roa = d.aprm64[a].w, dr = d.prm.delta_r;
                const double rax = centre64(d, a, 0), ray = centre64(d, a, 1), raz = centre64(d, a, 2);
                const int b = nl[j];
                const double ro = d.aprm64[b].w;
                const double qx = __dadd_rn(rax, __dmul_rn(Roa, d.Q64[3 * k]));
                const double qy = __dadd_rn(ray, __dmul_rn(Roa, d.Q64[3 * k + 1]));
                const double qz = __dadd_rn(raz, __dmul_rn(Roa, d.Q64[3 * k + 2]));
                return covers64(qx, qy, qz, centre64(d, b, 0), centre64(d, b, 1), centre64(d, b, 2), __dmul_rn(ro, ro),
                                s, dr);
            };
            for (int kb = 0; kb < d.N; kb += kBatch) {
                float qx[kPtsPerLane], qy[kPtsPerLane], qz[kPtsPerLane], mx[kPtsPerLane];
                unsigned valid = 0;
#pragma unroll
                for (int p = 0; p < kPtsPerLane; ++p) {
                    const int k = kb + lane + 32 * p;
                    const bool v = k < d.N;
                    const float4 qk = v ? d.Q4[k] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    qx[p] = qk.x;
                    qy[p] = qk.y;
                    qz[p] = qk.z;
                    valid |= v ? (1u << p) : 0u;
                    mx[p] = -INFINITY;
                }
                // step 1: the largest m of each point over all neighbours
#pragma unroll 2
                for (int j = 0; j < cnt; ++j) {
                    const float4 o = ol[j];
#pragma unroll
                    for (int p = 0; p < kPtsPerLane; ++p) {
                        const float m = fmaf(qz[p], o.z, fmaf(qy[p], o.y, fmaf(qx[p], o.x, -o.w)));
                        mx[p] = fmaxf(mx[p], m);
                    }
                }
                ntest += (unsigned long long)__popc(valid) * cnt;
                // decided points are counted; the rest are listed for the re-scan
                int nres = 0;
                const unsigned lt = (1u << lane) - 1u;
#pragma unroll
                for (int p = 0; p < kPtsPerLane; ++p) {
                    const bool v = (valid >> p) & 1u;
                    const bool res = v && mx[p] > -band && mx[p] <= band;
                    if (v && mx[p] > band) ++ncov;
                    const unsigned bm = __ballot_sync(0xffffffffu, res);
                    if (res) s_near[w][nres + __popc(bm & lt)] = (unsigned short)(lane + 32 * p);
                    nres += __popc(bm);
                }
                __syncwarp();
                // re-scan, one point at a time; lane t takes neighbours t, t + 32, ... (at most kMaxNbr / 32 = 12)
                for (int e = 0; e < nres; ++e) {
                    const int k = kb + s_near[w][e];
                    const float4 qk = d.Q4[k];
                    const float Qx = qk.x, Qy = qk.y, Qz = qk.z;
                    unsigned inb = 0, nrb = 0;
                    for (int r = 0; 32 * r < cnt; ++r) {
                        const int j = 32 * r + lane;
                        if (j < cnt) {
                            const float4 o = ol[j];
                            const float m = fmaf(Qz, o.z, fmaf(Qy, o.y, fmaf(Qx, o.x, -o.w)));
                            bool in = m > 0.0f;
                            if (fabsf(m) <= gd) in = recheck(j, k, -1);
                            inb |= in ? (1u << r) : 0u;
                            nrb |= fabsf(m) <= band ? (1u << r) : 0u;
                        }
                    }
                    const int C = (int)__reduce_add_sync(0xffffffffu, (unsigned)__popc(inb));
                    if (lane == 0) ncov += C >= 1;
                    // step 2 against neighbour j displaced along s; hs is h_js
                    auto covers_s = [&](int j, int s) -> bool {
                        const float4 o = ol[j];
                        const float os = s == 0 ? o.x : (s == 1 ? o.y : o.z);
                        const float Qs = s == 0 ? Qx : (s == 1 ? Qy : Qz);
                        const float hs = o.w + (2.0f * drf * os + drf * drf) * inv2R;
                        const float m = fmaf(Qz, o.z, fmaf(Qy, o.y, fmaf(Qx, o.x, fmaf(drf, Qs, -hs))));
                        ++ntest;
                        if (fabsf(m) > gd) return m >= 0.0f;
                        return recheck(j, k, s);
                    };
                    if (C == 0) {  // exposed: every near neighbour may cover it once displaced
                        for (unsigned b = nrb; b; b &= b - 1) {
                            const int j = 32 * (__ffs(b) - 1) + lane;
                            for (int s = 0; s < 3; ++s)
                                if (covers_s(j, s)) exchange(j, s, 1);
                        }
                    } else if (C == 1 && (inb & nrb)) {  // critically overlapped by a near neighbour
                        const int j = 32 * (__ffs(inb) - 1) + lane;
                        for (int s = 0; s < 3; ++s)
                            if (!covers_s(j, s)) exchange(j, s, -1);
                    }
                }
                __syncwarp();
            }
            // counts of the warp by 32-bit reductions (each below 2^31: at most 4096 points x kMaxNbr
            // neighbours x 3 axes); atom i's force is minus the quantum times its net exchanges
            ncov = (int)__reduce_add_sync(0xffffffffu, (unsigned)ncov);
            nguard = (int)__reduce_add_sync(0xffffffffu, (unsigned)nguard);
            const unsigned nt = __reduce_add_sync(0xffffffffu, (unsigned)ntest);
            __syncwarp();
            s0 = __reduce_add_sync(0xffffffffu, s0);
            s1 = __reduce_add_sync(0xffffffffu, s1);
            s2 = __reduce_add_sync(0xffffffffu, s2);
            if (lane == 0) {
                if (s0) atomicAdd((unsigned long long*)&d.Fcav[3 * a], (unsigned long long)(-qa * s0));
                if (s1) atomicAdd((unsigned long long*)&d.Fcav[3 * a + 1], (unsigned long long)(-qa * s1));
                if (s2) atomicAdd((unsigned long long*)&d.Fcav[3 * a + 2], (unsigned long long)(-qa * s2));
                d.covered[a] = ncov;
                d.sstat[a] = make_int2((int)nt, nguard);  // summed by the wrench kernel
            }
        }
    }
}

// ================================================================ pairwise solvation surrogate
// The smooth pairwise area approximation of Sec. 3.4 (solvation = 2): A_i = S_i prod_j f_ij with
// f_ij = 1 - b_ij / S_i, b_ij = pi Roff_i (Roff_i + Roff_j - d) (1 + (Roff_j - Roff_i) / d) (the area of
// sphere i inside sphere j, clamped to [0, S_i]), S_i = 4 pi Roff_i^2, E_i = gamma_i A_i. One warp per
// atom with gamma != 0, lanes over its solvation neighbours: pass 1 forms the product, pass 2 the pair
// forces c_ij e_ij (c_ij = E_i pi Roff_i (1 + (Roff_j^2 - Roff_i^2) / d^2) / (S_i f_ij), e_ij the unit
// vector from i to j), added to F_i and subtracted from F_j in the int64 fixed point of the solvation
// sums (2^-40), so they cancel exactly. A clamped factor (f_ij = 0: i inside j) zeroes E_i and its
// forces; j inside i buries nothing. Mixed mode: FP32 on the list offsets, the overlap decision
// d < Roff_i + Roff_j re-decided in FP64 inside the guard band (the force jumps there).
template <bool MIXED, int W>
__global__ void __launch_bounds__(W * 32) k_sasa_pw(const DevChain d) {
    grid_dep_sync();
    typedef typename std::conditional<MIXED, float, double>::type R;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int a = blockIdx.x * W + w;
    if (a >= d.n || d.status->done) return;
    if (d.chain_done[atom_chain(d, a)] || !d.gflag[a]) {
        if (lane == 0) { d.esolv[a] = 0.0; d.covered[a] = 0; d.sstat[a] = make_int2(0, 0); }
        return;
    }
    const int cnt = min(d.nbr_cnt[a], kMaxNbr);
    const int* nl = &d.nbr[(size_t)a * kMaxNbr];
    const float4* ol = &d.nbr_off[(size_t)a * kMaxNbr];
    const R Ri = MIXED ? (R)d.aprm32[a].w : (R)d.aprm64[a].w;
    const R Si = (R)(4.0 * 3.14159265358979323846) * Ri * Ri;
    const R kPi = (R)3.14159265358979323846;
    const float gp = d.grid[atom_chain(d, a)].gpf;
    int nguard = 0;
    // neighbour j: offset r_j - r_i, Roff_j, and whether the spheres overlap (d < Roff_i + Roff_j)
    auto geom = [&](int j, R& ox, R& oy, R& oz, R& d2, R& Rj) -> bool {
        const int b = nl[j];
        if constexpr (MIXED) {
            const float4 o = ol[j];
            ox = o.x; oy = o.y; oz = o.z;
            Rj = sqrtf(o.w);
            d2 = ox * ox + oy * oy + oz * oz;
            const float s = Ri + Rj;
            if (fabsf(d2 - s * s) > gp) return d2 < s * s;
            ++nguard;  // guard band: the FP64 decision of the FP64 path
        } else {
            ox = d.r[3 * b] - d.r[3 * a]; oy = d.r[3 * b + 1] - d.r[3 * a + 1]; oz = d.r[3 * b + 2] - d.r[3 * a + 2];
            Rj = d.aprm64[b].w;
            d2 = ox * ox + oy * oy + oz * oz;
            return d2 < (Ri + Rj) * (Ri + Rj);
        }
        const double ex = centre64(d, b, 0) - centre64(d, a, 0), ey = centre64(d, b, 1) - centre64(d, a, 1),
                     ez = centre64(d, b, 2) - centre64(d, a, 2);
        const double s64 = d.aprm64[a].w + d.aprm64[b].w;
        return ex * ex + ey * ey + ez * ez < s64 * s64;
    };
    // a force term in the solvation sums' fixed point, round(q 2^40): in mixed mode from FP32 pieces
    // of q 2^17 (exact scaling; see fx_add), FP64 only for terms of 32 kcal/mol/A or more
    auto fx40 = [&](R q) -> long long {
        if constexpr (MIXED) {
            const float v = q * 131072.0f;
            if (fabsf(v) < kPairFxMax) {
                int n, fr;
                fx_pieces(v, n, fr);
                return fx_units(n, fr);
            }
            return llrint((double)q * kFxScale);
        } else {
            return llrint(q * kFxScale);
        }
    };
    // pass 1: A_i / S_i = prod f_ij
    R prod = (R)1;
    bool clamped = false;
    for (int j = lane; j < cnt; j += 32) {
        R ox, oy, oz, d2, Rj;
        if (!geom(j, ox, oy, oz, d2, Rj)) continue;
        const R dd = sqrt(d2);
        const R b = fmax(kPi * Ri * (Ri + Rj - dd) * ((R)1 + (Rj - Ri) / dd), (R)0);
        const R f = (R)1 - b / Si;
        if (f <= (R)0) clamped = true;
        prod *= fmax(f, (R)0);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) prod *= __shfl_xor_sync(0xffffffffu, prod, o);
    clamped = __any_sync(0xffffffffu, clamped);
    const R Ei = (R)d.G0[a] * prod;  // G0_i = gamma_i S_i
    long long fi[3] = {0, 0, 0};
    if (!clamped && Ei != (R)0) {
        // pass 2: pair forces
        for (int j = lane; j < cnt; j += 32) {
            R ox, oy, oz, d2, Rj;
            if (!geom(j, ox, oy, oz, d2, Rj)) continue;
            const R dd = sqrt(d2);
            const R b = kPi * Ri * (Ri + Rj - dd) * ((R)1 + (Rj - Ri) / dd);
            if (b <= (R)0) continue;  // j inside i: no burial
            const R f = (R)1 - b / Si;
            const R mdb = kPi * Ri * ((R)1 + (Rj * Rj - Ri * Ri) / d2);
            const R cij = Ei * mdb / (Si * f) / dd;  // times r_j - r_i
            const long long qx = fx40(cij * ox), qy = fx40(cij * oy), qz = fx40(cij * oz);
            fi[0] += qx; fi[1] += qy; fi[2] += qz;
            unsigned long long* Fj = reinterpret_cast<unsigned long long*>(&d.Fcav[3 * nl[j]]);
            atomicAdd(Fj, (unsigned long long)(-qx));
            atomicAdd(Fj + 1, (unsigned long long)(-qy));
            atomicAdd(Fj + 2, (unsigned long long)(-qz));
        }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) fi[k] = warp_sum(fi[k]);
    nguard = (int)__reduce_add_sync(0xffffffffu, (unsigned)nguard);
    if (lane == 0) {
        unsigned long long* Fa = reinterpret_cast<unsigned long long*>(&d.Fcav[3 * a]);
        if (fi[0]) atomicAdd(Fa, (unsigned long long)fi[0]);
        if (fi[1]) atomicAdd(Fa + 1, (unsigned long long)fi[1]);
        if (fi[2]) atomicAdd(Fa + 2, (unsigned long long)fi[2]);
        d.esolv[a] = (double)Ei;
        d.covered[a] = 0;
        d.sstat[a] = make_int2(cnt, nguard);
    }
}

// loop state of a batch; with full, also the statistics and the chains' bounding boxes
__global__ void k_reset_loop(const DevChain d, int full) {
    grid_dep_sync();
    reset_loop_state(d, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x, full != 0);
}

__global__ void k_force_out(const DevChain d) {
    grid_dep_sync();
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= 3 * d.n) return;
    double fc = d.prm.solvation ? (double)d.Fcav[x] * kFxInv : 0.0;
    d.Fcav64[x] = fc;
    if (d.prm.precision == KCM_MIXED) d.Fpair[x] = (double)d.Fpx[x] * kPairFxInv + (double)d.Fox[x] * 0.5 + (double)d.Fov[x];
    d.Ftot[x] = d.Fpair[x] + fc;
}

inline int blocks(long long n, int tpb) { return (int)((n + tpb - 1) / tpb); }

}  // namespace

void launch_init_status(DevChain& d, cudaStream_t s) { launch_k(k_reset_loop, blocks(d.nchains, 256), 256, 0, s, d.pdl, d, 1); }
void launch_reset_loop(DevChain& d, cudaStream_t s) { launch_k(k_reset_loop, blocks(d.nchains, 256), 256, 0, s, d.pdl, d, 0); }

void launch_binning(DevChain& d, cudaStream_t s) {
    if (d.bin_c) {  // a single chain in mixed mode: one cluster
        launch_bin_cluster(d, s);
        return;
    }
    if (d.atom_off) {  // a batch in mixed mode: cells and starts by one block per chain, then the placement
        launch_k(k_bin_chains, d.nchains, kBinChainThreads, 0, s, d.pdl, d);
        launch_k(k_bin_place<true>, blocks(d.n, 256), 256, 0, s, d.pdl, d);
        return;
    }
    launch_k(k_bin_count, blocks(d.n, kBinThreads), kBinThreads, 0, s, d.pdl, d);
    if (!d.scan_fused) {
        launch_k(k_scan_sums, d.scan_blocks, kScanThreadsBig, 0, s, d.pdl, d);
        launch_k(k_scan_cells, d.scan_blocks, kScanThreadsBig, 0, s, d.pdl, d);
    }
    if (d.prm.precision == KCM_MIXED) {
        launch_k(k_bin_place<true>, blocks(d.n, 256), 256, 0, s, d.pdl, d);
    } else {
        launch_k(k_bin_place<false>, blocks(d.n, 256), 256, 0, s, d.pdl, d);
        launch_k(k_bin_stable, blocks(d.n, 256), 256, 0, s, d.pdl, d);
    }
}

template <int W>
void launch_pairs_w(DevChain& d, cudaStream_t s) {
    const bool mixed = d.prm.precision == KCM_MIXED;
    int nb = (d.n + W - 1) / W;
    if (d.pair_grid_cap > 0) nb = std::min(nb, d.pair_grid_cap);  // persistent grid
    if (d.stencil == 2) {
        if (mixed) launch_k(k_pair<true, 2, W>, nb, W * 32, 0, s, d.pdl, d);
        else launch_k(k_pair<false, 2, W>, nb, W * 32, 0, s, d.pdl, d);
    } else {
        if (mixed) launch_k(k_pair<true, 1, W>, nb, W * 32, 0, s, d.pdl, d);
        else launch_k(k_pair<false, 1, W>, nb, W * 32, 0, s, d.pdl, d);
    }
}

template <int W>
int pair_resident_w(const DevChain& d) {
    int b = 0;
    const bool mixed = d.prm.precision == KCM_MIXED;
    cudaError_t e;
    if (d.stencil == 2) {
        e = mixed ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_pair<true, 2, W>, W * 32, 0)
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_pair<false, 2, W>, W * 32, 0);
    } else {
        e = mixed ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_pair<true, 1, W>, W * 32, 0)
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_pair<false, 1, W>, W * 32, 0);
    }
    return e == cudaSuccess ? b : -1;
}

int pair_resident_blocks(const DevChain& d) {
    switch (d.pair_warps) {
        case 1: return pair_resident_w<1>(d);
        case 2: return pair_resident_w<2>(d);
        default: return pair_resident_w<4>(d);
    }
}

// the pair kernel: in mixed mode the cell-pair tile kernel when chosen, else the warp-per-atom kernel
// with pair_warps home atoms per block (a tile shape of kTileWarps)
void launch_pairs(DevChain& d, cudaStream_t s) {
    if (d.pair_tile && d.prm.precision == KCM_MIXED) {
        launch_pairs_tile(d, s);
        return;
    }
    switch (d.pair_warps) {
        case 1: launch_pairs_w<1>(d, s); break;
        case 2: launch_pairs_w<2>(d, s); break;
        default: launch_pairs_w<4>(d, s); break;
    }
}

void launch_sasa(DevChain& d, cudaStream_t s) {
    const int nb4 = (d.n + kSasaWarps - 1) / kSasaWarps;
    if (d.prm.solvation == 2) {  // sasa_warps atoms per block here too
        const int W = d.sasa_warps;
        const int nb = (d.n + W - 1) / W;
        if (d.prm.precision == KCM_MIXED) {
            if (W == 1) launch_k(k_sasa_pw<true, 1>, nb, 32, 0, s, d.pdl, d);
            else if (W == 2) launch_k(k_sasa_pw<true, 2>, nb, 64, 0, s, d.pdl, d);
            else launch_k(k_sasa_pw<true, 4>, nb, 128, 0, s, d.pdl, d);
        } else {
            if (W == 1) launch_k(k_sasa_pw<false, 1>, nb, 32, 0, s, d.pdl, d);
            else if (W == 2) launch_k(k_sasa_pw<false, 2>, nb, 64, 0, s, d.pdl, d);
            else launch_k(k_sasa_pw<false, 4>, nb, 128, 0, s, d.pdl, d);
        }
    } else if (d.prm.solvation) {
        if (d.prm.precision == KCM_MIXED) {  // sasa_warps atoms per block (a tile shape of kTileWarps)
            const int W = d.sasa_warps;
            const int nb = (d.n + W - 1) / W;
            if (W == 1) launch_k(k_sasa_mixed<1>, nb, 32, 0, s, d.pdl, d);
            else if (W == 2) launch_k(k_sasa_mixed<2>, nb, 64, 0, s, d.pdl, d);
            else launch_k(k_sasa_mixed<4>, nb, 128, 0, s, d.pdl, d);
        } else {
            launch_k(k_sasa, nb4, kSasaWarps * 32, 0, s, d.pdl, d);
        }
    }
}

void launch_sasa_long(DevChain& d, cudaStream_t s) {
    if (d.prm.solvation != 1) return;
    const int nb = std::max(1, std::min((d.n + kSasaWarps - 1) / kSasaWarps, kSasaLongBlocks));
    if (d.prm.precision == KCM_MIXED) launch_k(k_sasa_mixed_long, nb, kSasaWarps * 32, 0, s, d.pdl, d);
    else launch_k(k_sasa_long, nb, kSasaWarps * 32, 0, s, d.pdl, d);
}

void launch_force_out(DevChain& d, cudaStream_t s) { launch_k(k_force_out, blocks(3LL * d.n, 256), 256, 0, s, d.pdl, d); }

}  // namespace kcm
