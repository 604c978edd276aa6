// CUDA kernels of one KCM iteration for sm_103a (B300).
//
// Stages (Sec. 4.1 steps 4-8):
//   A1 forward kinematics: prefix product of per-joint affine transforms (FP64), Sec. 2.1 and
//      App. B; atom centres r = M_link(r^0)
//   A2 binning: bounding box, uniform grid (Sec. 3.2), counting sort by cell with warp-aggregated
//      atomics, cells ordered by atom index for determinism
//   A3-A5 pair forces over the 27-cell neighbourhood (eq. 02_2, 03_2, 03_8, 03_9) and the
//      solvation neighbour lists A'_i (Sec. 3.2 "neighbourhood matrix")
//   A6 surface enumeration, Algorithm 1 (Sec. 3.4), one warp per atom
//   A7-A8 link wrenches (eq. KCM_01/02) and the suffix sum of Sec. 3.5, tau_k = J_k^T P^agg_k
//   A9 clamped step (eq. KCM_07), A10 energies (eq. 01, G_cav_patch)
//
// B300 has about one FP64 FMA per 64 FP32 FMAs, so every FP64 stage is cut into many small blocks
// (a few threads each) that the scheduler spreads over all SMs; FP32 work uses full warps.
// Every reduction has a fixed order or is integer, so an iteration is bitwise reproducible.
#include <cuda_runtime.h>

#include <cstdio>
#include <type_traits>

#include "kcm_device.h"

namespace kcm {

namespace {

// ---------------------------------------------------------------- small helpers
__device__ __forceinline__ unsigned long long dkey(double x) {
    unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
    return (b & 0x8000000000000000ULL) ? ~b : (b | 0x8000000000000000ULL);
}
__device__ __forceinline__ double dkey_inv(unsigned long long k) {
    unsigned long long b = (k & 0x8000000000000000ULL) ? (k & 0x7FFFFFFFFFFFFFFFULL) : ~k;
    return __longlong_as_double(static_cast<long long>(b));
}

// affine transform: rows of the rotation a[0..8], translation a[9..11]; C = A o B
__device__ __forceinline__ void aff_compose(const double* A, const double* B, double* C) {
    double T[12];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int j = 0; j < 3; ++j) T[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
        T[9 + i] = A[3 * i] * B[9] + A[3 * i + 1] * B[10] + A[3 * i + 2] * B[11] + A[9 + i];
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) C[k] = T[k];
}
__device__ __forceinline__ void aff_identity(double* A) {
#pragma unroll
    for (int k = 0; k < 12; ++k) A[k] = (k == 0 || k == 4 || k == 8) ? 1.0 : 0.0;
}
__device__ __forceinline__ void aff_load(const double* src, double* A) {
#pragma unroll
    for (int k = 0; k < 12; ++k) A[k] = src[k];
}
__device__ __forceinline__ void aff_store(double* dst, const double* A) {
#pragma unroll
    for (int k = 0; k < 12; ++k) dst[k] = A[k];
}

// Local joint transform between consecutive link frames: L_j = Tr(step_j) o Rot(u_j, th), i.e.
// x -> R x + step_j with R = cos I + sin [u]x + (1 - cos) u u^T (right-hand rule). With link frame
// poses T_j = L_1 o ... o L_j the ZP-frame product of rotations about the joint axes (eq. kin_04)
// is T_j o Tr(-p0_j), and atom centres are T_link(r^0 - p0_link) (eq. r1/r2).
__device__ __forceinline__ void joint_tf(const double* u, const double* step, double th, double* G) {
    double s, c;
    sincos(th, &s, &c);
    double C = 1.0 - c;
    G[0] = c + u[0] * u[0] * C;        G[1] = u[0] * u[1] * C - u[2] * s; G[2] = u[0] * u[2] * C + u[1] * s;
    G[3] = u[1] * u[0] * C + u[2] * s; G[4] = c + u[1] * u[1] * C;        G[5] = u[1] * u[2] * C - u[0] * s;
    G[6] = u[2] * u[0] * C - u[1] * s; G[7] = u[2] * u[1] * C + u[0] * s; G[8] = c + u[2] * u[2] * C;
    G[9] = step[0];
    G[10] = step[1];
    G[11] = step[2];
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ int warp_max(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// The FP64 overlap test of Algorithm 1: || (r_a + Roff_a q_k) - r_b - dr e_s ||^2 <= Roff_b^2,
// written with explicit roundings so that the FP64 kernel and the FP32 guard-band recheck take
// identical decisions.
__device__ __forceinline__ bool covers64(double qx, double qy, double qz, double bx, double by, double bz,
                                         double roff2_b, int s, double dr) {
    double wx = __dsub_rn(qx, bx), wy = __dsub_rn(qy, by), wz = __dsub_rn(qz, bz);
    if (s == 0) wx = __dsub_rn(wx, dr);
    if (s == 1) wy = __dsub_rn(wy, dr);
    if (s == 2) wz = __dsub_rn(wz, dr);
    double d2 = __dadd_rn(__dadd_rn(__dmul_rn(wx, wx), __dmul_rn(wy, wy)), __dmul_rn(wz, wz));
    return d2 <= roff2_b;
}

// ================================================================ A1: forward kinematics
// chunk products P_c = G_{cC} o ... o G_{cC+C-1}; G_j stored for the apply pass
__global__ void k_fk_local(const DevChain d) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= d.nfk_chunks || d.status->done) return;
    int j0 = c * kFkChunk, j1 = min(d.l, j0 + kFkChunk);
    double P[12], Gj[12];
    joint_tf(&d.u0[3 * j0], &d.step0[3 * j0], d.theta[j0], P);
    aff_store(&d.G[12 * j0], P);
    for (int j = j0 + 1; j < j1; ++j) {
        joint_tf(&d.u0[3 * j], &d.step0[3 * j], d.theta[j], Gj);
        aff_store(&d.G[12 * j], Gj);
        aff_compose(P, Gj, P);
    }
    aff_store(&d.chunkP[12 * c], P);
}

// exclusive prefix of the chunk products, E_c = P_0 o ... o P_{c-1}, in one block: each thread
// folds a contiguous run, one thread scans the run totals, each thread rescans its run
__global__ void k_fk_scan(const DevChain d) {
    __shared__ double S[kScanThreads][12];
    if (d.status->done) return;
    int t = threadIdx.x, nc = d.nfk_chunks;
    int per = (nc + kScanThreads - 1) / kScanThreads;
    int c0 = min(nc, t * per), c1 = min(nc, c0 + per);
    double A[12], B[12];
    aff_identity(A);
    for (int c = c0; c < c1; ++c) {
        aff_load(&d.chunkP[12 * c], B);
        aff_compose(A, B, A);
    }
    for (int k = 0; k < 12; ++k) S[t][k] = A[k];
    __syncthreads();
    if (t == 0) {
        double X[12];
        aff_identity(X);
        for (int u = 0; u < kScanThreads; ++u) {
            for (int k = 0; k < 12; ++k) B[k] = S[u][k];
            for (int k = 0; k < 12; ++k) S[u][k] = X[k];
            aff_compose(X, B, X);
        }
    }
    __syncthreads();
    for (int k = 0; k < 12; ++k) A[k] = S[t][k];
    for (int c = c0; c < c1; ++c) {
        aff_store(&d.chunkE[12 * c], A);
        aff_load(&d.chunkP[12 * c], B);
        aff_compose(A, B, A);
    }
}

// link frame poses M_{j+1} = M_j o L_j; current axis u_j = R(M_j) u0_j through p_j = origin of
// frame j+1 (the joint's axis point)
__global__ void k_fk_apply(const DevChain d) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= d.nfk_chunks || d.status->done) return;
    int j0 = c * kFkChunk, j1 = min(d.l, j0 + kFkChunk);
    double X[12], Gj[12];
    aff_load(&d.chunkE[12 * c], X);
    for (int j = j0; j < j1; ++j) {
        const double* u = &d.u0[3 * j];
#pragma unroll
        for (int i = 0; i < 3; ++i) d.ucur[3 * j + i] = X[3 * i] * u[0] + X[3 * i + 1] * u[1] + X[3 * i + 2] * u[2];
        aff_load(&d.G[12 * j], Gj);
        aff_compose(X, Gj, X);
        aff_store(&d.M[12 * (j + 1)], X);
#pragma unroll
        for (int i = 0; i < 3; ++i) d.pcur[3 * j + i] = X[9 + i];
    }
}

__global__ void k_fk_atoms(const DevChain d) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= d.n || d.status->done) return;
    const double* M = &d.M[12 * d.link[a]];
    double x = d.r0[3 * a], y = d.r0[3 * a + 1], z = d.r0[3 * a + 2];
#pragma unroll
    for (int i = 0; i < 3; ++i) d.r[3 * a + i] = M[3 * i] * x + M[3 * i + 1] * y + M[3 * i + 2] * z + M[9 + i];
}

// ================================================================ A2: binning
__global__ void k_bbox(const DevChain d) {
    __shared__ double smin[3][8], smax[3][8];
    if (d.status->done) return;
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < d.n; a += gridDim.x * blockDim.x) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            double v = d.r[3 * a + i];
            mn[i] = fmin(mn[i], v);
            mx[i] = fmax(mx[i], v);
        }
    }
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        for (int o = 16; o > 0; o >>= 1) {
            mn[i] = fmin(mn[i], __shfl_down_sync(0xffffffffu, mn[i], o));
            mx[i] = fmax(mx[i], __shfl_down_sync(0xffffffffu, mx[i], o));
        }
        if (lane == 0) { smin[i][w] = mn[i]; smax[i][w] = mx[i]; }
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        int i = threadIdx.x;
        double a = INFINITY, b = -INFINITY;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { a = fmin(a, smin[i][k]); b = fmax(b, smax[i][k]); }
        atomicMin(&d.status->bbox[i], dkey(a));
        atomicMax(&d.status->bbox[3 + i], dkey(b));
    }
}

// grid from the bounding box; resets the box and the per-evaluation counters for the next pass
__global__ void k_grid_setup(const DevChain d) {
    Status* st = d.status;
    if (st->done) return;
    double mn[3], mx[3];
    for (int i = 0; i < 3; ++i) { mn[i] = dkey_inv(st->bbox[i]); mx[i] = dkey_inv(st->bbox[3 + i]); }
    double s = fmax(d.rmax * (1.0 + 1e-12) + 1e-9, d.prm.cell_size);
    s = ceil(s * 1024.0) / 1024.0;
    GridInfo g;
    bool finite = isfinite(mx[0] - mn[0]) && isfinite(mx[1] - mn[1]) && isfinite(mx[2] - mn[2]);
    if (!finite) {
        atomicOr(&st->error, kErrNonfinite);
        st->done = 1;
        for (int i = 0; i < 3; ++i) { mn[i] = 0.0; mx[i] = 0.0; }
    }
    for (;;) {
        long long nx = (long long)floor((mx[0] - mn[0]) / s) + 1;
        long long ny = (long long)floor((mx[1] - mn[1]) / s) + 1;
        long long nz = (long long)floor((mx[2] - mn[2]) / s) + 1;
        if (nx * ny * nz <= (long long)d.cell_cap) {
            g.nx = (int)nx; g.ny = (int)ny; g.nz = (int)nz;
            g.ncells = (int)(nx * ny * nz);
            break;
        }
        s = ceil(s * 1.25 * 1024.0) / 1024.0;
    }
    g.ox = mn[0]; g.oy = mn[1]; g.oz = mn[2];
    g.s = s;
    *d.grid = g;
    for (int i = 0; i < 3; ++i) { st->bbox[i] = ~0ULL; st->bbox[3 + i] = 0ULL; }
    st->pairs = 0;
    st->nbr_total = 0;
    st->guard = 0;
    st->sasa_tests = 0;
    st->max_nbr = 0;
}

__device__ __forceinline__ int cell_of(const GridInfo& g, double x, double y, double z) {
    int cx = min(max((int)floor((x - g.ox) / g.s), 0), g.nx - 1);
    int cy = min(max((int)floor((y - g.oy) / g.s), 0), g.ny - 1);
    int cz = min(max((int)floor((z - g.oz) / g.s), 0), g.nz - 1);
    return (cz * g.ny + cy) * g.nx + cx;
}

// cell counts with one atomic per group of lanes that share a cell (consecutive atoms of a chain
// mostly share one)
__global__ void k_bin_count(const DevChain d) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= d.n || d.status->done) return;
    const GridInfo g = *d.grid;
    int key = cell_of(g, d.r[3 * a], d.r[3 * a + 1], d.r[3 * a + 2]);
    d.key[a] = key;
    unsigned peers = __match_any_sync(__activemask(), key);
    int lane = threadIdx.x & 31;
    if (lane == __ffs(peers) - 1) atomicAdd(&d.cell_count[key], __popc(peers));
}

// exclusive scan of the cell counts (one block); zeroes the counts for the next pass
__global__ void k_bin_scan(const DevChain d) {
    __shared__ int wsum[32];
    if (d.status->done) return;
    int nc = d.grid->ncells;
    int t = threadIdx.x, T = blockDim.x;
    int per = (nc + T - 1) / T;
    int c0 = min(nc, t * per), c1 = min(nc, c0 + per);
    int local = 0;
    for (int c = c0; c < c1; ++c) local += d.cell_count[c];
    int lane = t & 31, w = t >> 5;
    int v = local;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) wsum[w] = v;
    __syncthreads();
    if (w == 0) {
        int x = (lane < (T >> 5)) ? wsum[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        wsum[lane] = x;  // inclusive over warps
    }
    __syncthreads();
    int base = v - local + (w > 0 ? wsum[w - 1] : 0);
    for (int c = c0; c < c1; ++c) {
        int cnt = d.cell_count[c];
        d.cell_start[c] = base;
        d.cell_cursor[c] = base;
        d.cell_count[c] = 0;
        base += cnt;
    }
    if (t == T - 1) d.cell_start[nc] = base;
}

__global__ void k_bin_scatter(const DevChain d) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= d.n || d.status->done) return;
    int key = d.key[a];
    unsigned peers = __match_any_sync(__activemask(), key);
    int lane = threadIdx.x & 31;
    int leader = __ffs(peers) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(&d.cell_cursor[key], __popc(peers));
    base = __shfl_sync(peers, base, leader);
    int rank = __popc(peers & ((1u << lane) - 1u));
    d.sorted[base + rank] = a;
}

// order each cell by atom index (the scatter order depends on timing)
__global__ void k_bin_sortcells(const DevChain d) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (d.status->done || c >= d.grid->ncells) return;
    int b0 = d.cell_start[c], b1 = d.cell_start[c + 1];
    for (int i = b0 + 1; i < b1; ++i) {
        int v = d.sorted[i];
        int j = i - 1;
        while (j >= b0 && d.sorted[j] > v) {
            d.sorted[j + 1] = d.sorted[j];
            --j;
        }
        d.sorted[j + 1] = v;
    }
}

// sorted copies: FP64 centres, or FP32 offsets from the cell corner (|offset| < s, so the FP32
// rounding error is below s * 2^-24)
template <bool MIXED>
__global__ void k_bin_gather(const DevChain d) {
    int sl = blockIdx.x * blockDim.x + threadIdx.x;
    if (sl >= d.n || d.status->done) return;
    const GridInfo g = *d.grid;
    int a = d.sorted[sl];
    int key = d.key[a];
    d.slot_cell[sl] = key;
    double x = d.r[3 * a], y = d.r[3 * a + 1], z = d.r[3 * a + 2];
    dbl4 pa = d.aprm64[a];
    if (MIXED) {
        int cx = key % g.nx, cy = (key / g.nx) % g.ny, cz = key / (g.nx * g.ny);
        float ox = (float)(x - (g.ox + cx * g.s));
        float oy = (float)(y - (g.oy + cy * g.s));
        float oz = (float)(z - (g.oz + cz * g.s));
        d.spos32[sl] = make_float4(ox, oy, oz, (float)pa.x);
        d.sprm32[sl] = d.aprm32[a];
    } else {
        d.spos64[sl] = make_dbl4(x, y, z, pa.x);
        d.sprm64[sl] = pa;
    }
}

// ================================================================ A3-A5: pair forces + lists
template <bool MIXED>
__global__ void __launch_bounds__(kPairTpb) k_pair(const DevChain d) {
    typedef typename std::conditional<MIXED, float, double>::type R;
    __shared__ double sE[2][kPairTpb / 32];
    __shared__ unsigned long long sC[3][kPairTpb / 32];
    __shared__ int sM[kPairTpb / 32];
    const int sl = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = sl < d.n && !d.status->done;
    double Eel = 0.0, Evdw = 0.0;
    unsigned long long npairs = 0, nguard = 0;
    int ncount = 0;
    if (active) {
        const GridInfo g = *d.grid;
        const int a = d.sorted[sl];
        const int cell = d.slot_cell[sl];
        const int cx = cell % g.nx, cy = (cell / g.nx) % g.ny, cz = cell / (g.nx * g.ny);
        const R K = (R)d.prm.coulomb_k;
        const R w14e = (R)d.prm.w14_elec, w14v = (R)d.prm.w14_vdw;
        const R rc2 = (R)d.rcut2, rv2 = (R)d.rvdw2;
        const R rall2 = (R)(d.rmax * d.rmax) + (R)d.guard_pair;
        const R gp = (R)d.guard_pair;
        const R dr = (R)d.prm.delta_r;
        const R pad = MIXED ? (R)0.01 : (R)0.0;
        const bool solv = d.prm.solvation != 0;
        const R sf = (R)g.s;
        R px, py, pz, qi, sei, Ri, Roi;
        if (MIXED) {
            float4 p = d.spos32[sl], q = d.sprm32[sl];
            px = p.x; py = p.y; pz = p.z; qi = p.w;
            sei = q.y; Ri = q.z; Roi = q.w;
        } else {
            dbl4 p = d.spos64[sl], q = d.sprm64[sl];
            px = p.x; py = p.y; pz = p.z; qi = p.w;
            sei = q.y; Ri = q.z; Roi = q.w;
        }
        const unsigned long long exa = d.exm[a], m14a = d.m14m[a];
        R fx = 0, fy = 0, fz = 0;
        R eel = 0, evdw = 0;
        for (int dz = -1; dz <= 1; ++dz) {
            int ncz = cz + dz;
            if (ncz < 0 || ncz >= g.nz) continue;
            for (int dy = -1; dy <= 1; ++dy) {
                int ncy = cy + dy;
                if (ncy < 0 || ncy >= g.ny) continue;
                for (int dx = -1; dx <= 1; ++dx) {
                    int ncx = cx + dx;
                    if (ncx < 0 || ncx >= g.nx) continue;
                    int nc = (ncz * g.ny + ncy) * g.nx + ncx;
                    int t0 = d.cell_start[nc], t1 = d.cell_start[nc + 1];
                    // r_i - r_j = (o_i - o_j) - (c_j - c_i) s for cell-relative offsets
                    const R shx = MIXED ? (R)dx * sf : (R)0, shy = MIXED ? (R)dy * sf : (R)0, shz = MIXED ? (R)dz * sf : (R)0;
                    for (int t = t0; t < t1; ++t) {
                        if (t == sl) continue;
                        R qj, sej, Rj, Roj, ddx, ddy, ddz;
                        if (MIXED) {
                            float4 p = d.spos32[t];
                            ddx = (px - p.x) - shx; ddy = (py - p.y) - shy; ddz = (pz - p.z) - shz;
                            qj = p.w;
                        } else {
                            dbl4 p = d.spos64[t];
                            ddx = __dsub_rn(px, p.x); ddy = __dsub_rn(py, p.y); ddz = __dsub_rn(pz, p.z);
                            qj = p.w;
                        }
                        R d2;
                        if constexpr (MIXED) d2 = ddx * ddx + ddy * ddy + ddz * ddz;
                        else d2 = __dadd_rn(__dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy)), __dmul_rn(ddz, ddz));
                        if (d2 > rall2) continue;
                        const int b = d.sorted[t];
                        if (MIXED) {
                            float4 q = d.sprm32[t];
                            sej = q.y; Rj = q.z; Roj = q.w;
                        } else {
                            dbl4 q = d.sprm64[t];
                            sej = q.y; Rj = q.z; Roj = q.w;
                        }
                        if (solv) {  // solvation neighbour A'_i: d_ij <= Roff_i + Roff_j + dr
                            R lim = Roi + Roj + dr + pad;
                            if (d2 <= lim * lim) {
                                if (ncount < kMaxNbr) {
                                    d.nbr[(size_t)a * kMaxNbr + ncount] = b;
                                    if (MIXED) d.nbr_off[(size_t)a * kMaxNbr + ncount] = make_float4(-(float)ddx, -(float)ddy, -(float)ddz, (float)(Roj * Roj));
                                }
                                ++ncount;
                            }
                        }
                        // bond class from the lower index's masks (Sec. 3.3)
                        int lo = min(a, b), off = max(a, b) - lo;
                        bool excl = false, is14 = false;
                        if (off <= kMaskWindow) {
                            unsigned long long em = (lo == a) ? exa : d.exm[b];
                            unsigned long long mm = (lo == a) ? m14a : d.m14m[b];
                            excl = (em >> off) & 1ULL;
                            is14 = (mm >> off) & 1ULL;
                        }
                        if (excl) continue;
                        bool inE = d2 <= rc2, inV = d2 <= rv2;
                        if (MIXED && (fabs(d2 - rc2) <= gp || fabs(d2 - rv2) <= gp)) {
                            // guard band: decide the cutoff in FP64 as the FP64 path does
                            double ex = __dsub_rn(d.r[3 * a], d.r[3 * b]), ey = __dsub_rn(d.r[3 * a + 1], d.r[3 * b + 1]),
                                   ez = __dsub_rn(d.r[3 * a + 2], d.r[3 * b + 2]);
                            double d64 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
                            inE = d64 <= d.rcut2;
                            inV = d64 <= d.rvdw2;
                            ++nguard;
                        }
                        if (!inE && !inV) continue;
                        R we = is14 ? w14e : (R)1, wv = is14 ? w14v : (R)1;
                        R inv2 = (R)1 / d2;
                        R coef = 0;
                        const bool count_e = a < b;
                        if (inE) {
                            R qq = we * K * qi * qj;
                            coef += (R)0.5 * qq * inv2 * inv2;
                            if (count_e) eel += (R)0.25 * qq * inv2;
                        }
                        if (inV) {
                            R D = Ri + Rj;
                            R D2 = D * D;
                            R t6 = D2 * D2 * D2 * inv2 * inv2 * inv2;
                            R t12 = t6 * t6;
                            R eij = wv * sei * sej;
                            coef += (R)12 * eij * (t12 - t6) * inv2;
                            if (count_e) evdw += eij * (t12 - (R)2 * t6);
                        }
                        if (count_e && (we != (R)0 || wv != (R)0)) ++npairs;
                        fx += coef * ddx; fy += coef * ddy; fz += coef * ddz;
                    }
                }
            }
        }
        d.Fpair[3 * a] = (double)fx;
        d.Fpair[3 * a + 1] = (double)fy;
        d.Fpair[3 * a + 2] = (double)fz;
        d.nbr_cnt[a] = ncount;
        if (ncount > kMaxNbr) atomicOr(&d.status->error, kErrOverflow);
        Eel = (double)eel;
        Evdw = (double)evdw;
    }
    // block partials (fixed tree: deterministic)
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    Eel = warp_sum(Eel);
    Evdw = warp_sum(Evdw);
    npairs = warp_sum(npairs);
    nguard = warp_sum(nguard);
    unsigned long long nc64 = warp_sum((unsigned long long)ncount);
    int mx = warp_max(ncount);
    if (lane == 0) { sE[0][w] = Eel; sE[1][w] = Evdw; sC[0][w] = npairs; sC[1][w] = nguard; sC[2][w] = nc64; sM[w] = mx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double e0 = 0, e1 = 0;
        unsigned long long c0 = 0, c1 = 0, c2 = 0;
        int m = 0;
        for (int k = 0; k < kPairTpb / 32; ++k) { e0 += sE[0][k]; e1 += sE[1][k]; c0 += sC[0][k]; c1 += sC[1][k]; c2 += sC[2][k]; m = max(m, sM[k]); }
        d.Epair[2 * blockIdx.x] = e0;
        d.Epair[2 * blockIdx.x + 1] = e1;
        if (c0) atomicAdd(&d.status->pairs, c0);
        if (c1) atomicAdd(&d.status->guard, c1);
        if (c2) atomicAdd(&d.status->nbr_total, c2);
        if (m) atomicMax(&d.status->max_nbr, m);
    }
}

// ================================================================ A6: Algorithm 1
// One warp per atom i; lane L takes the sample points k = L, L + 32, ... Step 1 counts the
// overlapping neighbours of each point up to two and keeps the critical one; step 2 re-tests
// exposed points (C = 0) against every neighbour displaced by dr e_s and critically overlapped
// points (C = 1) against their critical neighbour only. Net exchange counts per (j, s) go to
// shared memory; the force quantum G0_i / (N dr) is applied in fixed point, so
// F_j += q c_js and F_i -= q c_js are exact integer additions.
template <bool MIXED>
__global__ void __launch_bounds__(kSasaWarps * 32) k_sasa(const DevChain d) {
    __shared__ int s_idx[kSasaWarps][kMaxNbr];
    __shared__ int s_cnt[kSasaWarps][3 * kMaxNbr];
    __shared__ float4 s_off[kSasaWarps][MIXED ? kMaxNbr : 1];
    __shared__ dbl4 s_pos[kSasaWarps][MIXED ? 1 : kMaxNbr];
    __shared__ double s_E[kSasaWarps];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int a = blockIdx.x * kSasaWarps + w;
    double Ea = 0.0;
    if (a < d.n && !d.status->done) {
        const double G0a = d.G0[a];
        if (G0a == 0.0) {
            if (lane == 0) d.covered[a] = 0;
        } else {
            const int cnt = min(d.nbr_cnt[a], kMaxNbr);
            for (int k = lane; k < cnt; k += 32) {
                int b = d.nbr[(size_t)a * kMaxNbr + k];
                s_idx[w][k] = b;
                s_cnt[w][3 * k] = 0; s_cnt[w][3 * k + 1] = 0; s_cnt[w][3 * k + 2] = 0;
                if (MIXED) {
                    s_off[w][k] = d.nbr_off[(size_t)a * kMaxNbr + k];
                } else {
                    double ro = d.aprm64[b].w;
                    s_pos[w][k] = make_dbl4(d.r[3 * b], d.r[3 * b + 1], d.r[3 * b + 2], __dmul_rn(ro, ro));
                }
            }
            __syncwarp();
            const double Roa = d.aprm64[a].w;
            const double rax = d.r[3 * a], ray = d.r[3 * a + 1], raz = d.r[3 * a + 2];
            const float Raf = (float)Roa;
            const double dr = d.prm.delta_r;
            const float drf = (float)dr;
            const float gs = d.guard_sasa;
            int ncov = 0, nguard = 0;
            unsigned long long ntest = 0;
            for (int k = lane; k < d.N; k += 32) {
                // T_i(q_k) = r_i + Roff_i q_k (Sec. 3.4): FP64 always in the FP64 kernel, and only
                // for guard-band rechecks in the mixed kernel
                double qx = 0, qy = 0, qz = 0;
                float vx = 0, vy = 0, vz = 0;
                if constexpr (MIXED) {
                    vx = Raf * d.Q32[3 * k]; vy = Raf * d.Q32[3 * k + 1]; vz = Raf * d.Q32[3 * k + 2];
                } else {
                    qx = __dadd_rn(rax, __dmul_rn(Roa, d.Q64[3 * k]));
                    qy = __dadd_rn(ray, __dmul_rn(Roa, d.Q64[3 * k + 1]));
                    qz = __dadd_rn(raz, __dmul_rn(Roa, d.Q64[3 * k + 2]));
                }
                auto test = [&](int j, int s) -> bool {
                    ++ntest;
                    if constexpr (MIXED) {
                        float4 o = s_off[w][j];
                        float wx = vx - o.x, wy = vy - o.y, wz = vz - o.z;
                        if (s == 0) wx -= drf;
                        if (s == 1) wy -= drf;
                        if (s == 2) wz -= drf;
                        float diff = wx * wx + wy * wy + wz * wz - o.w;
                        if (fabsf(diff) > gs) return diff <= 0.0f;
                        ++nguard;
                        int b = s_idx[w][j];
                        double ro = d.aprm64[b].w;
                        double gx = __dadd_rn(rax, __dmul_rn(Roa, d.Q64[3 * k]));
                        double gy = __dadd_rn(ray, __dmul_rn(Roa, d.Q64[3 * k + 1]));
                        double gz = __dadd_rn(raz, __dmul_rn(Roa, d.Q64[3 * k + 2]));
                        return covers64(gx, gy, gz, d.r[3 * b], d.r[3 * b + 1], d.r[3 * b + 2], __dmul_rn(ro, ro), s, dr);
                    } else {
                        dbl4 p = s_pos[w][j];
                        return covers64(qx, qy, qz, p.x, p.y, p.z, p.w, s, dr);
                    }
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
            nguard = warp_sum(nguard);
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
            if (lane == 0) {
                if (f0) atomicAdd((unsigned long long*)&d.Fcav[3 * a], (unsigned long long)f0);
                if (f1) atomicAdd((unsigned long long*)&d.Fcav[3 * a + 1], (unsigned long long)f1);
                if (f2) atomicAdd((unsigned long long*)&d.Fcav[3 * a + 2], (unsigned long long)f2);
                d.covered[a] = ncov;
                if (nguard) atomicAdd(&d.status->guard, (unsigned long long)nguard);
                atomicAdd(&d.status->sasa_tests, ntest);
                Ea = G0a - G0a * (double)ncov / (double)d.N;  // G^cav_i = G0_i f_i
            }
        }
    }
    if (lane == 0) s_E[w] = Ea;
    __syncthreads();
    if (threadIdx.x == 0) {
        double e = 0.0;
        for (int k = 0; k < kSasaWarps; ++k) e += s_E[k];
        d.Ecav[blockIdx.x] = e;
    }
}

// ================================================================ A7-A8: wrenches, suffix sums, torques
__global__ void k_wrench(const DevChain d) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= d.nlink_chunks || d.status->done) return;
    int h0 = c * kLinkChunk, h1 = min(d.L, h0 + kLinkChunk);
    const bool solv = d.prm.solvation != 0;
    double S[6] = {0, 0, 0, 0, 0, 0};
    for (int h = h0; h < h1; ++h) {
        double T0 = 0, T1 = 0, T2 = 0, F0 = 0, F1 = 0, F2 = 0;
        for (int a = d.link_start[h]; a < d.link_start[h + 1]; ++a) {
            double fx = d.Fpair[3 * a], fy = d.Fpair[3 * a + 1], fz = d.Fpair[3 * a + 2];
            if (solv) {
                fx += (double)d.Fcav[3 * a] * kFxInv;
                fy += (double)d.Fcav[3 * a + 1] * kFxInv;
                fz += (double)d.Fcav[3 * a + 2] * kFxInv;
            }
            double x = d.r[3 * a], y = d.r[3 * a + 1], z = d.r[3 * a + 2];
            T0 += y * fz - z * fy;  // r x F about the origin (eq. KCM_02)
            T1 += z * fx - x * fz;
            T2 += x * fy - y * fx;
            F0 += fx; F1 += fy; F2 += fz;
        }
        double* P = &d.P[6 * h];
        P[0] = T0; P[1] = T1; P[2] = T2; P[3] = F0; P[4] = F1; P[5] = F2;
        if (h >= 1) { S[0] += T0; S[1] += T1; S[2] += T2; S[3] += F0; S[4] += F1; S[5] += F2; }
    }
    for (int k = 0; k < 6; ++k) d.chunkS[6 * c + k] = S[k];
}

// exclusive suffix sums of the chunk sums (one block)
__global__ void k_torque_scan(const DevChain d) {
    __shared__ double S[kScanThreads][6];
    if (d.status->done) return;
    int t = threadIdx.x, nc = d.nlink_chunks;
    int per = (nc + kScanThreads - 1) / kScanThreads;
    int c0 = min(nc, t * per), c1 = min(nc, c0 + per);
    double A[6] = {0, 0, 0, 0, 0, 0};
    for (int c = c1 - 1; c >= c0; --c)
        for (int k = 0; k < 6; ++k) A[k] += d.chunkS[6 * c + k];
    for (int k = 0; k < 6; ++k) S[t][k] = A[k];
    __syncthreads();
    if (t == 0) {
        double run[6] = {0, 0, 0, 0, 0, 0};
        for (int u = kScanThreads - 1; u >= 0; --u)
            for (int k = 0; k < 6; ++k) {
                double v = S[u][k];
                S[u][k] = run[k];
                run[k] += v;
            }
    }
    __syncthreads();
    for (int k = 0; k < 6; ++k) A[k] = S[t][k];
    for (int c = c1 - 1; c >= c0; --c)
        for (int k = 0; k < 6; ++k) {
            d.chunkSuf[6 * c + k] = A[k];
            A[k] += d.chunkS[6 * c + k];
        }
}

// P^agg_k = P_k + P^agg_{k+1} (Sec. 3.5); tau_k = u_k . T^agg_k + (p_k x u_k) . F^agg_k
__global__ void k_torque_apply(const DevChain d) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= d.nlink_chunks || d.status->done) return;
    int h0 = c * kLinkChunk, h1 = min(d.L, h0 + kLinkChunk);
    double A[6];
    for (int k = 0; k < 6; ++k) A[k] = d.chunkSuf[6 * c + k];
    double tmax = 0.0;
    bool bad = false;
    for (int h = h1 - 1; h >= h0; --h) {
        if (h < 1) break;
        for (int k = 0; k < 6; ++k) A[k] += d.P[6 * h + k];
        int j = h - 1;  // joint k = h (1-based) moves links h..l
        const double* u = &d.ucur[3 * j];
        const double* p = &d.pcur[3 * j];
        double px = p[1] * u[2] - p[2] * u[1], py = p[2] * u[0] - p[0] * u[2], pz = p[0] * u[1] - p[1] * u[0];
        double t = u[0] * A[0] + u[1] * A[1] + u[2] * A[2] + px * A[3] + py * A[4] + pz * A[5];
        d.tau[j] = t;
        if (!isfinite(t)) bad = true;
        tmax = fmax(tmax, fabs(t));
    }
    if (bad) atomicOr(&d.status->error, kErrNonfinite);
    else if (tmax > 0.0) atomicMax(&d.status->max_abs_tau, (unsigned long long)__double_as_longlong(tmax));
}

// ================================================================ A10: energies
__global__ void k_energy(const DevChain d) {
    __shared__ double s[3][256];
    if (d.status->done) return;
    double e0 = 0, e1 = 0, e2 = 0;
    for (int b = threadIdx.x; b < d.pair_blocks; b += blockDim.x) { e0 += d.Epair[2 * b]; e1 += d.Epair[2 * b + 1]; }
    if (d.prm.solvation)
        for (int b = threadIdx.x; b < d.sasa_blocks; b += blockDim.x) e2 += d.Ecav[b];
    s[0][threadIdx.x] = e0; s[1][threadIdx.x] = e1; s[2][threadIdx.x] = e2;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int k = 0; k < 3; ++k) s[k][threadIdx.x] += s[k][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) { d.E[0] = s[0][0]; d.E[1] = s[1][0]; d.E[2] = s[2][0]; }
}

// ================================================================ A9: step
__global__ void k_step(const DevChain d) {
    __shared__ double smax[4];
    Status* st = d.status;
    if (st->done) return;
    if (st->error) {
        if (blockIdx.x == 0 && threadIdx.x == 0) st->done = 1;
        return;
    }
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    double ad = 0.0;
    if (j < d.l) {
        double t = d.tau[j], dt;
        if (d.prm.step_mode == KCM_STEP_NORMALIZED) {
            double tm = __longlong_as_double((long long)st->max_abs_tau);
            dt = tm > 0.0 ? d.prm.kappa * t / tm : 0.0;
        } else {
            dt = fmin(fmax(d.prm.kappa * t, -d.prm.dtheta_max), d.prm.dtheta_max);
        }
        d.theta[j] += dt;
        d.dtheta[j] = dt;
        ad = fabs(dt);
    }
    for (int o = 16; o > 0; o >>= 1) ad = fmax(ad, __shfl_down_sync(0xffffffffu, ad, o));
    if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = ad;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) m = fmax(m, smax[k]);
        atomicMax(&st->max_dtheta, (unsigned long long)__double_as_longlong(m));
        __threadfence();
        unsigned int ticket = atomicAdd(&st->ticket, 1u);
        if (ticket == gridDim.x - 1) {  // last block: close the iteration
            __threadfence();
            double mall = __longlong_as_double((long long)atomicAdd(&st->max_dtheta, 0ULL));
            st->last_max_dtheta = mall;
            st->iters += 1;
            if (mall < d.prm.conv_tol) st->done = 1;
            st->max_dtheta = 0ULL;
            st->max_abs_tau = 0ULL;
            st->ticket = 0u;
        }
    }
}

__global__ void k_reset_loop(const DevChain d, int full) {
    Status* st = d.status;
    st->iters = 0;
    st->done = 0;
    st->error = 0;
    st->ticket = 0u;
    st->max_dtheta = 0ULL;
    st->max_abs_tau = 0ULL;
    st->last_max_dtheta = 0.0;
    if (full) {
        for (int i = 0; i < 3; ++i) { st->bbox[i] = ~0ULL; st->bbox[3 + i] = 0ULL; }
        st->pairs = 0; st->nbr_total = 0; st->guard = 0; st->sasa_tests = 0; st->max_nbr = 0;
    }
}

__global__ void k_force_out(const DevChain d) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= 3 * d.n) return;
    double fc = d.prm.solvation ? (double)d.Fcav[x] * kFxInv : 0.0;
    d.Fcav64[x] = fc;
    d.Ftot[x] = d.Fpair[x] + fc;
}

inline int blocks(long long n, int tpb) { return (int)((n + tpb - 1) / tpb); }

}  // namespace

void launch_init_status(DevChain& d, cudaStream_t s) { k_reset_loop<<<1, 1, 0, s>>>(d, 1); }
void launch_reset_loop(DevChain& d, cudaStream_t s) { k_reset_loop<<<1, 1, 0, s>>>(d, 0); }

void launch_fk(DevChain& d, cudaStream_t s) {
    k_fk_local<<<blocks(d.nfk_chunks, kFkTpb), kFkTpb, 0, s>>>(d);
    k_fk_scan<<<1, kScanThreads, 0, s>>>(d);
    k_fk_apply<<<blocks(d.nfk_chunks, kFkTpb), kFkTpb, 0, s>>>(d);
    k_fk_atoms<<<blocks(d.n, kApplyTpb), kApplyTpb, 0, s>>>(d);
}

void launch_binning(DevChain& d, cudaStream_t s) {
    k_bbox<<<std::min(blocks(d.n, 256), 4 * 148), 256, 0, s>>>(d);
    k_grid_setup<<<1, 1, 0, s>>>(d);
    k_bin_count<<<blocks(d.n, 256), 256, 0, s>>>(d);
    k_bin_scan<<<1, 1024, 0, s>>>(d);
    k_bin_scatter<<<blocks(d.n, 256), 256, 0, s>>>(d);
    k_bin_sortcells<<<blocks(d.cell_cap, 256), 256, 0, s>>>(d);
    if (d.prm.precision == KCM_MIXED)
        k_bin_gather<true><<<blocks(d.n, 256), 256, 0, s>>>(d);
    else
        k_bin_gather<false><<<blocks(d.n, 256), 256, 0, s>>>(d);
}

void launch_pairs(DevChain& d, cudaStream_t s) {
    if (d.prm.precision == KCM_MIXED)
        k_pair<true><<<d.pair_blocks, kPairTpb, 0, s>>>(d);
    else
        k_pair<false><<<d.pair_blocks, kPairTpb, 0, s>>>(d);
}

void launch_forces(DevChain& d, cudaStream_t s) {
    launch_pairs(d, s);
    launch_sasa(d, s);
}

void launch_sasa(DevChain& d, cudaStream_t s) {
    if (d.prm.solvation) {
        cudaMemsetAsync(d.Fcav, 0, sizeof(long long) * 3 * (size_t)d.n, s);
        if (d.prm.precision == KCM_MIXED)
            k_sasa<true><<<d.sasa_blocks, kSasaWarps * 32, 0, s>>>(d);
        else
            k_sasa<false><<<d.sasa_blocks, kSasaWarps * 32, 0, s>>>(d);
    }
}

void launch_torques(DevChain& d, cudaStream_t s) {
    k_wrench<<<blocks(d.nlink_chunks, kFkTpb), kFkTpb, 0, s>>>(d);
    k_torque_scan<<<1, kScanThreads, 0, s>>>(d);
    k_torque_apply<<<blocks(d.nlink_chunks, kFkTpb), kFkTpb, 0, s>>>(d);
}

void launch_energy(DevChain& d, cudaStream_t s) { k_energy<<<1, 256, 0, s>>>(d); }

void launch_step(DevChain& d, cudaStream_t s) { k_step<<<blocks(d.l, 128), 128, 0, s>>>(d); }

void launch_force_out(DevChain& d, cudaStream_t s) { k_force_out<<<blocks(3LL * d.n, 256), 256, 0, s>>>(d); }

}  // namespace kcm
