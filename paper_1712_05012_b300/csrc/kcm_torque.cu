// A7-A9: link wrenches, suffix sums over links, joint torques and the kinetostatic step: FP64 in
// FP64 mode, double-float (kcm_df.cuh) in mixed mode; the step itself updates theta in FP64. The
// wrench kernel, which visits every atom once with one thread each, also converts the mixed-mode
// fixed-point forces, adds the cavity energy G0_i f_i and the pair energies of its atoms per chain,
// and totals the per-atom counters of the pair and solvation kernels.
//
// Wrench of link h about the origin, P_h = [sum r x F ; sum F] (eq. KCM_01/02), and
// P^agg_k = sum_{h >= k} P_h (Sec. 3.5) as a reverse scan: k_wrench_tile forms P_h from the atoms of
// a 32-link tile and scans the tile, its last block scans the tile totals, and k_torque takes
// tau_k = u_k . T^agg_k + (p_k x u_k) . F^agg_k (eq. KCM_05/06).
// In the clamped step mode the same thread applies dtheta_k = clamp(kappa tau_k, +-dtheta_max)
// (eq. KCM_07); the last block to finish closes the iteration.
#include <cuda_runtime.h>

#include <type_traits>

#include "kcm_common.cuh"
#include "kcm_df.cuh"
#include "kcm_device.h"

namespace kcm {

namespace {
using namespace dev;

// Per-chain maxima of non-negative doubles (as bit patterns) and sums: one atomic per warp when the
// warp's lanes agree on the chain (c < 0: no value), else one per lane.
__device__ __forceinline__ void chain_max(unsigned long long* arr, int c, unsigned long long v) {
    const int cw = __reduce_max_sync(0xffffffffu, c);
    if (__all_sync(0xffffffffu, c == cw || c < 0)) {
        for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_down_sync(0xffffffffu, v, o));
        if ((threadIdx.x & 31) == 0 && cw >= 0 && v) atomicMax(&arr[cw], v);
    } else if (c >= 0 && v) {
        atomicMax(&arr[c], v);
    }
}
template <class V>
__device__ __forceinline__ void chain_add(double* arr, int stride, int c, V v) {
    const int cw = __reduce_max_sync(0xffffffffu, c);
    if (__all_sync(0xffffffffu, c == cw || c < 0)) {
        v = warp_sum(v);
        if ((threadIdx.x & 31) == 0 && cw >= 0 && v != (V)0) atomicAdd(&arr[stride * cw], (double)v);
    } else if (c >= 0 && v != (V)0) {
        atomicAdd(&arr[stride * c], (double)v);
    }
}

// Segmented exclusive suffix sums of the tile totals (component w) by the wrench kernel's last block:
// R_t = x_t + (a chain ends in tile t ? 0 : R_{t+1}), the suffix of tile totals from t to the first
// chain end; tileSuf_t = R_{t+1}. A lane takes K consecutive tiles (their loads issued together): its
// own segmented suffix over them, then a warp scan of the lanes' aggregates, then the tiles' R from
// the next lane's first R; rounds of 32 K tiles from the end, carrying R of the first tile of the
// later round. K = 1 for a few tiles (one round of single tiles is the shortest path), 8 for many.
template <int kSufK, class T>
__device__ __forceinline__ void tile_suffix(const DevChain& d, T* tileSuf, int w, int lane) {
    T carry = num_f<T>(0.0f);
    for (int top = d.ltiles; top > 0; top -= 32 * kSufK) {
        const int b = top - 32 * kSufK + lane * kSufK;  // the lane's first tile
        T x[kSufK];
        bool tl[kSufK];
#pragma unroll
        for (int k = 0; k < kSufK; ++k) {
            const int tt = b + k;
            x[k] = num_f<T>(0.0f);
            tl[k] = true;
            if (tt >= 0) {
                const double raw = __ldcg(&d.tileS[6 * (size_t)tt + w]);  // the slot of a T, read past L1
                x[k] = *reinterpret_cast<const T*>(&raw);
                tl[k] = __ldcg(&d.tileT[tt]) != 0;
            }
        }
        T r[kSufK];      // in-lane suffix from tile b + k to the first chain end or the lane's last tile
        bool op[kSufK];  // no chain end in tiles b + k .. of the lane: the next lane's R continues it
        r[kSufK - 1] = x[kSufK - 1];
        op[kSufK - 1] = !tl[kSufK - 1];
#pragma unroll
        for (int k = kSufK - 2; k >= 0; --k) {
            r[k] = tl[k] ? x[k] : add(x[k], r[k + 1]);
            op[k] = !tl[k] && op[k + 1];
        }
        T X = r[0];
        bool TL = !op[0];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const T y = shfl_down(X, off);
            const bool yt = __shfl_down_sync(0xffffffffu, TL, off);
            if (lane + off < 32 && !TL) { X = add(X, y); TL = yt; }
        }
        const T RL = TL ? X : add(X, carry);  // R of the lane's first tile
        T Rn = shfl_down(RL, 1);                // R of the next lane's first tile
        if (lane == 31) Rn = carry;
#pragma unroll
        for (int k = 0; k < kSufK; ++k) {
            const int tt = b + k;
            // tileSuf_t = R_{t+1}: the in-lane suffix of the next tile, continued by the next lane's R
            const T e = k + 1 < kSufK ? (op[k + 1] ? add(r[k + 1], Rn) : r[k + 1]) : Rn;
            if (tt >= 0) tileSuf[6 * (size_t)tt + w] = e;
        }
        carry = shfl(RL, 0);
    }
}

// One block per tile of 32 links h in [32 t, 32 t + 32). The block's threads take the tile's atoms
// (r x F and F, with the conversion of the mixed-mode fixed-point forces) into shared memory; one
// thread per (component, link) adds the link's atoms in atom order; warp q then scans component q of
// the tile's P_h from the end (Kogge-Stone, segmented at the last link of each chain: a chain's
// sums never take in the next chain), and the last block to finish (ticket, no waiting) forms the
// segmented exclusive suffix sums of the tile totals.
template <class T, bool SIDE>
__global__ void __launch_bounds__(kWrenchWarps * 32) k_wrench_tile(const DevChain d) {
    constexpr bool DF = std::is_same<T, df>::value;
    __shared__ T sV[kWrenchTileAtoms][6];
    __shared__ T sP[32][6];
    __shared__ unsigned long long sSt[kWrenchWarps][4];
    __shared__ int sMx[kWrenchWarps];
    __shared__ bool last;
    Status* st = d.status;
    if (st->done) return;
    const int t = blockIdx.x, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int h0 = 32 * t, h1 = min(h0 + 32, d.L);
    const int a0 = d.link_start[h0], a1 = d.link_start[h1];
    const T* rr = reinterpret_cast<const T*>(DF ? d.rdf : d.r);
    // side-chain joint of the thread among those of the tile's links (at most 64: four per CA link):
    // its bond a -> b, the end of the atoms it moves, the bond's first atom and unit direction
    // u = (b - a) / |b - a| (the ZP bond length), loaded here so that they arrive during the atom loop
    int sc = 0, sc1 = 0, sb = 0, se = 0;
    T sA[3], sU[3];
    if (SIDE) {
        sc = d.chi_tile[t] + threadIdx.x;
        sc1 = d.chi_tile[t + 1];
        if (sc < sc1) {
            const int a = d.chi_a[sc];
            sb = d.chi_b[sc];
            se = d.chi_end[sc];
            const T inv = reinterpret_cast<const T*>(d.chi_inv)[sc];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                sA[k] = rr[3 * a + k];
                sU[k] = mul(sub(rr[3 * sb + k], sA[k]), inv);
            }
        }
    }
    // energies of the thread's atoms (Coulomb, LJ, cavity) for the chain cc: FP64 mode / mixed mode
    double E[3] = {0.0, 0.0, 0.0};
    float Ef[3] = {0.0f, 0.0f, 0.0f};
    int cc = -1;
    // per-atom counters of the pair and solvation kernels: pairs, guard re-decisions, overlap tests,
    // list entries; the largest list
    unsigned long long cnt[4] = {0ULL, 0ULL, 0ULL, 0ULL};
    int mxn = 0;
    for (int a = a0 + threadIdx.x; a < a1; a += blockDim.x) {
        T f[3];
        const int ca = atom_chain(d, a);
        if (ca != cc) {  // the thread's atoms move on to the next chain
            if (cc >= 0) {
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    if constexpr (DF) { if (Ef[k] != 0.0f) atomicAdd(&d.chain_E[3 * cc + k], (double)Ef[k]); }
                    else { if (E[k] != 0.0) atomicAdd(&d.chain_E[3 * cc + k], E[k]); }
                    E[k] = 0.0;
                    Ef[k] = 0.0f;
                }
            }
        }
        cc = ca;
        if (!d.pair_tile) {  // the cell-pair tile kernel adds its energies and counters to the totals itself
            if constexpr (DF) {
                const float2 ep = reinterpret_cast<const float2*>(d.epair)[a];
                Ef[0] += ep.x;
                Ef[1] += ep.y;
            } else {
                const double2 ep = reinterpret_cast<const double2*>(d.epair)[a];
                E[0] += ep.x;
                E[1] += ep.y;
            }
            const int2 ps = d.pstat[a];
            cnt[0] += ps.x;
            cnt[1] += ps.y;
        }
        if (d.prm.solvation) {
            const int2 ss = d.sstat[a];
            const int nl = d.nbr_cnt[a];
            cnt[1] += ss.y;
            cnt[2] += (unsigned)ss.x;
            cnt[3] += nl;
            mxn = max(mxn, nl);
        }
        if constexpr (DF) {  // pair forces in fixed point (2^-23) plus oversized terms, solvation (2^-40)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                f[k] = add(ldexp2(df_from_i64(d.Fpx[3 * a + k]), 0x1p-23f), df{d.Fov[3 * a + k], 0.0f});
                if (d.prm.solvation) f[k] = add(f[k], ldexp2(df_from_i64(d.Fcav[3 * a + k]), 0x1p-40f));
            }
            if (d.prm.solvation == 2) Ef[2] += (float)d.esolv[a];  // pairwise surrogate: gamma_i A_i
            else if (d.prm.solvation && d.gflag[a])  // G^cav_i = G0_i f_i, f_i = 1 - covered_i / N (Sec. 3.4)
                Ef[2] += d.G0f[a] * (1.0f - (float)d.covered[a] * d.f_invN);
        } else {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                f[k] = d.Fpair[3 * a + k];
                if (d.prm.solvation) f[k] += (double)d.Fcav[3 * a + k] * kFxInv;
            }
            if (d.prm.solvation == 2) {
                E[2] += d.esolv[a];
            } else if (d.prm.solvation) {
                const double G0a = d.G0[a];
                if (G0a != 0.0) E[2] += G0a - G0a * (double)d.covered[a] / (double)d.N;
            }
        }
        const T x = rr[3 * a], y = rr[3 * a + 1], z = rr[3 * a + 2];
        T* v = sV[a - a0];
        v[0] = sub(mul(y, f[2]), mul(z, f[1]));
        v[1] = sub(mul(z, f[0]), mul(x, f[2]));
        v[2] = sub(mul(x, f[1]), mul(y, f[0]));
        v[3] = f[0]; v[4] = f[1]; v[5] = f[2];
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {  // energies of the block's atoms, per chain
        if constexpr (DF) chain_add(d.chain_E + k, 3, cc, Ef[k]);
        else chain_add(d.chain_E + k, 3, cc, E[k]);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) cnt[k] = warp_sum(cnt[k]);
    mxn = __reduce_max_sync(0xffffffffu, mxn);
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) sSt[w][k] = cnt[k];
        sMx[w] = mxn;
    }
    __syncthreads();
    if (threadIdx.x == 0) {  // the block's counters: one atomic each
        unsigned long long s[4] = {0ULL, 0ULL, 0ULL, 0ULL};
        int m = 0;
        for (int q = 0; q < kWrenchWarps; ++q) {
            for (int k = 0; k < 4; ++k) s[k] += sSt[q][k];
            m = max(m, sMx[q]);
        }
        if (s[0]) atomicAdd(&st->pairs, s[0]);
        if (s[1]) atomicAdd(&st->guard, s[1]);
        if (s[2]) atomicAdd(&st->sasa_tests, s[2]);
        if (s[3]) atomicAdd(&st->nbr_total, s[3]);
        if (m) atomicMax(&st->max_nbr, m);
    }
    for (int u = threadIdx.x; u < 6 * 32; u += blockDim.x) {  // P_h component u / 32 of link h0 + u % 32
        const int k = u >> 5, h = h0 + (u & 31);
        T s = num_f<T>(0.0f);
        if (h < h1 && !(d.lflag[h] & 1))  // a chain's base link has no joint
            for (int a = d.link_start[h]; a < d.link_start[h + 1]; ++a) s = add(s, sV[a - a0][k]);
        sP[u & 31][k] = s;
    }
    // side-chain joints of the tile's links: the branch sums of Sec. 3.5 over the side atoms each one
    // moves, tau = u . (sum_s r_s x F_s - a x sum_s F_s) from the atoms' r x F and F above (the bond
    // and its atoms were loaded at the start)
    if (SIDE && sc < sc1) {
        T S[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) S[k] = num_f<T>(0.0f);
        for (int s = sb + 1; s < se; ++s)
#pragma unroll
            for (int k = 0; k < 6; ++k) S[k] = add(S[k], sV[s - a0][k]);
        const T mx = sub(S[0], sub(mul(sA[1], S[5]), mul(sA[2], S[4])));
        const T my = sub(S[1], sub(mul(sA[2], S[3]), mul(sA[0], S[5])));
        const T mz = sub(S[2], sub(mul(sA[0], S[4]), mul(sA[1], S[3])));
        d.tau[d.l + sc] = to_double(add(add(mul(sU[0], mx), mul(sU[1], my)), mul(sU[2], mz)));
    }
    __syncthreads();
    T* lane_suf = reinterpret_cast<T*>(d.lane_suf);
    T* tileS = reinterpret_cast<T*>(d.tileS);
    if (w < 6) {  // segmented reverse inclusive scan of component w over the tile
        const int h = h0 + lane;
        T x = sP[lane][w];
        bool tl = h >= d.L - 1 || (h < h1 && (d.lflag[h] & 2));  // last link of a chain
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const T y = shfl_down(x, off);
            const bool yt = __shfl_down_sync(0xffffffffu, tl, off);
            if (lane + off < 32 && !tl) { x = add(x, y); tl = yt; }
        }
        if (h < d.L) {
            lane_suf[6 * (size_t)h + w] = x;
            if (w == 0) d.ltail[h] = (unsigned char)tl;  // a chain ends in the tile at or after h
        }
        if (lane == 0) {
            tileS[6 * (size_t)t + w] = x;
            if (w == 0) d.tileT[t] = tl;
        }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&st->ticket_w, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    T* tileSuf = reinterpret_cast<T*>(d.tileSuf);
    if (w < 6) {  // segmented exclusive suffix sums of the tile totals
        if (d.ltiles <= 64) tile_suffix<1>(d, tileSuf, w, lane);
        else tile_suffix<8>(d, tileSuf, w, lane);
    }
    if (threadIdx.x == 0) st->ticket_w = 0u;
}

// the last block of the step: close the iteration of every chain that took a step
__device__ __forceinline__ void close_iteration(const DevChain& d, Status* st) {
    __shared__ int s_run;
    __shared__ unsigned long long s_dm;
    if (d.nchains == 1) {  // one chain: one thread closes it, with every load issued before any store
        if (threadIdx.x == 0) {
            const unsigned long long m = __ldcg(&d.chain_maxdt[0]);
            const int err = __ldcg(&st->error), done0 = __ldcg(&d.chain_done[0]);
            const int it0 = __ldcg(&d.chain_iters[0]), maxit = __ldcg(&d.chain_maxit[0]), sit = __ldcg(&st->iters);
            d.chain_maxdt[0] = 0ULL;
            d.chain_maxtau[0] = 0ULL;
            bool done = done0 != 0;
            if (!err && !done) {
                const double mc = __longlong_as_double((long long)m);
                d.chain_lastdt[0] = mc;
                d.chain_iters[0] = it0 + 1;
                st->last_max_dtheta = mc;
                st->iters = sit + 1;
                if (mc < d.prm.conv_tol || it0 + 1 >= maxit) {
                    d.chain_done[0] = 1;
                    done = true;
                }
            }
            if (err || done) st->done = 1;
            st->ticket = 0u;
        }
        return;
    }
    if (threadIdx.x == 0) { s_run = 0; s_dm = 0ULL; }
    __syncthreads();
    int run = 0;
    unsigned long long dm = 0ULL;
    for (int c = threadIdx.x; c < d.nchains; c += blockDim.x) {
        const unsigned long long m = __ldcg(&d.chain_maxdt[c]);
        d.chain_maxdt[c] = 0ULL;
        d.chain_maxtau[c] = 0ULL;
        if (__ldcg(&d.chain_err[c])) d.chain_done[c] = 1;  // a failed chain stops; the others go on
        if (d.chain_done[c]) continue;
        const double mc = __longlong_as_double((long long)m);
        d.chain_lastdt[c] = mc;
        const int it = d.chain_iters[c] + 1;
        d.chain_iters[c] = it;
        dm = max(dm, m);
        if (mc < d.prm.conv_tol || it >= d.chain_maxit[c]) d.chain_done[c] = 1;  // converged or out of iterations
        else ++run;
    }
    if (run) atomicAdd(&s_run, run);
    if (dm) atomicMax(&s_dm, dm);
    __syncthreads();
    if (threadIdx.x == 0) {
        st->last_max_dtheta = __longlong_as_double((long long)s_dm);
        st->iters += 1;
        if (s_run == 0) st->done = 1;  // every chain converged, reached its cap or failed
        st->ticket = 0u;
    }
}

// tau_k from P^agg (main-chain joints; the side-chain joints after them have theirs from the wrench
// kernel); with STEP the clamped step of the chains still running and the end of the iteration
template <bool STEP, class T>
__global__ void __launch_bounds__(128) k_torque(const DevChain d) {
    constexpr bool DF = std::is_same<T, df>::value;
    __shared__ bool last;
    Status* st = d.status;
    if (st->done) return;
    const int jj = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long adt = 0ULL, atau = 0ULL;  // bit patterns of non-negative doubles
    bool bad = false;
    int cj = -1;
    if (jj < d.l + d.ls) {
        double t;
        if (jj < d.l) {
            cj = joint_chain(d, jj);
            const int h = jj + cj + 1, tile = h >> 5;  // joint jj moves links h .. the chain's last link
            const T* ls = reinterpret_cast<const T*>(d.lane_suf);
            const T* ts = reinterpret_cast<const T*>(d.tileSuf);
            const bool own = d.ltail[h] != 0;  // the chain ends within this tile
            T A[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) A[k] = own ? ls[6 * (size_t)h + k] : add(ls[6 * (size_t)h + k], ts[6 * (size_t)tile + k]);
            const T* u = reinterpret_cast<const T*>(DF ? d.ucurdf : d.ucur) + 3 * jj;
            const T* p = reinterpret_cast<const T*>(DF ? d.pcurdf : d.pcur) + 3 * jj;
            const T px = sub(mul(p[1], u[2]), mul(p[2], u[1]));
            const T py = sub(mul(p[2], u[0]), mul(p[0], u[2]));
            const T pz = sub(mul(p[0], u[1]), mul(p[1], u[0]));
            const T tt = add(add(add(mul(u[0], A[0]), mul(u[1], A[1])), add(mul(u[2], A[2]), mul(px, A[3]))),
                             add(mul(py, A[4]), mul(pz, A[5])));
            t = to_double(tt);
        } else {
            cj = atom_chain(d, d.chi_b[jj - d.l]);
            t = d.tau[jj];  // formed by the wrench kernel
        }
        d.tau[jj] = t;
        bad = !isfinite(t);
        if (bad) atomicOr(&d.chain_err[cj], kErrNonfinite);
        const bool fx = d.jfixed[jj] != 0;  // a fixed joint takes no step and has no say in max |tau|
        atau = fx ? 0ULL : (unsigned long long)__double_as_longlong(fabs(t));
        if (d.chain_done[cj] || d.chain_err[cj]) {
            cj = -1;  // a converged or failed chain takes no more steps
        } else if (STEP && !bad) {
            const double dt = fx ? 0.0 : fmin(fmax(d.prm.kappa * t, -d.prm.dtheta_max), d.prm.dtheta_max);
            if (!fx) d.theta[jj] += dt;
            d.dtheta[jj] = dt;
            adt = (unsigned long long)__double_as_longlong(fabs(dt));
        }
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&st->error, kErrNonfinite);
    chain_max(d.chain_maxtau, cj, atau);
    if (!STEP) return;
    chain_max(d.chain_maxdt, cj, adt);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&st->ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    close_iteration(d, st);
}

// the paper's normalised step (eq. KCM_07): dtheta_k = kappa tau_k / max |tau| over the free joints of
// the joint's chain, main and side (a fixed joint takes none)
__global__ void __launch_bounds__(128) k_step_normalized(const DevChain d) {
    __shared__ bool last;
    Status* st = d.status;
    if (st->done) return;
    const int jj = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long adt = 0ULL;
    int cj = -1;
    if (jj < d.l + d.ls && !st->error) {
        cj = jj < d.l ? joint_chain(d, jj) : atom_chain(d, d.chi_b[jj - d.l]);
        if (d.chain_done[cj]) {
            cj = -1;
        } else {
            const double tm = __longlong_as_double((long long)__ldcg(&d.chain_maxtau[cj]));
            const double dt = (tm > 0.0 && !d.jfixed[jj]) ? d.prm.kappa * d.tau[jj] / tm : 0.0;
            d.theta[jj] += dt;
            d.dtheta[jj] = dt;
            adt = (unsigned long long)__double_as_longlong(fabs(dt));
        }
    }
    chain_max(d.chain_maxdt, cj, adt);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&st->ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    close_iteration(d, st);
}

}  // namespace

template <class T>
void launch_wrench(DevChain& d, cudaStream_t s) {
    if (d.ls) k_wrench_tile<T, true><<<d.ltiles, kWrenchWarps * 32, 0, s>>>(d);
    else k_wrench_tile<T, false><<<d.ltiles, kWrenchWarps * 32, 0, s>>>(d);
}

void launch_torques(DevChain& d, cudaStream_t s) {
    if (d.prm.precision == KCM_MIXED) {
        launch_wrench<df>(d, s);
        k_torque<false, df><<<(d.l + d.ls + 127) / 128, 128, 0, s>>>(d);
    } else {
        launch_wrench<double>(d, s);
        k_torque<false, double><<<(d.l + d.ls + 127) / 128, 128, 0, s>>>(d);
    }
}

template <class T>
void launch_torques_step_t(DevChain& d, cudaStream_t s) {
    launch_wrench<T>(d, s);
    if (d.prm.step_mode == KCM_STEP_CLAMP) {
        k_torque<true, T><<<(d.l + d.ls + 127) / 128, 128, 0, s>>>(d);
    } else {
        k_torque<false, T><<<(d.l + d.ls + 127) / 128, 128, 0, s>>>(d);
        k_step_normalized<<<(d.l + d.ls + 127) / 128, 128, 0, s>>>(d);
    }
}

// torques plus the step of one iteration (the evaluation kernels must already be enqueued)
void launch_torques_step(DevChain& d, cudaStream_t s) {
    if (d.prm.precision == KCM_MIXED) launch_torques_step_t<df>(d, s);
    else launch_torques_step_t<double>(d, s);
}

}  // namespace kcm
