// A7-A9: link wrenches, suffix sums over links, joint torques and the kinetostatic step: FP64 in
// FP64 mode, double-float (kcm_df.cuh) in mixed mode; the step itself updates theta in FP64. The
// kernel visits every atom once with one thread each, so it also converts the mixed-mode fixed-point
// forces, adds the cavity energy G0_i f_i (and the warp-per-atom pair kernel's pair energies) of its
// atoms per chain, and totals the per-atom counters of the pair and solvation kernels.
//
// Wrench of link h about the origin, P_h = [sum r x F ; sum F] (eq. KCM_01/02), and
// P^agg_k = sum_{h >= k} P_h (Sec. 3.5) as a reverse scan, then tau_k = u_k . T^agg_k +
// (p_k x u_k) . F^agg_k (eq. KCM_05/06) and, in the clamped step mode, dtheta_k = clamp(kappa tau_k,
// +-dtheta_max) (eq. KCM_07), all in one kernel (k_wrench_step): a block per tile of 32 links forms
// the tile's P_h and their in-tile suffix sums, publishes the tile's total, sums the totals of the
// later tiles of its chain (published by blocks that took them earlier: tiles are handed out from the
// last one down, so a block only waits for blocks already running), and takes the tile's torques and
// steps; the last block to finish closes the iteration. Each block sums the later totals itself, in a
// fixed order, rather than taking a running prefix from whichever later block finished first, so the
// result does not depend on timing: the torques stay bitwise reproducible. Every wait is bounded: a
// block that waits too long sets the timeout error, and the kernel ends without torques.
#include <cuda_runtime.h>

#include <type_traits>

#include "kcm_common.cuh"
#include "kcm_df.cuh"
#include "kcm_device.h"
#include "kcm_launch.h"

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

// Waits of k_wrench_step on later tiles' totals poll with a growing pause and give up after kSpinLimit
// polls (about 0.2 s), which sets kErrTimeout: the kernel then ends without torques and the host reads
// KCM_E_TIMEOUT.
constexpr int kSpinLimit = 200000;

__device__ __forceinline__ bool wait_published(const unsigned int* flag, unsigned int want) {
    unsigned ns = 32;
    for (int it = 0; it < kSpinLimit; ++it) {
        if (__ldcg(flag) == want) return true;
        __nanosleep(ns);
        if (ns < 256) ns <<= 1;
    }
    return false;
}

// sum over the warp in a fixed tree (lane 0 holds it)
template <class T>
__device__ __forceinline__ T warp_reduce(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = add(v, shfl_down(v, o));
    return v;
}

// one step of a segmented reverse scan over the 32 lanes (component x, "a chain ends here" flag tl)
template <class T>
__device__ __forceinline__ void reverse_scan32(T& x, bool& tl, int lane) {
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const T y = shfl_down(x, off);
        const bool yt = __shfl_down_sync(0xffffffffu, tl, off);
        if (lane + off < 32 && !tl) { x = add(x, y); tl = yt; }
    }
}

// One block per tile of 32 links h in [32 t, 32 t + 32), the tiles taken from the last one down
// (ticket). The block's threads take the tile's atoms (r x F and F, with the conversion of the
// mixed-mode fixed-point forces) into shared memory; one thread per (component, link) adds the link's
// atoms in atom order; warp q scans component q of the tile's P_h from the end (segmented at the last
// link of each chain: a chain's sums never take in the next chain) and the tile's total is published.
// The block then sums, in a fixed order, the totals of the later tiles up to the first one in which a
// chain ends (rounds of blockDim tiles, a tree within each round), which is the part of P^agg of its
// links that lies beyond the tile, and forms tau, and with STEP the clamped step, of the tile's joints
// (side-chain joints from their branch sums). The last block to finish closes the iteration.
template <class T, bool SIDE, bool STEP>
__global__ void __launch_bounds__(kWrenchWarps * 32) k_wrench_step(const DevChain d) {
    grid_dep_sync();
    constexpr bool DF = std::is_same<T, df>::value;
    __shared__ T sV[kWrenchTileAtoms][6];
    __shared__ T sP[32][6];  // link wrenches, then their in-tile suffix sums
    __shared__ bool sTL[32];  // a chain ends in the tile at or after the link
    __shared__ T sW[kWrenchWarps][6];
    __shared__ T sSuf[6];
    __shared__ unsigned long long sSt[kWrenchWarps][4];
    __shared__ int sMx[kWrenchWarps];
    __shared__ int sTile, sEnd;
    __shared__ unsigned int sEpoch;
    __shared__ bool sLast, sTimeout;
    Status* st = d.status;
    if (st->done) return;
    if (threadIdx.x == 0) {
        // later tiles first: by ticket, so that a block that waits for later tiles never holds the slot
        // one of them needs; by block index where every block is resident at once
        sTile = d.ltiles - 1 - (d.wrench_static ? (int)blockIdx.x : (int)atomicAdd(&st->ticket_lb, 1u));
        sEpoch = __ldcg(d.lb_epoch) + 1u;
        sTimeout = false;
        sEnd = 0x7fffffff;
    }
    __syncthreads();
    const int t = sTile, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned int epoch = sEpoch;
    double side_tau = 0.0;
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
                f[k] = add(add(ldexp2(df_from_i64(d.Fpx[3 * a + k]), 0x1p-23f), ldexp2(df_from_i64(d.Fox[3 * a + k]), 0.5f)),
                           df{d.Fov[3 * a + k], 0.0f});
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
        side_tau = to_double(add(add(mul(sU[0], mx), mul(sU[1], my)), mul(sU[2], mz)));
    }
    __syncthreads();
    T* tileS = reinterpret_cast<T*>(d.tileS);
    if (w < 6) {  // segmented reverse inclusive scan of component w over the tile
        const int h = h0 + lane;
        T x = sP[lane][w];
        bool tl = h >= d.L - 1 || (h < h1 && (d.lflag[h] & 2));  // last link of a chain
        reverse_scan32(x, tl, lane);
        sP[lane][w] = x;  // warp w alone reads and writes column w
        if (w == 0) sTL[lane] = tl;
        if (lane == 0) {
            tileS[6 * (size_t)t + w] = x;
            if (w == 0) d.tileT[t] = tl;
            __threadfence();  // the total before its flag
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && t != d.lb_withhold) atomicExch(&d.tileStat[t], epoch);  // published
    // the joint of link h0 + lane (warp 0): its current axis and point, loaded before the wait
    int jj_l = -1, ch_l = 0;
    T uj[3], pj[3];
    if (w == 0) {
        const int h = h0 + lane;
        if (h < h1 && !(d.lflag[h] & 1)) {  // a chain's base link has no joint
            ch_l = d.nchains == 1 ? 0 : d.link_chain[h];
            jj_l = h - ch_l - 1;  // the joint that moves links h .. the chain's last link
            const T* u = reinterpret_cast<const T*>(DF ? d.ucurdf : d.ucur) + 3 * jj_l;
            const T* p = reinterpret_cast<const T*>(DF ? d.pcurdf : d.pcur) + 3 * jj_l;
#pragma unroll
            for (int k = 0; k < 3; ++k) { uj[k] = u[k]; pj[k] = p[k]; }
        }
    }
    // P^agg beyond the tile: the totals of the later tiles up to the first chain end, in a fixed order
    T acc[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) acc[k] = num_f<T>(0.0f);
    // uniform: needed unless a chain ends at the tile's last link (then no link of the tile reaches past it)
    if (!sTL[h1 - h0 - 1]) {
        // the tile that holds the last link of the chain of the tile's last link (the last link of chain c
        // is joint_off[c + 1] + c): no later tile is waited for, although a round may reach past it
        int te = d.ltiles - 1;
        if (d.nchains > 1) {
            const int ce = d.link_chain[h1 - 1];
            te = (d.joint_off[ce + 1] + ce) >> 5;
        }
        for (int base = t + 1; base < d.ltiles; base += blockDim.x) {  // uniform
            const int tt = base + threadIdx.x;
            T v[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) v[k] = num_f<T>(0.0f);
            bool ends = false;
            if (tt <= te) {
                if (!wait_published(&d.tileStat[tt], epoch)) {
                    sTimeout = true;
                } else {
                    __threadfence();
                    ends = __ldcg(&d.tileT[tt]) != 0;
                    const double* raw = &d.tileS[6 * (size_t)tt];
#pragma unroll
                    for (int k = 0; k < 6; ++k) {
                        const double r = __ldcg(&raw[k]);
                        v[k] = *reinterpret_cast<const T*>(&r);
                    }
                }
            }
            if (ends) atomicMin(&sEnd, tt);
            __syncthreads();
            const int e = sEnd;
            const bool out = sTimeout;
            if (tt > e) {
#pragma unroll
                for (int k = 0; k < 6; ++k) v[k] = num_f<T>(0.0f);
            }
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                const T r = warp_reduce(v[k]);
                if (lane == 0) sW[w][k] = r;
            }
            __syncthreads();
            if (threadIdx.x == 0)
                for (int q = 0; q < kWrenchWarps; ++q)
#pragma unroll
                    for (int k = 0; k < 6; ++k) acc[k] = add(acc[k], sW[q][k]);
            __syncthreads();
            if (out || e != 0x7fffffff) break;  // uniform
        }
    }
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < 6; ++k) sSuf[k] = acc[k];
    __syncthreads();
    // torques (and steps) of the tile's joints: link h's joint from P^agg_h = in-tile suffix (+ the
    // later tiles' part unless its chain ends in the tile), side-chain joints from their branch sums
    unsigned long long atau1 = 0ULL, adt1 = 0ULL, atau2 = 0ULL, adt2 = 0ULL;  // bit patterns of |.|
    int cj1 = -1, cj2 = -1;
    bool bad = false;
    auto step_joint = [&](int jj, int cj, double tq, int& cjo, unsigned long long& atau, unsigned long long& adt) {
        d.tau[jj] = tq;
        const bool nf = !isfinite(tq);
        bad = bad || nf;
        if (nf) atomicOr(&d.chain_err[cj], kErrNonfinite);
        const bool fx = d.jfixed[jj] != 0;  // a fixed joint takes no step and has no say in max |tau|
        atau = fx ? 0ULL : (unsigned long long)__double_as_longlong(fabs(tq));
        cjo = cj;
        if (d.chain_done[cj] || d.chain_err[cj]) {
            cjo = -1;  // a converged or failed chain takes no more steps
        } else if (STEP && !nf) {
            const double dt = fx ? 0.0 : fmin(fmax(d.prm.kappa * tq, -d.prm.dtheta_max), d.prm.dtheta_max);
            if (!fx) set_theta(d, jj, d.theta[jj] + dt);
            d.dtheta[jj] = dt;
            adt = (unsigned long long)__double_as_longlong(fabs(dt));
        }
    };
    if (!sTimeout) {
        if (jj_l >= 0) {
            T A[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) A[k] = sTL[lane] ? sP[lane][k] : add(sP[lane][k], sSuf[k]);
            const T* u = uj;
            const T* p = pj;
            const T px = sub(mul(p[1], u[2]), mul(p[2], u[1]));
            const T py = sub(mul(p[2], u[0]), mul(p[0], u[2]));
            const T pz = sub(mul(p[0], u[1]), mul(p[1], u[0]));
            const T tt = add(add(add(mul(u[0], A[0]), mul(u[1], A[1])), add(mul(u[2], A[2]), mul(px, A[3]))),
                             add(mul(py, A[4]), mul(pz, A[5])));
            step_joint(jj_l, ch_l, to_double(tt), cj1, atau1, adt1);
        }
        if (SIDE && sc < sc1) step_joint(d.l + sc, atom_chain(d, sb), side_tau, cj2, atau2, adt2);
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&st->error, kErrNonfinite);
    chain_max(d.chain_maxtau, cj1, atau1);
    chain_max(d.chain_maxtau, cj2, atau2);
    if (STEP) {
        chain_max(d.chain_maxdt, cj1, adt1);
        chain_max(d.chain_maxdt, cj2, adt2);
    }
    if (threadIdx.x == 0 && sTimeout) atomicOr(&st->error, kErrTimeout);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) sLast = atomicAdd(&st->ticket_w, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!sLast) return;
    __threadfence();
    if (threadIdx.x == 0) {  // every block is done: the next launch takes fresh tickets and flags
        st->ticket_w = 0u;
        st->ticket_lb = 0u;
        *d.lb_epoch = epoch;
    }
    if (STEP) close_iteration(d, st);
    if (threadIdx.x == 0) {
        if (__ldcg(&st->error) & kErrTimeout) st->done = 1;  // a timed-out iteration ends the loop
        export_status(d);  // (the normalised step's kernel exports it again when it closes the iteration)
    }
}

// the paper's normalised step (eq. KCM_07): dtheta_k = kappa tau_k / max |tau| over the free joints of
// the joint's chain, main and side (a fixed joint takes none)
__global__ void __launch_bounds__(128) k_step_normalized(const DevChain d) {
    grid_dep_sync();
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
            set_theta(d, jj, d.theta[jj] + dt);
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
    if (threadIdx.x == 0) export_status(d);
}

}  // namespace

template <class T, bool STEP>
void launch_wrench_step(DevChain& d, cudaStream_t s) {
    if (d.ls) launch_k(k_wrench_step<T, true, STEP>, d.ltiles, kWrenchWarps * 32, 0, s, d.pdl, d);
    else launch_k(k_wrench_step<T, false, STEP>, d.ltiles, kWrenchWarps * 32, 0, s, d.pdl, d);
}

// the fewest resident blocks per SM over the wrench kernel's forms (their resources differ a little)
int wrench_resident_blocks(const DevChain& d) {
    int best = 1 << 30;
    auto q = [&](auto kernel) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, kWrenchWarps * 32, 0) != cudaSuccess) nb = -1;
        best = std::min(best, nb);
    };
    if (d.prm.precision == KCM_MIXED) {
        q(k_wrench_step<df, false, false>); q(k_wrench_step<df, false, true>);
        q(k_wrench_step<df, true, false>); q(k_wrench_step<df, true, true>);
    } else {
        q(k_wrench_step<double, false, false>); q(k_wrench_step<double, false, true>);
        q(k_wrench_step<double, true, false>); q(k_wrench_step<double, true, true>);
    }
    return best;
}

void launch_torques(DevChain& d, cudaStream_t s) {
    if (d.prm.precision == KCM_MIXED) launch_wrench_step<df, false>(d, s);
    else launch_wrench_step<double, false>(d, s);
}

template <class T>
void launch_torques_step_t(DevChain& d, cudaStream_t s) {
    if (d.prm.step_mode == KCM_STEP_CLAMP) {
        launch_wrench_step<T, true>(d, s);
    } else {
        launch_wrench_step<T, false>(d, s);
        launch_k(k_step_normalized, (d.l + d.ls + 127) / 128, 128, 0, s, d.pdl, d);
    }
}

// torques plus the step of one iteration (the evaluation kernels must already be enqueued)
void launch_torques_step(DevChain& d, cudaStream_t s) {
    if (d.prm.precision == KCM_MIXED) launch_torques_step_t<df>(d, s);
    else launch_torques_step_t<double>(d, s);
}

}  // namespace kcm
