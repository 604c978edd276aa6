// Cell-pair tile kernel of the mixed-precision pair forces (A3-A5): Coulomb with the distance-dependent
// dielectric and Lennard-Jones (eq. 02_2, 03_2, weighted by eq. 03_8 / 03_9), exclusions (Sec. 3.3)
// and the solvation neighbour lists A'_i (Sec. 3.2), over the uniform grid of Sec. 3.2.
//
// Work unit: 32 consecutive sorted slots (home atoms, one per lane) against one x-row of their half
// stencil (the home row from the home atoms onward, the rows dy > 0 of their plane and the rows of the
// planes dz > 0), so each unordered pair within range is met once (Newton's third law). Slots are
// ordered by cell, so the 32 atoms lie in a few runs of cells along x; each run (a segment of one grid
// row) is one home tile whose candidates are the row's cells from its first cell's x index - KR to its
// last one's + KR. A warp owns one stencil row and one window of 32 slots (the set-up of its segments
// runs on one lane each, in parallel). The candidates are staged 32 at a time in shared memory as float4
// cell offsets and float4 constants (the next 32 are loaded while these are evaluated), and every lane
// tests its home atom against them from shared memory (a broadcast read per test). The in-range pairs of
// a 32 x 32 tile are compacted into a queue and evaluated with every lane busy. Each pair term is added
// to both atoms as exact fixed-point pieces (units of 2^-23, fx_pieces) with shared-memory integer
// atomics into per-tile sums; a tile's sums go to the global fixed-point forces with one 64-bit integer
// add per atom and tile instead of one per pair. The integer sums do not depend on the order of the
// terms, so the forces are bitwise those of every other evaluation order (the warp-per-atom kernel's
// among them). The solvation pairs of a tile are counted per atom with shared counters; one global
// reservation per atom and tile then gives the list slots, which the entries take in turn, so no global
// atomic waits inside the pair loop. Home atoms that a short segment leaves idle are replaced by copies:
// with H home atoms (rounded up to a power of two) the 32 / H lane groups each test a different part of
// the staged row.
#include <cuda_runtime.h>

#include "kcm_common.cuh"
#include "kcm_device.h"
#include "kcm_launch.h"

namespace kcm {

namespace {
using namespace dev;

constexpr int kPtWarps = 1;           // warps (independent work units) per block: one, so that a
                                      // finished warp's slot takes the next unit at once (with four, a
                                      // block held its slots until its slowest unit ended: chain8000
                                      // pairs 170 -> 145 us, batch 2.05 -> 1.61 ms)
constexpr int kPtQueue = 32 * 32;     // in-range pairs of one tile at most
constexpr int kPtFlushChunks = 8;     // staged rows between flushes of the home sums: 8 x 32 pieces of
                                      // |.| <= 2^22 stay within int32
constexpr float kPtFilterPad = 0.02f; // A^2 added to the filter's squared range: its rounded shifted
                                      // offsets differ from the exact ones by ~1e-5 A at most
// queue entry: staged index (bits 0-4), home index (5-9); the evaluation sets bit 10 for a solvation pair
constexpr unsigned kQNear = 1u << 10;
#ifndef KCM_PT_MIN_BLOCKS
#define KCM_PT_MIN_BLOCKS 28  // resident blocks per SM the register budget is set for (72 registers;
                              // shared memory allows 25 blocks of 8 KB)
#endif

// one warp's shared memory
struct PtSmem {
    float4 hpos[32];       // home atoms: cell offsets, cell x index
    float4 hprm[32];       // charge, sqrt(eps), R, Roff
    ulonglong2 hmask[32];  // bond-class masks
    int hatom[32];
    float4 jpos[32];       // staged row: cell offsets and the exact x shift (cx_j - cx_home) s
    float4 jfxy[16];       // the filter's copy, shifted into the frame of the segment's first cell, rounded
    float2 jfz[16];        // and negated, packed by pairs of staged atoms: (x_t, x_t+1, y_t, y_t+1), (z_t, z_t+1)
    float4 jprm[32];
    ulonglong2 jmask[32];
    int jatom[32];
    int iacc[6][32];       // fixed-point sums of the home atoms: integer parts x, y, z, then fractions
    int jacc[6][32];       // of the staged atoms (their negated terms)
    int icnt[32], jcnt[32];    // solvation-list entries of the chunk per home / staged atom
    int ibase[32], jbase[32];  // their first list slots, reserved once per chunk
    int iput[32], jput[32];    // entries written so far (each entry takes the next reserved slot)
    unsigned short queue[kPtQueue];  // in-range pairs (kQNear layout)
};

// SPLIT warps share one window and stencil row: warp s takes staged rows s, s + SPLIT, ... (more and
// shorter warps for small workloads; chosen by the tile autotuner)
template <int KR, int SPLIT>
__global__ void __launch_bounds__(kPtWarps * 32, KCM_PT_MIN_BLOCKS) k_pair_tile(const DevChain d) {
    grid_dep_sync();
    constexpr int kW = 2 * KR + 1;
    constexpr int kRows = 1 + KR + KR * kW;  // rows of the half stencil
    __shared__ PtSmem smem[kPtWarps];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    PtSmem& S = smem[w];
    const long long gw = (long long)blockIdx.x * kPtWarps + w;
    const int part = (int)(gw % SPLIT);
    const int win = (int)(gw / (SPLIT * kRows)), row = (int)((gw / SPLIT) % kRows);
    const int s0 = win * 32;
    if (s0 >= d.n || d.status->done) return;  // whole warps: no block-wide barrier in this kernel

    // the row's position in the half stencil: (dy, dz) and the lowest x offset
    int dyc, dzc, dxlo = -KR;
    if (row == 0) { dyc = 0; dzc = 0; dxlo = 0; }
    else if (row <= KR) { dyc = row; dzc = 0; }
    else { const int rr = row - 1 - KR; dyc = rr % kW - KR; dzc = 1 + rr / kW; }
    const float rall2 = d.f_rall2;

    // Set-up, one lane per slot of the window, all in parallel: the slot's cell, chain and grid; the
    // window splits into segments of one grid row each (same chain, y and z cell index; slots are ordered
    // by cell, so a segment's cells run from its first slot's x index to its last slot's)
    const int sl = s0 + lane;
    const bool valid = sl < d.n;
    int key = 0, ca = 0, cx = 0, cy = 0, cz = 0, nx = 1, ny = 1, nz = 1, cbase = 0;
    float sf = 0.0f, gpf = 0.0f;
    bool done = true;
    if (valid) {
        key = d.slot_cell[sl];
        ca = slot_chain(d, sl);
        done = d.chain_done[ca] != 0;
        const GridInfo* gp = &d.grid[ca];
        nx = gp->nx; ny = gp->ny; nz = gp->nz; cbase = gp->cbase;
        sf = gp->sf;
        gpf = gp->gpf;
        const int cell = key - cbase;
        cx = cell % nx;
        cy = (cell / nx) % ny;
        cz = cell / (nx * ny);
    }
    const int rowkey = valid ? key - cx : -1;  // the grid row's first cell (global numbering)
    const int prevkey = __shfl_up_sync(0xffffffffu, rowkey, 1);
    const unsigned segs = __ballot_sync(0xffffffffu, valid && (lane == 0 || rowkey != prevkey));
    // the segment of a first lane ends before the next first lane (or at the window's last valid slot)
    const unsigned later = lane == 31 ? 0u : segs & (0xffffffffu << (lane + 1));
    const int nvalid = min(32, d.n - s0);
    const int seg_end = later ? __ffs(later) - 1 : nvalid;  // one past the segment's last lane
    const int cxb = __shfl_sync(0xffffffffu, cx, max(seg_end - 1, 0));
    // a first lane: the slot range of this warp's stencil row over the segment's cells, trimmed to the cells
    // within reach of the segment's box (gaps of whole cells, less a margin over the FP32 cell assignment)
    int jrow = 0, jend = 0;
    bool ok = false;
    if (((segs >> lane) & 1u) && !done) {
        const int ncy = cy + dyc, ncz = cz + dzc;
        auto gapc = [&](int k) { return fmaxf((float)(abs(k) - 1) * sf - 0.02f, 0.0f); };
        const float gy = gapc(dyc), gz = gapc(dzc);
        const float rem = rall2 - (gy * gy + gz * gz);
        if (ncy >= 0 && ncy < ny && ncz >= 0 && ncz < nz && rem >= 0.0f) {
            int xlo = max(cx + dxlo, 0), xhi = min(cxb + KR, nx - 1);
#pragma unroll
            for (int k = 2; k <= KR; ++k) {
                const float gk = gapc(k);
                if (gk * gk > rem) {
                    if (dxlo < 0) xlo = max(xlo, cx - k + 1);
                    xhi = min(xhi, cxb + k - 1);
                }
            }
            if (xlo <= xhi) {
                const int rb = cbase + (ncz * ny + ncy) * nx;
                jend = d.cell_start[rb + xhi + 1];
                jrow = row == 0 ? sl : d.cell_start[rb + xlo];  // home row: from the segment's atoms on
                ok = jrow < jend;
            }
        }
    }
    const unsigned tiles = __ballot_sync(0xffffffffu, ok);
    if (!tiles) return;

    const float K = d.f_K, w14e = d.f_w14e, w14v = d.f_w14v, rc2 = d.f_rc2, rv2 = d.f_rv2;
    const float fr2 = rall2 + kPtFilterPad, dr = d.f_dr, pad = 0.01f;
    const bool solv = d.prm.solvation != 0;

    // per-lane totals of the current chain: energies (FP32), pairs, guard-band re-decisions, overflow
    float ove = 0.0f, ovv = 0.0f;
    unsigned npairs = 0, nguard = 0;
    bool ovf = false;
    int cur = -1;
    auto flush_chain = [&]() {  // uniform
        const float Ee = warp_sum(ove), Ev = warp_sum(ovv);
        const unsigned np = __reduce_add_sync(0xffffffffu, npairs), ng = __reduce_add_sync(0xffffffffu, nguard);
        const bool of = __any_sync(0xffffffffu, ovf);
        if (lane == 0) {
            if (Ee != 0.0f) atomicAdd(&d.chain_E[3 * cur], (double)Ee);
            if (Ev != 0.0f) atomicAdd(&d.chain_E[3 * cur + 1], (double)Ev);
            if (np) atomicAdd(&d.status->pairs, (unsigned long long)np);
            if (ng) atomicAdd(&d.status->guard, (unsigned long long)ng);
            if (of) {
                atomicOr(&d.status->error, kErrOverflow);
                atomicOr(&d.chain_err[cur], kErrOverflow);
            }
        }
        ove = ovv = 0.0f;
        npairs = nguard = 0;
        ovf = false;
    };
    // reserves `c` list slots of atom a (c > 0): the first one, overflow, and the long-list record (the
    // reservation that holds slot kSasaStage is unique)
    auto reserve = [&](int a, int c) -> int {
        const int base = atomicAdd(&d.nbr_cnt[a], c);
        ovf |= base + c > kMaxNbr;
        if (base <= kSasaStage && kSasaStage < base + c) d.long_atoms[atomicAdd(&d.status->nlong, 1)] = a;
        return base;
    };

    for (unsigned m = tiles; m; m &= m - 1) {  // uniform: the segments with work in this row
        const int b0 = __ffs(m) - 1;
        const int h0 = s0 + b0;
        const int hn = __shfl_sync(0xffffffffu, seg_end, b0) - b0;
        const int tca = __shfl_sync(0xffffffffu, ca, b0);
        const int tjb = __shfl_sync(0xffffffffu, jrow, b0), tjend = __shfl_sync(0xffffffffu, jend, b0);
        const float fcxa = (float)__shfl_sync(0xffffffffu, cx, b0);  // the segment's first cell x index
        const float tsf = __shfl_sync(0xffffffffu, sf, b0), tgp = __shfl_sync(0xffffffffu, gpf, b0);
        if (tca != cur) {
            if (cur >= 0) flush_chain();
            cur = tca;
        }
        const float shy = __fmul_rn((float)dyc, tsf), shz = __fmul_rn((float)dzc, tsf);
        const int H = hn <= 1 ? 1 : 1 << (32 - __clz(hn - 1));  // power of two >= hn
        const int lgH = __ffs(H) - 1;
        const int hi = lane & (H - 1), gi = lane >> lgH;  // home atom and lane group
        const int isl = h0 + hi;
        // the first staged row's loads, issued before the home atoms' so that both are in flight
        float4 np4 = make_float4(0.f, 0.f, 0.f, 0.f), nq4 = np4;
        ulonglong2 nm = make_ulonglong2(0ULL, 0ULL);
        int na = 0;
        auto fetch = [&](int jc) {
            if (jc + lane < tjend) {
                np4 = d.spos32[jc + lane];
                nq4 = d.sprm32[jc + lane];
                nm = d.smask[jc + lane];
                na = d.sorted[jc + lane];
            }
        };
        const int jfirst = tjb + 32 * part;
        if (jfirst >= tjend) continue;  // uniform: no staged row of this part
        fetch(jfirst);
        // home atoms: the filter's copy of the offsets in the frame of the segment's first cell
        float px = 0.0f, py = 0.0f, pz = 0.0f;
        if (hi < hn) {
            const float4 p = d.spos32[isl];
            px = __fadd_rn(p.x, __fmul_rn(__fsub_rn(p.w, fcxa), tsf));
            py = p.y;
            pz = p.z;
            if (gi == 0) {
                S.hpos[hi] = p;
                S.hprm[hi] = d.sprm32[isl];
                S.hmask[hi] = d.smask[isl];
                S.hatom[hi] = d.sorted[isl];
            }
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) S.iacc[k][lane] = 0;
        // the home atoms' sums to the global fixed-point forces (lanes of the first group)
        auto flush_home = [&]() {
            if (gi == 0 && hi < hn) {
                const int a = S.hatom[hi];
                unsigned long long* Fa = reinterpret_cast<unsigned long long*>(&d.Fpx[3 * a]);
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const long long v = fx_units(S.iacc[k][hi], S.iacc[3 + k][hi]);
                    S.iacc[k][hi] = 0;
                    S.iacc[3 + k][hi] = 0;
                    if (v) atomicAdd(Fa + k, (unsigned long long)v);
                }
            }
        };
        int nchunk = 0;
        for (int jc = jfirst; jc < tjend; jc += 32 * SPLIT) {  // the row staged 32 atoms at a time
            const int jn = min(32, tjend - jc);
            {
                // the filter's copy (lanes beyond jn: far away, never in range)
                const float fx = lane < jn ? __fadd_rn(np4.x, __fmul_rn(__fsub_rn(np4.w, fcxa), tsf)) : 1e30f;
                const float fy = __fadd_rn(np4.y, shy), fz = __fadd_rn(np4.z, shz);
                const float ox = __shfl_xor_sync(0xffffffffu, fx, 1), oy = __shfl_xor_sync(0xffffffffu, fy, 1),
                            oz = __shfl_xor_sync(0xffffffffu, fz, 1);
                if (!(lane & 1)) {  // negated: the filter adds them
                    S.jfxy[lane >> 1] = make_float4(-fx, -ox, -fy, -oy);
                    S.jfz[lane >> 1] = make_float2(-fz, -oz);
                }
            }
            if (lane < jn) {
                S.jpos[lane] = np4;  // cell offsets and the cell's x index
                S.jprm[lane] = nq4;
                S.jmask[lane] = nm;
                S.jatom[lane] = na;
            }
#pragma unroll
            for (int k = 0; k < 6; ++k) S.jacc[k][lane] = 0;
            S.icnt[lane] = 0;
            S.jcnt[lane] = 0;
            S.iput[lane] = 0;
            S.jput[lane] = 0;
            __syncwarp();
            if (jc + 32 * SPLIT < tjend) fetch(jc + 32 * SPLIT);  // the next staged row, in flight during this one
            // filter: lane (hi, gi) tests home atom hi against staged atoms gi H .. gi H + H - 1, two at a
            // time with packed FP32 pairs (staged atoms beyond jn sit at 1e30 and fail)
            unsigned mask = 0;
            if (hi < hn) {
                const int j0 = gi * H;
                if (H == 1) {
                    const float4 q = S.jfxy[j0 >> 1];
                    const float2 qz = S.jfz[j0 >> 1];
                    const float dx = px + ((j0 & 1) ? q.y : q.x), dy = py + ((j0 & 1) ? q.w : q.z),
                                dz = pz + ((j0 & 1) ? qz.y : qz.x);
                    mask = dx * dx + dy * dy + dz * dz <= fr2;
                } else {
                    const float2 p2x = make_float2(px, px), p2y = make_float2(py, py), p2z = make_float2(pz, pz);
                    const int np2 = min(H, jn - j0 + 1) >> 1;  // pairs holding a staged atom below jn
#pragma unroll 4
                    for (int t2 = 0; t2 < np2; ++t2) {
                        const float4 q = S.jfxy[(j0 >> 1) + t2];
                        const float2 qz = S.jfz[(j0 >> 1) + t2];
                        const float2 dx = __fadd2_rn(p2x, make_float2(q.x, q.y));
                        const float2 dy = __fadd2_rn(p2y, make_float2(q.z, q.w));
                        const float2 dz = __fadd2_rn(p2z, qz);
                        const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
                        mask |= ((unsigned)(r2.x <= fr2) | ((unsigned)(r2.y <= fr2) << 1)) << (2 * t2);
                    }
                }
                if (row == 0) {  // home row: only staged slots after the home atom's
                    const int jmin = isl - jc - j0;  // bit t is slot jc + j0 + t
                    if (jmin >= 0) mask &= jmin >= 31 ? 0u : ~0u << (jmin + 1);
                }
            }
            // compaction into the queue, home atom by home atom
            const int c = __popc(mask);
            int incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const int T = __shfl_sync(0xffffffffu, incl, 31);
            {
                int pos = incl - c;
                const unsigned tag = ((unsigned)hi << 5) | (unsigned)(gi * H);
                for (unsigned mm = mask; mm; mm &= mm - 1) S.queue[pos++] = (unsigned short)(tag + (unsigned)(__ffs(mm) - 1));
            }
            __syncwarp();
            // evaluation: lane L takes the queue entries L R .. L R + R - 1, R = ceil(T / 32), so the
            // entries of one round mostly belong to different home atoms
            const int R = (T + 31) >> 5;
            for (int r = 0; r < R; ++r) {
                const int e = lane * R + r;
                if (e >= T) break;
                const unsigned en = S.queue[e];
                const int ih = (int)((en >> 5) & 31u), jj = (int)(en & 31u);
                const float4 hp = S.hpos[ih], jp = S.jpos[jj];
                // r_i - r_j = (o_i - o_j) - (c_j - c_i) s; the shifts are exact
                const float ddx = pair_delta_f32(hp.x, jp.x, __fmul_rn(__fsub_rn(jp.w, hp.w), tsf));
                const float ddy = pair_delta_f32(hp.y, jp.y, shy);
                const float ddz = pair_delta_f32(hp.z, jp.z, shz);
                const float d2 = pair_d2_f32(ddx, ddy, ddz);
                if (!(d2 <= rall2)) continue;  // the filter's margin let it through
                const float4 hq = S.hprm[ih], jq = S.jprm[jj];
                if (solv && solv_near_f32(d2, hq.w, jq.w, dr, pad)) {
                    // counted here, the slots reserved below, the entries written after that
                    atomicAdd(&S.icnt[ih], 1);
                    atomicAdd(&S.jcnt[jj], 1);
                    S.queue[e] = (unsigned short)(en | kQNear);
                }
                const int a = S.hatom[ih], b = S.jatom[jj];
                const int lo = min(a, b), off = max(a, b) - lo;
                bool excl = false, is14 = false;
                if (off <= kMaskWindow) {
                    const ulonglong2 mk = lo == a ? S.hmask[ih] : S.jmask[jj];
                    excl = (mk.x >> off) & 1ULL;
                    is14 = (mk.y >> off) & 1ULL;
                }
                bool inE = !excl && d2 <= rc2, inV = !excl && d2 <= rv2;
                if (!excl && (fabsf(d2 - rc2) <= tgp || fabsf(d2 - rv2) <= tgp)) {
                    // guard band: the cutoff decided in FP64 exactly as the FP64 path decides it
                    const double ex = __dsub_rn(centre64(d, a, 0), centre64(d, b, 0)),
                                 ey = __dsub_rn(centre64(d, a, 1), centre64(d, b, 1)),
                                 ez = __dsub_rn(centre64(d, a, 2), centre64(d, b, 2));
                    const double d64 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
                    inE = d64 <= d.rcut2;
                    inV = d64 <= d.rvdw2;
                    ++nguard;
                }
                if (inE || inV) {
                    const float we = is14 ? w14e : 1.0f, wv = is14 ? w14v : 1.0f;
                    const PairTermF pt = pair_term_f32(d2, hq.x, jq.x, hq.y, jq.y, hq.z, jq.z, K, we, wv, inE, inV);
                    if (we != 0.0f || wv != 0.0f) ++npairs;
                    const float fx1 = __fmul_rn(pt.coef, ddx), fy1 = __fmul_rn(pt.coef, ddy),
                                fz1 = __fmul_rn(pt.coef, ddz);
                    if (fabsf(fx1) < kPairFxMax && fabsf(fy1) < kPairFxMax && fabsf(fz1) < kPairFxMax) {
                        int n0, f0, n1, f1, n2, f2;
                        fx_pieces(fx1, n0, f0);
                        fx_pieces(fy1, n1, f1);
                        fx_pieces(fz1, n2, f2);
                        atomicAdd(&S.iacc[0][ih], n0);
                        atomicAdd(&S.iacc[1][ih], n1);
                        atomicAdd(&S.iacc[2][ih], n2);
                        atomicAdd(&S.iacc[3][ih], f0);
                        atomicAdd(&S.iacc[4][ih], f1);
                        atomicAdd(&S.iacc[5][ih], f2);
                        // j's term is exactly the negative (the pieces round symmetrically)
                        atomicAdd(&S.jacc[0][jj], -n0);
                        atomicAdd(&S.jacc[1][jj], -n1);
                        atomicAdd(&S.jacc[2][jj], -n2);
                        atomicAdd(&S.jacc[3][jj], -f0);
                        atomicAdd(&S.jacc[4][jj], -f1);
                        atomicAdd(&S.jacc[5][jj], -f2);
                    } else {  // clash-sized (or non-finite) term
                        add_oversized(d, a, b, fx1, fy1, fz1);
                    }
                    ove += pt.e_el;
                    ovv += pt.e_vd;
                }
            }
            __syncwarp();
            // the staged atoms' sums to the global fixed-point forces; list slots of the chunk's
            // solvation pairs, one reservation per atom
            if (lane < jn) {
                const int b = S.jatom[lane];
                unsigned long long* Fb = reinterpret_cast<unsigned long long*>(&d.Fpx[3 * b]);
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const long long v = fx_units(S.jacc[k][lane], S.jacc[3 + k][lane]);
                    if (v) atomicAdd(Fb + k, (unsigned long long)v);
                }
                const int cj = S.jcnt[lane];
                if (cj) S.jbase[lane] = reserve(b, cj);
            }
            if (lane < hn) {
                const int ci = S.icnt[lane];
                if (ci) S.ibase[lane] = reserve(S.hatom[lane], ci);
            }
            __syncwarp();
            // list entries of both directions: j in i's list (r_j - r_i, Roff_j^2), i in j's (r_i - r_j,
            // Roff_i^2)
            if (solv) {
                for (int r = 0; r < R; ++r) {
                    const int e = lane * R + r;
                    if (e >= T) break;
                    const unsigned en = S.queue[e];
                    if (!(en & kQNear)) continue;
                    const int ih = (int)((en >> 5) & 31u), jj = (int)(en & 31u);
                    const float4 hp = S.hpos[ih], jp = S.jpos[jj];
                    const float ddx = pair_delta_f32(hp.x, jp.x, __fmul_rn(__fsub_rn(jp.w, hp.w), tsf));
                    const float ddy = pair_delta_f32(hp.y, jp.y, shy);
                    const float ddz = pair_delta_f32(hp.z, jp.z, shz);
                    const int a = S.hatom[ih], b = S.jatom[jj];
                    // each entry takes the next of its atoms' reserved slots (a list's order is free)
                    const int slot = S.ibase[ih] + atomicAdd(&S.iput[ih], 1);
                    const int rslot = S.jbase[jj] + atomicAdd(&S.jput[jj], 1);
                    if (slot < kMaxNbr) {
                        d.nbr[(size_t)a * kMaxNbr + slot] = b;
                        d.nbr_off[(size_t)a * kMaxNbr + slot] = make_float4(-ddx, -ddy, -ddz, __fmul_rn(S.jprm[jj].w, S.jprm[jj].w));
                    }
                    if (rslot < kMaxNbr) {
                        d.nbr[(size_t)b * kMaxNbr + rslot] = a;
                        d.nbr_off[(size_t)b * kMaxNbr + rslot] = make_float4(ddx, ddy, ddz, __fmul_rn(S.hprm[ih].w, S.hprm[ih].w));
                    }
                }
            }
            if (++nchunk == kPtFlushChunks) {
                flush_home();
                nchunk = 0;
            }
            __syncwarp();  // the next staged row overwrites this one
        }
        flush_home();
        __syncwarp();  // the next segment overwrites the home atoms
    }
    if (cur >= 0) flush_chain();
}

}  // namespace

int pair_tile_rows(int stencil) { return stencil == 2 ? 13 : 5; }

template <int KR>
void launch_pairs_tile_kr(DevChain& d, cudaStream_t s) {
    const int split = d.pair_warps;  // the tile autotuner's pair shape
    const long long warps = (long long)((d.n + 31) / 32) * pair_tile_rows(d.stencil) * split;
    const int nb = (int)((warps + kPtWarps - 1) / kPtWarps);
    if (split == 1) launch_k(k_pair_tile<KR, 1>, nb, kPtWarps * 32, 0, s, d.pdl, d);
    else if (split == 2) launch_k(k_pair_tile<KR, 2>, nb, kPtWarps * 32, 0, s, d.pdl, d);
    else launch_k(k_pair_tile<KR, 4>, nb, kPtWarps * 32, 0, s, d.pdl, d);
}

void launch_pairs_tile(DevChain& d, cudaStream_t s) {
    if (d.stencil == 2) launch_pairs_tile_kr<2>(d, s);
    else launch_pairs_tile_kr<1>(d, s);
}

}  // namespace kcm
