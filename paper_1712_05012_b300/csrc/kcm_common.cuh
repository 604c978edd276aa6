// Device helpers shared by the kernel files of the KCM library.
#pragma once

#include <cuda_runtime.h>

#include "kcm_device.h"

namespace kcm {
namespace dev {

// Programmatic dependent launch: the first statement of every kernel of the library. It waits until the
// previous grid of the stream has completed and its memory operations are visible (at once when the
// kernel was launched without the attribute, or has no such predecessor), then lets the stream's next
// grid be scheduled, so that its launch overlaps this kernel's run (launch_k).
__device__ __forceinline__ void grid_dep_sync() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// kcm_step_host's graphs: the status record to the caller's page-locked copy (one thread, after the
// iteration's last update of the record; 8-byte words read from L2, where other blocks' atomics landed).
// The host reads it after the stream's work has completed, which makes the writes visible.
__device__ __forceinline__ void export_status(const DevChain& d) {
    if (!d.status_io) return;
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(d.status);
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(d.status_io);
#pragma unroll
    for (int i = 0; i < (int)(sizeof(Status) / 8); ++i) dst[i] = __ldcg(src + i);
}

// a step's new angle of joint jj (main chain or side chain), and kcm_step_host's copy of a main-chain one
__device__ __forceinline__ void set_theta(const DevChain& d, int jj, double th) {
    d.theta[jj] = th;
    if (d.theta_io && jj < d.l) d.theta_io[jj] = th;
}

// The loop state of a step call (k_reset_loop, or the first kernel of the first iteration's graph):
// thread c of nthreads; c = 0 resets the status record, and the chains are taken in strides.
__device__ __forceinline__ void reset_loop_state(const DevChain& d, int c, int nthreads, bool full) {
    Status* st = d.status;
    if (c == 0) {
        st->iters = 0;
        st->done = 0;
        st->error = 0;
        st->ticket = 0u;
        st->ticket_w = 0u;
        st->ticket_lb = 0u;
        st->ticket_bin = 0u;
        st->last_max_dtheta = 0.0;
        if (full) {
            st->ticket_bbox = 0u;
            st->pairs = 0; st->nbr_total = 0; st->guard = 0; st->sasa_tests = 0; st->max_nbr = 0; st->nlong = 0;
        }
    }
    for (; c < d.nchains; c += nthreads) {
        d.chain_done[c] = d.chain_maxit[c] <= 0;  // a chain without iterations to take is done from the start
        d.chain_err[c] = 0;
        d.chain_iters[c] = 0;
        d.chain_maxdt[c] = 0ULL;
        d.chain_maxtau[c] = 0ULL;
        d.chain_lastdt[c] = 0.0;
        d.chain_E[3 * c] = 0.0; d.chain_E[3 * c + 1] = 0.0; d.chain_E[3 * c + 2] = 0.0;
        if (full)
            for (int i = 0; i < 3; ++i) { d.cbox[6 * c + i] = ~0ULL; d.cbox[6 * c + 3 + i] = 0ULL; }
    }
}

// ---------------------------------------------------------------- small helpers
// chain of an atom or joint (no load for a single chain)
__device__ __forceinline__ int atom_chain(const DevChain& d, int a) { return d.nchains == 1 ? 0 : d.atom_chain[a]; }
__device__ __forceinline__ int slot_chain(const DevChain& d, int sl) { return d.nchains == 1 ? 0 : d.slot_chain[sl]; }
__device__ __forceinline__ int joint_chain(const DevChain& d, int j) { return d.nchains == 1 ? 0 : d.joint_chain[j]; }

__device__ __forceinline__ unsigned long long dkey(double x) {
    unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
    return (b & 0x8000000000000000ULL) ? ~b : (b | 0x8000000000000000ULL);
}
__device__ __forceinline__ double dkey_inv(unsigned long long k) {
    unsigned long long b = (k & 0x8000000000000000ULL) ? (k & 0x7FFFFFFFFFFFFFFFULL) : ~k;
    return __longlong_as_double(static_cast<long long>(b));
}

// Mixed mode: coordinate i of atom a in FP64, from the double-float centres the kinematics keep (the
// exact double of hi + lo, as the FP64 centres are formed); the mixed kernels need it only on their rare
// FP64 re-decisions, so the kinematics need not store FP64 centres in this mode.
__device__ __forceinline__ double centre64(const DevChain& d, int a, int i) {
    const float2 v = reinterpret_cast<const float2*>(d.rdf)[3 * a + i];
    return __dadd_rn((double)v.x, (double)v.y);
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
// exact warp sum of int32 values with |v| <= 2^30, as int64: 32-bit reductions of the two 16-bit
// halves of v + 2^30 (each half-sum fits in 32 bits)
__device__ __forceinline__ long long warp_sum_i32(int v) {
    const unsigned u = (unsigned)(v + (1 << 30));
    const unsigned hs = __reduce_add_sync(0xffffffffu, u >> 16);
    const unsigned ls = __reduce_add_sync(0xffffffffu, u & 0xFFFFu);
    return ((long long)hs << 16) + (long long)ls - 32LL * (1LL << 30);
}
__device__ __forceinline__ int warp_max(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// Exact fixed-point pieces of an FP32 pair term v, |v| < 2^22, with FP32 adds and integer subtracts
// only (B300 runs 64-bit conversions on its slow FP64 pipe). Adding 1.5 * 2^23 moves v into the
// binade where the float spacing is 1, so the sum is v rounded to an integer (ties to even) and its
// bit pattern minus that of 1.5 * 2^23 is that integer n; f = v - n is exact and |f| <= 1/2; the
// same trick on f * 2^23 gives the fraction in units of 2^-23. Both roundings are symmetric in sign,
// so the pieces of the (i, j) and (j, i) terms are exact negatives.
constexpr float kMagic23 = 12582912.0f;  // 1.5 * 2^23
constexpr int kMagic23Bits = 0x4B400000;
__device__ __forceinline__ void fx_pieces(float v, int& n, int& f) {
    const float t = v + kMagic23;
    const float fr = v - (t - kMagic23);
    const float u = fmaf(fr, 8388608.0f, kMagic23);
    n = __float_as_int(t) - kMagic23Bits;
    f = __float_as_int(u) - kMagic23Bits;
}
__device__ __forceinline__ void fx_add(float v, int& hi, int& lo) {
    int n, f;
    fx_pieces(v, n, f);
    hi += n;
    lo += f;
}
// the whole term n 2^23 + f in units of 2^-23
__device__ __forceinline__ long long fx_units(int n, int f) { return (long long)n * 8388608LL + f; }

// A pair term with a component of 2^22 or more (a clash) on atoms a and b (b takes the negative), summed
// so that the total does not depend on the order of the additions: a component below 2^22 in the fixed
// point of the other terms (2^-23), one of 2^22 .. 2^50 exactly in units of 2^-1 (a float of magnitude
// 2^22 or more is a multiple of 2^-1), and only a larger or non-finite one in a plain float sum.
__device__ __forceinline__ void add_oversized(const DevChain& d, int a, int b, float fx, float fy, float fz) {
    const float v[3] = {fx, fy, fz};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float m = fabsf(v[k]);
        if (m < 4194304.0f) {  // 2^22
            int n, f;
            fx_pieces(v[k], n, f);
            const long long u = fx_units(n, f);
            atomicAdd(reinterpret_cast<unsigned long long*>(&d.Fpx[3 * a + k]), (unsigned long long)u);
            atomicAdd(reinterpret_cast<unsigned long long*>(&d.Fpx[3 * b + k]), (unsigned long long)(-u));
        } else if (m < 1125899906842624.0f) {  // 2^50
            const long long u = __float2ll_rn(v[k] * 2.0f);  // exact
            atomicAdd(reinterpret_cast<unsigned long long*>(&d.Fox[3 * a + k]), (unsigned long long)u);
            atomicAdd(reinterpret_cast<unsigned long long*>(&d.Fox[3 * b + k]), (unsigned long long)(-u));
        } else {
            atomicAdd(&d.Fov[3 * a + k], v[k]);
            atomicAdd(&d.Fov[3 * b + k], -v[k]);
        }
    }
}

// Mixed-precision pair geometry with every FP32 rounding written out, so that each pair kernel that
// evaluates a pair forms the same bits (a compiler left to itself may fuse these operations
// differently in different kernels). Offsets are from the corners of the atoms' cells; the x shift
// (cx_j - cx_i) s and the row shifts (dy s, dz s) are exact.
// r_i - r_j = (o_i - o_j) - shift, component by component
__device__ __forceinline__ float pair_delta_f32(float oi, float oj, float shift) {
    return __fsub_rn(__fsub_rn(oi, oj), shift);
}
__device__ __forceinline__ float pair_d2_f32(float dx, float dy, float dz) {
    return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
}
// solvation neighbour range (A'_i, reading c11) with the FP32 cell-offset margin pad
__device__ __forceinline__ bool solv_near_f32(float d2, float Roi, float Roj, float dr, float pad) {
    const float lim = __fadd_rn(__fadd_rn(__fadd_rn(Roi, Roj), dr), pad);
    return d2 <= __fmul_rn(lim, lim);
}

// Force coefficient c (F_i = c (r_i - r_j) = -F_j) and energies of one pair in FP32: Coulomb with
// the dielectric 4d, E = K q_i q_j / (4 d^2) (eq. 02_2 with reading c2), and Lennard-Jones in the
// AMBER form eps_ij [(D/d)^12 - 2 (D/d)^6], D = R_i + R_j, eps_ij = sqrt(eps_i) sqrt(eps_j) (eq. 03_2,
// reading c5), each weighted by its 1-4 factor (eq. 03_8 / 03_9). Every product of the two atoms'
// constants is formed symmetrically, so (i, j) and (j, i) give the same bits. A near-coincident pair
// (d of a few thousandths of an A) would overflow the FP32 coefficient, or make it NaN from
// inf - inf: it is held at kPairCoefMax, a huge finite repulsion.
struct PairTermF {
    float coef, e_el, e_vd;
};
__device__ __forceinline__ PairTermF pair_term_f32(float d2, float qi, float qj, float sei, float sej, float Ri,
                                                   float Rj, float K, float we, float wv, bool inE, bool inV) {
    const float inv2 = __frcp_rn(d2);
    float cE = 0.0f, cV = 0.0f, eel = 0.0f, evd = 0.0f;
    if (inE) {
        const float qq = __fmul_rn(__fmul_rn(we, K), __fmul_rn(qi, qj));
        cE = __fmul_rn(__fmul_rn(0.5f, qq), __fmul_rn(inv2, inv2));
        eel = __fmul_rn(__fmul_rn(0.25f, qq), inv2);
    }
    if (inV) {
        const float D = __fadd_rn(Ri, Rj);
        const float x2 = __fmul_rn(__fmul_rn(D, D), inv2);
        const float t6 = __fmul_rn(__fmul_rn(x2, x2), x2);
        const float t12 = __fmul_rn(t6, t6);
        const float eij = __fmul_rn(wv, __fmul_rn(sei, sej));
        cV = __fmul_rn(__fmul_rn(__fmul_rn(12.0f, eij), __fsub_rn(t12, t6)), inv2);
        evd = __fmul_rn(eij, __fsub_rn(t12, __fmul_rn(2.0f, t6)));
    }
    float coef = __fadd_rn(cE, cV);
    if (!(coef <= kPairCoefMax)) coef = kPairCoefMax;
    return PairTermF{coef, eel, evd};
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


// Grid of a chain's cell list from its bounding box (lo, hi; or kb, order-preserving keys: min x, y, z
// then max x, y, z): cube cells of edge s with d.stencil * s >= every interaction range (plus a margin that
// absorbs FP32 cell assignment, so that two atoms within range are at most d.stencil cells apart on
// every axis), and s >= the requested edge; s a multiple of 2^-10 A so that it is exact in float;
// coarsened when the box would need more cells than the chain's cap. Leaves cbase to the caller.
// Returns false for a non-finite box (the grid is then one cell at the origin).
// (s_base, stencil and cell: DevChain's s_base, stencil and prm.cell_size)
__device__ __forceinline__ bool grid_from_bounds_s(double s_base, int stencil, double cell, double* lo, double* hi,
                                                   long long cap, GridInfo* out) {
    GridInfo g;
    const bool finite = isfinite(hi[0] - lo[0]) && isfinite(hi[1] - lo[1]) && isfinite(hi[2] - lo[2]);
    if (!finite)
        for (int i = 0; i < 3; ++i) { lo[i] = 0.0; hi[i] = 0.0; }
    const double ext[3] = {hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]};
    // (the division by the stencil, 1 or 2, is exact: a multiplication)
    double s = fmax(fma(1e-6, fmax(ext[0], fmax(ext[1], ext[2])), s_base) * (stencil == 2 ? 0.5 : 1.0), cell);
    s = ceil(s * 1024.0) * (1.0 / 1024.0);
    for (;;) {
        // n_i = floor(ext_i / s) + 1 estimated in float, then raised until n_i s > ext_i holds exactly
        // (n_i s is exact: s is a multiple of 2^-10), so the cells cover the box
        const float inv = 1.0f / (float)s;
        long long nn[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            long long k = (long long)floorf((float)ext[i] * inv) + 1;
            while ((double)k * s <= ext[i]) ++k;
            nn[i] = k;
        }
        if (nn[0] * nn[1] * nn[2] <= cap) {
            g.nx = (int)nn[0]; g.ny = (int)nn[1]; g.nz = (int)nn[2];
            g.ncells = (int)(nn[0] * nn[1] * nn[2]);
            break;
        }
        s = ceil(s * 1.25 * 1024.0) * (1.0 / 1024.0);
    }
    g.ox = lo[0]; g.oy = lo[1]; g.oz = lo[2];
#pragma unroll
    for (int i = 0; i < 3; ++i) {  // hi + lo of each coordinate of the origin (as df_from(double))
        const float h = __double2float_rn(lo[i]);
        g.of[i] = make_float2(h, __double2float_rn(__dsub_rn(lo[i], (double)h)));
    }
    g.s = s;
    g.sf = (float)s;
    g.gpf = (float)(1e-3 + 2e-4 * s);
    g.inv_sf = 1.0f / (float)s;
    g.cbase = 0;
    g.pad = 0;
    *out = g;
    return finite;
}
__device__ __forceinline__ bool grid_from_bounds(const DevChain& d, double* lo, double* hi, long long cap, GridInfo* out) {
    return grid_from_bounds_s(d.s_base, d.stencil, d.prm.cell_size, lo, hi, cap, out);
}

__device__ __forceinline__ bool grid_from_box(const DevChain& d, const unsigned long long* kb, long long cap,
                                              GridInfo* out) {
    double lo[3], hi[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        lo[i] = dkey_inv(kb[i]);
        hi[i] = dkey_inv(kb[3 + i]);
    }
    return grid_from_bounds(d, lo, hi, cap, out);
}

// the grid of chain c from the box its atoms were added to (cbox), which is reset for the next evaluation
__device__ __forceinline__ bool chain_grid(const DevChain& d, int c, GridInfo* out) {
    unsigned long long kb[6];  // every load before the first store
#pragma unroll
    for (int i = 0; i < 6; ++i) kb[i] = __ldcg(&d.cbox[6 * c + i]);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        d.cbox[6 * c + i] = ~0ULL;
        d.cbox[6 * c + 3 + i] = 0ULL;
    }
    return grid_from_box(d, kb, d.ccap[c], out);
}

}  // namespace dev
}  // namespace kcm
