// A1: forward kinematics as a prefix product of local link-frame transforms (FP64).
//
// Link frame poses T_j = L_1 o ... o L_j with L_j = Tr(step_j) o Rot(u0_j, theta_j) (eq. kin_04 in
// local frames; App. B prefix computation). Atom centres are T_link(r0 - frame origin) (eq. r1, r2).
//
// On B300 an FP64 warp instruction occupies a sub-partition's FP64 pipe for about 84 cycles however
// many of its lanes are active, so the scan is laid out to need few of them on its critical path
// (FP64 mode), and the mixed mode runs the same kernels in double-float arithmetic (kcm_df.cuh) on
// the FP32 pipe, with positions rounded to double at the end:
// a transform [R | t] is held by a quad of four lanes, lane r of the quad holding row r (R_r0, R_r1,
// R_r2, t_r) (the fourth lane repeats row 2). A composition A o B then costs each lane one row, 12
// FP64 instructions, instead of 36 for a whole transform per lane, and a warp holds eight transforms.
//
// k_fk_scan: block b (four warps, one per SM sub-partition, 32 quads) takes joints [32 J b,
// 32 J (b + 1)), J consecutive joints per quad. Each quad forms its joints' local transforms and their
// running product (kept in G), the warp scans its eight quad products (Kogge-Stone, 3 levels), warp 0
// scans the four warp products, and each quad stores its exclusive prefix within the block; the
// block product goes to tileP. When every chain lies within kFkTreeTiles blocks (a single chain of up to
// 2,048 J joints; the chains of a batch), every apply block reduces in one tree the products of the
// blocks before it back to the one where its chain starts; otherwise a one-block kernel of eight warps
// (k_fk_tiles) scans all block products into every block's exclusive prefix (tileE). k_fk_apply: block b composes its prefix,
// quad prefix and running products into the link poses, the current axes u_j and axis points p_j,
// moves the atoms of its links and adds them to their chain's bounding box; its last block to finish
// sets the grids of the cell lists. A batch of chains is their concatenation: every product is
// segmented at the first joint of a chain.
#include <cuda_runtime.h>

#include <type_traits>

#include "kcm_cells.cuh"
#include "kcm_common.cuh"
#include "kcm_df.cuh"
#include "kcm_device.h"
#include "kcm_launch.h"

namespace kcm {

namespace {
using namespace dev;

constexpr int kFkWarps = 4;               // warps per block of the transform scan (one per sub-partition)
constexpr int kFkQuads = 8 * kFkWarps;    // quads (transform slots) per block
constexpr int kFkMaxTiles = 40 * kFkQuads;  // most scan blocks (k_fk_tiles' quads run through up to 20 products each)
constexpr int kFkTreeTiles = 2 * kFkQuads;  // up to this many, every apply block reduces the earlier products itself

// the grid of chain c from its box keys (chain_grid; mixed mode: keys of double-float pairs)
template <class T>
__device__ __forceinline__ bool chain_grid_t(const DevChain& d, int c, GridInfo* out) {
    if constexpr (std::is_same<T, double>::value) {
        return chain_grid(d, c, out);
    } else {
        unsigned long long kb[6];  // every load before the first store
#pragma unroll
        for (int i = 0; i < 6; ++i) kb[i] = __ldcg(&d.cbox[6 * c + i]);
        df lo[3], hi[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            lo[i] = dfkey_inv(kb[i]);
            hi[i] = dfkey_inv(kb[3 + i]);
            d.cbox[6 * c + i] = ~0ULL;
            d.cbox[6 * c + 3 + i] = 0ULL;
        }
        return grid_from_bounds_df(d.s_base, d.stencil, d.prm.cell_size, lo, hi, d.ccap[c], out);
    }
}

// FP64 centres from the double-float ones (mixed mode keeps only those), for the callers that read them
__global__ void k_centres64(const DevChain d) {
    grid_dep_sync();
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x < 3 * d.n) d.r[x] = centre64(d, x / 3, x % 3);
}

// row rr of the identity
template <class T>
__device__ __forceinline__ void row_identity(int rr, T* a) {
    a[0] = num_f<T>(rr == 0 ? 1.0f : 0.0f);
    a[1] = num_f<T>(rr == 1 ? 1.0f : 0.0f);
    a[2] = num_f<T>(rr == 2 ? 1.0f : 0.0f);
    a[3] = num_f<T>(0.0f);
}

// the three rows of the quad's transform b (lanes base, base + 1, base + 2), for every lane of the quad
template <class T>
__device__ __forceinline__ void quad_rows(const T* b, int base, T* B) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
#pragma unroll
        for (int m = 0; m < 4; ++m) B[4 * k + m] = shfl(b[m], base + k);
    }
}

// A row and a whole transform (rows B[0..3], B[4..7], B[8..11]) passed by value.
template <class T>
struct Row4 {
    T v[4];
};
template <class T>
struct Mat34 {
    T v[12];
};

// row of C = A o B from row a of A and the full B
template <class T>
__device__ __forceinline__ Row4<T> row_compose_v(const Row4<T>& a, const Mat34<T>& B) {
    Row4<T> c;
#pragma unroll
    for (int m = 0; m < 3; ++m) c.v[m] = fma(a.v[2], B.v[8 + m], fma(a.v[1], B.v[4 + m], mul(a.v[0], B.v[m])));
    c.v[3] = fma(a.v[2], B.v[11], fma(a.v[1], B.v[7], fma(a.v[0], B.v[3], a.v[3])));
    return c;
}

// The double-float composition (~150 float instructions) as one function that is not inlined. These
// kernels run their straight-line code once per SM, so their time goes largely to fetching it: the
// instruction caches start cold after other kernels (and after an L2 flush the code comes from DRAM),
// and a composition inlined at every site is fetched at every site. One shared copy is fetched once
// and then runs from the cache (measured on B300: a composition costs ~0.5 us as fresh inline code
// from L2, ~1.1 us from DRAM, ~0.3 us as a call).
__device__ __noinline__ Row4<df> row_compose_df(Row4<df> a, Mat34<df> B) { return row_compose_v(a, B); }

template <class T>
__device__ __forceinline__ void row_compose(const T* a, const T* B, T* c) {
    Row4<T> ra;
    Mat34<T> mb;
#pragma unroll
    for (int m = 0; m < 4; ++m) ra.v[m] = a[m];
#pragma unroll
    for (int m = 0; m < 12; ++m) mb.v[m] = B[m];
    Row4<T> rc;
    if constexpr (std::is_same<T, df>::value) rc = row_compose_df(ra, mb);
    else rc = row_compose_v(ra, mb);
#pragma unroll
    for (int m = 0; m < 4; ++m) c[m] = rc.v[m];
}

// row rr of the local joint transform L_j = Tr(step_j) o Rot(u_j, th) with
// R = cos I + sin [u]x + (1 - cos) u u^T (right-hand rule); the same arithmetic as joint_tf
__device__ __forceinline__ void joint_row(const DevChain& d, int j, double th, int rr, double* g) {
    const double* u = &d.u0[3 * j];
    double s, c;
    sincos(th, &s, &c);
    const double C = 1.0 - c;
    if (rr == 0) {
        g[0] = c + u[0] * u[0] * C; g[1] = u[0] * u[1] * C - u[2] * s; g[2] = u[0] * u[2] * C + u[1] * s;
    } else if (rr == 1) {
        g[0] = u[1] * u[0] * C + u[2] * s; g[1] = c + u[1] * u[1] * C; g[2] = u[1] * u[2] * C - u[0] * s;
    } else {
        g[0] = u[2] * u[0] * C - u[1] * s; g[1] = u[2] * u[1] * C + u[0] * s; g[2] = c + u[2] * u[2] * C;
    }
    g[3] = d.step0[3 * j + rr];
}
__device__ __forceinline__ void joint_row(const DevChain& d, int j, double th, int rr, df* g) {
    const df* u = reinterpret_cast<const df*>(d.u0df) + 3 * j;
    df s, c;
    df_sincos(th, &s, &c);
    const df C = sub(df{1.0f, 0.0f}, c);
    const df ur = u[rr];
    const df urC = mul(ur, C);
#pragma unroll
    for (int m = 0; m < 3; ++m) g[m] = mul(urC, u[m]);  // (1 - cos) u_r u_m
    g[rr] = add(g[rr], c);
    // + sin [u]x: row 0 (0, -u2, u1), row 1 (u2, 0, -u0), row 2 (-u1, u0, 0)
    const int m1 = rr == 0 ? 2 : (rr == 1 ? 0 : 1);  // column with +sin u_k
    const int m2 = rr == 0 ? 1 : (rr == 1 ? 2 : 0);  // column with -sin u_k
    const int k1 = rr == 0 ? 1 : (rr == 1 ? 2 : 0);
    const int k2 = rr == 0 ? 2 : (rr == 1 ? 0 : 1);
    g[m1] = fma(s, u[k1], g[m1]);
    g[m2] = fma(neg(s), u[k2], g[m2]);
    g[3] = reinterpret_cast<const df*>(d.step0df)[3 * j + rr];
}

template <class T>
__device__ __forceinline__ void store_row(T* M, int rr, const T* a) {
    M[3 * rr] = a[0];
    M[3 * rr + 1] = a[1];
    M[3 * rr + 2] = a[2];
    M[9 + rr] = a[3];
}
template <class T>
__device__ __forceinline__ void load_row(const T* M, int rr, T* a) {
    a[0] = M[3 * rr];
    a[1] = M[3 * rr + 1];
    a[2] = M[3 * rr + 2];
    a[3] = M[9 + rr];
}
template <class T>
__device__ __forceinline__ void load_rows(const T* M, T* B) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        B[4 * k] = M[3 * k];
        B[4 * k + 1] = M[3 * k + 1];
        B[4 * k + 2] = M[3 * k + 2];
        B[4 * k + 3] = M[9 + k];
    }
}

// row rr of a transform written by another block of the running kernel (L2, not a stale L1 line)
__device__ __forceinline__ void load_row_cg(const double* M, int rr, double* a) {
    a[0] = __ldcg(&M[3 * rr]);
    a[1] = __ldcg(&M[3 * rr + 1]);
    a[2] = __ldcg(&M[3 * rr + 2]);
    a[3] = __ldcg(&M[9 + rr]);
}
__device__ __forceinline__ void load_row_cg(const df* M, int rr, df* a) {
    const double* m = reinterpret_cast<const double*>(M);
    double t[4] = {__ldcg(&m[3 * rr]), __ldcg(&m[3 * rr + 1]), __ldcg(&m[3 * rr + 2]), __ldcg(&m[9 + rr])};
#pragma unroll
    for (int k = 0; k < 4; ++k) a[k] = *reinterpret_cast<const df*>(&t[k]);
}

// Segmented products: a quad carries (f, A) with f set when a chain starts within the range A covers;
// (f1, A1) followed by (f2, A2) combine to (f1 | f2, f2 ? A2 : A1 o A2), so products never reach
// across the first joint of a chain.

// inclusive segmented Kogge-Stone scan over the first NQ quads of a warp (composition on the left)
template <int NQ = 8, class T>
__device__ __forceinline__ void warp_scan_quads(T* a, bool& f, int q, int base) {
#pragma unroll
    for (int off = 1; off < NQ; off <<= 1) {
        T y[4], B[12];
#pragma unroll
        for (int m = 0; m < 4; ++m) y[m] = shfl_up(a[m], 4 * off);
        const bool yf = __shfl_up_sync(0xffffffffu, f, 4 * off);
        quad_rows(a, base, B);
        if (q >= off) {
            if (!f) row_compose(y, B, a);
            f = f || yf;
        }
    }
}

// Scans the transforms held by the block's quads (row a of slot 8 w + q, flag f) in place into
// inclusive segmented block prefixes; the block total is returned in (tf, tot) on every lane.
// sW: [NW][12], sF: [NW] shared (NW warps, at most 8).
template <class T, int NW = kFkWarps>
__device__ __forceinline__ void block_scan_quads(T* a, bool& f, T* tot, bool& tf, T (*sW)[12], int* sF, int w, int q,
                                                 int rr, int base, int lane) {
    warp_scan_quads(a, f, q, base);
    if (q == 7 && (lane & 3) < 3) store_row(sW[w], rr, a);
    if (lane == 28) sF[w] = f;
    __syncthreads();
    if (w == 0) {  // scan of the warp totals, quad q <- warp q
        T t[4];
        bool tfl = false;
        if (q < NW) { load_row(sW[q], rr, t); tfl = sF[q] != 0; }
        else row_identity(rr, t);
        warp_scan_quads<NW>(t, tfl, q, base);
        __syncwarp();
        if (q < NW && (lane & 3) < 3) store_row(sW[q], rr, t);  // inclusive prefix of warps 0..q
        if (q < NW && (lane & 3) == 0) sF[q] = tfl;
    }
    __syncthreads();
    if (w > 0) {  // prefix of the earlier warps o own warp prefix, unless a chain starts in between
        T P[4], B[12];
        load_row(sW[w - 1], rr, P);
        quad_rows(a, base, B);  // shuffles outside the per-quad condition
        if (!f) row_compose(P, B, a);
        f = f || sF[w - 1] != 0;
    }
    load_row(sW[NW - 1], rr, tot);
    tf = sF[NW - 1] != 0;
    __syncthreads();
}

// Side-chain joints (eq. kin_05, r2): the offsets, in the frame of their CA link, of the side atoms
// that chi_1 .. chi_k turn. In the ZP frame the rotations compose from the most distal joint inward,
// x = T_1(T_2(... T_k(x0))) with T_c(x) = a_c + Rot(u_c, chi_c)(x - a_c) about the ZP bond (a_c, u_c):
// each T_c then turns about its bond where the ZP has it, and the link pose (the main-chain joints)
// takes the result to the current frame like every other atom of the link. Run by extra blocks of
// the transform-scan kernel, beside the scan (the apply kernel reads the result). Block b takes 128
// moved atoms (residue by residue); its threads first form sin and cos of the joints those atoms need
// (at most 128 + 3: a residue has no more joints than moved atoms, so only the block's first residue
// can bring joints beyond its atoms) into shared memory, then each thread turns its atom (at most four
// rotations). FP64, or double-float on the FP32 pipe in mixed mode, as the main-chain kinematics.
template <class T>
__device__ __forceinline__ void side_fk_block(const DevChain& d, int b) {
    constexpr bool DF = std::is_same<T, df>::value;
    constexpr int kJ = kSideFkThreads + 4;
    __shared__ T sS[kJ], sC[kJ];
    const int t0 = b * kSideFkThreads, t = t0 + threadIdx.x;
    const int2 last = d.mv_chi[min(t0 + kSideFkThreads, d.nmv) - 1];
    const int j0 = d.mv_chi[t0].x, j1 = last.x + last.y;  // the joints of the block's atoms
    // the thread's atom, loaded before the barrier
    const T* r0 = reinterpret_cast<const T*>(DF ? d.r0df : d.r0);
    const bool act = t < d.nmv;
    const int a = act ? d.mv_atom[t] : 0;
    const int2 mc = act ? d.mv_chi[t] : make_int2(0, 0);
    T x = r0[3 * a], y = r0[3 * a + 1], z = r0[3 * a + 2];
    for (int j = j0 + threadIdx.x; j < j1; j += kSideFkThreads) {
        T sn, cs;
        if constexpr (DF) {
            df_sincos(d.theta[d.l + j], &sn, &cs);
        } else {
            sincos(d.theta[d.l + j], &sn, &cs);
        }
        sS[j - j0] = sn;
        sC[j - j0] = cs;
    }
    __syncthreads();
    if (!act) return;
    const T* P = reinterpret_cast<const T*>(d.chi_p0);
    const T* U = reinterpret_cast<const T*>(d.chi_u0);
    for (int k = mc.y - 1; k >= 0; --k) {
        const int c = mc.x + k;
        const T sn = sS[c - j0], cs = sC[c - j0];
        const T ux = U[3 * c], uy = U[3 * c + 1], uz = U[3 * c + 2];
        const T px = P[3 * c], py = P[3 * c + 1], pz = P[3 * c + 2];
        const T vx = sub(x, px), vy = sub(y, py), vz = sub(z, pz);
        // Rodrigues: v cos + (u x v) sin + u (u . v)(1 - cos)
        const T w = mul(fma(ux, vx, fma(uy, vy, mul(uz, vz))), sub(num_f<T>(1.0f), cs));
        x = add(add(px, mul(vx, cs)), fma(sub(mul(uy, vz), mul(uz, vy)), sn, mul(ux, w)));
        y = add(add(py, mul(vy, cs)), fma(sub(mul(uz, vx), mul(ux, vz)), sn, mul(uy, w)));
        z = add(add(pz, mul(vz, cs)), fma(sub(mul(ux, vy), mul(uy, vx)), sn, mul(uz, w)));
    }
    T* out = reinterpret_cast<T*>(d.r0fk);
    out[3 * a] = x;
    out[3 * a + 1] = y;
    out[3 * a + 2] = z;
}

template <int J, class T>
__global__ void __launch_bounds__(kFkWarps * 32) k_fk_scan(const DevChain d) {
    grid_dep_sync();
    __shared__ T sW[kFkWarps][12];
    __shared__ int sF[kFkWarps];
    if (d.status->done) return;
    if (blockIdx.x >= d.ntiles) {  // the blocks after the scan's: side-chain joints
        side_fk_block<T>(d, blockIdx.x - d.ntiles);
        return;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int q = lane >> 2, rr = min(lane & 3, 2), base = lane & ~3;
    const int slot = w * 8 + q;
    const int j0 = (blockIdx.x * kFkQuads + slot) * J;
    T* G = reinterpret_cast<T*>(d.G);
    // running product of the quad's J joints, restarted at the first joint of a chain (the first
    // J - 1 kept in G until the block prefix is known); lf: a chain starts in the quad at or before
    T a[4];
    row_identity(rr, a);
    bool lf = false;
    unsigned lfbits = 0;
#pragma unroll
    for (int i = 0; i < J; ++i) {
        const int j = j0 + i;
        T g[4];  // joints past the end act as the identity (every lane takes part in the shuffles)
        bool head = false;
        if (j < d.l) {
            double th;
            if (d.io_import) {  // kcm_step_host's first iteration: the angles from the caller's buffer
                th = d.theta_io[j];
                if ((lane & 3) == 0) d.theta[j] = th;
            } else {
                th = d.theta[j];
            }
            joint_row(d, j, th, rr, g);
            head = d.jhead[j] != 0;
        } else {
            row_identity(rr, g);
        }
        if (i == 0) {
#pragma unroll
            for (int m = 0; m < 4; ++m) a[m] = g[m];
        } else {
            T B[12];
            quad_rows(g, base, B);  // shuffles outside the per-quad condition
            if (head) {
#pragma unroll
                for (int m = 0; m < 4; ++m) a[m] = g[m];
            } else {
                row_compose(a, B, a);
            }
        }
        lf = lf || head;
        lfbits |= lf ? (1u << i) : 0u;
        if (i < J - 1 && j < d.l && (lane & 3) < 3) store_row(&G[12 * (size_t)j], rr, a);
    }
    // block-inclusive segmented prefix of the quad; G_j <- (block prefix before the quad) o running
    // product through joint j, the pose of link j + 1 relative to the block's first frame (or to its
    // chain's first frame when the chain starts inside the block: gseg_j)
    T incl[4], tot[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) incl[m] = a[m];
    bool f = lf, tf = false;
    block_scan_quads(incl, f, tot, tf, sW, sF, w, q, rr, base, lane);
    T ex[4];
    bool exf;
#pragma unroll
    for (int m = 0; m < 4; ++m) ex[m] = shfl_up(incl[m], 4);
    exf = __shfl_up_sync(0xffffffffu, f, 4);
    if (q == 0) {  // first quad of the warp: the inclusive prefix of the previous warp
        if (w == 0) { row_identity(rr, ex); exf = false; }
        else { load_row(sW[w - 1], rr, ex); exf = sF[w - 1] != 0; }  // written before the last barrier, not reused
    }
    if (J > 1) {
#pragma unroll
        for (int i = 0; i < J - 1; ++i) {  // uniform within the quad
            const int j = j0 + i;
            if (j < d.l) {
                const bool own = (lfbits >> i) & 1u;  // a chain starts in the quad at or before joint j
                if (!own) {
                    T B[12], y[4];
                    load_rows(&G[12 * (size_t)j], B);
                    row_compose(ex, B, y);
                    __syncwarp(0xfu << base);
                    if ((lane & 3) < 3) store_row(&G[12 * (size_t)j], rr, y);
                }
                if ((lane & 3) == 0) d.gseg[j] = (unsigned char)(own || exf);
            }
        }
    }
    const int jl = j0 + J - 1;
    if (jl < d.l) {
        if ((lane & 3) < 3) store_row(&G[12 * (size_t)jl], rr, incl);
        if ((lane & 3) == 0) d.gseg[jl] = (unsigned char)f;
    }
    T* tP = reinterpret_cast<T*>(d.tileP);
    if (threadIdx.x < 32 && q == 0) {
        if ((lane & 3) < 3) store_row(&tP[12 * (size_t)blockIdx.x], rr, tot);
        if (lane == 0) d.tileF[blockIdx.x] = tf;
    }
    // Many blocks: the last block scans the block products, E_b = segmented product of blocks 0 .. b-1.
    // Few: every apply block reduces the products before it in one tree (a shorter critical path).
}

// A chain longer than kFkTreeTiles scan blocks: one block of kTileWarps warps scans the block products
// into every block's exclusive segmented prefix (tileE); each of its quads runs through
// ceil(blocks / quads) products in order, then the quads' totals are scanned and each quad runs
// through its products again, writing the prefixes. Eight warps (64 quads) halve the serial runs
// of the scan kernel's own four-warp blocks.
constexpr int kTileWarps = 8;
constexpr int kTileQuads = 8 * kTileWarps;
template <class T>
__global__ void __launch_bounds__(kTileWarps * 32) k_fk_tiles(const DevChain d) {
    grid_dep_sync();
    __shared__ T sW[kTileWarps][12];
    __shared__ int sF[kTileWarps];
    if (d.status->done) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int q = lane >> 2, rr = min(lane & 3, 2), base = lane & ~3;
    const int slot = w * 8 + q;
    const T* tP = reinterpret_cast<const T*>(d.tileP);
    T tot[4], ex[4];
    bool tf = false, exf = false;
    const int nt = d.ntiles;
    const int per = (nt + kTileQuads - 1) / kTileQuads;  // block products per quad, in order
    const int t0 = slot * per;
    T run[4];
    bool rf = false;
    row_identity(rr, run);
    for (int i = 0; i < per; ++i) {  // the quad's running product (every lane takes part in the shuffles)
        const int tt = t0 + i;
        T p[4], B[12];
        bool pf = false;
        if (tt < nt) { load_row_cg(&tP[12 * (size_t)tt], rr, p); pf = __ldcg(&d.tileF[tt]) != 0; }
        else row_identity(rr, p);
        quad_rows(p, base, B);
        if (pf) { for (int m = 0; m < 4; ++m) run[m] = p[m]; }
        else row_compose(run, B, run);
        rf = rf || pf;
    }
    bool xf = rf;
    block_scan_quads<T, kTileWarps>(run, xf, tot, tf, sW, sF, w, q, rr, base, lane);
    // exclusive prefix of the quad: the inclusive prefix of the quad before it
#pragma unroll
    for (int m = 0; m < 4; ++m) ex[m] = shfl_up(run[m], 4);
    exf = __shfl_up_sync(0xffffffffu, xf, 4);
    if (q == 0) {
        if (w == 0) { row_identity(rr, ex); exf = false; }
        else { load_row(sW[w - 1], rr, ex); exf = sF[w - 1] != 0; }
    }
    T* tE = reinterpret_cast<T*>(d.tileE);
    for (int i = 0; i < per; ++i) {
        const int tt = t0 + i;
        T p[4], B[12];
        bool pf = false;
        if (tt < nt) {
            if ((lane & 3) < 3) store_row(&tE[12 * (size_t)tt], rr, ex);
            load_row_cg(&tP[12 * (size_t)tt], rr, p);
            pf = __ldcg(&d.tileF[tt]) != 0;
        } else {
            row_identity(rr, p);
        }
        quad_rows(p, base, B);
        if (pf) { for (int m = 0; m < 4; ++m) ex[m] = p[m]; }
        else row_compose(ex, B, ex);
    }
}

// row rr (and flag) of the segmented product of the block products b0 .. b1 - 1 (identity, no flag,
// when empty), all warps of the block taking part: two products per quad, a tree within each warp,
// then a tree over the warp products
template <class T>
__device__ __forceinline__ void block_prefix(const DevChain& d, int b0, int b1, T (*sW)[12], int* sF, int w, int q,
                                             int rr, int base, int lane, T* out, bool& of) {
    const T* P = reinterpret_cast<const T*>(d.tileP);
    const int slot = w * 8 + q;
    T a[4], B[12];
    bool f = false;
    const int i0 = b0 + 2 * slot, i1 = i0 + 1;
    if (i0 < b1) { load_row(&P[12 * (size_t)i0], rr, a); f = d.tileF[i0] != 0; }
    else row_identity(rr, a);
    if (i1 < b1) {  // uniform within the quad
        load_rows(&P[12 * (size_t)i1], B);
        const bool f1 = d.tileF[i1] != 0;
        if (f1) { T t[4]; load_row(&P[12 * (size_t)i1], rr, t); for (int m = 0; m < 4; ++m) a[m] = t[m]; }
        else row_compose(a, B, a);
        f = f || f1;
    }
#pragma unroll
    for (int off = 1; off < 8; off <<= 1) {  // tree over the quads of the warp: quad q <- q (+) q + off
        T y[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) y[m] = shfl_down(a[m], 4 * off);
        const bool yf = __shfl_down_sync(0xffffffffu, f, 4 * off);
        quad_rows(y, base, B);
        if ((q & (2 * off - 1)) == 0) {
            if (yf) { for (int m = 0; m < 4; ++m) a[m] = y[m]; }
            else row_compose(a, B, a);
            f = f || yf;
        }
    }
    if (q == 0 && (lane & 3) < 3) store_row(sW[w], rr, a);
    if (lane == 0) sF[w] = f;
    __syncthreads();
    if (w == 0) {  // tree over the warp products in warp 0, quad q <- warp q
        if (q < kFkWarps) { load_row(sW[q], rr, a); f = sF[q] != 0; }
        else { row_identity(rr, a); f = false; }
#pragma unroll
        for (int off = 1; off < kFkWarps; off <<= 1) {
            T y[4];
#pragma unroll
            for (int m = 0; m < 4; ++m) y[m] = shfl_down(a[m], 4 * off);
            const bool yf = __shfl_down_sync(0xffffffffu, f, 4 * off);
            quad_rows(y, base, B);
            if ((q & (2 * off - 1)) == 0) {
                if (yf) { for (int m = 0; m < 4; ++m) a[m] = y[m]; }
                else row_compose(a, B, a);
                f = f || yf;
            }
        }
        __syncwarp();
        if (q == 0 && (lane & 3) < 3) store_row(sW[0], rr, a);
        if (lane == 0) sF[0] = f;
    }
    __syncthreads();
    load_row(sW[0], rr, out);
    of = sF[0] != 0;
    __syncthreads();
}

// link poses M_{h(j)} = (segmented product of the earlier blocks) o G_j, or G_j alone when the
// joint's chain starts in this block (h(j) = j + chain + 1: each chain also owns its fixed base link);
// current axis u_j = R(M_{h(j)}) u0_j (the rotation about u0_j leaves u0_j fixed) through p_j = origin
// of that frame; then the atoms of the block's links, and the bounding box of every chain; the last
// block to finish (ticket, no waiting) sets the chains' grids and their cell bases
template <int J, class T>
__global__ void __launch_bounds__(kFkWarps * 32) k_fk_apply(const DevChain d) {
    grid_dep_sync();
    __shared__ T sW[kFkWarps][12];
    __shared__ int sF[kFkWarps];
    __shared__ int sScan[kFkWarps];
    __shared__ unsigned long long sB[6][kFkWarps];
    __shared__ int sC[kFkWarps];
    __shared__ bool sLast;
    Status* st = d.status;
    if (st->done) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int q = lane >> 2, rr = min(lane & 3, 2), base = lane & ~3;
    const int slot = w * 8 + q;
    const int j0 = (blockIdx.x * kFkQuads + slot) * J;
    T* M = reinterpret_cast<T*>(d.M);
    const T* G = reinterpret_cast<const T*>(d.G);
    // block prefix: the segmented product of the earlier blocks, scanned by the scan kernel's last
    // block, or (few blocks) reduced here in one tree
    T bE[4];
    if (!d.fk_chain_tree) {
        load_row(&reinterpret_cast<const T*>(d.tileE)[12 * (size_t)blockIdx.x], rr, bE);
    } else {  // the products of the blocks from the one where the chain of this block's first joint starts
        const int jb = (int)blockIdx.x * kFkQuads * J;
        const int t0 = d.nchains == 1 ? 0 : d.joint_off[joint_chain(d, jb)] / (kFkQuads * J);
        bool pf;
        block_prefix(d, t0, (int)blockIdx.x, sW, sF, w, q, rr, base, lane, bE, pf);
    }
#pragma unroll
    for (int i = 0; i < J; ++i) {
        const int j = j0 + i;
        if (j < d.l) {  // uniform within the quad; no shuffles here
            T Gj[12], Ma[4];
            load_rows(&G[12 * (size_t)j], Gj);
            if (d.gseg[j]) {
                load_row(&G[12 * (size_t)j], rr, Ma);
            } else {
                row_compose(bE, Gj, Ma);
            }
            if ((lane & 3) < 3) {
                // mixed mode keeps the axes and axis points as double-floats only (the torque kernel's
                // form): no FP64 conversion per joint
                const T* u = reinterpret_cast<const T*>(std::is_same<T, double>::value ? d.u0 : d.u0df) + 3 * j;
                const T uc = fma(Ma[2], u[2], fma(Ma[1], u[1], mul(Ma[0], u[0])));
                store_row(&M[12 * ((size_t)j + joint_chain(d, j) + 1)], rr, Ma);
                if constexpr (std::is_same<T, double>::value) {
                    d.ucur[3 * j + rr] = uc;
                    d.pcur[3 * j + rr] = Ma[3];
                } else {
                    reinterpret_cast<T*>(d.ucurdf)[3 * j + rr] = uc;
                    reinterpret_cast<T*>(d.pcurdf)[3 * j + rr] = Ma[3];
                }
            }
        }
    }
    __syncthreads();  // the block's link poses are visible to the whole block
    // atoms of the block's links: those after the link of the previous block's last joint up to the
    // link of this block's last joint (chains' base links included; their pose is the identity)
    const int jb0 = blockIdx.x * kFkQuads * J, jb1 = min((int)(blockIdx.x + 1) * kFkQuads * J, d.l);
    const int hfirst = blockIdx.x == 0 ? 0 : jb0 + joint_chain(d, jb0 - 1) + 1;
    const int hlast = blockIdx.x == gridDim.x - 1 ? d.L : jb1 + joint_chain(d, jb1 - 1) + 1;
    const int a1 = d.link_start[hlast];
    const T* r0 = reinterpret_cast<const T*>(d.r0fk);
    unsigned long long mn[3] = {~0ULL, ~0ULL, ~0ULL}, mx[3] = {0ULL, 0ULL, 0ULL};
    int cc = -1;  // chain of the keys held in mn, mx
    for (int a = d.link_start[hfirst] + threadIdx.x; a < a1; a += blockDim.x) {
        const int ca = atom_chain(d, a);
        if (ca != cc) {  // a thread's atoms move on to the next chain: hand in the box so far
            if (cc >= 0)
                for (int i = 0; i < 3; ++i) { atomicMin(&d.cbox[6 * cc + i], mn[i]); atomicMax(&d.cbox[6 * cc + 3 + i], mx[i]); }
            cc = ca;
            for (int i = 0; i < 3; ++i) { mn[i] = ~0ULL; mx[i] = 0ULL; }
        }
        const T* Ml = &M[12 * (size_t)d.link[a]];
        const T x = r0[3 * a], y = r0[3 * a + 1], z = r0[3 * a + 2];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const T vt = fma(Ml[3 * i + 2], z, fma(Ml[3 * i + 1], y, fma(Ml[3 * i], x, Ml[9 + i])));
            // bounding box as order-preserving integer keys; mixed mode keeps the centres as double-floats
            // only, keyed as pairs (no FP64 conversion per atom; FP64 centres are formed on request)
            unsigned long long key;
            if constexpr (std::is_same<T, double>::value) {
                d.r[3 * a + i] = vt;
                key = dkey(vt);
            } else {
                reinterpret_cast<T*>(d.rdf)[3 * a + i] = vt;
                key = dfkey(vt);
            }
            mn[i] = min(mn[i], key);
            mx[i] = max(mx[i], key);
        }
    }
    // warps whose threads all hold the same chain reduce first (and the block, when all its warps do);
    // the others hand in lane by lane
    const int cw = __reduce_max_sync(0xffffffffu, cc);
    const bool wuni = __all_sync(0xffffffffu, cc == cw || cc < 0);
    if (wuni) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                mn[i] = min(mn[i], __shfl_down_sync(0xffffffffu, mn[i], o));
                mx[i] = max(mx[i], __shfl_down_sync(0xffffffffu, mx[i], o));
            }
        }
        if (lane == 0)
            for (int i = 0; i < 3; ++i) { sB[i][w] = mn[i]; sB[3 + i][w] = mx[i]; }
    } else if (cc >= 0) {
        for (int i = 0; i < 3; ++i) { atomicMin(&d.cbox[6 * cc + i], mn[i]); atomicMax(&d.cbox[6 * cc + 3 + i], mx[i]); }
    }
    if (lane == 0) sC[w] = wuni ? cw : -2;
    __syncthreads();
    if (threadIdx.x < 6) {
        const int i = threadIdx.x;
        int cb = -1;
        bool buni = true;
        for (int k = 0; k < kFkWarps; ++k) {
            if (sC[k] == -2 || (sC[k] >= 0 && cb >= 0 && sC[k] != cb)) buni = false;
            if (sC[k] >= 0) cb = sC[k];
        }
        if (buni && cb >= 0) {  // one chain in the whole block: one atomic per component
            unsigned long long v = i < 3 ? ~0ULL : 0ULL;
            for (int k = 0; k < kFkWarps; ++k)
                if (sC[k] >= 0) v = i < 3 ? min(v, sB[i][k]) : max(v, sB[i][k]);
            if (i < 3) atomicMin(&d.cbox[6 * cb + i], v);
            else atomicMax(&d.cbox[6 * cb + i], v);
        } else if (!buni) {
            for (int k = 0; k < kFkWarps; ++k) {
                if (sC[k] < 0) continue;
                if (i < 3) atomicMin(&d.cbox[6 * sC[k] + i], sB[i][k]);
                else atomicMax(&d.cbox[6 * sC[k] + i], sB[i][k]);
            }
        }
    }
    if (d.grid_in_bin) return;  // the cluster binning kernel forms the grid from the box
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) sLast = atomicAdd(&st->ticket_bbox, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!sLast) return;
    __threadfence();
    // grids of all chains, one thread per chain; cell bases by a block scan over the chains
    int cbase = 0;
    bool bad = false;
    for (int c0 = 0; c0 < d.nchains; c0 += blockDim.x) {
        const int cch = c0 + threadIdx.x;
        GridInfo g;
        int ncl = 0;
        if (cch < d.nchains) {
            if (!chain_grid_t<T>(d, cch, &g)) {  // non-finite centres: the chain fails (alone, in a batch)
                bad = true;
                d.chain_err[cch] |= kErrNonfinite;
                d.chain_done[cch] = 1;
            }
            ncl = g.ncells;
            d.chain_E[3 * cch] = 0.0; d.chain_E[3 * cch + 1] = 0.0; d.chain_E[3 * cch + 2] = 0.0;
        }
        int v = ncl;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y2 = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y2;
        }
        if (lane == 31) sScan[w] = v;
        __syncthreads();
        int before = 0, total = 0;
        for (int k = 0; k < kFkWarps; ++k) { if (k < w) before += sScan[k]; total += sScan[k]; }
        if (cch < d.nchains) {
            g.cbase = cbase + before + v - ncl;
            d.grid[cch] = g;
        }
        cbase += total;
        __syncthreads();
    }
    const bool bad_any = __syncthreads_or(bad);
    if (bad_any && threadIdx.x == 0) {
        atomicOr(&st->error, kErrNonfinite);
        if (d.nchains == 1) st->done = 1;
    }
    if (threadIdx.x == 0) {
        st->ncells = cbase;
        st->ticket_bbox = 0u;
        st->pairs = 0;
        st->nbr_total = 0;
        st->guard = 0;
        st->sasa_tests = 0;
        st->max_nbr = 0;
        st->nlong = 0;
        if (bad_any && d.nchains == 1) export_status(d);  // the loop ends here: no step block closes it
    }
}

template <int J>
void launch_fk_j(DevChain& d, cudaStream_t s) {
    // the scan kernel's grid: ntiles scan blocks, then the side-chain joints' blocks
    const int nscan = d.ntiles + (d.nmv + kSideFkThreads - 1) / kSideFkThreads;
    const bool tiles = !d.fk_chain_tree;  // the block products scanned by k_fk_tiles
    if (d.prm.precision == KCM_MIXED) {
        launch_k(k_fk_scan<J, df>, nscan, kFkWarps * 32, 0, s, d.pdl, d);
        if (tiles) launch_k(k_fk_tiles<df>, 1, kTileWarps * 32, 0, s, d.pdl, d);
        launch_k(k_fk_apply<J, df>, d.ntiles, kFkWarps * 32, 0, s, d.pdl, d);
    } else {
        launch_k(k_fk_scan<J, double>, nscan, kFkWarps * 32, 0, s, d.pdl, d);
        if (tiles) launch_k(k_fk_tiles<double>, 1, kTileWarps * 32, 0, s, d.pdl, d);
        launch_k(k_fk_apply<J, double>, d.ntiles, kFkWarps * 32, 0, s, d.pdl, d);
    }
}

}  // namespace

// joints per quad: the smallest J that keeps the block count within what the scan kernel's last
// block scans (kFkMaxTiles)
int fk_joints_per_lane(int l) {
    int J = 1;
    while (J < 32 && (l + kFkQuads * J - 1) / (kFkQuads * J) > kFkMaxTiles) J *= 2;
    return J;
}

int fk_block_joints() { return kFkQuads; }

int fk_tree_tiles() { return kFkTreeTiles; }

void launch_centres64(DevChain& d, cudaStream_t s) {
    if (d.prm.precision == KCM_MIXED && d.n > 0) launch_k(k_centres64, (3 * d.n + 255) / 256, 256, 0, s, d.pdl, d);
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
