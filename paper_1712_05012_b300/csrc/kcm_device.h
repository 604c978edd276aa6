// Device-side state of one KCM handle and the launchers of its kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "kcm_internal.h"

namespace kcm {

// Four doubles on a 32-byte boundary (two 16-byte loads).
struct alignas(32) dbl4 {
    double x, y, z, w;
};
__host__ __device__ inline dbl4 make_dbl4(double x, double y, double z, double w) { return dbl4{x, y, z, w}; }

// Uniform binning grid of Sec. 3.2 of one chain, rebuilt on the device every iteration. The cells
// of all chains of a batch are numbered consecutively: chain c owns [cbase, cbase + ncells).
struct GridInfo {
    double ox, oy, oz;  // FP64 mode: the grid origin (bounding-box minimum); mixed mode: 0 (the origin is of)
    double s;           // cell edge, a multiple of 2^-10 A so that it is exact in float
    float sf, inv_sf;   // the edge in float and its reciprocal
    float gpf;          // guard band of the FP32 cutoff tests (A^2), grows with the cell edge
    int nx, ny, nz;
    int ncells;
    int cbase;
    int pad;
    float2 of[3];       // mixed mode: the origin as double-floats (hi, lo); exact, the origin being a centre
};

// Error bits in Status::error.
constexpr int kErrNonfinite = 1;
constexpr int kErrOverflow = 2;
constexpr int kErrTimeout = 4;  // a bounded wait of a kernel on another block gave up

// Device-resident loop state; the host reads it back only when asked.
struct Status {
    unsigned int ticket;  // last-block detection in the step kernel
    unsigned int ticket_bbox;  // last-block detection in the bounding-box kernel
    int iters;            // iterations of the batch loop since the last reset
    int done;             // every chain converged, or failure: the remaining iterations are no-ops
    int error;            // kErr* bits
    int ncells;           // cells of all chains' grids
    double last_max_dtheta;  // largest |dtheta| over the chains stepped in the last iteration
    unsigned long long pairs;
    unsigned long long nbr_total;
    unsigned long long guard;
    unsigned long long sasa_tests;  // overlap tests performed by Algorithm 1 (steps 1 and 2)
    int max_nbr;
    unsigned int ticket_w;  // last-block detection in the wrench / suffix-scan kernel
    unsigned int ticket_bin;  // last-block detection in the cell-count kernel
    int nlong;                // atoms with more than kSasaStage solvation neighbours (long_atoms)
    unsigned int ticket_lb;   // tiles handed out by the torque kernel (from the last one down)
};

// Launch shapes.
// tile shapes of the warp-per-atom kernels (pair kernel; mixed Algorithm 1 or the pairwise solvation
// surrogate): atoms (warps) per block, one of kTileWarps, chosen by kcm_autotune_tiles (default 1: a finished warp's slot is taken
// by the next atom at once instead of waiting for the rest of its block)
constexpr int kTileWarps[3] = {1, 2, 4};
constexpr int kScanCells = 2048;      // cells per block of the cell-count scan
constexpr int kScanThreadsBig = 256;
constexpr int kBinThreads = 1024;     // block of the cell-count kernel (its last block scans small grids)
constexpr int kScanFusedMaxCells = 128 * kBinThreads;  // largest cell array scanned by one block
constexpr double kPairFxInv = 1.0 / 8388608.0;  // unit of the fraction sums of mixed-mode pair forces
constexpr float kPairFxMax = 4194304.0f;        // |pair term| below which it is summed in fixed point (2^22)
constexpr float kPairCoefMax = 1e32f;           // mixed: largest pair force coefficient (kcal/mol/A^2); the
                                                // terms, r x F and their sums then stay below FP32's range
constexpr int kPairFoldRounds = 256;            // pair rounds between folds of the int32 lane sums
constexpr int kPairQueue = 64;                  // ring of in-range candidates per warp of the pair kernel (power of 2)
constexpr int kSasaWarps = 4;
constexpr int kSasaLongBlocks = 32;  // most blocks of the long-list solvation kernels
constexpr int kApplyTpb = 64;
constexpr int kWrenchTileAtoms = 352;  // atoms of 32 links of at most 11 atoms (checked at creation)
constexpr int kSideFkThreads = 128;  // moved side atoms per block of the side-chain kinematics
constexpr int kWrenchWarps = 6;        // warps per 32-link tile of the wrench kernel (one per wrench component in the scan)

struct DevChain {
    int m = 0, n = 0, l = 0, L = 0, N = 0;
    int ls = 0;          // side-chain joints (0 unless kcm_params.side_joints); theta, dtheta, tau and
                         // jfixed hold the l main-chain joints and then the ls side-chain joints
    int nmv = 0;         // atoms moved by side-chain joints
    int fk_j = 1;        // joints per quad (four-lane transform slot) in the transform scan
    int bin_c = 0;       // single chain, mixed mode: CTAs of the cluster kernel that bins the atoms in one
                         // launch (k_bin_cluster); 0: the count and placement kernels
    int bin_capc = 0;    // its cells per CTA in shared memory (a multiple of 4, >= ceil(cell cap / bin_c))
    int ntiles = 0;      // transform-scan blocks of 32 * fk_j joints
    int fk_chain_tree = 0;  // every chain spans at most fk_tree_tiles() scan blocks: each apply block reduces
                            // the block products of its own chain before it (no scan of all of them)
    int grid_in_bin = 0;    // set on the kinematics and binning launches of the step and evaluation graphs when
                            // the cluster kernel bins: it forms the grid from the box (k_fk_apply has no
                            // last-block tail then)
    int ltiles = 0;      // suffix-sum tiles of 32 links
    int wrench_static = 0;  // every wrench block is resident at once: block b takes tile ltiles - 1 - b
                            // (no ticket round trip before its first load)
    int cell_cap = 0;     // cells of all chains' caps
    long long cell_alloc = 0;  // cells the cell arrays hold
    int pair_warps = 1, sasa_warps = 1;  // tile shapes: atoms per block of k_pair and of k_sasa_mixed / k_sasa_pw
    int pair_tile = 0;         // mixed mode: the cell-pair tile kernel (k_pair_tile) instead of the warp-per-atom
                               // kernel; its pair energies and counters go straight to the chain and status totals
    int pdl = 0;               // launches allow programmatic dependent launch (set while the iteration graphs
                               // are captured; every kernel starts with grid_dep_sync)
    int pair_persistent = 0;   // the pair kernel on a persistent grid (one block per resident slot)
    int pair_grid_cap = 0;     // its block count then (SMs x resident blocks per SM); 0: one block per W atoms
    int scan_blocks = 0;
    int scan_fused = 0;  // cell scan by the last block of the count kernel (cell_cap <= kScanFusedMaxCells)
    int stencil = 1;     // cells searched on either side of the home cell: 1 (edge >= largest range) or 2 (>= half of it)
    kcm_params prm{};
    // derived constants
    double rcut2 = 0, rvdw2 = 0;  // squared pair cutoffs
    double rmax = 0;              // largest interaction range (pair cutoffs, solvation neighbour range)
    double roff_max = 0;          // largest offset-sphere radius
    double s_base = 0;            // cell edge before its extent-dependent margin: rmax (1 + 1e-5) + 0.01 A;
                                  // with the two-cell stencil the edge may be half of it
    // the same constants in float for the mixed kernels (no FP64 instruction per warp)
    float f_K = 0, f_w14e = 0, f_w14v = 0, f_rc2 = 0, f_rv2 = 0, f_rall2 = 0, f_dr = 0, f_invN = 0;

    // static data
    double* r0 = nullptr;          // ZP centres relative to their link frame origin [n*3]
    int* link = nullptr;           // [n]
    int* link_start = nullptr;     // [L+1]
    double* u0 = nullptr;          // [l*3]
    double* u0df = nullptr;        // the same as double-float pairs (float hi, lo) for the mixed kernels [l*3]
    double* step0df = nullptr;     // [l*3]
    double* r0df = nullptr;        // [n*3]
    double* r0fk = nullptr;        // the offsets the FK reads: r0 (FP64) or r0df (mixed), or with side-chain
                                   // joints a copy whose moved side atoms k_side_fk rewrites [n*3]
    int* chi_a = nullptr;          // side-chain joint c turns about the bond chi_a -> chi_b [ls]
    int* chi_b = nullptr;          // [ls]
    int* chi_end = nullptr;        // it moves atoms chi_b + 1 .. chi_end - 1 [ls]
    // in the mode's number format (double, or double-float pairs in mixed mode):
    double* chi_p0 = nullptr;      // the bond's first atom in its link frame (ZP) [ls*3]
    double* chi_u0 = nullptr;      // the bond's unit direction in its link frame (ZP) [ls*3]
    double* chi_inv = nullptr;     // 1 / the bond's length [ls]
    int* mv_atom = nullptr;        // atom moved by side-chain joints [nmv]
    int2* mv_chi = nullptr;        // its residue's first side-chain joint, how many joints act on it [nmv]
    int* chi_tile = nullptr;       // side-chain joints of the links of wrench tile t: [chi_tile[t], chi_tile[t+1]) [ltiles+1]
    double* step0 = nullptr;       // link frame steps p0_j - p0_{j-1} [l*3]
    dbl4* aprm64 = nullptr;     // per atom: q, sqrt(eps), R, Roff
    float4* aprm32 = nullptr;      // the same in float
    double* G0 = nullptr;          // 4 pi gamma Roff^2 [n]
    int* gflag = nullptr;          // G0 != 0 [n]
    float* G0f = nullptr;          // G0 in float (mixed-mode energies) [n]
    long long* qfx = nullptr;      // G0 / (N dr) in fixed point [n]
    unsigned long long* exm = nullptr;   // [n]
    unsigned long long* m14m = nullptr;  // [n]
    double* Q64 = nullptr;         // [N*3]
    float* Q32 = nullptr;          // [N*3]
    float4* Q4 = nullptr;          // the same as (x, y, z, 0) [N]

    // per-iteration data
    double* theta = nullptr;       // [l + ls]
    double* dtheta = nullptr;      // [l + ls]
    double* tau = nullptr;         // [l + ls]
    double* G = nullptr;           // pose of link j+1 relative to the first frame of its scan block [l*12]
    double* tileP = nullptr;       // scan block products [ntiles*12]
    double* tileE = nullptr;       // exclusive segmented prefixes of the scan block products [ntiles*12]
    double* M = nullptr;           // link frame poses [L*12] (double-float pairs in mixed mode)
    double* ucur = nullptr;        // current joint axes [l*3]
    double* pcur = nullptr;        // current axis points [l*3]
    double* ucurdf = nullptr;      // mixed mode: the same as double-float pairs [l*3]
    double* pcurdf = nullptr;      // [l*3]
    double* r = nullptr;           // centres [n*3] (mixed mode: formed on request from rdf)
    double* rdf = nullptr;         // mixed mode: centres as double-float pairs [n*3]
    int* key = nullptr;            // cell of each atom [n]
    int* cell_count = nullptr;     // [cell_cap]
    int* cell_start = nullptr;     // [cell_cap+1]
    int* rank = nullptr;           // rank of each atom within its cell [n]
    int* scan_part = nullptr;      // block sums of the cell scan [scan_blocks]
    int* sorted = nullptr;         // slot -> atom [n]
    int* slot_chain = nullptr;     // batches: slot -> chain [n] (the pair kernels' first load, beside the atom)
    int* sorted_tmp = nullptr;     // FP64 mode: slot -> atom in the order of the atomic ranks, before the
                                   // atoms of each cell are put in atom order [n]
    int* slot_cell = nullptr;      // slot -> cell [n]
    ulonglong2* smask = nullptr;   // slot -> bond-class masks (exm, m14m) [n]
    dbl4* spos64 = nullptr;     // sorted centres + charge [n]
    float4* spos32 = nullptr;      // sorted cell-relative offsets + charge [n]
    float4* sprm32 = nullptr;      // sorted sqrt(eps), R, Roff [n]
    dbl4* sprm64 = nullptr;     // [n]
    double* Fpair = nullptr;       // [n*3] (FP64 mode; mixed mode fills it on request)
    long long* Fpx = nullptr;      // mixed mode: pair forces in fixed point, units of 2^-23 [n*3]
    float* Fov = nullptr;          // mixed mode: non-finite pair terms and those of 2^50 or more [n*3]
    long long* Fox = nullptr;      // mixed mode: pair terms of 2^22 .. 2^50, units of 2^-1 (exact) [n*3]
    long long* Fcav = nullptr;     // fixed point [n*3]
    int* nbr_cnt = nullptr;        // [n]
    int* nbr = nullptr;            // [n*kMaxNbr]
    float4* nbr_off = nullptr;     // r_j - r_i and Roff_j^2 [n*kMaxNbr]
    int* covered = nullptr;        // [n]
    int* long_atoms = nullptr;     // atoms with more than kSasaStage solvation neighbours, in any order [n]
    // per-atom results that the wrench kernel sums per chain and per launch (the pair and solvation
    // kernels then need no atomics on shared totals)
    double* epair = nullptr;       // Coulomb and LJ energy of the atom's pairs [n*2] (mixed: a float pair per atom)
    int2* pstat = nullptr;         // pair kernel: pairs counted, guard-band re-decisions [n]
    int2* sstat = nullptr;         // Algorithm 1: overlap tests, guard-band re-decisions [n]
    double* esolv = nullptr;       // pairwise solvation surrogate: energy gamma_i A_i of each atom [n]
    // batches: chain of each atom, joint and link; joint offsets; per-chain cell caps, bounding
    // boxes (order-preserving keys: min x, y, z then max x, y, z), loop state and energies
    int nchains = 1;
    int* atom_chain = nullptr;     // [n]
    int* joint_chain = nullptr;    // [l]
    int* link_chain = nullptr;     // [L]
    int* joint_off = nullptr;      // [nchains + 1]
    int* atom_off = nullptr;       // batches in mixed mode: first atom of each chain [nchains + 1]
    int* ccap = nullptr;           // [nchains]
    unsigned long long* cbox = nullptr;       // [nchains * 6]
    int* chain_done = nullptr;     // converged (the chain takes no more steps) [nchains]
    int* chain_iters = nullptr;    // [nchains]
    int* chain_maxit = nullptr;    // iterations a chain may take per step call (<= 0: none) [nchains]
    int* chain_err = nullptr;      // kErr* bits of a chain; in a batch a failed chain stops alone [nchains]
    unsigned long long* chain_maxdt = nullptr;   // bits of max |dtheta| of the running iteration
    unsigned long long* chain_maxtau = nullptr;  // bits of max |tau| of the running iteration
    double* chain_lastdt = nullptr;              // max |dtheta| of the chain's last step
    double* chain_E = nullptr;     // Coulomb, LJ, solvation energies [nchains * 3]
    unsigned char* jhead = nullptr;  // the joint is the first of its chain [l]
    unsigned char* jfixed = nullptr; // the joint is held fixed: it takes no step (kcm_set_fixed_joints) [l + ls]
    unsigned char* lflag = nullptr;  // 1: a chain's base link (no joint), 2: the last link of a chain [L]
    unsigned char* gseg = nullptr; // FK: a chain starts in the joint's scan block at or before it [l]
    int* tileF = nullptr;          // FK: a chain starts in the scan block [ntiles]
    int* tileT = nullptr;          // torques: a chain ends in the tile [ltiles]
    double* tileS = nullptr;       // tile sums [ltiles*6]
    unsigned int* tileStat = nullptr;  // torque kernel: launch number with which the tile's total was
                                       // published (k_wrench_step waits for it) [ltiles]
    unsigned int* lb_epoch = nullptr;  // the torque kernel's launch number (never reset)
    int lb_withhold = -1;              // test only (kcm_set_test_withhold): a tile whose total is never
                                       // published, so that the waits on it time out
    double* Ftot = nullptr;        // [n*3] (on request)
    double* Fcav64 = nullptr;      // [n*3] (on request)
    GridInfo* grid = nullptr;      // [nchains]
    Status* status = nullptr;
    // Host exchange of kcm_step_host (device addresses of page-locked, mapped host memory; null in every
    // other graph): the first iteration's transform scan takes the main-chain angles from theta_io
    // (io_import) into theta, every step writes the angles it changes back to both, and the status record
    // goes to status_io when an iteration's last update of it is made (the step's last block, or the
    // kinematics when they end the loop), so that the call reads theta and its outcome without copies.
    double* theta_io = nullptr;    // [l]
    Status* status_io = nullptr;
    int io_import = 0;
};
static_assert(sizeof(Status) % 8 == 0, "the status record is exported in 8-byte words");

// launchers (kcm_kernels.cu)
void launch_init_status(DevChain& d, cudaStream_t s);
void launch_reset_loop(DevChain& d, cudaStream_t s);
void launch_fk(DevChain& d, cudaStream_t s);
// the FP64 centres r from the double-float ones (mixed mode keeps only those); nothing in FP64 mode
void launch_centres64(DevChain& d, cudaStream_t s);
void launch_binning(DevChain& d, cudaStream_t s);  // with bin_c: k_bin_cluster
void launch_bin_cluster(DevChain& d, cudaStream_t s);  // kcm_bin_cluster.cu
// the cluster shape of k_bin_cluster for the chain and its cell cap (bin_c, bin_capc; bin_c = 0 when not
// wanted, when the chain does not qualify or when no such cluster fits the device)
cudaError_t plan_bin_cluster(DevChain& d, bool want);
void launch_pairs(DevChain& d, cudaStream_t s);
void launch_pairs_tile(DevChain& d, cudaStream_t s);  // kcm_pair_tile.cu
int pair_tile_rows(int stencil);                      // warps per window of 32 slots of k_pair_tile
int pair_resident_blocks(const DevChain& d);  // resident blocks per SM of the current pair kernel (-1: error)
int wrench_resident_blocks(const DevChain& d);  // resident blocks per SM of the wrench kernels (-1: error)
void launch_sasa(DevChain& d, cudaStream_t s);
void launch_sasa_long(DevChain& d, cudaStream_t s);  // atoms with more than kSasaStage neighbours
void launch_torques(DevChain& d, cudaStream_t s);
void launch_torques_step(DevChain& d, cudaStream_t s);
int fk_joints_per_lane(int l);
int fk_block_joints();  // quads per transform-scan block
int fk_tree_tiles();    // most block products an apply block reduces itself
void launch_force_out(DevChain& d, cudaStream_t s);

}  // namespace kcm
