// Internal declarations of the KCM library (host builder, constants shared by host and device).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "kcm.h"

namespace kcm {

// Fixed-point scale of the solvation force accumulators: one unit is 2^-40 kcal mol^-1 A^-1.
// int64 then spans +-8.4e6 kcal mol^-1 A^-1, and integer addition makes the sum order-free.
constexpr double kFxScale = 1099511627776.0;  // 2^40
constexpr double kFxInv = 1.0 / 1099511627776.0;

// Largest solvation neighbour list per atom; more raises KCM_E_OVERFLOW. At protein-like packing
// (about 0.1 atoms per A^3 with hydrogens) the solvation range of an atom (Roff_i + Roff_j + dr, up to
// ~6.8 A) holds about 130 atoms; chains that the iteration packs more densely reach a little over 256
// (one served job in several hundred after 200 iterations), hence half as much room again. Lists up to
// kSasaStage are staged in shared memory by Algorithm 1's kernels; longer ones are read from global memory.
constexpr int kMaxNbr = 384;
constexpr int kSasaStage = 128;

// Largest sample count per offset sphere.
constexpr int kMaxSample = 4096;

// Mixed handles of at least this many atoms start with the cell-pair tile kernel, smaller ones with the
// warp-per-atom kernel. The tile kernel's warps (one per 32 sorted slots and stencil row) fill the SMs
// only on large inputs: measured on a B300, 26.6 against 36.5 us on 10,506 atoms, about equal on
// 83,746, 2.03 against 2.5 ms on 1.63 M atoms (the pair-kernel autotuner decides per handle).
constexpr int kPairTileDefaultAtoms = 65536;

// Bond classes are stored as two 64-bit masks per atom `lo`: bit d set means the pair
// (lo, lo + d) is excluded (1-2 / 1-3) or is a 1-4 pair. Pairs within three bonds always lie
// within this window for the chains built here (checked at build time).
constexpr int kMaskWindow = 63;

struct HostChain {
    int m = 0, n = 0, l = 0, L = 0;  // residues, atoms, joints, links (L = l + 1)
    std::vector<double> zp;          // ZP centres [n*3]
    std::vector<int> link;           // link of each atom [n]
    std::vector<int> link_start;     // first atom of each link [L+1]
    std::vector<int> parent;         // bond-tree parent (root N_1: -1) [n]
    std::vector<int> kind;           // 0 N, 1 H, 2 CA, 3 C, 4 O, 5 side
    std::vector<double> q, eps, R;   // per atom (R = sigma / 2)
    std::vector<int> cls;            // solvation class
    std::vector<double> u0;          // ZP joint axis directions [l*3]
    std::vector<double> step0;       // frame step: axis point of joint j minus that of joint j-1 [l*3]
    std::vector<double> zp_rel;      // ZP offset of each atom from its link frame origin [n*3]
    std::vector<uint64_t> ex_mask, m14_mask;  // bond-class masks [n]
    // side-chain joints (eq. kin_05, r2), residue by residue: joint c turns about the bond
    // chi_a[c] -> chi_b[c] (CA or side atom k - 2 -> side atom k - 1) and moves atoms
    // chi_b[c] + 1 .. chi_end[c] - 1 (the side atoms beyond it); chi_p0 / chi_u0 give the bond's first
    // atom and unit direction in the frame of the residue's CA link (the frame of zp_rel)
    int ls = 0;
    std::vector<int> chi_a, chi_b, chi_end;  // [ls]
    std::vector<double> chi_p0, chi_u0;      // [ls*3]
    std::vector<double> chi_inv;             // 1 / bond length (the kinematics keep it) [ls]
    // atoms that side-chain joints move: the atom, the first joint of its residue, how many act on it
    std::vector<int> mv_atom, mv_chi0, mv_nk;
    // a batch of chains is their concatenation (atoms, links and joints in chain order); chain c
    // owns atoms [atom_off[c], atom_off[c+1]), joints [joint_off[c], ...) and links [link_off[c], ...)
    int nchains = 1;
    std::vector<int> atom_off, joint_off, link_off;  // [nchains + 1]
    std::vector<int> side_off;                       // side-chain joints of chain c [nchains + 1]
};

double gamma_of_class(int cls);
int build_host_chain(const kcm_topology* top, HostChain* hc, std::string* err);
// the batch of the given chains (each built by build_host_chain) in order
void concat_chains(const std::vector<HostChain>& parts, HostChain* out);
int bond_class_tree(const HostChain& hc, int a, int b);  // 0 far, 1 excluded, 2 1-4
int sample_points(int N, double* Q);
int validate_params(const kcm_params* p, std::string* err);

}  // namespace kcm
