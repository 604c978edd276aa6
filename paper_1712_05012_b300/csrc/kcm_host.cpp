// Host-side construction of a chain for the KCM engine: ZP geometry, rigid-link layout, joint
// axes, bond-class masks, solvation constants and the unit-sphere sample set.
//
// Geometry (Sec. 2.1, Sec. 4.1 "Preprocessing"): the zero position (ZP) has every peptide plane
// coplanar, phi = psi = 180 deg (theta = 0, eq. theta_1/theta_2) and trans peptide bonds. Atoms
// are placed one at a time from their bond length, bond angle and dihedral relative to three
// already-placed atoms (natural extension reference frame).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "kcm_internal.h"

namespace kcm {

namespace {

constexpr double kPi = 3.14159265358979323846;

struct V3 {
    double x, y, z;
};
inline V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 operator*(double s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
inline V3 unit(V3 a) { return (1.0 / std::sqrt(dot(a, a))) * a; }

// Place D with |CD| = len, angle(B, C, D) = ang and IUPAC dihedral(A, B, C, D) = dih.
V3 place(V3 A, V3 B, V3 C, double len, double ang, double dih) {
    V3 bc = unit(C - B);
    V3 nrm = unit(cross(B - A, bc));
    V3 mid = cross(nrm, bc);
    double dx = -len * std::cos(ang);
    double dy = len * std::sin(ang) * std::cos(dih);
    double dz = len * std::sin(ang) * std::sin(dih);
    return C + dx * bc + dy * mid + dz * nrm;
}

double rad(double deg) { return deg * kPi / 180.0; }

}  // namespace

// Table 3 (Sharp et al. adjustment), kcal mol^-1 A^-2; H (not in the table) gets 0.
double gamma_of_class(int cls) {
    static const double g[6] = {0.012, -0.116, -0.018, -0.175, -0.186, 0.0};
    return (cls >= 0 && cls < 6) ? g[cls] : 0.0;
}

int validate_params(const kcm_params* p, std::string* err) {
    if (!p) { *err = "params is NULL"; return KCM_E_INVAL; }
    if (!(p->cutoff > 0.0) || !(p->vdw_cutoff >= 0.0) || !(p->kappa >= 0.0) || !(p->dtheta_max > 0.0) ||
        !(p->r_probe >= 0.0) || !(p->delta_r > 0.0) || !(p->conv_tol >= 0.0) || !(p->cell_size >= 0.0) ||
        !std::isfinite(p->coulomb_k) || !std::isfinite(p->w14_elec) || !std::isfinite(p->w14_vdw) ||
        !std::isfinite(p->cutoff) || !std::isfinite(p->vdw_cutoff) || !std::isfinite(p->cell_size)) {
        *err = "a parameter is out of range";
        return KCM_E_INVAL;
    }
    if (p->n_sample < 1 || p->n_sample > kMaxSample) { *err = "n_sample must be in [1, 4096]"; return KCM_E_INVAL; }
    if (p->precision != KCM_FP64 && p->precision != KCM_MIXED) { *err = "bad precision"; return KCM_E_INVAL; }
    if (p->step_mode != KCM_STEP_CLAMP && p->step_mode != KCM_STEP_NORMALIZED) { *err = "bad step_mode"; return KCM_E_INVAL; }
    if (p->solvation < 0 || p->solvation > 2) { *err = "solvation must be 0, 1 or 2"; return KCM_E_INVAL; }
    if (p->side_joints != 0 && p->side_joints != 1) { *err = "side_joints must be 0 or 1"; return KCM_E_INVAL; }
    return KCM_OK;
}

// Latitude-ring sample set of Sec. 3.4 (see kcm_sample_points in kcm.h for the recipe).
int sample_points(int N, double* Q) {
    if (N < 1) return KCM_E_INVAL;
    int K = static_cast<int>(std::floor(std::sqrt(kPi * static_cast<double>(N) / 4.0) + 0.5));
    if (K < 1) K = 1;
    std::vector<double> wt(K), frac(K);
    std::vector<int> cnt(K);
    double total = 0.0;
    for (int r = 1; r <= K; ++r) {
        wt[r - 1] = std::sin(kPi * (static_cast<double>(r) - 0.5) / static_cast<double>(K));
        total += wt[r - 1];
    }
    int given = 0;
    for (int r = 0; r < K; ++r) {
        double share = static_cast<double>(N) * wt[r] / total;
        cnt[r] = static_cast<int>(std::floor(share));
        frac[r] = share - std::floor(share);
        given += cnt[r];
    }
    while (given < N) {  // largest remainder first, lower ring on ties
        int pick = 0;
        for (int r = 1; r < K; ++r)
            if (frac[r] > frac[pick]) pick = r;
        cnt[pick] += 1;
        frac[pick] = -1.0;
        ++given;
    }
    int k = 0;
    for (int r = 1; r <= K; ++r) {
        double polar = kPi * (static_cast<double>(r) - 0.5) / static_cast<double>(K);
        for (int t = 0; t < cnt[r - 1]; ++t) {
            double lon = 2.0 * kPi * (static_cast<double>(t) + 0.5 * static_cast<double>(r % 2)) /
                         static_cast<double>(cnt[r - 1]);
            Q[3 * k + 0] = std::sin(polar) * std::cos(lon);
            Q[3 * k + 1] = std::sin(polar) * std::sin(lon);
            Q[3 * k + 2] = std::cos(polar);
            ++k;
        }
    }
    return KCM_OK;
}

// Bond class from parent pointers on the bond tree rooted at N_1 (Sec. 3.3): 1-2 when one atom
// is the other's parent; 1-3 when grandparent or sibling; 1-4 when great-grandparent or a
// sibling of the parent. Returns 1 for 1-2/1-3 (excluded), 2 for 1-4, 0 otherwise.
int bond_class_tree(const HostChain& hc, int a, int b) {
    const std::vector<int>& P = hc.parent;
    auto up = [&](int x, int k) {
        for (int i = 0; i < k && x >= 0; ++i) x = P[x];
        return x;
    };
    auto one_way = [&](int x, int y) -> int {
        if (P[x] == y) return 1;                                        // one bond
        if (up(x, 2) == y || (P[x] >= 0 && P[x] == P[y])) return 2;     // two bonds
        int gp = up(x, 2);
        if (up(x, 3) == y || (gp >= 0 && P[y] == gp && y != P[x])) return 3;  // three bonds
        return 9;
    };
    if (a == b) return 1;
    int len = std::min(one_way(a, b), one_way(b, a));
    if (len <= 2) return 1;
    if (len == 3) return 2;
    return 0;
}

int build_host_chain(const kcm_topology* top, HostChain* hc, std::string* err) {
    if (!top || top->n_res < 1 || top->n_types < 1 || !top->res_type || !top->types) {
        *err = "topology is empty or has NULL arrays";
        return KCM_E_INVAL;
    }
    kcm_geometry g;
    if (top->geometry) {
        g = *top->geometry;
    } else {
        g = kcm_geometry{1.458, 1.525, 1.329, 1.231, 1.0, 1.53, 111.2, 116.2, 121.7, 120.8, 109.47122063449069};
    }
    const int m = top->n_res;
    std::vector<int> first(m), nside(m);
    long long n = 0;
    for (int i = 0; i < m; ++i) {
        int t = top->res_type[i];
        if (t < 0 || t >= top->n_types) { *err = "residue type out of range"; return KCM_E_INVAL; }
        int k = top->types[t].n_side;
        if (k < 1 || k > KCM_MAX_SIDE) { *err = "side group size must be 1..10"; return KCM_E_INVAL; }
        first[i] = static_cast<int>(n);
        nside[i] = k;
        n += 5 + k;
        if (n > (1LL << 28)) { *err = "chain too long"; return KCM_E_INVAL; }
    }
    hc->m = m;
    hc->n = static_cast<int>(n);
    hc->l = 2 * m;
    hc->L = 2 * m + 1;
    hc->zp.assign(3 * n, 0.0);
    hc->link.assign(n, 0);
    hc->parent.assign(n, -1);
    hc->kind.assign(n, 0);
    hc->q.assign(n, 0.0);
    hc->eps.assign(n, 0.0);
    hc->R.assign(n, 0.0);
    hc->cls.assign(n, 0);
    auto iN = [&](int i) { return first[i]; };
    auto iH = [&](int i) { return first[i] + 1; };
    auto iCA = [&](int i) { return first[i] + 2; };
    auto iS = [&](int i, int t) { return first[i] + 3 + t; };
    auto iC = [&](int i) { return first[i] + 3 + nside[i]; };
    auto iO = [&](int i) { return first[i] + 4 + nside[i]; };

    // constants, links and bond-tree parents
    for (int i = 0; i < m; ++i) {
        const kcm_restype& rt = top->types[top->res_type[i]];
        auto setp = [&](int a, const kcm_atom_param& ap, int kind, int lnk, int par) {
            if (!(ap.sigma > 0.0) || !(ap.eps >= 0.0) || !std::isfinite(ap.q) || !std::isfinite(ap.sigma) ||
                !std::isfinite(ap.eps) || ap.solv_class < 0 || ap.solv_class > 5)
                return false;
            hc->q[a] = ap.q;
            hc->eps[a] = ap.eps;
            hc->R[a] = 0.5 * ap.sigma;
            hc->cls[a] = ap.solv_class;
            hc->kind[a] = kind;
            hc->link[a] = lnk;
            hc->parent[a] = par;
            return true;
        };
        int pep_prev = (i == 0) ? 0 : 2 * i;  // link holding N_i, H_i
        bool ok = setp(iN(i), rt.backbone[0], 0, pep_prev, i == 0 ? -1 : iC(i - 1));
        ok = ok && setp(iH(i), rt.backbone[1], 1, pep_prev, iN(i));
        ok = ok && setp(iCA(i), rt.backbone[2], 2, 2 * i + 1, iN(i));
        for (int t = 0; t < nside[i]; ++t) ok = ok && setp(iS(i, t), rt.side[t], 5, 2 * i + 1, t == 0 ? iCA(i) : iS(i, t - 1));
        ok = ok && setp(iC(i), rt.backbone[3], 3, 2 * i + 2, iCA(i));
        ok = ok && setp(iO(i), rt.backbone[4], 4, 2 * i + 2, iC(i));
        if (!ok) { *err = "atom constants out of range (sigma > 0, eps >= 0, class 0..5)"; return KCM_E_INVAL; }
    }
    hc->link_start.assign(hc->L + 1, 0);
    for (int a = 0, h = 0; a < hc->n; ++a) {
        if (a > 0 && hc->link[a] < hc->link[a - 1]) { *err = "internal: links are not contiguous"; return KCM_E_INVAL; }
        while (h <= hc->link[a]) hc->link_start[h++] = a;
    }
    hc->link_start[hc->L] = hc->n;

    // ZP, residue by residue, in a frame re-centred on each residue's N: every stored vector is
    // short (atom offsets from N_i, the step N_i -> N_{i+1}), so nothing is recovered by
    // subtracting coordinates of a ~3.8 A-per-residue extended chain.
    std::vector<V3> loc(n, V3{0, 0, 0});
    std::vector<V3> nstep(m, V3{0, 0, 0});
    const double a_ncac = rad(g.a_n_ca_c), a_cacn = rad(g.a_ca_c_n), a_cnca = rad(g.a_c_n_ca), a_caco = rad(g.a_ca_c_o);
    const double a_side = rad(g.a_side), a_h = rad((360.0 - g.a_c_n_ca) / 2.0);
    V3 pN{0, 0, 0}, pCA{0, 0, 0}, pC{0, 0, 0};  // previous residue's N, CA, C relative to its N
    for (int i = 0; i < m; ++i) {
        V3 N{0, 0, 0}, CA, C, H;
        if (i == 0) {
            CA = V3{g.b_n_ca, 0.0, 0.0};
            C = CA + g.b_ca_c * V3{std::cos(kPi - a_ncac), std::sin(kPi - a_ncac), 0.0};
            H = place(C, CA, N, g.b_n_h, a_h, 0.0);
        } else {
            V3 Nn = place(pN, pCA, pC, g.b_c_n, a_cacn, kPi);     // psi = 180
            V3 CAn = place(pCA, pC, Nn, g.b_n_ca, a_cnca, kPi);   // omega = 180
            V3 Cn = place(pC, Nn, CAn, g.b_ca_c, a_ncac, kPi);    // phi = 180
            nstep[i - 1] = Nn;
            pCA = pCA - Nn;
            pC = pC - Nn;
            CA = CAn - Nn;
            C = Cn - Nn;
            H = place(pCA, pC, N, g.b_n_h, a_h, 0.0);
        }
        loc[iN(i)] = N;
        loc[iH(i)] = H;
        loc[iCA(i)] = CA;
        loc[iC(i)] = C;
        loc[iO(i)] = place(N, CA, C, g.b_c_o, a_caco, 0.0);
        // CB: the N-CA-C bisector (pointing away from N and C), turned by half the side angle
        // toward n x c, which gives the L configuration
        V3 nh = unit(N - CA);
        V3 ch = unit(C - CA);
        V3 bis = unit(-1.0 * (nh + ch));
        V3 w = unit(cross(nh, ch));
        loc[iS(i, 0)] = CA + g.b_side * (std::cos(0.5 * a_side) * bis + std::sin(0.5 * a_side) * w);
        V3 A = N, B = CA, D = loc[iS(i, 0)];
        for (int t = 1; t < nside[i]; ++t) {
            V3 E = place(A, B, D, g.b_side, a_side, kPi);
            loc[iS(i, t)] = E;
            A = B;
            B = D;
            D = E;
        }
        pN = N;
        pCA = CA;
        pC = C;
    }
    if (m > 0) nstep[m - 1] = place(pN, pCA, pC, g.b_c_n, a_cacn, kPi);  // where N_{m+1} would be
    // absolute ZP centres (reported by kcm_build_zp only)
    V3 Nabs{0, 0, 0};
    for (int i = 0; i < m; ++i) {
        for (int a = iN(i); a <= iO(i); ++a) {
            V3 x = Nabs + loc[a];
            hc->zp[3 * (size_t)a] = x.x;
            hc->zp[3 * (size_t)a + 1] = x.y;
            hc->zp[3 * (size_t)a + 2] = x.z;
        }
        Nabs = Nabs + nstep[i];
    }
    // joint axes and local link frames: link 2i+1 (CA_i, side) has its origin at N_i on the phi_i
    // axis, link 2i+2 (C_i, O_i, N_{i+1}, H_{i+1}) at CA_i on the psi_i axis, the base link at N_1
    hc->u0.assign(3 * hc->l, 0.0);
    hc->step0.assign(3 * hc->l, 0.0);
    hc->zp_rel.assign(3 * n, 0.0);
    auto put = [](std::vector<double>& v, long long k, V3 x) {
        v[3 * k] = x.x;
        v[3 * k + 1] = x.y;
        v[3 * k + 2] = x.z;
    };
    for (int i = 0; i < m; ++i) {
        put(hc->u0, 2 * i, unit(loc[iCA(i)]));
        put(hc->u0, 2 * i + 1, unit(loc[iC(i)] - loc[iCA(i)]));
        put(hc->step0, 2 * i, i == 0 ? V3{0, 0, 0} : nstep[i - 1] - loc[iCA(i - 1)]);  // CA_{i-1} -> N_i
        put(hc->step0, 2 * i + 1, loc[iCA(i)]);                                          // N_i -> CA_i
        if (i == 0) {
            put(hc->zp_rel, iN(0), loc[iN(0)]);
            put(hc->zp_rel, iH(0), loc[iH(0)]);
        }
        put(hc->zp_rel, iCA(i), loc[iCA(i)]);
        for (int t = 0; t < nside[i]; ++t) put(hc->zp_rel, iS(i, t), loc[iS(i, t)]);
        put(hc->zp_rel, iC(i), loc[iC(i)] - loc[iCA(i)]);
        put(hc->zp_rel, iO(i), loc[iO(i)] - loc[iCA(i)]);
        if (i + 1 < m) {
            put(hc->zp_rel, iN(i + 1), nstep[i] - loc[iCA(i)]);
            put(hc->zp_rel, iH(i + 1), nstep[i] + loc[iH(i + 1)] - loc[iCA(i)]);
        }
    }
    // side-chain joints: chi_k of residue i (k = 1 .. min(4, nside - 1)) about the ZP bond from CA
    // (k = 1) or side atom k - 2 to side atom k - 1, in the frame of link 2i+1 (origin N_i, where
    // zp_rel of CA and the side atoms is loc)
    for (int i = 0; i < m; ++i) {
        const int nchi = std::min(4, nside[i] - 1);
        const int c0 = hc->ls;
        for (int k = 1; k <= nchi; ++k) {
            const int a = k == 1 ? iCA(i) : iS(i, k - 2), b = iS(i, k - 1);
            const V3 ab = loc[b] - loc[a];
            const V3 u = unit(ab);
            hc->chi_inv.push_back(1.0 / std::sqrt(dot(ab, ab)));
            hc->chi_a.push_back(a);
            hc->chi_b.push_back(b);
            hc->chi_end.push_back(iS(i, 0) + nside[i]);
            hc->chi_p0.insert(hc->chi_p0.end(), {loc[a].x, loc[a].y, loc[a].z});
            hc->chi_u0.insert(hc->chi_u0.end(), {u.x, u.y, u.z});
            ++hc->ls;
        }
        for (int s = 1; s < nside[i] && nchi > 0; ++s) {  // side atom s turns with chi_1 .. chi_min(s, nchi)
            hc->mv_atom.push_back(iS(i, s));
            hc->mv_chi0.push_back(c0);
            hc->mv_nk.push_back(std::min(s, nchi));
        }
    }
    hc->side_off = {0, hc->ls};
    // bond-class masks over the window (lo, lo + d), d = 1..63, from a breadth-first walk of at most
    // three bonds out of every atom over the bond tree (parent and children): pairs one or two bonds
    // apart are excluded, three bonds apart are 1-4; every such pair must fall inside the window (a
    // pair with a residue gap of two or more is never that close)
    hc->ex_mask.assign(n, 0);
    hc->m14_mask.assign(n, 0);
    std::vector<int> coff(n + 1, 0), kids(n > 0 ? n - 1 : 0);
    for (int a = 0; a < hc->n; ++a)
        if (hc->parent[a] >= 0) ++coff[hc->parent[a] + 1];
    for (int a = 0; a < hc->n; ++a) coff[a + 1] += coff[a];
    {
        std::vector<int> fill(coff.begin(), coff.end() - 1);
        for (int a = 0; a < hc->n; ++a)
            if (hc->parent[a] >= 0) kids[fill[hc->parent[a]]++] = a;
    }
    int frontier[2][64], nf[2];
    for (int a = 0; a < hc->n; ++a) {
        // depth 1..3 from a, never stepping back to the atom it came from (the graph is a tree)
        int from[2][64];
        nf[0] = 1;
        frontier[0][0] = a;
        from[0][0] = -1;
        for (int depth = 1; depth <= 3; ++depth) {
            const int cur = (depth - 1) & 1, nxt = depth & 1;
            nf[nxt] = 0;
            for (int k = 0; k < nf[cur]; ++k) {
                const int x = frontier[cur][k], back = from[cur][k];
                auto visit = [&](int y) {
                    if (y == back || nf[nxt] >= 64) return;
                    frontier[nxt][nf[nxt]] = y;
                    from[nxt][nf[nxt]] = x;
                    ++nf[nxt];
                    if (y > a) {
                        const int d = y - a;
                        if (d > kMaskWindow) return;  // reported below
                        if (depth <= 2) hc->ex_mask[a] |= (1ULL << d);
                        else hc->m14_mask[a] |= (1ULL << d);
                    }
                };
                if (hc->parent[x] >= 0) visit(hc->parent[x]);
                for (int c = coff[x]; c < coff[x + 1]; ++c) visit(kids[c]);
            }
            for (int k = 0; k < nf[nxt]; ++k)
                if (frontier[nxt][k] - a > kMaskWindow) {
                    *err = "internal: bonded pair outside the class window";
                    return KCM_E_INVAL;
                }
        }
    }
    return KCM_OK;
}

void concat_chains(const std::vector<HostChain>& parts, HostChain* out) {
    HostChain& b = *out;
    b = HostChain();
    b.nchains = static_cast<int>(parts.size());
    b.atom_off.assign(1, 0);
    b.joint_off.assign(1, 0);
    b.link_off.assign(1, 0);
    b.side_off.assign(1, 0);
    for (const HostChain& p : parts) {
        const int a0 = b.n, h0 = b.L, c0 = b.ls;
        b.m += p.m;
        b.n += p.n;
        b.l += p.l;
        b.L += p.L;
        b.atom_off.push_back(b.n);
        b.joint_off.push_back(b.l);
        b.link_off.push_back(b.L);
        for (int c = 0; c < p.ls; ++c) {
            b.chi_a.push_back(p.chi_a[c] + a0);
            b.chi_b.push_back(p.chi_b[c] + a0);
            b.chi_end.push_back(p.chi_end[c] + a0);
        }
        b.chi_p0.insert(b.chi_p0.end(), p.chi_p0.begin(), p.chi_p0.end());
        b.chi_u0.insert(b.chi_u0.end(), p.chi_u0.begin(), p.chi_u0.end());
        b.chi_inv.insert(b.chi_inv.end(), p.chi_inv.begin(), p.chi_inv.end());
        for (size_t k = 0; k < p.mv_atom.size(); ++k) {
            b.mv_atom.push_back(p.mv_atom[k] + a0);
            b.mv_chi0.push_back(p.mv_chi0[k] + c0);
            b.mv_nk.push_back(p.mv_nk[k]);
        }
        b.ls += p.ls;
        b.side_off.push_back(b.ls);
        b.zp.insert(b.zp.end(), p.zp.begin(), p.zp.end());
        for (int a = 0; a < p.n; ++a) {
            b.link.push_back(p.link[a] + h0);
            b.parent.push_back(p.parent[a] < 0 ? -1 : p.parent[a] + a0);
        }
        for (int h = 0; h < p.L; ++h) b.link_start.push_back(p.link_start[h] + a0);
        b.kind.insert(b.kind.end(), p.kind.begin(), p.kind.end());
        b.q.insert(b.q.end(), p.q.begin(), p.q.end());
        b.eps.insert(b.eps.end(), p.eps.begin(), p.eps.end());
        b.R.insert(b.R.end(), p.R.begin(), p.R.end());
        b.cls.insert(b.cls.end(), p.cls.begin(), p.cls.end());
        b.u0.insert(b.u0.end(), p.u0.begin(), p.u0.end());
        b.step0.insert(b.step0.end(), p.step0.begin(), p.step0.end());
        b.zp_rel.insert(b.zp_rel.end(), p.zp_rel.begin(), p.zp_rel.end());
        // masks hold bits for partners at index offsets within the same chain, unchanged by the shift
        b.ex_mask.insert(b.ex_mask.end(), p.ex_mask.begin(), p.ex_mask.end());
        b.m14_mask.insert(b.m14_mask.end(), p.m14_mask.begin(), p.m14_mask.end());
    }
    b.link_start.push_back(b.n);
}

}  // namespace kcm
