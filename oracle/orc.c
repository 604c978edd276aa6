/*
 * KCM oracle — TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously-correct FP64 CPU statement of one iteration of the kinetostatic
 * compliance method (KCM) of Protofold II (Behandish & Ilies, arXiv 1712.05012). Only the test
 * suite, the package smoke check and the CPU-baseline leg of the benchmark call it; the CUDA
 * library neither links nor calls it, and it includes none of the library's headers.
 *
 * What it computes, in the paper's order and notation:
 *   - zero position (ZP) chain geometry (Sec. 2.1, Sec. 4.1 "Preprocessing"): planar extended
 *     backbone built by turning angles in the xy-plane, side groups by Rodrigues rotations;
 *   - forward kinematics exactly in the paper's form: M_j = R_1 ... R_j about the ZP axes
 *     (eq. kin_04), body vectors b = M b^0 (eq. kin_03), atom centres as prefix sums of body
 *     vectors (eq. r1, r2);
 *   - pairwise Coulomb with distance-dependent dielectric and Lennard-Jones 6-12 over ALL pairs,
 *     O(n^2), classified 1-2 / 1-3 / 1-4 by breadth-first search on the bond graph (eq. 02_2,
 *     03_2, 03_8, 03_9; Sec. 3.3);
 *   - solvation by surface enumeration, Algorithm 1 with the three-state count rules (Sec. 3.4),
 *     neighbour candidates found by an all-pairs scan; and a definition-level brute-force
 *     recount of f_{i,j,s} (eq. finitediff, F_cav_patch) for tiny inputs;
 *   - link wrenches (eq. KCM_01, KCM_02) and joint torques as the O(l^2) column sums of the
 *     matrix eq. 04_9, plus the row-scan (suffix sum) form of Sec. 3.5 for comparison;
 *   - the kinetostatic step (eq. KCM_07) in the per-joint clamped form and the normalised form.
 *
 * Readings of the paper used here (the CUDA library takes the same ones):
 *   energies sum unordered pairs once; F = -grad E with eps = 4 d, so the Coulomb force is
 *   K q_i q_j / (2 d^3) along e_ij; a single cutoff (optionally a separate LJ cutoff), d <= r_c
 *   included; w = 0 for 1-2 and 1-3 pairs, w14 for pairs exactly 3 bonds apart, 1 otherwise;
 *   R_i = sigma_i / 2; Algorithm 1's dagger lines update F_j (not F_i) and step 2 tests every
 *   neighbour (no break) unless `literal_break` asks for the printed break; the torque centre
 *   of every link is the origin, so J_k = [u_k ; p_k x u_k]; the sample set is the polar
 *   latitude-ring recipe documented at orc_sample_points.
 *
 * Pins (tests/test_oracle_*.py, all run without a GPU): bond lengths/angles kept under FK,
 * IUPAC dihedrals equal theta - pi, L chirality of CB, extended-chain closed forms; F = -grad E
 * by central differences; Newton's third law and zero net moment; LJ minimum at d = D with depth
 * eps; Coulomb 1/d^2 scaling; torques = -dE/dtheta by central differences; column form equals
 * row-scan form; isolated sphere exposure 1; two-sphere cap area convergence; Algorithm 1 equals
 * the brute-force recount exactly; solvation forces sum to zero; two-sphere solvation force
 * against the analytic cap derivative; step clamp. Parity unpinned: none.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

/* ---------------------------------------------------------------- small vector helpers */
static void v_sub(const double* a, const double* b, double* o) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static void v_add(const double* a, const double* b, double* o) { o[0] = a[0] + b[0]; o[1] = a[1] + b[1]; o[2] = a[2] + b[2]; }
static double v_dot(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void v_cross(const double* a, const double* b, double* o) {
    double x = a[1] * b[2] - a[2] * b[1], y = a[2] * b[0] - a[0] * b[2], z = a[0] * b[1] - a[1] * b[0];
    o[0] = x; o[1] = y; o[2] = z;
}
static void v_scale(const double* a, double s, double* o) { o[0] = a[0] * s; o[1] = a[1] * s; o[2] = a[2] * s; }
static void v_unit(const double* a, double* o) { double n = sqrt(v_dot(a, a)); v_scale(a, 1.0 / n, o); }

/* Rodrigues rotation matrix about unit axis u by angle t (right-hand rule). */
static void rot_matrix(const double* u, double t, double R[9]) {
    double c = cos(t), s = sin(t), C = 1.0 - c;
    R[0] = c + u[0] * u[0] * C;        R[1] = u[0] * u[1] * C - u[2] * s; R[2] = u[0] * u[2] * C + u[1] * s;
    R[3] = u[1] * u[0] * C + u[2] * s; R[4] = c + u[1] * u[1] * C;        R[5] = u[1] * u[2] * C - u[0] * s;
    R[6] = u[2] * u[0] * C - u[1] * s; R[7] = u[2] * u[1] * C + u[0] * s; R[8] = c + u[2] * u[2] * C;
}
static void mat_mul(const double A[9], const double B[9], double O[9]) {
    double T[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) T[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
    memcpy(O, T, sizeof T);
}
static void mat_vec(const double A[9], const double* v, double* o) {
    double x = A[0] * v[0] + A[1] * v[1] + A[2] * v[2];
    double y = A[3] * v[0] + A[4] * v[1] + A[5] * v[2];
    double z = A[6] * v[0] + A[7] * v[1] + A[8] * v[2];
    o[0] = x; o[1] = y; o[2] = z;
}
/* rotate vector v about unit axis u by angle t */
static void rodrigues(const double* v, const double* u, double t, double* o) {
    double R[9];
    rot_matrix(u, t, R);
    mat_vec(R, v, o);
}

/* ---------------------------------------------------------------- chain topology */
enum { K_N = 0, K_H = 1, K_CA = 2, K_C = 3, K_O = 4, K_SIDE = 5 };

typedef struct {
    int m, n;
    int* res;        /* residue of atom */
    int* kind;       /* K_* */
    int* slot;       /* type-table slot (0..4 backbone N,H,CA,C,O; 5.. side) */
    int* link;       /* link index 0..2m */
    int* first;      /* first atom of residue i: N_i */
    int* nside;      /* side atoms of residue i */
    double* q; double* eps; double* R; int* cls;
    double* zp;      /* ZP coordinates [n*3] (output only) */
    double* loc;     /* ZP offset of each atom from its residue's N [n*3] */
    double* nstep;   /* ZP vector N_i -> N_{i+1} [m*3] */
    int* adj_start;  /* bond graph CSR */
    int* adj;
    int* near_start; /* atoms within 3 bonds (excluding self): partner and bond distance */
    int* near_j;
    int* near_d;
    double geom[11];
    int* nchi;       /* side-chain joints chi_1 .. chi_nchi of residue i (eq. kin_05: at most 4) */
    int* chi_first;  /* index of residue i's chi_1 among all side-chain joints [m+1] */
} Chain;

/* atom index helpers: per residue order N, H, CA, side 1..k, C, O */
static int at_N(const Chain* c, int i) { return c->first[i]; }
static int at_H(const Chain* c, int i) { return c->first[i] + 1; }
static int at_CA(const Chain* c, int i) { return c->first[i] + 2; }
static int at_S(const Chain* c, int i, int t) { return c->first[i] + 3 + t; } /* t = 0..k-1 */
static int at_C(const Chain* c, int i) { return c->first[i] + 3 + c->nside[i]; }
static int at_O(const Chain* c, int i) { return c->first[i] + 4 + c->nside[i]; }

static double deg(double d) { return d * ORC_PI / 180.0; }

/* ZP geometry (Sec. 2.1): all peptide planes coplanar, phi = psi = omega = 180 deg. The backbone
 * is a planar zig-zag in the xy-plane, N_1 at the origin, CA_1 on +x, C_1 at y > 0; with every
 * backbone dihedral at 180 deg consecutive turns alternate in sign, so the direction of the bond
 * leaving backbone atom t depends on t mod 6 only. The ZP is kept the way eq. kin_03 uses it, as
 * short vectors: loc[a] is atom a's offset from the N of its residue and nstep[i] = N_{i+1} - N_i.
 * Absolute ZP centres (zp[], output only) are the running sums of nstep plus loc. */
static void zp_build(Chain* c) {
    const double* g = c->geom;
    double b_n_ca = g[0], b_ca_c = g[1], b_c_n = g[2], b_c_o = g[3], b_n_h = g[4], b_side = g[5];
    double a_n_ca_c = deg(g[6]), a_ca_c_n = deg(g[7]), a_c_n_ca = deg(g[8]), a_ca_c_o = deg(g[9]), a_side = deg(g[10]);
    int m = c->m;
    /* heading of the bond leaving backbone atom t (t mod 6): left turn at CA_1, then alternate */
    double hout[6];
    double heading = 0.0;
    hout[0] = 0.0;
    for (int t = 1; t < 6; t++) {
        int kk = t % 3;
        double interior = kk == 0 ? a_c_n_ca : (kk == 1 ? a_n_ca_c : a_ca_c_n);
        double sign = (t % 2 == 1) ? 1.0 : -1.0;
        heading += sign * (ORC_PI - interior);
        hout[t] = heading;
    }
    /* the bond arriving at atom t left atom t - 1; for N_1 this continues the zig-zag backwards */
#define HOUT(t) hout[((t) % 6 + 6) % 6]
#define HIN(t) hout[(((t) - 1) % 6 + 6) % 6]
    for (int i = 0; i < m; i++) {
        int tN = 3 * i, tCA = 3 * i + 1, tC = 3 * i + 2;
        int aN = at_N(c, i), aH = at_H(c, i), aCA = at_CA(c, i), aC = at_C(c, i), aO = at_O(c, i);
        double* L = c->loc;
        for (int x = 0; x < 3; x++) L[3 * aN + x] = 0.0;
        L[3 * aCA + 0] = b_n_ca * cos(HOUT(tN));
        L[3 * aCA + 1] = b_n_ca * sin(HOUT(tN));
        L[3 * aCA + 2] = 0.0;
        L[3 * aC + 0] = L[3 * aCA + 0] + b_ca_c * cos(HOUT(tCA));
        L[3 * aC + 1] = L[3 * aCA + 1] + b_ca_c * sin(HOUT(tCA));
        L[3 * aC + 2] = 0.0;
        c->nstep[3 * i + 0] = L[3 * aC + 0] + b_c_n * cos(HOUT(tC));
        c->nstep[3 * i + 1] = L[3 * aC + 1] + b_c_n * sin(HOUT(tC));
        c->nstep[3 * i + 2] = 0.0;
        /* O_i: in the plane at C_i, on the side away from N_{i+1}; angle CA-C-O fixed */
        double sC = (tC % 2 == 1) ? 1.0 : -1.0;
        double hO = HIN(tC) - sC * (ORC_PI - a_ca_c_o);
        L[3 * aO + 0] = L[3 * aC + 0] + b_c_o * cos(hO);
        L[3 * aO + 1] = L[3 * aC + 1] + b_c_o * sin(hO);
        L[3 * aO + 2] = 0.0;
        /* H_i: on the bisector of the external C(prev)-N-CA angle */
        double u1[3] = {cos(HIN(tN) + ORC_PI), sin(HIN(tN) + ORC_PI), 0.0};
        double u2[3] = {cos(HOUT(tN)), sin(HOUT(tN)), 0.0};
        double s_[3], d[3];
        v_add(u1, u2, s_);
        v_scale(s_, -1.0, s_);
        v_unit(s_, d);
        for (int x = 0; x < 3; x++) L[3 * aH + x] = b_n_h * d[x];
        /* side group: CB at the tetrahedral L position, then a planar all-trans zig-zag */
        double* N = &L[3 * aN];
        double* CA = &L[3 * aCA];
        double* C = &L[3 * aC];
        double nh[3], ch[3], bis[3], bh[3], w[3], wh[3], ax[3], tmp[3];
        v_sub(N, CA, tmp); v_unit(tmp, nh);
        v_sub(C, CA, tmp); v_unit(tmp, ch);
        v_add(nh, ch, bis); v_scale(bis, -1.0, bis); v_unit(bis, bh);
        v_cross(nh, ch, w); v_unit(w, wh);
        v_cross(bh, wh, tmp); v_unit(tmp, ax);
        double dir[3];
        rodrigues(bh, ax, 0.5 * a_side, dir); /* bisector turned toward n x c by half the tetrahedral angle */
        int aS = at_S(c, i, 0);
        for (int x = 0; x < 3; x++) L[3 * aS + x] = CA[x] + b_side * dir[x];
        double pn[3], cb[3];
        v_sub(&L[3 * aS], CA, cb);
        v_sub(N, CA, tmp);
        v_cross(tmp, cb, pn); v_unit(pn, pn);
        for (int t = 1; t < c->nside[i]; t++) {
            double turn = (t % 2 == 1) ? (ORC_PI - a_side) : -(ORC_PI - a_side);
            double nd[3];
            rodrigues(dir, pn, turn, nd);
            memcpy(dir, nd, sizeof nd);
            int prev = at_S(c, i, t - 1), cur = at_S(c, i, t);
            for (int x = 0; x < 3; x++) L[3 * cur + x] = L[3 * prev + x] + b_side * dir[x];
        }
    }
#undef HOUT
#undef HIN
    double Nabs[3] = {0, 0, 0};
    for (int i = 0; i < m; i++) {
        int a0 = at_N(c, i), a1 = at_O(c, i);
        for (int a = a0; a <= a1; a++)
            for (int x = 0; x < 3; x++) c->zp[3 * a + x] = Nabs[x] + c->loc[3 * a + x];
        for (int x = 0; x < 3; x++) Nabs[x] += c->nstep[3 * i + x];
    }
}

/* Bond graph of the chain: N-H, N-CA, CA-side1, side_t-side_{t+1}, CA-C, C-O, C-N(next). */
static void bonds_build(Chain* c) {
    int m = c->m, n = c->n;
    int maxb = 8 * n;
    int* bi = (int*)malloc(sizeof(int) * maxb);
    int* bj = (int*)malloc(sizeof(int) * maxb);
    int nb = 0;
#define ADDB(x, y) do { bi[nb] = (x); bj[nb] = (y); nb++; } while (0)
    for (int i = 0; i < m; i++) {
        ADDB(at_N(c, i), at_H(c, i));
        ADDB(at_N(c, i), at_CA(c, i));
        ADDB(at_CA(c, i), at_S(c, i, 0));
        for (int t = 1; t < c->nside[i]; t++) ADDB(at_S(c, i, t - 1), at_S(c, i, t));
        ADDB(at_CA(c, i), at_C(c, i));
        ADDB(at_C(c, i), at_O(c, i));
        if (i + 1 < m) ADDB(at_C(c, i), at_N(c, i + 1));
    }
#undef ADDB
    int* deg_ = (int*)calloc(n + 1, sizeof(int));
    for (int b = 0; b < nb; b++) { deg_[bi[b]]++; deg_[bj[b]]++; }
    c->adj_start = (int*)malloc(sizeof(int) * (n + 1));
    c->adj_start[0] = 0;
    for (int a = 0; a < n; a++) c->adj_start[a + 1] = c->adj_start[a] + deg_[a];
    c->adj = (int*)malloc(sizeof(int) * (c->adj_start[n] + 1));
    int* fill = (int*)calloc(n, sizeof(int));
    for (int b = 0; b < nb; b++) {
        c->adj[c->adj_start[bi[b]] + fill[bi[b]]++] = bj[b];
        c->adj[c->adj_start[bj[b]] + fill[bj[b]]++] = bi[b];
    }
    free(fill); free(deg_); free(bi); free(bj);
    /* breadth-first search from every atom to depth 3 (Sec. 3.3: interaction type = shortest
     * path length on the bond graph) */
    int cap = 64 * n + 64;
    c->near_start = (int*)malloc(sizeof(int) * (n + 1));
    c->near_j = (int*)malloc(sizeof(int) * cap);
    c->near_d = (int*)malloc(sizeof(int) * cap);
    int* dist = (int*)malloc(sizeof(int) * n);
    for (int a = 0; a < n; a++) dist[a] = -1;
    int* queue = (int*)malloc(sizeof(int) * n);
    int cnt = 0;
    for (int a = 0; a < n; a++) {
        c->near_start[a] = cnt;
        int qh = 0, qt = 0;
        queue[qt++] = a;
        dist[a] = 0;
        while (qh < qt) {
            int x = queue[qh++];
            if (dist[x] == 3) continue;
            for (int e = c->adj_start[x]; e < c->adj_start[x + 1]; e++) {
                int y = c->adj[e];
                if (dist[y] < 0) { dist[y] = dist[x] + 1; queue[qt++] = y; }
            }
        }
        for (int t = 1; t < qt; t++) {
            if (cnt >= cap) abort();
            c->near_j[cnt] = queue[t];
            c->near_d[cnt] = dist[queue[t]];
            cnt++;
        }
        for (int t = 0; t < qt; t++) dist[queue[t]] = -1;
    }
    c->near_start[n] = cnt;
    free(dist); free(queue);
}

/* Table 3, adjustment of Sharp et al.: atomic solvation parameters gamma in kcal mol^-1 A^-2,
 * for the classes C, O/N, S, O-, N+; hydrogen (absent from the table) carries gamma = 0. */
static double gamma_of_class(int k) {
    switch (k) {
        case 0: return 0.012;
        case 1: return -0.116;
        case 2: return -0.018;
        case 3: return -0.175;
        case 4: return -0.186;
        default: return 0.0;
    }
}

void* orc_chain_new(int m, const int* res_type, const int* n_side, const double* tq, const double* teps,
                    const double* tsigma, const int* tcls, const double* geom) {
    Chain* c = (Chain*)calloc(1, sizeof(Chain));
    c->m = m;
    memcpy(c->geom, geom, sizeof c->geom);
    c->first = (int*)malloc(sizeof(int) * m);
    c->nside = (int*)malloc(sizeof(int) * m);
    c->nchi = (int*)malloc(sizeof(int) * m);
    c->chi_first = (int*)malloc(sizeof(int) * (m + 1));
    int n = 0;
    for (int i = 0; i < m; i++) {
        c->first[i] = n;
        c->nside[i] = n_side[res_type[i]];
        /* a side-chain joint turns about the bond to side atom k - 1 (CA -> CB for k = 1) and moves
         * the side atoms beyond it: at most 4 (eq. kin_05), and one fewer than the side atoms */
        c->nchi[i] = c->nside[i] >= 2 ? (c->nside[i] - 1 < 4 ? c->nside[i] - 1 : 4) : 0;
        n += 5 + c->nside[i];
    }
    c->n = n;
    c->chi_first[0] = 0;
    for (int i = 0; i < m; i++) c->chi_first[i + 1] = c->chi_first[i] + c->nchi[i];
    c->res = (int*)malloc(sizeof(int) * n);
    c->kind = (int*)malloc(sizeof(int) * n);
    c->slot = (int*)malloc(sizeof(int) * n);
    c->link = (int*)malloc(sizeof(int) * n);
    c->q = (double*)malloc(sizeof(double) * n);
    c->eps = (double*)malloc(sizeof(double) * n);
    c->R = (double*)malloc(sizeof(double) * n);
    c->cls = (int*)malloc(sizeof(int) * n);
    c->zp = (double*)calloc(3 * (size_t)n, sizeof(double));
    c->loc = (double*)calloc(3 * (size_t)n, sizeof(double));
    c->nstep = (double*)calloc(3 * (size_t)m, sizeof(double));
    for (int i = 0; i < m; i++) {
        int t = res_type[i], k = c->nside[i];
        /* links: base link 0 = {N_1, H_1}; CA-link 2i+1 = {CA_i, side_i}; peptide link 2i+2 =
         * {C_i, O_i, N_{i+1}, H_{i+1}} (two rigid links per residue, Sec. 2.1) */
        int nl = (i == 0) ? 0 : 2 * i;
        struct { int a, kind, slot, link; } at[15];
        int na = 0;
        at[na].a = at_N(c, i); at[na].kind = K_N; at[na].slot = 0; at[na].link = nl; na++;
        at[na].a = at_H(c, i); at[na].kind = K_H; at[na].slot = 1; at[na].link = nl; na++;
        at[na].a = at_CA(c, i); at[na].kind = K_CA; at[na].slot = 2; at[na].link = 2 * i + 1; na++;
        for (int s = 0; s < k; s++) { at[na].a = at_S(c, i, s); at[na].kind = K_SIDE; at[na].slot = 5 + s; at[na].link = 2 * i + 1; na++; }
        at[na].a = at_C(c, i); at[na].kind = K_C; at[na].slot = 3; at[na].link = 2 * i + 2; na++;
        at[na].a = at_O(c, i); at[na].kind = K_O; at[na].slot = 4; at[na].link = 2 * i + 2; na++;
        for (int x = 0; x < na; x++) {
            int a = at[x].a;
            c->res[a] = i; c->kind[a] = at[x].kind; c->slot[a] = at[x].slot; c->link[a] = at[x].link;
            c->q[a] = tq[15 * t + at[x].slot];
            c->eps[a] = teps[15 * t + at[x].slot];
            c->R[a] = 0.5 * tsigma[15 * t + at[x].slot]; /* R_i = sigma_i / 2 */
            c->cls[a] = tcls[15 * t + at[x].slot];
        }
    }
    zp_build(c);
    bonds_build(c);
    return c;
}

void orc_chain_free(void* p) {
    Chain* c = (Chain*)p;
    if (!c) return;
    free(c->res); free(c->kind); free(c->slot); free(c->link); free(c->first); free(c->nside);
    free(c->nchi); free(c->chi_first);
    free(c->q); free(c->eps); free(c->R); free(c->cls); free(c->zp); free(c->loc); free(c->nstep);
    free(c->adj_start); free(c->adj); free(c->near_start); free(c->near_j); free(c->near_d);
    free(c);
}

int orc_natoms(void* p) { return ((Chain*)p)->n; }

void orc_atom_info(void* p, int* res, int* kind, int* link, double* q, double* eps, double* R, double* gamma) {
    Chain* c = (Chain*)p;
    for (int a = 0; a < c->n; a++) {
        if (res) res[a] = c->res[a];
        if (kind) kind[a] = c->kind[a];
        if (link) link[a] = c->link[a];
        if (q) q[a] = c->q[a];
        if (eps) eps[a] = c->eps[a];
        if (R) R[a] = c->R[a];
        if (gamma) gamma[a] = gamma_of_class(c->cls[a]);
    }
}

void orc_zp(void* p, double* xyz) {
    Chain* c = (Chain*)p;
    memcpy(xyz, c->zp, sizeof(double) * 3 * (size_t)c->n);
}

/* the ZP as short vectors: loc[n*3] (offset of each atom from its residue's N) and
 * nstep[m*3] (N_i -> N_{i+1}; the last entry is where N_{m+1} would be) */
void orc_zp_local(void* p, double* loc, double* nstep) {
    Chain* c = (Chain*)p;
    memcpy(loc, c->loc, sizeof(double) * 3 * (size_t)c->n);
    memcpy(nstep, c->nstep, sizeof(double) * 3 * (size_t)c->m);
}

/* number of bonds between a and b on the bond graph, or 4 when more than 3 */
int orc_bond_distance(void* p, int a, int b) {
    Chain* c = (Chain*)p;
    if (a == b) return 0;
    for (int e = c->near_start[a]; e < c->near_start[a + 1]; e++)
        if (c->near_j[e] == b) return c->near_d[e];
    return 4;
}

/* list of bonds, as pairs (a, b) with a < b; returns the count */
int orc_bonds(void* p, int* out_pairs) {
    Chain* c = (Chain*)p;
    int cnt = 0;
    for (int a = 0; a < c->n; a++)
        for (int e = c->adj_start[a]; e < c->adj_start[a + 1]; e++)
            if (c->adj[e] > a) {
                if (out_pairs) { out_pairs[2 * cnt] = a; out_pairs[2 * cnt + 1] = c->adj[e]; }
                cnt++;
            }
    return cnt;
}

/* ---------------------------------------------------------------- forward kinematics */
/* One residue of the forward kinematics: given M = M_{2i} (rotation through the previous psi)
 * and the current centre of N_i, place CA_i, the side group, C_i, O_i, N_{i+1}, H_{i+1}; return
 * M_{2i+2} in Mout and N_{i+1} in rN_out. Optionally writes the current axes and axis points of
 * joints 2i+1 (phi_i) and 2i+2 (psi_i). */
/* ZP offset of atom a from CA_i, for atoms of residue i and the N, H of residue i+1 (short
 * vectors built from loc and nstep, never from differences of absolute ZP centres) */
static void zp_from_ca(const Chain* c, int i, int a, double* v) {
    const double* ca = &c->loc[3 * at_CA(c, i)];
    if (c->res[a] == i) {
        v_sub(&c->loc[3 * a], ca, v);
    } else { /* N_{i+1} or H_{i+1}: through N_i -> N_{i+1} */
        double t[3];
        v_add(&c->nstep[3 * i], &c->loc[3 * a], t);
        v_sub(t, ca, v);
    }
}

/* ZP offset from CA_i of side atom s of residue i after the side-chain rotations th_side[0 ..
 * nchi-1] (eq. kin_05, r2): chi_k turns by th_side[k-1] about the ZP bond from side atom k - 2 (CA
 * for k = 1) to side atom k - 1 and moves side atoms s >= k; in the ZP frame the rotations compose
 * from the most distal: x = T_1(T_2(... T_min(s, nchi)(x0))), T_k(x) = R_k (x - a_k) + a_k. */
static void side_offset(const Chain* c, int i, int s, const double* th_side, double* x) {
    zp_from_ca(c, i, at_S(c, i, s), x);
    const int kmax = s < c->nchi[i] ? s : c->nchi[i];
    for (int k = kmax; k >= 1; k--) {
        double a[3] = {0, 0, 0}, b[3], u[3], R[9], t[3], r[3];
        if (k >= 2) zp_from_ca(c, i, at_S(c, i, k - 2), a);
        zp_from_ca(c, i, at_S(c, i, k - 1), b);
        v_sub(b, a, u);
        v_unit(u, u);
        rot_matrix(u, th_side[k - 1], R);
        v_sub(x, a, t);
        mat_vec(R, t, r);
        v_add(r, a, x);
    }
}

static void fk_residue(const Chain* c, int i, double th_phi, double th_psi, const double* th_side, const double M[9],
                       const double* rN, double* xyz, double Mout[9], double* rN_out, double* u2, double* p2) {
    int aCA = at_CA(c, i), aC = at_C(c, i);
    double u0[3], b0[3], R[9], Mphi[9], Mpsi[9], b[3], rCA[3], v0[3], v[3];
    /* phi_i: rotation about the ZP axis N_i -> CA_i (eq. kin_04) */
    memcpy(b0, &c->loc[3 * aCA], sizeof b0); /* ZP body vector N_i -> CA_i */
    v_unit(b0, u0);
    rot_matrix(u0, th_phi, R);
    mat_mul(M, R, Mphi);
    if (u2) mat_vec(Mphi, u0, &u2[0]);
    if (p2) memcpy(&p2[0], rN, 3 * sizeof(double));
    mat_vec(Mphi, b0, b); /* body vector N_i -> CA_i (eq. kin_03) */
    v_add(rN, b, rCA);    /* eq. r1 */
    memcpy(&xyz[3 * aCA], rCA, sizeof rCA);
    for (int s = 0; s < c->nside[i]; s++) { /* eq. r2 */
        int aS = at_S(c, i, s);
        if (th_side) side_offset(c, i, s, th_side, v0);
        else zp_from_ca(c, i, aS, v0);
        mat_vec(Mphi, v0, v);
        v_add(rCA, v, &xyz[3 * aS]);
    }
    /* psi_i: rotation about the ZP axis CA_i -> C_i */
    zp_from_ca(c, i, aC, v0);
    v_unit(v0, u0);
    rot_matrix(u0, th_psi, R);
    mat_mul(Mphi, R, Mpsi);
    if (u2) mat_vec(Mpsi, u0, &u2[3]);
    if (p2) memcpy(&p2[3], rCA, sizeof rCA);
    int pep[4], np_ = 0;
    pep[np_++] = aC;
    pep[np_++] = at_O(c, i);
    if (i + 1 < c->m) { pep[np_++] = at_N(c, i + 1); pep[np_++] = at_H(c, i + 1); }
    for (int x = 0; x < np_; x++) { /* peptide-plane atoms, rigid with the psi link */
        zp_from_ca(c, i, pep[x], v0);
        mat_vec(Mpsi, v0, v);
        v_add(rCA, v, &xyz[3 * pep[x]]);
    }
    if (i + 1 < c->m) memcpy(rN_out, &xyz[3 * at_N(c, i + 1)], 3 * sizeof(double));
    memcpy(Mout, Mpsi, 9 * sizeof(double));
}

/* eq. kin_04: M_j = R_1 R_2 ... R_j with R_r the rotation by theta_r about the ZP axis u^0_r;
 * eq. kin_02/03: u = M u^0, b = M b^0; eq. r1/r2: atom centres as prefix sums of body vectors,
 * N_1 anchored at the origin. Joint 2i+1 (phi of residue i) turns about N_i -> CA_i, joint 2i+2
 * (psi) about CA_i -> C_i. Outputs: atom centres [n*3]; optionally the current joint axes
 * u [2m*3] and a point on each axis p [2m*3] (N_i for phi, CA_i for psi). */
/* the same with the side-chain joints at theta_side [orc_nside_joints] (NULL: the ZP side groups) */
void orc_fk_x(void* p, const double* theta, const double* theta_side, double* xyz, double* u_out, double* p_out) {
    Chain* c = (Chain*)p;
    double M[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    double rN[3] = {0, 0, 0};
    /* base link: N_1 and H_1 never move */
    memcpy(&xyz[3 * at_N(c, 0)], &c->zp[3 * at_N(c, 0)], 3 * sizeof(double));
    memcpy(&xyz[3 * at_H(c, 0)], &c->zp[3 * at_H(c, 0)], 3 * sizeof(double));
    for (int i = 0; i < c->m; i++) {
        double Mn[9], rn[3] = {0, 0, 0};
        fk_residue(c, i, theta[2 * i], theta[2 * i + 1], theta_side ? &theta_side[c->chi_first[i]] : NULL, M, rN,
                   xyz, Mn, rn, u_out ? &u_out[6 * i] : NULL, p_out ? &p_out[6 * i] : NULL);
        memcpy(M, Mn, sizeof M);
        memcpy(rN, rn, sizeof rN);
    }
}

void orc_fk(void* p, const double* theta, double* xyz, double* u_out, double* p_out) {
    orc_fk_x(p, theta, NULL, xyz, u_out, p_out);
}

int orc_nside_joints(void* p) { return ((Chain*)p)->chi_first[((Chain*)p)->m]; }

/* Torques of the side-chain joints (eq. KCM_06 for the branches of Sec. 3.5): the moment, about the
 * joint's current axis (its bond, from side atom k - 2 or CA to side atom k - 1), of the forces on
 * the side atoms it moves, tau = u . sum_s (r_s - a) x F_s. */
void orc_side_torques(void* p, const double* xyz, const double* F, double* tau_side) {
    Chain* c = (Chain*)p;
    for (int i = 0; i < c->m; i++) {
        for (int k = 1; k <= c->nchi[i]; k++) {
            const double* a = &xyz[3 * (k >= 2 ? at_S(c, i, k - 2) : at_CA(c, i))];
            const double* b = &xyz[3 * at_S(c, i, k - 1)];
            double u[3];
            v_sub(b, a, u);
            v_unit(u, u);
            double t = 0.0;
            for (int s = k; s < c->nside[i]; s++) {
                double r[3], m[3];
                v_sub(&xyz[3 * at_S(c, i, s)], a, r);
                v_cross(r, &F[3 * at_S(c, i, s)], m);
                t += v_dot(u, m);
            }
            tau_side[c->chi_first[i] + k - 1] = t;
        }
    }
}

/* ---------------------------------------------------------------- compact random-walk starts */
/* Input generation for the compact workloads (not part of the method): grow the chain residue by
 * residue, drawing (theta_phi, theta_psi) uniformly (phi, psi uniform in [-pi, pi)) and redrawing
 * up to max_retries times until no heavy-atom pair more than three bonds apart is closer than
 * min_dist; when every draw fails, back up `backtrack` residues and regrow. Angles are drawn as
 * 16-bit codes (theta = code * 2 pi / 65536) from SplitMix64 (Steele, Lea & Flood 2014) so that
 * they are exact in float64; the codes are written to codes_out [2m]. Returns 0, or -1 when the
 * attempt budget runs out. */
static uint64_t splitmix64(uint64_t* s) {
    uint64_t z = (*s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

typedef struct { int nb; int* head; int* next; double cell; } Grid;
static uint32_t grid_hash(long long x, long long y, long long z, int nb) {
    uint64_t h = (uint64_t)(x * 73856093LL) ^ (uint64_t)(y * 19349663LL) ^ (uint64_t)(z * 83492791LL);
    return (uint32_t)(h % (uint64_t)nb);
}
static void grid_insert(Grid* g, const double* xyz, int a) {
    long long x = (long long)floor(xyz[3 * a] / g->cell), y = (long long)floor(xyz[3 * a + 1] / g->cell),
              z = (long long)floor(xyz[3 * a + 2] / g->cell);
    uint32_t h = grid_hash(x, y, z, g->nb);
    g->next[a] = g->head[h];
    g->head[h] = a;
}
static int heavy(const Chain* c, int a) { return c->kind[a] != K_H; }

static int clash_free(const Chain* c, const Grid* g, const double* xyz, const int* cand, int nc, double dmin) {
    double d2min = dmin * dmin;
    for (int t = 0; t < nc; t++) {
        int a = cand[t];
        long long x = (long long)floor(xyz[3 * a] / g->cell), y = (long long)floor(xyz[3 * a + 1] / g->cell),
                  z = (long long)floor(xyz[3 * a + 2] / g->cell);
        for (long long dx = -1; dx <= 1; dx++)
            for (long long dy = -1; dy <= 1; dy++)
                for (long long dz = -1; dz <= 1; dz++) {
                    uint32_t h = grid_hash(x + dx, y + dy, z + dz, g->nb);
                    for (int b = g->head[h]; b >= 0; b = g->next[b]) {
                        double r[3];
                        v_sub(&xyz[3 * a], &xyz[3 * b], r);
                        if (v_dot(r, r) < d2min && orc_bond_distance((void*)c, a, b) > 3) return 0;
                    }
                }
        for (int u = 0; u < t; u++) { /* among the new atoms themselves */
            int b = cand[u];
            double r[3];
            v_sub(&xyz[3 * a], &xyz[3 * b], r);
            if (v_dot(r, r) < d2min && orc_bond_distance((void*)c, a, b) > 3) return 0;
        }
    }
    return 1;
}

int orc_grow_start(void* p, unsigned long long seed, double min_dist, int max_retries, int backtrack,
                   unsigned short* codes_out) {
    Chain* c = (Chain*)p;
    int m = c->m, n = c->n;
    uint64_t st = (uint64_t)seed;
    double* xyz = (double*)calloc(3 * (size_t)n, sizeof(double));
    double* Ms = (double*)malloc(sizeof(double) * 9 * (m + 1)); /* M before residue i */
    double* rNs = (double*)malloc(sizeof(double) * 3 * (m + 1));
    Grid g;
    g.cell = min_dist;
    g.nb = 1;
    while (g.nb < 2 * n) g.nb <<= 1;
    g.head = (int*)malloc(sizeof(int) * g.nb);
    g.next = (int*)malloc(sizeof(int) * n);
    for (int h = 0; h < g.nb; h++) g.head[h] = -1;
    double I[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    memcpy(&Ms[0], I, sizeof I);
    memset(&rNs[0], 0, 3 * sizeof(double));
    memcpy(&xyz[3 * at_N(c, 0)], &c->zp[3 * at_N(c, 0)], 3 * sizeof(double));
    memcpy(&xyz[3 * at_H(c, 0)], &c->zp[3 * at_H(c, 0)], 3 * sizeof(double));
    grid_insert(&g, xyz, at_N(c, 0));
    long long budget = (long long)m * max_retries * 50 + 1000;
    int i = 0, rc = 0;
    while (i < m) {
        int ok = 0;
        for (int r = 0; r < max_retries && !ok; r++) {
            if (--budget < 0) { rc = -1; goto done; }
            unsigned short cp = (unsigned short)(splitmix64(&st) >> 48), cs = (unsigned short)(splitmix64(&st) >> 48);
            double tp = (double)cp * (2.0 * ORC_PI / 65536.0), ts = (double)cs * (2.0 * ORC_PI / 65536.0);
            double Mn[9], rn[3] = {0, 0, 0};
            fk_residue(c, i, tp, ts, NULL, &Ms[9 * i], &rNs[3 * i], xyz, Mn, rn, NULL, NULL);
            int cand[16], nc = 0;
            cand[nc++] = at_CA(c, i);
            for (int s = 0; s < c->nside[i]; s++) cand[nc++] = at_S(c, i, s);
            cand[nc++] = at_C(c, i);
            cand[nc++] = at_O(c, i);
            if (i + 1 < m) cand[nc++] = at_N(c, i + 1);
            if (clash_free(c, &g, xyz, cand, nc, min_dist)) {
                ok = 1;
                codes_out[2 * i] = cp;
                codes_out[2 * i + 1] = cs;
                memcpy(&Ms[9 * (i + 1)], Mn, sizeof Mn);
                memcpy(&rNs[3 * (i + 1)], rn, sizeof rn);
                for (int t = 0; t < nc; t++) if (heavy(c, cand[t])) grid_insert(&g, xyz, cand[t]);
            }
        }
        if (ok) { i++; continue; }
        /* back up and rebuild the grid from the atoms that stay */
        i = i > backtrack ? i - backtrack : 0;
        for (int h = 0; h < g.nb; h++) g.head[h] = -1;
        int lastatom = (i < m) ? at_CA(c, i) : n; /* atoms before CA_i stay placed */
        for (int a = 0; a < lastatom; a++) if (heavy(c, a)) grid_insert(&g, xyz, a);
    }
done:
    free(xyz); free(Ms); free(rNs); free(g.head); free(g.next);
    return rc;
}

/* ---------------------------------------------------------------- pairwise forces */
/* Coulomb with eps_ij = 4 d (kappa_ij = 4 d, eq. 02 with the distance-dependent dielectric) and
 * Lennard-Jones 6-12 in the AMBER form (eq. 03), each weighted by w_ij (eq. 03_8, 03_9).
 * Pair energy:  w_e K q_i q_j / (4 d^2)  +  w_v eps_ij [ (D/d)^12 - 2 (D/d)^6 ],
 * D = R_i + R_j, eps_ij = sqrt(eps_i eps_j). Force on i is -grad_{r_i} of the pair energy:
 * [ w_e K q_i q_j / (2 d^4) + 12 w_v eps_ij (D^12/d^14 - D^6/d^8) ] (r_i - r_j).
 * Pairs farther than the cutoff (d > r_c) are dropped (eq. 02_2, 03_2).
 *
 * `cls` gives each pair's bond class through `bond_class(i, j)`: 1 for 1-2 or 1-3 (w = 0),
 * 2 for 1-4 (w = w14), 0 otherwise (w = 1). E[0] = electrostatic, E[1] = van der Waals, both
 * summed over unordered pairs once; F[n*3] = force per atom. Returns the number of unordered
 * pairs within the cutoff that carry w != 0. */
typedef struct {
    const int* start; const int* j; const int* d; /* atoms within 3 bonds, from BFS */
} BondInfo;

static int bond_class(const BondInfo* bi, int a, int b) {
    if (!bi || !bi->start) return 0;
    for (int e = bi->start[a]; e < bi->start[a + 1]; e++)
        if (bi->j[e] == b) return bi->d[e] <= 2 ? 1 : 2;
    return 0;
}

static long long pair_forces_core(int n, const double* xyz, const double* q, const double* eps, const double* R,
                                  const BondInfo* bi, const double* prm, double* F, double* E) {
    double rc = prm[0], rcv = prm[1] > 0 ? prm[1] : prm[0], K = prm[2], w14e = prm[3], w14v = prm[4];
    double rc2 = rc * rc, rcv2 = rcv * rcv;
    /* per-atom partial energies, summed afterwards in atom order so that the result does not
     * depend on the thread count */
    double* Ei = (double*)calloc(2 * (size_t)n + 2, sizeof(double));
    long long npairs = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : npairs)
    for (int i = 0; i < n; i++) {
        double Fi[3] = {0, 0, 0};
        double Eel = 0.0, Evdw = 0.0;
        for (int j = 0; j < n; j++) {
            if (j == i) continue;
            double r[3];
            v_sub(&xyz[3 * i], &xyz[3 * j], r);
            double d2 = v_dot(r, r);
            if (d2 > rc2 && d2 > rcv2) continue;
            int cl = bond_class(bi, i, j);
            if (cl == 1) continue;
            double we = cl == 2 ? w14e : 1.0, wv = cl == 2 ? w14v : 1.0;
            double coef = 0.0;
            if (d2 <= rc2) {
                double d4 = d2 * d2;
                coef += we * K * q[i] * q[j] / (2.0 * d4);
                if (j > i) Eel += we * K * q[i] * q[j] / (4.0 * d2);
            }
            if (d2 <= rcv2) {
                double D = R[i] + R[j];
                double eij = sqrt(eps[i] * eps[j]);
                double D2 = D * D, D6 = D2 * D2 * D2, D12 = D6 * D6;
                double d6 = d2 * d2 * d2, d8 = d6 * d2, d12 = d6 * d6, d14 = d12 * d2;
                coef += 12.0 * wv * eij * (D12 / d14 - D6 / d8);
                if (j > i) Evdw += wv * eij * (D12 / d12 - 2.0 * D6 / d6);
            }
            if (j > i && (we != 0.0 || wv != 0.0)) npairs++;
            Fi[0] += coef * r[0]; Fi[1] += coef * r[1]; Fi[2] += coef * r[2];
        }
        F[3 * i] = Fi[0]; F[3 * i + 1] = Fi[1]; F[3 * i + 2] = Fi[2];
        Ei[2 * i] = Eel; Ei[2 * i + 1] = Evdw;
    }
    E[0] = 0.0; E[1] = 0.0;
    for (int i = 0; i < n; i++) { E[0] += Ei[2 * i]; E[1] += Ei[2 * i + 1]; }
    free(Ei);
    return npairs;
}

/* prm = {cutoff, vdw_cutoff (0 = same), coulomb_k, w14_elec, w14_vdw} */
long long orc_pair_forces_chain(void* p, const double* xyz, const double* prm, double* F, double* E) {
    Chain* c = (Chain*)p;
    BondInfo bi = {c->near_start, c->near_j, c->near_d};
    return pair_forces_core(c->n, xyz, c->q, c->eps, c->R, &bi, prm, F, E);
}

/* the same for free atoms (no bonds) */
long long orc_pair_forces_free(int n, const double* xyz, const double* q, const double* eps, const double* R,
                               const double* prm, double* F, double* E) {
    return pair_forces_core(n, xyz, q, eps, R, NULL, prm, F, E);
}

/* ---------------------------------------------------------------- sample set on the unit sphere */
/* Quasi-uniform polar sampling (Sec. 3.4: orbits at uniform angular spacing, points on each orbit
 * in proportion to its circumference). The paper defers the details to another report, so the
 * recipe here is: K = round(sqrt(pi N / 4)) latitude rings at polar angles pi (r - 1/2) / K,
 * r = 1..K; ring r receives n_r points in proportion to sin of its polar angle, rounded by the
 * largest-remainder rule (ties to the smaller r) so that the n_r sum to N; point t of ring r sits
 * at longitude 2 pi (t + (r mod 2)/2) / n_r. Points are listed ring by ring. */
int orc_sample_points(int N, double* Q) {
    if (N < 1) return -1;
    int K = (int)floor(sqrt(ORC_PI * (double)N / 4.0) + 0.5);
    if (K < 1) K = 1;
    double* w = (double*)malloc(sizeof(double) * K);
    int* nr = (int*)malloc(sizeof(int) * K);
    double* frac = (double*)malloc(sizeof(double) * K);
    double wsum = 0.0;
    for (int r = 1; r <= K; r++) {
        w[r - 1] = sin(ORC_PI * ((double)r - 0.5) / (double)K);
        wsum += w[r - 1];
    }
    int assigned = 0;
    for (int r = 0; r < K; r++) {
        double ideal = (double)N * w[r] / wsum;
        nr[r] = (int)floor(ideal);
        frac[r] = ideal - floor(ideal);
        assigned += nr[r];
    }
    for (int left = N - assigned; left > 0; left--) {
        int best = -1;
        for (int r = 0; r < K; r++)
            if (best < 0 || frac[r] > frac[best]) best = r;
        nr[best] += 1;
        frac[best] = -1.0;
    }
    int k = 0;
    for (int r = 1; r <= K; r++) {
        double th = ORC_PI * ((double)r - 0.5) / (double)K;
        for (int t = 0; t < nr[r - 1]; t++) {
            double lon = 2.0 * ORC_PI * ((double)t + 0.5 * (double)(r % 2)) / (double)nr[r - 1];
            Q[3 * k + 0] = sin(th) * cos(lon);
            Q[3 * k + 1] = sin(th) * sin(lon);
            Q[3 * k + 2] = cos(th);
            k++;
        }
    }
    free(w); free(nr); free(frac);
    return k;
}

/* ---------------------------------------------------------------- solvation (Algorithm 1) */
/* Neighbour candidates A'_i: every j != i with d_ij <= Roff_i + Roff_j + dr. No farther sphere
 * can reach atom i's offset sphere even after a displacement by dr (Sec. 2.2, eq. 04_3). */
static int* sasa_candidates(int n, const double* xyz, const double* Roff, double dr, int** start_out) {
    int* start = (int*)malloc(sizeof(int) * (n + 1));
    int* cnt = (int*)calloc(n, sizeof(int));
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < n; i++) {
        int c_ = 0;
        for (int j = 0; j < n; j++) {
            if (j == i) continue;
            double r[3];
            v_sub(&xyz[3 * i], &xyz[3 * j], r);
            double lim = Roff[i] + Roff[j] + dr;
            if (v_dot(r, r) <= lim * lim) c_++;
        }
        cnt[i] = c_;
    }
    start[0] = 0;
    for (int i = 0; i < n; i++) start[i + 1] = start[i] + cnt[i];
    int* list = (int*)malloc(sizeof(int) * ((size_t)start[n] + 1));
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < n; i++) {
        int c_ = start[i];
        for (int j = 0; j < n; j++) {
            if (j == i) continue;
            double r[3];
            v_sub(&xyz[3 * i], &xyz[3 * j], r);
            double lim = Roff[i] + Roff[j] + dr;
            if (v_dot(r, r) <= lim * lim) list[c_++] = j;
        }
    }
    free(cnt);
    *start_out = start;
    return list;
}

/* overlap test of Algorithm 1: ||q - (r_j + disp)|| <= Roff_j, compared squared */
static int covers(const double* qk, const double* rj, double Roffj, int s, double dr) {
    double w[3] = {qk[0] - rj[0], qk[1] - rj[1], qk[2] - rj[2]};
    if (s >= 0) w[s] -= dr;
    return v_dot(w, w) <= Roffj * Roffj;
}

/* Algorithm 1 for all atoms. Inputs: centres r [n*3], offset radii Roff = R + R_probe [n],
 * solvation parameters gamma [n] (Table 3), the unit sample set Q [N*3], finite difference dr.
 * Outputs: F [n*3] solvation forces, E_atom [n] = G^cav_i = 4 pi gamma_i Roff_i^2 f_i,
 * covered [n] = number of samples with C_ik >= 1 (so f_i = 1 - covered_i / N).
 * Optional: counts [n_pairs*3] with per-(i, candidate slot, s) net exchange counts; the force
 * exchanged between i and its candidate j along e_s is G0_i / (N dr) times that count.
 * stats[0] = step-1 overlap tests, stats[1] = step-2 tests, stats[2] = candidate pairs.
 * literal_break = 1 keeps the printed `break` after the first newly-overlapping neighbour in the
 * C = 0 branch (comparison only); 0 tests every neighbour. */
void orc_sasa(int n, const double* xyz, const double* Roff, const double* gamma, int N, const double* Q,
              double dr, int literal_break, double* F, double* E_atom, int* covered, long long* stats,
              int* cand_start_out, int* cand_out, int* counts_out) {
    int* cstart;
    int* cand = sasa_candidates(n, xyz, Roff, dr, &cstart);
    int* cnt = (int*)calloc((size_t)cstart[n] * 3 + 1, sizeof(int)); /* net exchange counts */
    long long t1 = 0, t2 = 0;
#pragma omp parallel for schedule(dynamic, 8) reduction(+ : t1, t2)
    for (int i = 0; i < n; i++) {
        /* Step 1: energy. C_ik counts overlapping neighbours and stops at 2; j_over keeps the
         * critical neighbour when C_ik = 1. */
        double G0 = 4.0 * ORC_PI * gamma[i] * Roff[i] * Roff[i];
        int nc = cstart[i + 1] - cstart[i];
        const int* A = &cand[cstart[i]];
        int* Cik = (int*)malloc(sizeof(int) * N);
        int* jover = (int*)malloc(sizeof(int) * N);
        int cov = 0;
        for (int k = 0; k < N; k++) {
            double qk[3];
            for (int x = 0; x < 3; x++) qk[x] = xyz[3 * i + x] + Roff[i] * Q[3 * k + x]; /* T_i(q_k) */
            Cik[k] = 0;
            jover[k] = -1;
            for (int a = 0; a < nc; a++) {
                int j = A[a];
                t1++;
                if (covers(qk, &xyz[3 * j], Roff[j], -1, dr)) {
                    Cik[k]++;
                    if (Cik[k] == 1) { jover[k] = a; cov++; }
                    else { jover[k] = -1; break; }
                }
            }
        }
        covered[i] = cov;
        E_atom[i] = G0 - G0 * (double)cov / (double)N;
        /* Step 2: forces. Exposed points (C = 0) re-test every neighbour displaced by dr e_s;
         * critically overlapped points (C = 1) re-test only the critical neighbour. */
        int* my = &cnt[3 * (size_t)cstart[i]];
        for (int k = 0; k < N; k++) {
            if (Cik[k] >= 2) continue;
            double qk[3];
            for (int x = 0; x < 3; x++) qk[x] = xyz[3 * i + x] + Roff[i] * Q[3 * k + x];
            for (int s = 0; s < 3; s++) {
                if (Cik[k] == 0) {
                    for (int a = 0; a < nc; a++) {
                        int j = A[a];
                        t2++;
                        if (covers(qk, &xyz[3 * j], Roff[j], s, dr)) {
                            my[3 * a + s] += 1; /* F_i,s -= G0/(N dr), F_j,s += G0/(N dr) */
                            if (literal_break) break;
                        }
                    }
                } else {
                    int a = jover[k];
                    int j = A[a];
                    t2++;
                    if (!covers(qk, &xyz[3 * j], Roff[j], s, dr)) my[3 * a + s] -= 1; /* F_i,s += .., F_j,s -= .. */
                }
            }
        }
        free(Cik); free(jover);
        (void)G0;
    }
    /* apply the pairwise exchanges in a fixed order (deterministic for any thread count) */
    for (int x = 0; x < 3 * n; x++) F[x] = 0.0;
    for (int i = 0; i < n; i++) {
        double quantum = 4.0 * ORC_PI * gamma[i] * Roff[i] * Roff[i] / ((double)N * dr);
        for (int a = cstart[i]; a < cstart[i + 1]; a++) {
            int j = cand[a];
            for (int s = 0; s < 3; s++) {
                int c_ = cnt[3 * (size_t)a + s];
                if (!c_) continue;
                F[3 * i + s] -= quantum * c_;
                F[3 * j + s] += quantum * c_;
            }
        }
    }
    if (stats) { stats[0] = t1; stats[1] = t2; stats[2] = cstart[n]; }
    if (cand_start_out) memcpy(cand_start_out, cstart, sizeof(int) * (n + 1));
    if (cand_out) memcpy(cand_out, cand, sizeof(int) * cstart[n]);
    if (counts_out) memcpy(counts_out, cnt, sizeof(int) * 3 * (size_t)cstart[n]);
    free(cnt); free(cand); free(cstart);
}

/* number of candidate pairs (ordered) for sizing the optional outputs of orc_sasa */
int orc_sasa_ncand(int n, const double* xyz, const double* Roff, double dr) {
    int* cstart;
    int* cand = sasa_candidates(n, xyz, Roff, dr, &cstart);
    int r = cstart[n];
    free(cand); free(cstart);
    return r;
}

/* Definition-level solvation for tiny inputs: f_i by enumeration of all N points against all
 * other atoms (exposure ratio, Sec. 3.4), f_{i,j,s} by re-enumeration with r_j moved by dr e_s,
 * the forward difference of eq. finitediff, and the forces of eq. F_cav_patch:
 *   F_i = G0_i sum_j grad_{r_j} f_i - sum_j G0_j grad_{r_i} f_j,  G0 = 4 pi gamma Roff^2.
 * dcount[(i*n + j)*3 + s] = N (f_{i,j,s} - f_i) as an exact integer. */
void orc_sasa_bruteforce(int n, const double* xyz, const double* Roff, const double* gamma, int N, const double* Q,
                         double dr, double* F, double* E_atom, int* covered, int* dcount) {
    int* exposed = (int*)malloc(sizeof(int) * n);
    for (int i = 0; i < n; i++) {
        int e = 0;
        for (int k = 0; k < N; k++) {
            double qk[3];
            for (int x = 0; x < 3; x++) qk[x] = xyz[3 * i + x] + Roff[i] * Q[3 * k + x];
            int hit = 0;
            for (int j = 0; j < n && !hit; j++)
                if (j != i && covers(qk, &xyz[3 * j], Roff[j], -1, dr)) hit = 1;
            if (!hit) e++;
        }
        exposed[i] = e;
        covered[i] = N - e;
        E_atom[i] = 4.0 * ORC_PI * gamma[i] * Roff[i] * Roff[i] * (double)e / (double)N;
    }
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++)
            for (int s = 0; s < 3; s++) {
                int e = 0;
                if (j != i) {
                    for (int k = 0; k < N; k++) {
                        double qk[3];
                        for (int x = 0; x < 3; x++) qk[x] = xyz[3 * i + x] + Roff[i] * Q[3 * k + x];
                        int hit = 0;
                        for (int h = 0; h < n && !hit; h++)
                            if (h != i && covers(qk, &xyz[3 * h], Roff[h], h == j ? s : -1, dr)) hit = 1;
                        if (!hit) e++;
                    }
                } else {
                    e = exposed[i];
                }
                dcount[((size_t)i * n + j) * 3 + s] = e - exposed[i];
            }
    for (int i = 0; i < n; i++)
        for (int s = 0; s < 3; s++) {
            double f = 0.0;
            for (int j = 0; j < n; j++) {
                if (j == i) continue;
                double G0i = 4.0 * ORC_PI * gamma[i] * Roff[i] * Roff[i];
                double G0j = 4.0 * ORC_PI * gamma[j] * Roff[j] * Roff[j];
                double grad_j_fi = (double)dcount[((size_t)i * n + j) * 3 + s] / (double)N / dr;
                double grad_i_fj = (double)dcount[((size_t)j * n + i) * 3 + s] / (double)N / dr;
                f += G0i * grad_j_fi - G0j * grad_i_fj;
            }
            F[3 * i + s] = f;
        }
    free(exposed);
}

/* ---------------------------------------------------------------- torques */
/* Link wrenches (eq. KCM_01, KCM_02), moments about the origin: P_h = [T_h ; F_h]. */
static void link_wrench(int n, int L, const int* link, const double* xyz, const double* F, double* P) {
    memset(P, 0, sizeof(double) * 6 * (size_t)L);
    for (int a = 0; a < n; a++) {
        double t[3];
        v_cross(&xyz[3 * a], &F[3 * a], t);
        int h = link[a];
        for (int x = 0; x < 3; x++) { P[6 * h + x] += t[x]; P[6 * h + 3 + x] += F[3 * a + x]; }
    }
}

/* Joint torques as the column sums of eq. 04_9: tau_k = sum_{h >= k} J_k^T P_h with
 * J_k = [u_k ; p_k x u_k] (eq. KCM_05 with every link's torque centre at the origin). Links are
 * numbered 0..l; joint k (1..l) moves links k..l. Protofold I's O(l^2) order. */
void orc_torques_columns(int n, int l, const int* link, const double* xyz, const double* F, const double* u,
                         const double* pk, double* tau) {
    double* P = (double*)malloc(sizeof(double) * 6 * (size_t)(l + 1));
    link_wrench(n, l + 1, link, xyz, F, P);
    for (int k = 1; k <= l; k++) {
        const double* uk = &u[3 * (k - 1)];
        double pxu[3];
        v_cross(&pk[3 * (k - 1)], uk, pxu);
        double t = 0.0;
        for (int h = k; h <= l; h++) t += v_dot(uk, &P[6 * h]) + v_dot(pxu, &P[6 * h + 3]);
        tau[k - 1] = t;
    }
    free(P);
}

/* Row-scan form of Sec. 3.5: P^agg_k = P_k + P^agg_{k+1}, tau_k = J_k^T P^agg_k. */
void orc_torques_rowscan(int n, int l, const int* link, const double* xyz, const double* F, const double* u,
                         const double* pk, double* tau) {
    double* P = (double*)malloc(sizeof(double) * 6 * (size_t)(l + 1));
    link_wrench(n, l + 1, link, xyz, F, P);
    double agg[6] = {0, 0, 0, 0, 0, 0};
    for (int k = l; k >= 1; k--) {
        for (int x = 0; x < 6; x++) agg[x] += P[6 * k + x];
        const double* uk = &u[3 * (k - 1)];
        double pxu[3];
        v_cross(&pk[3 * (k - 1)], uk, pxu);
        tau[k - 1] = v_dot(uk, agg) + v_dot(pxu, agg + 3);
    }
    free(P);
}

/* ---------------------------------------------------------------- pairwise solvation surrogate */
/* The smooth pairwise approximation of the solvent-accessible area that preceded surface enumeration
 * (Sec. 3.4: probabilistic pairwise formulae): the exposed area of atom i is
 *   A_i = S_i prod_{j != i} (1 - b_ij / S_i),   S_i = 4 pi Roff_i^2,
 * with b_ij the area of the offset sphere of i inside that of j,
 *   b_ij = pi Roff_i (Roff_i + Roff_j - d) (1 + (Roff_j - Roff_i) / d)   for d < Roff_i + Roff_j,
 * clamped to [0, S_i] (j inside i: 0; i inside j: S_i), and every overlap parameter of the
 * probabilistic formulae equal to 1. Energy G^cav = sum_i gamma_i A_i (eq. 04 with the areas A_i).
 * Forces are the exact negative gradient: with c_ij = dE_i/dd_ij = E_i (-db_ij/dd) / (S_i f_ij),
 * f_ij = 1 - b_ij/S_i and -db/dd = pi Roff_i (1 + (Roff_j^2 - Roff_i^2) / d^2), the pair (i, j)
 * adds c_ij e_ij to F_i and -c_ij e_ij to F_j, e_ij = (r_j - r_i) / d. Where a factor is clamped
 * (f_ij = 0 or b_ij = 0 inside the overlap range) its derivative is taken as 0.
 * Inputs: centres xyz [n*3], Roff [n], gamma [n]; outputs F [n*3], E_atom [n] (may be NULL). */
static double pw_dist(const double* a, const double* b) {
    const double x = a[0] - b[0], y = a[1] - b[1], z = a[2] - b[2];
    return sqrt(x * x + y * y + z * z);
}

void orc_sasa_pairwise(int n, const double* xyz, const double* Roff, const double* gamma, double* F, double* E_atom) {
    memset(F, 0, sizeof(double) * 3 * n);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int i = 0; i < n; i++) {
        const double Ri = Roff[i], Si = 4.0 * ORC_PI * Ri * Ri;
        double A = Si;
        for (int j = 0; j < n; j++) {
            if (j == i) continue;
            const double d = pw_dist(&xyz[3 * i], &xyz[3 * j]);
            if (d >= Ri + Roff[j]) continue;
            double b = ORC_PI * Ri * (Ri + Roff[j] - d) * (1.0 + (Roff[j] - Ri) / d);
            if (b < 0.0) b = 0.0;
            double f = 1.0 - b / Si;
            if (f < 0.0) f = 0.0;
            A *= f;
        }
        if (E_atom) E_atom[i] = gamma[i] * A;
    }
    /* forces: a second pass needs every A_i; E_i = gamma_i A_i (serial over i: each pair writes to j) */
    for (int i = 0; i < n; i++) {
        const double Ri = Roff[i], Si = 4.0 * ORC_PI * Ri * Ri;
        double A = Si;
        int clamped = 0;
        for (int j = 0; j < n; j++) {
            if (j == i) continue;
            const double d = pw_dist(&xyz[3 * i], &xyz[3 * j]);
            if (d >= Ri + Roff[j]) continue;
            double b = ORC_PI * Ri * (Ri + Roff[j] - d) * (1.0 + (Roff[j] - Ri) / d);
            if (b < 0.0) b = 0.0;
            double f = 1.0 - b / Si;
            if (f <= 0.0) { clamped = 1; f = 0.0; }
            A *= f;
        }
        const double Ei = gamma[i] * A;
        if (Ei == 0.0 || clamped) continue;
        for (int j = 0; j < n; j++) {
            if (j == i) continue;
            const double d = pw_dist(&xyz[3 * i], &xyz[3 * j]);
            if (d >= Ri + Roff[j]) continue;
            const double b = ORC_PI * Ri * (Ri + Roff[j] - d) * (1.0 + (Roff[j] - Ri) / d);
            if (b <= 0.0) continue;  /* j inside i: no burial, no derivative */
            const double f = 1.0 - b / Si;
            const double mdb = ORC_PI * Ri * (1.0 + (Roff[j] * Roff[j] - Ri * Ri) / (d * d));
            const double cij = Ei * mdb / (Si * f);
            for (int x = 0; x < 3; x++) {
                const double e = (xyz[3 * j + x] - xyz[3 * i + x]) / d;
                F[3 * i + x] += cij * e;
                F[3 * j + x] -= cij * e;
            }
        }
    }
}

/* ---------------------------------------------------------------- kinetostatic step */
/* mode 0: dtheta_k = clamp(kappa tau_k, -dmax, +dmax); mode 1: the paper's normalised step
 * dtheta_k = kappa tau_k / max_j |tau_j| (eq. KCM_07). theta_{t+1} = theta_t + dtheta (Sec. 3.1).
 * fixed (may be NULL): joints held fixed (Sec. 4.1, the option of fixing dihedral angles so that
 * groups of residues move as rigid bodies); they take no step and do not enter max_j |tau_j|.
 * Returns max_k |dtheta_k|. */
double orc_step(int l, double* theta, const double* tau, double kappa, double dmax, int mode, double* dtheta,
                const unsigned char* fixed) {
    double tmax = 0.0, dm = 0.0;
    for (int k = 0; k < l; k++)
        if (!(fixed && fixed[k])) tmax = fmax(tmax, fabs(tau[k]));
    for (int k = 0; k < l; k++) {
        double d;
        if (fixed && fixed[k]) d = 0.0;
        else if (mode == 1) d = tmax > 0.0 ? kappa * tau[k] / tmax : 0.0;
        else {
            d = kappa * tau[k];
            if (d > dmax) d = dmax;
            if (d < -dmax) d = -dmax;
        }
        if (dtheta) dtheta[k] = d;
        theta[k] += d;
        dm = fmax(dm, fabs(d));
    }
    return dm;
}

/* ---------------------------------------------------------------- one full iteration */
/* prm = {cutoff, vdw_cutoff, coulomb_k, w14_elec, w14_vdw, r_probe, delta_r, kappa, dtheta_max,
 *        conv_tol, solvation, n_sample, step_mode}
 * Evaluates at theta: positions, pair and solvation forces, torques, energies E[3] (elec, vdw,
 * cav). Optional outputs may be NULL. */
void orc_evaluate_x(void* p, const double* prm, const double* theta, const double* theta_side, double* xyz,
                    double* F_pair, double* F_cav, double* tau, double* tau_side, double* E, int* covered,
                    long long* stats) {
    Chain* c = (Chain*)p;
    int n = c->n, l = 2 * c->m, N = (int)prm[11];
    double* X = xyz ? xyz : (double*)malloc(sizeof(double) * 3 * n);
    double* Fp = F_pair ? F_pair : (double*)malloc(sizeof(double) * 3 * n);
    double* Fc = F_cav ? F_cav : (double*)malloc(sizeof(double) * 3 * n);
    double* u = (double*)malloc(sizeof(double) * 3 * l);
    double* pk = (double*)malloc(sizeof(double) * 3 * l);
    double Ep[2];
    orc_fk_x(p, theta, theta_side, X, u, pk);
    double pprm[5] = {prm[0], prm[1], prm[2], prm[3], prm[4]};
    long long npairs = orc_pair_forces_chain(p, X, pprm, Fp, Ep);
    double Ecav = 0.0;
    long long st[3] = {0, 0, 0};
    if (prm[10] == 2.0) {  /* the pairwise surrogate */
        double* Roff = (double*)malloc(sizeof(double) * n);
        double* gam = (double*)malloc(sizeof(double) * n);
        double* Ea = (double*)malloc(sizeof(double) * n);
        for (int a = 0; a < n; a++) { Roff[a] = c->R[a] + prm[5]; gam[a] = gamma_of_class(c->cls[a]); }
        orc_sasa_pairwise(n, X, Roff, gam, Fc, Ea);
        for (int a = 0; a < n; a++) Ecav += Ea[a];
        if (covered) memset(covered, 0, sizeof(int) * n);
        free(Roff); free(gam); free(Ea);
    } else if (prm[10] != 0.0) {
        double* Roff = (double*)malloc(sizeof(double) * n);
        double* gam = (double*)malloc(sizeof(double) * n);
        double* Ea = (double*)malloc(sizeof(double) * n);
        int* cov = covered ? covered : (int*)malloc(sizeof(int) * n);
        double* Q = (double*)malloc(sizeof(double) * 3 * N);
        orc_sample_points(N, Q);
        for (int a = 0; a < n; a++) { Roff[a] = c->R[a] + prm[5]; gam[a] = gamma_of_class(c->cls[a]); }
        orc_sasa(n, X, Roff, gam, N, Q, prm[6], 0, Fc, Ea, cov, st, NULL, NULL, NULL);
        for (int a = 0; a < n; a++) Ecav += Ea[a];
        free(Roff); free(gam); free(Ea); free(Q);
        if (!covered) free(cov);
    } else {
        memset(Fc, 0, sizeof(double) * 3 * n);
        if (covered) memset(covered, 0, sizeof(int) * n);
    }
    if (tau || tau_side) {
        double* Ft = (double*)malloc(sizeof(double) * 3 * n);
        for (int x = 0; x < 3 * n; x++) Ft[x] = Fp[x] + Fc[x];
        if (tau) orc_torques_columns(n, l, c->link, X, Ft, u, pk, tau);
        if (tau_side) orc_side_torques(p, X, Ft, tau_side);
        free(Ft);
    }
    if (E) { E[0] = Ep[0]; E[1] = Ep[1]; E[2] = Ecav; }
    if (stats) { stats[0] = npairs; stats[1] = st[0]; stats[2] = st[1]; stats[3] = st[2]; }
    if (!xyz) free(X);
    if (!F_pair) free(Fp);
    if (!F_cav) free(Fc);
    free(u); free(pk);
}

void orc_evaluate(void* p, const double* prm, const double* theta, double* xyz, double* F_pair, double* F_cav,
                  double* tau, double* E, int* covered, long long* stats) {
    orc_evaluate_x(p, prm, theta, NULL, xyz, F_pair, F_cav, tau, NULL, E, covered, stats);
}

/* The KCM loop (Sec. 4.1 steps 4-9): evaluate, step, stop once max |dtheta| < conv_tol.
 * theta is updated in place; E_trace [n_iters*3], dmax_trace [n_iters] and fixed [l] (joints held
 * fixed) are optional; with theta_side (NULL: none) the side-chain joints are stepped together with
 * the main-chain joints, as one vector of joint angles. Returns the number of iterations taken. */
int orc_run_x(void* p, const double* prm, double* theta, double* theta_side, int n_iters, double* E_trace,
              double* dmax_trace, const unsigned char* fixed) {
    Chain* c = (Chain*)p;
    const int l = 2 * c->m, ls = theta_side ? orc_nside_joints(p) : 0;
    double* tau = (double*)malloc(sizeof(double) * (l + ls + 1));
    double* all = (double*)malloc(sizeof(double) * (l + ls + 1));
    unsigned char* fx = NULL;
    if (fixed) {
        fx = (unsigned char*)calloc(l + ls + 1, 1);
        memcpy(fx, fixed, l);
    }
    int it;
    for (it = 0; it < n_iters; it++) {
        double E[3];
        orc_evaluate_x(p, prm, theta, theta_side, NULL, NULL, NULL, tau, ls ? tau + l : NULL, E, NULL, NULL);
        memcpy(all, theta, sizeof(double) * l);
        if (ls) memcpy(all + l, theta_side, sizeof(double) * ls);
        double dm = orc_step(l + ls, all, tau, prm[7], prm[8], (int)prm[12], NULL, fx);
        memcpy(theta, all, sizeof(double) * l);
        if (ls) memcpy(theta_side, all + l, sizeof(double) * ls);
        if (E_trace) memcpy(&E_trace[3 * it], E, sizeof E);
        if (dmax_trace) dmax_trace[it] = dm;
        if (dm < prm[9]) { it++; break; }
    }
    free(tau); free(all); free(fx);
    return it;
}

int orc_run(void* p, const double* prm, double* theta, int n_iters, double* E_trace, double* dmax_trace,
            const unsigned char* fixed) {
    return orc_run_x(p, prm, theta, NULL, n_iters, E_trace, dmax_trace, fixed);
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}
