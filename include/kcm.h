/*
 * kcm.h — C ABI of the B300-native kinetostatic compliance method (KCM) step.
 *
 * One KCM iteration (Behandish & Ilies, "Protofold II", arXiv 1712.05012, Sec. 4.1 steps 4-8)
 * maps the chain's joint angles theta to atom centres by forward kinematics over rigid links
 * (Sec. 2.1, eq. kin_02..kin_05, r1, r2), bins the atoms into a uniform cell grid (Sec. 3.2),
 * evaluates cutoff Coulomb with the distance-dependent dielectric eps = 4 d, Lennard-Jones 6-12
 * (Sec. 2.2, eq. 02_2, 03_2, 03_8, 03_9) and the surface-enumeration solvation forces
 * (Sec. 3.4, Algorithm 1), reduces forces to link wrenches and joint torques with a suffix sum
 * (eq. KCM_01, KCM_02, KCM_06, Sec. 3.5) and steps theta <- theta + dtheta (eq. KCM_07).
 *
 * Conventions
 *   Units: Angstrom, elementary charge, kcal/mol, radian.
 *   Atom order (inputs and outputs): per residue N, H, CA, side atoms 1..k, C, O. With this order
 *     the atoms of every rigid link are contiguous: base link {N_1, H_1}; CA link i = {CA_i, side_i};
 *     peptide link i = {C_i, O_i, N_{i+1}, H_{i+1}} (the last one is {C_m, O_m}).
 *   Joint order: theta[2i] = phi joint of residue i (about N_i -> CA_i), theta[2i+1] = psi joint
 *     (about CA_i -> C_i), i = 0..m-1, so l = 2m joints. theta = 0 is the zero position (ZP,
 *     phi = psi = 180 deg, eq. theta_1/theta_2); phi_i = theta[2i] - pi, psi_i = theta[2i+1] - pi.
 *     A joint rotates everything distal to it by the right-hand rule about its axis; N_1 stays at
 *     the origin. ZP frame: N_1 at the origin, CA_1 on +x, C_1 in the xy-plane at y > 0.
 *   Every call returns an int status: KCM_OK (0) or a negative KCM_E_* code; kcm_strerror names it
 *     and kcm_last_error(h) gives the last message for a handle.
 *   Host buffers passed to the library are caller-owned; the library copies what it keeps. The
 *     handle owns all device memory it allocates; nothing is freed before kcm_destroy.
 *   A handle is not thread-safe; distinct handles are independent. All device work of a handle is
 *     ordered on the CUDA stream given at kcm_create (an internal stream when NULL). Calls taking
 *     host buffers synchronise that stream before returning; *_dev calls take device pointers and
 *     are ordered on the stream without synchronising.
 */
#ifndef KCM_H
#define KCM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define KCM_OK 0
#define KCM_E_INVAL (-1)     /* invalid argument or size mismatch */
#define KCM_E_NOMEM (-2)     /* device or host allocation failed */
#define KCM_E_CUDA (-3)      /* a CUDA runtime call failed */
#define KCM_E_TIMEOUT (-4)   /* a bounded device wait gave up (the torque kernel's blocks wait for later tiles' totals) */
#define KCM_E_NONFINITE (-5) /* a torque came out NaN or infinite */
#define KCM_E_OVERFLOW (-6)  /* an atom had more solvation neighbours than the list holds */
#define KCM_E_NODEVICE (-8)  /* no CUDA device, or the device is not sm_103 */
#define KCM_E_CANCELLED (-9) /* a served job was cancelled (kcm_server_cancel) */

/* precision of the pair and solvation arithmetic; kinematics and torque scans are FP64 always */
#define KCM_FP64 0
#define KCM_MIXED 1

/* step rule (eq. KCM_07) */
#define KCM_STEP_CLAMP 0      /* dtheta_k = clamp(kappa tau_k, -dtheta_max, +dtheta_max) */
#define KCM_STEP_NORMALIZED 1 /* dtheta_k = kappa tau_k / max_j |tau_j| (the paper's form) */

/* solvation classes: the rows of Table 3 (atomic solvation parameters, Sharp et al. adjustment)
 * plus hydrogen, which Table 3 does not list and which gets gamma = 0 */
#define KCM_CLS_C 0      /* gamma = +0.012 kcal mol^-1 A^-2 */
#define KCM_CLS_ON 1     /* -0.116 */
#define KCM_CLS_S 2      /* -0.018 */
#define KCM_CLS_OMINUS 3 /* -0.175 */
#define KCM_CLS_NPLUS 4  /* -0.186 */
#define KCM_CLS_H 5      /* 0 */

#define KCM_MAX_SIDE 10

/* Atomic constants of one atom (the tuple a_i of Sec. 2.2): charge q (e), LJ well depth eps
 * (kcal/mol), LJ size sigma (A; the van der Waals radius is R = sigma / 2, so the LJ distance is
 * D_ij = R_i + R_j) and the solvation class. */
typedef struct {
    double q;
    double eps;
    double sigma;
    int32_t solv_class;
    int32_t reserved;
} kcm_atom_param;

/* One residue type: its rigid side group size (1..10 atoms, a planar all-trans zig-zag hung on
 * CA, first atom at the L-chirality CB position) and the constants of its backbone atoms
 * (N, H, CA, C, O in that order) and side atoms. */
typedef struct {
    int32_t n_side;
    int32_t reserved;
    kcm_atom_param backbone[5];
    kcm_atom_param side[KCM_MAX_SIDE];
} kcm_restype;

/* Fixed bond lengths (A) and bond angles (degrees) of the rigid links (Sec. 2.1, App. A:
 * bond lengths and angles are constant, omega = 180 deg). H sits on the bisector of the external
 * C-N-CA angle; side groups use b_side and the angle a_side throughout. */
typedef struct {
    double b_n_ca, b_ca_c, b_c_n, b_c_o, b_n_h, b_side;
    double a_n_ca_c, a_ca_c_n, a_c_n_ca, a_ca_c_o, a_side;
} kcm_geometry;

/* A chain: n_res residues with types res_type[i] in [0, n_types) drawn from the table `types`.
 * geometry may be NULL for the library defaults (N-CA 1.458, CA-C 1.525, C-N 1.329, C=O 1.231,
 * N-H 1.0, side 1.53 A; N-CA-C 111.2, CA-C-N 116.2, C-N-CA 121.7, CA-C-O 120.8, side 109.4712
 * degrees). All pointers are read during kcm_create only. */
typedef struct {
    int32_t n_res;
    int32_t n_types;
    const int32_t* res_type;
    const kcm_restype* types;
    const kcm_geometry* geometry;
} kcm_topology;

/* Run parameters. cutoff: Coulomb and LJ cutoff (pairs with d <= cutoff interact, eq. 02_2);
 * vdw_cutoff: separate LJ cutoff when > 0 (the paper uses 9 A and 5 A); kappa: step gain
 * (rad per kcal/mol); dtheta_max: clamp (rad); w14_elec, w14_vdw: weights of pairs three bonds
 * apart (1-2 and 1-3 pairs get 0, all others 1; eq. 03_8/03_9); r_probe: solvent probe radius
 * (the offset sphere is R + r_probe, Sec. 3.4); delta_r: finite-difference displacement of
 * eq. finitediff; coulomb_k: 332.0636 kcal A mol^-1 e^-2; conv_tol: the step loop stops once
 * max_k |dtheta_k| < conv_tol; cell_size: requested edge of the binning cells of Sec. 3.2 (0 =
 * the smallest edge that covers the largest interaction range rmax with the 27 cells around an
 * atom's cell; an edge below rmax switches the pair search to the 125 cells two cells out, and
 * is raised to rmax / 2 plus a rounding margin if smaller; a grid that would exceed its cell cap
 * is coarsened);
 * n_sample: sample points per offset sphere N; solvation: 0 off, 1 surface enumeration (Algorithm 1),
 * 2 the pairwise surrogate that preceded it (Sec. 3.4: A_i = S_i prod_j (1 - b_ij / S_i), b_ij the
 * area of offset sphere i inside offset sphere j, S_i = 4 pi Roff_i^2; smooth, with exact gradient
 * forces); precision: KCM_FP64/KCM_MIXED;
 * step_mode: KCM_STEP_CLAMP/KCM_STEP_NORMALIZED; side_joints: 1 adds the side-chain joints (eq. kin_05,
 * r2: residue i gets chi_1 .. chi_k, k = min(4, side atoms - 1); chi_k turns about the bond from side
 * atom k - 2 (CA for k = 1) to side atom k - 1 and moves side atoms k, k + 1, ...), stepped by the
 * loop together with the main-chain joints as one vector (kcm_set_side_theta and the calls after
 * it); 0 (the default) holds every side group in its ZP form. */
typedef struct {
    double cutoff;
    double vdw_cutoff;
    double kappa;
    double dtheta_max;
    double w14_elec;
    double w14_vdw;
    double r_probe;
    double delta_r;
    double coulomb_k;
    double conv_tol;
    double cell_size;
    int32_t n_sample;
    int32_t solvation;
    int32_t precision;
    int32_t step_mode;
    int32_t side_joints;
} kcm_params;

/* Counters of the last evaluation (device-side, read back by kcm_get_stats). */
typedef struct {
    int64_t pairs;          /* unordered pairs within the cutoff with w != 0 */
    int64_t sasa_neighbors; /* ordered solvation neighbour entries (sum over atoms of |A'_i|) */
    int64_t max_neighbors;  /* largest |A'_i| */
    int64_t guard_rechecks; /* FP32 tests inside the guard band re-decided in FP64 */
    int64_t cells;          /* cells of the binning grid */
    double cell_size;       /* edge actually used (A) */
    int64_t iterations;     /* iterations taken by the last kcm_step */
    int64_t sasa_tests;     /* overlap tests performed by Algorithm 1 (steps 1 and 2) */
} kcm_stats;

typedef struct kcm_ctx* kcm_handle;

/* Fill `p` with the defaults: cutoff 10, vdw_cutoff 0, kappa 1e-3, dtheta_max 0.02,
 * w14 0.5/0.5, r_probe 1.4, delta_r 0.02, coulomb_k 332.0636, conv_tol 1e-4, cell_size 0,
 * n_sample 256, solvation 1, KCM_FP64, KCM_STEP_CLAMP, side_joints 0. */
int kcm_params_default(kcm_params* p);

/* Build the chain (ZP geometry, bond-class tables, sample set) on the host and upload it to the
 * current CUDA device. cuda_stream is a cudaStream_t (NULL: the library makes its own stream).
 * theta starts at 0 (the ZP). Errors: KCM_E_INVAL (bad sizes, types or parameters),
 * KCM_E_NODEVICE, KCM_E_NOMEM, KCM_E_CUDA. On error *out is NULL. */
int kcm_create(const kcm_topology* top, const kcm_params* prm, void* cuda_stream, kcm_handle* out);

/* A batch of n_chains independent chains tops[0..n_chains-1] in one handle, stepped together by the
 * same kernels (one launch per stage for all chains; every scan is segmented at chain boundaries and
 * every chain gets its own cell grid). The chains are concatenated: atoms, joints and theta of chain
 * c follow those of chain c-1 (kcm_chain_offsets), so every per-atom and per-joint call of this
 * header covers the whole batch. Each chain converges on its own (its max |dtheta| below conv_tol)
 * and then takes no more steps; kcm_step returns when every chain has converged or after n_iters.
 * kcm_energy returns the sums over the chains (kcm_chain_energies gives them per chain). The paper
 * steps one chain; batching many independent chains is a throughput layer over the same
 * iteration (Sec. 4.1). Errors as kcm_create, also KCM_E_INVAL for n_chains < 1. */
int kcm_create_batch(const kcm_topology* tops, int32_t n_chains, const kcm_params* prm, void* cuda_stream,
                     kcm_handle* out);

/* Number of chains of the handle (1 for kcm_create), -1 for NULL. */
int32_t kcm_nchains(kcm_handle h);

/* Offsets of every chain: atoms of chain c are [atom_off[c], atom_off[c+1]), its joints (theta,
 * tau) [joint_off[c], joint_off[c+1]); both arrays hold kcm_nchains + 1 entries (either may be
 * NULL). Host memory, caller-owned. */
int kcm_chain_offsets(kcm_handle h, int64_t* atom_off, int64_t* joint_off);

/* Energies of every chain at the current theta (evaluates): E[3c..3c+2] = Coulomb, Lennard-Jones,
 * solvation of chain c (eq. 01). E has 3 * kcm_nchains doubles, host memory. */
int kcm_chain_energies(kcm_handle h, double* E);

/* Loop state of every chain since the last kcm_step or kcm_step_async: iterations taken, whether it
 * has stopped (1: converged, reached its cap or failed) or is still running (0), the max |dtheta| of
 * its last step, and its status (KCM_OK, KCM_E_OVERFLOW or KCM_E_NONFINITE). In a batch a failing
 * chain stops alone (the others go on; kcm_step still reports the error); a single chain stops the
 * loop. Arrays of kcm_nchains entries, host memory, any may be NULL; waits for the handle's stream. */
int kcm_chain_state(kcm_handle h, int32_t* iters, int32_t* converged, double* max_dtheta, int32_t* errors);

/* Cap on the iterations every chain may take in each later kcm_step / kcm_step_async call:
 * max_iters[c] for chain c (kcm_nchains entries, host memory; NULL removes every cap). A chain with
 * a cap <= 0 takes no step at all and costs no pair or solvation work; a chain that reaches its cap
 * stops like a converged one (kcm_chain_state reports converged = 1 and its iterations). The
 * serving loop below uses it to advance chains of a batch by different amounts. */
int kcm_set_chain_max_iters(kcm_handle h, const int32_t* max_iters);

/* Device memory held by the handle, in bytes (-1 for NULL). */
int64_t kcm_device_bytes(kcm_handle h);

/* ---------------------------------------------------------------- serving loop
 * A request loop for folding jobs (no counterpart in the paper, which folds one chain at a time):
 * jobs of any chain length are submitted at any time, admitted as device memory frees up under a
 * budget, stepped with all other admitted jobs on the device (continuous batching: a batch on a stream
 * of its own advances in chunks of iterations launched without waiting), and retired when they
 * converge (max |dtheta| < conv_tol) or reach their iteration cap. Free slots are refilled by
 * compaction: the next batch takes the waiting jobs together with the running jobs of the batch with
 * the most retired slots, which move over with the angles they reached at its next chunk boundary;
 * the old batch is then freed, so the memory of retired jobs returns to the budget. New batches are
 * made on worker threads (up to four admission waves and one compaction at a time) while ticks go on. Coordinates, cell lists and theta stay
 * on the device from admission to retirement (a move copies theta once). Single-threaded: one thread
 * calls the kcm_server_* functions of a server. Times are seconds since creation (host clock). */
typedef struct kcm_server kcm_server;

#define KCM_JOB_WAITING 0
#define KCM_JOB_RUNNING 1
#define KCM_JOB_DONE 2

typedef struct {
    int32_t state;       /* KCM_JOB_* */
    int32_t error;       /* KCM_OK, or the status that ended the job (e.g. KCM_E_NONFINITE, KCM_E_NOMEM) */
    int32_t iters;       /* iterations taken */
    int32_t converged;   /* 1: stopped because max |dtheta| < conv_tol */
    double max_dtheta;   /* max |dtheta| of its last step */
    int64_t natoms;
    double t_submit, t_admit, t_done;
} kcm_job_info;

/* params: as kcm_create (all jobs of a server share them); hbm_budget_bytes: device memory the
 * server's batches may hold together (a job that cannot fit even alone ends with KCM_E_NOMEM);
 * max_chains_per_batch: most chains a batch holds; chunk_iters: iterations a batch takes between two
 * looks at its chains. Errors: KCM_E_INVAL, KCM_E_NOMEM. */
int kcm_server_create(const kcm_params* params, int64_t hbm_budget_bytes, int32_t max_chains_per_batch,
                      int32_t chunk_iters, kcm_server** out);
void kcm_server_destroy(kcm_server* s);

/* Queue a job: the chain `top` (copied), its start theta0[l] (l = 2 n_res, host memory, copied) and
 * its iteration cap. *job_id > 0 names it. With params.side_joints = 1 the job's side-chain joints
 * start at 0 and are stepped with its main chain; kcm_server_job reports the main-chain angles.
 * Errors: KCM_E_INVAL (bad topology, sizes or cap). */
int kcm_server_submit(kcm_server* s, const kcm_topology* top, const double* theta0, int64_t l, int32_t max_iters,
                      int64_t* job_id);

/* Make progress without waiting for the device: collect the batches whose chunk has finished (retire
 * their done jobs, launch their next chunk, free emptied batches) and admit waiting jobs as the
 * budget allows. Reports the jobs still waiting and running (either pointer may be NULL). */
int kcm_server_tick(kcm_server* s, int32_t* n_waiting, int32_t* n_running);

/* Admission waves: a tick admits waiting jobs once min_jobs of them wait, once the oldest has waited
 * max_wait_s seconds, or at once when no job is running (default 1 and 0: every tick admits what
 * waits). Larger waves make fewer, larger batches (each batch's creation and per-iteration launches
 * are paid once for all its jobs) at the price of queueing. Errors: KCM_E_INVAL (min_jobs < 1,
 * max_wait_s negative or not finite). */
int kcm_server_set_admission(kcm_server* s, int32_t min_jobs, double max_wait_s);

/* Ids of jobs retired since the last poll (at most `capacity`; *n of them written to ids). The
 * server keeps the records of the last 65,536 polled jobs; older ones are dropped. */
int kcm_server_poll(kcm_server* s, int64_t* ids, int32_t capacity, int32_t* n);

/* State of a job and, once it is done, its final theta (theta may be NULL; l = 2 n_res). Errors:
 * KCM_E_INVAL (unknown id, a record already dropped, l mismatch). */
int kcm_server_job(kcm_server* s, int64_t job_id, kcm_job_info* info, double* theta, int64_t l);

/* Cancel a job: a waiting job retires at once; a job that has a slot takes no step after the chunk
 * that is running and retires at the end of it, with the angles it reached. Either way it ends with
 * error KCM_E_CANCELLED (a job that converges or reaches its cap in that chunk ends as it would have).
 * The other jobs are not affected. Errors: KCM_E_INVAL (unknown id, or the job has finished). */
int kcm_server_cancel(kcm_server* s, int64_t job_id);

/* Device memory held by the server's batches, in bytes (-1 for NULL). */
int64_t kcm_server_device_bytes(kcm_server* s);

/* Free everything the handle owns. NULL is accepted. */
void kcm_destroy(kcm_handle h);

int64_t kcm_natoms(kcm_handle h);  /* n, or -1 for a NULL handle */
int64_t kcm_njoints(kcm_handle h); /* l = 2 m, or -1 */

/* Joint angles theta[l] (rad), host copies. l must equal kcm_njoints. */
int kcm_set_theta(kcm_handle h, const double* theta, int64_t l);
int kcm_get_theta(kcm_handle h, double* theta, int64_t l);
/* The same with device pointers (stream-ordered, no synchronisation). */
int kcm_set_theta_dev(kcm_handle h, const double* theta_dev, int64_t l);
int kcm_get_theta_dev(kcm_handle h, double* theta_dev, int64_t l);

/* Atom centres xyz[n*3] at the current theta (forward kinematics only: eq. kin_04, r1, r2). */
int kcm_positions(kcm_handle h, double* xyz, int64_t n);

/* Total force per atom F[n*3] (kcal mol^-1 A^-1) at the current theta: pair forces
 * (eq. 03_8 + 03_9) plus solvation forces (Algorithm 1) when solvation is on. */
int kcm_forces(kcm_handle h, double* F, int64_t n);

/* The two terms separately: F_pair[n*3] (Coulomb + LJ) and F_cav[n*3] (solvation). Either
 * pointer may be NULL. */
int kcm_force_terms(kcm_handle h, double* F_pair, double* F_cav, int64_t n);

/* Joint torques tau[l] (kcal/mol per rad) at the current theta: tau_k = J_k^T sum_{h>=k} P_h with
 * J_k = [u_k ; p_k x u_k] and link wrenches P_h taken about the origin (eq. KCM_01..06). */
int kcm_torques(kcm_handle h, double* tau, int64_t l);
int kcm_torques_dev(kcm_handle h, double* tau_dev, int64_t l);

/* Energies at the current theta: E[0] Coulomb, E[1] Lennard-Jones (unordered pairs once),
 * E[2] solvation sum_i 4 pi gamma_i Roff_i^2 f_i (eq. G_cav_patch; 0 when solvation is off). */
int kcm_energy(kcm_handle h, double E[3]);

/* Covered sample counts per atom (f_i = 1 - covered_i / N, Sec. 3.4), int32[n]. Atoms with
 * gamma = 0 contribute neither energy nor force and are not enumerated: their count reads 0; with
 * the pairwise surrogate (solvation = 2) nothing is enumerated and every count reads 0. */
int kcm_sasa_counts(kcm_handle h, int32_t* covered, int64_t n);

/* Run up to n_iters KCM iterations from the current theta (evaluate, then theta += dtheta); stop
 * early once max |dtheta| < conv_tol. The loop runs as a captured CUDA graph with no host round
 * trip per iteration. iters_done and max_dtheta (of the last iteration taken) may be NULL.
 * Errors: KCM_E_NONFINITE, KCM_E_OVERFLOW (results of that iteration are not valid), KCM_E_CUDA. */
int kcm_step(kcm_handle h, int32_t n_iters, int32_t* iters_done, double* max_dtheta);

/* kcm_set_theta, kcm_step and kcm_get_theta in one call with one wait: theta_in[l] (host, NULL: the
 * current theta) goes to the device, up to n_iters iterations run as in kcm_step, and the final theta
 * comes back in theta_out[l] (host, may be NULL); this is the host round trip of a caller that owns
 * theta on the host. With both buffers and n_iters >= 1 the angles pass through a page-locked, mapped
 * buffer of the handle (made at the first such call, l doubles): the first iteration's transform scan
 * reads them from it and every step writes the angles it changes back, and the kernel that ends an
 * iteration writes the status record to page-locked host memory, so the call is a host copy in, one
 * graph launch per iteration, one wait and a host copy out, with no copy on the stream. Otherwise the
 * copies are enqueued on the handle's stream (asynchronous for page-locked buffers). Errors as
 * kcm_set_theta and kcm_step. */
int kcm_step_host(kcm_handle h, const double* theta_in, double* theta_out, int64_t l, int32_t n_iters,
                  int32_t* iters_done, double* max_dtheta);

/* Enqueue n_iters iterations without synchronising (for timing with CUDA events on the stream);
 * read the outcome later with kcm_step_status. */
int kcm_step_async(kcm_handle h, int32_t n_iters);
int kcm_step_status(kcm_handle h, int32_t* iters_done, double* max_dtheta);

int kcm_get_stats(kcm_handle h, kcm_stats* st);

/* Joints held fixed (Sec. 4.1: the user may fix as many dihedral angles as desired, so that groups of
 * residues such as secondary elements or domains move as rigid bodies and only the loops between
 * them deform). fixed[l] (l = kcm_njoints; a batch's joints in chain order): nonzero holds the joint.
 * A fixed joint takes no step; its torque is still computed (kcm_torques), but it has no part in the
 * normalised step's max |tau| nor in the convergence test (max |dtheta| over the moved joints).
 * NULL clears all flags (the default). Synchronises. Errors: KCM_E_INVAL (l does not match). */
int kcm_set_fixed_joints(kcm_handle h, const uint8_t* fixed, int64_t l);

/* Side-chain joints (kcm_params.side_joints = 1; eq. kin_05, r2 and the branch torques of Sec. 3.5).
 * Joint chi_k of residue i turns the side atoms beyond the bond (side atom k - 2, or CA for k = 1) ->
 * (side atom k - 1) about that bond; chi = 0 is the ZP side group. The side-chain joints of a handle
 * are numbered residue by residue, chi_1 first (a batch: chain by chain); there are
 * kcm_nside_joints of them (0 when side_joints = 0, -1 for a NULL handle). They start at 0; the
 * loop (kcm_step) steps them with the main-chain joints as one vector of joint angles: the same
 * clamp or normalisation (max |tau| over the main and side joints of a chain) and the same
 * convergence test (max |dtheta| over both). They are never held fixed (kcm_set_fixed_joints covers
 * the main-chain joints). Arrays are host memory of ls = kcm_nside_joints doubles (rad; kcal/mol per
 * rad); errors: KCM_E_INVAL (ls does not match, NULL array, a non-finite angle). */
int64_t kcm_nside_joints(kcm_handle h);
int kcm_set_side_theta(kcm_handle h, const double* chi, int64_t ls);
int kcm_get_side_theta(kcm_handle h, double* chi, int64_t ls);
/* The same with device pointers (stream-ordered, no synchronisation; no finiteness check). */
int kcm_set_side_theta_dev(kcm_handle h, const double* chi_dev, int64_t ls);
int kcm_get_side_theta_dev(kcm_handle h, double* chi_dev, int64_t ls);
/* torques of the side-chain joints at the current angles: tau = u . sum_s (r_s - a) x F_s over the side
 * atoms s the joint moves, u its current unit bond axis and a the bond's first atom (evaluates) */
int kcm_side_torques(kcm_handle h, double* tau, int64_t ls);
/* side-chain joints of chain c: [side_off[c], side_off[c+1]) (kcm_nchains + 1 entries, host memory) */
int kcm_side_offsets(kcm_handle h, int64_t* side_off);

/* Cell-edge autotuner. For each candidate edge (A; meaning as kcm_params.cell_size, so 0 is the
 * smallest 27-cell edge) evaluate the chain (forces and torques at the current theta, no step:
 * theta is not changed) once to warm up and then `reps` times, timed with CUDA events on the
 * handle's stream; keep the fastest edge for all later calls. The pair set, and so the result,
 * does not depend on the edge: only the rounding of the FP32 cell offsets and the order of
 * floating-point sums do. times_ms[n_candidates] (may be NULL) receives the mean time of one
 * evaluation per candidate; *chosen (may be NULL) the winning candidate. Synchronises. Errors:
 * KCM_E_INVAL (n_candidates not in [1, KCM_AUTOTUNE_MAX], reps not in [1, 1000], a negative
 * or non-finite candidate), the errors of an evaluation (the previous edge is then restored). */
#define KCM_AUTOTUNE_MAX 64
int kcm_autotune_cell(kcm_handle h, const double* candidates, int32_t n_candidates, int32_t reps,
                      double* times_ms, double* chosen);

/* Tile shapes of the warp-per-atom kernels: atoms (warps) per thread block of the pair kernel and of
 * the solvation kernel (Algorithm 1's mixed-precision kernel, or the pairwise surrogate's kernel in
 * either precision), each 1, 2 or 4, and the pair kernel's grid: one block per group of atoms
 * (pair_persistent = 0) or a persistent grid of one block per resident slot, each block taking every
 * so-many-th group (1). Defaults 1, 1, 0. The result does not depend on them (each atom's work is its
 * warp's; sums are exact or the same per atom), only the scheduling does. kcm_set_tiles sets them
 * (synchronises; KCM_E_INVAL for another value); kcm_get_tiles reads them (any pointer may be NULL).
 * kcm_autotune_tiles evaluates the chain at the current theta and cell edge with every combination (a
 * warm-up, then `reps` evaluations timed with CUDA events on the handle's stream) and keeps the
 * fastest: times_ms[18] (may be NULL) indexed [persistent][pair shape][solvation shape], shapes in the
 * order 1, 2, 4; the choice in the three outputs (may be NULL). With the cell-pair tile kernel
 * (KCM_PAIR_CELL_TILES, below) the pair shape is its split instead: the warps that share one window of
 * 32 home slots and one stencil row (each taking every pair_warps-th staged group of 32 candidates);
 * that kernel has no persistent grid, so the other grid's entries repeat the current one's times.
 * Synchronises. Errors: KCM_E_INVAL (reps not in [1, 1000]), the errors of an evaluation (the previous
 * shapes are then restored). */
#define KCM_TILE_CHOICES 3
int kcm_set_tiles(kcm_handle h, int32_t pair_warps, int32_t sasa_warps, int32_t pair_persistent);
int kcm_get_tiles(kcm_handle h, int32_t* pair_warps, int32_t* sasa_warps, int32_t* pair_persistent);
int kcm_autotune_tiles(kcm_handle h, int32_t reps, double* times_ms, int32_t* pair_warps, int32_t* sasa_warps,
                       int32_t* pair_persistent);

/* Pair kernel of mixed precision (A3-A5: Coulomb and LJ forces, exclusions, solvation neighbour
 * lists; eq. 02_2, 03_2, 03_8 / 03_9 and the grid of Sec. 3.2). KCM_PAIR_CELL_TILES: a home cell's
 * atoms against one row of its half stencil staged in shared memory, in-range pairs compacted and
 * evaluated with every lane busy, per-tile fixed-point sums added to the global forces once per atom and
 * tile. KCM_PAIR_WARP_PER_ATOM: one warp per home atom (the FP64 path's kernel; its mixed form takes the
 * tile shapes above). A mixed handle starts with the tile kernel from 65,536 atoms on (batches, long
 * chains) and with the warp-per-atom kernel below (the tile kernel's warps fill the SMs only on large
 * inputs); kcm_autotune_pair_kernel measures both. Both give bitwise the same pair forces and
 * solvation lists (up to the order of a list's entries, which no result depends on); energies agree to
 * FP32 rounding. kcm_set_pair_kernel synchronises and drops the captured graphs; KCM_E_INVAL for
 * another value, or for KCM_PAIR_CELL_TILES on an FP64 handle. kcm_get_pair_kernel reads it. */
#define KCM_PAIR_WARP_PER_ATOM 0
#define KCM_PAIR_CELL_TILES 1
int kcm_set_pair_kernel(kcm_handle h, int32_t kind);
int kcm_get_pair_kernel(kcm_handle h, int32_t* kind);
/* Pair-kernel autotuner: runs kcm_autotune_tiles with each pair kernel (mixed precision; an FP64
 * handle has only the warp-per-atom kernel) and keeps the kernel and tile shapes of the fastest
 * evaluation. times_ms[2] (may be NULL): the best evaluation time of each kernel, indexed by
 * KCM_PAIR_* (0 for a kernel not tried); *kind (may be NULL): the choice. Synchronises; errors as
 * kcm_autotune_tiles (the previous kernel is then restored). */
int kcm_autotune_pair_kernel(kcm_handle h, int32_t reps, double* times_ms, int32_t* kind);

/* Launch overlap in the captured step graphs (on = 1, the default): every kernel of an iteration is
 * launched with programmatic stream serialization and begins by waiting for the previous kernel to
 * complete (griddepcontrol.wait), so that each kernel's launch overlaps the previous one's run; results
 * are unchanged. Worth it when the handle has the GPU to itself (1,000-residue chain: 102.6 -> 101.0 us
 * per iteration); for handles that share the GPU with other streams' kernels it costs more than it saves
 * (the next kernel's blocks hold SM slots while they wait: the serving loop's p50 latency 0.13-0.15 s
 * without, 0.20-0.25 s with), and the serving loop turns it off for its batches. Synchronises and drops
 * the captured graphs. Errors: KCM_E_INVAL (on not 0 or 1). */
int kcm_set_graph_overlap(kcm_handle h, int32_t on);

/* Binning kernel (A2, Sec. 3.2: cell counts, their scan, the atoms in slot order). KCM_BIN_CLUSTER (the
 * default): a single chain of up to 32,768 atoms in mixed precision is binned in one launch of one
 * thread-block cluster of up to 16 CTAs, the cell counts kept in the CTAs' shared memory (atomics through distributed shared
 * memory) and the stages joined by cluster barriers; it applies when the chain's cell cap split over
 * the cluster fits in shared memory (at most 53,248 cells per CTA) and the device can place the
 * cluster. Otherwise, and for batches and FP64, KCM_BIN_BLOCKS: a count kernel whose last block scans
 * the counts, then a placement kernel. The cluster kernel forms an atom's cell and its offset from the
 * cell corner in double-float and rounds once to float, where the blocks round the FP64 difference, so
 * pair forces agree to FP32 rounding, not bit for bit. kcm_set_binning_kernel synchronises and drops
 * the captured graphs; KCM_E_INVAL for another value. kcm_get_binning_kernel reads the kernel in use
 * and the CTAs of its cluster (0 for the blocks; `ctas` may be NULL). */
#define KCM_BIN_BLOCKS 0
#define KCM_BIN_CLUSTER 1
int kcm_set_binning_kernel(kcm_handle h, int32_t kind);
int kcm_get_binning_kernel(kcm_handle h, int32_t* kind, int32_t* ctas);

/* Test only: the torque kernel never publishes the total of link tile `tile` (tiles of 32 links; -1,
 * the default, publishes all), so that the blocks waiting for it give up after their bounded wait
 * (about 0.2 s) and the call reports KCM_E_TIMEOUT, with the device context still usable. It exists to
 * test that failure path; a handle with it set yields no valid torques. Synchronises and drops the
 * captured graphs. Errors: KCM_E_INVAL (tile out of range). */
int kcm_set_test_withhold(kcm_handle h, int32_t tile);

/* Stages of one iteration, in launch order, as timed by kcm_step_timed. */
#define KCM_STAGE_KINEMATICS 0 /* transform scan and atom centres (eq. kin_04, r1, r2) */
#define KCM_STAGE_BINNING 1    /* bounding box, grid, counting sort (Sec. 3.2) */
#define KCM_STAGE_PAIRS 2      /* Coulomb + LJ forces, their energies, solvation neighbour lists */
#define KCM_STAGE_SOLVATION 3  /* Algorithm 1 and the solvation energy */
#define KCM_STAGE_TORQUES 4    /* link wrenches, suffix sums, joint torques (Sec. 3.5) and the step (eq. KCM_07) */
#define KCM_NUM_STAGES 5

/* Run ONE iteration (as kcm_step(h, 1, ...)) through a copy of the iteration graph that records
 * CUDA events between stages on the handle's stream, synchronise, and return the stage durations
 * stage_ms[n_stages] (n_stages <= KCM_NUM_STAGES) and the whole iteration's duration total_ms.
 * Either output may be NULL. Same errors as kcm_step. */
int kcm_step_timed(kcm_handle h, float* stage_ms, int32_t n_stages, float* total_ms);

/* The cudaStream_t the handle works on. */
void* kcm_stream(kcm_handle h);

/* Joint torques from given atom forces without allocating device memory.
 *
 * The paper has no counterpart: this exists for callers that cannot allocate device memory when
 * they need torques, such as a serving process that reserved all GPU memory up front for its own
 * pool allocator (a cudaMalloc there fails or fragments the pool), or a latency-critical host
 * loop that must not wait on the driver's allocator. The computation is the one kcm_torques runs
 * (link wrenches about the origin, suffix sums over links, tau_k = u_k . T^agg_k +
 * (p_k x u_k) . F^agg_k), on data the caller provides.
 *
 * Arguments (all device pointers; nothing is copied or allocated):
 *   n_links      number of links L = l + 1 (the base link 0 plus one per joint), 2..KCM_NOALLOC_MAX_LINKS
 *   link_start   int32[L+1]: the atoms of link h are link_start[h] .. link_start[h+1]-1
 *   xyz, F       double[n*3]: atom centres and forces, n = link_start[L]
 *   axis, point  double[l*3]: unit axis u_k and a point p_k on it for joint k (0-based), joint k
 *                moving links k+1..l
 *   tau          double[l]: output
 *   cuda_stream  cudaStream_t the kernels are launched on (NULL: the legacy default stream)
 * The call only enqueues work; synchronise the stream before reading tau. Returns KCM_E_INVAL for
 * sizes beyond the limit or NULL pointers (nothing is launched), KCM_E_NODEVICE / KCM_E_CUDA when
 * the scratch cannot be located or a launch fails.
 *
 * Scratch: a fixed array of about 2 MB that is part of the library image; every GPU that loads the
 * library holds it until the process exits, which is what limits L. The first call on a device,
 * with that device current, looks up the array's device address (cudaGetSymbolAddress) and keeps it
 * for the life of the process; make that first call before any stream capture. Do not call this
 * entry point again on a device after cudaDeviceReset (or after its primary context was released
 * and made again) in the same process: the library reloads with the new context and the kept address
 * may no longer be the array's. All calls on a device share the array and each call
 * writes every scratch word it reads, so nothing carries over from an earlier call; calls that
 * overlap on the GPU (different streams, or different host threads) race on it. */
#define KCM_NOALLOC_MAX_LINKS 32768
int kcm_torques_noalloc(int32_t n_links, const int32_t* link_start, const double* xyz, const double* F,
                        const double* axis, const double* point, double* tau, void* cuda_stream);

/* Host-only helpers (no device needed). */

/* The unit-sphere sample set Q[N*3] of Sec. 3.4: K = round(sqrt(pi N / 4)) latitude rings at polar
 * angles pi (r - 1/2) / K, ring r holding a share of N proportional to the sine of its polar
 * angle (largest-remainder rounding, ties to the lower ring), point t of ring r at longitude
 * 2 pi (t + (r mod 2)/2) / n_r; listed ring by ring. Returns KCM_OK or KCM_E_INVAL (N < 1). */
int kcm_sample_points(int32_t N, double* Q);

/* The ZP coordinates xyz0[n*3] and link index link[n] of a topology, as kcm_create builds them
 * (n must equal the chain's atom count). Either output may be NULL. */
int kcm_build_zp(const kcm_topology* top, double* xyz0, int32_t* link, int64_t n);

/* Bond class of atom pairs of a topology as the kernels see them: 0 = interacts fully,
 * 1 = excluded (1-2 or 1-3), 2 = 1-4 (weighted by w14). Writes n_pairs classes for the index
 * pairs a[k], b[k]. */
int kcm_pair_class(const kcm_topology* top, const int32_t* a, const int32_t* b, int64_t n_pairs, int32_t* cls);

/* Atom count of a topology (or a negative status). */
int64_t kcm_topology_natoms(const kcm_topology* top);

const char* kcm_strerror(int code);
const char* kcm_last_error(kcm_handle h);

#ifdef __cplusplus
}
#endif

#endif /* KCM_H */
