/*
 * dpslab.h -- C ABI of the doubly-periodic slab spectral Ewald solver.
 *
 * The solver computes, for N Gaussian charges (Eq. (gcharge), width g_w) in a
 * slab 0 < z < H that is periodic on [0, Lx) x [0, Ly), with permittivity eps
 * inside, eps_b below z = 0 and eps_t above z = H (Sec. 2):
 *   - the Gaussian-averaged potential phibar_k at every charge, Eq. (pbar),
 *     in the gauge phi(0) = 0, Eq. (phi00);
 *   - the force F_k = q_k Ebar(z_k), Eq. (fqE);
 *   - the energy U = 1/2 sum_k q_k phibar_k of Eq. (Ufinal), plus, when wall
 *     charge densities are set (dpslab_plan_set_wall_charge), their term
 *     1/2 int (sigma_b phi(x, y, 0) + sigma_t phi(x, y, H)) dx dy.
 * It follows the far-field algorithm of Sec. 5.2.2 (steps 1-7, a Fourier
 * grid in x, y and a second-kind Chebyshev grid in z on [-3 H_E, H + 3 H_E],
 * one boundary value problem per transverse mode solved as in Appendix A,
 * the harmonic correction Eq. (inphisc) and the k = 0 mode of Sec. 4.3.4)
 * plus the near field of Sec. 4.2 over a cell list.
 *
 * Units are those of the paper: rationalised electrostatics, a Gaussian
 * charge interacts as q / (4 pi eps r) at long range; there is no Coulomb
 * constant.
 *
 * Conventions for every call:
 *   - Return value 0 (DPSLAB_OK) or a negative DPSLAB_ERR_* code; the
 *     message is dpslab_strerror(code). No call aborts the process.
 *   - Pointers documented "device" must be CUDA device pointers on the
 *     plan's device, "host" ones ordinary host memory. The caller owns
 *     every buffer it passes; the plan owns all its work space.
 *   - Arrays are dense, row-major, double precision, with no padding.
 */
#ifndef DPSLAB_H
#define DPSLAB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ codes */
#define DPSLAB_OK                     0
#define DPSLAB_ERR_INVALID_ARG       -1  /* a parameter is out of range or a pointer is NULL */
#define DPSLAB_ERR_NOT_NEUTRAL       -2  /* |sum q + wall charges| > 1e-12 (sum |q| + |wall charges|) (Eq. (elecneu)) */
#define DPSLAB_ERR_OUT_OF_SLAB       -3  /* a charge has z outside (0, H) or a non-finite value */
#define DPSLAB_ERR_CUTOFF_TOO_LARGE  -4  /* r_cut >= min(Lx, Ly)/2: nearest-image rule of Sec. 4.2 fails */
#define DPSLAB_ERR_SPLIT_CONSTRAINT  -5  /* strict mode: 2 H_E >= H or r_cut >= H (Sec. 5.3, Table (ewconstraints)) */
#define DPSLAB_ERR_CAPACITY          -6  /* n > max_n of the plan */
#define DPSLAB_ERR_CUDA              -7  /* a CUDA runtime call failed */
#define DPSLAB_ERR_NO_DEVICE         -8  /* no usable CUDA device */
#define DPSLAB_ERR_GRID              -9  /* grid too small for the Gaussian support, or a size the kernels do not support */
#define DPSLAB_ERR_UNSUPPORTED      -10  /* option not built into this library */
#define DPSLAB_ERR_BD_REJECTED      -11  /* every proposal of a Brownian-dynamics step left the slab */
#define DPSLAB_ERR_TIMEOUT          -12  /* a bounded wait on the tensor-core pipeline gave up (dpslab_plan_set_wait_limit) */
#define DPSLAB_PENDING                1  /* dpslab_solve_poll: the enqueued solve has not finished yet */

/* ------------------------------------------------------------- precision */
#define DPSLAB_FP64   0   /* every stage in double precision */
#define DPSLAB_MIXED  1   /* FP32 spreading, FFT, interpolation and near field; the z Chebyshev
                             transforms as tensor-core GEMMs on three-piece BF16 splits with FP32
                             accumulation (Nz <= 256 and ny (nx/2+1) even; otherwise as
                             DPSLAB_MIXED_SIMT); the banded BVP of k != 0 in FP32; in double:
                             the whole k = 0 mode (z transform, BVP, slope A_i), every mode's
                             boundary-condition correction (mismatches, coefficients of
                             Eq. (inphisc)), the gauge and the energy reduction */
#define DPSLAB_MIXED_SIMT 2  /* DPSLAB_MIXED with the z transforms in FP32 on the CUDA cores */

/* Bits of dpslab_derived.violations (Sec. 5.3): */
#define DPSLAB_VIOL_FAR_FIELD   1  /* 2 H_E >= H: images of images reach [-H_E, H+H_E] (Eq. (farconstraint), with h = 0) */
#define DPSLAB_VIOL_NEAR_FIELD  2  /* r_cut >= H: a second image would be needed (Eq. (nearapprox), n_img = 1, h = 0) */

/*
 * Problem and discretisation. Fields set to 0 are derived (Sec. 5.1):
 *   tol      1e-4 (~4 digits) or 5e-4 (~3 digits) -> h factor c_h (1.4 / 1.2)
 *            and Gaussian support n_g (12 / 10), Table (ewconstraints);
 *   xi       0: paper rule g_t = c_h h_xy, xi from Eq. (gt) -- unless r_cut
 *            is given, then xi is the smallest value with
 *            |dGbar(r_cut; g_w, xi)/dr| < tol |dGbar(r_cut; g_w, 0)/dr|
 *            (Eq. (GnearK)), for grids that resolve g_w itself;
 *            INFINITY: no splitting (the smooth solver of Sec. 3.1, no near field);
 *   r_cut    0: r_nf of Eq. (rnf) + n_sigma g_w;
 *   nz       0: ceil(pi (H + 6 H_E) / (2 h_xy)), Sec. 5.1;
 *   n_sigma  0: n_g / (2 c_h); H_E = n_sigma g_t, Eq. (He).
 * eps_b or eps_t = INFINITY selects a metallic wall (the eps_w -> inf limit
 * of every formula; with one metallic wall the k = 0 slope uses the other
 * wall's displacement condition, with two the walls are at equal potential).
 */
typedef struct dpslab_params {
    double Lx, Ly, H;          /* box [0,Lx) x [0,Ly), slab 0 < z < H; > 0            */
    double eps, eps_b, eps_t;  /* permittivities; > 0, eps_b/eps_t may be INFINITY    */
    double gw;                 /* Gaussian charge width g_w > 0                        */
    double tol;                /* 1e-4 or 5e-4                                         */
    int    nx, ny, nz;         /* grid; nx, ny >= 4 required; nz 0 = derive            */
    double xi;                 /* splitting parameter; 0 = derive; INFINITY = none     */
    double r_cut;              /* near-field cutoff; 0 = derive                        */
    double n_sigma;            /* Gaussian truncation in standard deviations; 0 = table */
    int    precision;          /* DPSLAB_FP64, DPSLAB_MIXED or DPSLAB_MIXED_SIMT        */
    int    strict;             /* nonzero: constraint violations are errors            */
} dpslab_params;

/* Every derived quantity of a parameter set (host values). */
typedef struct dpslab_derived {
    double hx, hy, h;          /* grid spacings; h = max(hx, hy) = h_xy                */
    double xi, gt;             /* splitting parameter, g_t of Eq. (gt)                 */
    double n_sigma, HE;        /* truncation, H_E = n_sigma g_t                        */
    double r_cut, r_nf;        /* near-field cutoff (r_nf = 0 when r_cut was given)    */
    double a, b, Hbar;         /* Chebyshev domain [a, b] = [-3 H_E, H + 3 H_E]         */
    double kmax;               /* correction applied for 0 < |k| <= kmax = pi / h_xy   */
    int    nx, ny, nz;
    int    support_x, support_y;  /* maximum Gaussian support in grid points          */
    int    violations;         /* DPSLAB_VIOL_* bits                                   */
} dpslab_derived;

typedef struct dpslab_plan dpslab_plan;

/*
 * Derive every quantity of Sec. 5.1 / Table (ewconstraints) from p, on the
 * host only (no CUDA call). Returns DPSLAB_ERR_INVALID_ARG for bad
 * parameters, DPSLAB_ERR_GRID / _CUTOFF_TOO_LARGE / _SPLIT_CONSTRAINT as
 * dpslab_plan_create would.
 */
int dpslab_derive(const dpslab_params* p, dpslab_derived* out);

/*
 * Host copies of plan tables, for inspection (no CUDA call):
 *   which = 0: Chebyshev nodes z_j, j = 0..nz-1 (z_0 = b, z_{nz-1} = a), Sec. 5.2.2;
 *           1: quadrature weights of the z grid (Clenshaw-Curtis, Hbar/2 scaled);
 *           2: gauge weights int gamma_z(z) T_n(s(z)) dz, n = 0..nz-1.
 * out must hold nz doubles.
 */
int dpslab_table(const dpslab_params* p, int which, double* out, int n_out);

/*
 * Create a plan on the current CUDA device for up to max_n charges:
 * derives the parameters, builds the tables and allocates all device work
 * space (the only allocation; dpslab_solve allocates nothing).
 * *out receives the plan, or NULL on error.
 */
int dpslab_plan_create(const dpslab_params* p, int64_t max_n, dpslab_plan** out);

/* The derived parameters of a plan. */
int dpslab_plan_derived(const dpslab_plan* plan, dpslab_derived* out);

/* Bytes of device memory the plan holds. */
int64_t dpslab_plan_device_bytes(const dpslab_plan* plan);

/*
 * Wall charge densities (Eq. (rho) and Sec. 4.3.1, the paper's sigma_b at
 * z = 0 and sigma_t at z = H), fixed for every later solve of the plan.
 *   sigma_b, sigma_t  host arrays of ny*nx doubles, [j*nx + i] the density at
 *                     (i*hx, j*hy) (nx, ny the plan's grid); NULL for an
 *                     uncharged wall. Both NULL removes the wall charges.
 *   stream            CUDA stream (cudaStream_t) for the set-up work.
 * They enter the displacement mismatches Eq. (mm2), (mm4) for 0 < |k| <= pi/h
 * (modes above are dropped: the density must be resolved by the grid) and
 * Eq. (ai1), (ai2) for k = 0, so potentials and forces include their field.
 * The energy gains 1/2 int (sigma_b phi(x, y, 0) + sigma_t phi(x, y, H)),
 * evaluated per xy mode: for k = 0 from the plane-averaged potential at the
 * walls (far field plus the near field's planar integral in closed form), for
 * k != 0 by Green's reciprocity (the wall charges' own correction averaged
 * at the charges, plus its Parseval self term), so -dU/dz_k is the force.
 * Electroneutrality (Eq. (elecneu)) then covers charges and wall charges
 * together. The set-up runs once: two xy transforms, the correction grid
 * (one grid of the plan's precision, held by the plan) and its self term;
 * each solve adds one gather kernel. Needs a bound workspace (its arrays are
 * used as scratch) and no solve in flight. Errors: DPSLAB_ERR_INVALID_ARG
 * (no workspace, a solve in flight, non-finite values),
 * DPSLAB_ERR_UNSUPPORTED (a charge density on a metallic wall),
 * DPSLAB_ERR_CUDA.
 */
int dpslab_plan_set_wall_charge(dpslab_plan* plan, const double* sigma_b, const double* sigma_t, void* stream);

/*
 * Brownian dynamics of the ions (Sec. 7.1): one step of Eq. (leimkuhler)
 *   z^{n+1} = z^n + mu (F_steric(z^n) + F(z^n)) dt + sqrt(kT mu dt / 2) (W^n + W^{n+1})
 * with F the electrostatic force of a solve with this plan (Eq. (fqE)) and
 * F_steric the capped Lennard-Jones repulsion of Eq. (steric), (lj) between
 * ions (nearest periodic image in x, y) and between each ion and its own
 * mirror image in each wall.
 */
typedef struct dpslab_bd_params {
    double dt;          /* time step */
    double mu;          /* scalar mobility */
    double kT;          /* thermal energy */
    double a;           /* ion radius: the repulsion acts below 2^(1/p) 2a */
    double U0;          /* strength of Eq. (lj) */
    double r_m;         /* below r_m the force is F_LJ(r_m) */
    int p;              /* exponent of Eq. (lj), >= 1 */
    int max_retries;    /* proposals per step, 1 .. DPSLAB_BD_MAX_RETRIES */
    double max_disp;    /* > 0: an ion's displacement per step is capped at this length */
    uint64_t seed;      /* key of the noise generator */
} dpslab_bd_params;

#define DPSLAB_BD_MAX_RETRIES 32

/*
 * The noise W_i = (W_x, W_y, W_z) of ion i at (step, retry): Philox4x32-10
 * (Salmon et al., SC 2011) with key = seed and counter = (i, step low word,
 * step high word, retry); its four words u_k = (w_k + 1/2) 2^-32 give two
 * Box-Muller pairs, of which the first three numbers are used. W^{n+1} of step
 * n is drawn with step index n + 1. This call writes W^0 (step 0, retry 0)
 * for n ions into the device array W [n][3] on `stream`.
 */
int dpslab_bd_init_noise(uint64_t seed, int64_t n, double* W, void* stream);

/*
 * Enqueue step `step` (n -> n + 1) on `stream` and return at once; completion
 * and errors through dpslab_solve_poll (the plan is in flight until then).
 *   pos    device [n][3] positions z^n, replaced by z^{n+1} (x, y wrapped into
 *          the box) when the step is accepted
 *   q      device [n] charges (electroneutral with any wall charges)
 *   W      device [n][3] noise W^n, replaced by the accepted W^{n+1}
 *   force  device [n][3] receives the electrostatic force at z^n, or NULL
 * The solve at z^n, the steric forces (on the solve's cell list) and up to
 * max_retries proposals run as kernels in stream order. A proposal with any
 * ion outside 0 < z < H is discarded and the next one (new W^{n+1}) tried;
 * if all are discarded nothing changes and the poll returns
 * DPSLAB_ERR_BD_REJECTED. Requires the near field (xi finite) with
 * 2^(1/p) 2a <= r_cut; the energy is computed as in dpslab_solve.
 * Errors at enqueue: DPSLAB_ERR_INVALID_ARG, DPSLAB_ERR_CAPACITY, DPSLAB_ERR_CUDA.
 */
int dpslab_bd_step_enqueue(dpslab_plan* plan, const dpslab_bd_params* bp, int64_t n, double* pos, const double* q,
                           double* W, uint64_t step, double* force, void* stream);

/* Proposals discarded by the last completed step (0 .. max_retries). */
int dpslab_bd_last_retries(const dpslab_plan* plan);

/*
 * Launch-shape autotuning. DPSLAB_NKNOBS knobs set the launch shapes of the
 * solve's kernels:
 *   knobs[0]  x forward FFT: rows per block     knobs[1]  y forward FFT: columns per block
 *   knobs[2]  y inverse FFT: columns per block  knobs[3]  x inverse FFT: rows per block
 *   knobs[4]  interpolation: charges (warps) per block: 1, 2, 4 or 8
 *   knobs[5]  column kernel (per-mode BVP): k modes per block: 8, 16 or 32
 *             (DPSLAB_MIXED with tensor-core z transforms), 4 or 8 (with
 *             CUDA-core z transforms), 2 or 4 (DPSLAB_FP64)
 *   knobs[6]  spreading: x grid columns per thread: 1, 2 or 4 (DPSLAB_MIXED),
 *             1 (DPSLAB_FP64)
 * A value sets the block size and shared memory of its kernel; the results
 * do not depend on it beyond the order of floating-point sums. The FFT knobs
 * take 1, 2, 4, ..., 32 within the kernel's thread and shared-memory limits.
 * dpslab_plan_autotune runs the solve on the caller's device inputs (as
 * dpslab_solve, outputs discarded), and for each knob in turn times its
 * stage with CUDA events (median of `reps` solves after one warm-up) at each
 * allowed value, keeping a value only when it is at least 2% faster. Needs a
 * bound workspace and no solve in flight. dpslab_plan_tuning writes the
 * first n >= 4 knobs (n < DPSLAB_NKNOBS: the FFT knobs only);
 * dpslab_plan_set_tuning applies the first n >= 4 knobs (for example cached
 * from an earlier autotune of the same grid) and leaves the others; it
 * returns DPSLAB_ERR_INVALID_ARG and changes nothing if a value is outside
 * its kernel's limits.
 */
#define DPSLAB_NKNOBS 7
int dpslab_plan_autotune(dpslab_plan* plan, int64_t n, const double* pos, const double* q, int reps, void* stream);
int dpslab_plan_tuning(const dpslab_plan* plan, int* knobs, int n);
int dpslab_plan_set_tuning(dpslab_plan* plan, const int* knobs, int n);

/*
 * A plan without a workspace: tables and derived parameters only (a few MB);
 * the caller binds a workspace of at least dpslab_plan_work_bytes bytes with
 * dpslab_plan_bind_work before solving. Serving loops keep many such plans
 * resident and give the large per-solve arrays (grids, cell list) only to
 * the solves admitted at a time. Errors as dpslab_plan_create.
 */
int dpslab_plan_create_unbound(const dpslab_params* p, int64_t max_n, dpslab_plan** out);

/* Bytes of the per-solve workspace the plan needs (grids, spectra, field
 * grids, charge arrays, buckets, cell list, partial sums). */
int64_t dpslab_plan_work_bytes(const dpslab_plan* plan);

/*
 * Bind the caller's device workspace to an unbound plan: `work` (256-byte
 * aligned, at least dpslab_plan_work_bytes bytes) is carved into the plan's
 * per-solve arrays and used by every later solve until rebound; work == NULL
 * unbinds (solves then fail with DPSLAB_ERR_INVALID_ARG). The caller keeps
 * ownership and must not free or reuse it while a solve of the plan is in
 * flight; nothing in it needs to survive between solves, so plans may take
 * turns on one workspace. DPSLAB_ERR_INVALID_ARG for a plan that owns its
 * workspace (dpslab_plan_create), one with a solve in flight, a misaligned
 * pointer or too few bytes.
 */
int dpslab_plan_bind_work(dpslab_plan* plan, void* work, int64_t bytes);

/*
 * Bytes of device memory dpslab_plan_create(p, max_n) would take, computed on
 * the host without a device and without allocating (for admission control
 * by memory footprint). Errors as dpslab_plan_create's parameter checks;
 * *bytes is 0 on error.
 */
int dpslab_plan_footprint(const dpslab_params* p, int64_t max_n, int64_t* bytes);

/*
 * One solve (Sec. 5.2.2 far field + Sec. 4.2 near field + gauge + energy).
 *   n        number of charges, 1 <= n <= max_n;
 *   pos      device, [n][3] (x, y, z); x and y are wrapped into [0, L);
 *            z must lie in (0, H);
 *   q        device, [n] charges; sum must vanish (Eq. (elecneu));
 *   U        host scalar, or NULL;
 *   phi      device, [n] averaged potentials, or NULL;
 *   force    device, [n][3] forces, or NULL;
 *   stream   cudaStream_t to run on (NULL = legacy default stream).
 * The call enqueues all work on stream and waits for it before returning
 * (it reads back the status word and U). Invalid charges do not fault: they
 * are replaced by zero charges and the call returns DPSLAB_ERR_OUT_OF_SLAB.
 */
int dpslab_solve(dpslab_plan* plan, int64_t n, const double* pos, const double* q,
                 double* U, double* phi, double* force, void* stream);

/*
 * Same as dpslab_solve with host buffers: copies pos and q to the device,
 * solves, and copies phi and force back (each output may be NULL). Host
 * buffers that are page-locked copy faster.
 */
int dpslab_solve_host(dpslab_plan* plan, int64_t n, const double* pos, const double* q,
                      double* U, double* phi, double* force, void* stream);

/*
 * Copy an intermediate device buffer of the last solve to host memory, for
 * stage-by-stage checks:
 *   which = 0: rho_i then rho_o, 2 x [nz][ny][nx] (Sec. 5.2.2 steps 2-3);
 *           1: fields phi, E_x, E_y, E_z on the grid, [nz][ny][nx][4];
 *           2: far-field phibar, Ebar at the charges, [n][4];
 *           3: near-field phibar, Ebar at the charges, [n][4];
 *           4: scalars (B_i(0), A_i(0), phi^(f)(0), phi^(n)(0)).
 * bytes must equal the buffer's size for that n.
 */
int dpslab_debug_fetch(dpslab_plan* plan, int which, void* host_dst, size_t bytes);

/* Number of kernels the last solve launched. */
int dpslab_last_launch_count(const dpslab_plan* plan);

/*
 * Asynchronous form of dpslab_solve, for serving loops that overlap many
 * solves. dpslab_solve_enqueue validates the arguments and enqueues the
 * whole solve on `stream` (the same work as dpslab_solve), then returns
 * without waiting. dpslab_solve_poll never blocks. It returns DPSLAB_PENDING
 * while the enqueued solve runs, and then the solve's own result code, as
 * dpslab_solve would have returned it, with *U set (U may be NULL). At most
 * one solve per plan may be in flight; enqueueing another before the poll
 * has returned a result gives DPSLAB_ERR_INVALID_ARG. The output buffers
 * must stay valid until then.
 */
int dpslab_solve_enqueue(dpslab_plan* plan, int64_t n, const double* pos, const double* q, double* phi,
                         double* force, void* stream);
int dpslab_solve_poll(dpslab_plan* plan, double* U);

/*
 * Batches of independent systems, each with its own box, walls, grid and
 * charge count (the paper's solve, per system; systems never interact).
 *
 * dpslab_batch_create makes one plan per system (params[i], max_n[i]: as
 * dpslab_plan_create) and nstreams CUDA streams (1 <= nstreams; at most
 * count are used). System i runs on stream i mod nstreams. The plans of one
 * stream share one workspace sized for the largest of them, since they run
 * one after another. The batch's device footprint is therefore the tables of
 * every system plus nstreams workspaces (dpslab_batch_device_bytes). Errors
 * are as dpslab_plan_create, for the first system that fails; nothing is
 * left allocated then.
 *
 * dpslab_batch_solve solves every system. It forks the caller's stream into
 * the batch's streams, enqueues the solves there and joins them back, in
 * one of two schedules (dpslab_batch_set_schedule). DPSLAB_BATCH_STREAMS:
 * system i's whole solve runs on stream i mod nstreams. DPSLAB_BATCH_WAVES:
 * in waves of nstreams systems (systems w .. w + nstreams - 1, whose
 * workspaces are distinct), each system's solve runs up to its column stage
 * on its stream; then the column stage of the whole wave (the per-mode BVP,
 * Appendix A, and the boundary-condition correction, Sec. 4.3.3, whose
 * modes are independent, Sec. 5.2.2) runs as one launch per kind of column
 * kernel over every k mode of every system of the wave; then the rest of
 * each solve on its stream. With nstreams >= count the batch is one wave.
 * The first call with a given set of arguments (the n[i], every pointer and
 * the schedule) captures this into a CUDA graph; later calls with the same
 * arguments replay it (new values in the same buffers are fine). It returns
 * when the batch is done.
 *   n[count]; pos[count] ([n_i][3] device), q[count] ([n_i] device): the
 *   inputs of system i, as dpslab_solve.
 *   U[count]: host, may be NULL; phi, force: arrays of count device
 *   pointers, may be NULL, and so may their entries (that output is skipped).
 *   status[count]: host, may be NULL; the dpslab_solve code of each system.
 * Returns DPSLAB_OK if every system succeeded, else the code of the first
 * failing one. A batch is not thread-safe; one call at a time per batch.
 */
typedef struct dpslab_batch dpslab_batch;
int dpslab_batch_create(const dpslab_params* params, const int64_t* max_n, int count, int nstreams,
                        dpslab_batch** out);
int dpslab_batch_solve(dpslab_batch* batch, const int64_t* n, const double* const* pos, const double* const* q,
                       double* U, double* const* phi, double* const* force, int* status, void* stream);
int64_t dpslab_batch_device_bytes(const dpslab_batch* batch);
/* Kernels the last dpslab_batch_solve launched, over all systems. */
int dpslab_batch_last_launch_count(const dpslab_batch* batch);
/*
 * Schedule of a batch solve:
 *   DPSLAB_BATCH_STREAMS (the default): each system's whole solve runs on
 *     its stream, and the streams run freely beside one another;
 *   DPSLAB_BATCH_WAVES: the waves described above, with the column stage of
 *     each wave as one launch per kind of column kernel (and per 21 systems)
 *     over all its systems' k modes.
 * Both give the same results. dpslab_batch_set_schedule returns
 * DPSLAB_ERR_INVALID_ARG for any other value; the next solve captures a new
 * graph. dpslab_batch_autotune times both schedules on the caller's device
 * inputs (as dpslab_batch_solve, outputs discarded; the median of `reps`
 * solves after one warm-up each, CUDA events on `stream`) and keeps the
 * other schedule only when it is at least 2% faster.
 */
#define DPSLAB_BATCH_STREAMS 0
#define DPSLAB_BATCH_WAVES   1
int dpslab_batch_set_schedule(dpslab_batch* batch, int schedule);
int dpslab_batch_schedule(const dpslab_batch* batch);
int dpslab_batch_autotune(dpslab_batch* batch, const int64_t* n, const double* const* pos, const double* const* q,
                          int reps, void* stream);
int dpslab_batch_destroy(dpslab_batch* batch);

/*
 * Per-stage timing. With profiling on, every solve records CUDA events on its
 * stream around each stage; dpslab_stage_times writes the last solve's
 * stage durations in milliseconds (device time) to ms[0 .. DPSLAB_NSTAGES-1].
 * Stage i is named by dpslab_stage_name(i): prepare (validation, cell
 * list), spread (sources, buckets, spreading), fft_x_fwd, fft_y_fwd, z_fwd
 * (the k = 0 column in double, then the tensor-core z transform; only the
 * former when the z transforms run inside the BVP kernel), bvp (per-mode
 * BVP, correction coefficients), z_inv (tensor-core inverse z transform with
 * the correction at the nodes; 0 as z_fwd), fft_y_inv, fft_x_inv, interp,
 * near (pairs), finish (gauge + assembly + energy).
 * on: 0 = off; 1 = on, the solve unchanged: the near field still runs on the
 * plan's second stream beside the far field, and its stage time is taken by
 * events on that stream (the stage times then add up to more than the
 * solve); 2 = on, with the near field run in line on the solve's stream, so
 * that the stages follow one another. Other values: DPSLAB_ERR_INVALID_ARG.
 */
/*
 * Watchdog of the tensor-core z transforms (DPSLAB_MIXED with Nz <= 256).
 * Their kernels wait on the tensor cores and on bulk copies with bounded
 * waits of at most `polls` polls each (default 2^26, seconds); a wait that
 * runs out makes the kernel stop, wait for the work it has in flight, free
 * its tensor memory and return, and the solve then reports
 * DPSLAB_ERR_TIMEOUT (its outputs are not valid; the plan stays usable).
 * polls = 0 makes every such wait give up at once, which is how that path is
 * tested. Returns DPSLAB_ERR_INVALID_ARG for polls < 0 or a solve in flight.
 * Not part of the paper's method.
 */
int dpslab_plan_set_wait_limit(dpslab_plan* plan, int64_t polls);

#define DPSLAB_NSTAGES 12
int dpslab_profile(dpslab_plan* plan, int on);
int dpslab_stage_times(const dpslab_plan* plan, double* ms, int n);
const char* dpslab_stage_name(int stage);

/*
 * Near field only, allocating nothing (the paper has no counterpart: this
 * call exists for callers that cannot call cudaMalloc, e.g. code running
 * inside an allocator's callbacks, under a device memory pool that must not
 * grow, or in a loop that reserves all memory up front). It computes the
 * same near-field part as dpslab_solve (Gaussian-averaged kernels, one image
 * per wall, pairs closer than r_cut) without a plan:
 *   p        parameters as for dpslab_plan_create (derived on the host);
 *   n        1 <= n <= 65536 charges, else DPSLAB_ERR_CAPACITY; the cell
 *            list may have at most 65536 cells (floor(Lx/r_cut) *
 *            floor(Ly/r_cut) * floor(H/r_cut)), else DPSLAB_ERR_CAPACITY;
 *   pos, q   device, [n][3] and [n], as for dpslab_solve;
 *   out      device, [n][4]: near-field phibar and Ebar (x, y, z) per charge;
 *   stream   cudaStream_t (NULL = legacy default stream).
 * The scratch space is one file-scope device array of about 8.3 MiB that every
 * GPU loading this library holds until the process exits. All calls share
 * it: calls that overlap on the GPU (other streams, other threads) race and
 * must be serialised by the caller. The first call on a device looks up the
 * array's device address; make that first call before any stream capture.
 * The call waits for its stream before returning.
 */
int dpslab_near_field_static(const dpslab_params* p, int64_t n, const double* pos, const double* q,
                             double* out, void* stream);

/* Release the plan and all its device memory; NULL is accepted. */
int dpslab_plan_destroy(dpslab_plan* plan);

/* Static message for an error code. */
const char* dpslab_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* DPSLAB_H */
