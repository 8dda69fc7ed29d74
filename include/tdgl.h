/*
 * tdgl.h -- C ABI of the GB300 implicit TDGL solver.
 *
 * The solver advances the complex order parameter psi of the dimensionless
 * time-dependent Ginzburg-Landau equation (arXiv:1409.8340, Sec. 2, Eq.
 * GL_dimensionless with the external-current gauge of Eq. GL_external_current)
 * on an Nx x Ny x Nz grid, together with the scalar potential mu (Eq. Poisson)
 * and the phase-gradient variable K (Eq. K_ODE).  Each time step is the
 * Crank-Nicolson step of Eq. GL_numCN, linearised with |psi_est|^2 = |psi^-|^2,
 * solved by Jacobi iteration (Eq. final) to the squared max-norm tolerance of
 * Eq. convergence; then K (periodic x) and mu are updated (Sec. 3, order psi,
 * K, mu).
 *
 * Conventions for every entry point:
 *   - Return value: TDGL_OK (0) or a negative TDGL_ERR_* code.  No exception
 *     crosses the ABI.  tdgl_error_string() names a code.
 *   - Grid index m = i + Nx*(j + Ny*k), x fastest (Sec. 3).  Complex arrays
 *     are interleaved float pairs (re, im) = 8 bytes per site.
 *   - Device memory is owned by the caller.  The library never allocates
 *     device memory: tdgl_create() carves its arrays out of a caller-provided
 *     workspace of tdgl_workspace_bytes() bytes, and the caller keeps it alive
 *     until tdgl_destroy().  The handle itself is a small host object.
 *   - All work is enqueued on the stream given at creation (a cudaStream_t
 *     passed as void*; NULL = legacy default stream).  Entry points that return
 *     host-visible results synchronise that stream; the others are asynchronous.
 *   - A handle is used by one host thread and one stream at a time.
 *   - After TDGL_ERR_NOT_CONVERGED or TDGL_ERR_NONFINITE from a step, the
 *     state (psi, mu, K) is left at the last completed step.
 */
#ifndef TDGL_H
#define TDGL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TDGL_OK 0
#define TDGL_ERR_INVALID_ARG (-1)
#define TDGL_ERR_NOT_CONVERGED (-2)
#define TDGL_ERR_NONFINITE (-3)
#define TDGL_ERR_TIMEOUT (-4)
#define TDGL_ERR_CUDA (-5)
#define TDGL_ERR_WORKSPACE (-6)

#define TDGL_PERIODIC 0
#define TDGL_OPEN 1

#define TDGL_LINKS_LANDAU 0   /* yz-plane field, Landau gauge A = xbar [0, Bz, -By] (Eq. A_yz) */
#define TDGL_LINKS_GENERAL 1  /* explicit per-link phases (gauge tests)                         */
#define TDGL_LINKS_XZ 2       /* xz-plane field, Landau gauge A = ybar [-Bz, 0, Bx] (Eq. A_xz)   */

/*
 * Problem description.
 *   nx, ny, nz      grid points per axis (nx, ny >= 2; nz >= 1, nz = 1 is a film).
 *   bc[3]           TDGL_PERIODIC or TDGL_OPEN per axis (Sec. 3.3).  Periodic x
 *                   with a field uses the quasi-periodic wrap phase of Sec. 3.3.1;
 *                   periodic x and y then require Bz Lx Ly = 2 pi n_z, periodic x
 *                   and z require By Lx Lz = 2 pi n_y (flux quantisation).  In the
 *                   xz gauge the wrap is along y instead: periodic y and x require
 *                   Bz Lx Ly = 2 pi n_z, periodic y and z require Bx Ly Lz = 2 pi n_x.
 *   hx, hy, hz      grid spacings in units of xi_0 (L = N h periodic, (N-1) h open).
 *   g               anisotropy: z derivatives carry 1/g^2 (Sec. 2.1).
 *   u, beta         u of Eq. GL_dimensionless (absorbed into ht as in the
 *                   footnote of Eq. GL_numCN) and the |psi|^2 psi coefficient.
 *   ht              time step h_t.
 *   By, Bz          field in the yz plane, units of H_c2(0) (Eq. B_yz); in the xz
 *                   gauge By must be 0.
 *   Jext            applied current along x.  Periodic x: enters through the K
 *                   ODE (Eq. K_ODE).  Open x: injected as normal current through
 *                   the x faces via the Neumann condition d(mu)/dx = -Jext.
 *   eps             Jacobi tolerance on max_m |r_m|^2 (Eq. convergence).
 *   max_iter        sweep cap per step; exceeding it is TDGL_ERR_NOT_CONVERGED.
 *   check_every     convergence is tested after every check_every-th sweep
 *                   (1 = the paper's per-sweep test).
 *   fixed_sweeps    > 0: run exactly this many sweeps per step, no test.
 *   freeze_mu_K     1: keep mu and K fixed (no K ODE, no Poisson solve).
 *   poisson_cycles  multigrid V-cycles per step (>= 1).
 *   poisson_tol     > 0: keep cycling (up to poisson_max_cycles) until
 *                   max|F - Lap mu| <= poisson_tol * max|F|.
 *   links_mode      TDGL_LINKS_LANDAU (field (0, By, Bz)), TDGL_LINKS_XZ (field
 *                   (Bx, 0, Bz), links built on the device from FP64 phases and kept
 *                   as a 3N table; tdgl_batch_*, the adjoint and tdgl_sweep_noalloc
 *                   take Landau links only) or TDGL_LINKS_GENERAL.
 *   sweeps_per_pass 0 or 1: one Jacobi sweep per pass over memory.  2: where the
 *                   grid allows (Landau links, nx even), two sweeps per pass
 *                   (temporal blocking) with the per-sweep test kept exactly, so
 *                   the results are those of one sweep at a time (to FP32
 *                   rounding).  On GB300 the two-sweep pass is slower than two
 *                   single sweeps at every size measured, so 1 is the default.
 *   noise_T         thermal noise of Eq. b (Sec. 3.1.2): the grid-independent
 *                   parameter T_zeta = h_t hx hy hz zeta_max^2 (hz dropped on a
 *                   film); 0 = no noise.  Each step adds h_t zeta_m to b_m with
 *                   zeta = zeta_max (v1 + i v2), v1, v2 uniform on [-1, 1) drawn by
 *                   Philox4x32-10 with counter (site m, step n) and key noise_seed;
 *                   n counts the handle's steps since creation or the last
 *                   tdgl_set_state / tdgl_upload_state, or is set by tdgl_set_step.
 *   noise_seed      key of the noise generator.
 *   Bx              field along x (Eq. B_xz), TDGL_LINKS_XZ only (0 otherwise).
 *   sweep_kernel    Jacobi sweep kernel: 1 register-tiled (two sites per thread,
 *                   the next plane prefetched in registers); 2 staged in shared
 *                   memory by the tensor memory accelerator (a producer thread
 *                   keeps three planes of boxes in flight; Landau links of either
 *                   plane, with or without insulating sites, even nx, else the
 *                   register-tiled kernel runs); 0 the default, which is 2.  With 2,
 *                   the init + first sweep is staged too (16-byte asynchronous
 *                   copies of psi, mu, alpha and the previous mu; yz links without
 *                   insulating sites and nx % 4 == 0, else register-tiled).  The
 *                   kernels do the same arithmetic in the same order (the staged
 *                   sweep's 1 / |diag M|^2 is the hardware reciprocal, about one
 *                   ulp from the correctly rounded one).
 *   poisson_guess   starting guess of each Poisson solve: 1 the previous step's mu;
 *                   2 its linear extrapolation in time, 2 mu^(n-1) - mu^(n-2) (the
 *                   previous mu on the first step after creation or a state load);
 *                   0 the default, which is 2.  With insulating sites, and
 *                   for tdgl_solve_mu called on its own (not after the psi solve of
 *                   a step), the guess is the current mu.  The solution the solve
 *                   converges to does not depend on it; with a fixed number of
 *                   V-cycles the extrapolated guess leaves a smaller error (one cycle
 *                   from it about as small as two from the previous mu on flux flow).
 *   d_insulating    device u8[N] or NULL: nonzero marks an insulating site
 *                   (Sec. 3.4 (ii), e.g. the mask of tdgl_pattern_ex).  Every link
 *                   that touches an insulating site carries no current: it leaves
 *                   the psi stencil and its diagonal, J_av, the energy, and the
 *                   Poisson operator and right-hand side; insulating sites hold
 *                   psi = mu = 0 and take no injected current.  Read once by
 *                   tdgl_create.  Needs Landau links (either plane) and even nx;
 *                   unless freeze_mu_K, the conducting sites must form one
 *                   connected domain (and, with current injected through open x
 *                   faces, touch both faces), else TDGL_ERR_INVALID_ARG.  The
 *                   Poisson solve is then conjugate gradients preconditioned by
 *                   V-cycles: poisson_cycles iterations, or with poisson_tol > 0
 *                   until the relative residual is below it.  Not for batches, the
 *                   adjoint or two sweeps per pass.
 *   d_alpha         device f32[N], eps(r) of Eq. epsilon (caller-owned, read-only
 *                   for the handle's lifetime).
 *   d_link_phase    device f32[3N] link phases theta_{a,m} of the link from m to
 *                   m+a (general mode only; NULL otherwise).  The x links are
 *                   further multiplied by exp(i hx K).
 */
typedef struct tdgl_config {
    int32_t nx, ny, nz;
    int32_t bc[3];
    double hx, hy, hz;
    double g, u, beta, ht;
    double By, Bz;
    double Jext;
    double eps;
    int32_t max_iter;
    int32_t check_every;
    int32_t fixed_sweeps;
    int32_t freeze_mu_K;
    int32_t poisson_cycles;
    int32_t poisson_max_cycles;
    double poisson_tol;
    int32_t links_mode;
    int32_t sweeps_per_pass;
    double noise_T;
    uint64_t noise_seed;
    double Bx;
    const float *d_alpha;
    const float *d_link_phase;
    const uint8_t *d_insulating;
    int32_t sweep_kernel;
    int32_t poisson_guess;
} tdgl_config;

typedef struct tdgl_handle tdgl_handle;

/* Observables (Sec. 2.1 Eq. J, Sec. 3.1.1 J_av, Sec. 2.2 K and E_x).  energy is the
 * discrete GL free energy with trapezoid face weights; vortices come from the
 * winding of xy plaquettes (arg of psi*_a U_ab psi_b summed with the plaquette
 * flux hx hy Bz).  FP64 accumulations. */
typedef struct tdgl_obs {
    double psi2_mean;        /* (1/N) sum |psi|^2                                     */
    double energy;           /* free energy                                            */
    double javg;             /* J_av of the last step (periodic x), else 0             */
    double K;                /* current K                                              */
    double Ex;               /* electric field of the last step                        */
    double vortex_unsigned;  /* sum_p |n_p| per z layer, averaged over layers          */
    double vortex_signed;    /* sum_p n_p per z layer, averaged over layers            */
    double last_r2;          /* max |r|^2 at the last convergence test                 */
    double poisson_res;      /* max|F - Lap mu| / max|F| after the last Poisson solve  */
                             /* (0 before the first solve; with a fixed number of     */
                             /* V-cycles measured when the observables are computed)  */
    int32_t last_sweeps;     /* Jacobi sweeps of the last step                         */
    int32_t poisson_cycles;  /* V-cycles of the last step                              */
    int64_t step;            /* completed time steps                                   */
} tdgl_obs;

/* Device pointers into the handle's workspace, where the current state lies: the
 * arrays rotate among buffers, so fetch them again after each step. */
typedef struct tdgl_state_ptrs {
    float *psi;   /* complex64[N], current psi^n                  */
    float *mu;    /* f32[N], current mu^n                         */
    float *b;     /* complex64[N], b of the last step (Eq. b)     */
    float *D;     /* complex64[N], diag M of the last step        */
    float *f;     /* f32[N], Poisson right-hand side, last step   */
} tdgl_state_ptrs;

/* Per-phase device time (CUDA events on the handle's stream, summed over steps
 * since tdgl_profile_enable) and host-side launch counters.  ms_sweeps covers
 * only the batches of Jacobi sweeps (host gaps between batches excluded);
 * launches that found the solve already converged return immediately and are
 * counted in sweep_launches but not in sweeps. */
typedef struct tdgl_profile {
    double ms_init;          /* fused init + first sweep                        */
    double ms_sweeps;        /* Jacobi sweeps 2..n                              */
    double ms_K;             /* J_av and the K ODE                              */
    double ms_poisson;       /* right-hand side, V-cycles, projection, voltage  */
    int64_t steps;           /* time steps                                      */
    int64_t sweeps;          /* Jacobi sweeps that did work, all steps          */
    int64_t sweep_launches;  /* sweep kernels launched (after the init sweep)   */
    int64_t kernel_launches; /* every kernel launch of the library              */
    int64_t vcycles;         /* multigrid V-cycles                              */
} tdgl_profile;

const char *tdgl_error_string(int code);

/* sizeof of the ABI structs, so that a binding can check its own layout:
 * which = 0 tdgl_config, 1 tdgl_obs, 2 tdgl_state_ptrs, 3 tdgl_profile,
 * 4 tdgl_adjoint_config, 5 tdgl_adjoint_stats, 6 tdgl_batch_tuning,
 * 7 tdgl_batch_stats, 8 tdgl_batch_tune_report, 9 tdgl_shape, 10 tdgl_lattice,
 * 11 tdgl_background; 0 for any other value.
 * Host only, needs no device. */
size_t tdgl_abi_struct_size(int32_t which);

/* Bytes of device workspace tdgl_create() needs for cfg (0 if cfg is invalid). */
size_t tdgl_workspace_bytes(const tdgl_config *cfg);

/* Validate cfg, carve the workspace (d_workspace must be 256-byte aligned and
 * ws_bytes >= tdgl_workspace_bytes(cfg)), build link tables on the device and
 * set psi = 0, mu = 0, K = 0.  Synchronises the stream before returning. */
int tdgl_create(const tdgl_config *cfg, void *d_workspace, size_t ws_bytes, void *stream, tdgl_handle **out);

void tdgl_destroy(tdgl_handle *h);

/* Copy a state in from DEVICE arrays (psi complex64[N], mu f32[N] or NULL = 0). */
int tdgl_set_state(tdgl_handle *h, const float *d_psi, const float *d_mu, double K);

/* Copy a state in from / out to HOST arrays (pinned or pageable). */
int tdgl_upload_state(tdgl_handle *h, const float *host_psi, const float *host_mu, double K);
int tdgl_download_state(tdgl_handle *h, float *host_psi, float *host_mu, double *K);

int tdgl_get_state(tdgl_handle *h, tdgl_state_ptrs *out);

/* Set the step index: the count of completed steps that tdgl_obs.step reports, and
 * the counter n of the thermal noise (Philox4x32-10 counter (site, n), Sec. 3.1.2)
 * that the next step draws with.  A state load (tdgl_set_state, tdgl_upload_state)
 * restarts the noise counter at 0.  Synchronises. */
int tdgl_set_step(tdgl_handle *h, int64_t step);

/* The previous step's mu (f32[N]), which the extrapolated Poisson guess of the next
 * step reads (tdgl_config.poisson_guess).  tdgl_get_mu_prev copies it to out (host
 * memory if out_on_host, else device memory) and returns 1, or returns 0 when the
 * handle holds none (after creation or a state load, or without the extrapolated
 * guess).  tdgl_set_mu_prev copies one in (NULL: none); it is refused without the
 * extrapolated guess.  A state load clears it, so load the state first.  (Single
 * handles only: a batch member keeps its previous mu inside the batch, and a state
 * load clears it.)
 *
 * Checkpoints: psi, mu and K (tdgl_download_state), the previous mu and the step
 * index, restored by a state load, tdgl_set_mu_prev and tdgl_set_step, continue the
 * run exactly as if it had not been interrupted, noise included.  Both synchronise. */
int tdgl_get_mu_prev(tdgl_handle *h, float *out, int32_t out_on_host);
int tdgl_set_mu_prev(tdgl_handle *h, const float *in, int32_t in_on_host);

/* Advance n_steps full time steps (psi, K, mu).  Synchronises once per step to
 * read the convergence status; returns the first error met. */
int tdgl_step(tdgl_handle *h, int n_steps);

/* Advance n_steps full time steps like tdgl_step, as ONE CUDA graph launch with a
 * single synchronisation at the end (the kernel loop of Sec. 4.1 kept on the
 * device).  A WHILE conditional node runs the steps; in each, IF nodes select the
 * launch sequence of the state's psi and mu buffers, a nested WHILE node repeats
 * two Jacobi sweeps until the sweep kernels' own convergence test (Eq. 11) has
 * decided, and IF nodes select the Poisson solve of the buffer holding the result.
 * Same kernels and arguments as tdgl_step, so the same results bit for bit.
 *   The graph is built on the first call (tens of milliseconds) and kept with the
 * handle; where the driver cannot build it, the steps run as tdgl_step.  The first step after creation or a state load (with the extrapolated
 * Poisson guess: until a previous mu exists) runs launch by launch, as tdgl_step.
 *   Returns TDGL_ERR_INVALID_ARG for handles the loop does not cover: insulating
 * sites, poisson_tol > 0, fixed_sweeps > 0, two sweeps per pass, batch members,
 * slabs and Poisson-only handles.  A step whose Jacobi solve fails (not converged
 * within max_iter, non-finite, a wait that timed out) stops the loop with the state
 * of the step before it and the error returned; the steps before it count. */
int tdgl_step_resident(tdgl_handle *h, int32_t n_steps);

/* The same steps as tdgl_step_resident, enqueued on the handle's stream without waiting
 * for them: the call returns once the graph is launched (after the launch-by-launch first
 * step, where one is due).  Steps enqueued while others are pending continue from their
 * device state; a failure halts every step enqueued after it.  tdgl_sync waits for the
 * enqueued steps and returns their status (the first error met; the state is then that of
 * the last good step).  Every other call on the handle first does the same, and returns
 * that error in place of its own work when the enqueued steps failed.  Handles the
 * resident loop does not cover: TDGL_ERR_INVALID_ARG. */
int tdgl_step_enqueue(tdgl_handle *h, int32_t n_steps);
int tdgl_sync(tdgl_handle *h);

/* Choose the Jacobi sweep of this handle by timing (Sec. 3.1; the two-sweep pass is
 * temporal blocking, not in the paper): the staged sweep (sweep_kernel 2), the
 * register-tiled one (1), and two sweeps per pass (sweeps_per_pass 2), as far as the
 * grid supports each.  Every candidate takes one warm-up step and trial_steps timed
 * steps from the current state; the state (psi, mu, the previous mu, K, the step and
 * noise counters, the profile counters) is restored before every trial and at the end,
 * so the run continues as if the call had not been made, with the fastest candidate.
 * Host memory holds the saved state (12 N + 4 N bytes); the device gets no allocation.
 * ms[c]: ms per step of candidate c (0 staged, 1 register-tiled, 2 two sweeps per pass;
 * 0 where not supported); chosen: the one kept.  Synchronises.  Handles the step does
 * not cover (batch members, slabs, Poisson-only): TDGL_ERR_INVALID_ARG. */
typedef struct tdgl_tune_report {
    double ms[3];
    int32_t chosen;
    int32_t candidates;
} tdgl_tune_report;
int tdgl_autotune(tdgl_handle *h, int32_t trial_steps, tdgl_tune_report *report);

/* Only the implicit psi solve of one step (init, Jacobi sweeps, residual
 * reductions), without the K and mu updates; *sweeps_out may be NULL. */
int tdgl_solve_psi(tdgl_handle *h, int32_t *sweeps_out);

/* Only the Poisson solve for the current psi and K (right-hand side, V-cycles,
 * zero-mode projection). */
int tdgl_solve_mu(tdgl_handle *h);

/* Start (on != 0) or stop collecting tdgl_profile data; enabling resets it. */
int tdgl_profile_enable(tdgl_handle *h, int on);
int tdgl_profile_read(tdgl_handle *h, tdgl_profile *out);

/* Test hook for the bounded waits of the staged kernels (the Jacobi sweep and the
 * Poisson right-hand side staged by the tensor memory accelerator, and the staged
 * line smoother).  Each of their mbarrier waits ends after wait_ns nanoseconds
 * (0: the default of 2 s; at most 2 s); extra_tx_bytes (0 .. 65536) is added to the
 * bytes that the stages of the first block of each staged sweep or right-hand-side
 * launch, and the boxes of the first warp of each staged smoother launch, expect.
 * With a value > 0 those stages never complete and their waits run out while the
 * rest of the launch completes -- no copy faults, the copies land and are waited
 * for as in a real timeout.  The waits that run out record TDGL_ERR_TIMEOUT, which
 * the step reports.  (0, 0), the state at creation, is normal use.  Synchronises the stream
 * and drops the handle's captured Poisson graphs (captured again on the next solve).
 *
 * After TDGL_ERR_TIMEOUT, from this hook or from a copy that never landed, the
 * handle's psi, mu and K stay at the last completed step and every later step
 * reports TDGL_ERR_TIMEOUT again; tdgl_observables still works.  Loading a state
 * (tdgl_set_state or tdgl_upload_state) clears the error and the handle steps
 * normally again. */
int tdgl_test_staged_waits(tdgl_handle *h, int64_t wait_ns, int32_t extra_tx_bytes);

/* Compute observables of the current state (synchronises). */
int tdgl_observables(tdgl_handle *h, tdgl_obs *out);

/*
 * z-slab decomposition (a grid split along z over several GPUs or processes; the
 * paper names multi-GPU runs as future work, Sec. 5).  A slab handle holds the
 * planes z0 .. z0 + nz_local - 1 of a grid described by global_cfg, between two halo
 * planes: its arrays (psi, mu, alpha, f, as for tdgl_create) have nz_local + 2
 * planes, plane 1 being global plane z0; the halo planes hold copies of the
 * neighbouring slabs' edge planes, which the caller keeps current.  global_cfg must
 * be periodic in z, open in x, with Landau links, even nx, no insulating sites, no
 * thermal noise, one sweep per pass, check_every 1 and no fixed sweep count;
 * global_cfg->d_alpha points at the slab's alpha with its halo planes (f32 of
 * nx ny (nz_local + 2); the halo planes are not read).
 *
 * A step, driven by the caller over all slabs (Sec. 3.1 and 3.2 in the paper's order):
 *   1. the halo planes of the state psi (tdgl_slab_planes, latest = 0) are exchanged;
 *   2. tdgl_slab_sweep(first = 1) forms b and diag M (Eq. b) and runs the first
 *      Jacobi sweep (Eq. final); *r2_local is max |b - M psi|^2 of the sweep's input
 *      over the slab's own planes;
 *   3. the caller takes the maximum of r2_local over all slabs; if it is below eps
 *      (Eq. convergence) the output of that sweep is the result, else the halos of
 *      the latest iterate (latest = 1) are exchanged and tdgl_slab_sweep(first = 0)
 *      runs the next sweep (up to max_iter);
 *   4. tdgl_slab_accept makes the result the state, whose halos are exchanged again;
 *   5. tdgl_slab_rhs writes the Poisson right-hand side of the slab's planes into f
 *      (tdgl_get_state: f, planes 1 .. nz_local);
 *   6. the caller solves the potential of the whole grid's f (for instance on a
 *      Poisson-only handle, below) and writes the slab's part into the slab's mu
 *      (planes 1 .. nz_local), where the next init reads it.
 * tdgl_slab_planes: planes[0], planes[1] = the slab's first and last plane (to send
 * down and up), planes[2], planes[3] = the halo planes below and above (to receive),
 * device pointers to complex64[nx ny] of the state (latest = 0) or of the latest
 * iterate (latest = 1).  tdgl_slab_sweep synchronises; it returns the step's
 * TDGL_ERR_NONFINITE like tdgl_step.  tdgl_step, tdgl_solve_psi, tdgl_solve_mu and
 * tdgl_observables refuse slab handles.
 */
size_t tdgl_slab_workspace_bytes(const tdgl_config *global_cfg, int32_t z0, int32_t nz_local);
int tdgl_slab_create(const tdgl_config *global_cfg, int32_t z0, int32_t nz_local, void *d_workspace, size_t ws_bytes,
                     void *stream, tdgl_handle **out);
int tdgl_slab_sweep(tdgl_handle *h, int32_t first, double *r2_local);
int tdgl_slab_accept(tdgl_handle *h);
int tdgl_slab_planes(tdgl_handle *h, int32_t latest, float **planes);
int tdgl_slab_rhs(tdgl_handle *h);

/*
 * Poisson-only handle: the multigrid Poisson solve of Sec. 3.2 (the operator, the
 * boundary conditions of cfg and the zero-mode projection of tdgl_step) for a
 * right-hand side the caller writes into the handle's f (tdgl_get_state: f; mu is
 * the result, psi NULL).  No psi arrays are allocated and cfg->d_alpha may be NULL;
 * Landau links, no insulating sites.  tdgl_solve_mu_f runs poisson_cycles V-cycles
 * (or to poisson_tol) from the starting guess of poisson_guess (the extrapolation
 * of the last two solutions of this handle), projects out the weighted mean and,
 * with open x, computes E_x from the face potentials; it works on single handles
 * too (after a step: the f of that step).  tdgl_read_ctl_scalars returns E_x and the
 * relative residual max|F - Lap mu| / max|F| of the last solve (synchronises).
 */
size_t tdgl_poisson_workspace_bytes(const tdgl_config *cfg);
int tdgl_poisson_create(const tdgl_config *cfg, void *d_workspace, size_t ws_bytes, void *stream, tdgl_handle **out);
int tdgl_solve_mu_f(tdgl_handle *h);
int tdgl_read_ctl_scalars(tdgl_handle *h, double *Ex, double *poisson_res);

/*
 * Inclusion pattern generator (Sec. 3.4), standalone.  Candidates (host array,
 * 10 doubles each: centre cx cy cz, semi-axes a b c, unit quaternion q0..q3 of
 * the body rotation) are consumed in order; a site r = (i hx, j hy, k hz) lies
 * inside candidate n when d^T R diag(a^-2) R^T d <= 1, d = r - c with the
 * minimum-image convention on periodic axes, evaluated in FP64.  A site belongs
 * to the first candidate containing it; candidates are added until at least
 * target_sites sites are inside (target_sites <= 0: all candidates).
 * d_alpha[m] = alpha_in inside, alpha_out elsewhere.  Only nx..nz, bc and h of
 * grid are read.  d_scratch: device bytes >= tdgl_pattern_scratch_bytes().
 * Synchronises; *n_used and *n_marked (may be NULL) receive the counts.
 */
size_t tdgl_pattern_scratch_bytes(const tdgl_config *grid, int64_t n_candidates);
int tdgl_pattern(const tdgl_config *grid, const double *host_candidates, int64_t n_candidates,
                 int64_t target_sites, float alpha_in, float alpha_out, float *d_alpha,
                 void *d_scratch, size_t scratch_bytes, void *stream, int64_t *n_used, int64_t *n_marked);

/*
 * Pattern generator, full form (Sec. 3.4): pinning landscapes from shapes,
 * lattices of a shape, shapes that claim their outside (a shaped integration
 * domain) and tessellated backgrounds.
 *
 * Shapes.  A site r = (i hx, j hy, k hz) is tested in the body frame of the
 * shape: d = r - c with the minimum image on periodic axes, e_a = sum_r R_ra d_r,
 * R the rotation of the unit quaternion q (body -> lab).  All in FP64 with each
 * product and sum rounded separately, so the decision at every site is
 * reproducible.  A shape with TDGL_SHAPE_INVERT claims the sites it does not
 * contain.  A site takes the value of the first shape (list order) that claims
 * it.  Shapes are taken in order while fewer than target_sites sites are
 * claimed (target_sites <= 0: all).  TDGL_SHAPE_INSULATING marks the claimed
 * sites in d_insulating (the insulating inclusions of Sec. 3.4 (ii)).
 */
#define TDGL_SHAPE_ELLIPSOID 0   /* sum_a (e_a / a_a)^2 <= 1: spheres, ellipsoids, circles on a film   */
#define TDGL_SHAPE_CUBOID 1      /* |e_a| <= a_a: cuboids, rectangles on a film                     */
#define TDGL_SHAPE_CYLINDER 2    /* (e_x/a_x)^2 + (e_y/a_y)^2 <= 1 and |e_z| <= a_z (axis body z)     */
#define TDGL_SHAPE_CROSS 3       /* bar (a_x, a_y, a_z) united with bar (a_y, a_x, a_z)              */
#define TDGL_SHAPE_OCTANT 4      /* ellipsoid restricted to e_x, e_y, e_z >= 0                        */
#define TDGL_SHAPE_INVERT 1      /* flags: claims the outside                                         */
#define TDGL_SHAPE_INSULATING 2  /* flags: claimed sites are insulating                               */

typedef struct tdgl_shape {
    int32_t kind;
    int32_t flags;
    double c[3];     /* centre, units of xi_0                                   */
    double a[3];     /* semi-axes / half-extents (> 0)                          */
    double q[4];     /* unit quaternion (w, x, y, z)                            */
    double value;    /* eps(r) of the claimed sites                             */
} tdgl_shape;

/*
 * Lattices of a motif shape, expanded on the device: point = origin + n1 a1 +
 * n2 a2 + n3 a3 + basis_b (0 <= n_i < count[i]), motif centred at point +
 * motif.c; shapes ordered n3, n2, n1, basis (fastest).  With spacing (a, b, c):
 *   SQUARE      a1 = (a,0,0), a2 = (0,a,0)
 *   TRIANGULAR  a1 = (a,0,0), a2 = (a/2, a sqrt(3)/2, 0)
 *   HONEYCOMB   triangular, basis {0, (a/2, a sqrt(3)/6, 0)}
 *   KAGOME      triangular, basis {0, a1/2, a2/2}
 *   RECTANGULAR a1 = (a,0,0), a2 = (0,b,0), a3 = (0,0,c)      (3-D)
 *   HEXAGONAL   triangular layers stacked with a3 = (0,0,c)     (3-D)
 * The 2-D kinds stack count[2] layers with a3 = (0,0,c) (count[2] = 1: one layer).
 */
#define TDGL_LATTICE_SQUARE 0
#define TDGL_LATTICE_TRIANGULAR 1
#define TDGL_LATTICE_HONEYCOMB 2
#define TDGL_LATTICE_KAGOME 3
#define TDGL_LATTICE_RECTANGULAR 4
#define TDGL_LATTICE_HEXAGONAL 5

typedef struct tdgl_lattice {
    int32_t kind;
    int32_t count[3];
    double origin[3];
    double spacing[3];
    tdgl_shape motif;
} tdgl_lattice;

/*
 * Background of the sites no shape claims.
 *   CONSTANT  value.
 *   CHECKER   cells of size cell[a] (<= 0: axis not divided), cell index
 *             c_a = floor(i_a h_a / cell[a]).  p_odd < 0: values[(c_x+c_y+c_z) & 1].
 *             p_odd in [0, 1]: random checkerboard, a cell takes values[1] when
 *             u < p_odd, u = (x0 >> 8) 2^-24 from Philox4x32-10 with counter
 *             (cell, 0, 0x4B434548) and key = seed, cell = c_x + n_x (c_y + n_y c_z),
 *             n_a = floor((N_a - 1) h_a / cell[a]) + 1; else values[0].
 *   VORONOI   the value of the nearest seed (host_seeds: n_seeds x (x, y, z, value))
 *             under the metric (Euclidean, absolute = sum |d_a|, maximum = max |d_a|),
 *             minimum image on periodic axes, equal distances to the lower seed index.
 */
#define TDGL_BG_CONSTANT 0
#define TDGL_BG_CHECKER 1
#define TDGL_BG_VORONOI 2
#define TDGL_METRIC_EUCLIDEAN 0
#define TDGL_METRIC_ABSOLUTE 1
#define TDGL_METRIC_MAXIMUM 2

typedef struct tdgl_background {
    int32_t kind;
    int32_t metric;
    double value;
    double cell[3];
    double values[2];
    double p_odd;
    uint64_t seed;
    const double *host_seeds;
    int64_t n_seeds;
} tdgl_background;

/* Scratch for tdgl_pattern_ex (0: invalid arguments).  bg may be NULL (constant 1). */
size_t tdgl_pattern_ex_scratch_bytes(const tdgl_config *grid, int64_t n_shapes, const tdgl_lattice *lattices,
                                     int32_t n_lattices, const tdgl_background *bg);
/* Shapes (host, n_shapes), then the shapes of each lattice (host, n_lattices) in order;
 * d_alpha f32[N] receives the pattern, d_insulating (u8[N], may be NULL) 1 where the
 * claiming shape is insulating.  Only nx..nz, bc and h of grid are read.  Synchronises;
 * *n_used (shapes taken) and *n_marked (claimed sites) may be NULL.
 * Errors: TDGL_ERR_INVALID_ARG (bad kind, non-positive size, quaternion not of unit
 * norm within 1e-6, more than 2^31 - 16 shapes, Voronoi without seeds),
 * TDGL_ERR_WORKSPACE (scratch too small or not 256-byte aligned). */
int tdgl_pattern_ex(const tdgl_config *grid, const tdgl_shape *shapes, int64_t n_shapes,
                    const tdgl_lattice *lattices, int32_t n_lattices, const tdgl_background *bg,
                    int64_t target_sites, float *d_alpha, uint8_t *d_insulating, void *d_scratch,
                    size_t scratch_bytes, void *stream, int64_t *n_used, int64_t *n_marked);

/*
 * Adjoint of the time loop: gradient of the time-averaged electric field with
 * respect to the pinning map alpha (inverse design of inclusions).  The paper
 * has no adjoint; this differentiates its discrete step (Sec. 3.1, Crank-
 * Nicolson residual R = psi' - psi + (ht/2) H (psi' + psi), H = diag(beta|psi|^2
 * + i u mu - alpha) - Lap_U; Sec. 3.2 Poisson solve), taking every linear solve
 * as exact.  Starting from the handle's current state, tdgl_adjoint runs
 * n_steps forward steps exactly as tdgl_step (the handle ends in the state
 * after them), storing (psi, mu) every checkpoint_every steps in d_ws; then,
 * segment by segment from the end, recomputes the segment's states from its
 * checkpoint and runs the reverse steps: adjoint Poisson, adjoint of the
 * right-hand side Im[psi* NS psi], adjoint implicit solve M^H lam = g by
 * Jacobi to a relative tolerance, and accumulation of dJ/dalpha.
 *   J = (1/(n_steps - window_start)) sum_{n > window_start} E_x^n
 * Requires open x (E_x from the face potentials), Landau links and even nx.
 * d_grad_alpha: device f32[N], overwritten.  *objective: J.  d_ws: device bytes
 * >= tdgl_adjoint_workspace_bytes(), 256-byte aligned, caller-owned.
 * Synchronises the stream once per step.
 */
typedef struct tdgl_adjoint_config {
    int32_t n_steps;           /* forward steps                                   */
    int32_t checkpoint_every;  /* steps between stored states (>= 1)              */
    int32_t window_start;      /* J averages E_x over steps window_start+1..n     */
    int32_t adj_max_iter;      /* sweep cap of each adjoint solve                 */
    double adj_eps;            /* adjoint Jacobi stops when max |r|^2 <= adj_eps  */
                               /* times max |r|^2 of its first sweep (relative)   */
    int32_t poisson_cycles;    /* V-cycles of each adjoint Poisson solve (>= 1)   */
    int32_t reserved;
    double poisson_tol;        /* > 0: more cycles until the relative residual    */
} tdgl_adjoint_config;         /*      is below it (up to poisson_max_cycles)     */

typedef struct tdgl_adjoint_stats {
    double ms_forward;         /* first forward pass (device time)                */
    double ms_recompute;       /* recomputed segments                             */
    double ms_reverse;         /* reverse steps                                   */
    int64_t adjoint_sweeps;    /* adjoint Jacobi sweeps, all steps                */
} tdgl_adjoint_stats;

size_t tdgl_adjoint_workspace_bytes(const tdgl_handle *h, const tdgl_adjoint_config *acfg);
int tdgl_adjoint(tdgl_handle *h, const tdgl_adjoint_config *acfg, void *d_ws, size_t ws_bytes, float *d_grad_alpha,
                 double *objective, tdgl_adjoint_stats *stats);

/*
 * Allocation-free Jacobi sweep.  The paper has no counterpart: this entry point
 * exists for callers that cannot call cudaMalloc -- code running inside a host
 * application whose memory manager owns the device heap, or a real-time loop
 * that must not allocate once it runs -- but that hold device buffers for their
 * inputs and outputs.  It performs one sweep of Eq. final, exactly as the sweeps
 * of tdgl_step do, with the Landau links of cfg and exp(i hx K) on x links:
 *   d_psi_out = D^{-1} (b - R psi_in),   *r2max = max_m |b - M psi_in|^2,
 * for complex64 arrays d_psi_in, d_b (Eq. b), d_D (diag M) and d_psi_out of
 * nx*ny*nz sites (d_psi_out must not alias d_psi_in).  Only nx..Bz of cfg are
 * read; d_alpha may be NULL; links_mode must be TDGL_LINKS_LANDAU.
 * Its scratch (control block, link tables, per-block maxima) is one static
 * device array of TDGL_NOALLOC_SCRATCH_BYTES bytes that every GPU loading the
 * library holds until exit; nothing is allocated.  Grids with an axis longer
 * than TDGL_NOALLOC_MAX_AXIS, or needing more than TDGL_NOALLOC_MAX_BLOCKS sweep
 * blocks, are rejected with TDGL_ERR_WORKSPACE.  The first call on a device
 * looks the array's address up (make it before any stream capture).  All calls
 * share the array, so calls that overlap on the GPU race; each call rewrites
 * what it uses before it runs.  Synchronises the stream.
 */
#define TDGL_NOALLOC_MAX_AXIS 4096
#define TDGL_NOALLOC_MAX_BLOCKS 65536
#define TDGL_NOALLOC_SCRATCH_BYTES (512 + 32 * TDGL_NOALLOC_MAX_AXIS + 8 * TDGL_NOALLOC_MAX_BLOCKS)
int tdgl_sweep_noalloc(const tdgl_config *cfg, const float *d_psi_in, const float *d_b, const float *d_D, double K,
                       float *d_psi_out, double *r2max, void *stream);

/*
 * Batched ensembles.  The paper steps one sample at a time; a batch advances up
 * to TDGL_BATCH_MAX independent instances (own grid size, boundary conditions,
 * field, current, time step, tolerance and alpha map) with one persistent,
 * cooperative kernel launch per time step.  That launch runs, for every
 * instance, the whole step of tdgl_step: init and Jacobi sweeps of the implicit
 * psi solve (Sec. 3.1, Eq. b, Eq. final) with the convergence test of each
 * instance applied after every sweep (Eq. convergence; an instance that has
 * converged stops while the others go on), J_av and the K ODE on periodic x
 * (Sec. 2.2), the Poisson right-hand side and poisson_cycles multigrid V-cycles
 * (Sec. 3.2), the zero-mode projection of mu and the open-x voltage.  Phases
 * are separated by a grid barrier whose waits end after timeout_ms; a timeout
 * sets a sticky error that tdgl_batch_status reports, and every later launch
 * returns at once.  Launches are replayed from a CUDA graph of graph_steps
 * steps.  Work items are (instance, tile) pairs, distributed over the
 * persistent blocks phase by phase.
 *
 * Requirements per instance: links_mode TDGL_LINKS_LANDAU, nx even, nx*ny*nz <
 * 2^31, poisson_tol == 0 (a fixed number of V-cycles), and a coarsest multigrid
 * level of at most 1024 y-z modes.  Violations return TDGL_ERR_INVALID_ARG.
 * The instances' handles (tdgl_batch_instance) serve tdgl_set_state,
 * tdgl_upload_state, tdgl_download_state, tdgl_get_state and tdgl_observables;
 * tdgl_step, tdgl_solve_psi, tdgl_solve_mu and tdgl_adjoint refuse them
 * (TDGL_ERR_INVALID_ARG).  After an instance fails (no convergence within
 * max_iter, or a non-finite residual) its state stays at its last good step
 * and later steps skip it.
 */
#define TDGL_BATCH_MAX 256

typedef struct tdgl_batch tdgl_batch;

typedef struct tdgl_batch_tuning {
    int32_t blocks_per_sm;        /* persistent blocks per SM (<= the occupancy limit; 0 = that limit) */
    int32_t graph_steps;          /* steps per CUDA graph replay (0: plain launches)                   */
    int32_t timeout_ms;           /* bound of every grid-barrier wait                                  */
    int32_t test_extra_arrivals;  /* 0.  > 0 makes every barrier wait for blocks that do not exist,    */
                                  /* so that the timeout path can be tested                            */
    int32_t sweep_kernel;         /* init, Jacobi sweep and Poisson right-hand-side tiles: 0 staged in */
                                  /* shared memory by asynchronous copies (default; the init where     */
                                  /* nx % 4 == 0), 1 register-tiled                                    */
    int32_t kz[TDGL_BATCH_MAX];   /* z planes per sweep tile, per instance (0: default rule)           */
} tdgl_batch_tuning;

typedef struct tdgl_batch_stats {
    int64_t steps;                /* batch steps enqueued since creation                               */
    int64_t sweeps;               /* Jacobi sweeps, summed over instances                              */
    double site_iters;            /* sum over instances of sites x sweeps                              */
    int32_t grid_blocks;          /* persistent blocks of the launch                                   */
    int32_t blocks_per_sm;
    int32_t graph;                /* 1: steps are replayed from a captured CUDA graph                  */
    int32_t smem_bytes;           /* dynamic shared memory per block                                   */
} tdgl_batch_stats;

typedef struct tdgl_batch_tune_report {
    double ms_default;            /* ms per step of the starting configuration                        */
    double ms_best;               /* ms per step of the chosen configuration                          */
    int32_t candidates;           /* configurations timed                                              */
    int32_t classes;              /* distinct instance grid sizes tuned separately                     */
} tdgl_batch_tune_report;

/* Device bytes for the instances' workspaces, the instance table and the batch
 * scratch (0 if any cfg is invalid for a batch). */
size_t tdgl_batch_workspace_bytes(const tdgl_config *cfgs, int32_t n);
/* Create n instances in d_workspace (256-byte aligned); states start at psi = 0,
 * mu = 0, K = 0.  Synchronises the stream. */
int tdgl_batch_create(const tdgl_config *cfgs, int32_t n, void *d_workspace, size_t ws_bytes, void *stream,
                      tdgl_batch **out);
void tdgl_batch_destroy(tdgl_batch *b);
int tdgl_batch_instance(tdgl_batch *b, int32_t i, tdgl_handle **out);
/* Enqueue n_steps batch steps on the stream (asynchronous). */
int tdgl_batch_step(tdgl_batch *b, int32_t n_steps);
/* Synchronise; status[i] (may be NULL) = 0 or the error that stopped instance i.
 * Returns TDGL_ERR_TIMEOUT after a barrier timeout, else the first nonzero
 * instance status, else TDGL_OK. */
int tdgl_batch_status(tdgl_batch *b, int32_t *status);
/* Synchronise and compute every instance's observables into out[n]. */
int tdgl_batch_observables(tdgl_batch *b, tdgl_obs *out);
/* Synchronise; sweeps (may be NULL) receives each instance's cumulative sweeps. */
int tdgl_batch_stats_read(tdgl_batch *b, tdgl_batch_stats *out, int64_t *sweeps);
int tdgl_batch_get_tuning(tdgl_batch *b, tdgl_batch_tuning *out);
int tdgl_batch_set_tuning(tdgl_batch *b, const tdgl_batch_tuning *in);
/* Phase log: with logging on, every launch records when each of its phases ended
 * (device globaltimer, read by one thread after the phase's grid barrier).
 * tdgl_batch_phase_read sums the last launch's phase durations by kind into
 * ms_by_op[TDGL_BATCH_OPS] and counts the phases into phases_by_op; the kinds are
 * 0 init + first sweep, 1 Jacobi sweep, 2 J_av and K, 3 Poisson right-hand side,
 * 4 line smoothing, 5 residual (no phase: formed inside the restriction), 6 restriction
 * with the residual, 7-9 coarsest-level transform,
 * line solve and inverse transform, 10 prolongation, 11 zero mode and voltage,
 * 12 projection.  Synchronises. */
#define TDGL_BATCH_OPS 13
int tdgl_batch_phase_log(tdgl_batch *b, int32_t on);
int tdgl_batch_phase_read(tdgl_batch *b, double *ms_by_op, int32_t *phases_by_op, int32_t nops);
/* The last launch's phases one by one, in order: ms[i] and ops[i] (the kinds above) for
 * the first cap of them; *n_out = the number of phases.  Synchronises. */
int tdgl_batch_phase_list(tdgl_batch *b, double *ms, int32_t *ops, int32_t cap, int32_t *n_out);

/* Time trial_steps steps (after one warm-up step) for each candidate launch
 * shape, sweep tile kind (staged or register-tiled) and per-size-class sweep
 * tile depth, restoring the states before every
 * trial and at the end; keeps the fastest.  The states are left unchanged. */
int tdgl_batch_autotune(tdgl_batch *b, int32_t trial_steps, tdgl_batch_tune_report *report);

#ifdef __cplusplus
}
#endif

#endif /* TDGL_H */
