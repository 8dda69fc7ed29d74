// Internal declarations shared by the CUDA translation units of the solver.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/tdgl.h"

namespace tdgl {

constexpr int kPeriodic = TDGL_PERIODIC;
constexpr int kOpen = TDGL_OPEN;
constexpr int kMaxLevels = 16;

// Grid and coefficients as the kernels see them (passed by value).
struct DevGrid {
    int nx, ny, nz;
    long long N;
    int bcx, bcy, bcz;
    float cx, cy, cz;          // 1/hx^2, 1/hy^2, 1/(g^2 hz^2); 0 on an inactive axis
    float S;                   // cx + cy + cz
    float ht2, u, beta;        // ht/2, u, beta
    const float2 *Uy;          // [nx] y links exp(-i hy Bz xbar_i)
    const float2 *Uz;          // [nx] z links exp(+i hz By xbar_i)
    const float2 *Py;          // [ny] periodic-x wrap phase, y part
    const float2 *Pz;          // [nz] periodic-x wrap phase, z part
    const float2 *L;           // [3N] general links, or nullptr (Landau)
    // xz-plane gauge (Eq. A_xz), nullptr otherwise; L then holds the same links as a 3N table
    const float2 *Xj;          // [ny] x links exp(i hx Bz ybar_j) (times exp(i hx K))
    const float2 *Zj;          // [ny] z links exp(-i hz Bx ybar_j)
    const float2 *Wx;          // [nx] periodic-y wrap link, x part exp(-i i hx Ly Bz)
    const float2 *Wz;          // [nz] periodic-y wrap link, z part exp(+i k hz Ly Bx)
    const uint8_t *lk;         // [N] link bits (insulating inclusions), or nullptr: every link present
    // z window: the planes kw0 .. kw1-1 are updated and reduced over (kw1 = 0: all planes).
    // A z-slab of a larger grid holds its planes between two halo planes (window 1 .. nz-2)
    // whose values come from the neighbouring slabs.
    int kw0, kw1;
};
__host__ __device__ __forceinline__ int zlo(const DevGrid &g) { return g.kw1 ? g.kw0 : 0; }
__host__ __device__ __forceinline__ int zhi(const DevGrid &g) { return g.kw1 ? g.kw1 : g.nz; }

// Link bits of a site (insulating inclusions, Sec. 3.4 (ii)): the link to the +x,
// -x, +y, -y, +z, -z neighbour exists and joins two conducting sites; kLkIns: the
// site itself is insulating (psi = mu = 0, no links).
constexpr unsigned kLkXp = 1u, kLkXm = 2u, kLkYp = 4u, kLkYm = 8u, kLkZp = 16u, kLkZm = 32u, kLkIns = 64u;

// Device-resident control block.  Written only by single threads at the end of
// kernels (last-block reductions), read by later launches on the same stream.
struct DevCtl {
    double K;                  // current K
    double r2ref;              // max |r|^2 of the first sweep (relative tolerance)
    double Ex;                 // electric field of the last step
    double javg;               // J_av of the last step
    double r2;                 // max |r|^2 of the last tested sweep
    double fmean;              // weighted mean of the Poisson right-hand side
    double fmax;               // max |F| (after projection)
    double res;                // last Poisson residual max-norm
    double wsum;               // sum of trapezoid weights
    double mu_mean;            // weighted mean of mu before projection
    double sums[8];            // scratch results of observable reductions
    float2 Ux;                 // exp(i hx K), from K in FP64
    int iter;                  // sweeps done in this step
    int done;                  // 1: this step's Jacobi solve finished
    int status;                // TDGL_OK or error
    int result;                // buffer index holding the solve's result
    unsigned int ticket;       // last-block ticket (reset by the last block)
    int redo;                  // 1: the result is the first sweep of the last two-sweep pass (recompute it)
    int mu_prev_ok;            // batch member: the solve buffer holds the previous step's mu
    int pad1;
    unsigned long long nstep;  // time steps initialised since creation or the last state load (noise counter)
    unsigned long long pad2;
    // weighted mean not yet subtracted from each mu buffer: the state mu is mu_buf[q] -
    // mu_off[q] (the zero-mode projection of a fixed-cycle solve is applied where mu is
    // read, or when the state is handed out)
    double mu_off[2];
    // the device-resident step loop (tdgl_step_resident)
    int rcur, rq;              // psi buffer and mu buffer of the state
    int rleft, rdone;          // steps still to run; steps run (their solves succeeded)
    int rspare, rlast;         // (unused); sweeps of the last step run
    int rok;                   // 1: this step's Jacobi solve succeeded (its tail runs)
    int rhalt;                 // 1: a failure stopped the enqueued steps (later ones do nothing)
    long long rsweeps;         // sweeps of the steps run
    long long rloops;          // two-sweep loop iterations of all steps entered
    // batch member: sum of w mu and the x-face difference of mu (open x), accumulated by the
    // finest level's last two smoothing passes (cleared when the right-hand side is formed)
    double bmean[2];
};

// ----------------------------------------------------------------------------
// complex64 helpers
// ----------------------------------------------------------------------------
__host__ __device__ __forceinline__ float2 cmk(float x, float y) { return make_float2(x, y); }
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 cscale(float s, float2 a) { return make_float2(s * a.x, s * a.y); }
__host__ __device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
__host__ __device__ __forceinline__ float2 cmulc(float2 a, float2 b)
{
    return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ __forceinline__ float cabs2(float2 a) { return a.x * a.x + a.y * a.y; }
// acc += a * b
__host__ __device__ __forceinline__ void cfma(float2 &acc, float2 a, float2 b)
{
    acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
    acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
}
// acc += conj(a) * b
__host__ __device__ __forceinline__ void cfmac(float2 &acc, float2 a, float2 b)
{
    acc.x = fmaf(a.x, b.x, fmaf(a.y, b.y, acc.x));
    acc.y = fmaf(a.x, b.y, fmaf(-a.y, b.x, acc.y));
}

// ----------------------------------------------------------------------------
// reductions
// ----------------------------------------------------------------------------
__device__ __forceinline__ float warp_max(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sumf(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide max of a float (all threads get the result).  sh: >= 32 floats.
__device__ __forceinline__ float block_max(float v, float *sh)
{
    int lane = threadIdx.x & 31;
    int wid = (threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z)) >> 5;
    int nthreads = blockDim.x * blockDim.y * blockDim.z;
    int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    lane = tid & 31;
    v = warp_max(v);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    int nw = (nthreads + 31) >> 5;
    float r = (tid < nw) ? sh[tid] : 0.0f;
    if (wid == 0) r = warp_max(r);
    if (tid == 0) sh[0] = r;
    __syncthreads();
    r = sh[0];
    return r;
}

// Block-wide FP64 sum (result valid in thread 0).  sh: >= 32 doubles.
__device__ __forceinline__ double block_sum(double v, double *sh)
{
    int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    int nthreads = blockDim.x * blockDim.y * blockDim.z;
    int lane = tid & 31, wid = tid >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    int nw = (nthreads + 31) >> 5;
    double r = (tid < nw) ? sh[tid] : 0.0;
    if (wid == 0) r = warp_sum(r);
    return r;
}

// Load through L2 only (CG) or a plain dereference that the compiler may turn
// into a read-only-path load.  A persistent kernel reads data that other blocks
// wrote earlier in the same launch, so it uses the L2 form (L2 is the point of
// coherence; the non-coherent read-only path has no such guarantee).  Measured
// on the batched step, L1-cached loads were not faster.
template <bool CG, class T>
__device__ __forceinline__ T ldx(const T *p)
{
    if constexpr (CG) return __ldcg(p);
    else return *p;
}

// Last-block ticket: returns true in every thread of the block that finishes
// last.  The caller has already written its per-block partial.
__device__ __forceinline__ bool last_block(unsigned int *ticket, unsigned int nblocks, int *sh_flag)
{
    int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        unsigned int t = atomicAdd(ticket, 1u);
        *sh_flag = (t == nblocks - 1u);
    }
    __syncthreads();
    bool last = *sh_flag != 0;
    if (last) __threadfence();
    return last;
}

// ----------------------------------------------------------------------------
// host-side launchers (defined in the .cu files)
// ----------------------------------------------------------------------------
struct SweepArgs {
    DevGrid g;
    DevCtl *ctl;
    double *blockred;          // per-block partials
    const float2 *src;         // input iterate (init: psi^-)
    float2 *dst;               // output iterate
    float2 *b;
    float2 *D;
    const float *mu;           // init only
    const float *alpha;        // init only
    int dst_index;             // buffer index of dst
    int check_every;
    int fixed_sweeps;
    int max_iter;
    double eps;
    int rel_eps;               // 1: converge when max|r|^2 <= eps * (max|r|^2 of the first sweep)
    float *f;                  // Poisson right-hand side (right-hand-side mode)
    float inj;                 // 2 J / hx at open x faces (right-hand-side mode)
    double wsum;               // sum of trapezoid weights (right-hand-side mode)
    float noise_amp;           // h_t zeta_max (init mode; 0: no noise)
    unsigned long long noise_seed;
    // staged (tensor-map) kernels: bound of each mbarrier wait in ns (0: the kernel's
    // default) and bytes added to each stage's expected transaction count (0 in normal
    // use; > 0 makes every wait run out, for the timeout test)
    unsigned long long wait_ns;
    unsigned int extra_tx;
    // init only: starting guess of the coming Poisson solve, written in place over the
    // previous-but-one mu: mu_guess = ex_a mu + ex_b mu_guess (nullptr: none)
    float *mu_guess;
    float ex_a, ex_b;
    // 1: write the guess on the rows of zebra colour 1 ((j + k) odd) only: the first pass
    // of the coming V-cycle solves the colour-0 lines from their colour-1 neighbours and
    // never reads colour-0 values (a proper colouring and a smoothed finest level)
    int guess_odd_only;
    // init only: the pending mean of mu and of the previous-but-one mu (nullptr: none)
    const double *mu_off, *mu_off_prev;
    // device-resident step loop (has_loop 1): the condition of the WHILE graph node that
    // repeats the sweeps, set by the block that decides a sweep (1 while the solve goes on)
    // and by a sweep that finds the solve already decided (0); and, when the decision ends
    // the solve, the value of the SWITCH node of the step's tail: tail_base + the result's
    // buffer after a successful solve, else kNoBranch
    cudaGraphConditionalHandle loop_cond, tail_cond;
    int has_loop, tail_base;
};
constexpr unsigned int kNoBranch = 6;

// staged: the tile staged in shared memory where init_staged_supported (else register-tiled)
cudaError_t launch_init_sweep(const SweepArgs &a, cudaStream_t s, bool staged = false);
bool init_staged_supported(const DevGrid &g);
cudaError_t init_staged_setup();   // the staged init's shared-memory attribute (set once per process)
// the guess of launch_init_sweep on its own: P = a S + b P over N sites
cudaError_t launch_mu_guess(long long N, const float *S, float *P, float a, float b, const double *offS,
                            const double *offP, cudaStream_t s);
cudaError_t launch_sweep(const SweepArgs &a, cudaStream_t s);
// one sweep src -> dst that neither tests nor touches the control block
cudaError_t launch_sweep_redo(const SweepArgs &a, cudaStream_t s);
// the Jacobi sweep with its tile staged in shared memory by the tensor memory
// accelerator (k_sweep_tma.cu); tensor maps of the psi buffers, b and diag M
struct TmaMaps {
    CUtensorMap psi[3], b, D;
};
// cuTensorMapEncodeTiled from the driver (nullptr if unavailable)
void *tma_encode_entry();
bool tma_sweep_supported(const DevGrid &g);
bool tma_encode_maps(const DevGrid &g, float2 *const psi[3], const float2 *b, const float2 *D, TmaMaps *m);
cudaError_t launch_sweep_tma(const SweepArgs &a, const CUtensorMap &map_psi, const TmaMaps &m, cudaStream_t s);
int sweep_blocks(const DevGrid &g);
// two sweeps per pass (k_pair.cu); the decision is the per-sweep one
bool pair_supported(const DevGrid &g);
size_t pair_blocks(const DevGrid &g);
cudaError_t launch_sweep_pair(const SweepArgs &a, cudaStream_t s);

struct KArgs {
    DevGrid g;
    DevCtl *ctl;
    double *blockred;
    const float2 *psi;
    double hx, dtK, Jext;
    int update_K;              // 1: integrate the K ODE
};
cudaError_t launch_javg_K(const KArgs &a, cudaStream_t s);
cudaError_t launch_set_Ux(DevCtl *ctl, double hx, cudaStream_t s);

// Explicit-Euler step of the K ODE (Sec. 2.2, Eq. K_ODE) from J_av, E_x = dK/dt,
// and the rewind of K into [0, 2 pi / hx); run by one thread.
__device__ __forceinline__ void k_ode_update(DevCtl *c, double jav, double hx, double dtK, double Jext, int update_K)
{
    c->javg = jav;
    if (!update_K) return;
    double K0 = c->K;
    double K1 = K0 + dtK * (Jext - jav);
    c->Ex = (K1 - K0) / dtK;
    const double twopi = 6.283185307179586476925286766559;
    K1 = K1 - (twopi / hx) * floor(K1 * hx / twopi);
    c->K = K1;
    double sn, cs;
    sincos(hx * K1, &sn, &cs);
    c->Ux = make_float2((float)cs, (float)sn);
}

// Multigrid Poisson solver
struct MGLevel {
    int nx, ny, nz;
    long long N;
    int fy, fz;                // coarsening factor from this level to the next (1 or 2)
    float cx, cy, cz;
    float *u;                  // solution / correction
    float *r;                  // right-hand side
    float *t;                  // residual scratch
    float *G;                  // x-line inverse kernel G_k, k = kmin..kmax (device)
    int P;                     // period of the extended x line: nx (periodic) or 2(nx-1) (open)
    int kmin, kmax;            // kernel support (kmax - kmin + 1 <= P)
    float *cw;                 // coarsest level only: [W (M x M) | V (M x M) | G_q (M x P)], or nullptr
    int M;                     // number of y-z modes of the coarsest level (ny * nz)
    // recursive exact line solve (short decay): chunk C = nx / 32 sites per lane, or 0;
    // rho = t - sqrt(t^2 - 1), t = 1 + s / (2 cx), and the output scale rho / cx
    int iir, iir_w;    // recursive line solve: C sites per lane, warm-up length iir_w (0: exact scan)
    float rho, rscale;
    // exact scan: rho^(C 2^q) (q = 0..4), log2 rho, 1 / (1 - rho^P) (P the period of the
    // extended line), 1 / (1 - rho^2)
    float rhoC[5], l2rho, gf, gb;
};
int mg_period(int nx, int bcx);
// x lines of colour c ((j + k) % 2 == c) on an ny x nz line grid
long long mg_lines_of_colour(int ny, int nz, int c);
// Line-inverse kernel of a level with shift s = 2 cy + 2 cz; returns kmin.
int mg_line_kernel(int nx, int bcx, double cx, double s, std::vector<float> &Gs);
// Eigen-decomposition of the coarsest level's y-z operator and per-mode kernels
// (host, FP64 -> f32), M = ny*nz.  Returns false if the basis is singular.
size_t mg_coarse_floats(int nx, int bcx, int M);
bool mg_coarse_factors(int nx, int bcx, double cx, int ny, int nz, int bcy, int bcz, double cy, double cz, float *cw);
struct PoissonArgs {
    DevGrid g;
    DevCtl *ctl;
    double *blockred;
    int nlevels;
    MGLevel lev[kMaxLevels];
    float *f;                  // level-0 right-hand side (= lev[0].r)
    float *mu;                 // level-0 solution (= lev[0].u)
    double hx, Jext;
    int inject;                // open x with applied current
    double wsum;
    // levels smoothed by the recursive line solve: 2-D tensor maps of u viewed as rows of
    // 32 floats, a box being one 512-site line (16 rows, 128-byte swizzle), and the u each
    // map was made for (nullptr: none; a copy of these arguments pointing its u elsewhere
    // falls back to the asynchronous-copy smoother)
    CUtensorMap umap[kMaxLevels];
    const float *umap_u[kMaxLevels];
    int mu_q;                  // the handle's mu buffer that mu points at (-1: another array)
    // staged kernels' wait bound and extra expected bytes (as in SweepArgs; 0: normal use)
    unsigned long long wait_ns;
    unsigned int extra_tx;
    // mean_dot 1: a cycle's fused closing sum (mean_out) is the weighted inner product of
    // the right-hand side and the result, sum w f u, into ctl->sums[dot_slot], instead of
    // the mean of u
    int mean_dot, dot_slot;
};
// tensor maps for the levels of pa that the recursive smoother handles (false: none made)
bool mg_encode_line_maps(PoissonArgs &pa);
cudaError_t launch_poisson_rhs(const PoissonArgs &a, const float2 *psi, cudaStream_t s);
// the right-hand side through the staged sweep tile (psi boxes only); map_psi describes psi
cudaError_t launch_poisson_rhs_tma(const PoissonArgs &pa, const float2 *psi, const CUtensorMap &map_psi,
                                   const TmaMaps &m, cudaStream_t s);
// after_cycle: the call directly follows a V-cycle on the same right-hand side
// mean_out: the cycle's closing finest-level passes also leave the weighted mean of mu in
// ctl->mu_mean, where vcycle_mean_fusable allows (launch_project_mu then skips its own sum)
cudaError_t launch_vcycle(const PoissonArgs &a, cudaStream_t s, long long *launches, bool after_cycle = false,
                          bool mean_out = false);
bool vcycle_mean_fusable(const PoissonArgs &a);
cudaError_t launch_poisson_residual(const PoissonArgs &a, cudaStream_t s);
cudaError_t launch_project_mu(const PoissonArgs &a, cudaStream_t s, bool mean_done = false);
// ctl->fmean = the trapezoid-weighted mean of the level-0 right-hand side f
cudaError_t launch_f_mean(const PoissonArgs &a, cudaStream_t s);
// the projection left pending: ctl->mu_off[a.mu_q] = ctl->mu_mean (the fused mean of the cycle)
cudaError_t launch_commit_mean(const PoissonArgs &a, cudaStream_t s);
// subtract the pending mean from mu_buf (mu_off[q]) and clear it
cudaError_t launch_mu_materialize(long long N, float *mu, DevCtl *ctl, int q, cudaStream_t s);
cudaError_t launch_voltage(const PoissonArgs &a, cudaStream_t s);

// Insulating inclusions (k_insulating.cu)
cudaError_t launch_link_bits(const DevGrid &g, const uint8_t *ins, uint8_t *lk, cudaStream_t s);
constexpr int kMaxIslands = 1 << 16;   // conducting components besides the largest one
struct InsPoisson {
    float *r, *z, *p, *q;      // residual, preconditioned residual, direction, A p
    int *comp;                 // [N] 0: largest conducting component, 1..: islands, -1: insulating
    double *isl_w, *isl_acc;   // [kMaxIslands] sum of w per island, per-island scratch sums
    int n_isl;                 // islands (conducting components enclosed by insulators)
    double wsum_c;             // sum of w over the largest component
    double n_face0, n_face1;   // its sites on the x = 0 and x = L faces
    CUtensorMap zmap;          // the finest smoother's map of z for the preconditioning V-cycle
    const float *zmap_u;       // z when zmap is valid, else nullptr
};
// Conducting components (labels by propagation in r..z as scratch), their compact ids,
// and the weights of each; TDGL_ERR_INVALID_ARG beyond kMaxIslands islands.
int build_components(const DevGrid &g, InsPoisson &ip, DevCtl *ctl, double *blockred, cudaStream_t s);
// Poisson solve with the links next to insulating sites removed: CG in the trapezoid-
// weighted inner product, preconditioned by one V-cycle of the plain operator.
// iters > 0: exactly that many iterations; else up to max_iters until res <= tol
// (a host read per iteration).  Returns a TDGL_* code and the iterations done.
int masked_poisson_solve(const PoissonArgs &pa, const InsPoisson &ip, double tol, int iters, int max_iters,
                         cudaStream_t s, int *done, long long *launches);
cudaError_t launch_voltage_masked(const PoissonArgs &a, const InsPoisson &ip, cudaStream_t s);

// Observables
cudaError_t launch_observables(const DevGrid &g, DevCtl *ctl, double *blockred, const float2 *psi,
                               const float *alpha, int32_t *scratch_i, double flux, cudaStream_t s);

// Pattern generator (k_pattern.cu): the work of tdgl_pattern_ex after argument checks
size_t pattern_ex_scratch(const tdgl_config *grid, int64_t n_shapes, const tdgl_lattice *lats, int32_t n_lattices,
                          const tdgl_background *bg);
int pattern_ex_run(const tdgl_config *grid, const tdgl_shape *shapes, int64_t n_shapes, const tdgl_lattice *lats,
                   int32_t n_lattices, const tdgl_background *bg, int64_t target, float *d_alpha,
                   uint8_t *d_insulating, void *d_scratch, size_t scratch_bytes, cudaStream_t s, int64_t *n_used,
                   int64_t *n_marked);

// Adjoint kernels (k_adjoint.cu) and the adjoint sweep (k_jacobi.cu)
cudaError_t launch_adj_sweep(const SweepArgs &a, cudaStream_t s);
bool adj_supported(const DevGrid &g);
cudaError_t launch_adj_fterm(const DevGrid &g, float2 Ux, const float2 *psi, const float *u, const float2 *psibar,
                             float2 *gout, cudaStream_t s);
cudaError_t launch_adj_diag(const DevGrid &g, const float2 *psi_p, const float *mu_p, const float *alpha,
                            const float2 *gv, float2 *D, float2 *lam0, cudaStream_t s);
cudaError_t launch_adj_update(const DevGrid &g, const float2 *lam, const float2 *psi_n, const float2 *psi_p,
                              const float2 *gv, float *grad, float *mubar, float2 *psibar, cudaStream_t s);
cudaError_t launch_adj_voltage_source(const DevGrid &g, float *mubar, float s_val, cudaStream_t s);
cudaError_t launch_adj_rhs(const DevGrid &g, const float *mubar, float *r, DevCtl *ctl, double *blockred, double wsum,
                           cudaStream_t s);

// Batched persistent step (k_batch.cu).  One entry per instance, in device memory.
constexpr int kBatchMax = TDGL_BATCH_MAX;
struct BatchHead {
    SweepArgs a;               // sweep arguments (src/dst set per phase)
    float2 *psi[3];            // the handle's three iterate buffers
    int iS, iA, iB;            // state buffer and the two Jacobi buffers
    int kz, gx, gy, gz;        // sweep tiling: tiles = gx gy gz
    int tiles;
    int split_max;             // z parts a sweep tile may be split into (1, 2 or 4: divides kz, fits the partial slots)
    int mean_fused;            // 1: the zero mode and the voltage are summed by the finest smoothing passes
    int red_chunk, red_items;  // sites per reduction item, items (<= half the partial slots)
    int periodic_x, open_x, freeze, cycles;
    double hx, dtK, Jext;
    int nlev;                  // multigrid levels
    int lpb[kMaxLevels];       // lines per smoothing tile
    long long nlines[kMaxLevels][2];
    // the Poisson solve's buffer: the state mu itself, or (extrapolated guess) the second
    // mu buffer, which holds the previous step's mu until the init writes the guess there;
    // the closing shift then writes the new state into mu and the old one into this buffer
    float *mu_solve;
};
struct BatchInst {
    BatchHead h;               // staged in shared memory by every work item
    PoissonArgs pa;
};
struct BatchParams {
    const BatchInst *inst;     // [n]
    int n;
    int lmax;                  // max over instances of (levels - 1)
    int cycles_max;
    int any_px;                // some instance has a periodic x axis
    int max_phases;            // bound on Jacobi phases per launch
    int staged;                // 1: Jacobi sweep tiles staged in shared memory; 0: register-tiled
    int any_mean;              // 1: some instance needs the separate mean phase (no fused sums)
    // [n]: the instances in the order their items are dealt, the largest sweep tiles first, so
    // that a phase ends on small items
    const int *order;
    int *act;                  // [2][n]: instance still iterating after a phase of that parity
    int *bst;                  // [n]: 0, or the error that stopped the instance
    long long *sweeps;         // [n]: cumulative Jacobi sweeps
    unsigned int *bar;         // [0] barrier arrivals (zeroed before each launch), [1] error flag
    unsigned int extra;        // arrivals a barrier waits for beyond the grid (0; >0 only to test the timeout)
    unsigned long long timeout_ns;
    unsigned long long *plog;  // optional phase log: [2 i] globaltimer at the end of phase i, [2 i + 1] its op
    int plog_cap;              // entries in plog (0: no log)
};
size_t batch_smem_bytes(const BatchInst &I);
// Occupancy of the kernel variant built for bps (2 or 3) resident blocks per SM.
cudaError_t batch_max_blocks_per_sm(size_t smem, int bps, int *out);
cudaError_t launch_batch_step(const BatchParams &p, int grid, int bps, size_t smem, cudaStream_t s);
int batch_default_kz(const DevGrid &g);
void batch_tiling(BatchInst &I, int kz);

}  // namespace tdgl

// Host-side solver handle (shared by the C ABI translation units).
struct tdgl_handle {
    tdgl_config cfg;
    tdgl::DevGrid g;
    cudaStream_t stream;
    tdgl::DevCtl *ctl;
    double *blockred;
    float2 *psi[3];
    int cur;
    float2 *b, *D;
    float *mu, *f;             // mu: the current state, mu_buf[mu_q]
    // Poisson guess by extrapolation in time: the solve of a step runs in the other buffer,
    // which the init has overwritten with 2 mu^(n-1) - mu^(n-2) (mu^(n-1) when prev_valid is
    // 0), and then becomes the state; the old state is the next step's mu^(n-2)
    float *mu_buf[2];
    int mu_q;
    int prev_valid;            // 1: mu_buf[1 - mu_q] holds the state of the step before
    int mu_pend[2];            // 1: a pending mean was recorded for the buffer (ctl->mu_off[q])
    int guess_ready;           // 1: the init of this step has written the guess
    CUtensorMap umap0[2];      // the finest level's smoother maps for each mu buffer
    const float *umap0_u[2];
    float2 *links;
    tdgl::PoissonArgs pa;
    size_t nblockred;          // capacity of blockred (doubles)
    int batch_owned;           // 1: stepped only through a batch
    float noise_amp;           // h_t zeta_max, 0 without noise
    int last_sweeps;
    int last_cycles;
    int64_t step;
    double wsum;
    double dtK;
    double last_javg;
    uint8_t *lk;               // link bits when insulating sites are given, else nullptr
    int use_tma;               // 1: Jacobi sweeps by the shared-memory staged kernel
    int mu_solved;             // 1: a Poisson solve has run (f and mu hold its right-hand side and result)
    int in_adjoint;            // 1: tdgl_adjoint is running (projections applied at once)
    // z-slab of a larger grid (tdgl_slab_create): planes 1 .. slab_nz of the arrays are the
    // slab (global planes slab_z0 ..), planes 0 and slab_nz + 1 the halos
    int slab, slab_z0, slab_nz;
    int slab_n;                // sweeps of the current slab solve
    int slab_last;             // buffer of the latest slab iterate
    int poisson_only;          // 1: no psi arrays (tdgl_poisson_create)
    unsigned long long dbg_wait_ns;   // tdgl_test_staged_waits: wait bound (0: default)
    unsigned int dbg_extra_tx;        // tdgl_test_staged_waits: extra expected bytes (0: none)
    // the Poisson solve of a step (right-hand side, V-cycles, projection) as CUDA graphs,
    // one per psi buffer, captured on a private stream and replayed on the handle's stream
    cudaStream_t cap_stream;
    cudaGraphExec_t pgraph[6];   // per psi buffer (3) and mu buffer (2)
    int pgraph_fail;
    int poisson_calls;
    long long pgraph_launches;
    // the device-resident step loop: one graph of conditional nodes for any number of steps
    cudaGraphExec_t rgraph;
    int rgraph_fail;
    int stepped;                 // 1: a host-driven step has run on the handle
    int res_pending;             // 1: resident steps enqueued, not yet accounted on the host
    long long rgraph_launches;   // launches of one step outside the sweep loop
    tdgl::TmaMaps tmaps;       // its tensor maps
    tdgl::InsPoisson ip;
    // profiling
    int prof_on;
    static constexpr int kEvents = 10;
    cudaEvent_t ev[kEvents];
    bool ev_made;
    bool pend_K, pend_P, pend_R;   // K / Poisson / recomputed-sweep event pairs recorded but not yet read
    tdgl_profile prof;
};

namespace tdgl {
bool handle_extrapolates(const tdgl_handle *h);
void use_mu_buffer(tdgl_handle *h, int q);
int mu_materialize(tdgl_handle *h, int q);
void drop_poisson_graphs(tdgl_handle *h);
// pieces of the host-driven step (tdgl_api.cu) used by the device-resident loop
SweepArgs step_sweep_args(tdgl_handle *h);
void step_guess_args(const tdgl_handle *h, SweepArgs &a, int q);
long long step_poisson_sequence(tdgl_handle *h, cudaStream_t s, cudaError_t *err);
bool step_lazy_projection(const tdgl_handle *h);
bool step_pairs(const tdgl_handle *h);
int step_read_ctl(tdgl_handle *h, DevCtl *out);
// wait for the resident steps enqueued on the handle and account for them on the host;
// returns their status (TDGL_OK when none are pending)
int resident_sync(tdgl_handle *h);
}  // namespace tdgl
