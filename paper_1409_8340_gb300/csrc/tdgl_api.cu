// C ABI of the solver: configuration checks, workspace layout, link tables,
// and the order of launches within a time step (arXiv:1409.8340, Sec. 3 and
// Sec. 4.1: psi first, then K, then mu).
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "tdgl_internal.cuh"

using namespace tdgl;

namespace tdgl {

// The Poisson solve starts from the extrapolated guess (tdgl_config.poisson_guess 0 or 2),
// where the handle has the second mu buffer and solves mu itself
bool handle_extrapolates(const tdgl_handle *h)
{
    const int gm = h->cfg.poisson_guess;
    return h->mu_buf[1] != nullptr && !h->batch_owned && !h->cfg.freeze_mu_K && (gm == 0 || gm == 2);
}

// make mu_buf[q] the state: the finest multigrid level solves in it
void use_mu_buffer(tdgl_handle *h, int q)
{
    h->mu_q = q;
    h->mu = h->mu_buf[q];
    h->pa.mu = h->pa.lev[0].u = h->mu;
    h->pa.mu_q = q;
    h->pa.umap[0] = h->umap0[q];
    h->pa.umap_u[0] = h->umap0_u[q];
}

// Apply the pending zero-mode projection of mu buffer q (a fixed-cycle solve leaves it in
// ctl->mu_off[q]; nothing to do without one)
int mu_materialize(tdgl_handle *h, int q)
{
    if (h->lk || h->batch_owned || !h->mu_buf[q] || !h->mu_pend[q]) return TDGL_OK;
    h->mu_pend[q] = 0;
    return launch_mu_materialize(h->g.N, h->mu_buf[q], h->ctl, q, h->stream) == cudaSuccess ? TDGL_OK : TDGL_ERR_CUDA;
}

void drop_poisson_graphs(tdgl_handle *h)
{
    for (int q = 0; q < 6; ++q)
        if (h->pgraph[q]) {
            cudaGraphExecDestroy(h->pgraph[q]);
            h->pgraph[q] = nullptr;
        }
    if (h->rgraph) {
        cudaGraphExecDestroy(h->rgraph);
        h->rgraph = nullptr;
    }
}

}  // namespace tdgl

namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int active(int n) { return n >= 2; }

double box_len(int n, double h, int bc) { return bc == TDGL_PERIODIC ? n * h : (n - 1) * h; }

// flux quantum count n = B L1 L2 / 2 pi; returns false if not an integer
bool quantised(double B, double L1, double L2, long long *n)
{
    double q = B * L1 * L2 / kTwoPi;
    double r = floor(q + 0.5);
    *n = (long long)r;
    return fabs(q - r) <= 1e-9 * (1.0 + fabs(q));
}

// pon: a Poisson-only handle (tdgl_poisson_create), which has no psi and reads no alpha
int validate(const tdgl_config *c, bool pon = false)
{
    if (!c) return TDGL_ERR_INVALID_ARG;
    if (c->nx < 2 || c->ny < 2 || c->nz < 1) return TDGL_ERR_INVALID_ARG;
    if ((long long)c->nx * c->ny * c->nz > (1LL << 33)) return TDGL_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a)
        if (c->bc[a] != TDGL_PERIODIC && c->bc[a] != TDGL_OPEN) return TDGL_ERR_INVALID_ARG;
    if ((c->bc[0] == TDGL_PERIODIC && c->nx < 3) || (c->bc[1] == TDGL_PERIODIC && c->ny < 3) ||
        (c->bc[2] == TDGL_PERIODIC && c->nz == 2))
        return TDGL_ERR_INVALID_ARG;   // a periodic axis needs distinct forward and backward neighbours
    if (!(c->hx > 0) || !(c->hy > 0) || !(c->hz > 0) || !(c->g > 0) || !(c->ht > 0)) return TDGL_ERR_INVALID_ARG;
    if (!(c->u > 0) || !(c->beta >= 0)) return TDGL_ERR_INVALID_ARG;
    if (c->max_iter < 1 || c->check_every < 1 || c->fixed_sweeps < 0) return TDGL_ERR_INVALID_ARG;
    if (c->sweeps_per_pass < 0 || c->sweeps_per_pass > 2) return TDGL_ERR_INVALID_ARG;
    if (c->sweep_kernel < 0 || c->sweep_kernel > 2) return TDGL_ERR_INVALID_ARG;
    if (c->poisson_guess < 0 || c->poisson_guess > 2) return TDGL_ERR_INVALID_ARG;
    if (!(c->noise_T >= 0)) return TDGL_ERR_INVALID_ARG;
    if (c->fixed_sweeps == 0 && !(c->eps > 0)) return TDGL_ERR_INVALID_ARG;
    if (c->poisson_cycles < 1 || c->poisson_max_cycles < c->poisson_cycles) return TDGL_ERR_INVALID_ARG;
    if (!c->d_alpha && !pon) return TDGL_ERR_INVALID_ARG;
    if (c->links_mode != TDGL_LINKS_LANDAU && c->links_mode != TDGL_LINKS_GENERAL && c->links_mode != TDGL_LINKS_XZ)
        return TDGL_ERR_INVALID_ARG;
    if (c->links_mode == TDGL_LINKS_GENERAL && !c->d_link_phase) return TDGL_ERR_INVALID_ARG;
    if (c->nx > 1500) return TDGL_ERR_INVALID_ARG;   // x lines of the Poisson smoother live in shared memory
    if (!(c->Bx == c->Bx) || !(c->By == c->By) || !(c->Bz == c->Bz)) return TDGL_ERR_INVALID_ARG;
    // insulating inclusions run on the tiled kernels: Landau links of either plane, even nx
    if (c->d_insulating && (c->links_mode == TDGL_LINKS_GENERAL || (c->nx % 2) != 0)) return TDGL_ERR_INVALID_ARG;
    // each gauge carries the field components of its plane only
    if (c->links_mode == TDGL_LINKS_LANDAU && c->Bx != 0.0) return TDGL_ERR_INVALID_ARG;
    if (c->links_mode == TDGL_LINKS_XZ && c->By != 0.0) return TDGL_ERR_INVALID_ARG;
    const double Lx = box_len(c->nx, c->hx, c->bc[0]), Ly = box_len(c->ny, c->hy, c->bc[1]);
    const double Lz = box_len(c->nz, c->hz, c->bc[2]);
    const bool pz = c->bc[2] == TDGL_PERIODIC && c->nz >= 2;
    long long n;
    if (c->links_mode == TDGL_LINKS_LANDAU && c->bc[0] == TDGL_PERIODIC) {
        // quasi-periodic x wrap (Sec. 3.3.1)
        if (c->bc[1] == TDGL_PERIODIC && !quantised(c->Bz, Lx, Ly, &n)) return TDGL_ERR_INVALID_ARG;
        if (pz && !quantised(c->By, Lx, Lz, &n)) return TDGL_ERR_INVALID_ARG;
    }
    if (c->links_mode == TDGL_LINKS_XZ && c->bc[1] == TDGL_PERIODIC) {
        // quasi-periodic y wrap of the xz-plane gauge
        if (c->bc[0] == TDGL_PERIODIC && !quantised(c->Bz, Lx, Ly, &n)) return TDGL_ERR_INVALID_ARG;
        if (pz && !quantised(c->Bx, Ly, Lz, &n)) return TDGL_ERR_INVALID_ARG;
    }
    return TDGL_OK;
}

struct Layout {
    size_t ctl, blockred, psi[3], b, D, mu, mu2, f, t, links, xzt, lk, insv, comp, isl, Uy, Uz, Py, Pz, total;
    int nlevels;
    int ny[kMaxLevels], nz[kMaxLevels], fy[kMaxLevels], fz[kMaxLevels];
    size_t u[kMaxLevels], r[kMaxLevels], tri[kMaxLevels];
    size_t nblockred;
    size_t cw;        // coarsest-level eigen-factors (0: none, the coarsest level is relaxed)
};

constexpr int kCoarseModes = 128;

bool can_coarsen(int n, int bc)
{
    if (bc == TDGL_PERIODIC) return (n % 2 == 0) && n >= 8;
    return (n % 2 == 1) && n >= 5;
}
int coarse_n(int n, int bc) { return bc == TDGL_PERIODIC ? n / 2 : (n - 1) / 2 + 1; }

Layout layout(const tdgl_config *c, bool pon = false)
{
    Layout L;
    memset(&L, 0, sizeof(L));
    const long long N = (long long)c->nx * c->ny * c->nz;
    DevGrid g;
    memset(&g, 0, sizeof(g));
    g.nx = c->nx;
    g.ny = c->ny;
    g.nz = c->nz;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    L.ctl = take(sizeof(DevCtl));
    size_t nb = (size_t)sweep_blocks(g);
    if (nb < 4 * 4096) nb = 4 * 4096;
    const size_t nb2d = 2 * (size_t)((c->nx + 127) / 128) * (size_t)c->ny;   // 2-D reduction grids, 2 values each
    if (nb < nb2d) nb = nb2d;
    if (nb < 2 * pair_blocks(g)) nb = 2 * pair_blocks(g);
    L.nblockred = nb;
    L.blockred = take(sizeof(double) * nb);
    const size_t npsi = pon ? 0 : (size_t)N;   // a Poisson-only handle holds no psi, b or diag M
    for (int q = 0; q < 3; ++q) L.psi[q] = take(8 * npsi);
    L.b = take(8 * npsi);
    L.D = take(8 * npsi);
    L.mu = take(4 * (size_t)N);
    // the second mu buffer: the previous step's mu, over which the init writes the guess
    // that the next Poisson solve starts from (the multigrid solve and the masked CG)
    L.mu2 = take(4 * (size_t)N);
    L.f = take(4 * (size_t)N);
    L.t = take(4 * (size_t)N);
    L.links = (c->links_mode != TDGL_LINKS_LANDAU) ? take(8 * 3 * (size_t)N) : 0;
    L.xzt = (c->links_mode == TDGL_LINKS_XZ) ? take(8 * (2 * (size_t)c->ny + c->nx + c->nz)) : 0;
    // insulating inclusions: link bits, and r, z, p, q of the Poisson CG (also the labels
    // of the connectivity check, 8 bytes per site, at creation)
    L.lk = c->d_insulating ? take((size_t)N) : 0;
    L.insv = c->d_insulating ? take(16 * (size_t)N) : 0;
    L.comp = c->d_insulating ? take(4 * (size_t)N) : 0;
    L.isl = c->d_insulating ? take(16 * (size_t)kMaxIslands) : 0;
    L.Uy = take(8 * (size_t)c->nx);
    L.Uz = take(8 * (size_t)c->nx);
    L.Py = take(8 * (size_t)c->ny);
    L.Pz = take(8 * (size_t)c->nz);
    // multigrid levels
    int ny = c->ny, nz = c->nz, l = 0;
    for (;;) {
        L.ny[l] = ny;
        L.nz[l] = nz;
        L.tri[l] = take(4 * (size_t)mg_period(c->nx, c->bc[0]));
        if (l > 0) {
            L.u[l] = take(4 * (size_t)c->nx * ny * nz);
            L.r[l] = take(4 * (size_t)c->nx * ny * nz);
        }
        bool cy = can_coarsen(ny, c->bc[1]);
        bool cz = nz >= 2 && can_coarsen(nz, c->bc[2]);
        // a level with at most kCoarseModes y-z modes is solved exactly (dense basis)
        if ((!cy && !cz) || ny * nz <= kCoarseModes || l + 1 >= kMaxLevels) {
            L.fy[l] = L.fz[l] = 1;
            break;
        }
        L.fy[l] = cy ? 2 : 1;
        L.fz[l] = cz ? 2 : 1;
        ny = cy ? coarse_n(ny, c->bc[1]) : ny;
        nz = cz ? coarse_n(nz, c->bc[2]) : nz;
        ++l;
    }
    L.nlevels = l + 1;
    {
        // exact coarsest solve when the dense y-z basis stays small
        const int M = L.ny[l] * L.nz[l];
        L.cw = (M <= 1024) ? take(sizeof(float) * mg_coarse_floats(c->nx, c->bc[0], M)) : 0;
    }
    L.total = off;
    return L;
}

template <class T>
T *at(void *base, size_t off)
{
    return reinterpret_cast<T *>(reinterpret_cast<char *>(base) + off);
}

int cuda_err(cudaError_t e) { return e == cudaSuccess ? TDGL_OK : TDGL_ERR_CUDA; }

__global__ void phases_to_links(const float *theta, float2 *L, long long n3)
{
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n3; q += (long long)gridDim.x * blockDim.x) {
        float s, c;
        sincosf(theta[q], &s, &c);
        L[q] = make_float2(c, s);
    }
}

// Links of the xz-plane Landau gauge (A = ybar [-Bz, 0, Bx], ybar = j hy - Ly/2): the
// x and z links depend on j only (tables X[j], Z[j]); on a periodic y axis the wrap link
// from j = Ny-1 to j = 0 is Wx[i] Wz[k] = exp(-i(i hx Ly Bz - k hz Ly Bx)), the conjugate
// of the quasi-periodic factor psi_{i,-1,k} = P_{i,k} psi_{i,Ny-1,k} (Sec. 3.3.1).
// t = [X ny][Z ny][Wx nx][Wz nz], each entry rounded from FP64 once.
__global__ void xz_links(const float2 *t, float2 *L, int nx, int ny, int nz, int wrap_y)
{
    const long long N = (long long)nx * ny * nz;
    const float2 *X = t, *Z = t + ny, *Wx = t + 2 * ny, *Wz = Wx + nx;
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < N; m += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(m % nx);
        const long long jk = m / nx;
        const int j = (int)(jk % ny), k = (int)(jk / ny);
        L[m] = X[j];
        L[N + m] = (wrap_y && j == ny - 1) ? cmul(Wx[i], Wz[k]) : make_float2(1.f, 0.f);
        L[2 * N + m] = Z[j];
    }
}

void ev_collect(tdgl_handle *h);

int read_ctl(tdgl_handle *h, DevCtl *out)
{
    cudaError_t e = cudaMemcpyAsync(out, h->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return TDGL_ERR_CUDA;
    int rc = cuda_err(cudaStreamSynchronize(h->stream));
    ev_collect(h);
    return rc;
}

SweepArgs sweep_args(tdgl_handle *h)
{
    SweepArgs a;
    memset(&a, 0, sizeof(a));
    a.g = h->g;
    a.ctl = h->ctl;
    a.blockred = h->blockred;
    a.b = h->b;
    a.D = h->D;
    a.mu = h->mu;
    a.alpha = h->cfg.d_alpha;
    a.check_every = h->cfg.check_every;
    a.fixed_sweeps = h->cfg.fixed_sweeps;
    a.max_iter = h->cfg.max_iter;
    a.eps = h->cfg.eps;
    a.noise_amp = h->noise_amp;
    a.noise_seed = h->cfg.noise_seed;
    a.wait_ns = h->dbg_wait_ns;
    a.extra_tx = h->dbg_extra_tx;
    return a;
}

bool extrapolating(const tdgl_handle *h) { return handle_extrapolates(h); }

// The init also writes the coming Poisson solve's guess over mu^(n-2), the buffer other than
// the state's q: 2 mu^(n-1) - mu^(n-2) with a previous mu (prev), else mu^(n-1)
void guess_args(const tdgl_handle *h, SweepArgs &a, int q, bool prev)
{
    const tdgl_config &c = h->cfg;
    a.mu_off_prev = &h->ctl->mu_off[1 - q];
    a.mu_guess = h->mu_buf[1 - q];
    a.ex_a = prev ? 2.f : 1.f;
    a.ex_b = prev ? -1.f : 0.f;
    // the V-cycle's first pass reads only the colour-1 rows of the guess when the zebra
    // colouring (j + k) % 2 is proper and the finest level is smoothed (the masked CG's
    // first residual reads every site)
    const bool proper = (c.bc[1] == TDGL_OPEN || (c.ny % 2) == 0) && (c.bc[2] == TDGL_OPEN || c.nz == 1 || (c.nz % 2) == 0);
    a.guess_odd_only = (proper && h->pa.nlevels > 1 && !h->lk) ? 1 : 0;
}

void ev_rec(tdgl_handle *h, int i)
{
    if (h->prof_on) cudaEventRecord(h->ev[i], h->stream);
}

double ev_ms(tdgl_handle *h, int a, int b)
{
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->ev[a], h->ev[b]) != cudaSuccess) return 0.0;
    return (double)ms;
}

// Read K / Poisson timings recorded in an earlier step (the stream has been
// synchronised since, so the events are complete).
void ev_collect(tdgl_handle *h)
{
    if (!h->prof_on) return;
    if (h->pend_K) h->prof.ms_K += ev_ms(h, 4, 5);
    if (h->pend_P) h->prof.ms_poisson += ev_ms(h, 6, 7);
    if (h->pend_R) h->prof.ms_sweeps += ev_ms(h, 8, 9);
    h->pend_K = h->pend_P = h->pend_R = false;
}

}  // namespace

extern "C" {

const char *tdgl_error_string(int code)
{
    switch (code) {
    case TDGL_OK: return "ok";
    case TDGL_ERR_INVALID_ARG: return "invalid argument";
    case TDGL_ERR_NOT_CONVERGED: return "Jacobi iteration did not converge within max_iter sweeps";
    case TDGL_ERR_NONFINITE: return "non-finite residual";
    case TDGL_ERR_TIMEOUT: return "device wait timed out";
    case TDGL_ERR_CUDA: return "CUDA runtime error";
    case TDGL_ERR_WORKSPACE: return "workspace too small or misaligned";
    default: return "unknown error";
    }
}

size_t tdgl_abi_struct_size(int32_t which)
{
    switch (which) {
    case 0: return sizeof(tdgl_config);
    case 1: return sizeof(tdgl_obs);
    case 2: return sizeof(tdgl_state_ptrs);
    case 3: return sizeof(tdgl_profile);
    case 4: return sizeof(tdgl_adjoint_config);
    case 5: return sizeof(tdgl_adjoint_stats);
    case 6: return sizeof(tdgl_batch_tuning);
    case 7: return sizeof(tdgl_batch_stats);
    case 8: return sizeof(tdgl_batch_tune_report);
    case 9: return sizeof(tdgl_shape);
    case 10: return sizeof(tdgl_lattice);
    case 11: return sizeof(tdgl_background);
    case 12: return sizeof(tdgl_tune_report);
    default: return 0;
    }
}

size_t tdgl_workspace_bytes(const tdgl_config *cfg)
{
    if (validate(cfg) != TDGL_OK) return 0;
    return layout(cfg).total;
}

static int create_impl(const tdgl_config *cfg, void *ws, size_t ws_bytes, void *stream, tdgl_handle **out, bool pon);

int tdgl_create(const tdgl_config *cfg, void *ws, size_t ws_bytes, void *stream, tdgl_handle **out)
{
    return create_impl(cfg, ws, ws_bytes, stream, out, false);
}

static int create_impl(const tdgl_config *cfg, void *ws, size_t ws_bytes, void *stream, tdgl_handle **out, bool pon)
{
    if (!out) return TDGL_ERR_INVALID_ARG;
    *out = nullptr;
    int v = validate(cfg, pon);
    if (v != TDGL_OK) return v;
    Layout L = layout(cfg, pon);
    if (!ws || ((uintptr_t)ws & 255u) || ws_bytes < L.total) return TDGL_ERR_WORKSPACE;
    tdgl_handle *h = new tdgl_handle();
    h->cfg = *cfg;
    h->stream = (cudaStream_t)stream;
    const tdgl_config &c = *cfg;
    const long long N = (long long)c.nx * c.ny * c.nz;
    DevGrid &g = h->g;
    g.nx = c.nx;
    g.ny = c.ny;
    g.nz = c.nz;
    g.N = N;
    g.bcx = c.bc[0];
    g.bcy = c.bc[1];
    g.bcz = c.bc[2];
    g.cx = (float)(1.0 / (c.hx * c.hx));
    g.cy = (float)(1.0 / (c.hy * c.hy));
    g.cz = active(c.nz) ? (float)(1.0 / (c.g * c.g * c.hz * c.hz)) : 0.f;
    g.S = (float)(1.0 / (c.hx * c.hx) + 1.0 / (c.hy * c.hy) + (active(c.nz) ? 1.0 / (c.g * c.g * c.hz * c.hz) : 0.0));
    g.ht2 = (float)(0.5 * c.ht);
    g.u = (float)c.u;
    g.beta = (float)c.beta;
    g.Uy = at<float2>(ws, L.Uy);
    g.Uz = at<float2>(ws, L.Uz);
    g.Py = at<float2>(ws, L.Py);
    g.Pz = at<float2>(ws, L.Pz);
    g.L = (c.links_mode != TDGL_LINKS_LANDAU) ? at<float2>(ws, L.links) : nullptr;
    if (c.links_mode == TDGL_LINKS_XZ) {
        float2 *t = at<float2>(ws, L.xzt);   // [X ny][Z ny][Wx nx][Wz nz]
        g.Xj = t;
        g.Zj = t + c.ny;
        g.Wx = t + 2 * (size_t)c.ny;
        g.Wz = t + 2 * (size_t)c.ny + c.nx;
    } else {
        g.Xj = g.Zj = g.Wx = g.Wz = nullptr;
    }
    g.lk = c.d_insulating ? at<uint8_t>(ws, L.lk) : nullptr;
    h->lk = const_cast<uint8_t *>(g.lk);
    memset(&h->ip, 0, sizeof(h->ip));
    if (c.d_insulating) {
        float *v = at<float>(ws, L.insv);
        h->ip.r = v;
        h->ip.z = v + N;
        h->ip.p = v + 2 * N;
        h->ip.q = v + 3 * N;
        h->ip.comp = at<int>(ws, L.comp);
        h->ip.isl_w = at<double>(ws, L.isl);
        h->ip.isl_acc = h->ip.isl_w + kMaxIslands;
    }
    h->ctl = at<DevCtl>(ws, L.ctl);
    h->blockred = at<double>(ws, L.blockred);
    for (int q = 0; q < 3; ++q) h->psi[q] = at<float2>(ws, L.psi[q]);
    h->cur = 0;
    h->b = at<float2>(ws, L.b);
    h->D = at<float2>(ws, L.D);
    h->mu_buf[0] = at<float>(ws, L.mu);
    h->mu_buf[1] = at<float>(ws, L.mu2);
    h->mu_q = 0;
    h->mu = h->mu_buf[0];
    h->f = at<float>(ws, L.f);
    h->links = g.L ? at<float2>(ws, L.links) : nullptr;
    h->nblockred = L.nblockred;
    // Jacobi sweep kernel: 1 register-tiled; 2 or 0 (default) staged in shared memory by the
    // tensor memory accelerator where it applies (Landau links of either plane, even nx),
    // measured faster at every size tried; the register-tiled kernel elsewhere
    h->poisson_only = pon ? 1 : 0;
    h->use_tma = (!pon && c.sweep_kernel != 1 && tma_sweep_supported(g)) ? 1 : 0;
    if (h->use_tma && !tma_encode_maps(g, h->psi, h->b, h->D, &h->tmaps)) h->use_tma = 0;
    h->batch_owned = 0;
    {
        // h_t zeta_max, zeta_max = (T_zeta / (h_t hx hy hz))^(1/2) (Sec. 3.1.2); a film drops hz
        const double vol = c.hx * c.hy * (c.nz >= 2 ? c.hz : 1.0);
        h->noise_amp = c.noise_T > 0 ? (float)(c.ht * sqrt(c.noise_T / (c.ht * vol))) : 0.f;
    }
    h->last_sweeps = 8;
    h->last_cycles = c.poisson_cycles;
    h->step = 0;
    h->dtK = c.u * c.ht;
    h->wsum = 1.0;
    for (int a = 0; a < 3; ++a) {
        int n = (a == 0) ? c.nx : (a == 1 ? c.ny : c.nz);
        h->wsum *= (c.bc[a] == TDGL_OPEN && n >= 2) ? (double)(n - 1) : (double)n;
    }

    // link tables in FP64 (Eq. link_variables with A~ of Eq. A_yz), wrap phase of Sec. 3.3.1
    const double Lx = box_len(c.nx, c.hx, c.bc[0]);
    std::vector<float2> Uy(c.nx), Uz(c.nx), Py(c.ny), Pz(c.nz);
    for (int i = 0; i < c.nx; ++i) {
        double xbar = i * c.hx - 0.5 * Lx;
        double ay = fmod(-c.hy * c.Bz * xbar, kTwoPi), az = fmod(c.hz * c.By * xbar, kTwoPi);
        Uy[i] = make_float2((float)cos(ay), (float)sin(ay));
        Uz[i] = make_float2((float)cos(az), (float)sin(az));
    }
    // P_{j,k} = exp(i(-j hy Lx Bz + k hz Lx By)) = Py[j] Pz[k]
    long long nzq = 0, nyq = 0;
    bool qy = c.bc[1] == TDGL_PERIODIC && quantised(c.Bz, Lx, box_len(c.ny, c.hy, c.bc[1]), &nzq);
    bool qz = c.bc[2] == TDGL_PERIODIC && quantised(c.By, Lx, box_len(c.nz, c.hz, c.bc[2]), &nyq);
    for (int j = 0; j < c.ny; ++j) {
        double ph;
        if (qy) {
            long long r = ((nzq * j) % c.ny + c.ny) % c.ny;       // j hy Lx Bz = 2 pi nz j / Ny
            ph = -kTwoPi * (double)r / (double)c.ny;
        } else {
            ph = -fmod(j * c.hy * Lx * c.Bz, kTwoPi);
        }
        Py[j] = make_float2((float)cos(ph), (float)sin(ph));
    }
    for (int k = 0; k < c.nz; ++k) {
        double ph;
        if (qz) {
            long long r = ((nyq * k) % c.nz + c.nz) % c.nz;
            ph = kTwoPi * (double)r / (double)c.nz;
        } else {
            ph = fmod(k * c.hz * Lx * c.By, kTwoPi);
        }
        Pz[k] = make_float2((float)cos(ph), (float)sin(ph));
    }
    cudaStream_t s = h->stream;
    int rc = TDGL_OK;
    auto chk = [&](cudaError_t e) {
        if (e != cudaSuccess && rc == TDGL_OK) rc = TDGL_ERR_CUDA;
    };
    chk(cudaMemcpyAsync((void *)g.Uy, Uy.data(), 8 * c.nx, cudaMemcpyHostToDevice, s));
    chk(cudaMemcpyAsync((void *)g.Uz, Uz.data(), 8 * c.nx, cudaMemcpyHostToDevice, s));
    chk(cudaMemcpyAsync((void *)g.Py, Py.data(), 8 * c.ny, cudaMemcpyHostToDevice, s));
    chk(cudaMemcpyAsync((void *)g.Pz, Pz.data(), 8 * c.nz, cudaMemcpyHostToDevice, s));
    std::vector<float2> xzt;
    if (c.links_mode == TDGL_LINKS_GENERAL) {
        long long n3 = 3 * N;
        int nb = (int)((n3 + 255) / 256 < 8192 ? (n3 + 255) / 256 : 8192);
        phases_to_links<<<nb, 256, 0, s>>>(c.d_link_phase, h->links, n3);
        chk(cudaGetLastError());
    } else if (c.links_mode == TDGL_LINKS_XZ) {
        // Eq. A_xz: U_x(j) = exp(i hx Bz ybar_j) (K is applied by the kernels), U_y = 1 inside
        // the box, U_z(j) = exp(-i hz Bx ybar_j); FP64 phases, whole flux quanta reduced exactly
        const double Ly = box_len(c.ny, c.hy, c.bc[1]), Lz = box_len(c.nz, c.hz, c.bc[2]);
        xzt.resize(2 * (size_t)c.ny + c.nx + c.nz);
        float2 *X = xzt.data(), *Z = X + c.ny, *Wx = Z + c.ny, *Wz = Wx + c.nx;
        auto e = [](double ph) { return make_float2((float)cos(ph), (float)sin(ph)); };
        for (int j = 0; j < c.ny; ++j) {
            double ybar = j * c.hy - 0.5 * Ly;
            X[j] = e(fmod(c.hx * c.Bz * ybar, kTwoPi));
            Z[j] = e(fmod(-c.hz * c.Bx * ybar, kTwoPi));
        }
        long long nzq = 0, nxq = 0;
        bool qx = c.bc[0] == TDGL_PERIODIC && quantised(c.Bz, Lx, Ly, &nzq);
        bool qz = c.bc[2] == TDGL_PERIODIC && quantised(c.Bx, Ly, Lz, &nxq);
        for (int i = 0; i < c.nx; ++i) {   // -i hx Ly Bz; periodic x: = -2 pi nz i / Nx
            double ph = qx ? -kTwoPi * (double)(((nzq * i) % c.nx + c.nx) % c.nx) / (double)c.nx
                           : -fmod(i * c.hx * Ly * c.Bz, kTwoPi);
            Wx[i] = e(ph);
        }
        for (int k = 0; k < c.nz; ++k) {   // +k hz Ly Bx; periodic z: = 2 pi nx k / Nz
            double ph = qz ? kTwoPi * (double)(((nxq * k) % c.nz + c.nz) % c.nz) / (double)c.nz
                           : fmod(k * c.hz * Ly * c.Bx, kTwoPi);
            Wz[k] = e(ph);
        }
        float2 *dt = at<float2>(ws, L.xzt);
        chk(cudaMemcpyAsync((void *)dt, xzt.data(), 8 * xzt.size(), cudaMemcpyHostToDevice, s));
        int nb = (int)((N + 255) / 256 < 8192 ? (N + 255) / 256 : 8192);
        xz_links<<<nb, 256, 0, s>>>(dt, h->links, c.nx, c.ny, c.nz, c.bc[1] == TDGL_PERIODIC);
        chk(cudaGetLastError());
    }
    DevCtl ctl0;
    memset(&ctl0, 0, sizeof(ctl0));
    ctl0.Ux = make_float2(1.f, 0.f);
    chk(cudaMemcpyAsync(h->ctl, &ctl0, sizeof(DevCtl), cudaMemcpyHostToDevice, s));
    if (!pon) chk(cudaMemsetAsync(h->psi[0], 0, 8 * (size_t)N, s));
    chk(cudaMemsetAsync(h->mu, 0, 4 * (size_t)N, s));
    if (h->mu_buf[1]) chk(cudaMemsetAsync(h->mu_buf[1], 0, 4 * (size_t)N, s));
    chk(cudaMemsetAsync(h->f, 0, 4 * (size_t)N, s));
    if (c.d_insulating && rc == TDGL_OK) {
        // link bits and conducting components; current injected through the x faces needs
        // the largest component on both faces
        chk(launch_link_bits(g, c.d_insulating, h->lk, s));
        if (rc == TDGL_OK) {
            int r2 = build_components(g, h->ip, h->ctl, h->blockred, s);
            if (r2 != TDGL_OK) rc = r2;
            else if (!(h->ip.wsum_c > 0) || (c.bc[0] == TDGL_OPEN && (h->ip.n_face0 < 1 || h->ip.n_face1 < 1)))
                rc = TDGL_ERR_INVALID_ARG;
        }
    }

    // multigrid
    PoissonArgs &pa = h->pa;
    memset(&pa, 0, sizeof(pa));
    pa.g = g;
    pa.ctl = h->ctl;
    pa.blockred = h->blockred;
    pa.nlevels = L.nlevels;
    pa.f = h->f;
    pa.mu = h->mu;
    pa.hx = c.hx;
    pa.Jext = c.Jext;
    pa.inject = (c.bc[0] == TDGL_OPEN && c.Jext != 0.0) ? 1 : 0;
    pa.wsum = h->wsum;
    std::vector<float> tri;
    double hy = c.hy, hz = c.hz;
    for (int l = 0; l < L.nlevels; ++l) {
        MGLevel &M = pa.lev[l];
        M.nx = c.nx;
        M.ny = L.ny[l];
        M.nz = L.nz[l];
        M.N = (long long)c.nx * M.ny * M.nz;
        M.fy = L.fy[l];
        M.fz = L.fz[l];
        M.cx = g.cx;
        M.cy = (float)(1.0 / (hy * hy));
        M.cz = active(M.nz) ? (float)(1.0 / (c.g * c.g * hz * hz)) : 0.f;
        M.u = (l == 0) ? h->mu : at<float>(ws, L.u[l]);
        M.r = (l == 0) ? h->f : at<float>(ws, L.r[l]);
        M.t = at<float>(ws, L.t);
        M.G = at<float>(ws, L.tri[l]);
        M.P = mg_period(c.nx, c.bc[0]);
        M.kmin = mg_line_kernel(c.nx, c.bc[0], M.cx, 2.0 * M.cy + 2.0 * M.cz, tri);
        {
            // the line operator (2 cx + s) - cx (shift + shift^-1) = (cx / rho)(1 - rho S-)(1 - rho S+):
            // a causal and an anticausal first-order recursion.  With 16 sites per lane: each
            // lane starts them 12 values before (after) its chunk where rho^12 <= 1e-8 (the
            // dropped terms fall below FP32 rounding), else the exact scan over the lanes
            // (iir_w = 0).  With 32 sites per lane: a 32-value warm-up where rho^32 <= 1e-9.
            const double sx = 2.0 * M.cy + 2.0 * M.cz, tt = 1.0 + sx / (2.0 * M.cx);
            const double rho = tt - sqrt(tt * tt - 1.0);
            M.rho = (float)rho;
            M.rscale = (float)(rho / M.cx);
            const int C = c.nx / 32;
            const bool shape = (C == 16 || C == 32) && c.nx == 32 * C && sx > 0;
            M.iir = 0;
            M.iir_w = 0;
            if (shape && C == 16 && rho <= 0.999) {
                // (rho closer to 1, a line barely coupled in y and z, keeps the convolution:
                // the scan's seeds would divide by 1 - rho^P near cancellation)
                M.iir = 16;
                M.iir_w = (pow(rho, 12.0) <= 1e-8) ? 12 : 0;
            } else if (shape && pow(rho, 32.0) <= 1e-9) {
                M.iir = 32;
                M.iir_w = 32;
            }
            const int P = (c.bc[0] == TDGL_OPEN) ? 2 * c.nx - 2 : c.nx;
            for (int q = 0; q < 5; ++q) M.rhoC[q] = (float)pow(rho, (double)C * (1 << q));
            M.l2rho = (float)log2(rho);
            M.gf = (float)(1.0 / (1.0 - pow(rho, (double)P)));
            M.gb = (float)(1.0 / (1.0 - rho * rho));
        }
        M.kmax = M.kmin + (int)tri.size() - 1;
        chk(cudaMemcpyAsync(M.G, tri.data(), 4 * tri.size(), cudaMemcpyHostToDevice, s));
        M.cw = nullptr;
        M.M = M.ny * M.nz;
        std::vector<float> cwh;
        if (l == L.nlevels - 1 && L.cw) {
            cwh.resize(mg_coarse_floats(c.nx, c.bc[0], M.M));
            if (mg_coarse_factors(c.nx, c.bc[0], M.cx, M.ny, M.nz, c.bc[1], c.bc[2], M.cy, M.nz >= 2 ? M.cz : 0.0,
                                  cwh.data())) {
                M.cw = at<float>(ws, L.cw);
                chk(cudaMemcpyAsync(M.cw, cwh.data(), 4 * cwh.size(), cudaMemcpyHostToDevice, s));
            }
        }
        if (M.fy == 2) hy *= 2.0;
        if (M.fz == 2) hz *= 2.0;
        // a synchronous wait keeps `tri` valid for the copy above
        chk(cudaStreamSynchronize(s));
    }
    // tensor maps for the recursive smoother's row staging (none: per-lane copies), for
    // each of the two mu buffers that the finest level can solve in
    if (h->lk) {
        // and of z, in which the masked solve's preconditioning V-cycle smooths
        pa.lev[0].u = h->ip.z;
        mg_encode_line_maps(pa);
        h->ip.zmap = pa.umap[0];
        h->ip.zmap_u = pa.umap_u[0];
    }
    for (int q = 1; q >= 0; --q) {
        if (!h->mu_buf[q]) continue;
        pa.lev[0].u = pa.mu = h->mu_buf[q];
        mg_encode_line_maps(pa);
        h->umap0[q] = pa.umap[0];
        h->umap0_u[q] = pa.umap_u[0];
    }
    // with the staged sweep, the init's tile is staged too (asynchronous copies) where it applies
    if (h->use_tma && init_staged_supported(g)) chk(init_staged_setup());
    chk(cudaStreamSynchronize(s));
    if (rc != TDGL_OK) {
        delete h;
        return rc;
    }
    *out = h;
    return TDGL_OK;
}

void tdgl_destroy(tdgl_handle *h)
{
    if (!h) return;
    if (h->res_pending) resident_sync(h);   // the enqueued steps finish before the handle goes
    drop_poisson_graphs(h);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->ev_made)
        for (int i = 0; i < tdgl_handle::kEvents; ++i) cudaEventDestroy(h->ev[i]);
    delete h;
}

int tdgl_profile_enable(tdgl_handle *h, int on)
{
    if (h && h->res_pending) {   // resident steps enqueued: finish and account for them first
        const int rs = resident_sync(h);
        if (rs != TDGL_OK) return rs;
    }
    if (!h) return TDGL_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return TDGL_ERR_CUDA;
    if (on && !h->ev_made) {
        for (int i = 0; i < tdgl_handle::kEvents; ++i)
            if (cudaEventCreate(&h->ev[i]) != cudaSuccess) return TDGL_ERR_CUDA;
        h->ev_made = true;
    }
    h->prof_on = on ? 1 : 0;
    h->pend_K = h->pend_P = h->pend_R = false;
    memset(&h->prof, 0, sizeof(h->prof));
    return TDGL_OK;
}

int tdgl_test_staged_waits(tdgl_handle *h, int64_t wait_ns, int32_t extra_tx_bytes)
{
    if (h && h->res_pending) {   // resident steps enqueued: finish and account for them first
        const int rs = resident_sync(h);
        if (rs != TDGL_OK) return rs;
    }
    if (!h || wait_ns < 0 || wait_ns > 2000000000LL || extra_tx_bytes < 0 || extra_tx_bytes > 65536)
        return TDGL_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return TDGL_ERR_CUDA;
    h->dbg_wait_ns = (unsigned long long)wait_ns;
    h->dbg_extra_tx = (unsigned int)extra_tx_bytes;
    h->pa.wait_ns = h->dbg_wait_ns;
    h->pa.extra_tx = h->dbg_extra_tx;
    // the captured Poisson graphs hold the old kernel arguments: capture again on the next solve
    drop_poisson_graphs(h);
    return TDGL_OK;
}

int tdgl_profile_read(tdgl_handle *h, tdgl_profile *out)
{
    if (h && h->res_pending) {   // resident steps enqueued: finish and account for them first
        const int rs = resident_sync(h);
        if (rs != TDGL_OK) return rs;
    }
    if (!h || !out) return TDGL_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return TDGL_ERR_CUDA;
    ev_collect(h);
    *out = h->prof;
    return TDGL_OK;
}

int tdgl_set_state(tdgl_handle *h, const float *d_psi, const float *d_mu, double K)
{
    if (h && h->res_pending) {   // resident steps enqueued: finish and account for them first
        const int rs = resident_sync(h);
        if (rs != TDGL_OK) return rs;
    }
    if (!h || !d_psi) return TDGL_ERR_INVALID_ARG;
    if (h->poisson_only) return TDGL_ERR_INVALID_ARG;
    const size_t N = (size_t)h->g.N;
    cudaStream_t s = h->stream;
    if (cudaMemcpyAsync(h->psi[h->cur], d_psi, 8 * N, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return TDGL_ERR_CUDA;
    cudaError_t e = d_mu ? cudaMemcpyAsync(h->mu, d_mu, 4 * N, cudaMemcpyDeviceToDevice, s)
                         : cudaMemsetAsync(h->mu, 0, 4 * N, s);
    if (e != cudaSuccess) return TDGL_ERR_CUDA;
    DevCtl c;
    memset(&c, 0, sizeof(c));
    c.K = K;
    c.Ux = make_float2((float)cos(h->cfg.hx * K), (float)sin(h->cfg.hx * K));
    if (cudaMemcpyAsync(h->ctl, &c, sizeof(DevCtl), cudaMemcpyHostToDevice, s) != cudaSuccess) return TDGL_ERR_CUDA;
    if (launch_set_Ux(h->ctl, h->cfg.hx, s) != cudaSuccess) return TDGL_ERR_CUDA;
    h->mu_solved = 0;   // f no longer belongs to mu
    h->prev_valid = 0;  // no mu of an earlier step to extrapolate from
    h->guess_ready = 0;
    h->mu_pend[0] = h->mu_pend[1] = 0;   // the control block (and its pending means) was cleared
    return cuda_err(cudaStreamSynchronize(s));
}

int tdgl_upload_state(tdgl_handle *h, const float *host_psi, const float *host_mu, double K)
{
    if (h && h->res_pending) {   // resident steps enqueued: finish and account for them first
        const int rs = resident_sync(h);
        if (rs != TDGL_OK) return rs;
    }
    if (!h || !host_psi) return TDGL_ERR_INVALID_ARG;
    if (h->poisson_only) return TDGL_ERR_INVALID_ARG;
    const size_t N = (size_t)h->g.N;
    cudaStream_t s = h->stream;
    if (cudaMemcpyAsync(h->psi[h->cur], host_psi, 8 * N, cudaMemcpyHostToDevice, s) != cudaSuccess) return TDGL_ERR_CUDA;
    cudaError_t e = host_mu ? cudaMemcpyAsync(h->mu, host_mu, 4 * N, cudaMemcpyHostToDevice, s)
                            : cudaMemsetAsync(h->mu, 0, 4 * N, s);
    if (e != cudaSuccess) return TDGL_ERR_CUDA;
    DevCtl c;
    memset(&c, 0, sizeof(c));
    c.K = K;
    if (cudaMemcpyAsync(h->ctl, &c, sizeof(DevCtl), cudaMemcpyHostToDevice, s) != cudaSuccess) return TDGL_ERR_CUDA;
    if (launch_set_Ux(h->ctl, h->cfg.hx, s) != cudaSuccess) return TDGL_ERR_CUDA;
    h->mu_solved = 0;   // f no longer belongs to mu
    h->prev_valid = 0;  // no mu of an earlier step to extrapolate from
    h->guess_ready = 0;
    h->mu_pend[0] = h->mu_pend[1] = 0;   // the control block (and its pending means) was cleared
    return cuda_err(cudaStreamSynchronize(s));
}

int tdgl_get_mu_prev(tdgl_handle *h, float *out, int32_t out_on_host)
{
    if (h && h->res_pending) {   // resident steps enqueued: finish and account for them first
        const int rs = resident_sync(h);
        if (rs != TDGL_OK) return rs;
    }
    if (!h || !out) return TDGL_ERR_INVALID_ARG;
    if (!extrapolating(h) || !h->prev_valid) return 0;
    cudaStream_t s = h->stream;
    const size_t N = (size_t)h->g.N;
    if (mu_materialize(h, 1 - h->mu_q) != TDGL_OK) return TDGL_ERR_CUDA;
    if (cudaMemcpyAsync(out, h->mu_buf[1 - h->mu_q], 4 * N, out_on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                        s) != cudaSuccess)
        return TDGL_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return TDGL_ERR_CUDA;
    return 1;
}

int tdgl_set_mu_prev(tdgl_handle *h, const float *in, int32_t in_on_host)
{
    if (h && h->res_pending) {   // resident steps enqueued: finish and account for them first
        const int rs = resident_sync(h);
        if (rs != TDGL_OK) return rs;
    }
    if (!h) return TDGL_ERR_INVALID_ARG;
    h->guess_ready = 0;
    if (!in) {
        h->prev_valid = 0;
        return TDGL_OK;
    }
    if (!extrapolating(h)) return TDGL_ERR_INVALID_ARG;
    cudaStream_t s = h->stream;
    const size_t N = (size_t)h->g.N;
    if (cudaMemcpyAsync(h->mu_buf[1 - h->mu_q], in, 4 * N, in_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                        s) != cudaSuccess)
        return TDGL_ERR_CUDA;
    if (cudaMemsetAsync(&h->ctl->mu_off[1 - h->mu_q], 0, sizeof(double), s) != cudaSuccess) return TDGL_ERR_CUDA;
    h->mu_pend[1 - h->mu_q] = 0;
    if (cudaStreamSynchronize(s) != cudaSuccess) return TDGL_ERR_CUDA;
    h->prev_valid = 1;
    return TDGL_OK;
}

int tdgl_set_step(tdgl_handle *h, int64_t step)
{
    if (h && h->res_pending) {   // resident steps enqueued: finish and account for them first
        const int rs = resident_sync(h);
        if (rs != TDGL_OK) return rs;
    }
    if (!h || step < 0) return TDGL_ERR_INVALID_ARG;
    cudaStream_t s = h->stream;
    const unsigned long long n = (unsigned long long)step;
    if (cudaMemcpyAsync(&h->ctl->nstep, &n, sizeof(n), cudaMemcpyHostToDevice, s) != cudaSuccess) return TDGL_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return TDGL_ERR_CUDA;
    h->step = step;
    return TDGL_OK;
}

int tdgl_download_state(tdgl_handle *h, float *host_psi, float *host_mu, double *K)
{
    if (h && h->res_pending) {   // resident steps enqueued: finish and account for them first
        const int rs = resident_sync(h);
        if (rs != TDGL_OK) return rs;
    }
    if (!h || (h->poisson_only && host_psi)) return TDGL_ERR_INVALID_ARG;
    const size_t N = (size_t)h->g.N;
    cudaStream_t s = h->stream;
    if (mu_materialize(h, h->mu_q) != TDGL_OK) return TDGL_ERR_CUDA;
    if (host_psi && cudaMemcpyAsync(host_psi, h->psi[h->cur], 8 * N, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return TDGL_ERR_CUDA;
    if (host_mu && cudaMemcpyAsync(host_mu, h->mu, 4 * N, cudaMemcpyDeviceToHost, s) != cudaSuccess) return TDGL_ERR_CUDA;
    DevCtl c;
    int rc = read_ctl(h, &c);
    if (rc != TDGL_OK) return rc;
    if (K) *K = c.K;
    return TDGL_OK;
}

int tdgl_get_state(tdgl_handle *h, tdgl_state_ptrs *out)
{
    if (h && h->res_pending) {   // resident steps enqueued: finish and account for them first
        const int rs = resident_sync(h);
        if (rs != TDGL_OK) return rs;
    }
    if (!h || !out) return TDGL_ERR_INVALID_ARG;
    if (mu_materialize(h, h->mu_q) != TDGL_OK) return TDGL_ERR_CUDA;
    out->psi = reinterpret_cast<float *>(h->psi[h->cur]);
    out->mu = h->mu;
    out->b = reinterpret_cast<float *>(h->b);
    out->D = reinterpret_cast<float *>(h->D);
    out->f = h->f;
    return TDGL_OK;
}

int tdgl_solve_psi(tdgl_handle *h, int32_t *sweeps_out)
{
    if (h && h->res_pending) {   // resident steps enqueued: finish and account for them first
        const int rs = resident_sync(h);
        if (rs != TDGL_OK) return rs;
    }
    if (!h || h->batch_owned || h->slab || h->poisson_only) return TDGL_ERR_INVALID_ARG;
    const tdgl_config &c = h->cfg;
    cudaStream_t s = h->stream;
    SweepArgs a = sweep_args(h);
    const int ia = (h->cur + 1) % 3, ib = (h->cur + 2) % 3;
    // two sweeps per pass over memory on request, where the grid allows (same results)
    const bool pairs = c.sweeps_per_pass == 2 && pair_supported(h->g);
    a.src = h->psi[h->cur];
    a.dst = h->psi[ia];
    a.dst_index = ia;
    a.mu_off = &h->ctl->mu_off[h->mu_q];   // the pending projection of mu
    if (extrapolating(h)) {
        guess_args(h, a, h->mu_q, h->prev_valid != 0);
        h->guess_ready = 1;
        h->mu_pend[1 - h->mu_q] = 0;   // the guess over the previous mu carries no pending mean
    }
    ev_rec(h, 0);
    if (launch_init_sweep(a, s, h->use_tma != 0) != cudaSuccess) return TDGL_ERR_CUDA;
    a.mu_guess = nullptr;
    a.mu_off = a.mu_off_prev = nullptr;
    ev_rec(h, 1);
    h->prof.kernel_launches += 1;
    int launched = 1;   // sweeps enqueued (the init fuses the first)
    bool first_sync = true;
    auto collect = [&]() {
        if (!h->prof_on) return;
        if (first_sync) h->prof.ms_init += ev_ms(h, 0, 1);
        first_sync = false;
        h->prof.ms_sweeps += ev_ms(h, 2, 3);
    };
    // enqueue at least n more sweeps
    auto enqueue = [&](int n) -> int {
        ev_rec(h, 2);
        int launches = 0;
        for (int q = 0; q < n;) {
            if (pairs) {
                // pass p covers sweeps 2p and 2p+1: p odd reads A and writes B, p even the reverse
                const int p = (launched + 1) / 2;
                a.src = (p & 1) ? h->psi[ia] : h->psi[ib];
                a.dst = (p & 1) ? h->psi[ib] : h->psi[ia];
                a.dst_index = (p & 1) ? ib : ia;
                if (launch_sweep_pair(a, s) != cudaSuccess) return TDGL_ERR_CUDA;
                launched += 2;
                q += 2;
            } else {
                // sweep number `launched` (1-based count of sweeps before it) reads the
                // output of the previous one: odd -> A to B, even -> B to A
                const bool odd = (launched % 2) == 1;
                a.src = odd ? h->psi[ia] : h->psi[ib];
                a.dst = odd ? h->psi[ib] : h->psi[ia];
                a.dst_index = odd ? ib : ia;
                cudaError_t e;
                if (h->use_tma) {
                    int src = 0;
                    while (src < 2 && h->psi[src] != a.src) ++src;
                    e = launch_sweep_tma(a, h->tmaps.psi[src], h->tmaps, s);
                } else {
                    e = launch_sweep(a, s);
                }
                if (e != cudaSuccess) return TDGL_ERR_CUDA;
                ++launched;
                ++q;
            }
            ++launches;
        }
        h->prof.sweep_launches += launches;
        h->prof.kernel_launches += launches;
        ev_rec(h, 3);
        return TDGL_OK;
    };
    DevCtl ctl;
    if (c.fixed_sweeps > 0) {
        int rc = enqueue(c.fixed_sweeps - 1);
        if (rc != TDGL_OK) return rc;
        rc = read_ctl(h, &ctl);
        if (rc != TDGL_OK) return rc;
        collect();
    } else {
        int batch = h->last_sweeps;
        for (;;) {
            int n = batch - launched;
            if (n < 1) n = 1;
            if (launched + n > c.max_iter) n = c.max_iter - launched;
            if (n > 0) {
                int rc = enqueue(n);
                if (rc != TDGL_OK) return rc;
            } else {
                ev_rec(h, 2);
                ev_rec(h, 3);
            }
            int rc = read_ctl(h, &ctl);
            if (rc != TDGL_OK) return rc;
            collect();
            if (ctl.done || launched >= c.max_iter) break;
            batch = launched + 4;
        }
    }
    if (ctl.status != TDGL_OK || !ctl.done) {
        // the init has written the Poisson guess over the previous mu: a retry starts afresh
        if (extrapolating(h)) h->prev_valid = h->guess_ready = 0;
        return ctl.status != TDGL_OK ? ctl.status : TDGL_ERR_NOT_CONVERGED;
    }
    if (ctl.redo) {
        // the first sweep of the deciding pass is the result: recompute it from
        // the pass's input into the pass's output buffer
        const int p = ctl.iter / 2;
        a.src = (p & 1) ? h->psi[ia] : h->psi[ib];
        a.dst = (p & 1) ? h->psi[ib] : h->psi[ia];
        a.dst_index = (p & 1) ? ib : ia;
        if (h->prof_on) cudaEventRecord(h->ev[8], s);
        if (launch_sweep_redo(a, s) != cudaSuccess) return TDGL_ERR_CUDA;
        if (h->prof_on) cudaEventRecord(h->ev[9], s);
        h->pend_R = h->prof_on;
        h->prof.sweep_launches += 1;
        h->prof.kernel_launches += 1;
    }
    h->cur = ctl.result;
    h->last_sweeps = ctl.iter;
    h->prof.sweeps += ctl.iter;
    if (sweeps_out) *sweeps_out = ctl.iter;
    return TDGL_OK;
}

// The fixed launch sequence of a plain Poisson solve (poisson_tol == 0): right-hand side,
// poisson_cycles V-cycles, projection.  Returns the launches enqueued.
static cudaError_t poisson_rhs(tdgl_handle *h, cudaStream_t s)
{
    if (h->use_tma) return launch_poisson_rhs_tma(h->pa, h->psi[h->cur], h->tmaps.psi[h->cur], h->tmaps, s);
    return launch_poisson_rhs(h->pa, h->psi[h->cur], s);
}

static bool lazy_projection(const tdgl_handle *h, bool fm)
{
    return fm && !h->lk && !h->batch_owned && !h->in_adjoint;
}

static long long poisson_sequence(tdgl_handle *h, cudaStream_t s, cudaError_t *err)
{
    long long nl = 1;
    const int nc = h->cfg.poisson_cycles;
    const bool fm = nc > 0 && vcycle_mean_fusable(h->pa);   // the last cycle leaves the mean of mu
    cudaError_t e = poisson_rhs(h, s);
    for (int q = 0; q < nc && e == cudaSuccess; ++q) e = launch_vcycle(h->pa, s, &nl, q > 0, fm && q == nc - 1);
    // with the mean summed by the cycle, the projection is left pending (applied where mu is read)
    if (e == cudaSuccess) e = lazy_projection(h, fm) ? launch_commit_mean(h->pa, s) : launch_project_mu(h->pa, s, fm);
    *err = e;
    return nl + (fm ? 1 : 2);
}

// Capture the sequence for the current psi buffer (false: graphs are not used).
static bool build_poisson_graph(tdgl_handle *h)
{
    if (!h->cap_stream && cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        h->cap_stream = nullptr;
        return false;
    }
    if (cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return false;
    cudaError_t e;
    const long long nl = poisson_sequence(h, h->cap_stream, &e);
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(h->cap_stream, &graph);
    if (e != cudaSuccess || ee != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return false;
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    h->pgraph[h->cur + 3 * h->mu_q] = exec;
    h->pgraph_launches = nl;
    return true;
}

int tdgl_solve_mu(tdgl_handle *h)
{
    if (h && h->res_pending) {   // resident steps enqueued: finish and account for them first
        const int rs = resident_sync(h);
        if (rs != TDGL_OK) return rs;
    }
    if (!h || h->batch_owned || h->slab || h->poisson_only) return TDGL_ERR_INVALID_ARG;
    const tdgl_config &c = h->cfg;
    cudaStream_t s = h->stream;
    h->mu_solved = 1;
    if (extrapolating(h) && h->guess_ready) {
        // the step's init wrote the guess over the other mu buffer: solve there; the old
        // state becomes the previous mu of the next extrapolation.  (A solve that no init
        // prepared -- repeated solves of one right-hand side -- starts from the current mu
        // in place: on a fixed right-hand side the extrapolation of two iterates would
        // converge more slowly than the plain restart.)
        use_mu_buffer(h, 1 - h->mu_q);
        h->prev_valid = 1;
    }
    h->guess_ready = 0;
    // plain solve from the second call on: replay a captured graph (the first call runs the
    // launches directly, which also sets the kernels' one-time attributes outside a capture)
    const int gk = h->cur + 3 * h->mu_q;
    if (!h->lk && c.poisson_tol <= 0 && !h->pgraph_fail && h->poisson_calls++ >= 1) {
        if (!h->pgraph[gk] && !build_poisson_graph(h)) h->pgraph_fail = 1;
        if (h->pgraph[gk]) {
            if (cudaGraphLaunch(h->pgraph[gk], s) != cudaSuccess) return TDGL_ERR_CUDA;
            h->mu_pend[h->mu_q] = lazy_projection(h, vcycle_mean_fusable(h->pa) && c.poisson_cycles > 0) ? 1 : 0;
            h->last_cycles = c.poisson_cycles;
            h->prof.vcycles += c.poisson_cycles;
            h->prof.kernel_launches += h->pgraph_launches;
            return TDGL_OK;
        }
    }
    if (poisson_rhs(h, s) != cudaSuccess) return TDGL_ERR_CUDA;
    if (h->lk) {
        // removed links: CG iterations preconditioned by V-cycles; poisson_cycles of them, or
        // (poisson_tol > 0) until max|F - Lap mu| <= poisson_tol max|F|, at most poisson_max_cycles
        long long nl = 1;
        int it = 0;
        int rc = masked_poisson_solve(h->pa, h->ip, c.poisson_tol, c.poisson_tol > 0 ? 0 : c.poisson_cycles,
                                      c.poisson_max_cycles, s, &it, &nl);
        h->last_cycles = it;
        h->prof.vcycles += it + 1;
        h->prof.kernel_launches += nl;
        return rc;
    }
    long long nl = 1;
    int cycles = 0;
    // a fixed number of cycles: the last one leaves the mean of mu
    const bool fm = c.poisson_tol <= 0 && c.poisson_cycles > 0 && vcycle_mean_fusable(h->pa);
    for (int q = 0; q < c.poisson_cycles; ++q, ++cycles)
        if (launch_vcycle(h->pa, s, &nl, q > 0, fm && q == c.poisson_cycles - 1) != cudaSuccess) return TDGL_ERR_CUDA;
    if (c.poisson_tol > 0) {
        for (;;) {
            if (launch_poisson_residual(h->pa, s) != cudaSuccess) return TDGL_ERR_CUDA;
            ++nl;
            DevCtl ctl;
            int rc = read_ctl(h, &ctl);
            if (rc != TDGL_OK) return rc;
            if (ctl.res <= c.poisson_tol || cycles >= c.poisson_max_cycles) break;
            if (launch_vcycle(h->pa, s, &nl, true) != cudaSuccess) return TDGL_ERR_CUDA;
            ++cycles;
        }
    }
    if ((lazy_projection(h, fm) ? launch_commit_mean(h->pa, s) : launch_project_mu(h->pa, s, fm)) != cudaSuccess)
        return TDGL_ERR_CUDA;
    h->mu_pend[h->mu_q] = lazy_projection(h, fm) ? 1 : 0;
    nl += fm ? 1 : 2;
    h->last_cycles = cycles;
    h->prof.vcycles += cycles;
    h->prof.kernel_launches += nl;
    return TDGL_OK;
}

// ---------------------------------------------------------------------------------
// z-slab decomposition: a handle for the planes z0 .. z0 + nz_local - 1 of a grid
// periodic in z, with one halo plane on each side; sweeps one at a time, the
// convergence decision and the halo exchange left to the caller.
// ---------------------------------------------------------------------------------
static int slab_config(const tdgl_config *gcfg, int32_t z0, int32_t nz_local, tdgl_config *lc)
{
    if (!gcfg || validate(gcfg) != TDGL_OK) return TDGL_ERR_INVALID_ARG;
    const tdgl_config &c = *gcfg;
    if (c.bc[2] != TDGL_PERIODIC || c.nz < 3 || c.bc[0] != TDGL_OPEN || c.links_mode != TDGL_LINKS_LANDAU ||
        (c.nx % 2) != 0 || c.d_insulating || c.noise_T != 0.0 || c.sweeps_per_pass == 2 || c.fixed_sweeps > 0 ||
        c.check_every != 1)
        return TDGL_ERR_INVALID_ARG;
    if (nz_local < 1 || z0 < 0 || (long long)z0 + nz_local > c.nz) return TDGL_ERR_INVALID_ARG;
    *lc = c;
    lc->nz = nz_local + 2;
    return validate(lc);
}

size_t tdgl_slab_workspace_bytes(const tdgl_config *global_cfg, int32_t z0, int32_t nz_local)
{
    tdgl_config lc;
    if (slab_config(global_cfg, z0, nz_local, &lc) != TDGL_OK) return 0;
    return layout(&lc).total;
}

int tdgl_slab_create(const tdgl_config *global_cfg, int32_t z0, int32_t nz_local, void *d_workspace, size_t ws_bytes,
                     void *stream, tdgl_handle **out)
{
    tdgl_config lc;
    int rc = slab_config(global_cfg, z0, nz_local, &lc);
    if (rc != TDGL_OK) return rc;
    rc = create_impl(&lc, d_workspace, ws_bytes, stream, out, false);
    if (rc != TDGL_OK) return rc;
    tdgl_handle *h = *out;
    h->slab = 1;
    h->slab_z0 = z0;
    h->slab_nz = nz_local;
    h->g.kw0 = h->pa.g.kw0 = 1;
    h->g.kw1 = h->pa.g.kw1 = nz_local + 1;
    return TDGL_OK;
}

int tdgl_slab_sweep(tdgl_handle *h, int32_t first, double *r2_local)
{
    if (!h || !h->slab) return TDGL_ERR_INVALID_ARG;
    if (!first && h->slab_n < 1) return TDGL_ERR_INVALID_ARG;
    cudaStream_t s = h->stream;
    SweepArgs a = sweep_args(h);
    a.fixed_sweeps = 1 << 30;   // never decided on the device: the caller takes the global maximum
    a.max_iter = 1 << 30;
    a.check_every = 1;
    const int ia = (h->cur + 1) % 3, ib = (h->cur + 2) % 3;
    cudaError_t e;
    if (first) {
        a.src = h->psi[h->cur];
        a.dst = h->psi[ia];
        a.dst_index = ia;
        e = launch_init_sweep(a, s, h->use_tma != 0);
        h->slab_n = 1;
    } else {
        // sweep number slab_n reads the previous output: odd A -> B, even B -> A
        const bool odd = (h->slab_n % 2) == 1;
        a.src = odd ? h->psi[ia] : h->psi[ib];
        a.dst = odd ? h->psi[ib] : h->psi[ia];
        a.dst_index = odd ? ib : ia;
        if (h->use_tma) {
            int src = 0;
            while (src < 2 && h->psi[src] != a.src) ++src;
            e = launch_sweep_tma(a, h->tmaps.psi[src], h->tmaps, s);
        } else {
            e = launch_sweep(a, s);
        }
        h->slab_n += 1;
    }
    if (e != cudaSuccess) return TDGL_ERR_CUDA;
    h->slab_last = a.dst_index;
    h->prof.kernel_launches += 1;
    DevCtl ctl;
    int rc = read_ctl(h, &ctl);
    if (rc != TDGL_OK) return rc;
    if (r2_local) *r2_local = ctl.r2;
    return ctl.status;
}

int tdgl_slab_accept(tdgl_handle *h)
{
    if (!h || !h->slab || h->slab_n < 1) return TDGL_ERR_INVALID_ARG;
    h->cur = h->slab_last;
    h->last_sweeps = h->slab_n;
    h->prof.sweeps += h->slab_n;
    h->slab_n = 0;
    ++h->step;
    return TDGL_OK;
}

int tdgl_slab_planes(tdgl_handle *h, int32_t latest, float **planes)
{
    if (!h || !h->slab || !planes || (latest && h->slab_n < 1)) return TDGL_ERR_INVALID_ARG;
    float2 *buf = h->psi[latest ? h->slab_last : h->cur];
    const long long pl = (long long)h->g.nx * h->g.ny;
    planes[0] = reinterpret_cast<float *>(buf + pl);                        // first slab plane
    planes[1] = reinterpret_cast<float *>(buf + pl * h->slab_nz);           // last slab plane
    planes[2] = reinterpret_cast<float *>(buf);                             // halo below
    planes[3] = reinterpret_cast<float *>(buf + pl * (h->slab_nz + 1));     // halo above
    return TDGL_OK;
}

int tdgl_slab_rhs(tdgl_handle *h)
{
    if (!h || !h->slab) return TDGL_ERR_INVALID_ARG;
    if (poisson_rhs(h, h->stream) != cudaSuccess) return TDGL_ERR_CUDA;
    h->prof.kernel_launches += 1;
    return cuda_err(cudaGetLastError());
}

// ---------------------------------------------------------------------------------
// Poisson-only handle: the potential of a right-hand side the caller writes into f
// ---------------------------------------------------------------------------------
size_t tdgl_poisson_workspace_bytes(const tdgl_config *cfg)
{
    if (validate(cfg, true) != TDGL_OK || cfg->d_insulating || cfg->links_mode != TDGL_LINKS_LANDAU) return 0;
    return layout(cfg, true).total;
}

int tdgl_poisson_create(const tdgl_config *cfg, void *d_workspace, size_t ws_bytes, void *stream, tdgl_handle **out)
{
    if (!cfg || cfg->d_insulating || cfg->links_mode != TDGL_LINKS_LANDAU) return TDGL_ERR_INVALID_ARG;
    return create_impl(cfg, d_workspace, ws_bytes, stream, out, true);
}

int tdgl_solve_mu_f(tdgl_handle *h)
{
    if (!h || h->batch_owned || h->slab || h->lk) return TDGL_ERR_INVALID_ARG;
    const tdgl_config &c = h->cfg;
    cudaStream_t s = h->stream;
    h->mu_solved = 1;
    h->guess_ready = 0;   // the guess is formed here, from the state and the previous mu
    long long nl = 1;
    if (launch_f_mean(h->pa, s) != cudaSuccess) return TDGL_ERR_CUDA;
    if (extrapolating(h)) {
        // the guess 2 mu^(n-1) - mu^(n-2) over the previous mu, then solve there
        const int q = h->mu_q;
        if (launch_mu_guess(h->g.N, h->mu, h->mu_buf[1 - q], h->prev_valid ? 2.f : 1.f, h->prev_valid ? -1.f : 0.f,
                            &h->ctl->mu_off[q], &h->ctl->mu_off[1 - q], s) != cudaSuccess)
            return TDGL_ERR_CUDA;
        use_mu_buffer(h, 1 - q);
        h->prev_valid = 1;
        nl += 1;
    }
    const bool fm = c.poisson_tol <= 0 && c.poisson_cycles > 0 && vcycle_mean_fusable(h->pa);
    int cycles = 0;
    for (; cycles < c.poisson_cycles; ++cycles)
        if (launch_vcycle(h->pa, s, &nl, cycles > 0, fm && cycles == c.poisson_cycles - 1) != cudaSuccess)
            return TDGL_ERR_CUDA;
    if (c.poisson_tol > 0) {
        for (;;) {
            if (launch_poisson_residual(h->pa, s) != cudaSuccess) return TDGL_ERR_CUDA;
            ++nl;
            DevCtl ctl;
            int rc = read_ctl(h, &ctl);
            if (rc != TDGL_OK) return rc;
            if (ctl.res <= c.poisson_tol || cycles >= c.poisson_max_cycles) break;
            if (launch_vcycle(h->pa, s, &nl, true) != cudaSuccess) return TDGL_ERR_CUDA;
            ++cycles;
        }
    }
    if ((lazy_projection(h, fm) ? launch_commit_mean(h->pa, s) : launch_project_mu(h->pa, s, fm)) != cudaSuccess)
        return TDGL_ERR_CUDA;
    h->mu_pend[h->mu_q] = lazy_projection(h, fm) ? 1 : 0;
    if (c.bc[0] == TDGL_OPEN && launch_voltage(h->pa, s) != cudaSuccess) return TDGL_ERR_CUDA;
    h->last_cycles = cycles;
    h->prof.vcycles += cycles;
    h->prof.kernel_launches += nl + 2;
    return cuda_err(cudaGetLastError());
}

int tdgl_read_ctl_scalars(tdgl_handle *h, double *Ex, double *poisson_res)
{
    if (!h) return TDGL_ERR_INVALID_ARG;
    if (poisson_res && h->mu_solved && !h->lk && h->cfg.poisson_tol <= 0 &&
        launch_poisson_residual(h->pa, h->stream) != cudaSuccess)
        return TDGL_ERR_CUDA;
    DevCtl ctl;
    int rc = read_ctl(h, &ctl);
    if (rc != TDGL_OK) return rc;
    if (Ex) *Ex = ctl.Ex;
    if (poisson_res) *poisson_res = ctl.res;
    return TDGL_OK;
}

int tdgl_step(tdgl_handle *h, int n_steps)
{
    if (h && h->res_pending) {   // resident steps enqueued: finish and account for them first
        const int rs = resident_sync(h);
        if (rs != TDGL_OK) return rs;
    }
    if (!h || h->batch_owned || h->slab || h->poisson_only || n_steps < 0) return TDGL_ERR_INVALID_ARG;
    const tdgl_config &c = h->cfg;
    cudaStream_t s = h->stream;
    for (int n = 0; n < n_steps; ++n) {
        int rc = tdgl_solve_psi(h, nullptr);
        if (rc != TDGL_OK) return rc;
        if (c.bc[0] == TDGL_PERIODIC) {
            KArgs k;
            k.g = h->g;
            k.ctl = h->ctl;
            k.blockred = h->blockred;
            k.psi = h->psi[h->cur];
            k.hx = c.hx;
            k.dtK = h->dtK;
            k.Jext = c.Jext;
            k.update_K = c.freeze_mu_K ? 0 : 1;
            ev_rec(h, 4);
            if (launch_javg_K(k, s) != cudaSuccess) return TDGL_ERR_CUDA;
            ev_rec(h, 5);
            h->pend_K = h->prof_on;
            h->prof.kernel_launches += 1;
        }
        ev_rec(h, 6);
        if (!c.freeze_mu_K) {
            rc = tdgl_solve_mu(h);
            if (rc != TDGL_OK) return rc;
        }
        if (c.bc[0] == TDGL_OPEN) {
            if ((h->lk ? launch_voltage_masked(h->pa, h->ip, s) : launch_voltage(h->pa, s)) != cudaSuccess)
                return TDGL_ERR_CUDA;
            h->prof.kernel_launches += 1;
        }
        ev_rec(h, 7);
        h->pend_P = h->prof_on;
        ++h->step;
        ++h->prof.steps;
        h->stepped = 1;
    }
    return cuda_err(cudaGetLastError());
}

// The state a trial of tdgl_autotune changes, saved in host memory and put back.
struct TuneSave {
    std::vector<float2> psi;
    std::vector<float> mu[2];
    DevCtl ctl;
    int cur, mu_q, prev_valid, guess_ready, last_sweeps, last_cycles, stepped;
    int mu_pend[2];
    int64_t step;
    tdgl_profile prof;
};

static int tune_save(tdgl_handle *h, TuneSave &t)
{
    const size_t N = (size_t)h->g.N;
    cudaStream_t s = h->stream;
    t.psi.resize(N);
    if (cudaMemcpyAsync(t.psi.data(), h->psi[h->cur], 8 * N, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return TDGL_ERR_CUDA;
    for (int q = 0; q < 2; ++q) {
        if (!h->mu_buf[q]) continue;
        t.mu[q].resize(N);
        if (cudaMemcpyAsync(t.mu[q].data(), h->mu_buf[q], 4 * N, cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return TDGL_ERR_CUDA;
    }
    if (cudaMemcpyAsync(&t.ctl, h->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, s) != cudaSuccess) return TDGL_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return TDGL_ERR_CUDA;
    t.cur = h->cur;
    t.mu_q = h->mu_q;
    t.prev_valid = h->prev_valid;
    t.guess_ready = h->guess_ready;
    t.last_sweeps = h->last_sweeps;
    t.last_cycles = h->last_cycles;
    t.stepped = h->stepped;
    t.mu_pend[0] = h->mu_pend[0];
    t.mu_pend[1] = h->mu_pend[1];
    t.step = h->step;
    t.prof = h->prof;
    return TDGL_OK;
}

static int tune_restore(tdgl_handle *h, const TuneSave &t)
{
    const size_t N = (size_t)h->g.N;
    cudaStream_t s = h->stream;
    if (cudaMemcpyAsync(h->psi[t.cur], t.psi.data(), 8 * N, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return TDGL_ERR_CUDA;
    for (int q = 0; q < 2; ++q)
        if (h->mu_buf[q] &&
            cudaMemcpyAsync(h->mu_buf[q], t.mu[q].data(), 4 * N, cudaMemcpyHostToDevice, s) != cudaSuccess)
            return TDGL_ERR_CUDA;
    if (cudaMemcpyAsync(h->ctl, &t.ctl, sizeof(DevCtl), cudaMemcpyHostToDevice, s) != cudaSuccess) return TDGL_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return TDGL_ERR_CUDA;
    h->cur = t.cur;
    use_mu_buffer(h, t.mu_q);
    h->mu_solved = 0;   // f holds a trial's right-hand side: the saved residual stands
    h->prev_valid = t.prev_valid;
    h->guess_ready = t.guess_ready;
    h->last_sweeps = t.last_sweeps;
    h->last_cycles = t.last_cycles;
    h->stepped = t.stepped;
    h->mu_pend[0] = t.mu_pend[0];
    h->mu_pend[1] = t.mu_pend[1];
    h->step = t.step;
    h->prof = t.prof;
    return TDGL_OK;
}

// candidate c: 0 the staged sweep, 1 the register-tiled sweep, 2 two sweeps per pass
static void tune_apply(tdgl_handle *h, int c)
{
    h->use_tma = (c == 0) ? 1 : 0;
    h->cfg.sweeps_per_pass = (c == 2) ? 2 : 1;
    drop_poisson_graphs(h);   // captured with the previous kernels (and the resident loop's graph)
    h->pgraph_fail = 0;
    h->rgraph_fail = 0;
}

int tdgl_autotune(tdgl_handle *h, int32_t trial_steps, tdgl_tune_report *report)
{
    if (!h || !report || trial_steps < 1 || h->batch_owned || h->slab || h->poisson_only) return TDGL_ERR_INVALID_ARG;
    if (h->res_pending) {   // resident steps enqueued: finish and account for them first
        const int rs = resident_sync(h);
        if (rs != TDGL_OK) return rs;
    }
    memset(report, 0, sizeof(*report));
    bool ok[3];
    ok[0] = tma_sweep_supported(h->g) && (h->use_tma || tma_encode_maps(h->g, h->psi, h->b, h->D, &h->tmaps));
    ok[1] = true;
    ok[2] = pair_supported(h->g) && h->cfg.fixed_sweeps <= 0;
    const int start = h->cfg.sweeps_per_pass == 2 && ok[2] ? 2 : (h->use_tma ? 0 : 1);
    TuneSave t;
    int rc = tune_save(h, t);
    if (rc != TDGL_OK) return rc;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return TDGL_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return TDGL_ERR_CUDA;
    }
    int best = start;
    for (int c = 0; c < 3 && rc == TDGL_OK; ++c) {
        if (!ok[c]) continue;
        tune_apply(h, c);
        rc = tdgl_step(h, 1);   // warm-up (and the first replay-captured Poisson sequence)
        if (rc == TDGL_OK && cudaEventRecord(e0, h->stream) != cudaSuccess) rc = TDGL_ERR_CUDA;
        if (rc == TDGL_OK) rc = tdgl_step(h, trial_steps);
        if (rc == TDGL_OK && (cudaEventRecord(e1, h->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
            rc = TDGL_ERR_CUDA;
        float ms = 0.f;
        if (rc == TDGL_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = TDGL_ERR_CUDA;
        if (rc == TDGL_OK) {
            report->ms[c] = ms / trial_steps;
            report->candidates += 1;
            if (report->ms[c] < report->ms[best] || !ok[best] || report->ms[best] == 0.0) best = c;
        }
        const int rr = tune_restore(h, t);
        if (rc == TDGL_OK) rc = rr;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // a failed trial leaves the starting configuration
    tune_apply(h, rc == TDGL_OK ? best : start);
    report->chosen = rc == TDGL_OK ? best : start;
    return rc;
}

int tdgl_observables(tdgl_handle *h, tdgl_obs *out)
{
    if (h && h->res_pending) {   // resident steps enqueued: finish and account for them first
        const int rs = resident_sync(h);
        if (rs != TDGL_OK) return rs;
    }
    if (!h || !out || h->slab || h->poisson_only) return TDGL_ERR_INVALID_ARG;
    const tdgl_config &c = h->cfg;
    double flux = c.hx * c.hy * c.Bz;
    // a solve with a fixed number of V-cycles never measured its residual: measure it now
    // (max|F - Lap mu| / max|F| of the last solve's right-hand side and result)
    if (h->mu_solved && !h->batch_owned && !h->lk && c.poisson_tol <= 0 &&
        launch_poisson_residual(h->pa, h->stream) != cudaSuccess)
        return TDGL_ERR_CUDA;
    if (launch_observables(h->g, h->ctl, h->blockred, h->psi[h->cur], c.d_alpha, nullptr, flux, h->stream) != cudaSuccess)
        return TDGL_ERR_CUDA;
    DevCtl ctl;
    int rc = read_ctl(h, &ctl);
    if (rc != TDGL_OK) return rc;
    double dV = c.hx * c.hy * (c.nz >= 2 ? c.hz : 1.0);
    memset(out, 0, sizeof(*out));
    out->psi2_mean = ctl.sums[0] / (double)h->g.N;
    out->energy = ctl.sums[1] * dV;
    out->vortex_unsigned = ctl.sums[2] / (double)c.nz;
    out->vortex_signed = ctl.sums[3] / (double)c.nz;
    out->javg = ctl.javg;
    out->K = ctl.K;
    out->Ex = ctl.Ex;
    out->last_r2 = ctl.r2;
    out->poisson_res = ctl.res;
    out->last_sweeps = h->batch_owned ? ctl.iter : h->last_sweeps;
    out->poisson_cycles = h->last_cycles;
    out->step = h->step;
    return TDGL_OK;
}

// The candidates of tdgl_pattern (centre, semi-axes, quaternion) as ellipsoid shapes.
static std::vector<tdgl_shape> candidates_as_shapes(const double *c, int64_t n, float alpha_in)
{
    std::vector<tdgl_shape> v((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        const double *q = c + 10 * i;
        tdgl_shape &S = v[(size_t)i];
        S.kind = TDGL_SHAPE_ELLIPSOID;
        S.flags = 0;
        for (int a = 0; a < 3; ++a) {
            S.c[a] = q[a];
            S.a[a] = q[3 + a];
        }
        for (int a = 0; a < 4; ++a) S.q[a] = q[6 + a];
        S.value = (double)alpha_in;
    }
    return v;
}

size_t tdgl_pattern_scratch_bytes(const tdgl_config *grid, int64_t n_candidates)
{
    if (n_candidates < 0 || n_candidates > 0x7ffffff0LL) return 0;
    tdgl_background bg;
    memset(&bg, 0, sizeof(bg));
    return pattern_ex_scratch(grid, n_candidates, nullptr, 0, &bg);
}

int tdgl_pattern(const tdgl_config *grid, const double *host_candidates, int64_t n_candidates, int64_t target_sites,
                 float alpha_in, float alpha_out, float *d_alpha, void *d_scratch, size_t scratch_bytes, void *stream,
                 int64_t *n_used, int64_t *n_marked)
{
    if (!grid || !d_alpha || n_candidates < 0 || (n_candidates > 0 && !host_candidates)) return TDGL_ERR_INVALID_ARG;
    if (n_candidates > 0x7ffffff0LL) return TDGL_ERR_INVALID_ARG;
    for (int64_t n = 0; n < n_candidates; ++n) {
        const double *q = host_candidates + 10 * n;
        if (!(q[3] > 0) || !(q[4] > 0) || !(q[5] > 0)) return TDGL_ERR_INVALID_ARG;
    }
    std::vector<tdgl_shape> sh = candidates_as_shapes(host_candidates, n_candidates, alpha_in);
    tdgl_background bg;
    memset(&bg, 0, sizeof(bg));
    bg.kind = TDGL_BG_CONSTANT;
    bg.value = (double)alpha_out;
    return pattern_ex_run(grid, sh.data(), n_candidates, nullptr, 0, &bg, target_sites, d_alpha, nullptr, d_scratch,
                          scratch_bytes, (cudaStream_t)stream, n_used, n_marked);
}

size_t tdgl_pattern_ex_scratch_bytes(const tdgl_config *grid, int64_t n_shapes, const tdgl_lattice *lattices,
                                     int32_t n_lattices, const tdgl_background *bg)
{
    return pattern_ex_scratch(grid, n_shapes, lattices, n_lattices, bg);
}

int tdgl_pattern_ex(const tdgl_config *grid, const tdgl_shape *shapes, int64_t n_shapes, const tdgl_lattice *lattices,
                    int32_t n_lattices, const tdgl_background *bg, int64_t target_sites, float *d_alpha,
                    uint8_t *d_insulating, void *d_scratch, size_t scratch_bytes, void *stream, int64_t *n_used,
                    int64_t *n_marked)
{
    return pattern_ex_run(grid, shapes, n_shapes, lattices, n_lattices, bg, target_sites, d_alpha, d_insulating,
                          d_scratch, scratch_bytes, (cudaStream_t)stream, n_used, n_marked);
}

}  // extern "C"

// Pieces of the host-driven step shared with the device-resident step loop
namespace tdgl {
SweepArgs step_sweep_args(tdgl_handle *h) { return sweep_args(h); }
void step_guess_args(const tdgl_handle *h, SweepArgs &a, int q) { guess_args(h, a, q, true); }
long long step_poisson_sequence(tdgl_handle *h, cudaStream_t s, cudaError_t *err) { return poisson_sequence(h, s, err); }
bool step_lazy_projection(const tdgl_handle *h)
{
    return lazy_projection(h, h->cfg.poisson_cycles > 0 && vcycle_mean_fusable(h->pa));
}
bool step_pairs(const tdgl_handle *h) { return h->cfg.sweeps_per_pass == 2 && pair_supported(h->g); }
int step_read_ctl(tdgl_handle *h, DevCtl *out) { return read_ctl(h, out); }
}  // namespace tdgl
