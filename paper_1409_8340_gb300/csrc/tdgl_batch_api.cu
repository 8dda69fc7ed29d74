// C ABI of batched ensembles: instance creation in one caller-owned workspace,
// the instance table of the persistent kernel, CUDA-graph replay of its
// launches, per-instance status, and the autotuner (launch shape, sweep tile kind
// and sweep tile depth per grid-size class, timed on the batch itself).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <tuple>
#include <vector>

#include "mg_tile.cuh"

using namespace tdgl;

namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr int kPhaseLogCap = 8192;   // phase-log entries (one launch)

int batch_check(const tdgl_config *c)
{
    if (!c) return TDGL_ERR_INVALID_ARG;
    if (tdgl_workspace_bytes(c) == 0) return TDGL_ERR_INVALID_ARG;
    if (c->links_mode != TDGL_LINKS_LANDAU || (c->nx % 2) != 0 || c->d_insulating) return TDGL_ERR_INVALID_ARG;
    if ((long long)c->nx * c->ny * c->nz >= (1LL << 31)) return TDGL_ERR_INVALID_ARG;
    if (c->poisson_tol > 0) return TDGL_ERR_INVALID_ARG;

    return TDGL_OK;
}

struct BLayout {
    std::vector<size_t> inst;   // offset of each instance's workspace
    size_t table, order, act, bst, sweeps, bar, plog, save, total;
    std::vector<size_t> save_psi, save_mu, save_mu2, save_ctl;
};

BLayout blayout(const tdgl_config *cfgs, int n)
{
    BLayout L;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    for (int i = 0; i < n; ++i) L.inst.push_back(take(tdgl_workspace_bytes(&cfgs[i])));
    L.table = take(sizeof(BatchInst) * (size_t)n);
    L.order = take(sizeof(int) * (size_t)n);
    L.act = take(sizeof(int) * 2 * (size_t)n);
    L.bst = take(sizeof(int) * (size_t)n);
    L.sweeps = take(sizeof(long long) * (size_t)n);
    // psi-solve count, error flag, mu-solve count, log index, two item counters per launch
    L.bar = take(8 * sizeof(unsigned int));
    L.plog = take(2 * sizeof(unsigned long long) * kPhaseLogCap);
    L.save = off;
    for (int i = 0; i < n; ++i) {
        const size_t N = (size_t)cfgs[i].nx * cfgs[i].ny * cfgs[i].nz;
        L.save_psi.push_back(take(8 * N));
        L.save_mu.push_back(take(4 * N));
        L.save_mu2.push_back(take(4 * N));   // the second mu buffer (previous mu)
        L.save_ctl.push_back(take(sizeof(DevCtl)));
    }
    L.total = off;
    return L;
}

template <class T>
T *at(void *base, size_t off)
{
    return reinterpret_cast<T *>(reinterpret_cast<char *>(base) + off);
}

}  // namespace

struct tdgl_batch {
    int n;
    cudaStream_t stream;        // the caller's stream: launches and graph replays
    cudaStream_t cap;           // private stream the graph is captured on
    void *ws;
    BLayout L;
    std::vector<tdgl_handle *> h;
    std::vector<BatchInst> inst;
    BatchParams P;
    int sms;
    int occ2, occ3;             // resident blocks per SM of the two kernel variants
    int bps, grid;
    size_t smem;
    tdgl_batch_tuning tune;
    std::vector<int> order;     // dealing order of the instances (device copy at L.order)
    cudaGraphExec_t gexec;
    int graph_built;            // gexec matches the current table and launch shape
    int graph_ok;               // capture worked (0: plain launches)
    int log_on;                 // phase log of every launch
    int64_t steps;
};

namespace {

void fill_instance(tdgl_batch *b, int i, int kz)
{
    tdgl_handle *h = b->h[i];
    const tdgl_config &c = h->cfg;
    BatchInst &I = b->inst[i];
    memset(&I, 0, sizeof(I));
    BatchHead &H = I.h;
    SweepArgs &a = H.a;
    a.g = h->g;
    a.ctl = h->ctl;
    a.blockred = h->blockred;
    a.b = h->b;
    a.D = h->D;
    a.mu = h->mu;
    a.alpha = c.d_alpha;
    a.check_every = c.check_every;
    a.fixed_sweeps = c.fixed_sweeps;
    a.max_iter = c.max_iter;
    a.eps = c.eps;
    a.rel_eps = 0;
    a.noise_amp = h->noise_amp;
    a.noise_seed = c.noise_seed;
    a.f = h->f;
    a.inj = h->pa.inject ? (float)(2.0 * c.Jext / c.hx) : 0.f;
    a.wsum = h->wsum;
    for (int q = 0; q < 3; ++q) H.psi[q] = h->psi[q];
    H.iS = h->cur;
    H.iA = (h->cur + 1) % 3;
    H.iB = (h->cur + 2) % 3;
    // sweep tiles and reduction items must fit the instance's partial slots
    if (kz <= 0) kz = batch_default_kz(h->g);
    batch_tiling(I, kz);
    while ((size_t)H.tiles > h->nblockred && H.kz < c.nz) batch_tiling(I, H.kz * 2);
    H.split_max = 1;
    for (int sp = 2; sp <= 4; sp *= 2)
        if (H.kz % sp == 0 && (size_t)H.tiles * sp <= h->nblockred) H.split_max = sp;
    const long long N = h->g.N;
    const long long half = (long long)(h->nblockred / 2);
    long long chunk = std::max<long long>(32768, (N + half - 1) / half);
    chunk = (chunk + 255) / 256 * 256;
    H.red_chunk = (int)chunk;
    H.red_items = (int)((N + chunk - 1) / chunk);
    H.periodic_x = c.bc[0] == TDGL_PERIODIC;
    H.open_x = !H.periodic_x;
    H.freeze = c.freeze_mu_K ? 1 : 0;
    H.cycles = c.poisson_cycles;
    H.hx = c.hx;
    H.dtK = h->dtK;
    H.Jext = c.Jext;
    H.nlev = h->pa.nlevels;
    H.mean_fused = (!H.freeze && H.nlev >= 2) ? 1 : 0;
    for (int l = 0; l < H.nlev; ++l) {
        const MGLevel &M = h->pa.lev[l];
        H.lpb[l] = line_shape(M.nx, M.kmin, M.kmax, 256).lpb;
        for (int col = 0; col < 2; ++col) H.nlines[l][col] = mg_lines_of_colour(M.ny, M.nz, col);
    }
    I.pa = h->pa;
    // Poisson guess: the linear extrapolation in time (tdgl_config.poisson_guess 0 or 2),
    // solved in the second mu buffer; else the previous mu, solved in place
    const bool ex = h->mu_buf[1] && !c.freeze_mu_K && (c.poisson_guess == 0 || c.poisson_guess == 2);
    H.mu_solve = ex ? h->mu_buf[1] : h->mu;
    I.pa.lev[0].u = I.pa.mu = H.mu_solve;
    I.pa.mu_q = -1;
    for (int l = 0; l < kMaxLevels; ++l) I.pa.umap_u[l] = nullptr;   // the batch smoother reads u directly
}

void fill_params(tdgl_batch *b)
{
    BatchParams &P = b->P;
    memset(&P, 0, sizeof(P));
    P.inst = at<BatchInst>(b->ws, b->L.table);
    P.n = b->n;
    P.act = at<int>(b->ws, b->L.act);
    P.bst = at<int>(b->ws, b->L.bst);
    P.sweeps = at<long long>(b->ws, b->L.sweeps);
    P.bar = at<unsigned int>(b->ws, b->L.bar);
    P.extra = (unsigned int)std::max(0, b->tune.test_extra_arrivals);
    P.staged = b->tune.sweep_kernel == 0 ? 1 : 0;
    P.timeout_ns = (unsigned long long)std::max(1, b->tune.timeout_ms) * 1000000ull;
    P.plog = b->log_on ? at<unsigned long long>(b->ws, b->L.plog) : nullptr;
    P.plog_cap = b->log_on ? kPhaseLogCap : 0;
    int phases = 1;
    for (int i = 0; i < b->n; ++i) {
        const BatchHead &H = b->inst[i].h;
        P.lmax = std::max(P.lmax, H.nlev - 1);
        if (!H.freeze) P.cycles_max = std::max(P.cycles_max, H.cycles);
        P.any_px |= H.periodic_x;
        if (H.freeze ? H.open_x : !H.mean_fused) P.any_mean = 1;
        phases = std::max(phases, H.a.fixed_sweeps > 0 ? H.a.fixed_sweeps : H.a.max_iter);
    }
    P.max_phases = phases + 1;
    // dealing order: sites per sweep tile, largest first (ties by index)
    std::vector<int> ord(b->n);
    for (int i = 0; i < b->n; ++i) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
        const BatchHead &X = b->inst[x].h, &Y = b->inst[y].h;
        return (double)X.a.g.N / X.tiles > (double)Y.a.g.N / Y.tiles;
    });
    b->order = ord;
    P.order = at<int>(b->ws, b->L.order);
}

// Push the table and launch shape of the current tuning to the device.
int apply_tuning(tdgl_batch *b)
{
    size_t smem = 0;
    for (int i = 0; i < b->n; ++i) {
        fill_instance(b, i, b->tune.kz[i]);
        b->tune.kz[i] = b->inst[i].h.kz;
        smem = std::max(smem, batch_smem_bytes(b->inst[i]));
    }
    b->smem = smem;
    if (batch_max_blocks_per_sm(smem, 2, &b->occ2) != cudaSuccess) return TDGL_ERR_CUDA;
    if (batch_max_blocks_per_sm(smem, 3, &b->occ3) != cudaSuccess) return TDGL_ERR_CUDA;
    int want = b->tune.blocks_per_sm;
    if (want <= 0) want = b->occ3 >= 3 ? 3 : std::min(2, b->occ2);
    if (want >= 3 && b->occ3 < 3) want = 2;
    if (want == 2 && b->occ2 < 2) want = 1;
    if (want < 1 || b->occ2 < 1) return TDGL_ERR_INVALID_ARG;
    b->bps = want;
    b->tune.blocks_per_sm = want;
    b->grid = b->sms * want;
    fill_params(b);
    if (cudaMemcpyAsync(at<BatchInst>(b->ws, b->L.table), b->inst.data(), sizeof(BatchInst) * b->n,
                        cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
        cudaMemcpyAsync(at<int>(b->ws, b->L.order), b->order.data(), sizeof(int) * b->n, cudaMemcpyHostToDevice,
                        b->stream) != cudaSuccess)
        return TDGL_ERR_CUDA;
    b->graph_built = 0;
    return cudaStreamSynchronize(b->stream) == cudaSuccess ? TDGL_OK : TDGL_ERR_CUDA;
}

void drop_graph(tdgl_batch *b)
{
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
    b->graph_built = 0;
}

// Capture graph_steps launches on the private stream; on failure fall back to
// plain launches.
void build_graph(tdgl_batch *b)
{
    drop_graph(b);
    b->graph_ok = 0;
    b->graph_built = 1;
    if (b->tune.graph_steps <= 0) return;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    bool ok = true;
    for (int q = 0; q < b->tune.graph_steps && ok; ++q)
        ok = launch_batch_step(b->P, b->grid, b->bps, b->smem, b->cap) == cudaSuccess;
    cudaError_t e = cudaStreamEndCapture(b->cap, &g);
    if (!ok || e != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return;
    }
    e = cudaGraphInstantiate(&b->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->gexec = nullptr;
        cudaGetLastError();
        return;
    }
    b->graph_ok = 1;
}

int enqueue_steps(tdgl_batch *b, int n, bool allow_graph)
{
    int done = 0;
    if (allow_graph) {
        if (!b->graph_built) build_graph(b);
        if (b->graph_ok) {
            for (; done + b->tune.graph_steps <= n; done += b->tune.graph_steps)
                if (cudaGraphLaunch(b->gexec, b->stream) != cudaSuccess) return TDGL_ERR_CUDA;
        }
    }
    for (; done < n; ++done)
        if (launch_batch_step(b->P, b->grid, b->bps, b->smem, b->stream) != cudaSuccess) return TDGL_ERR_CUDA;
    b->steps += n;
    for (tdgl_handle *h : b->h) h->step += n;
    return TDGL_OK;
}

int read_error_flag(tdgl_batch *b, unsigned int *err)
{
    if (cudaMemcpyAsync(err, b->P.bar + 1, sizeof(unsigned int), cudaMemcpyDeviceToHost, b->stream) != cudaSuccess)
        return TDGL_ERR_CUDA;
    return cudaStreamSynchronize(b->stream) == cudaSuccess ? TDGL_OK : TDGL_ERR_CUDA;
}

int save_states(tdgl_batch *b, std::vector<int> &bst, std::vector<long long> &sw)
{
    cudaStream_t s = b->stream;
    for (int i = 0; i < b->n; ++i) {
        tdgl_handle *h = b->h[i];
        const size_t N = (size_t)h->g.N;
        if (cudaMemcpyAsync(at<char>(b->ws, b->L.save_psi[i]), h->psi[h->cur], 8 * N, cudaMemcpyDeviceToDevice, s) ||
            cudaMemcpyAsync(at<char>(b->ws, b->L.save_mu[i]), h->mu, 4 * N, cudaMemcpyDeviceToDevice, s) ||
            cudaMemcpyAsync(at<char>(b->ws, b->L.save_ctl[i]), h->ctl, sizeof(DevCtl), cudaMemcpyDeviceToDevice, s))
            return TDGL_ERR_CUDA;
        if (h->mu_buf[1] &&
            cudaMemcpyAsync(at<char>(b->ws, b->L.save_mu2[i]), h->mu_buf[1], 4 * N, cudaMemcpyDeviceToDevice, s))
            return TDGL_ERR_CUDA;
    }
    bst.resize(b->n);
    sw.resize(b->n);
    if (cudaMemcpyAsync(bst.data(), b->P.bst, sizeof(int) * b->n, cudaMemcpyDeviceToHost, s) ||
        cudaMemcpyAsync(sw.data(), b->P.sweeps, sizeof(long long) * b->n, cudaMemcpyDeviceToHost, s))
        return TDGL_ERR_CUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? TDGL_OK : TDGL_ERR_CUDA;
}

int restore_states(tdgl_batch *b, const std::vector<int> &bst, const std::vector<long long> &sw)
{
    cudaStream_t s = b->stream;
    for (int i = 0; i < b->n; ++i) {
        tdgl_handle *h = b->h[i];
        const size_t N = (size_t)h->g.N;
        if (cudaMemcpyAsync(h->psi[h->cur], at<char>(b->ws, b->L.save_psi[i]), 8 * N, cudaMemcpyDeviceToDevice, s) ||
            cudaMemcpyAsync(h->mu, at<char>(b->ws, b->L.save_mu[i]), 4 * N, cudaMemcpyDeviceToDevice, s) ||
            cudaMemcpyAsync(h->ctl, at<char>(b->ws, b->L.save_ctl[i]), sizeof(DevCtl), cudaMemcpyDeviceToDevice, s))
            return TDGL_ERR_CUDA;
        if (h->mu_buf[1] &&
            cudaMemcpyAsync(h->mu_buf[1], at<char>(b->ws, b->L.save_mu2[i]), 4 * N, cudaMemcpyDeviceToDevice, s))
            return TDGL_ERR_CUDA;
    }
    if (cudaMemcpyAsync(b->P.bst, bst.data(), sizeof(int) * b->n, cudaMemcpyHostToDevice, s) ||
        cudaMemcpyAsync(b->P.sweeps, sw.data(), sizeof(long long) * b->n, cudaMemcpyHostToDevice, s))
        return TDGL_ERR_CUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? TDGL_OK : TDGL_ERR_CUDA;
}

}  // namespace

extern "C" {

size_t tdgl_batch_workspace_bytes(const tdgl_config *cfgs, int32_t n)
{
    if (!cfgs || n < 1 || n > TDGL_BATCH_MAX) return 0;
    for (int i = 0; i < n; ++i)
        if (batch_check(&cfgs[i]) != TDGL_OK) return 0;
    return blayout(cfgs, n).total;
}

int tdgl_batch_create(const tdgl_config *cfgs, int32_t n, void *d_workspace, size_t ws_bytes, void *stream,
                      tdgl_batch **out)
{
    if (!out) return TDGL_ERR_INVALID_ARG;
    *out = nullptr;
    if (!cfgs || n < 1 || n > TDGL_BATCH_MAX) return TDGL_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i) {
        int rc = batch_check(&cfgs[i]);
        if (rc != TDGL_OK) return rc;
    }
    BLayout L = blayout(cfgs, n);
    if (!d_workspace || ((uintptr_t)d_workspace & 255u) || ws_bytes < L.total) return TDGL_ERR_WORKSPACE;
    tdgl_batch *b = new tdgl_batch();
    b->n = n;
    b->stream = (cudaStream_t)stream;
    b->ws = d_workspace;
    b->L = L;
    b->inst.resize(n);
    b->tune.graph_steps = 10;
    b->tune.timeout_ms = 2000;
    int rc = TDGL_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess)
        rc = TDGL_ERR_CUDA;
    for (int i = 0; i < n && rc == TDGL_OK; ++i) {
        tdgl_handle *h = nullptr;
        rc = tdgl_create(&cfgs[i], at<char>(d_workspace, L.inst[i]), tdgl_workspace_bytes(&cfgs[i]), stream, &h);
        if (rc != TDGL_OK) break;
        h->batch_owned = 1;
        b->h.push_back(h);
        if (!h->pa.lev[h->pa.nlevels - 1].cw) rc = TDGL_ERR_INVALID_ARG;   // coarsest level too large to solve exactly
    }
    if (rc == TDGL_OK) {
        if (cudaMemsetAsync(at<char>(d_workspace, L.act), 0, L.save - L.act, b->stream) != cudaSuccess) rc = TDGL_ERR_CUDA;
    }
    if (rc == TDGL_OK) rc = apply_tuning(b);
    if (rc != TDGL_OK) {
        tdgl_batch_destroy(b);
        return rc;
    }
    *out = b;
    return TDGL_OK;
}

void tdgl_batch_destroy(tdgl_batch *b)
{
    if (!b) return;
    drop_graph(b);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (tdgl_handle *h : b->h) tdgl_destroy(h);
    delete b;
}

int tdgl_batch_instance(tdgl_batch *b, int32_t i, tdgl_handle **out)
{
    if (!b || !out || i < 0 || i >= b->n) return TDGL_ERR_INVALID_ARG;
    *out = b->h[i];
    return TDGL_OK;
}

int tdgl_batch_step(tdgl_batch *b, int32_t n_steps)
{
    if (!b || n_steps < 0) return TDGL_ERR_INVALID_ARG;
    return enqueue_steps(b, n_steps, true);
}

int tdgl_batch_status(tdgl_batch *b, int32_t *status)
{
    if (!b) return TDGL_ERR_INVALID_ARG;
    std::vector<int> st(b->n);
    if (cudaMemcpyAsync(st.data(), b->P.bst, sizeof(int) * b->n, cudaMemcpyDeviceToHost, b->stream) != cudaSuccess)
        return TDGL_ERR_CUDA;
    unsigned int err = 0;
    int rc = read_error_flag(b, &err);
    if (rc != TDGL_OK) return rc;
    if (status)
        for (int i = 0; i < b->n; ++i) status[i] = st[i];
    if (err == 1u) return TDGL_ERR_TIMEOUT;
    if (err != 0u) return TDGL_ERR_NOT_CONVERGED;
    for (int i = 0; i < b->n; ++i)
        if (st[i] != 0) return st[i];
    return TDGL_OK;
}

int tdgl_batch_observables(tdgl_batch *b, tdgl_obs *out)
{
    if (!b || !out) return TDGL_ERR_INVALID_ARG;
    for (int i = 0; i < b->n; ++i) {
        int rc = tdgl_observables(b->h[i], &out[i]);
        if (rc != TDGL_OK) return rc;
    }
    return TDGL_OK;
}

int tdgl_batch_stats_read(tdgl_batch *b, tdgl_batch_stats *out, int64_t *sweeps)
{
    if (!b || !out) return TDGL_ERR_INVALID_ARG;
    std::vector<long long> sw(b->n);
    if (cudaMemcpyAsync(sw.data(), b->P.sweeps, sizeof(long long) * b->n, cudaMemcpyDeviceToHost, b->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return TDGL_ERR_CUDA;
    memset(out, 0, sizeof(*out));
    out->steps = b->steps;
    for (int i = 0; i < b->n; ++i) {
        out->sweeps += sw[i];
        out->site_iters += (double)sw[i] * (double)b->h[i]->g.N;
        if (sweeps) sweeps[i] = sw[i];
    }
    out->grid_blocks = b->grid;
    out->blocks_per_sm = b->bps;
    if (!b->graph_built && b->tune.graph_steps > 0) build_graph(b);
    out->graph = b->graph_ok;
    out->smem_bytes = (int32_t)b->smem;
    return TDGL_OK;
}

int tdgl_batch_get_tuning(tdgl_batch *b, tdgl_batch_tuning *out)
{
    if (!b || !out) return TDGL_ERR_INVALID_ARG;
    *out = b->tune;
    return TDGL_OK;
}

int tdgl_batch_set_tuning(tdgl_batch *b, const tdgl_batch_tuning *in)
{
    if (!b || !in) return TDGL_ERR_INVALID_ARG;
    if (in->blocks_per_sm < 0 || in->blocks_per_sm > 3 || in->graph_steps < 0 || in->timeout_ms < 1 ||
        in->test_extra_arrivals < 0 || in->sweep_kernel < 0 || in->sweep_kernel > 1)
        return TDGL_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return TDGL_ERR_CUDA;
    b->tune = *in;
    return apply_tuning(b);
}

int tdgl_batch_phase_log(tdgl_batch *b, int32_t on)
{
    if (!b) return TDGL_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return TDGL_ERR_CUDA;
    b->log_on = on ? 1 : 0;
    return apply_tuning(b);
}

int tdgl_batch_phase_read(tdgl_batch *b, double *ms_by_op, int32_t *phases_by_op, int32_t nops)
{
    if (!b || !ms_by_op || !phases_by_op || nops < TDGL_BATCH_OPS) return TDGL_ERR_INVALID_ARG;
    if (!b->log_on) return TDGL_ERR_INVALID_ARG;
    std::vector<unsigned long long> log(2 * (size_t)kPhaseLogCap);
    if (cudaMemcpyAsync(log.data(), at<char>(b->ws, b->L.plog), sizeof(unsigned long long) * log.size(),
                        cudaMemcpyDeviceToHost, b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return TDGL_ERR_CUDA;
    for (int q = 0; q < nops; ++q) {
        ms_by_op[q] = 0.0;
        phases_by_op[q] = 0;
    }
    unsigned long long t_prev = log[0];
    for (int i = 1; i < kPhaseLogCap; ++i) {
        const unsigned long long tag = log[2 * i + 1];
        if (tag == 0xffffull) break;
        const int op = (int)(tag >> 8);
        if (op < 0 || op >= TDGL_BATCH_OPS) break;
        ms_by_op[op] += (double)(log[2 * i] - t_prev) * 1e-6;
        phases_by_op[op] += 1;
        t_prev = log[2 * i];
    }
    return TDGL_OK;
}

int tdgl_batch_phase_list(tdgl_batch *b, double *ms, int32_t *ops, int32_t cap, int32_t *n_out)
{
    if (!b || !ms || !ops || !n_out || cap < 0) return TDGL_ERR_INVALID_ARG;
    if (!b->log_on) return TDGL_ERR_INVALID_ARG;
    std::vector<unsigned long long> log(2 * (size_t)kPhaseLogCap);
    if (cudaMemcpyAsync(log.data(), at<char>(b->ws, b->L.plog), sizeof(unsigned long long) * log.size(),
                        cudaMemcpyDeviceToHost, b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return TDGL_ERR_CUDA;
    int n = 0;
    unsigned long long t_prev = log[0];
    for (int i = 1; i < kPhaseLogCap; ++i) {
        const unsigned long long tag = log[2 * i + 1];
        if (tag == 0xffffull) break;
        const int op = (int)(tag >> 8);
        if (op < 0 || op >= TDGL_BATCH_OPS) break;
        if (n < cap) {
            ms[n] = (double)(log[2 * i] - t_prev) * 1e-6;
            ops[n] = op;
        }
        ++n;
        t_prev = log[2 * i];
    }
    *n_out = n;
    return TDGL_OK;
}

int tdgl_batch_autotune(tdgl_batch *b, int32_t trial_steps, tdgl_batch_tune_report *report)
{
    if (!b || trial_steps < 1) return TDGL_ERR_INVALID_ARG;
    std::vector<int> bst;
    std::vector<long long> sw;
    int rc = save_states(b, bst, sw);
    if (rc != TDGL_OK) return rc;
    const int64_t steps0 = b->steps;
    std::vector<int64_t> hsteps;
    for (tdgl_handle *h : b->h) hsteps.push_back(h->step);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return TDGL_ERR_CUDA;
    int candidates = 0;
    // ms per step of the current tuning, from the saved states
    auto trial = [&](double *ms) -> int {
        int r = apply_tuning(b);
        if (r != TDGL_OK) return r;
        r = restore_states(b, bst, sw);
        if (r != TDGL_OK) return r;
        r = enqueue_steps(b, 1, false);
        if (r != TDGL_OK) return r;
        cudaEventRecord(e0, b->stream);
        r = enqueue_steps(b, trial_steps, false);
        if (r != TDGL_OK) return r;
        cudaEventRecord(e1, b->stream);
        unsigned int err = 0;
        r = read_error_flag(b, &err);
        if (r != TDGL_OK) return r;
        if (err) return TDGL_ERR_TIMEOUT;
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        *ms = (double)t / trial_steps;
        ++candidates;
        return TDGL_OK;
    };
    tdgl_batch_tuning best = b->tune;
    double ms_best = 0.0, ms_default = 0.0;
    rc = trial(&ms_default);
    ms_best = ms_default;
    best = b->tune;
    // launch shape
    for (int bps = 1; bps <= 3 && rc == TDGL_OK; ++bps) {
        if (bps == best.blocks_per_sm) continue;
        if ((bps == 3 && b->occ3 < 3) || (bps < 3 && b->occ2 < bps)) continue;
        tdgl_batch_tuning t = best;
        t.blocks_per_sm = bps;
        b->tune = t;
        double ms = 0.0;
        rc = trial(&ms);
        if (rc == TDGL_OK && ms < ms_best) {
            ms_best = ms;
            best = b->tune;
        }
    }
    // sweep tiles staged in shared memory or register-tiled
    if (rc == TDGL_OK) {
        tdgl_batch_tuning t = best;
        t.sweep_kernel = 1 - best.sweep_kernel;
        b->tune = t;
        double ms = 0.0;
        rc = trial(&ms);
        if (rc == TDGL_OK && ms < ms_best) {
            ms_best = ms;
            best = b->tune;
        }
    }
    // sweep tile depth per grid-size class
    std::map<std::tuple<int, int, int>, std::vector<int>> classes;
    for (int i = 0; i < b->n; ++i) classes[std::make_tuple(b->h[i]->g.nx, b->h[i]->g.ny, b->h[i]->g.nz)].push_back(i);
    for (auto &cl : classes) {
        if (rc != TDGL_OK) break;
        const std::vector<int> &members = cl.second;
        const int nz = std::get<2>(cl.first);
        for (int kz : {1, 2, 4, 8, 16, 32}) {
            if (kz > nz || kz == best.kz[members[0]]) continue;
            tdgl_batch_tuning t = best;
            for (int i : members) t.kz[i] = kz;
            b->tune = t;
            double ms = 0.0;
            rc = trial(&ms);
            if (rc != TDGL_OK) break;
            if (ms < ms_best) {
                ms_best = ms;
                best = b->tune;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->tune = best;
    int rc2 = apply_tuning(b);
    if (rc2 == TDGL_OK) rc2 = restore_states(b, bst, sw);
    b->steps = steps0;
    for (int i = 0; i < b->n; ++i) b->h[i]->step = hsteps[i];
    if (report) {
        report->ms_default = ms_default;
        report->ms_best = ms_best;
        report->candidates = candidates;
        report->classes = (int32_t)classes.size();
    }
    return rc != TDGL_OK ? rc : rc2;
}

}  // extern "C"
