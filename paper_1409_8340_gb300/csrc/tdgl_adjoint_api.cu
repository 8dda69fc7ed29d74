// Adjoint driver: forward pass with checkpoints, then segment-wise recompute
// and reverse steps (see k_adjoint.cu for the reverse-step equations).
#include <string.h>

#include <vector>

#include "tdgl_internal.cuh"

using namespace tdgl;

namespace {

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

struct AdjLayout {
    size_t slot_psi, slot_mu, slot_bytes;
    int nck, nseg;
    size_t ck, seg, fin, psibar, gv, lam0, lam1, mubar, au, ar, total;
};

int adj_validate(const tdgl_handle *h, const tdgl_adjoint_config *a)
{
    if (!h || !a) return TDGL_ERR_INVALID_ARG;
    if (a->n_steps < 1 || a->checkpoint_every < 1 || a->window_start < 0 || a->window_start >= a->n_steps)
        return TDGL_ERR_INVALID_ARG;
    if (a->adj_max_iter < 1 || !(a->adj_eps > 0) || a->poisson_cycles < 1) return TDGL_ERR_INVALID_ARG;
    if (h->cfg.bc[0] != TDGL_OPEN || h->g.L != nullptr || h->lk || !adj_supported(h->g) || h->cfg.freeze_mu_K)
        return TDGL_ERR_INVALID_ARG;
    return TDGL_OK;
}

AdjLayout adj_layout(const tdgl_handle *h, const tdgl_adjoint_config *a)
{
    AdjLayout L;
    const size_t N = (size_t)h->g.N;
    L.slot_psi = al256(8 * N);
    L.slot_mu = al256(4 * N);
    // psi, mu and, where the Poisson guess is extrapolated, the previous step's mu
    L.slot_bytes = L.slot_psi + L.slot_mu + (handle_extrapolates(h) ? al256(4 * N) : 0);
    L.nck = (a->n_steps + a->checkpoint_every - 1) / a->checkpoint_every;
    L.nseg = a->checkpoint_every + 1;
    size_t off = 0;
    L.ck = off;
    off += L.slot_bytes * (size_t)L.nck;
    L.seg = off;
    off += L.slot_bytes * (size_t)L.nseg;
    L.fin = off;
    off += L.slot_bytes;
    L.psibar = off;
    off += al256(8 * N);
    L.gv = off;
    off += al256(8 * N);
    L.lam0 = off;
    off += al256(8 * N);
    L.lam1 = off;
    off += al256(8 * N);
    L.mubar = off;
    off += al256(4 * N);
    L.au = off;
    off += al256(4 * N);
    L.ar = off;
    off += al256(4 * N);
    L.total = off;
    return L;
}

int sync_ctl(tdgl_handle *h, DevCtl *out)
{
    if (cudaMemcpyAsync(out, h->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
        return TDGL_ERR_CUDA;
    return cudaStreamSynchronize(h->stream) == cudaSuccess ? TDGL_OK : TDGL_ERR_CUDA;
}

}  // namespace

extern "C" size_t tdgl_adjoint_workspace_bytes(const tdgl_handle *h, const tdgl_adjoint_config *acfg)
{
    if (adj_validate(h, acfg) != TDGL_OK) return 0;
    return adj_layout(h, acfg).total;
}

extern "C" int tdgl_adjoint(tdgl_handle *h, const tdgl_adjoint_config *acfg, void *d_ws, size_t ws_bytes,
                            float *d_grad_alpha, double *objective, tdgl_adjoint_stats *stats)
{
    if (h && h->res_pending) {   // resident steps enqueued: finish and account for them first
        const int rs = resident_sync(h);
        if (rs != TDGL_OK) return rs;
    }
    int rc = adj_validate(h, acfg);
    if (rc != TDGL_OK) return rc;
    // the reverse pass assumes a deterministic forward without noise
    if (!d_grad_alpha || h->batch_owned || h->noise_amp != 0.f) return TDGL_ERR_INVALID_ARG;
    // every stored state holds its own projected mu: apply the pending projections now and
    // project at once inside (the captured Poisson graphs are recaptured either way)
    if ((rc = mu_materialize(h, 0)) != TDGL_OK || (rc = mu_materialize(h, 1)) != TDGL_OK) return rc;
    drop_poisson_graphs(h);
    h->in_adjoint = 1;
    struct Leave {
        tdgl_handle *h;
        ~Leave()
        {
            h->in_adjoint = 0;
            drop_poisson_graphs(h);
        }
    } leave{h};
    const tdgl_adjoint_config &A = *acfg;
    const AdjLayout L = adj_layout(h, acfg);
    if (!d_ws || ((uintptr_t)d_ws & 255u) || ws_bytes < L.total) return TDGL_ERR_WORKSPACE;
    char *ws = static_cast<char *>(d_ws);
    const DevGrid &g = h->g;
    const size_t N = (size_t)g.N;
    cudaStream_t s = h->stream;
    const int T = A.n_steps, C = A.checkpoint_every;
    auto slot_psi = [&](size_t base, int q) { return reinterpret_cast<float2 *>(ws + base + L.slot_bytes * (size_t)q); };
    auto slot_mu = [&](size_t base, int q) {
        return reinterpret_cast<float *>(ws + base + L.slot_bytes * (size_t)q + L.slot_psi);
    };
    // with the extrapolated Poisson guess a state also holds the previous step's mu (and
    // whether there is one), so that a recomputed step repeats the forward one exactly
    const bool ex = handle_extrapolates(h);
    auto slot_mup = [&](size_t base, int q) {
        return reinterpret_cast<float *>(ws + base + L.slot_bytes * (size_t)q + L.slot_psi + L.slot_mu);
    };
    std::vector<char> pv_ck((size_t)L.nck), pv_seg((size_t)L.nseg), pv_fin(1);
    auto pv_of = [&](size_t base) -> std::vector<char> & {
        return base == L.ck ? pv_ck : (base == L.seg ? pv_seg : pv_fin);
    };
    auto save = [&](size_t base, int q) -> int {
        if (cudaMemcpyAsync(slot_psi(base, q), h->psi[h->cur], 8 * N, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return TDGL_ERR_CUDA;
        if (cudaMemcpyAsync(slot_mu(base, q), h->mu, 4 * N, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return TDGL_ERR_CUDA;
        if (ex) {
            if (cudaMemcpyAsync(slot_mup(base, q), h->mu_buf[1 - h->mu_q], 4 * N, cudaMemcpyDeviceToDevice, s) !=
                cudaSuccess)
                return TDGL_ERR_CUDA;
            pv_of(base)[(size_t)q] = (char)h->prev_valid;
        }
        return TDGL_OK;
    };
    auto restore = [&](size_t base, int q) -> int {
        if (cudaMemcpyAsync(h->psi[h->cur], slot_psi(base, q), 8 * N, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return TDGL_ERR_CUDA;
        if (cudaMemcpyAsync(h->mu, slot_mu(base, q), 4 * N, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return TDGL_ERR_CUDA;
        if (ex) {
            if (cudaMemcpyAsync(h->mu_buf[1 - h->mu_q], slot_mup(base, q), 4 * N, cudaMemcpyDeviceToDevice, s) !=
                cudaSuccess)
                return TDGL_ERR_CUDA;
            h->prev_valid = pv_of(base)[(size_t)q];
            h->guess_ready = 0;
        }
        return TDGL_OK;
    };
    float2 *psibar = reinterpret_cast<float2 *>(ws + L.psibar);
    float2 *gv = reinterpret_cast<float2 *>(ws + L.gv);
    float2 *lam[2] = {reinterpret_cast<float2 *>(ws + L.lam0), reinterpret_cast<float2 *>(ws + L.lam1)};
    float *mubar = reinterpret_cast<float *>(ws + L.mubar);
    float *au = reinterpret_cast<float *>(ws + L.au);
    float *ar = reinterpret_cast<float *>(ws + L.ar);

    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return TDGL_ERR_CUDA;
    tdgl_adjoint_stats st;
    memset(&st, 0, sizeof(st));
    auto elapsed = [&]() {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        return (double)ms;
    };
    auto fail = [&](int code) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return code;
    };

    // ---- forward pass with checkpoints
    double sumEx = 0.0;
    cudaEventRecord(e0, s);
    for (int n = 0; n < T; ++n) {
        if (n % C == 0 && (rc = save(L.ck, n / C)) != TDGL_OK) return fail(rc);
        if ((rc = tdgl_step(h, 1)) != TDGL_OK) return fail(rc);
        DevCtl c;
        if ((rc = sync_ctl(h, &c)) != TDGL_OK) return fail(rc);
        if (n + 1 > A.window_start) sumEx += c.Ex;
    }
    if ((rc = save(L.fin, 0)) != TDGL_OK) return fail(rc);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    st.ms_forward = elapsed();
    const int nwin = T - A.window_start;
    if (objective) *objective = sumEx / nwin;

    // ---- reverse pass
    if (cudaMemsetAsync(psibar, 0, 8 * N, s) != cudaSuccess || cudaMemsetAsync(mubar, 0, 4 * N, s) != cudaSuccess ||
        cudaMemsetAsync(au, 0, 4 * N, s) != cudaSuccess || cudaMemsetAsync(d_grad_alpha, 0, 4 * N, s) != cudaSuccess)
        return fail(TDGL_ERR_CUDA);
    const float vsrc = (float)(1.0 / ((double)nwin * g.ny * g.nz * (g.nx - 1) * h->cfg.hx));
    PoissonArgs pa = h->pa;
    pa.mu_q = -1;   // not one of the handle's mu buffers
    pa.lev[0].u = au;
    pa.lev[0].r = ar;
    pa.mu = au;
    pa.f = ar;
    const float2 Ux0 = make_float2(1.f, 0.f);   // open x: K = 0
    // the fixed adjoint Poisson sequence (right-hand side, V-cycles, projection) on stream q
    auto adj_poisson_fixed = [&](cudaStream_t q) -> cudaError_t {
        cudaError_t e = launch_adj_rhs(g, mubar, ar, h->ctl, h->blockred, h->wsum, q);
        long long nl = 0;
        for (int c = 0; c < A.poisson_cycles && e == cudaSuccess; ++c) e = launch_vcycle(pa, q, &nl);
        if (e == cudaSuccess) e = launch_project_mu(pa, q);
        return e;
    };
    cudaGraphExec_t rgraph = nullptr;
    bool graph_fail = false;
    long long rev_solves = 0;
    cudaStream_t cap = nullptr;
    if (A.poisson_tol <= 0 && cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) {
        cap = nullptr;
        graph_fail = true;
    }
    struct GraphGuard {
        cudaGraphExec_t *g;
        cudaStream_t *c;
        ~GraphGuard()
        {
            if (*g) cudaGraphExecDestroy(*g);
            if (*c) cudaStreamDestroy(*c);
        }
    } graph_guard{&rgraph, &cap};
    for (int c = L.nck - 1; c >= 0; --c) {
        const int s0 = c * C, s1 = (s0 + C < T) ? s0 + C : T;
        cudaEventRecord(e0, s);
        if ((rc = restore(L.ck, c)) != TDGL_OK || (rc = save(L.seg, 0)) != TDGL_OK) return fail(rc);
        for (int n = s0 + 1; n <= s1; ++n) {
            if ((rc = tdgl_step(h, 1)) != TDGL_OK) return fail(rc);
            if ((rc = save(L.seg, n - s0)) != TDGL_OK) return fail(rc);
        }
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        st.ms_recompute += elapsed();
        cudaEventRecord(e0, s);
        for (int n = s1; n > s0; --n) {
            const float2 *psi_n = slot_psi(L.seg, n - s0), *psi_p = slot_psi(L.seg, n - 1 - s0);
            const float *mu_p = slot_mu(L.seg, n - 1 - s0);
            if (n > A.window_start && launch_adj_voltage_source(g, mubar, vsrc, s) != cudaSuccess)
                return fail(TDGL_ERR_CUDA);
            // adjoint Poisson: w = W * G(mubar / W); with a fixed number of V-cycles the whole
            // sequence is replayed from a graph from the second reverse step on (the first runs
            // the launches directly, which also sets the kernels' one-time attributes)
            const bool replay = A.poisson_tol <= 0 && !graph_fail && rev_solves++ > 0;
            if (replay) {
                if (!rgraph) {
                    cudaGraph_t gr = nullptr;
                    cudaError_t e1 = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
                    cudaError_t e2 = (e1 == cudaSuccess) ? adj_poisson_fixed(cap) : e1;
                    cudaError_t e3 = (e1 == cudaSuccess) ? cudaStreamEndCapture(cap, &gr) : e1;
                    if (e2 != cudaSuccess || e3 != cudaSuccess || !gr ||
                        cudaGraphInstantiate(&rgraph, gr, 0) != cudaSuccess) {
                        rgraph = nullptr;
                        graph_fail = true;
                        cudaGetLastError();
                    }
                    if (gr) cudaGraphDestroy(gr);
                }
                if (rgraph && cudaGraphLaunch(rgraph, s) != cudaSuccess) return fail(TDGL_ERR_CUDA);
            }
            if (!replay || graph_fail) {
                if (launch_adj_rhs(g, mubar, ar, h->ctl, h->blockred, h->wsum, s) != cudaSuccess)
                    return fail(TDGL_ERR_CUDA);
                long long nl = 0;
                int cycles = 0;
                for (; cycles < A.poisson_cycles; ++cycles)
                    if (launch_vcycle(pa, s, &nl) != cudaSuccess) return fail(TDGL_ERR_CUDA);
                if (A.poisson_tol > 0) {
                    for (;;) {
                        if (launch_poisson_residual(pa, s) != cudaSuccess) return fail(TDGL_ERR_CUDA);
                        DevCtl cc;
                        if ((rc = sync_ctl(h, &cc)) != TDGL_OK) return fail(rc);
                        if (cc.res <= A.poisson_tol || cycles >= h->cfg.poisson_max_cycles) break;
                        if (launch_vcycle(pa, s, &nl) != cudaSuccess) return fail(TDGL_ERR_CUDA);
                        ++cycles;
                    }
                }
                if (launch_project_mu(pa, s) != cudaSuccess) return fail(TDGL_ERR_CUDA);
            }
            // g = psibar + i [NS^H(w psi^n) - w NS(psi^n)]
            if (launch_adj_fterm(g, Ux0, psi_n, au, psibar, gv, s) != cudaSuccess) return fail(TDGL_ERR_CUDA);
            // M^H lam = g
            if (launch_adj_diag(g, psi_p, mu_p, h->cfg.d_alpha, gv, h->D, lam[0], s) != cudaSuccess)
                return fail(TDGL_ERR_CUDA);
            int zero3[3] = {0, 0, 0};   // iter, done, status
            if (cudaMemcpyAsync(&h->ctl->iter, zero3, sizeof(zero3), cudaMemcpyHostToDevice, s) != cudaSuccess)
                return fail(TDGL_ERR_CUDA);
            SweepArgs sa;
            memset(&sa, 0, sizeof(sa));
            sa.g = g;
            sa.ctl = h->ctl;
            sa.blockred = h->blockred;
            sa.b = gv;
            sa.D = h->D;
            sa.check_every = 1;
            sa.fixed_sweeps = 0;
            sa.max_iter = A.adj_max_iter;
            sa.eps = A.adj_eps;
            sa.rel_eps = 1;
            int launched = 0, batch = 6;
            DevCtl cc;
            for (;;) {
                int nb = batch;
                if (launched + nb > A.adj_max_iter) nb = A.adj_max_iter - launched;
                for (int q = 0; q < nb; ++q, ++launched) {
                    sa.src = lam[launched & 1];
                    sa.dst = lam[(launched + 1) & 1];
                    sa.dst_index = (launched + 1) & 1;
                    if (launch_adj_sweep(sa, s) != cudaSuccess) return fail(TDGL_ERR_CUDA);
                }
                if ((rc = sync_ctl(h, &cc)) != TDGL_OK) return fail(rc);
                if (cc.done || launched >= A.adj_max_iter) break;
                batch = 4;
            }
            if (cc.status != TDGL_OK) return fail(cc.status);
            if (!cc.done) return fail(TDGL_ERR_NOT_CONVERGED);
            st.adjoint_sweeps += cc.iter;
            if (launch_adj_update(g, lam[cc.result], psi_n, psi_p, gv, d_grad_alpha, mubar, psibar, s) != cudaSuccess)
                return fail(TDGL_ERR_CUDA);
        }
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        st.ms_reverse += elapsed();
    }
    if ((rc = restore(L.fin, 0)) != TDGL_OK) return fail(rc);
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(TDGL_ERR_CUDA);
    if (stats) *stats = st;
    return fail(TDGL_OK);
}
