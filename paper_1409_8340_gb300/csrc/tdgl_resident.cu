// The device-resident time step: the kernel loop of Sec. 4.1 (Jacobi sweeps until the
// convergence test, then the Poisson solve) for any number of steps as ONE CUDA graph,
// with no host round trip between sweeps or between steps.
//
// The host-driven step (tdgl_step) reads the control block after a batch of sweeps to
// learn whether the Jacobi solve converged and which psi buffer holds its result.  Here
// those decisions stay on the device and steer conditional graph nodes:
//
//   WHILE (steps left, status OK)                         outer loop, one step per pass
//     SWITCH on the state's (psi buffer c, mu buffer q):
//       init sweep psi[c] -> psi[c+1]  (Eq. 10 right-hand side, first sweep, Poisson
//       guess of Sec. 3.2 over mu buffer 1 - q)
//       WHILE (not decided)  sweep c+1 -> c+2, sweep c+2 -> c+1
//     SWITCH on the (result buffer r, mu buffer of the solve q'), none after a failure:
//       [K ODE, Eq. K_ODE]  Poisson right-hand side, V-cycles, projection  [voltage, Sec. 2.3]
//     step end: the result becomes the state; next step or stop
//
// Every launch in the branches is the one the host-driven step makes (same kernels, same
// arguments), so the two paths give the same bits.  The convergence decision is the
// sweep kernels' own (Eq. 11 tested by their last block), and the block that takes it
// also sets the sweep loop's condition and, when the solve ends, the tail's branch; a
// sweep after the deciding one returns at once and clears the loop condition.  Both loops
// are bounded: the sweep loop by the decision itself, which ends every solve by max_iter
// sweeps (not converged), the step loop by a counter of the steps asked for in the
// control block.
#include "tdgl_internal.cuh"

#include <cstddef>
#include <cstring>

using namespace tdgl;

namespace {

// the SWITCH node of the step's solve: the branch of the state's psi buffer and mu buffer
// (b + 3 q when the mu buffers swap every step, else b), none once a failure has halted
// the enqueued steps; the tail's SWITCH runs nothing until a solve ends successfully
__global__ void res_select_state(DevCtl *c, cudaGraphConditionalHandle hs, cudaGraphConditionalHandle ht, int flip)
{
    cudaGraphSetConditional(hs, c->rhalt ? kNoBranch : (unsigned int)(c->rcur + (flip ? 3 * c->rq : 0)));
    cudaGraphSetConditional(ht, kNoBranch);
    c->rok = 0;
}

__global__ void res_step_end(DevCtl *c, cudaGraphConditionalHandle ho, int flip)
{
    // a failed Jacobi solve leaves the state as it was (the tail did not run); a failure in
    // the tail (a Poisson wait that timed out) ends the loop after the step
    bool go = false;
    if (c->rhalt) {
        cudaGraphSetConditional(ho, 0u);
        return;
    }
    c->rloops += c->iter / 2;   // passes of the sweep loop after the init's sweep
    if (c->rok) {
        c->rcur = c->result;
        if (flip) c->rq = 1 - c->rq;
        c->rdone += 1;
        c->rsweeps += c->iter;
        c->rlast = c->iter;
        c->rleft -= 1;
        go = c->rleft > 0 && c->status == TDGL_OK;
    }
    if (!c->rok || c->status != TDGL_OK) c->rhalt = 1;
    cudaGraphSetConditional(ho, go ? 1u : 0u);
}

// append a conditional node with n bodies after everything captured so far on s; its
// body graphs out
cudaError_t cap_cond(cudaStream_t s, cudaGraph_t g, cudaGraphConditionalHandle hd, cudaGraphConditionalNodeType t,
                     cudaGraph_t *body, unsigned int n = 1)
{
    cudaStreamCaptureStatus st;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(s, &st, nullptr, nullptr, &deps, nullptr, &nd);
    if (e != cudaSuccess) return e;
    if (st != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = hd;
    p.conditional.type = t;
    p.conditional.size = n;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &p);
    if (e != cudaSuccess) return e;
    for (unsigned int i = 0; i < n; ++i) body[i] = p.conditional.phGraph_out[i];
    return cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

struct Builder {
    tdgl_handle *h;
    cudaStream_t s[3];
    long long tail_launches;
    cudaGraphConditionalHandle htail;   // the SWITCH node of the step's tail

    cudaError_t sweep(SweepArgs a, int src, int dst, cudaStream_t st)
    {
        a.src = h->psi[src];
        a.dst = h->psi[dst];
        a.dst_index = dst;
        return h->use_tma ? launch_sweep_tma(a, h->tmaps.psi[src], h->tmaps, st) : launch_sweep(a, st);
    }

    // branch (c, q): init sweep and the sweep loop; the deciding sweep selects the tail
    // branch tail_base + result
    cudaError_t solve_branch(cudaGraph_t g, int c, int q, int tail_base)
    {
        cudaStream_t st = s[1];
        cudaError_t e = cudaStreamBeginCaptureToGraph(st, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        const int ia = (c + 1) % 3, ib = (c + 2) % 3;
        SweepArgs a = step_sweep_args(h);
        a.mu = h->mu_buf[q];   // the state's potential, which the sweeps read (Eq. 10)
        a.src = h->psi[c];
        a.dst = h->psi[ia];
        a.dst_index = ia;
        a.mu_off = &h->ctl->mu_off[q];
        if (handle_extrapolates(h)) step_guess_args(h, a, q);
        // the sweeps' deciding block sets the loop's condition (the init's decision the first)
        cudaGraphConditionalHandle hw;
        e = cudaGraphConditionalHandleCreate(&hw, g, 0, 0);
        a.loop_cond = hw;
        a.has_loop = 1;
        a.tail_cond = htail;
        a.tail_base = tail_base;
        if (e == cudaSuccess) e = launch_init_sweep(a, st, h->use_tma != 0);
        a.mu_guess = nullptr;
        a.mu_off = a.mu_off_prev = nullptr;
        cudaGraph_t wb = nullptr;
        if (e == cudaSuccess) e = cap_cond(st, g, hw, cudaGraphCondTypeWhile, &wb);
        if (e == cudaSuccess) {
            cudaStream_t sw = s[2];
            e = cudaStreamBeginCaptureToGraph(sw, wb, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaError_t e1 = sweep(a, ia, ib, sw);
                if (e1 == cudaSuccess) e1 = sweep(a, ib, ia, sw);
                cudaGraph_t out = nullptr;
                e = cudaStreamEndCapture(sw, &out);
                if (e1 != cudaSuccess) e = e1;
            }
        }
        cudaGraph_t out = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(st, &out);
        return e != cudaSuccess ? e : ee;
    }

    // branch (r, q): what the host-driven step runs after the Jacobi solve, with psi[r]
    // the solution and mu buffer q the Poisson solve's
    cudaError_t tail_branch(cudaGraph_t g, int r, int q)
    {
        cudaStream_t st = s[1];
        cudaError_t e = cudaStreamBeginCaptureToGraph(st, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        const tdgl_config &c = h->cfg;
        const int cur0 = h->cur, q0 = h->mu_q;
        h->cur = r;
        use_mu_buffer(h, q);
        long long nl = 0;
        if (c.bc[0] == TDGL_PERIODIC) {
            KArgs k;
            k.g = h->g;
            k.ctl = h->ctl;
            k.blockred = h->blockred;
            k.psi = h->psi[r];
            k.hx = c.hx;
            k.dtK = h->dtK;
            k.Jext = c.Jext;
            k.update_K = c.freeze_mu_K ? 0 : 1;
            e = launch_javg_K(k, st);
            nl += 1;
        }
        if (e == cudaSuccess && !c.freeze_mu_K) nl += step_poisson_sequence(h, st, &e);
        if (e == cudaSuccess && c.bc[0] == TDGL_OPEN) {
            e = launch_voltage(h->pa, st);
            nl += 1;
        }
        h->cur = cur0;
        use_mu_buffer(h, q0);
        tail_launches = nl;
        cudaGraph_t out = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(st, &out);
        return e != cudaSuccess ? e : ee;
    }

    cudaError_t build(cudaGraph_t top)
    {
        const bool flip = handle_extrapolates(h);
        cudaGraphConditionalHandle ho;
        cudaError_t e = cudaGraphConditionalHandleCreate(&ho, top, 1, cudaGraphCondAssignDefault);
        if (e != cudaSuccess) return e;
        cudaGraphNodeParams p = {};
        p.type = cudaGraphNodeTypeConditional;
        p.conditional.handle = ho;
        p.conditional.type = cudaGraphCondTypeWhile;
        p.conditional.size = 1;
        cudaGraphNode_t on;
        e = cudaGraphAddNode(&on, top, nullptr, nullptr, 0, &p);
        if (e != cudaSuccess) return e;
        cudaGraph_t ob = p.conditional.phGraph_out[0];
        cudaStream_t so = s[0];
        e = cudaStreamBeginCaptureToGraph(so, ob, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        // the mu buffers a state can be in: both when each step swaps them, else the current
        // one; body b + 3 t of either SWITCH is psi buffer b with the t-th of them
        const int nq = flip ? 2 : 1;
        const int qs[2] = {flip ? 0 : h->mu_q, 1};
        cudaGraphConditionalHandle hsel;
        e = cudaGraphConditionalHandleCreate(&hsel, ob, 0, 0);
        if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&htail, ob, 0, 0);
        if (e == cudaSuccess) {
            res_select_state<<<1, 1, 0, so>>>(h->ctl, hsel, htail, flip ? 1 : 0);
            e = cudaGetLastError();
        }
        cudaGraph_t body[6] = {};
        if (e == cudaSuccess) e = cap_cond(so, ob, hsel, cudaGraphCondTypeSwitch, body, 3 * nq);
        for (int t = 0; t < nq && e == cudaSuccess; ++t)
            for (int c = 0; c < 3 && e == cudaSuccess; ++c)
                // the solve of a step from mu buffer q runs in the other one when they swap
                e = solve_branch(body[c + 3 * t], c, qs[t], flip ? 3 * (1 - t) : 0);
        if (e == cudaSuccess) e = cap_cond(so, ob, htail, cudaGraphCondTypeSwitch, body, 3 * nq);
        for (int t = 0; t < nq && e == cudaSuccess; ++t)
            for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = tail_branch(body[r + 3 * t], r, qs[t]);
        if (e == cudaSuccess) {
            res_step_end<<<1, 1, 0, so>>>(h->ctl, ho, flip ? 1 : 0);
            e = cudaGetLastError();
        }
        cudaGraph_t out = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(so, &out);
        return e != cudaSuccess ? e : ee;
    }
};

int build_resident(tdgl_handle *h)
{
    Builder B;
    memset(&B, 0, sizeof(B));
    B.h = h;
    for (int i = 0; i < 3; ++i)
        if (cudaStreamCreateWithFlags(&B.s[i], cudaStreamNonBlocking) != cudaSuccess) {
            for (int j = 0; j < i; ++j) cudaStreamDestroy(B.s[j]);
            return TDGL_ERR_CUDA;
        }
    cudaGraph_t top = nullptr;
    cudaError_t e = cudaGraphCreate(&top, 0);
    if (e == cudaSuccess) e = B.build(top);
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, top, 0);
    if (top) cudaGraphDestroy(top);
    for (int i = 0; i < 3; ++i) cudaStreamDestroy(B.s[i]);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return TDGL_ERR_CUDA;
    }
    h->rgraph = exec;
    // per step outside the sweep loop: state select, init, tail, step end
    h->rgraph_launches = 3 + B.tail_launches;
    return TDGL_OK;
}

}  // namespace

// Enqueue n resident steps (n >= 1) on the handle's stream; the first step after creation
// or a state load runs launch by launch first.  Steps enqueued while others are pending
// continue from their device state (the host has not accounted for them yet).
static int resident_enqueue(tdgl_handle *h, int n)
{
    // the first step after creation or a state load runs launch by launch: it sets the
    // kernels' one-time attributes outside a capture and leaves a previous mu to extrapolate from
    while (n > 0 && !h->res_pending && (!h->stepped || (handle_extrapolates(h) && !h->prev_valid))) {
        const int rc = tdgl_step(h, 1);
        if (rc != TDGL_OK) return rc;
        --n;
    }
    if (n == 0) return TDGL_OK;
    // a driver that cannot build the graph runs the same launches from the host
    if (!h->rgraph && !h->rgraph_fail && build_resident(h) != TDGL_OK) h->rgraph_fail = 1;
    if (h->rgraph_fail) {
        const int rc = resident_sync(h);
        return rc != TDGL_OK ? rc : tdgl_step(h, n);
    }
    cudaStream_t s = h->stream;
    if (h->res_pending) {
        // after the pending steps (stream order): n more; the counters keep accumulating
        if (cudaMemcpyAsync(&h->ctl->rleft, &n, sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess)
            return TDGL_ERR_CUDA;
    } else {
        // the loop's part of the control block: state buffers, steps to run, counters cleared
        struct {
            int rcur, rq, rleft, rdone, rspare, rlast, rok, rhalt;
            long long rsweeps, rloops;
        } r = {h->cur, h->mu_q, n, 0, 0, h->last_sweeps, 0, 0, 0, 0};
        static_assert(sizeof(r) == offsetof(DevCtl, rloops) + sizeof(long long) - offsetof(DevCtl, rcur), "layout");
        if (cudaMemcpyAsync(&h->ctl->rcur, &r, sizeof(r), cudaMemcpyHostToDevice, s) != cudaSuccess)
            return TDGL_ERR_CUDA;
    }
    // (a copy from pageable host memory is staged before the call returns: the stack values
    // above may go)
    if (cudaGraphLaunch(h->rgraph, s) != cudaSuccess) return TDGL_ERR_CUDA;
    h->res_pending = 1;
    h->guess_ready = 0;
    return TDGL_OK;
}

namespace tdgl {

int resident_sync(tdgl_handle *h)
{
    if (!h->res_pending) return TDGL_OK;
    h->res_pending = 0;
    const tdgl_config &c = h->cfg;
    DevCtl ctl;
    const int rc = step_read_ctl(h, &ctl);
    if (rc != TDGL_OK) return rc;
    const int done = ctl.rdone;
    if (done > 0) {
        h->cur = ctl.rcur;
        if (ctl.rq != h->mu_q) use_mu_buffer(h, ctl.rq);
        h->last_sweeps = ctl.rlast;
        h->step += done;
        h->prof.steps += done;
        if (!c.freeze_mu_K) {
            h->mu_solved = 1;
            h->last_cycles = c.poisson_cycles;
            h->prof.vcycles += (long long)c.poisson_cycles * done;
            // the solves leave their means pending in the state (and, after two steps, in the
            // previous mu)
            const int lazy = step_lazy_projection(h) ? 1 : 0;
            h->mu_pend[h->mu_q] = lazy;
            if (handle_extrapolates(h)) {
                if (done >= 2) h->mu_pend[1 - h->mu_q] = lazy;
                h->prev_valid = 1;
            }
        }
    }
    h->prof.sweeps += ctl.rsweeps;
    h->prof.sweep_launches += 2 * ctl.rloops + done;
    h->prof.kernel_launches += 2 * ctl.rloops + (long long)done * h->rgraph_launches;
    if (!ctl.rhalt) return TDGL_OK;
    if (handle_extrapolates(h)) {
        // a failed step's init has written the Poisson guess over the previous mu: a retry
        // starts afresh (as after tdgl_step), and that buffer holds no pending mean
        h->prev_valid = 0;
        h->mu_pend[1 - h->mu_q] = 0;
    }
    return ctl.status != TDGL_OK ? ctl.status : TDGL_ERR_NOT_CONVERGED;
}

}  // namespace tdgl

extern "C" {

static bool resident_covers(const tdgl_handle *h)
{
    const tdgl_config &c = h->cfg;
    return !h->batch_owned && !h->slab && !h->poisson_only && !h->lk && c.poisson_tol <= 0 && c.fixed_sweeps <= 0 &&
           !step_pairs(h);
}

int tdgl_step_resident(tdgl_handle *h, int32_t n_steps)
{
    if (!h || n_steps < 0 || !resident_covers(h)) return TDGL_ERR_INVALID_ARG;
    if (n_steps > 0) {
        const int rc = resident_enqueue(h, n_steps);
        if (rc != TDGL_OK) return rc;
    }
    return resident_sync(h);
}

int tdgl_step_enqueue(tdgl_handle *h, int32_t n_steps)
{
    if (!h || n_steps < 0 || !resident_covers(h)) return TDGL_ERR_INVALID_ARG;
    return n_steps > 0 ? resident_enqueue(h, n_steps) : TDGL_OK;
}

int tdgl_sync(tdgl_handle *h)
{
    if (!h) return TDGL_ERR_INVALID_ARG;
    const int rc = resident_sync(h);
    if (rc != TDGL_OK) return rc;
    return cudaStreamSynchronize(h->stream) == cudaSuccess ? TDGL_OK : TDGL_ERR_CUDA;
}

}  // extern "C"
