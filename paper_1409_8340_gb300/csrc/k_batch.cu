// Batched persistent step: one cooperative launch advances every instance of a
// batch by one full time step (Sec. 3.1 implicit psi solve with its per-sweep
// convergence test, Sec. 2.2 K ODE, Sec. 3.2 Poisson solve).  The launch walks
// a fixed sequence of phases; in each phase the blocks share out the work items
// (instance, tile) of the instances taking part, and a grid barrier ends the
// phase.  The Jacobi phases repeat while any instance is still iterating: the
// last tile of an instance to finish a sweep reduces that instance's residual
// maxima and decides (the same decision as the per-instance kernels), so
// converged instances drop out while the others go on.
//
// All loads of arrays written earlier in the same launch go through L2
// (ld.global.cg): the non-coherent path is never used for them.
#include <float.h>
#include <stddef.h>
#include <string.h>

#include "mg_tile.cuh"
#include "staged_tile.cuh"
#include "sweep_tile.cuh"

namespace tdgl {

constexpr int kBT = kBX * kBY;   // threads per block
constexpr int kFlat = 1024;      // sites per flat work item (4 per thread)
constexpr int kQ = 4;            // site quads per thread in a prolongation item
constexpr int kFlatQ = 4 * kQ * kBX * kBY;   // sites per prolongation item

enum BatchOp {
    OP_INIT,
    OP_SWEEP,
    OP_JAVG,
    OP_RHS,
    OP_SMOOTH,
    OP_RESID,      // (a phase-log kind no phase has: the residual is formed inside the restriction)
    OP_RESTRICT,
    OP_CFWD,
    OP_CCONV,
    OP_CINV,
    OP_PROLONG,
    OP_MEAN,
    OP_SHIFT
};

struct BatchSmem {
    int start[kBatchMax + 1];   // exclusive prefix of the phase's item counts
    int cnt[kBatchMax];
    int active[kBatchMax];      // instance takes part in the current Jacobi phase
    int ok[kBatchMax];          // instance finished its Jacobi solve without error
    int alive[kBatchMax];       // instance not stopped by an earlier error
    BatchHead H;
    MGLevel L0, L1;
    int cached;                 // instance whose head is in H (-1: none)
    int flag;
    int cw;                     // barrier count word of this launch: bar[0] (psi solve), bar[2] (mu solve)
    unsigned int log0;          // phase-log index of this launch's start
    int grab;                   // the item this block took last (dynamic phases)
    unsigned short order[kBatchMax];   // instances in dealing order (copied from P.order)
    int split;                  // sweep phases: z parts per tile (1, or 2 or 4 when the phase has few tiles)
};

__device__ __forceinline__ int btid() { return threadIdx.x + kBX * threadIdx.y; }

__device__ __forceinline__ unsigned long long gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void copy_words(void *dst, const void *src, int bytes)
{
    int *d = reinterpret_cast<int *>(dst);
    const int *s = reinterpret_cast<const int *>(src);
    for (int w = btid(); w < bytes / 4; w += kBT) d[w] = s[w];
}

// Grid barrier with a bounded wait.  Arrivals accumulate in *count over the
// launch (zeroed before it); barrier number nb completes at nb * (grid + extra)
// arrivals.  A wait that passes timeout_ns, or sees the error flag bar[1], sets the
// flag and returns false in every thread of the block.
__device__ __forceinline__ bool grid_barrier(unsigned int *bar, unsigned int *count, unsigned int extra,
                                             unsigned long long timeout_ns, unsigned int nb, int *flag)
{
    __syncthreads();
    if (btid() == 0) {
        const unsigned int target = nb * (gridDim.x + extra);
        volatile unsigned int *cnt = count;
        volatile unsigned int *err = bar + 1;
        __threadfence();
        atomicAdd(count, 1u);
        const unsigned long long t0 = gtimer();
        int good = 1;
        unsigned int back = 32;
        for (;;) {
            if (*cnt >= target) break;
            if (*err != 0u) {
                good = 0;
                break;
            }
            if (gtimer() - t0 > timeout_ns) {
                atomicCAS(bar + 1, 0u, 1u);
                good = 0;
                break;
            }
            __nanosleep(back);
            if (back < 256) back <<= 1;
        }
        __threadfence();
        *flag = good;
    }
    __syncthreads();
    return *flag != 0;
}

// A proper zebra colouring of a level: no two lines of one colour are neighbours across a
// periodic wrap (y and z extents even, or open, or a single line).  Then the
// post-smoothing's first pass (colour 1) solves its lines from F and the colour-0 lines
// alone, and the prolongation needs to correct the colour-0 lines only.
__device__ __forceinline__ bool proper_zebra(const MGLevel &L, int bcy, int bcz)
{
    return (bcy == kOpen || L.ny == 1 || (L.ny & 1) == 0) && (bcz == kOpen || L.nz == 1 || (L.nz & 1) == 0);
}

// Sites the prolongation of level l corrects: the colour-0 lines' under a proper zebra
// colouring, else every site.
__device__ __forceinline__ long long prolong_sites(const BatchInst &I, int l)
{
    const MGLevel &L = I.pa.lev[l];
    return proper_zebra(L, I.h.a.g.bcy, I.h.a.g.bcz) ? I.h.nlines[l][0] * L.nx : L.N;
}

// Work items of instance t in a phase (0: not taking part).
__device__ int items_of(const BatchParams &P, const BatchSmem &S, int t, int op, int l)
{
    const BatchInst &I = P.inst[t];
    switch (op) {
    case OP_INIT: return S.alive[t] ? I.h.tiles : 0;
    case OP_SWEEP: return S.active[t] ? I.h.tiles * min(S.split, I.h.split_max) : 0;
    case OP_JAVG: return (S.ok[t] && I.h.periodic_x) ? I.h.red_items : 0;
    case OP_RHS: return S.ok[t] ? I.h.tiles : 0;
    case OP_MEAN: return (S.ok[t] && (I.h.freeze ? I.h.open_x : !I.h.mean_fused)) ? I.h.red_items : 0;
    case OP_SHIFT: return (S.ok[t] && !I.h.freeze) ? I.h.red_items : 0;
    default: break;
    }
    // multigrid phases: l is the level, or the cycle for the coarsest-level ops
    if (!S.ok[t] || I.h.freeze) return 0;
    const int top = I.h.nlev - 1;
    switch (op) {
    case OP_SMOOTH: {
        const int lev = l >> 1, c = l & 1;
        if (lev >= top) return 0;
        return (int)((I.h.nlines[lev][c] + I.h.lpb[lev] - 1) / I.h.lpb[lev]);
    }
    case OP_PROLONG: return (l < top) ? (int)((prolong_sites(I, l) + kFlatQ - 1) / kFlatQ) : 0;
    case OP_RESTRICT: return (l < top) ? (int)((I.pa.lev[l + 1].N + kFlat - 1) / kFlat) : 0;
    case OP_CFWD:
    case OP_CINV: return (int)(((long long)I.pa.lev[top].M * I.pa.lev[top].nx + kFlat - 1) / kFlat);
    case OP_CCONV: return I.pa.lev[top].M;
    default: return 0;
    }
}

// Item counts and their exclusive prefix for a phase, by dealing position (instance
// S.order[t] at position t); returns the total.
__device__ int build_phase(const BatchParams &P, BatchSmem &S, int op, int l)
{
    __syncthreads();
    if (btid() == 0) S.split = 1;
    __syncthreads();
    for (int pass = 0;; ++pass) {
    for (int t = btid(); t < P.n; t += kBT) S.cnt[t] = items_of(P, S, S.order[t], op, l);
    __syncthreads();
    if (btid() < 32) {
        const int lane = btid();
        const int per = (P.n + 31) / 32;
        int sum = 0;
        for (int q = 0; q < per; ++q) {
            const int t = lane * per + q;
            if (t < P.n) sum += S.cnt[t];
        }
        int incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        int run = incl - sum;
        for (int q = 0; q < per; ++q) {
            const int t = lane * per + q;
            if (t < P.n) {
                S.start[t] = run;
                run += S.cnt[t];
            }
        }
        if (lane == 31) S.start[P.n] = incl;
    }
    __syncthreads();
    // A sweep phase with fewer tiles than twice the blocks (the members still iterating at
    // the end of a solve) splits each tile into 2 or 4 parts along z, so that its last
    // items are short: the phase is counted again with the parts.
    const int total = S.start[P.n];
    if (pass > 0 || op != OP_SWEEP || total >= 2 * (int)gridDim.x || total == 0) break;
    if (btid() == 0) S.split = (2 * total < (int)gridDim.x) ? 4 : 2;
    __syncthreads();
    }
    if (btid() == 0) S.cached = -1;
    __syncthreads();
    return S.start[P.n];
}

// Dealing position holding item `it` (the last t with start[t] <= it; it < total).
__device__ __forceinline__ int find_instance(const BatchSmem &S, int n, int it)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (S.start[mid] <= it) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Stage instance m's head (and the levels op needs) in shared memory and point
// the sweep arguments at the phase's buffers.
__device__ void stage(const BatchParams &P, BatchSmem &S, int m, int op, int l, int parity)
{
    if (S.cached == m) return;
    __syncthreads();
    const BatchInst &I = P.inst[m];
    copy_words(&S.H, &I.h, sizeof(BatchHead));
    int la = -1, lb = -1;
    const int top = I.h.nlev - 1;
    if (op == OP_SMOOTH) la = l >> 1;
    else if (op == OP_RESTRICT || op == OP_PROLONG) {
        la = l;
        lb = l + 1;
    } else if (op == OP_CFWD || op == OP_CCONV || op == OP_CINV) la = top;
    if (la >= 0) copy_words(&S.L0, &I.pa.lev[la], sizeof(MGLevel));
    if (lb >= 0) copy_words(&S.L1, &I.pa.lev[lb], sizeof(MGLevel));
    __syncthreads();
    if (btid() == 0) {
        SweepArgs &a = S.H.a;
        if (op == OP_INIT) {
            a.src = S.H.psi[S.H.iS];
            a.dst = S.H.psi[S.H.iA];
            a.dst_index = S.H.iA;
            if (S.H.mu_solve != a.mu) {
                // the init writes the Poisson guess 2 mu^(n-1) - mu^(n-2) (mu^(n-1) on the
                // first step after a state load) over the previous mu in the solve buffer
                const bool prev = ldx<true>(&a.ctl->mu_prev_ok) != 0;
                a.mu_guess = S.H.mu_solve;
                a.ex_a = prev ? 2.f : 1.f;
                a.ex_b = prev ? -1.f : 0.f;
            }
        } else if (op == OP_SWEEP) {
            // sweep p reads the output of sweep p-1: odd p A -> B, even p B -> A
            const int ia = parity ? S.H.iA : S.H.iB, ib = parity ? S.H.iB : S.H.iA;
            a.src = S.H.psi[ia];
            a.dst = S.H.psi[ib];
            a.dst_index = ib;
        } else if (op == OP_RHS || op == OP_JAVG) {
            a.src = S.H.psi[ldx<true>(&a.ctl->result)];
            a.dst = S.H.psi[S.H.iS];
        }
        S.cached = m;
    }
    __syncthreads();
}

// site (i, j, k) of flat index m on an nx x ny x nz grid
__device__ __forceinline__ void flat_ijk(unsigned int m, int nx, int ny, int &i, int &j, int &k)
{
    const unsigned int r = m / (unsigned int)nx;
    i = (int)(m - r * (unsigned int)nx);
    k = (int)(r / (unsigned int)ny);
    j = (int)(r - (unsigned int)k * (unsigned int)ny);
}

// Im[conj(psi_m) (Ux' psi_{m+x} - conj(Ux'') psi_{m-x})]: the x-link current at
// site m (Sec. 3.1.1, J_av), Landau links with the periodic-x wrap phase.
__device__ __forceinline__ double javg_site(const DevGrid &g, float2 Ux, const float2 *psi, long long m)
{
    int i, j, k;
    flat_ijk((unsigned int)m, g.nx, g.ny, i, j, k);
    const float2 p = ldx<true>(psi + m);
    const long long mp = (i == g.nx - 1) ? m - (g.nx - 1) : m + 1;
    const long long mm = (i == 0) ? m + (g.nx - 1) : m - 1;
    const float2 lf = (i == g.nx - 1) ? cmulc(cmul(g.Py[j], g.Pz[k]), Ux) : Ux;
    const float2 lb = (i == 0) ? cmulc(cmul(g.Py[j], g.Pz[k]), Ux) : Ux;
    const float2 d = csub(cmul(lf, ldx<true>(psi + mp)), cmulc(lb, ldx<true>(psi + mm)));
    return (double)(p.x * d.y - p.y * d.x);
}


__device__ void run_item(const BatchParams &P, BatchSmem &S, float *dsm, int op, int l, int parity, int m, int li)
{
    BatchHead &H = S.H;
    const int tid = btid();
    switch (op) {
    case OP_INIT:
    case OP_SWEEP: {
        // a sweep phase's item is part `part` of `spl` along z of a tile
        const int spl = (op == OP_SWEEP) ? min(S.split, H.split_max) : 1;
        const int tile = li / spl, part = li - tile * spl;
        const int bx = tile % H.gx, r = tile / H.gx;
        const int by = r % H.gy, bz = r / H.gy * spl + part;
        const int kz = H.kz / spl;
        float rmax = 0.f, facc = 0.f;
        if (zlo(H.a.g) + bz * kz >= zhi(H.a.g)) {
            // an empty part of the last z tile
        } else if (op == OP_INIT) {
            // staged init where mu's rows sit on 16-byte boundaries
            if (P.staged && (H.a.g.nx & 3) == 0)
                sweep_staged_tile<1>(H.a, kz, bx, by, bz, rmax, facc, reinterpret_cast<IStage *>(dsm));
            else
                sweep2_body<1, true>(H.a, kz, bx, by, bz, rmax, facc);
        }
        else if (P.staged) sweep_staged_tile<0>(H.a, kz, bx, by, bz, rmax, facc, reinterpret_cast<BStage *>(dsm));
        else sweep2_body<0, true>(H.a, kz, bx, by, bz, rmax, facc);
        if (finish_sweep_at<false>(H.a, rmax, op == OP_INIT, li, H.tiles * spl) && tid == 0)
            P.act[(parity & 1) * P.n + m] = H.a.ctl->done ? 0 : 1;
        break;
    }
    case OP_RHS: {
        const int bx = li % H.gx, r = li / H.gx;
        const int by = r % H.gy, bz = r / H.gy;
        float rmax = 0.f, facc = 0.f;
        if (P.staged) sweep_staged_tile<4>(H.a, H.kz, bx, by, bz, rmax, facc, reinterpret_cast<RStage *>(dsm));
        else sweep2_body<4, true>(H.a, H.kz, bx, by, bz, rmax, facc);
        // the deciding block also clears the sums the finest smoothing passes will accumulate
        if (finish_rhs_sum_at(H.a.ctl, H.a.blockred, (double)facc, H.a.wsum, li, H.tiles) && tid == 0) {
            H.a.ctl->bmean[0] = 0.0;
            H.a.ctl->bmean[1] = 0.0;
        }
        break;
    }
    case OP_JAVG: {
        const DevGrid &g = H.a.g;
        const float2 Ux = ldx<true>(&H.a.ctl->Ux);
        const long long m0 = (long long)li * H.red_chunk;
        const long long m1 = min(m0 + H.red_chunk, g.N);
        double acc = 0.0;
        for (long long q = m0 + tid; q < m1; q += kBT) acc += javg_site(g, Ux, H.a.src, q);
        __shared__ double shd[32];
        double s = block_sum(acc, shd);
        if (tid == 0) H.a.blockred[li] = s;
        if (!last_block(&H.a.ctl->ticket, H.red_items, &S.flag)) break;
        double t = 0.0;
        for (int q = tid; q < H.red_items; q += kBT) t += ((volatile double *)H.a.blockred)[q];
        t = block_sum(t, shd);
        if (tid == 0) {
            H.a.ctl->ticket = 0u;
            k_ode_update(H.a.ctl, t / (2.0 * (double)g.N * H.hx), H.hx, H.dtK, H.Jext, H.freeze ? 0 : 1);
        }
        break;
    }
    case OP_SMOOTH: {
        const int lev = l >> 1, c = l & 1;
        const float fsub = (lev == 0) ? (float)ldx<true>(&H.a.ctl->fmean) : 0.f;
        const DevGrid &g = H.a.g;
        const LineShape sh = line_shape(S.L0.nx, S.L0.kmin, S.L0.kmax, kBT);
        if (parity && lev == 0 && H.mean_fused) {
            // the last cycle's finest passes: each line's new values are final, so their
            // weighted sum and x-face difference (the zero mode, the voltage) are summed here
            float sw = 0.f, sv = 0.f;
            line_smooth_lines<true, true>(S.L0, sh, g.bcx, g.bcy, g.bcz, c, H.nlines[lev][c], fsub, li, tid, kBT,
                                          dsm, &sw, &sv);
            // per warp, without a block barrier: the warp's sums added to the instance's
            for (int o = 16; o > 0; o >>= 1) {
                sw += __shfl_xor_sync(0xffffffffu, sw, o);
                sv += __shfl_xor_sync(0xffffffffu, sv, o);
            }
            if ((tid & 31) == 0) {
                atomicAdd(&H.a.ctl->bmean[0], (double)sw);
                atomicAdd(&H.a.ctl->bmean[1], (double)sv);
            }
            break;
        }
        line_smooth_lines<true>(S.L0, sh, g.bcx, g.bcy, g.bcz, c, H.nlines[lev][c], fsub, li, tid, kBT, dsm);
        break;
    }
    case OP_RESTRICT: {
        // full weighting in (y, z) of the fine residual, formed on the fly (never stored):
        // each coarse site weights the residuals of its fine rows and planes as restrict4_at
        // weights the stored ones, in the same order
        const MGLevel &F = S.L0, &C = S.L1;
        const DevGrid &g = H.a.g;
        const float fsub = (l == 0) ? (float)ldx<true>(&H.a.ctl->fmean) : 0.f;
        const int nk = (F.fz == 2) ? 3 : 1, nj = (F.fy == 2) ? 3 : 1;
        if ((C.nx & 3) == 0) {
            const long long m0 = (long long)li * kFlat + 4 * tid;
            if (m0 < C.N) {
                int i, J, K;
                flat_ijk((unsigned int)m0, C.nx, C.ny, i, J, K);
                float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
                for (int a2 = 0; a2 < nk; ++a2) {
                    const int dk = (nk == 3) ? a2 - 1 : 0;
                    const float wk = (nk == 3) ? (dk == 0 ? 0.5f : 0.25f) : 1.f;
                    const int kf = (F.nz >= 2) ? nb_idx(F.fz * K, dk, F.nz, g.bcz) : 0;
                    for (int b2 = 0; b2 < nj; ++b2) {
                        const int dj = (nj == 3) ? b2 - 1 : 0;
                        const float wj = (nj == 3) ? (dj == 0 ? 0.5f : 0.25f) : 1.f;
                        const int jf = nb_idx(F.fy * J, dj, F.ny, g.bcy);
                        const float4 t = residual4_at<true>(F, g.bcx, g.bcy, g.bcz, fsub, i, jf, kf);
                        acc.x += wk * wj * t.x;
                        acc.y += wk * wj * t.y;
                        acc.z += wk * wj * t.z;
                        acc.w += wk * wj * t.w;
                    }
                }
                *reinterpret_cast<float4 *>(C.r + m0) = acc;
                *reinterpret_cast<float4 *>(C.u + m0) = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            break;
        }
#pragma unroll 1
        for (int r = 0; r < kFlat / kBT; ++r) {
            const long long mm = (long long)li * kFlat + r * kBT + tid;
            if (mm >= C.N) break;
            int i, J, K;
            flat_ijk((unsigned int)mm, C.nx, C.ny, i, J, K);
            float acc = 0.f;
            for (int a2 = 0; a2 < nk; ++a2) {
                const int dk = (nk == 3) ? a2 - 1 : 0;
                const float wk = (nk == 3) ? (dk == 0 ? 0.5f : 0.25f) : 1.f;
                const int kf = (F.nz >= 2) ? nb_idx(F.fz * K, dk, F.nz, g.bcz) : 0;
                for (int b2 = 0; b2 < nj; ++b2) {
                    const int dj = (nj == 3) ? b2 - 1 : 0;
                    const float wj = (nj == 3) ? (dj == 0 ? 0.5f : 0.25f) : 1.f;
                    const int jf = nb_idx(F.fy * J, dj, F.ny, g.bcy);
                    const long long mf = (long long)F.nx * (jf + (long long)F.ny * kf) + i;
                    acc += wk * wj * residual_at<true>(F, g.bcx, g.bcy, g.bcz, fsub, i, jf, kf, mf);
                }
            }
            C.r[mm] = acc;
            C.u[mm] = 0.f;
        }
        break;
    }
    case OP_PROLONG: {
        // u += P e on the colour-0 lines (a proper zebra colouring: the colour-1 lines are
        // solved next without reading their old values), else on every site; sites are
        // enumerated line by line
        const MGLevel &F = S.L0, &C = S.L1;
        const DevGrid &g = H.a.g;
        const bool zeb = proper_zebra(F, g.bcy, g.bcz);
        const unsigned int ns = (unsigned int)(zeb ? H.nlines[l][0] * F.nx : F.N);
        const unsigned int nxu = (unsigned int)F.nx;
        // site s of the enumeration: (i, j, k) and its index
        auto site = [&](unsigned int sc, int &i, int &j, int &k) -> long long {
            if (zeb) {
                const unsigned int q = sc / nxu;
                i = (int)(sc - q * nxu);
                line_jk(q, 0, F.ny, F.nz, j, k);
                return (long long)F.nx * (j + (long long)F.ny * k) + i;
            }
            flat_ijk(sc, F.nx, F.ny, i, j, k);
            return (long long)sc;
        };
        if ((F.nx & 3) == 0) {
            // kQ quads per thread, every quad's loads before any store (lanes past the end
            // compute a valid quad and store nothing)
            float4 res[kQ];
            long long mq[kQ];
#pragma unroll
            for (int u = 0; u < kQ; ++u) {
                const unsigned int sq = (unsigned int)li * kFlatQ + 4u * (tid + u * kBT);
                int i, j, k;
                const long long mc = site(min(sq, ns - 4u), i, j, k);
                mq[u] = (sq < ns) ? mc : -1;
                const float4 v = prolong4_at<true>(F, C, g.bcy, g.bcz, i, j, k);
                const float4 o = ld4<true>(F.u + mc);
                res[u] = make_float4(o.x + v.x, o.y + v.y, o.z + v.z, o.w + v.w);
            }
#pragma unroll
            for (int u = 0; u < kQ; ++u)
                if (mq[u] >= 0) *reinterpret_cast<float4 *>(F.u + mq[u]) = res[u];
            break;
        }
#pragma unroll 4
        for (int r = 0; r < kFlatQ / kBT; ++r) {
            const unsigned int sc = (unsigned int)li * kFlatQ + r * kBT + tid;
            if (sc >= ns) break;
            int i, j, k;
            const long long mm = site(sc, i, j, k);
            const float v = prolong_at<true>(F, C, g.bcy, g.bcz, i, j, k);
            F.u[mm] = ldx<true>(F.u + mm) + v;
        }
        break;
    }
    case OP_CFWD:
    case OP_CINV: {
        const MGLevel &L = S.L0;
        const float fsub = (H.nlev == 1) ? (float)ldx<true>(&H.a.ctl->fmean) : 0.f;
        const long long ne = (long long)L.M * L.nx;
#pragma unroll
        for (int r = 0; r < kFlat / kBT; ++r) {
            const long long e = (long long)li * kFlat + r * kBT + tid;
            if (e >= ne) break;
            if (op == OP_CFWD) L.t[e] = coarse_fwd_at<true>(L, fsub, e);
            else L.u[e] = coarse_inv_at<true>(L, e);
        }
        break;
    }
    case OP_CCONV: coarse_conv_line<true>(S.L0, H.a.g.bcx, li, tid, kBT, dsm); break;
    case OP_MEAN: {
        // sum w mu (zero mode) and the x-face difference of mu (open-x voltage)
        const DevGrid &g = H.a.g;
        const float *mu = H.mu_solve;
        const unsigned int m0 = (unsigned int)li * (unsigned int)H.red_chunk;
        const unsigned int m1 = (unsigned int)min((long long)m0 + H.red_chunk, g.N);
        const bool ox = g.bcx == kOpen, oy = g.bcy == kOpen, oz = g.bcz == kOpen && g.nz >= 2;
        float accf = 0.f;
        double accv = 0.0;
        auto site = [&](unsigned int q, int i, int j, int k, float v) {
            float w = 1.f;
            if (ox && (i == 0 || i == g.nx - 1)) w *= 0.5f;
            if (oy && (j == 0 || j == g.ny - 1)) w *= 0.5f;
            if (oz && (k == 0 || k == g.nz - 1)) w *= 0.5f;
            accf += w * v;
            if (H.open_x) {
                if (i == 0) accv += (double)v;
                if (i == g.nx - 1) accv -= (double)v;
            }
        };
        if ((g.nx & 3) == 0 && !oy && !oz) {
            // periodic y and z: only the x faces carry a weight (1/2) and the face sums of E_x.
            // Four sites of one row per thread and pass; the site's x index advances by the
            // pass stride modulo nx instead of being divided out per site.
            // The loads of kU passes are issued before their sums (one load in flight per
            // thread left the pass latency-bound); the sums keep the pass order.
            const unsigned int stride = 4u * kBT, dstep = stride % (unsigned int)g.nx;
            unsigned int i = (m0 + 4u * tid) % (unsigned int)g.nx;
            constexpr int kU = 4;
            for (unsigned int q0 = m0 + 4u * tid; q0 < m1; q0 += kU * stride) {
                float4 xs[kU];
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const unsigned int q = q0 + u * stride;
                    xs[u] = (q < m1) ? ld4<true>(mu + q) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    if (q0 + u * stride >= m1) break;
                    const float4 x = xs[u];
                    float sum = (x.x + x.y) + (x.z + x.w);
                    if (ox && i == 0) sum -= 0.5f * x.x;
                    if (ox && i + 3 == (unsigned int)g.nx - 1) sum -= 0.5f * x.w;
                    accf += sum;
                    if (H.open_x) {
                        if (i == 0) accv += (double)x.x;
                        if (i + 3 == (unsigned int)g.nx - 1) accv -= (double)x.w;
                    }
                    i += dstep;
                    if (i >= (unsigned int)g.nx) i -= (unsigned int)g.nx;
                }
            }
        } else if ((g.nx & 3) == 0) {
            // four sites of one row per thread and pass; the loads of all passes first
            constexpr int kMP = 8;
            float4 v[kMP];
#pragma unroll
            for (int r = 0; r < kMP; ++r) {
                const unsigned int q = m0 + 4u * (tid + r * kBT);
                if (q < m1) v[r] = ld4<true>(mu + q);
            }
            for (unsigned int base = m0; base < m1; base += 4u * kBT * kMP) {
#pragma unroll
                for (int r = 0; r < kMP; ++r) {
                    const unsigned int q = base + 4u * (tid + r * kBT);
                    if (q < m1) {
                        const float4 x = (base == m0) ? v[r] : ld4<true>(mu + q);
                        int i, j, k;
                        flat_ijk(q, g.nx, g.ny, i, j, k);
                        site(q, i, j, k, x.x);
                        site(q + 1, i + 1, j, k, x.y);
                        site(q + 2, i + 2, j, k, x.z);
                        site(q + 3, i + 3, j, k, x.w);
                    }
                }
            }
        } else {
            for (unsigned int q = m0 + tid; q < m1; q += kBT) {
                int i, j, k;
                flat_ijk(q, g.nx, g.ny, i, j, k);
                site(q, i, j, k, ldx<true>(mu + q));
            }
        }
        __shared__ double shd[32];
        const double s0 = block_sum((double)accf, shd);
        const double s1 = block_sum(accv, shd);
        if (tid == 0) {
            H.a.blockred[2 * li] = s0;
            H.a.blockred[2 * li + 1] = s1;
        }
        if (!last_block(&H.a.ctl->ticket, H.red_items, &S.flag)) break;
        double t0 = 0.0, t1 = 0.0;
        for (int q = tid; q < H.red_items; q += kBT) {
            t0 += ((volatile double *)H.a.blockred)[2 * q];
            t1 += ((volatile double *)H.a.blockred)[2 * q + 1];
        }
        t0 = block_sum(t0, shd);
        t1 = block_sum(t1, shd);
        if (tid == 0) {
            DevCtl *c = H.a.ctl;
            c->ticket = 0u;
            if (!H.freeze) c->mu_mean = t0 / H.a.wsum;
            if (H.open_x) c->Ex = t1 / (double)((long long)g.ny * g.nz) / ((g.nx - 1) * H.hx);
            // after the shift the solve buffer holds this step's starting mu
            if (!H.freeze && H.mu_solve != H.a.mu) c->mu_prev_ok = 1;
        }
        break;
    }
    case OP_SHIFT: {
        if (H.mean_fused) {
            // the sums of the finest smoothing passes: the mean, the voltage and the guess flag
            // (what the mean phase records otherwise), written by the first item
            DevCtl *cc = H.a.ctl;
            const double t0 = ldx<true>(&cc->bmean[0]), t1 = ldx<true>(&cc->bmean[1]);
            if (li == 0 && tid == 0) {
                const DevGrid &g = H.a.g;
                cc->mu_mean = t0 / H.a.wsum;
                if (H.open_x) cc->Ex = t1 / (double)((long long)g.ny * g.nz) / ((g.nx - 1) * H.hx);
                if (H.mu_solve != H.a.mu) cc->mu_prev_ok = 1;
            }
        }
        const float c = H.mean_fused ? (float)(ldx<true>(&H.a.ctl->bmean[0]) / H.a.wsum)
                                     : (float)ldx<true>(&H.a.ctl->mu_mean);
        float *mu = const_cast<float *>(H.a.mu);
        const long long m0 = (long long)li * H.red_chunk;
        const long long m1 = min(m0 + H.red_chunk, H.a.g.N);
        if (H.mu_solve != H.a.mu) {
            // state <- solution - mean; the solve buffer keeps the old state (mu^(n-1)) for
            // the next step's extrapolation
            float *sv = H.mu_solve;
            if ((H.a.g.N & 3) == 0) {
                // the loads of kU passes first (the two buffers are distinct, the passes'
                // sites disjoint), then their stores
                constexpr int kU = 4;
                const long long stride = 4 * kBT;
                for (long long q0 = m0 + 4 * tid; q0 < m1; q0 += kU * stride) {
                    float4 vs[kU], os[kU];
#pragma unroll
                    for (int u = 0; u < kU; ++u) {
                        const long long q = q0 + u * stride;
                        if (q < m1) {
                            vs[u] = ld4<true>(sv + q);
                            os[u] = ld4<true>(mu + q);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < kU; ++u) {
                        const long long q = q0 + u * stride;
                        if (q < m1) {
                            const float4 v = vs[u];
                            *reinterpret_cast<float4 *>(mu + q) = make_float4(v.x - c, v.y - c, v.z - c, v.w - c);
                            *reinterpret_cast<float4 *>(sv + q) = os[u];
                        }
                    }
                }
            } else {
                for (long long q = m0 + tid; q < m1; q += kBT) {
                    const float v = ldx<true>(sv + q), o = ldx<true>(mu + q);
                    mu[q] = v - c;
                    sv[q] = o;
                }
            }
            break;
        }
        if ((H.a.g.N & 3) == 0) {
            for (long long q = m0 + 4 * tid; q < m1; q += 4 * kBT) {
                const float4 v = ld4<true>(mu + q);
                *reinterpret_cast<float4 *>(mu + q) = make_float4(v.x - c, v.y - c, v.z - c, v.w - c);
            }
        } else {
            for (long long q = m0 + tid; q < m1; q += kBT) mu[q] = ldx<true>(mu + q) - c;
        }
        break;
    }
    default: break;
    }
}

// This block's share of a phase's items (total from build_phase); ph: the phase's index in
// the launch.  Items are dealt on demand from a counter, tiles one at a time and the other
// items in runs of ch (about eight runs per block), so that blocks whose items ran faster
// take more and the phase ends together.  Two counters per launch alternate between phases: at the start of every phase
// block 0 clears the one the phase before used (the next phase's; every block has passed
// the barrier that ended the one before).
__device__ void run_items(const BatchParams &P, BatchSmem &S, float *dsm, int op, int l, int parity, int total,
                          unsigned int ph)
{
    const int tid = btid();
    unsigned int *ctr = P.bar + 4 + (S.cw ? 2 : 0);
    if (blockIdx.x == 0 && tid == 0) atomicExch(ctr + ((ph + 1) & 1), 0u);
    // tiles (init, sweeps, right-hand side) one at a time: they are few and long
    const bool tiles = op == OP_INIT || op == OP_SWEEP || op == OP_RHS;
    const int ch = tiles ? 1 : max(1, total / (int)(8 * gridDim.x));
    for (;;) {
        __syncthreads();
        if (tid == 0) S.grab = (int)atomicAdd(ctr + (ph & 1), (unsigned int)ch);
        __syncthreads();
        const int i0 = S.grab;
        if (i0 >= total) break;
        const int i1 = min(i0 + ch, total);
        for (int it = i0; it < i1; ++it) {
            const int pos = find_instance(S, P.n, it);
            const int m = S.order[pos];
            stage(P, S, m, op, l, parity);
            run_item(P, S, dsm, op, l, parity, m, it - S.start[pos]);
        }
    }
}

// Phase log entry (block 0): the time every block has finished phase nb, and its op.
__device__ __forceinline__ void log_phase(const BatchParams &P, unsigned int nb, int op, int l)
{
    if (P.plog && blockIdx.x == 0 && btid() == 0 && (int)nb < P.plog_cap) {
        P.plog[2 * nb] = gtimer();
        P.plog[2 * nb + 1] = (unsigned long long)(op * 256 + l);
    }
}

// One phase: item table, this block's items, then the grid barrier.
__device__ __forceinline__ bool phase(const BatchParams &P, BatchSmem &S, float *dsm, unsigned int &nbar, int op,
                                      int l, int parity)
{
    run_items(P, S, dsm, op, l, parity, build_phase(P, S, op, l), nbar);
    if (!grid_barrier(P.bar, P.bar + S.cw, P.extra, P.timeout_ns, ++nbar, &S.flag)) return false;
    log_phase(P, S.log0 + nbar, op, l);
    return true;
}

// A time step is two cooperative launches: the implicit psi solve, then K, the Poisson
// solve and the projection.  Each is compiled alone, so each gets the registers its own
// phases need (one kernel with every phase spilled more in the Jacobi sweeps).
// MINB: resident blocks per SM the register budget is sized for (2: no spills;
// 3: a few spilled registers, more warps to cover memory latency).
template <int MINB>
__global__ void __launch_bounds__(kBT, MINB) batch_psi_kernel(BatchParams P)
{
    extern __shared__ __align__(16) float dsm[];
    __shared__ BatchSmem S;
    if (*(volatile unsigned int *)(P.bar + 1) != 0u) return;   // sticky error from an earlier launch
    const int tid = btid();
    unsigned int nbar = 0;
    if (tid == 0) {
        S.cw = 0;
        S.log0 = 0;
    }
    log_phase(P, 0, 255, 0);   // launch start
    for (int t = tid; t < P.n; t += kBT) {
        S.order[t] = (unsigned short)P.order[t];
        S.alive[t] = (ldx<true>(P.bst + t) == 0) ? 1 : 0;
        S.active[t] = S.alive[t];
        S.ok[t] = 0;
    }
    // implicit psi solve: init + first sweep, then sweeps while any instance iterates
    if (!phase(P, S, dsm, nbar, OP_INIT, 0, 0)) return;
    for (int p = 1;; ++p) {
        __syncthreads();
        for (int t = tid; t < P.n; t += kBT)
            S.active[t] = S.active[t] && ldx<true>(P.act + ((p - 1) & 1) * P.n + t);
        if (p > P.max_phases) {
            // every instance stops at its own max_iter; this bound is never reached
            if (blockIdx.x == 0 && tid == 0) atomicCAS(P.bar + 1, 0u, 2u);
            return;
        }
        const int total = build_phase(P, S, OP_SWEEP, 0);
        if (total == 0) break;
        run_items(P, S, dsm, OP_SWEEP, 0, p & 1, total, nbar);
        if (!grid_barrier(P.bar, P.bar, P.extra, P.timeout_ns, ++nbar, &S.flag)) return;
        log_phase(P, nbar, OP_SWEEP, 0);
    }
    // block 0 records each instance's sweeps and failure (which the second launch reads)
    // and where the second launch's phase log continues
    __syncthreads();
    if (blockIdx.x == 0) {
        for (int t = tid; t < P.n; t += kBT) {
            if (!S.alive[t]) continue;
            const DevCtl *c = P.inst[t].h.a.ctl;
            const int st = ldx<true>(&c->status);
            P.sweeps[t] += ldx<true>(&c->iter);
            if (st != TDGL_OK) P.bst[t] = st;
        }
        if (tid == 0) P.bar[3] = nbar;
    }
}

template <int MINB>
__global__ void __launch_bounds__(kBT, MINB) batch_mu_kernel(BatchParams P)
{
    extern __shared__ __align__(16) float dsm[];
    __shared__ BatchSmem S;
    if (*(volatile unsigned int *)(P.bar + 1) != 0u) return;   // sticky error (either launch)
    const int tid = btid();
    unsigned int nbar = 0;
    if (tid == 0) {
        S.cw = 2;
        S.log0 = ldx<true>(P.bar + 3);
    }
    // the instances whose psi solve succeeded: no failure recorded
    for (int t = tid; t < P.n; t += kBT) {
        S.order[t] = (unsigned short)P.order[t];
        S.ok[t] = (ldx<true>(P.bst + t) == 0) ? 1 : 0;
        S.alive[t] = S.active[t] = 0;
    }
    __syncthreads();
    if (P.any_px && !phase(P, S, dsm, nbar, OP_JAVG, 0, 0)) return;
    if (!phase(P, S, dsm, nbar, OP_RHS, 0, 0)) return;
    for (int cyc = 0; cyc < P.cycles_max; ++cyc) {
        for (int l = 0; l < P.lmax; ++l) {
            if (!phase(P, S, dsm, nbar, OP_SMOOTH, 2 * l, 0)) return;
            if (!phase(P, S, dsm, nbar, OP_SMOOTH, 2 * l + 1, 0)) return;
            if (!phase(P, S, dsm, nbar, OP_RESTRICT, l, 0)) return;
        }
        if (!phase(P, S, dsm, nbar, OP_CFWD, 0, 0)) return;
        if (!phase(P, S, dsm, nbar, OP_CCONV, 0, 0)) return;
        if (!phase(P, S, dsm, nbar, OP_CINV, 0, 0)) return;
        // (the finest level's passes of the last cycle sum the zero mode and the voltage:
        // parity 1 of a smoothing phase)
        const int last = (cyc == P.cycles_max - 1) ? 1 : 0;
        for (int l = P.lmax - 1; l >= 0; --l) {
            if (!phase(P, S, dsm, nbar, OP_PROLONG, l, 0)) return;
            if (!phase(P, S, dsm, nbar, OP_SMOOTH, 2 * l + 1, l == 0 ? last : 0)) return;
            if (!phase(P, S, dsm, nbar, OP_SMOOTH, 2 * l, l == 0 ? last : 0)) return;
        }
    }
    if (P.any_mean && !phase(P, S, dsm, nbar, OP_MEAN, 0, 0)) return;
    run_items(P, S, dsm, OP_SHIFT, 0, 0, build_phase(P, S, OP_SHIFT, 0), nbar);
    log_phase(P, S.log0 + nbar + 1, OP_SHIFT, 0);   // block 0's own end (no barrier follows)
    if (P.plog && blockIdx.x == 0 && tid == 0 && (int)(S.log0 + nbar + 2) < P.plog_cap)
        P.plog[2 * (S.log0 + nbar + 2) + 1] = 0xffffull;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
int batch_default_kz(const DevGrid &g)
{
    // enough tiles for the instance to spread over the GPU, planes deep enough to
    // amortise the two halo planes
    const int gx = (g.nx + kPX - 1) / kPX, gy = (g.ny + kBY - 1) / kBY;
    int kz = 8;
    while (kz > 1 && (long long)gx * gy * ((g.nz + kz - 1) / kz) < 64) kz >>= 1;
    return kz > g.nz ? g.nz : kz;
}

void batch_tiling(BatchInst &I, int kz)
{
    const DevGrid &g = I.h.a.g;
    if (kz < 1) kz = 1;
    if (kz > g.nz) kz = g.nz;
    BatchHead &H = I.h;
    H.kz = kz;
    H.gx = (g.nx + kPX - 1) / kPX;
    H.gy = (g.ny + kBY - 1) / kBY;
    H.gz = (g.nz + kz - 1) / kz;
    H.tiles = H.gx * H.gy * H.gz;
}

size_t batch_smem_bytes(const BatchInst &I)
{
    long long fl = 0;
    const int top = I.h.nlev - 1;
    for (int l = 0; l < top; ++l) {
        const MGLevel &L = I.pa.lev[l];
        const long long v = line_tile_floats(line_shape(L.nx, L.kmin, L.kmax, kBT));
        if (v > fl) fl = v;
    }
    const MGLevel &C = I.pa.lev[top];
    const long long v = coarse_line_floats(C.nx, C.P);
    if (v > fl) fl = v;
    return sizeof(float) * (size_t)fl;
}

// Kernel variant for a target of bps resident blocks per SM.
// the two launches of a step for a target of bps resident blocks per SM
static const void *batch_kernel(int which, int bps)
{
    if (which == 0) return bps >= 3 ? (const void *)batch_psi_kernel<3> : (const void *)batch_psi_kernel<2>;
    return bps >= 3 ? (const void *)batch_mu_kernel<3> : (const void *)batch_mu_kernel<2>;
}

// resident blocks per SM of the step's launches (the smaller of the two): the psi solve with
// the sweep ring, the mu solve with smem bytes of line tiles
cudaError_t batch_max_blocks_per_sm(size_t smem, int bps, int *out)
{
    int occ[2] = {0, 0};
    for (int w = 0; w < 2; ++w) {
        const void *k = batch_kernel(w, bps);
        const size_t dyn = w == 0 ? kRingBytes : std::max(smem, kRingRBytes);
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[w], k, kBT, dyn);
        if (e != cudaSuccess) return e;
    }
    *out = occ[0] < occ[1] ? occ[0] : occ[1];
    return cudaSuccess;
}

cudaError_t launch_batch_step(const BatchParams &p, int grid, int bps, size_t smem, cudaStream_t s)
{
    // the two launches' barrier counts, the log index and the item counters; the error flag
    // (bar[1]) stays
    cudaError_t e = cudaMemsetAsync(p.bar, 0, sizeof(unsigned int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p.bar + 2, 0, 6 * sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kBX, kBY);
    cfg.dynamicSmemBytes = kRingBytes;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = bps >= 3 ? cudaLaunchKernelEx(&cfg, batch_psi_kernel<3>, p) : cudaLaunchKernelEx(&cfg, batch_psi_kernel<2>, p);
    if (e != cudaSuccess) return e;
    cfg.dynamicSmemBytes = std::max(smem, kRingRBytes);
    return bps >= 3 ? cudaLaunchKernelEx(&cfg, batch_mu_kernel<3>, p) : cudaLaunchKernelEx(&cfg, batch_mu_kernel<2>, p);
}

}  // namespace tdgl
