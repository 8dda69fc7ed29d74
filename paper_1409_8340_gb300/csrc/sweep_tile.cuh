// One tile of the Landau-gauge Jacobi sweep (yz- or xz-plane field) and the per-block finishing
// reductions, shared by the per-instance kernels and the batched persistent
// kernel (arXiv:1409.8340, Sec. 3.1: matrix M, Eq. b, Eq. final, Eq. convergence).
#pragma once
#include <float.h>

#include "philox.cuh"
#include "tdgl_internal.cuh"

namespace tdgl {

constexpr int kBX = 32;
constexpr int kBY = 8;

// Convergence decision of one sweep (Sec. 3.1, Eq. convergence) on the grid
// maximum gf of |r|^2 of the sweep's input iterate.  Run by one thread.
__device__ __forceinline__ void sweep_decide_ctl(const SweepArgs &a, float gf, bool init)
{
    DevCtl *c = a.ctl;
    int it = init ? 1 : c->iter + 1;
    if (init) {
        // a timed-out wait of a staged kernel (sweep or smoother) stays reported
        if (c->status != TDGL_ERR_TIMEOUT) c->status = TDGL_OK;
        c->nstep += 1;   // the init blocks have all read the noise counter
    }
    c->iter = it;
    if (*(volatile int *)&c->status == TDGL_ERR_TIMEOUT) {
        // a block of this sweep (or an earlier staged kernel) gave up waiting: end the solve
        c->done = 1;
        return;
    }
    c->r2 = (double)gf;
    c->result = a.dst_index;
    if (!(gf <= FLT_MAX)) {
        c->status = TDGL_ERR_NONFINITE;
        c->done = 1;
    } else if (a.fixed_sweeps > 0) {
        c->done = (it >= a.fixed_sweeps) ? 1 : 0;
    } else if (a.rel_eps && (it == 1 ? (c->r2ref = (double)gf, gf == 0.f) : (double)gf <= a.eps * c->r2ref)) {
        c->done = 1;
    } else if (!a.rel_eps && (it % a.check_every) == 0 && (double)gf < a.eps) {
        c->done = 1;
    } else if (it >= a.max_iter) {
        c->status = TDGL_ERR_NOT_CONVERGED;
        c->done = 1;
    } else {
        c->done = 0;
    }
}

// The decision, and in the device-resident loop the condition of its sweep loop: every
// path above ends the solve by max_iter sweeps, so the loop ends.  LOOP false: a kernel
// never launched inside that loop (the batched step), compiled without the graph calls.
template <bool LOOP = true>
__device__ __forceinline__ void sweep_decide(const SweepArgs &a, float gf, bool init)
{
    sweep_decide_ctl(a, gf, init);
    if (LOOP && a.has_loop) {
        DevCtl *c = a.ctl;
        cudaGraphSetConditional(a.loop_cond, c->done ? 0u : 1u);
        if (c->done) {
            const bool ok = c->status == TDGL_OK;
            c->rok = ok ? 1 : 0;
            cudaGraphSetConditional(a.tail_cond, ok ? (unsigned int)(a.tail_base + c->result) : kNoBranch);
        }
    }
}

// Start of a sweep that the solve may no longer need: true when an earlier sweep has
// decided (every block then returns); block (0, 0, 0) clears the loop condition.
__device__ __forceinline__ bool sweep_already_decided(const SweepArgs &a)
{
    if (!*(volatile int *)&a.ctl->done) return false;
    if (a.has_loop && (blockIdx.x | blockIdx.y | blockIdx.z | threadIdx.x | threadIdx.y | threadIdx.z) == 0)
        cudaGraphSetConditional(a.loop_cond, 0u);
    return true;
}

// Block maximum of |r|^2 into blockred[bid]; the last of nb blocks reduces the
// partials and decides.  Returns true in the block that decided.
template <bool LOOP = true>
__device__ __forceinline__ bool finish_sweep_at(const SweepArgs &a, float bmax, bool init, unsigned int bid,
                                                unsigned int nb)
{
    __shared__ float shf[32];
    __shared__ int flag;
    float m = block_max(bmax, shf);
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    if (tid == 0) a.blockred[bid] = (double)m;
    if (!last_block(&a.ctl->ticket, nb, &flag)) return false;
    double g = 0.0;
    for (unsigned int q = tid; q < nb; q += blockDim.x * blockDim.y) {
        double v = ((volatile double *)a.blockred)[q];
        g = v > g ? v : g;
    }
    float gf = block_max((float)g, shf);
    if (tid == 0) {
        a.ctl->ticket = 0u;
        sweep_decide<LOOP>(a, gf, init);
    }
    return true;
}

// ---------------------------------------------------------------------------
// Landau-gauge sweep, two sites per thread (even nx): each thread owns the x pair
// (x, x+1) of one row and marches in z.  16-byte loads of psi, b and D; the x
// neighbours of the pair come from the adjacent lanes by warp shuffles; the
// next plane's b, D and psi(k+1) are requested before the current plane is
// computed, so each thread keeps two planes of loads in flight.
// INIT: also forms b and diag M from psi^-, mu and alpha (first sweep).
// ---------------------------------------------------------------------------
constexpr int kPX = 64;   // x sites per block (32 lanes x 2)

__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }

// Block FP64 sum of w f into blockred[bid]; the last of nb blocks writes
// ctl->fmean = sum / wsum.  Returns true in the block that finished.
__device__ __forceinline__ bool finish_rhs_sum_at(DevCtl *ctl, double *blockred, double v, double wsum,
                                                  unsigned int bid, unsigned int nb)
{
    __shared__ double shd[32];
    __shared__ int flag;
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    double s = block_sum(v, shd);
    if (tid == 0) blockred[bid] = s;
    if (!last_block(&ctl->ticket, nb, &flag)) return false;
    double t = 0.0;
    for (unsigned int q = tid; q < nb; q += blockDim.x * blockDim.y) t += ((volatile double *)blockred)[q];
    t = block_sum(t, shd);
    if (tid == 0) {
        ctl->ticket = 0u;
        ctl->fmean = t / wsum;
    }
    return true;
}

// MODE 0: Jacobi sweep; 1: init + first sweep; 2: Poisson right-hand side;
// 3: adjoint sweep; 4: right-hand side that also copies psi (src) to a.dst.
// One tile (block coordinates bx, by, bz of the sweep2 grid) of a sweep; returns the
// thread's max |r|^2 in rmax (sweep modes) or its sum of w f in facc (right-hand side).
// CG: loads of data written earlier in the same launch go through L2 only.
// XZ: links of the xz-plane gauge (Eq. A_xz) from the j-indexed tables Xj, Zj and, on a
// periodic y axis, the wrap link Wx[i] Wz[k] from row ny-1 to row 0 (x wrap plain U_x).
// MASK: insulating inclusions (Sec. 3.4 (ii)): the link bits g.lk remove the links next
// to insulating sites from the neighbour sum and from the diagonal; an insulating site
// gets b = 0, diag M = 1 (psi = 0) and no injected current.
template <int MODE, bool CG = false, bool XZ = false, bool MASK = false>
__device__ __forceinline__ void sweep2_body(const SweepArgs &a, int kz, int bx, int by, int bz, float &rmax,
                                            float &facc)
{
    constexpr bool INIT = (MODE == 1);
    constexpr bool RHS = (MODE == 2 || MODE == 4);
    constexpr bool COPY = (MODE == 4);
    constexpr bool ADJ = (MODE == 3);   // adjoint solve M^H lam = g: conj(D), transposed open-face rows
    const DevGrid &g = a.g;
    const int tx = threadIdx.x;
    const int x = (bx * kBX + tx) * 2;
    const int j = by * kBY + threadIdx.y;
    const int k0 = zlo(g) + bz * kz;
    const int k1 = min(k0 + kz, zhi(g));
    const bool in = (x < g.nx) && (j < g.ny);
    const float2 Ux = ldx<CG>(&a.ctl->Ux);
    const unsigned long long nstep = INIT ? ldx<CG>(&a.ctl->nstep) : 0ull;
    const float4 *__restrict__ src = reinterpret_cast<const float4 *>(a.src);
    const float2 *__restrict__ src2 = a.src;
    const float4 *__restrict__ bq = reinterpret_cast<const float4 *>(a.b);
    const float4 *__restrict__ Dq = reinterpret_cast<const float4 *>(a.D);
    const float2 *__restrict__ mu2 = reinterpret_cast<const float2 *>(a.mu);
    const float2 *__restrict__ al2 = reinterpret_cast<const float2 *>(a.alpha);
    float4 *__restrict__ dst = reinterpret_cast<float4 *>(a.dst);
    float4 *__restrict__ bout = reinterpret_cast<float4 *>(a.b);
    float4 *__restrict__ Dout = reinterpret_cast<float4 *>(a.D);

    const long long rowq = g.nx >> 1;                       // float4 per row
    const long long plq = rowq * g.ny;                       // float4 per plane
    const long long sz = (long long)g.nx * g.ny;             // sites per plane
    const bool xper = (g.bcx == kPeriodic), yper = (g.bcy == kPeriodic), zper = (g.bcz == kPeriodic);
    const bool xlo = (x == 0), xhi = (x + 2 >= g.nx);
    const bool ylo = (j == 0), yhi = (j == g.ny - 1);
    const int jc = min(j, g.ny - 1);
    const int jp = yhi ? (yper ? 0 : jc) : jc + 1;
    const int jm = ylo ? (yper ? g.ny - 1 : jc) : jc - 1;
    const long long q0 = (x >> 1) + rowq * jc;               // float4 index in plane 0
    // Neighbour coefficients of the pair, constant along z: (ht/2) * c_axis *
    // (open-face weight 2 or 0) * link, so that S = (ht/2) NS is six complex
    // multiply-adds per site.  Forward neighbours use U, backward ones conj(U).
    const bool zact = g.nz >= 2;
    // open-face weights of the y neighbours: the forward operator doubles the inner
    // neighbour on a face row; its transpose doubles the face value on the next row
    const float wy_f = yper ? 1.f
                            : (ADJ ? (yhi ? 0.f : (j + 1 == g.ny - 1 ? 2.f : 1.f)) : (ylo ? 2.f : (yhi ? 0.f : 1.f)));
    const float wy_b = yper ? 1.f
                            : (ADJ ? (ylo ? 0.f : (j - 1 == 0 ? 2.f : 1.f)) : (yhi ? 2.f : (ylo ? 0.f : 1.f)));
    const bool yedge = (wy_f != 1.f) || (wy_b != 1.f);
    float2 yf0 = cmk(0.f, 0.f), yf1 = yf0, zf0 = yf0, zf1 = yf0;
    const bool ywrap = XZ && yper && (ylo || yhi);   // a row next to the xz gauge's y wrap
    float4 wxq = make_float4(1.f, 0.f, 1.f, 0.f);
    if (in) {
        const float sy = g.ht2 * g.cy, szc = g.ht2 * g.cz;
        if (XZ) {
            yf0 = yf1 = cmk(sy, 0.f);
            zf0 = zf1 = cscale(szc, g.Zj[jc]);
            if (ywrap) wxq = reinterpret_cast<const float4 *>(g.Wx)[x >> 1];
        } else {
            const float4 uy = reinterpret_cast<const float4 *>(g.Uy)[x >> 1];
            const float4 uz = reinterpret_cast<const float4 *>(g.Uz)[x >> 1];
            yf0 = cscale(sy, lo2(uy));
            yf1 = cscale(sy, hi2(uy));
            zf0 = cscale(szc, lo2(uz));
            zf1 = cscale(szc, hi2(uz));
        }
    }
    // x: site x has forward neighbour c1 and backward xl; site x+1 has forward xr and backward c0.
    // Backward coefficients are the conjugates of the forward ones.
    const float2 xf = cscale(g.ht2 * g.cx, XZ ? cmul(Ux, g.Xj[jc]) : Ux);
    const float inv_ht2 = 1.0f / g.ht2;

    auto knext = [&](int k) { return (k == g.nz - 1) ? (zper ? 0 : g.nz - 2) : k + 1; };
    float4 pzm = make_float4(0.f, 0.f, 0.f, 0.f), pc = pzm, pzp_n = pzm, b_n = pzm, D_n = pzm;
    float2 mu_n = cmk(0.f, 0.f), al_n = mu_n, pg_n = mu_n;
    float2 *__restrict__ guess2 = reinterpret_cast<float2 *>(a.mu_guess);
    const bool guess = INIT && guess2 != nullptr;
    // pending means of mu and of the previous-but-one mu (the zero-mode projection)
    const float offS = (INIT && a.mu_off) ? (float)ldx<CG>(a.mu_off) : 0.f;
    const float offP = (INIT && a.mu_off_prev) ? (float)ldx<CG>(a.mu_off_prev) : 0.f;
    const uchar2 *__restrict__ lk2 = reinterpret_cast<const uchar2 *>(g.lk);
    uchar2 lk_n = make_uchar2(0, 0);
    if (MASK && in) lk_n = ldx<CG>(lk2 + q0 + plq * k0);
    if (in) {
        if (zact) pzm = ldx<CG>(src + q0 + plq * ((k0 == 0) ? (zper ? g.nz - 1 : 1) : k0 - 1));
        pc = ldx<CG>(src + q0 + plq * k0);
        if (zact) pzp_n = ldx<CG>(src + q0 + plq * knext(k0));
        if (INIT) {
            mu_n = ldx<CG>(mu2 + q0 + plq * k0);
            al_n = ldx<CG>(al2 + q0 + plq * k0);
            if (guess && (!a.guess_odd_only || ((j + k0) & 1))) pg_n = ldx<CG>(guess2 + q0 + plq * k0);
        } else if (!RHS) {
            b_n = ldx<CG>(bq + q0 + plq * k0);
            D_n = ldx<CG>(Dq + q0 + plq * k0);
        }
    }
    float wxy0 = 1.f, wxy1 = 1.f;
    if (RHS) {
        const float wy = (g.bcy == kOpen && (j == 0 || j == g.ny - 1)) ? 0.5f : 1.f;
        wxy0 = wy * ((g.bcx == kOpen && x == 0) ? 0.5f : 1.f);
        wxy1 = wy * ((g.bcx == kOpen && x + 1 == g.nx - 1) ? 0.5f : 1.f);
    }
    for (int k = k0; k < k1; ++k) {
        const float4 pzp = pzp_n;
        const float4 bc = b_n, Dc = D_n;
        const float2 muc = make_float2(mu_n.x - offS, mu_n.y - offS), alc = al_n, pgc = pg_n;
        const uchar2 lkc = lk_n;
        const long long q = q0 + plq * k;
        float4 yf = make_float4(0.f, 0.f, 0.f, 0.f), yb = yf;
        float2 xl = cmk(0.f, 0.f), xr = xl;
        if (in) {
            if (k + 1 < k1) {
                if (MASK) lk_n = ldx<CG>(lk2 + q + plq);
                if (zact) pzp_n = ldx<CG>(src + q0 + plq * knext(k + 1));
                if (INIT) {
                    mu_n = ldx<CG>(mu2 + q + plq);
                    al_n = ldx<CG>(al2 + q + plq);
                    if (guess && (!a.guess_odd_only || ((j + k + 1) & 1))) pg_n = ldx<CG>(guess2 + q + plq);
                } else if (!RHS) {
                    b_n = ldx<CG>(bq + q + plq);
                    D_n = ldx<CG>(Dq + q + plq);
                }
            }
            yf = ldx<CG>(src + (x >> 1) + rowq * jp + plq * k);
            yb = ldx<CG>(src + (x >> 1) + rowq * jm + plq * k);
        }
        // x neighbours: left of x from lane tx-1, right of x+1 from lane tx+1
        const float2 from_left = make_float2(__shfl_up_sync(0xffffffffu, pc.z, 1), __shfl_up_sync(0xffffffffu, pc.w, 1));
        const float2 from_right =
            make_float2(__shfl_down_sync(0xffffffffu, pc.x, 1), __shfl_down_sync(0xffffffffu, pc.y, 1));
        const long long m = (long long)x + (long long)g.nx * jc + sz * k;   // site index of x
        if (in) {
            if (tx > 0) xl = from_left;
            else if (!xlo) xl = ldx<CG>(src2 + m - 1);
            else if (xper) xl = ldx<CG>(src2 + m + g.nx - 1);
            if (!xhi && tx < kBX - 1) xr = from_right;
            else if (!xhi) xr = ldx<CG>(src2 + m + 2);
            else if (xper) xr = ldx<CG>(src2 + m + 2 - g.nx);
        }
        if (in) {
            const float2 c0 = lo2(pc), c1 = hi2(pc);
            // x neighbours with the boundary rules: open faces double the inner
            // neighbour; the periodic wrap link (i = nx-1 -> 0) carries conj(P_jk)
            // in the yz gauge and is the plain x link in the xz gauge.
            float2 xl0 = xl, xr1 = xr, c1x = c1, c0x = c0;
            if (xlo || xhi) {
                if (xper) {
                    if (!XZ) {
                        const float2 P = cmul(g.Py[jc], g.Pz[k]);
                        if (xlo) xl0 = cmul(P, xl);      // conj(Ux conj(P)) xl = conj(Ux) (P xl)
                        if (xhi) xr1 = cmulc(P, xr);     // Ux conj(P) xr = Ux (conj(P) xr)
                    }
                } else if (!ADJ) {
                    if (xlo) {
                        c1x = cscale(2.f, c1);
                        xl0 = cmk(0.f, 0.f);
                    }
                    if (xhi) {
                        c0x = cscale(2.f, c0);
                        xr1 = cmk(0.f, 0.f);
                    }
                } else {
                    // transpose: site 1 sees the low face value twice, site nx-2 the high one
                    if (xlo) {
                        c0x = cscale(2.f, c0);
                        xl0 = cmk(0.f, 0.f);
                    }
                    if (xhi) {
                        c1x = cscale(2.f, c1);
                        xr1 = cmk(0.f, 0.f);
                    }
                }
            }
            float2 yf_0 = lo2(yf), yf_1 = hi2(yf), yb_0 = lo2(yb), yb_1 = hi2(yb);
            if (ywrap) {
                // wrap link W = Wx[i] Wz[k] from row ny-1 to row 0: forward W psi, backward conj(W) psi
                const float2 wz = g.Wz[k];
                const float2 W0 = cmul(lo2(wxq), wz), W1 = cmul(hi2(wxq), wz);
                if (yhi) {
                    yf_0 = cmul(W0, yf_0);
                    yf_1 = cmul(W1, yf_1);
                }
                if (ylo) {
                    yb_0 = cmulc(W0, yb_0);
                    yb_1 = cmulc(W1, yb_1);
                }
            }
            if (yedge) {
                yf_0 = cscale(wy_f, yf_0);
                yf_1 = cscale(wy_f, yf_1);
                yb_0 = cscale(wy_b, yb_0);
                yb_1 = cscale(wy_b, yb_1);
            }
            if (MASK) {
                // removed links (0) and present ones (1) of each site of the pair
                const unsigned l0 = lkc.x, l1 = lkc.y;
                c1x = cscale((l0 & kLkXp) ? 1.f : 0.f, c1x);
                xl0 = cscale((l0 & kLkXm) ? 1.f : 0.f, xl0);
                xr1 = cscale((l1 & kLkXp) ? 1.f : 0.f, xr1);
                c0x = cscale((l1 & kLkXm) ? 1.f : 0.f, c0x);
                yf_0 = cscale((l0 & kLkYp) ? 1.f : 0.f, yf_0);
                yb_0 = cscale((l0 & kLkYm) ? 1.f : 0.f, yb_0);
                yf_1 = cscale((l1 & kLkYp) ? 1.f : 0.f, yf_1);
                yb_1 = cscale((l1 & kLkYm) ? 1.f : 0.f, yb_1);
            }
            // S = (ht/2) NS for both sites
            float2 ns0 = cmul(xf, c1x), ns1 = cmulc(xf, c0x);
            cfmac(ns0, xf, xl0);
            cfma(ns1, xf, xr1);
            cfma(ns0, yf0, yf_0);
            cfmac(ns0, yf0, yb_0);
            cfma(ns1, yf1, yf_1);
            cfmac(ns1, yf1, yb_1);
            if (zact) {
                float wz_f = 1.f, wz_b = 1.f;
                if (!zper && ADJ) {
                    wz_f = (k == g.nz - 1) ? 0.f : (k + 1 == g.nz - 1 ? 2.f : 1.f);
                    wz_b = (k == 0) ? 0.f : (k - 1 == 0 ? 2.f : 1.f);
                } else if (!zper) {
                    if (k == 0) {
                        wz_f = 2.f;
                        wz_b = 0.f;
                    } else if (k == g.nz - 1) {
                        wz_f = 0.f;
                        wz_b = 2.f;
                    }
                }
                float4 zpp = (wz_f == 1.f) ? pzp : make_float4(wz_f * pzp.x, wz_f * pzp.y, wz_f * pzp.z, wz_f * pzp.w);
                float4 zmm = (wz_b == 1.f) ? pzm : make_float4(wz_b * pzm.x, wz_b * pzm.y, wz_b * pzm.z, wz_b * pzm.w);
                if (MASK) {
                    const float f0 = (lkc.x & kLkZp) ? 1.f : 0.f, b0 = (lkc.x & kLkZm) ? 1.f : 0.f;
                    const float f1 = (lkc.y & kLkZp) ? 1.f : 0.f, b1 = (lkc.y & kLkZm) ? 1.f : 0.f;
                    zpp = make_float4(f0 * zpp.x, f0 * zpp.y, f1 * zpp.z, f1 * zpp.w);
                    zmm = make_float4(b0 * zmm.x, b0 * zmm.y, b1 * zmm.z, b1 * zmm.w);
                }
                cfma(ns0, zf0, lo2(zpp));
                cfmac(ns0, zf0, lo2(zmm));
                cfma(ns1, zf1, hi2(zpp));
                cfmac(ns1, zf1, hi2(zmm));
            }
            if (RHS) {
                // f = Im[conj(psi) NS(psi)] plus the open-x injection terms
                float f0 = (c0.x * ns0.y - c0.y * ns0.x) * inv_ht2;
                float f1 = (c1.x * ns1.y - c1.y * ns1.x) * inv_ht2;
                if (!xper) {
                    if (xlo && !(MASK && (lkc.x & kLkIns))) f0 -= a.inj;
                    if (xhi && !(MASK && (lkc.y & kLkIns))) f1 += a.inj;
                }
                reinterpret_cast<float2 *>(a.f)[q] = make_float2(f0, f1);
                if (COPY) dst[q] = pc;
                const float wz = (g.bcz == kOpen && g.nz >= 2 && (k == 0 || k == g.nz - 1)) ? 0.5f : 1.f;
                facc += wz * (wxy0 * f0 + wxy1 * f1);
                pzm = pc;
                pc = pzp;
                continue;
            }
            float2 b0, b1, D0, D1;
            if (INIT) {
                const float2 cs[2] = {c0, c1};
                const float2 nss[2] = {ns0, ns1};
                const float mus[2] = {muc.x, muc.y}, als[2] = {alc.x, alc.y};
                float S2[2] = {2.f * g.S, 2.f * g.S};
                if (MASK) {
                    // diagonal: c_a per present link, the ghost doubling an open face's inner link
                    const unsigned ls[2] = {lkc.x, lkc.y};
                    const float fy = (!yper && (ylo || yhi)) ? 2.f : 1.f;
                    const float fz = (zact && !zper && (k == 0 || k == g.nz - 1)) ? 2.f : 1.f;
#pragma unroll
                    for (int s2 = 0; s2 < 2; ++s2) {
                        const unsigned l = ls[s2];
                        const float fx = (!xper && (s2 == 0 ? xlo : xhi)) ? 2.f : 1.f;
                        const float nxl = (float)(((l & kLkXp) ? 1 : 0) + ((l & kLkXm) ? 1 : 0));
                        const float nyl = (float)(((l & kLkYp) ? 1 : 0) + ((l & kLkYm) ? 1 : 0));
                        const float nzl = (float)(((l & kLkZp) ? 1 : 0) + ((l & kLkZm) ? 1 : 0));
                        S2[s2] = g.cx * fx * nxl + g.cy * fy * nyl + (zact ? g.cz * fz * nzl : 0.f);
                    }
                }
                float2 bo[2], Do[2];
#pragma unroll
                for (int s2 = 0; s2 < 2; ++s2) {
                    const float a2 = cabs2(cs[s2]);
                    Do[s2] = cmk(1.f + g.ht2 * (g.beta * a2 + S2[s2] - als[s2]), g.ht2 * g.u * mus[s2]);
                    const float cr = als[s2] - g.beta * a2 - S2[s2];
                    const float ci = -g.u * mus[s2];
                    const float2 lin = cmk(cr * cs[s2].x - ci * cs[s2].y, cr * cs[s2].y + ci * cs[s2].x);
                    bo[s2] = cadd(cadd(cs[s2], cscale(g.ht2, lin)), nss[s2]);   // nss = (ht/2) NS
                    if (a.noise_amp != 0.f) {
                        // thermal noise h_t zeta_m (Sec. 3.1.2), counter (site, step)
                        const float2 v = noise_uv(a.noise_seed, m + s2, nstep);
                        bo[s2] = cmk(bo[s2].x + a.noise_amp * v.x, bo[s2].y + a.noise_amp * v.y);
                    }
                    if (MASK && ((s2 == 0 ? lkc.x : lkc.y) & kLkIns)) {   // insulating: psi = 0
                        bo[s2] = cmk(0.f, 0.f);
                        Do[s2] = cmk(1.f, 0.f);
                    }
                }
                b0 = bo[0];
                b1 = bo[1];
                D0 = Do[0];
                D1 = Do[1];
                bout[q] = make_float4(b0.x, b0.y, b1.x, b1.y);
                Dout[q] = make_float4(D0.x, D0.y, D1.x, D1.y);
                // the coming Poisson solve starts from a mu^(n-1) + b mu^(n-2), written over the latter
                if (guess && (!a.guess_odd_only || ((j + k) & 1)))
                    guess2[q] = make_float2(a.ex_a * muc.x + a.ex_b * (pgc.x - offP),
                                            a.ex_a * muc.y + a.ex_b * (pgc.y - offP));
            } else {
                b0 = lo2(bc);
                b1 = hi2(bc);
                D0 = ADJ ? cconj(lo2(Dc)) : lo2(Dc);
                D1 = ADJ ? cconj(hi2(Dc)) : hi2(Dc);
            }
            const float2 s0 = cadd(b0, ns0), s1 = cadd(b1, ns1);
            const float2 r0 = csub(s0, cmul(D0, c0)), r1 = csub(s1, cmul(D1, c1));
            // 1 / |D|^2, correctly rounded (the same value as 1.0f / |D|^2)
            const float2 n0 = cscale(__frcp_rn(cabs2(D0)), cmulc(D0, s0));
            const float2 n1 = cscale(__frcp_rn(cabs2(D1)), cmulc(D1, s1));
            dst[q] = make_float4(n0.x, n0.y, n1.x, n1.y);
            float r2a = cabs2(r0), r2b = cabs2(r1);
            r2a = (r2a <= FLT_MAX) ? r2a : INFINITY;
            r2b = (r2b <= FLT_MAX) ? r2b : INFINITY;
            rmax = fmaxf(rmax, fmaxf(r2a, r2b));
        }
        pzm = pc;
        pc = pzp;
    }
}

}  // namespace tdgl
