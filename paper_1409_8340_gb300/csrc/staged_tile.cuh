// Sweep tiles staged in shared memory by 16-byte asynchronous copies, shared by the
// batched persistent kernel and the per-instance init kernel (arXiv:1409.8340, Sec. 3.1:
// Eq. b, Eq. final, Eq. convergence; Sec. 3.3: the Poisson right-hand side).
#pragma once
#include <float.h>

#include "philox.cuh"
#include "sweep_tile.cuh"
#include "tdgl_internal.cuh"

namespace tdgl {

// ---------------------------------------------------------------------------
// Sweep tiles staged in shared memory (Sec. 3.1, Eq. b, Eq. final and Eq. convergence;
// and the Poisson right-hand side of Sec. 3.3).
//
// A tile is 64 x-sites by 8 rows, marching along z.  Every thread streams, per z
// plane, its own site pair of psi (and of b and diag M for a sweep; the first half
// warp the row's mu, alpha and previous-but-one mu for the init) into a ring of
// plane stages with 16-byte asynchronous copies through L2 (cp.async.cg), the edge
// warps and lanes also the tile's y halo rows and x halo pairs.  Planes stay in flight
// ahead of the plane being updated, held in shared memory instead of registers.  The
// copies bypass L1 as the batched kernel's loads do: there, data written earlier in the
// same launch by other blocks is copied after the grid barrier that ended its phase.
// ---------------------------------------------------------------------------
constexpr int kRing = 5;                 // plane stages
constexpr int kRowQ = kBX + 2;           // float4 per staged psi row: [pair x0-2 | 32 pairs | pair x0+64]
struct BStage {
    float4 psi[kBY + 2][kRowQ];          // rows j0-1 .. j0+8
    float4 b[kBY][kBX];
    float4 D[kBY][kBX];
};
static_assert(sizeof(BStage) % 16 == 0, "16-byte stage elements");
constexpr size_t kRingBytes = kRing * sizeof(BStage);
// right-hand side: psi alone, through a deeper ring of smaller stages
constexpr int kRingR = 8;
struct RStage {
    float4 psi[kBY + 2][kRowQ];
};
constexpr size_t kRingRBytes = kRingR * sizeof(RStage);
// init + first sweep: psi, and the tile's mu, alpha and previous-but-one mu (the Poisson
// guess's source) as rows of 64 floats
struct IStage {
    float4 psi[kBY + 2][kRowQ];
    float mu[kBY][kPX];
    float al[kBY][kPX];
    float pg[kBY][kPX];
};
static_assert(kRing * sizeof(IStage) <= kRingBytes, "the init ring fits the sweep ring's shared memory");
// stage kind and ring depth of a tile mode (0 sweep, 1 init + first sweep, 4 right-hand side)
template <int MODE>
struct StageOf {
    using T = BStage;
    static constexpr int n = kRing;
};
template <>
struct StageOf<1> {
    using T = IStage;
    static constexpr int n = kRing;
};
template <>
struct StageOf<4> {
    using T = RStage;
    static constexpr int n = kRingR;
};
// b and diag M of a stage (the right-hand side's stages hold none)
__device__ __forceinline__ float4 *stage_b_ptr(BStage &S, int r, int tx) { return &S.b[r][tx]; }
__device__ __forceinline__ float4 *stage_D_ptr(BStage &S, int r, int tx) { return &S.D[r][tx]; }
__device__ __forceinline__ float4 *stage_b_ptr(RStage &, int, int) { return nullptr; }
__device__ __forceinline__ float4 *stage_D_ptr(RStage &, int, int) { return nullptr; }
__device__ __forceinline__ float4 stage_b(const BStage &S, int r, int tx) { return S.b[r][tx]; }
__device__ __forceinline__ float4 stage_D(const BStage &S, int r, int tx) { return S.D[r][tx]; }
__device__ __forceinline__ float4 stage_b(const RStage &, int, int) { return make_float4(0.f, 0.f, 0.f, 0.f); }
__device__ __forceinline__ float4 stage_D(const RStage &, int, int) { return make_float4(0.f, 0.f, 0.f, 0.f); }
__device__ __forceinline__ float4 *stage_b_ptr(IStage &, int, int) { return nullptr; }
__device__ __forceinline__ float4 *stage_D_ptr(IStage &, int, int) { return nullptr; }
__device__ __forceinline__ float4 stage_b(const IStage &, int, int) { return make_float4(0.f, 0.f, 0.f, 0.f); }
__device__ __forceinline__ float4 stage_D(const IStage &, int, int) { return make_float4(0.f, 0.f, 0.f, 0.f); }
// mu, alpha and previous-but-one mu rows of an init stage (other stages hold none)
__device__ __forceinline__ float *stage_row(IStage &S, int w, int r)
{
    return w == 0 ? &S.mu[r][0] : (w == 1 ? &S.al[r][0] : &S.pg[r][0]);
}
template <class St>
__device__ __forceinline__ float *stage_row(St &, int, int) { return nullptr; }
__device__ __forceinline__ float2 stage_pair(const IStage &S, int w, int r, int tx)
{
    const float *row = w == 0 ? &S.mu[r][0] : (w == 1 ? &S.al[r][0] : &S.pg[r][0]);
    return *reinterpret_cast<const float2 *>(row + 2 * tx);
}
template <class St>
__device__ __forceinline__ float2 stage_pair(const St &, int, int, int) { return make_float2(0.f, 0.f); }

__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// index c wrapped onto 0 .. n-1 (periodic) or clamped to it (open)
__device__ __forceinline__ int wrap_or_clamp(int c, int n, bool per)
{
    if (per) {
        c %= n;
        return c < 0 ? c + n : c;
    }
    return min(max(c, 0), n - 1);
}


// stored plane of z plane z (one beyond either end: the periodic image, or the
// mirrored inner plane on an open face, whose term carries weight 0)
__device__ __forceinline__ int batch_plane(const DevGrid &g, int z)
{
    if (z < 0) return (g.bcz == kPeriodic) ? z + g.nz : (g.nz >= 2 ? 1 : 0);
    if (z >= g.nz) return (g.bcz == kPeriodic) ? z - g.nz : (g.nz >= 2 ? g.nz - 2 : 0);
    return z;
}

// One staged tile: plane p of the tile (z plane k0 - 1 + p) in stage p % NS.  The plane
// below the tile enters as the first plane's lower neighbour only and is read directly;
// each later plane's lower neighbour is carried in a register, so the step of plane t
// reads the stages of planes t and t + 1 and the one of plane t - 1 takes plane t + NS - 1.
//
// MODE 4, the Poisson right-hand side (Sec. 3.3): psi alone is staged; each site pair
// writes f = Im[conj(psi) NS(psi)] / (ht/2) plus the injected current on the open x
// faces, copies psi to a.dst, and adds its trapezoid-weighted f to facc.  MODE 1, the
// init (Sec. 3.1, Eq. b; nx % 4 == 0): b and diag M from psi^n, mu and alpha (with the
// thermal noise), written out, then the first sweep; and the Poisson guess.  MODE 0, the
// Jacobi sweep.  Per site the arithmetic is sweep2_body's (without insulating sites), in the
// same order; each stage element maps to a grid site with the periodic wraps applied (open
// faces clamp to the face; the boundary rules zero or double those terms), so every x and
// y neighbour, the wrap neighbours included, is a plain read of the stage.
template <int MODE>
__device__ __forceinline__ void sweep_staged_tile(const SweepArgs &a, int kz, int bx, int by, int bz, float &rmax, float &facc,
                                  typename StageOf<MODE>::T *ring)
{
    constexpr bool RHS = (MODE == 4), INIT = (MODE == 1);
    constexpr int NS = StageOf<MODE>::n;
    const DevGrid &g = a.g;
    const int tx = threadIdx.x, r = threadIdx.y;
    const int x0 = bx * kPX, j0 = by * kBY;
    const int x = x0 + 2 * tx, j = j0 + r;
    const int k0 = zlo(g) + bz * kz, k1 = min(k0 + kz, zhi(g));
    const int nplanes = (k1 - k0) + 2;   // k0 - 1 .. k1
    const bool in = (x < g.nx) && (j < g.ny);
    const bool xper = (g.bcx == kPeriodic), yper = (g.bcy == kPeriodic), zper = (g.bcz == kPeriodic);
    const bool xlo = (x == 0), xhi = (x + 2 >= g.nx);
    const bool ylo = (j == 0), yhi = (j == g.ny - 1);
    const bool zact = g.nz >= 2;
    const int jc = min(j, g.ny - 1);
    const int rowq = g.nx >> 1;
    const long long plq = (long long)rowq * g.ny;
    const float4 *__restrict__ src = reinterpret_cast<const float4 *>(a.src);
    const float4 *__restrict__ bq = reinterpret_cast<const float4 *>(a.b);
    const float4 *__restrict__ Dq = reinterpret_cast<const float4 *>(a.D);
    float4 *__restrict__ dst = reinterpret_cast<float4 *>(a.dst);

    // in-plane float4 offsets of this thread's copies: its own pair (read by itself and,
    // past the grid's last pair or row, as the wrap neighbour of the pair or row before),
    // the y halo rows (first and last warp) and the x halo pairs (first and last lane)
    const int cq = wrap_or_clamp(x0 / 2 + tx, rowq, xper);
    const int own = wrap_or_clamp(j, g.ny, yper) * rowq + cq;
    const int yh = (r == 0) ? wrap_or_clamp(j0 - 1, g.ny, yper) * rowq + cq
                            : wrap_or_clamp(j0 + kBY, g.ny, yper) * rowq + cq;
    const int xh = wrap_or_clamp(j, g.ny, yper) * rowq +
                   wrap_or_clamp(tx == 0 ? x0 / 2 - 1 : x0 / 2 + kBX, rowq, xper);
    const bool need = (x <= g.nx) && (j <= g.ny);
    const long long sz = (long long)g.nx * g.ny;   // sites per plane
    const bool guess = INIT && a.mu_guess != nullptr;
    auto issue = [&](int t) {
        if (t < nplanes) {
            auto &S = ring[t % NS];
            const long long base = plq * batch_plane(g, k0 - 1 + t);
            if (need) cp_async16(&S.psi[r + 1][tx + 1], src + base + own);
            if (r == 0) cp_async16(&S.psi[0][tx + 1], src + base + yh);
            if (r == kBY - 1) cp_async16(&S.psi[kBY + 1][tx + 1], src + base + yh);
            if (tx == 0) cp_async16(&S.psi[r + 1][0], src + base + xh);
            if (tx == kBX - 1) cp_async16(&S.psi[r + 1][kBX + 1], src + base + xh);
            if (!RHS && !INIT && in && t + 1 < nplanes) {   // b and diag M of the updated planes only
                cp_async16(stage_b_ptr(S, r, tx), bq + base + own);
                cp_async16(stage_D_ptr(S, r, tx), Dq + base + own);
            }
            // init: the updated planes' mu, alpha and (on the rows that take the guess)
            // previous-but-one mu, 16 bytes per lane of the first half warp (nx % 4 == 0)
            if (INIT && t + 1 < nplanes && j < g.ny && tx < kPX / 4 && x0 + 4 * tx < g.nx) {
                const int k = k0 - 1 + t;
                const long long fb = sz * k + (long long)g.nx * j + x0 + 4 * tx;
                cp_async16(stage_row(S, 0, r) + 4 * tx, a.mu + fb);
                cp_async16(stage_row(S, 1, r) + 4 * tx, a.alpha + fb);
                if (guess && (!a.guess_odd_only || ((j + k) & 1))) cp_async16(stage_row(S, 2, r) + 4 * tx, a.mu_guess + fb);
            }
        }
        cp_async_commit();
    };

    // coefficients of the pair, constant along z (as in sweep2_body)
    const float wy_f = yper ? 1.f : (ylo ? 2.f : (yhi ? 0.f : 1.f));
    const float wy_b = yper ? 1.f : (yhi ? 2.f : (ylo ? 0.f : 1.f));
    const bool yedge = (wy_f != 1.f) || (wy_b != 1.f);
    float2 yf0 = cmk(0.f, 0.f), yf1 = yf0, zf0 = yf0, zf1 = yf0;
    if (in) {
        const float sy = g.ht2 * g.cy, szc = g.ht2 * g.cz;
        const float4 uy = reinterpret_cast<const float4 *>(g.Uy)[x >> 1];
        const float4 uz = reinterpret_cast<const float4 *>(g.Uz)[x >> 1];
        yf0 = cscale(sy, lo2(uy));
        yf1 = cscale(sy, hi2(uy));
        zf0 = cscale(szc, lo2(uz));
        zf1 = cscale(szc, hi2(uz));
    }
    const float2 xf = cscale(g.ht2 * g.cx, ldx<true>(&a.ctl->Ux));
    const long long q0 = (x >> 1) + (long long)rowq * jc;
    // RHS: trapezoid weights of the pair on open faces, 1 / (ht/2)
    const float wy = (g.bcy == kOpen && (j == 0 || j == g.ny - 1)) ? 0.5f : 1.f;
    const float wxy0 = wy * ((g.bcx == kOpen && x == 0) ? 0.5f : 1.f);
    const float wxy1 = wy * ((g.bcx == kOpen && x + 1 == g.nx - 1) ? 0.5f : 1.f);
    const float inv_ht2 = 1.0f / g.ht2;
    // init: the noise counter and the pending means of mu and of the previous-but-one mu
    const unsigned long long nstep = INIT ? ldx<true>(&a.ctl->nstep) : 0ull;
    const float offS = (INIT && a.mu_off) ? (float)ldx<true>(a.mu_off) : 0.f;
    const float offP = (INIT && a.mu_off_prev) ? (float)ldx<true>(a.mu_off_prev) : 0.f;

    float4 pzm = make_float4(0.f, 0.f, 0.f, 0.f);
    if (in && zact) pzm = ldx<true>(src + plq * batch_plane(g, k0 - 1) + own);
    // the ring is free: the block's previous item waited for all of its copies
    __syncthreads();
    for (int t = 1; t < NS; ++t) issue(t);
    for (int t = 1; t + 1 < nplanes; ++t) {
        // planes up to t + 1 have landed (NS - 3 newer groups may still be in flight), and
        // every thread has finished plane t - 1, so its stage takes plane t + NS - 1
        cp_async_wait<NS - 3>();
        __syncthreads();
        issue(t + NS - 1);
        const int k = k0 - 1 + t;
        const auto &Pc = ring[t % NS], &Pp = ring[(t + 1) % NS];
        if (!in) continue;
        const float4 pc = Pc.psi[r + 1][tx + 1];
        const float2 c0 = lo2(pc), c1 = hi2(pc);
        const float2 xl = hi2(Pc.psi[r + 1][tx]), xr = lo2(Pc.psi[r + 1][tx + 2]);
        const float4 yf = Pc.psi[r + 2][tx + 1], yb = Pc.psi[r][tx + 1];
        float2 xl0 = xl, xr1 = xr, c1x = c1, c0x = c0;
        if (xlo || xhi) {
            if (xper) {
                const float2 Pw = cmul(g.Py[jc], g.Pz[k]);
                if (xlo) xl0 = cmul(Pw, xl);
                if (xhi) xr1 = cmulc(Pw, xr);
            } else {
                if (xlo) {
                    c1x = cscale(2.f, c1);
                    xl0 = cmk(0.f, 0.f);
                }
                if (xhi) {
                    c0x = cscale(2.f, c0);
                    xr1 = cmk(0.f, 0.f);
                }
            }
        }
        float2 yf_0 = lo2(yf), yf_1 = hi2(yf), yb_0 = lo2(yb), yb_1 = hi2(yb);
        if (yedge) {
            yf_0 = cscale(wy_f, yf_0);
            yf_1 = cscale(wy_f, yf_1);
            yb_0 = cscale(wy_b, yb_0);
            yb_1 = cscale(wy_b, yb_1);
        }
        float2 ns0 = cmul(xf, c1x), ns1 = cmulc(xf, c0x);
        cfmac(ns0, xf, xl0);
        cfma(ns1, xf, xr1);
        cfma(ns0, yf0, yf_0);
        cfmac(ns0, yf0, yb_0);
        cfma(ns1, yf1, yf_1);
        cfmac(ns1, yf1, yb_1);
        if (zact) {
            float wz_f = 1.f, wz_b = 1.f;
            if (!zper) {
                if (k == 0) {
                    wz_f = 2.f;
                    wz_b = 0.f;
                } else if (k == g.nz - 1) {
                    wz_f = 0.f;
                    wz_b = 2.f;
                }
            }
            const float4 pzp = Pp.psi[r + 1][tx + 1];
            const float4 zpp = (wz_f == 1.f) ? pzp : make_float4(wz_f * pzp.x, wz_f * pzp.y, wz_f * pzp.z, wz_f * pzp.w);
            const float4 zmm = (wz_b == 1.f) ? pzm : make_float4(wz_b * pzm.x, wz_b * pzm.y, wz_b * pzm.z, wz_b * pzm.w);
            cfma(ns0, zf0, lo2(zpp));
            cfmac(ns0, zf0, lo2(zmm));
            cfma(ns1, zf1, hi2(zpp));
            cfmac(ns1, zf1, hi2(zmm));
        }
        pzm = pc;
        if (RHS) {
            float f0 = (c0.x * ns0.y - c0.y * ns0.x) * inv_ht2;
            float f1 = (c1.x * ns1.y - c1.y * ns1.x) * inv_ht2;
            if (!xper) {
                if (xlo) f0 -= a.inj;
                if (xhi) f1 += a.inj;
            }
            reinterpret_cast<float2 *>(a.f)[q0 + plq * k] = make_float2(f0, f1);
            dst[q0 + plq * k] = pc;
            const float wz = (g.bcz == kOpen && g.nz >= 2 && (k == 0 || k == g.nz - 1)) ? 0.5f : 1.f;
            facc += wz * (wxy0 * f0 + wxy1 * f1);
            continue;
        }
        float2 b0, b1, D0, D1;
        if (INIT) {
            // b and diag M of the pair from psi^n, mu and alpha (sweep2_body's MODE 1 order)
            const float2 mu_n = stage_pair(Pc, 0, r, tx);
            const float2 muc = make_float2(mu_n.x - offS, mu_n.y - offS), alc = stage_pair(Pc, 1, r, tx);
            const float2 cs[2] = {c0, c1};
            const float2 nss[2] = {ns0, ns1};
            const float mus[2] = {muc.x, muc.y}, als[2] = {alc.x, alc.y};
            const float S2 = 2.f * g.S;
            const long long m = (long long)x + (long long)g.nx * jc + sz * k;
            float2 bo[2], Do[2];
#pragma unroll
            for (int s2 = 0; s2 < 2; ++s2) {
                const float a2 = cabs2(cs[s2]);
                Do[s2] = cmk(1.f + g.ht2 * (g.beta * a2 + S2 - als[s2]), g.ht2 * g.u * mus[s2]);
                const float cr = als[s2] - g.beta * a2 - S2;
                const float ci = -g.u * mus[s2];
                const float2 lin = cmk(cr * cs[s2].x - ci * cs[s2].y, cr * cs[s2].y + ci * cs[s2].x);
                bo[s2] = cadd(cadd(cs[s2], cscale(g.ht2, lin)), nss[s2]);
                if (a.noise_amp != 0.f) {
                    // thermal noise h_t zeta_m (Sec. 3.1.2), counter (site, step)
                    const float2 v = noise_uv(a.noise_seed, m + s2, nstep);
                    bo[s2] = cmk(bo[s2].x + a.noise_amp * v.x, bo[s2].y + a.noise_amp * v.y);
                }
            }
            b0 = bo[0];
            b1 = bo[1];
            D0 = Do[0];
            D1 = Do[1];
            reinterpret_cast<float4 *>(a.b)[q0 + plq * k] = make_float4(b0.x, b0.y, b1.x, b1.y);
            reinterpret_cast<float4 *>(a.D)[q0 + plq * k] = make_float4(D0.x, D0.y, D1.x, D1.y);
            // the coming Poisson solve starts from a mu^(n-1) + b mu^(n-2), written over the latter
            if (guess && (!a.guess_odd_only || ((j + k) & 1))) {
                const float2 pgc = stage_pair(Pc, 2, r, tx);
                reinterpret_cast<float2 *>(a.mu_guess)[q0 + plq * k] =
                    make_float2(a.ex_a * muc.x + a.ex_b * (pgc.x - offP), a.ex_a * muc.y + a.ex_b * (pgc.y - offP));
            }
        } else {
            const float4 bc = stage_b(Pc, r, tx), Dc = stage_D(Pc, r, tx);
            b0 = lo2(bc);
            b1 = hi2(bc);
            D0 = lo2(Dc);
            D1 = hi2(Dc);
        }
        const float2 s0 = cadd(b0, ns0), s1 = cadd(b1, ns1);
        const float2 r0 = csub(s0, cmul(D0, c0)), r1 = csub(s1, cmul(D1, c1));
        const float2 n0 = cscale(__frcp_rn(cabs2(D0)), cmulc(D0, s0));
        const float2 n1 = cscale(__frcp_rn(cabs2(D1)), cmulc(D1, s1));
        dst[q0 + plq * k] = make_float4(n0.x, n0.y, n1.x, n1.y);
        float r2a = cabs2(r0), r2b = cabs2(r1);
        r2a = (r2a <= FLT_MAX) ? r2a : INFINITY;
        r2b = (r2b <= FLT_MAX) ? r2b : INFINITY;
        rmax = fmaxf(rmax, fmaxf(r2a, r2b));
    }
    // every copy has landed (the groups still counted are empty) before the ring is reused
    cp_async_wait<0>();
}

}  // namespace tdgl
