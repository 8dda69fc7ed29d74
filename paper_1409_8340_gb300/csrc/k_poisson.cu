// Scalar potential: exact discrete solve of Lap mu = F (arXiv:1409.8340, Sec. 3.2,
// Eq. Poisson; the fixed point of the paper's pseudo-time relaxation) by
// geometric multigrid.
//
// x is never coarsened: every level keeps all Nx points and is smoothed by
// zebra x-line Gauss-Seidel.  Every x line of a level carries the same
// constant-coefficient operator T = tridiag(-cx, 2cx + s, -cx) (s = 2 cy + 2 cz),
// periodic on a periodic x axis; on an open x axis the Neumann rows make it the
// restriction of the periodic operator on the mirrored line of period
// P = 2(Nx - 1).  So T^{-1} is a circular convolution with the periodized Green's
// function G_k = (1/P) sum_m cos(2 pi m k / P) / (2 cx (1 - cos(2 pi m / P)) + s),
// which decays like rho^|k| (rho = 0.17 on the finest level of an isotropic
// grid): it is precomputed in FP64 on the host and truncated where it falls
// below 2e-9 G_0, so a line solve is a short, fully parallel convolution.
//
// y and z are coarsened by 2 while the size allows (periodic: even N >= 8; open:
// odd N >= 5), with full weighting and bilinear interpolation.  The coarsest
// level is solved exactly: its small y-z operator is diagonalised by a dense
// basis V (Fourier modes on periodic axes, DCT-I modes on open axes), and each
// mode q is a line problem with shift sigma_q, solved with its own Green's
// function (the pseudo-inverse for the singular mode).  The zero mode
// (constants) is removed in FP64: the right-hand side is projected onto
// sum_m w_m F_m = 0 and the solution onto sum_m w_m mu_m = 0, w the trapezoid
// weights (1/2 per open face).
#include <cudaTypedefs.h>
#include <float.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "mg_tile.cuh"
#include "tma_util.cuh"

namespace tdgl {

constexpr int kThreads = 256;

static int grid_blocks(long long n, int per_thread = 4)
{
    long long b = (n + (long long)kThreads * per_thread - 1) / ((long long)kThreads * per_thread);
    if (b < 1) b = 1;
    if (b > 8192) b = 8192;
    return (int)b;
}

// ---------------------------------------------------------------------------
// host: Green's functions
// ---------------------------------------------------------------------------
int mg_period(int nx, int bcx) { return bcx == kOpen ? 2 * (nx - 1) : nx; }

// G_k, k = 0..P-1, of T = tridiag(-cx, 2cx + s, -cx) on a ring of P points.
// s == 0: pseudo-inverse (the constant mode dropped).
static void green(int P, double cx, double s, std::vector<double> &G)
{
    const double pi = 3.14159265358979323846;
    std::vector<double> ct(P), inv(P);
    for (int j = 0; j < P; ++j) ct[j] = cos(2.0 * pi * j / P);
    for (int m = 0; m < P; ++m) {
        double lam = 2.0 * cx * (1.0 - ct[m]) + s;
        inv[m] = (s == 0.0 && m == 0) ? 0.0 : 1.0 / lam;
    }
    G.assign(P, 0.0);
    for (int k = 0; k < P; ++k) {
        double acc = 0.0;
        long long idx = 0;
        for (int m = 0; m < P; ++m) {
            acc += ct[idx] * inv[m];
            idx += k;
            if (idx >= P) idx -= P;
        }
        G[k] = acc / P;
    }
}

// Fills Gs (length kmax - kmin + 1, Gs[k - kmin] = G_k) for the line operator of
// a level; returns kmin (kmax = -kmin for a truncated kernel, P - 1 for a full one).
int mg_line_kernel(int nx, int bcx, double cx, double s, std::vector<float> &Gs)
{
    const int P = mg_period(nx, bcx);
    std::vector<double> G;
    green(P, cx, s, G);
    int B = 0;
    for (int k = 1; k <= P / 2; ++k)
        if (fabs(G[k]) > 2e-9 * fabs(G[0])) B = k;
    Gs.clear();
    if (2 * B + 1 < P) {
        for (int k = -B; k <= B; ++k) Gs.push_back((float)G[(k + P) % P]);
        return -B;
    }
    for (int k = 0; k < P; ++k) Gs.push_back((float)G[k]);
    return 0;
}

long long mg_lines_of_colour(int ny, int nz, int c)
{
    long long n = 0;
    for (int k = 0; k < nz; ++k) n += (ny + 1 - ((c + k) & 1)) / 2;
    return n;
}

// ---------------------------------------------------------------------------
// zebra x-line smoother
// ---------------------------------------------------------------------------
struct LineArgs {
    MGLevel L;
    int bcx, bcy, bcz;
    int color;
    long long nlines;
    LineShape sh;
    const DevCtl *ctl;
    int level0;
    // weighted sum of the final mu over the last two finest-level passes (recursive
    // smoother only): stage 1 (colour 1) leaves block partials in blockred[0, nb1);
    // stage 2 (colour 0) adds its own at blockred[kMeanOff + b] and its last block writes
    // ctl->mu_mean.  0: off.
    int mean_stage, mean_nb1;
    int mean_dot, dot_slot;   // the sum is of w r u, into ctlw->sums[dot_slot] (PoissonArgs)
    DevCtl *ctlw;
    double *blockred;
    double wsum;
    unsigned long long wait_ns;   // staged smoother: wait bound (0: default)
    unsigned int extra_tx;        // staged smoother: extra expected bytes (0 in normal use)
};
constexpr int kMeanOff = 4096;

__global__ void __launch_bounds__(kThreads) line_smooth_kernel(LineArgs A)
{
    extern __shared__ __align__(16) float sm[];
    const float fsub = A.level0 ? (float)A.ctl->fmean : 0.f;
    line_smooth_lines<false>(A.L, A.sh, A.bcx, A.bcy, A.bcz, A.color, A.nlines, fsub, blockIdx.x, threadIdx.x,
                             blockDim.x, sm);
}

// 2D launch over (x, y) with a loop over z: thread (i, j) walks its z column.
constexpr int kGX = 128;
static dim3 grid_xy(int nx, int ny) { return dim3((nx + kGX - 1) / kGX, ny); }
// 3D launch: (x, y, z-chunk of kGZ planes), enough independent threads to cover memory latency
constexpr int kGZ = 4;
static dim3 grid_xyz(int nx, int ny, int nz) { return dim3((nx + kGX - 1) / kGX, ny, (nz + kGZ - 1) / kGZ); }

// t = F - L u on one level (level 0: F = f - fmean)
// skip_color >= 0: rows (j, k) of that zebra colour are left out (their residual is zero
// right after that colour's exact line solves; the restriction does not read them)
__global__ void __launch_bounds__(kGX) residual_kernel(MGLevel L, int bcx, int bcy, int bcz, const DevCtl *ctl, int level0,
                                                      int skip_color)
{
    const int i = blockIdx.x * kGX + threadIdx.x, j = blockIdx.y;
    if (i >= L.nx) return;
    const float fsub = level0 ? (float)ctl->fmean : 0.f;
    const long long pl = (long long)L.nx * L.ny;
    float *__restrict__ tt = L.t;
    const int ka = blockIdx.z * kGZ, kb = min(ka + kGZ, L.nz);
#pragma unroll
    for (int dk = 0; dk < kGZ; ++dk) {
        const int k = ka + dk;
        if (k >= kb) break;
        if (skip_color >= 0 && ((j + k) & 1) == skip_color) continue;
        const long long m = i + (long long)L.nx * j + pl * k;
        tt[m] = residual_at<false>(L, bcx, bcy, bcz, fsub, i, j, k, m);
    }
}

// Four-site versions (nx % 4 == 0): thread (i0 / 4, j) of a kGX-thread block over
// 4 kGX x sites, kGZ planes per block.
static dim3 grid_xyz4(int nx, int ny, int nz) { return dim3((nx / 4 + kGX - 1) / kGX, ny, (nz + kGZ - 1) / kGZ); }

__global__ void __launch_bounds__(kGX) residual4_kernel(MGLevel L, int bcx, int bcy, int bcz, const DevCtl *ctl,
                                                       int level0, int skip_color)
{
    const int i0 = (blockIdx.x * kGX + threadIdx.x) * 4, j = blockIdx.y;
    if (i0 >= L.nx) return;
    const float fsub = level0 ? (float)ctl->fmean : 0.f;
    const long long pl = (long long)L.nx * L.ny;
    const int ka = blockIdx.z * kGZ, kb = min(ka + kGZ, L.nz);
#pragma unroll
    for (int dk = 0; dk < kGZ; ++dk) {
        const int k = ka + dk;
        if (k >= kb) break;
        if (skip_color >= 0 && ((j + k) & 1) == skip_color) continue;
        *reinterpret_cast<float4 *>(L.t + i0 + (long long)L.nx * j + pl * k) = residual4_at<false>(L, bcx, bcy, bcz, fsub, i0, j, k);
    }
}

__global__ void __launch_bounds__(kGX) restrict4_kernel(MGLevel F, MGLevel C, int bcy, int bcz, int zero_color)
{
    const int i0 = (blockIdx.x * kGX + threadIdx.x) * 4, J = blockIdx.y;
    if (i0 >= C.nx) return;
    const int nx = C.nx;
    const int Ka = blockIdx.z * kGZ, Kb = min(Ka + kGZ, C.nz);
#pragma unroll
    for (int dK = 0; dK < kGZ; ++dK) {
        const int K = Ka + dK;
        if (K >= Kb) break;
        const long long m = i0 + (long long)nx * (J + (long long)C.ny * K);
        *reinterpret_cast<float4 *>(C.r + m) = restrict4_at<false>(F, bcy, bcz, i0, J, K, zero_color);
        *reinterpret_cast<float4 *>(C.u + m) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

constexpr int kRZ = 4;   // coarse planes per block (at most; fewer on small levels)
struct Rows3 {
    float4 m, c, p;   // rows 2J-1, 2J, 2J+1 of one fine plane
};

__device__ __forceinline__ float4 ldg4(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }

// FAST: every fine row and plane the block touches is interior (no wrap or mirror), so
// the plane and row bookkeeping is fixed at compile time and each coarse plane's loads
// are independent of one another.
template <bool FAST>
__device__ __forceinline__ void residual_restrict_march(const MGLevel &F, const MGLevel &C, int bcx, int bcy, int bcz,
                                                        float fsub, int i0, int J, int Ka, int Kb)
{
    const int nx = F.nx, ny = F.ny, nz = F.nz;
    const long long pl = (long long)nx * ny;
    const int j0 = 2 * J, jm = nb_idx(j0, -1, ny, bcy), jp = nb_idx(j0, 1, ny, bcy);
    // y neighbours of the outer rows (those of the centre row are jm and jp)
    const int jmm = nb_idx(jm, -1, ny, bcy), jmp = nb_idx(jm, 1, ny, bcy);
    const int jpm = nb_idx(jp, -1, ny, bcy), jpp = nb_idx(jp, 1, ny, bcy);
    const int xl = nb_idx(i0, -1, nx, bcx), xr = nb_idx(i0 + 3, 1, nx, bcx);
    const float *u = F.u;
    auto load3 = [&](int k) {
        const float *b = u + pl * k + i0;
        Rows3 t;
        t.m = ldg4(b + (long long)nx * jm);
        t.c = ldg4(b + (long long)nx * j0);
        t.p = ldg4(b + (long long)nx * jp);
        return t;
    };
    // residual of the three rows of plane k from its rows U and the rows of the planes
    // below (Zm) and above (Zp)
    auto resid3 = [&](int k, const Rows3 &U, const Rows3 &Zm, const Rows3 &Zp, float4 &tm, float4 &tc, float4 &tp) {
        const float *ub = u + pl * k;
        const float *rb = F.r + pl * k + i0;
        {
            const float *row = ub + (long long)nx * jm;
            const float4 ym = ldg4(ub + (long long)nx * jmm + i0);
            const float4 yp = (FAST || jmp == j0) ? U.c : ldg4(ub + (long long)nx * jmp + i0);
            tm = residual4_core(F, fsub, U.m, ldg4(rb + (long long)nx * jm), __ldg(row + xl), __ldg(row + xr), true, yp,
                                ym, true, Zp.m, Zm.m);
        }
        {
            const float *row = ub + (long long)nx * j0;
            tc = residual4_core(F, fsub, U.c, ldg4(rb + (long long)nx * j0), __ldg(row + xl), __ldg(row + xr), true, U.p,
                                U.m, true, Zp.c, Zm.c);
        }
        {
            const float *row = ub + (long long)nx * jp;
            const float4 ym = (FAST || jpm == j0) ? U.c : ldg4(ub + (long long)nx * jpm + i0);
            const float4 yp = ldg4(ub + (long long)nx * jpp + i0);
            tp = residual4_core(F, fsub, U.p, ldg4(rb + (long long)nx * jp), __ldg(row + xl), __ldg(row + xr), true, yp,
                                ym, true, Zp.p, Zm.p);
        }
    };
    // acc += w t in restrict4_at's order (rows 2J-1, 2J, 2J+1 of one fine plane)
    auto add3 = [](float4 &acc, float wk, const float4 &tm, const float4 &tc, const float4 &tp) {
        const float4 ts[3] = {tm, tc, tp};
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const float wj = (b == 1) ? 0.5f : 0.25f;
            acc.x += wk * wj * ts[b].x;
            acc.y += wk * wj * ts[b].y;
            acc.z += wk * wj * ts[b].z;
            acc.w += wk * wj * ts[b].w;
        }
    };
    // plane 2Ka - 1 (A) and 2Ka (B)
    int pA = FAST ? 2 * Ka - 1 : nb_idx(2 * Ka, -1, nz, bcz);
    Rows3 uA = load3(pA), uB = load3(2 * Ka);
    float4 tAm, tAc, tAp;
    {
        const int zm = FAST ? pA - 1 : nb_idx(pA, -1, nz, bcz), zp = FAST ? pA + 1 : nb_idx(pA, 1, nz, bcz);
        const Rows3 Zm = (!FAST && zm == 2 * Ka) ? uB : load3(zm);
        const Rows3 Zp = (FAST || zp == 2 * Ka) ? uB : load3(zp);
        resid3(pA, uA, Zm, Zp, tAm, tAc, tAp);
    }
    for (int K = Ka; K < Kb; ++K) {
        // planes A = nb(2K, -1) (pA), B = 2K, C = nb(2K, +1); N = nb(C, +1)
        const int pB = 2 * K;
        const int pC = FAST ? pB + 1 : nb_idx(pB, 1, nz, bcz);
        const int pN = FAST ? pB + 2 : nb_idx(pC, 1, nz, bcz);
        const Rows3 uC = (!FAST && pC == pA) ? uA : load3(pC);
        const Rows3 uN = (!FAST && pN == pB) ? uB : load3(pN);
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        add3(acc, 0.25f, tAm, tAc, tAp);
        {
            float4 tBm, tBc, tBp;
            resid3(pB, uB, uA, uC, tBm, tBc, tBp);
            add3(acc, 0.5f, tBm, tBc, tBp);
        }
        {
            const int cm = FAST ? pB : nb_idx(pC, -1, nz, bcz);
            const Rows3 Zm = (FAST || cm == pB) ? uB : load3(cm);
            resid3(pC, uC, Zm, uN, tAm, tAc, tAp);   // plane C's residual, carried as the next A
            add3(acc, 0.25f, tAm, tAc, tAp);
        }
        const long long m = i0 + (long long)C.nx * (J + (long long)C.ny * K);
        *reinterpret_cast<float4 *>(C.r + m) = acc;
        *reinterpret_cast<float4 *>(C.u + m) = make_float4(0.f, 0.f, 0.f, 0.f);
        if (K + 1 < Kb) {
            uA = uC;
            pA = pC;
            uB = (FAST || pN == pB + 2) ? uN : load3(pB + 2);
        }
    }
}

// Residual and full-weighting restriction in one pass, for a level coarsened by 2 in
// both y and z (the fine residual t is never stored).  Thread (i0 / 4, J) marches over
// the coarse planes K of its block: coarse site (J, K) sums t over the fine rows
// 2J-1, 2J, 2J+1 (mirrored or wrapped at the ends) of the fine planes 2K-1, 2K, 2K+1
// with the weights of restrict4_at, in its order.  The residual of plane 2K+1 is the
// 2K'-1 plane of the next coarse plane and is carried over; the u rows of a fine plane
// are loaded once and kept while the planes next to it need them.  The residual of each
// fine site is residual4_at's arithmetic, so the coarse right-hand side equals that of
// residual4_kernel followed by restrict4_kernel.
// Six blocks per SM (80 registers, a few spilled bytes) hide more of the load latency
// than four without spills: 138 against 154 us at 512x512x256.
template <int RZ>
__global__ void __launch_bounds__(kGX, 6) residual_restrict4_kernel(MGLevel F, MGLevel C, int bcx, int bcy, int bcz,
                                                                    const DevCtl *ctl, int level0)
{
    const int i0 = (blockIdx.x * kGX + threadIdx.x) * 4, J = blockIdx.y;
    if (i0 >= F.nx) return;
    const float fsub = level0 ? (float)ctl->fmean : 0.f;
    const int Ka = blockIdx.z * RZ, Kb = min(Ka + RZ, C.nz);
    // interior block: rows 2J-2 .. 2J+2 and planes 2Ka-2 .. 2Kb exist without wrap or mirror
    const bool fast = (2 * J - 2 >= 0) && (2 * J + 2 <= F.ny - 1) && (2 * Ka - 2 >= 0) && (2 * Kb <= F.nz - 1);
    if (fast) residual_restrict_march<true>(F, C, bcx, bcy, bcz, fsub, i0, J, Ka, Kb);
    else residual_restrict_march<false>(F, C, bcx, bcy, bcz, fsub, i0, J, Ka, Kb);
}

// only_color >= 0: only rows of that zebra colour take the correction (the other
// colour's lines are solved exactly next, from r and these rows alone).  GZ planes per
// block (one on small levels, for more blocks).
template <int GZ>
__global__ void __launch_bounds__(kGX) prolong4_kernel(MGLevel F, MGLevel C, int bcy, int bcz, int only_color)
{
    const int i0 = (blockIdx.x * kGX + threadIdx.x) * 4, j = blockIdx.y;
    if (i0 >= F.nx) return;
    const int nx = F.nx;
    const int ka = blockIdx.z * GZ, kb = min(ka + GZ, F.nz);
#pragma unroll
    for (int dk = 0; dk < GZ; ++dk) {
        const int k = ka + dk;
        if (k >= kb) break;
        if (only_color >= 0 && ((j + k) & 1) != only_color) continue;
        float4 *p = reinterpret_cast<float4 *>(F.u + i0 + (long long)nx * (j + (long long)F.ny * k));
        const float4 v = prolong4_at<false>(F, C, bcy, bcz, i0, j, k);
        const float4 o = *p;
        *p = make_float4(o.x + v.x, o.y + v.y, o.z + v.z, o.w + v.w);
    }
}

// max |F - L u| and max |F| on level 0 (ctl->res = ratio)
__global__ void __launch_bounds__(kGX) residual_norm_kernel(MGLevel L, int bcx, int bcy, int bcz, DevCtl *ctl,
                                                            double *blockred)
{
    const int i = blockIdx.x * kGX + threadIdx.x, j = blockIdx.y;
    const float fsub = (float)ctl->fmean;
    float rmax = 0.f, fmax = 0.f;
    if (i < L.nx) {
        const long long pl = (long long)L.nx * L.ny;
        for (int k = 0; k < L.nz; ++k) {
            const long long m = i + (long long)L.nx * j + pl * k;
            const float F = L.r[m] - fsub;
            rmax = fmaxf(rmax, fabsf(F - lap_at<false>(L, L.u, i, j, k, m, bcx, bcy, bcz)));
            fmax = fmaxf(fmax, fabsf(F));
        }
    }
    __shared__ float shf[32];
    __shared__ int flag;
    const unsigned int bid = blockIdx.x + gridDim.x * blockIdx.y, nb = gridDim.x * gridDim.y;
    float a = block_max(rmax, shf);
    float b = block_max(fmax, shf);
    if (threadIdx.x == 0) {
        blockred[2 * bid] = a;
        blockred[2 * bid + 1] = b;
    }
    if (!last_block(&ctl->ticket, nb, &flag)) return;
    float ra = 0.f, rb = 0.f;
    for (unsigned int q = threadIdx.x; q < nb; q += blockDim.x) {
        ra = fmaxf(ra, (float)((volatile double *)blockred)[2 * q]);
        rb = fmaxf(rb, (float)((volatile double *)blockred)[2 * q + 1]);
    }
    ra = block_max(ra, shf);
    rb = block_max(rb, shf);
    if (threadIdx.x == 0) {
        ctl->ticket = 0u;
        ctl->fmax = rb;
        ctl->res = rb > 0.f ? (double)ra / (double)rb : (double)ra;
    }
}

// r_c = full weighting of t_f (y, z); u_c = 0.  Grid over the coarse (x, y).
__global__ void __launch_bounds__(kGX) restrict_kernel(MGLevel F, MGLevel C, int bcy, int bcz, int zero_color)
{
    const int i = blockIdx.x * kGX + threadIdx.x, J = blockIdx.y;
    if (i >= C.nx) return;
    const int nx = C.nx;
    const int Ka = blockIdx.z * kGZ, cnt = min(kGZ, C.nz - Ka);
    float acc[kGZ];
#pragma unroll
    for (int dK = 0; dK < kGZ; ++dK)
        if (dK < cnt) acc[dK] = restrict_at<false>(F, bcy, bcz, i, J, Ka + dK, zero_color);
#pragma unroll
    for (int dK = 0; dK < kGZ; ++dK) {
        if (dK < cnt) {
            const long long m = i + (long long)nx * (J + (long long)C.ny * (Ka + dK));
            C.r[m] = acc[dK];
            C.u[m] = 0.f;
        }
    }
}

// u_f += bilinear interpolation of u_c.  Grid over the fine (x, y).
__global__ void __launch_bounds__(kGX) prolong_kernel(MGLevel F, MGLevel C, int bcy, int bcz, int only_color)
{
    const int i = blockIdx.x * kGX + threadIdx.x, j = blockIdx.y;
    if (i >= F.nx) return;
    const int nx = F.nx;
    const int ka = blockIdx.z * kGZ, kb = min(ka + kGZ, F.nz);
#pragma unroll
    for (int dk = 0; dk < kGZ; ++dk) {
        const int k = ka + dk;
        if (k >= kb) break;
        if (only_color >= 0 && ((j + k) & 1) != only_color) continue;
        const float v = prolong_at<false>(F, C, bcy, bcz, i, j, k);
        F.u[i + (long long)nx * (j + (long long)F.ny * k)] += v;
    }
}

// Zebra x-line Gauss-Seidel by the recursive exact line solve (levels with short
// decay): one warp per line, C = nx / 32 consecutive sites per lane.  The line
// operator T = (2 cx + s) - cx (S- + S+) equals (cx / rho)(1 - rho S-)(1 - rho S+), so
// u = (rho / cx) (1 - rho S+)^-1 (1 - rho S-)^-1 E: a forward recursion w_x = E_x +
// rho w_(x-1), then a backward one z_x = w_x + rho z_(x+1), u = (rho / cx) z.  Each lane
// starts its forward recursion from the C values before its chunk (the previous lane's,
// by shuffle) and its backward recursion from the C w-values after it (the next
// lane's): the dropped terms carry rho^C <= 1e-9.  The ends of the line use the
// periodic wrap or the Neumann mirror of the extended line, as the convolution does.
template <int C>
__global__ void __launch_bounds__(kThreads) line_iir_kernel(LineArgs A)
{
    const MGLevel &L = A.L;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const long long line = (long long)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
    if (line >= A.nlines) return;   // whole warps
    const float fsub = A.level0 ? (float)A.ctl->fmean : 0.f;
    int j, k;
    line_jk(line, A.color, L.ny, L.nz, j, k);
    const int nx = L.nx;
    const long long plane = (long long)nx * L.ny;
    const long long base = (long long)nx * j + plane * k;
    const bool ya = L.ny >= 2, za = L.nz >= 2;
    const float *rr = L.r + base;
    const float *up = ya ? L.u + (long long)nx * nb_idx(j, 1, L.ny, A.bcy) + plane * k : rr;
    const float *um = ya ? L.u + (long long)nx * nb_idx(j, -1, L.ny, A.bcy) + plane * k : rr;
    const float *zp = za ? L.u + (long long)nx * j + plane * nb_idx(k, 1, L.nz, A.bcz) : rr;
    const float *zm = za ? L.u + (long long)nx * j + plane * nb_idx(k, -1, L.nz, A.bcz) : rr;
    const int i0 = lane * C;
    float e[C];
#pragma unroll
    for (int h = 0; h < C; h += 4) {
        const float4 a = *reinterpret_cast<const float4 *>(rr + i0 + h);
        const float4 yp = *reinterpret_cast<const float4 *>(up + i0 + h);
        const float4 ym = *reinterpret_cast<const float4 *>(um + i0 + h);
        const float4 kp = *reinterpret_cast<const float4 *>(zp + i0 + h);
        const float4 km = *reinterpret_cast<const float4 *>(zm + i0 + h);
        const float av[4] = {a.x, a.y, a.z, a.w}, ypv[4] = {yp.x, yp.y, yp.z, yp.w}, ymv[4] = {ym.x, ym.y, ym.z, ym.w},
                    kpv[4] = {kp.x, kp.y, kp.z, kp.w}, kmv[4] = {km.x, km.y, km.z, km.w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float x = -(av[c] - fsub);
            if (ya) x += L.cy * (ypv[c] + ymv[c]);
            if (za) x += L.cz * (kpv[c] + kmv[c]);
            e[h + c] = x;
        }
    }
    const bool open = (A.bcx == kOpen);
    const float rho = L.rho;
    // values beyond the chunk that the two mirrored ends need: e(C) from lane 1 (left
    // mirror, lane 0) and e(nx - 1 - C) from lane 30 (right mirror, lane 31)
    const float e_next0 = __shfl_sync(FULL, e[0], 1);
    const float e_prevlast = __shfl_sync(FULL, e[C - 1], 30);
    // forward warm-up over x = i0 - C .. i0 - 1
    float w = 0.f;
#pragma unroll
    for (int m = 0; m < C; ++m) {
        float v = __shfl_sync(FULL, e[m], (lane + 31) & 31);
        if (open && lane == 0) v = (m == 0) ? e_next0 : e[C - m];   // e_ext(-d) = e(d), d = C - m
        w = fmaf(rho, w, v);
    }
    float wv[C];
#pragma unroll
    for (int m = 0; m < C; ++m) {
        w = fmaf(rho, w, e[m]);
        wv[m] = w;
    }
    // right mirror: the forward recursion continued over e_ext(nx + m) = e(nx - 2 - m)
    float wext[C];
    {
        float wc = wv[C - 1];
#pragma unroll
        for (int m = 0; m < C; ++m) {
            const float v = (m <= C - 2) ? e[C - 2 - m] : e_prevlast;
            wc = fmaf(rho, wc, v);
            wext[m] = wc;
        }
    }
    // backward warm-up over x = i0 + 2C - 1 down to i0 + C
    float z = 0.f;
#pragma unroll
    for (int m = C - 1; m >= 0; --m) {
        float v = __shfl_sync(FULL, wv[m], (lane + 1) & 31);
        if (open && lane == 31) v = wext[m];
        z = fmaf(rho, z, v);
    }
    float out[C];
#pragma unroll
    for (int m = C - 1; m >= 0; --m) {
        z = fmaf(rho, z, wv[m]);
        out[m] = z * L.rscale;
    }
    float *dst = L.u + base + i0;
#pragma unroll
    for (int h = 0; h < C; h += 4)
        *reinterpret_cast<float4 *>(dst + h) = make_float4(out[h], out[h + 1], out[h + 2], out[h + 3]);
}

// The same recursive line solve with the line's four neighbour rows brought into shared
// memory by 16-byte asynchronous copies, one buffer per warp: as soon as a line's
// right-hand side e is in registers the buffer takes the next line's copies, which fly
// while the warp runs the recursions (the long part of a line), so the loads of a whole
// line are in flight without holding them in registers.  The line's own row of r (16
// values per lane) goes to registers one line ahead.  At 9 KB of shared memory per warp,
// up to 24 warps (independent recursion chains) fit on an SM.  Rows are stored with 4
// floats of padding per 32 (the lanes' 16-site chunks then fall on distinct banks).
constexpr int kIirWarps = 4;
__device__ __forceinline__ int pad32(int t) { return t + 4 * (t >> 5); }

__device__ __forceinline__ void cp_async16(float *dst, const float *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}

// W = 12 (levels with rho^12 <= 1e-8, below FP32 rounding): each lane warms its
// recursions up over the last 12 values of the previous lane (the first 12 of the next).
// W = 0 (every other level): the exact solve by scans over the lanes, for any rho < 1.
// Each lane runs both recursions from zero over its chunk; the value entering a chunk is
// a linear recurrence over the lanes (c_L = rho^C c_(L-1) + end_(L-1)), evaluated by a
// five-step shuffle scan; it is seeded at the line's ends in closed form: w(-1) is a
// weighted sum over the periodic or mirrored extension (a warp reduction), and the
// backward seed z(N) follows from the mirror symmetry of the solution (z(N) = z(N - 2))
// or, on a periodic line, from a second weighted sum.
// TMA: the four rows come as four boxes of the level's tensor map (one lane issues them,
// completing the warp's mbarrier) into an unpadded 8 KB buffer in the 128-byte swizzled
// layout, which keeps the lanes' 16-byte reads on distinct banks: no per-lane copies.
// Each wait is bounded; one that runs out records TDGL_ERR_TIMEOUT and ends the warp's
// lines after its copies in flight have landed (again bounded).
constexpr int kIirTmaBytes = 4 * 512 * 4;   // a warp's buffer: four 512-site rows
constexpr unsigned long long kIirWaitNs = 2000000000ull;
template <int C, int W, bool TMA>
__global__ void __launch_bounds__(kIirWarps * 32, 6)
    line_iir_async_kernel(LineArgs A, const __grid_constant__ CUtensorMap map_u)
{
    static_assert(W >= 0 && W <= C, "warm-up within the previous lane (0: exact scan)");
    static_assert(!TMA || C == 16, "tensor-map boxes hold 512-site lines");
    constexpr int NX = 32 * C, ROW = TMA ? NX : NX + NX / 8;   // row length in floats (padded for copies)
    extern __shared__ __align__(16) float sm_iir[];
    const MGLevel &L = A.L;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    float *sm_base = sm_iir;
    if (TMA)   // the swizzled layout repeats every 1024 bytes: buffers on 1024-byte boundaries
        sm_base = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(sm_iir) + 1023) & ~(uintptr_t)1023);
    float *buf = sm_base + (size_t)wib * 4 * ROW;   // [4 rows][ROW]
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(sm_base + (size_t)kIirWarps * 4 * ROW) + wib;
    unsigned parity = 0u;
    bool issued = false;   // TMA: a line's boxes are in flight
    if (TMA) {
        if (lane == 0) {
            mbar_init(bar, 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncwarp();
    }
    const unsigned long long wait_ns = A.wait_ns ? A.wait_ns : kIirWaitNs;
    // timeout test only: the first warp's boxes expect bytes that never come
    const unsigned xtx = (blockIdx.x == 0 && wib == 0) ? A.extra_tx : 0u;
    const unsigned long long deadline = TMA ? gtime() + wait_ns : 0ull;
    // exact solve (W = 0): the lane's powers of rho, once per kernel: the weights of its
    // first (pw_f1) and last (pw_f2) site in w(-1), of its first site in z(N) (pw_b), and
    // the carries' seeds rho^(C(L+1)) (pw_c1) and rho^(C(32-L)) (pw_c2)
    float pw_f1 = 0.f, pw_f2 = 0.f, pw_b = 0.f, pw_c1 = 0.f, pw_c2 = 0.f;
    if (W == 0) {
        const int N = 32 * C, x0 = lane * C, x1 = x0 + C - 1;
        const bool op = (A.bcx == kOpen);
        pw_f1 = exp2f(L.l2rho * (float)(x0 - 1));
        pw_f2 = exp2f(L.l2rho * (float)(op ? 2 * N - 3 - x1 : N - 1 - x1));
        pw_b = exp2f(L.l2rho * (float)x0);
        pw_c1 = exp2f(L.l2rho * (float)(C * (lane + 1)));
        pw_c2 = exp2f(L.l2rho * (float)(C * (32 - lane)));
    }
    const long long nwarps = (long long)gridDim.x * kIirWarps;
    const long long first = (long long)blockIdx.x * kIirWarps + wib;
    const float fsub = A.level0 ? (float)A.ctl->fmean : 0.f;
    const long long plane = (long long)NX * L.ny;
    const bool ya = L.ny >= 2, za = L.nz >= 2;
    const int i0 = lane * C;
    // the staged rows of a line: u(j+1), u(j-1), u(k+1), u(k-1) (an inactive axis points
    // at the line's own row, whose values are not used); its r row goes to registers
    auto issue = [&](long long line, float *dst, float4 *rv) {
        int j, k;
        line_jk(line, A.color, L.ny, L.nz, j, k);
        const long long base = (long long)NX * j + plane * k;
        long long src[4];   // float offsets of the rows in u
        src[0] = ya ? (long long)NX * nb_idx(j, 1, L.ny, A.bcy) + plane * k : base;
        src[1] = ya ? (long long)NX * nb_idx(j, -1, L.ny, A.bcy) + plane * k : base;
        src[2] = za ? (long long)NX * j + plane * nb_idx(k, 1, L.nz, A.bcz) : base;
        src[3] = za ? (long long)NX * j + plane * nb_idx(k, -1, L.nz, A.bcz) : base;
        if constexpr (TMA) {
            if (lane == 0) {
                // the warp's reads of the buffer (generic proxy) precede these writes
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_expect(bar, (unsigned)kIirTmaBytes + xtx);
#pragma unroll
                for (int a = 0; a < 4; ++a) tma_load2(dst + a * ROW, &map_u, 0, (int)(src[a] >> 5), bar);
            }
            issued = true;
        } else {
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int h = 0; h < C / 4; ++h) {
                    const int t = 4 * (h * 32 + lane);   // coalesced: lane-consecutive 16-byte chunks
                    cp_async16(dst + a * ROW + pad32(t), L.u + src[a] + t);
                }
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
#pragma unroll
        for (int h = 0; h < C / 4; ++h) rv[h] = __ldg(reinterpret_cast<const float4 *>(L.r + base + i0 + 4 * h));
    };
    // shared-memory offset of the float4 holding sites i0 + h .. i0 + h + 3 of a row
    auto slot = [&](int h) {
        if constexpr (TMA) {
            // 16-byte chunk c = (i0 + h) / 4 lies in 128-byte row c / 8 at chunk c % 8, which
            // the 128-byte swizzle stores at chunk (c % 8) ^ (row % 8)
            const int c = (i0 + h) >> 2, r = c >> 3;
            return r * 32 + (((c & 7) ^ (r & 7)) << 2);
        } else {
            return pad32(i0 + h);
        }
    };
    float macc = 0.f;   // mean stage: this lane's weighted sum of the new values
    if (first < A.nlines) {
    float4 rc[C / 4], rn[C / 4];
    issue(first, buf, rc);
    for (long long line = first; line < A.nlines; line += nwarps) {
        if constexpr (TMA) {
            const bool ok = mbar_wait(bar, parity, deadline);
            if (!__all_sync(FULL, ok)) {
                if (lane == 0) A.ctlw->status = TDGL_ERR_TIMEOUT;
                break;
            }
            parity ^= 1u;
            issued = false;
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncwarp();
        const float *cur = buf;
        float e[C];
#pragma unroll
        for (int h = 0; h < C; h += 4) {
            const int t = slot(h);
            const float4 a = rc[h / 4];
            const float4 yp = *reinterpret_cast<const float4 *>(cur + t);
            const float4 ym = *reinterpret_cast<const float4 *>(cur + ROW + t);
            const float4 kp = *reinterpret_cast<const float4 *>(cur + 2 * ROW + t);
            const float4 km = *reinterpret_cast<const float4 *>(cur + 3 * ROW + t);
            const float av[4] = {a.x, a.y, a.z, a.w}, ypv[4] = {yp.x, yp.y, yp.z, yp.w},
                        ymv[4] = {ym.x, ym.y, ym.z, ym.w}, kpv[4] = {kp.x, kp.y, kp.z, kp.w},
                        kmv[4] = {km.x, km.y, km.z, km.w};
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float x = -(av[c] - fsub);
                if (ya) x += L.cy * (ypv[c] + ymv[c]);
                if (za) x += L.cz * (kpv[c] + kmv[c]);
                e[h + c] = x;
            }
        }
        __syncwarp();   // every lane has read the buffer: it takes the next line
        if (line + nwarps < A.nlines) issue(line + nwarps, buf, rn);
        const bool open = (A.bcx == kOpen);
        const float rho = L.rho;
        float wv[C];
        float z = 0.f;
        float out[C];
        if constexpr (W == 0) {
            // exact: each lane runs its recursions from zero over its chunk; the values
            // entering a chunk follow from a scan over the lanes (carry c_L = rho^C c_(L-1)
            // + end_(L-1)), seeded at the line's ends in closed form
            // w(-1) over the extended line: open, sum_x (rho^(x-1) [x >= 1] + rho^(2N-3-x)
            // [x <= N-2]) e(x) / (1 - rho^(2N-2)); periodic, sum_x rho^(N-1-x) e(x) / (1 - rho^N)
            float ps = 0.f;
            {
                float p1 = pw_f1, p2 = pw_f2;   // at m = 0 and m = C - 1
#pragma unroll
                for (int m = 0; m < C; ++m) {
                    const float t1 = (open && !(lane == 0 && m == 0)) ? p1 : 0.f;
                    ps = fmaf(t1, e[m], ps);
                    p1 *= rho;
                }
#pragma unroll
                for (int m = C - 1; m >= 0; --m) {
                    const float t2 = (open && lane == 31 && m == C - 1) ? 0.f : p2;
                    ps = fmaf(t2, e[m], ps);
                    p2 *= rho;
                }
            }
            float w = 0.f;
#pragma unroll
            for (int m = 0; m < C; ++m) {
                w = fmaf(rho, w, e[m]);
                wv[m] = w;
            }
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) ps += __shfl_xor_sync(FULL, ps, o);
            const float wm1 = ps * L.gf;
            // forward carries: S_L = sum_(l <= L) rho^(C(L-l)) end_l + rho^(C(L+1)) w(-1)
            float S = w;
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                const float t = __shfl_up_sync(FULL, S, 1 << q);
                if (lane >= (1 << q)) S = fmaf(L.rhoC[q], t, S);
            }
            S = fmaf(pw_c1, wm1, S);
            float cin = __shfl_up_sync(FULL, S, 1);
            if (lane == 0) cin = wm1;
            {
                float p = rho;
#pragma unroll
                for (int m = 0; m < C; ++m) {
                    wv[m] = fmaf(p, cin, wv[m]);
                    p *= rho;
                }
            }
            // backward, from zero over the chunk
#pragma unroll
            for (int m = C - 1; m >= 0; --m) {
                z = fmaf(rho, z, wv[m]);
                out[m] = z;
            }
            // z(N): open, by the mirror symmetry of the solution z(N) = z(N-2), hence
            // z(N) = (rho w(N-1) + w(N-2)) / (1 - rho^2); periodic, z(N) = z(0) =
            // sum_x rho^x w(x) / (1 - rho^N)
            float zN;
            if (open) {
                zN = __shfl_sync(FULL, fmaf(rho, wv[C - 1], wv[C - 2]) * L.gb, 31);
            } else {
                float pz = 0.f, p = pw_b;
#pragma unroll
                for (int m = 0; m < C; ++m) {
                    pz = fmaf(p, wv[m], pz);
                    p *= rho;
                }
#pragma unroll
                for (int o = 16; o >= 1; o >>= 1) pz += __shfl_xor_sync(FULL, pz, o);
                zN = pz * L.gf;
            }
            // backward carries: T_L = sum_(l >= L) rho^(C(l-L)) start_l + rho^(C(32-L)) z(N)
            float T = z;
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                const float t = __shfl_down_sync(FULL, T, 1 << q);
                if (lane + (1 << q) < 32) T = fmaf(L.rhoC[q], t, T);
            }
            T = fmaf(pw_c2, zN, T);
            float din = __shfl_down_sync(FULL, T, 1);
            if (lane == 31) din = zN;
            {
                float p = rho;
#pragma unroll
                for (int m = C - 1; m >= 0; --m) {
                    out[m] = fmaf(p, din, out[m]) * L.rscale;
                    p *= rho;
                }
            }
        } else if constexpr (W <= C) {
            const float e_next0 = __shfl_sync(FULL, e[0], 1);
            const float e_prevlast = __shfl_sync(FULL, e[C - 1], 30);
            // forward warm-up over x = i0 - W .. i0 - 1 (the previous lane's last W values);
            // on an open line lane 0 reads the mirror e_ext(-d) = e(d), d = W - m
            float w = 0.f;
#pragma unroll
            for (int m = 0; m < W; ++m) {
                float v = __shfl_sync(FULL, e[C - W + m], (lane + 31) & 31);
                if (open && lane == 0) v = (W - m == C) ? e_next0 : e[(W - m) % C];
                w = fmaf(rho, w, v);
            }
#pragma unroll
            for (int m = 0; m < C; ++m) {
                w = fmaf(rho, w, e[m]);
                wv[m] = w;
            }
            // right mirror: lane 31 continues the forward recursion over e(nx - 2 - m)
            float wext[W];
            {
                float wc = wv[C - 1];
#pragma unroll
                for (int m = 0; m < W; ++m) {
                    const float v = (m <= C - 2) ? e[(C - 2 - m + C) % C] : e_prevlast;
                    wc = fmaf(rho, wc, v);
                    wext[m] = wc;
                }
            }
            // backward warm-up over x = i0 + C + W - 1 down to i0 + C
#pragma unroll
            for (int m = W - 1; m >= 0; --m) {
                float v = __shfl_sync(FULL, wv[m], (lane + 1) & 31);
                if (open && lane == 31) v = wext[m];
                z = fmaf(rho, z, v);
            }
        }
        if constexpr (W != 0) {
#pragma unroll
            for (int m = C - 1; m >= 0; --m) {
                z = fmaf(rho, z, wv[m]);
                out[m] = z * L.rscale;
            }
        }
        int j, k;
        line_jk(line, A.color, L.ny, L.nz, j, k);
        float *dst = L.u + (long long)NX * j + plane * k + i0;
#pragma unroll
        for (int h = 0; h < C; h += 4)
            *reinterpret_cast<float4 *>(dst + h) = make_float4(out[h], out[h + 1], out[h + 2], out[h + 3]);
        if (A.mean_stage) {
            // trapezoid weights: 1/2 on each open face
            float ls = 0.f;
#pragma unroll
            for (int m = 0; m < C; ++m) {
                const bool face = open && ((lane == 0 && m == 0) || (lane == 31 && m == C - 1));
                const float4 r4 = rc[m / 4];
                const float rm = (m % 4 == 0) ? r4.x : (m % 4 == 1) ? r4.y : (m % 4 == 2) ? r4.z : r4.w;
                ls += (face ? 0.5f : 1.f) * (A.mean_dot ? rm * out[m] : out[m]);
            }
            float wyz = (A.bcy == kOpen && L.ny >= 2 && (j == 0 || j == L.ny - 1)) ? 0.5f : 1.f;
            if (A.bcz == kOpen && L.nz >= 2 && (k == 0 || k == L.nz - 1)) wyz *= 0.5f;
            macc += wyz * ls;
        }
#pragma unroll
        for (int h = 0; h < C / 4; ++h) rc[h] = rn[h];
    }
    }
    // a wait that ran out: the boxes in flight land before the buffer is given up
    if (TMA && issued) mbar_wait(bar, parity, deadline + wait_ns);
    if (!A.mean_stage) return;
    __shared__ double shd[32];
    __shared__ int flag;
    const double bs = block_sum((double)macc, shd);
    if (threadIdx.x == 0) A.blockred[(A.mean_stage == 2 ? kMeanOff : 0) + blockIdx.x] = bs;
    if (A.mean_stage != 2 || !last_block(&A.ctlw->ticket, gridDim.x, &flag)) return;
    double t = 0.0;
    for (int q = threadIdx.x; q < A.mean_nb1; q += blockDim.x) t += ((volatile double *)A.blockred)[q];
    for (int q = threadIdx.x; q < (int)gridDim.x; q += blockDim.x) t += ((volatile double *)A.blockred)[kMeanOff + q];
    t = block_sum(t, shd);
    if (threadIdx.x == 0) {
        A.ctlw->ticket = 0u;
        if (A.mean_dot) A.ctlw->sums[A.dot_slot] = t;
        else A.ctlw->mu_mean = t / A.wsum;
    }
}

bool mg_encode_line_maps(PoissonArgs &pa)
{
    bool any = false;
    for (int l = 0; l < kMaxLevels; ++l) pa.umap_u[l] = nullptr;
    const auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(tma_encode_entry());
    if (!encode) return false;
    for (int l = 0; l < pa.nlevels; ++l) {
        const MGLevel &L = pa.lev[l];
        if (L.iir != 16 || L.nx != 512 || (reinterpret_cast<uintptr_t>(L.u) & 15) != 0) continue;
        // u as rows of 32 floats (128 bytes); a box of 16 rows is one line
        const cuuint64_t dims[2] = {32, (cuuint64_t)(L.N / 32)};
        const cuuint64_t strides[1] = {128};
        const cuuint32_t box[2] = {32, 16};
        const cuuint32_t estr[2] = {1, 1};
        if (encode(&pa.umap[l], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, L.u, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS) {
            pa.umap_u[l] = L.u;
            any = true;
        }
    }
    return any;
}

// blocks of one recursive-smoother pass over nlines lines: a warp per line up to one
// resident wave (small levels are latency-bound, so every line gets its own warp)
static long long async_grid(long long nlines, int occ, int sms)
{
    long long nb = (nlines + kIirWarps - 1) / kIirWarps;
    const long long cap = (long long)occ * sms;
    return nb > cap ? cap : nb;
}

static cudaError_t smooth(const PoissonArgs &a, int l, int color, cudaStream_t s, long long *nl, int mean_stage = 0)
{
    const MGLevel &L = a.lev[l];
    LineArgs A;
    A.L = L;
    A.bcx = a.g.bcx;
    A.bcy = a.g.bcy;
    A.bcz = a.g.bcz;
    A.color = color;
    A.nlines = mg_lines_of_colour(L.ny, L.nz, color);
    A.ctl = a.ctl;
    A.level0 = (l == 0);
    A.mean_stage = 0;
    A.mean_nb1 = 0;
    A.mean_dot = a.mean_dot;
    A.dot_slot = a.dot_slot;
    A.ctlw = a.ctl;
    A.blockred = a.blockred;
    A.wsum = a.wsum;
    A.wait_ns = a.wait_ns;
    A.extra_tx = a.extra_tx;
    if (A.nlines == 0 && mean_stage == 0) return cudaSuccess;
    if (L.iir == 16) {
        // staged by the tensor memory accelerator where this level's map describes its u,
        // else by per-lane asynchronous copies; one resident wave of blocks (shared memory
        // and registers decide how many fit on an SM)
        const bool tma = a.umap_u[l] != nullptr && a.umap_u[l] == L.u;
        const size_t smem_cp = (size_t)kIirWarps * 4 * (512 + 64) * sizeof(float);
        const size_t smem_tma = (size_t)kIirWarps * kIirTmaBytes + 1024 + kIirWarps * sizeof(unsigned long long);
        const size_t smem = tma ? smem_tma : smem_cp;
        using KFn = void (*)(LineArgs, const CUtensorMap);
        static const KFn kfn[2][2] = {{line_iir_async_kernel<16, 12, false>, line_iir_async_kernel<16, 0, false>},
                                      {line_iir_async_kernel<16, 12, true>, line_iir_async_kernel<16, 0, true>}};
        static int sms = 0, occ[2][2];
        if (!sms) {
            int dev = 0;
            if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
                sms = 152;
            for (int t = 0; t < 2; ++t)
                for (int w = 0; w < 2; ++w) {
                    const size_t sz = t ? smem_tma : smem_cp;
                    cudaFuncSetAttribute(kfn[t][w], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sz);
                    // a failed query leaves one block per SM (and clears its error)
                    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[t][w], kfn[t][w], kIirWarps * 32, sz) !=
                        cudaSuccess) {
                        cudaGetLastError();
                        occ[t][w] = 1;
                    }
                    if (occ[t][w] < 1) occ[t][w] = 1;
                }
        }
        const int wi = (L.iir_w == 12) ? 0 : 1;
        const int occ_l = occ[tma ? 1 : 0][wi];
        long long nb = async_grid(A.nlines, occ_l, sms);
        if (mean_stage) {
            A.mean_stage = mean_stage;
            A.mean_nb1 = (int)async_grid(mg_lines_of_colour(L.ny, L.nz, 1), occ_l, sms);
            if (nb < 1) nb = 1;   // the reduction runs even without lines of this colour
        }
        kfn[tma ? 1 : 0][wi]<<<(int)nb, kIirWarps * 32, smem, s>>>(A, a.umap[tma ? l : 0]);
        ++*nl;
        return cudaGetLastError();
    }
    if (L.iir == 32) {
        const int nb = (int)((A.nlines + kThreads / 32 - 1) / (kThreads / 32));
        line_iir_kernel<32><<<nb, kThreads, 0, s>>>(A);
        ++*nl;
        return cudaGetLastError();
    }
    const LineShape sh = line_shape(L.nx, L.kmin, L.kmax, kThreads);
    A.sh = sh;
    const size_t smem = sizeof(float) * (size_t)line_tile_floats(sh);
    int nb = (int)((A.nlines + sh.lpb - 1) / sh.lpb);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(line_smooth_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr_set = true;
    }
    line_smooth_kernel<<<nb, kThreads, smem, s>>>(A);
    ++*nl;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Exact solve on the coarsest level: forward y-z transform, per-mode line
// convolution, inverse transform.  cw = [W (M x M) | V (M x M) | Gq (M x P)].
// ---------------------------------------------------------------------------
static void yz_basis(int n, int bc, double c, std::vector<double> &V, std::vector<double> &lam)
{
    const double pi = 3.14159265358979323846;
    V.assign((size_t)n * n, 0.0);
    lam.assign(n, 0.0);
    if (n == 1) {
        V[0] = 1.0;
        return;
    }
    if (bc == kOpen) {
        for (int k = 0; k < n; ++k) {
            for (int j = 0; j < n; ++j) V[(size_t)j * n + k] = cos(pi * k * j / (n - 1));
            double sn = sin(pi * k / (2.0 * (n - 1)));
            lam[k] = -4.0 * c * sn * sn;
        }
        return;
    }
    int col = 0;
    for (int j = 0; j < n; ++j) V[(size_t)j * n + col] = 1.0;
    lam[col++] = 0.0;
    for (int k = 1; 2 * k < n; ++k) {
        double sn = sin(pi * k / n);
        for (int j = 0; j < n; ++j) V[(size_t)j * n + col] = cos(2.0 * pi * k * j / n);
        lam[col++] = -4.0 * c * sn * sn;
        for (int j = 0; j < n; ++j) V[(size_t)j * n + col] = sin(2.0 * pi * k * j / n);
        lam[col++] = -4.0 * c * sn * sn;
    }
    if (n % 2 == 0) {
        for (int j = 0; j < n; ++j) V[(size_t)j * n + col] = (j % 2) ? -1.0 : 1.0;
        lam[col++] = -4.0 * c;
    }
}

static bool invert(int n, const std::vector<double> &A, std::vector<double> &Ainv)
{
    std::vector<double> a(A);
    Ainv.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) Ainv[(size_t)i * n + i] = 1.0;
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(a[(size_t)r * n + c]) > fabs(a[(size_t)p * n + c])) p = r;
        if (fabs(a[(size_t)p * n + c]) < 1e-300) return false;
        for (int k = 0; k < n; ++k) {
            std::swap(a[(size_t)c * n + k], a[(size_t)p * n + k]);
            std::swap(Ainv[(size_t)c * n + k], Ainv[(size_t)p * n + k]);
        }
        double d = 1.0 / a[(size_t)c * n + c];
        for (int k = 0; k < n; ++k) {
            a[(size_t)c * n + k] *= d;
            Ainv[(size_t)c * n + k] *= d;
        }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            double f = a[(size_t)r * n + c];
            if (f == 0.0) continue;
            for (int k = 0; k < n; ++k) {
                a[(size_t)r * n + k] -= f * a[(size_t)c * n + k];
                Ainv[(size_t)r * n + k] -= f * Ainv[(size_t)c * n + k];
            }
        }
    }
    return true;
}

size_t mg_coarse_floats(int nx, int bcx, int M) { return 2 * (size_t)M * M + (size_t)M * mg_period(nx, bcx); }

bool mg_coarse_factors(int nx, int bcx, double cx, int ny, int nz, int bcy, int bcz, double cy, double cz, float *cw)
{
    std::vector<double> Vy, Vz, ly, lz, Wy, Wz;
    yz_basis(ny, bcy, cy, Vy, ly);
    yz_basis(nz, bcz, cz, Vz, lz);
    if (!invert(ny, Vy, Wy) || !invert(nz, Vz, Wz)) return false;
    const int M = ny * nz, P = mg_period(nx, bcx);
    float *W = cw, *V = cw + (size_t)M * M, *Gq = cw + 2 * (size_t)M * M;
    // site s = j + ny k, mode q = p + ny r
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int r = 0; r < nz; ++r)
                for (int p = 0; p < ny; ++p) {
                    const int s = j + ny * k, q = p + ny * r;
                    V[(size_t)s * M + q] = (float)(Vy[(size_t)j * ny + p] * Vz[(size_t)k * nz + r]);
                    W[(size_t)q * M + s] = (float)(Wy[(size_t)p * ny + j] * Wz[(size_t)r * nz + k]);
                }
    std::vector<double> G;
    for (int r = 0; r < nz; ++r)
        for (int p = 0; p < ny; ++p) {
            const int q = p + ny * r;
            double sigma = -(ly[p] + lz[r]);
            if (sigma < 1e-12 * cx) sigma = 0.0;
            green(P, cx, sigma, G);
            for (int k = 0; k < P; ++k) Gq[(size_t)q * P + k] = (float)G[k];
        }
    return true;
}

struct CoarseArgs {
    MGLevel L;
    int bcx;
    const DevCtl *ctl;
    int level0;
};

// The two basis changes of the coarsest level as tiled products: Out[a][i] = sum_b
// Mat[a][b] In[b][i] over the M y-z modes.  Block (x-tile, a-tile) stages In[b][64 x-sites]
// and Mat[4 rows][b] in shared memory, kCB terms of the sum at a time; each thread sums
// one output in the order of coarse_fwd_at / coarse_inv_at (b ascending).
// FWD: Mat = W, In = -(r - fsub), Out = H in t.  Otherwise Mat = V, In = X, Out = u.
constexpr int kCT = 64, kCA = 4, kCB = 128;
template <bool FWD>
__global__ void __launch_bounds__(256) coarse_mat_kernel(CoarseArgs A, const float *X)
{
    __shared__ float In[kCB][kCT];
    __shared__ float Mt[kCA][kCB + 1];
    const MGLevel &L = A.L;
    const int nx = L.nx, M = L.M;
    const float fsub = (FWD && A.level0) ? (float)A.ctl->fmean : 0.f;
    const float *Mat = FWD ? L.cw : L.cw + (size_t)M * M;
    const float *src = FWD ? L.r : (X ? X : L.t);
    float *out = FWD ? L.t : L.u;
    const int i0 = blockIdx.x * kCT, a0 = blockIdx.y * kCA;
    const int ii = threadIdx.x % kCT, aa = threadIdx.x / kCT;   // row aa
    float acc0 = 0.f;
    for (int b0 = 0; b0 < M; b0 += kCB) {
        const int nb = min(kCB, M - b0);
        __syncthreads();
        for (int e = threadIdx.x; e < nb * kCT; e += 256) {
            const int b = e / kCT, x = e % kCT;
            float v = 0.f;
            if (i0 + x < nx) {
                v = src[(size_t)(b0 + b) * nx + i0 + x];
                if (FWD) v = -(v - fsub);
            }
            In[b][x] = v;
        }
        for (int e = threadIdx.x; e < kCA * nb; e += 256) {
            const int a = e / nb, b = e % nb;
            Mt[a][b] = (a0 + a < M) ? Mat[(size_t)(a0 + a) * M + b0 + b] : 0.f;
        }
        __syncthreads();
        for (int b = 0; b < nb; ++b) {
            const float v = In[b][ii];
            acc0 += Mt[aa][b] * v;
        }
    }
    if (i0 + ii < nx) {
        if (a0 + aa < M) out[(size_t)(a0 + aa) * nx + i0 + ii] = acc0;
    }
}

// X[q][i] = sum_k Gq[q][k] H~[q][i + k] over one period.  With X null, in place in t:
// one block owns a whole mode line, so it reads the line before writing it.  Otherwise
// block (c, q) writes the c-th of gridDim.x chunks of line q into X.
__global__ void __launch_bounds__(kThreads) coarse_conv_kernel(CoarseArgs A, float *X)
{
    extern __shared__ __align__(16) float sm[];
    const int nx = A.L.nx;
    const int chunk = ((nx + gridDim.x - 1) / gridDim.x + kCR - 1) / kCR * kCR;
    const int ib = blockIdx.x * chunk, ie = min(nx, ib + chunk);
    coarse_conv_line<false>(A.L, A.bcx, blockIdx.y, threadIdx.x, blockDim.x, sm, X, ib, X ? ie : -1);
}


static cudaError_t coarse_solve(const PoissonArgs &a, int l, cudaStream_t s, long long *nl)
{
    CoarseArgs C;
    C.L = a.lev[l];
    C.bcx = a.g.bcx;
    C.ctl = a.ctl;
    C.level0 = (l == 0);
    const long long n = (long long)C.L.M * C.L.nx;
    const dim3 mgrid((C.L.nx + kCT - 1) / kCT, (C.L.M + kCA - 1) / kCA);
    coarse_mat_kernel<true><<<mgrid, 256, 0, s>>>(C, nullptr);
    // below the finest level the shared scratch t (finest-level size) has room for X after
    // H, and each mode line is split over four blocks
    float *X = (l > 0 && 2 * n <= a.lev[0].N) ? C.L.t + n : nullptr;
    dim3 grid(X ? 4 : 1, C.L.M);
    size_t smem = sizeof(float) * (size_t)coarse_line_floats(C.L.nx, C.L.P);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(coarse_conv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr = true;
    }
    coarse_conv_kernel<<<grid, kThreads, smem, s>>>(C, X);
    coarse_mat_kernel<false><<<mgrid, 256, 0, s>>>(C, X);
    *nl += 3;
    return cudaGetLastError();
}

// skip_first: the finest level's first colour-0 pass is left out.  Right after a
// V-cycle (which ends with a colour-0 pass on the same right-hand side) it would repeat
// exact line solves on identical input: the same bits.
// mean_out (finest level only): the closing two passes also sum the weighted final mu
// into ctl->mu_mean (vcycle_mean_fusable says when the smoother there can)
static cudaError_t vcycle(const PoissonArgs &a, int l, cudaStream_t s, long long *nl, bool skip_first = false,
                          bool mean_out = false)
{
    const int bcx = a.g.bcx, bcy = a.g.bcy, bcz = a.g.bcz;
    if (l == a.nlevels - 1) {
        if (a.lev[l].cw) return coarse_solve(a, l, s, nl);
        // no exact factors (too many y-z modes): relax
        int n = 2 * (a.lev[l].ny + a.lev[l].nz) + 8;
        for (int it = 0; it < n; ++it) {
            smooth(a, l, 0, s, nl);
            smooth(a, l, 1, s, nl);
        }
        return cudaGetLastError();
    }
    if (!skip_first) smooth(a, l, 0, s, nl);
    smooth(a, l, 1, s, nl);
    const MGLevel &F = a.lev[l], &C = a.lev[l + 1];
    const bool v4 = (F.nx % 4) == 0;   // rows on 16-byte boundaries (x is never coarsened)
    // With a proper zebra colouring the post-smoothing starts with colour 1, whose lines are
    // solved from r and the colour-0 rows alone (their old values are never read): only
    // colour 0 takes the prolonged correction, with the same result bit for bit.  (After the
    // pre-smoothing the colour-1 rows' residual is zero in exact arithmetic, but in FP32 it
    // is rounding noise of the size of the colour-0 residual near convergence, so it is
    // still computed and restricted: zc = -1.)
    const bool proper = (bcy == kOpen || F.ny == 1 || (F.ny % 2) == 0) && (bcz == kOpen || F.nz == 1 || (F.nz % 2) == 0);
    const int zc = -1, oc = proper ? 0 : -1;
    // residual and restriction in one pass wherever the level is coarsened in y and z
    // (measured faster than the two kernels on every level of a 512x512x256 grid); a
    // thread marches over kRZ coarse planes, or over one where the level has too few
    // blocks to fill the GPU (short chains hide the latency of small levels better)
    if (v4 && F.fy == 2 && F.fz == 2 && zc < 0) {
        const long long cols = (long long)((F.nx / 4 + kGX - 1) / kGX) * C.ny;
        if (cols * C.nz >= 2048LL * kRZ) {
            const dim3 grid((F.nx / 4 + kGX - 1) / kGX, C.ny, (C.nz + kRZ - 1) / kRZ);
            residual_restrict4_kernel<kRZ><<<grid, kGX, 0, s>>>(F, C, bcx, bcy, bcz, a.ctl, l == 0);
        } else {
            const dim3 grid((F.nx / 4 + kGX - 1) / kGX, C.ny, C.nz);
            residual_restrict4_kernel<1><<<grid, kGX, 0, s>>>(F, C, bcx, bcy, bcz, a.ctl, l == 0);
        }
        *nl -= 1;
    } else if (v4) {
        residual4_kernel<<<grid_xyz4(F.nx, F.ny, F.nz), kGX, 0, s>>>(F, bcx, bcy, bcz, a.ctl, l == 0, zc);
        restrict4_kernel<<<grid_xyz4(C.nx, C.ny, C.nz), kGX, 0, s>>>(F, C, bcy, bcz, zc);
    } else {
        residual_kernel<<<grid_xyz(F.nx, F.ny, F.nz), kGX, 0, s>>>(F, bcx, bcy, bcz, a.ctl, l == 0, zc);
        restrict_kernel<<<grid_xyz(C.nx, C.ny, C.nz), kGX, 0, s>>>(F, C, bcy, bcz, zc);
    }
    *nl += 3;
    vcycle(a, l + 1, s, nl);
    if (v4) {
        const dim3 g4 = grid_xyz4(F.nx, F.ny, F.nz);
        if ((long long)g4.x * g4.y * g4.z >= 2048)
            prolong4_kernel<kGZ><<<g4, kGX, 0, s>>>(F, C, bcy, bcz, oc);
        else
            prolong4_kernel<1><<<dim3(g4.x, F.ny, F.nz), kGX, 0, s>>>(F, C, bcy, bcz, oc);
    }
    else prolong_kernel<<<grid_xyz(F.nx, F.ny, F.nz), kGX, 0, s>>>(F, C, bcy, bcz, oc);
    smooth(a, l, 1, s, nl, mean_out ? 1 : 0);
    smooth(a, l, 0, s, nl, mean_out ? 2 : 0);
    return cudaGetLastError();
}

bool vcycle_mean_fusable(const PoissonArgs &a) { return a.nlevels > 1 && a.lev[0].iir == 16; }

cudaError_t launch_vcycle(const PoissonArgs &a, cudaStream_t s, long long *launches, bool after_cycle, bool mean_out)
{
    // the zebra colouring (j + k) % 2 is a proper two-colouring of the lines unless a
    // periodic axis has odd length; only then is a repeated colour-0 pass not a no-op
    const MGLevel &F = a.lev[0];
    const bool proper = (a.g.bcy == kOpen || F.ny == 1 || (F.ny % 2) == 0) &&
                        (a.g.bcz == kOpen || F.nz == 1 || (F.nz % 2) == 0);
    return vcycle(a, 0, s, launches, after_cycle && proper && a.nlevels > 1, mean_out && vcycle_mean_fusable(a));
}

cudaError_t launch_poisson_residual(const PoissonArgs &a, cudaStream_t s)
{
    residual_norm_kernel<<<grid_xy(a.lev[0].nx, a.lev[0].ny), kGX, 0, s>>>(a.lev[0], a.g.bcx, a.g.bcy, a.g.bcz, a.ctl,
                                                                          a.blockred);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Zero mode of mu: subtract the weighted mean (FP64 sum).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kGX) mu_mean_kernel(DevGrid g, const float *mu, DevCtl *ctl, double *blockred,
                                                      double wsum, int to_fmean)
{
    const int i = blockIdx.x * kGX + threadIdx.x, j = blockIdx.y;
    float accf = 0.f;
    if (i < g.nx) {
        float wxy = 1.f;
        if (g.bcx == kOpen && (i == 0 || i == g.nx - 1)) wxy *= 0.5f;
        if (g.bcy == kOpen && (j == 0 || j == g.ny - 1)) wxy *= 0.5f;
        const long long pl = (long long)g.nx * g.ny;
        for (int k = 0; k < g.nz; ++k) {
            float w = wxy;
            if (g.bcz == kOpen && g.nz >= 2 && (k == 0 || k == g.nz - 1)) w *= 0.5f;
            accf += w * mu[i + (long long)g.nx * j + pl * k];
        }
    }
    __shared__ double shd[32];
    __shared__ int flag;
    const unsigned int bid = blockIdx.x + gridDim.x * blockIdx.y, nb = gridDim.x * gridDim.y;
    double s = block_sum((double)accf, shd);
    if (threadIdx.x == 0) blockred[bid] = s;
    if (!last_block(&ctl->ticket, nb, &flag)) return;
    double t = 0.0;
    for (unsigned int q = threadIdx.x; q < nb; q += blockDim.x) t += ((volatile double *)blockred)[q];
    t = block_sum(t, shd);
    if (threadIdx.x == 0) {
        ctl->ticket = 0u;
        (to_fmean ? ctl->fmean : ctl->mu_mean) = t / wsum;
    }
}

// mu -= mean, four sites per thread per pass, loads of a pass before its stores
// mu -= c with c the weighted mean (from_off: the pending mean mu_off[q] instead); thread 0
// clears mu_off[q] (zero_q >= 0), which no thread of this launch reads unless from_off
__global__ void mu_shift_kernel(long long N, float *mu, DevCtl *ctl, int zero_q, int from_off)
{
    const float c = (float)(from_off ? ctl->mu_off[zero_q] : ctl->mu_mean);
    if (!from_off && zero_q >= 0 && blockIdx.x == 0 && threadIdx.x == 0) ctl->mu_off[zero_q] = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long m0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; m0 < N; m0 += 4 * stride) {
        float v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (m0 + q * stride < N) v[q] = mu[m0 + q * stride];
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (m0 + q * stride < N) mu[m0 + q * stride] = v[q] - c;
    }
}

cudaError_t launch_project_mu(const PoissonArgs &a, cudaStream_t s, bool mean_done)
{
    if (!mean_done) mu_mean_kernel<<<grid_xy(a.g.nx, a.g.ny), kGX, 0, s>>>(a.g, a.mu, a.ctl, a.blockred, a.wsum, 0);
    mu_shift_kernel<<<grid_blocks(a.g.N, 8), kThreads, 0, s>>>(a.g.N, a.mu, a.ctl, a.mu_q, 0);
    return cudaGetLastError();
}

cudaError_t launch_f_mean(const PoissonArgs &a, cudaStream_t s)
{
    mu_mean_kernel<<<grid_xy(a.g.nx, a.g.ny), kGX, 0, s>>>(a.g, a.f, a.ctl, a.blockred, a.wsum, 1);
    return cudaGetLastError();
}

__global__ void commit_mean_kernel(DevCtl *ctl, int q) { ctl->mu_off[q] = ctl->mu_mean; }

cudaError_t launch_commit_mean(const PoissonArgs &a, cudaStream_t s)
{
    if (a.mu_q < 0) return cudaErrorInvalidValue;
    commit_mean_kernel<<<1, 1, 0, s>>>(a.ctl, a.mu_q);
    return cudaGetLastError();
}

cudaError_t launch_mu_materialize(long long N, float *mu, DevCtl *ctl, int q, cudaStream_t s)
{
    mu_shift_kernel<<<grid_blocks(N, 8), kThreads, 0, s>>>(N, mu, ctl, q, 1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaMemsetAsync(&ctl->mu_off[q], 0, sizeof(double), s);
}

// ---------------------------------------------------------------------------
// Voltage for open x: E_x = (<mu>_{i=0} - <mu>_{i=Nx-1}) / ((Nx-1) hx).
// ---------------------------------------------------------------------------
__global__ void voltage_kernel(DevGrid g, const float *mu, DevCtl *ctl, double *blockred, double hx)
{
    const long long nf = (long long)g.ny * g.nz;
    double acc = 0.0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nf; q += (long long)gridDim.x * blockDim.x)
        acc += (double)mu[q * g.nx] - (double)mu[q * g.nx + g.nx - 1];
    __shared__ double shd[32];
    __shared__ int flag;
    double s = block_sum(acc, shd);
    if (threadIdx.x == 0) blockred[blockIdx.x] = s;
    if (!last_block(&ctl->ticket, gridDim.x, &flag)) return;
    double t = 0.0;
    for (unsigned int q = threadIdx.x; q < gridDim.x; q += blockDim.x) t += ((volatile double *)blockred)[q];
    t = block_sum(t, shd);
    if (threadIdx.x == 0) {
        ctl->ticket = 0u;
        ctl->Ex = t / (double)nf / ((g.nx - 1) * hx);
    }
}

cudaError_t launch_voltage(const PoissonArgs &a, cudaStream_t s)
{
    long long nf = (long long)a.g.ny * a.g.nz;
    int nb = (int)((nf + kThreads - 1) / kThreads);
    if (nb > 256) nb = 256;
    voltage_kernel<<<nb, kThreads, 0, s>>>(a.g, a.mu, a.ctl, a.blockred, a.hx);
    return cudaGetLastError();
}

}  // namespace tdgl
