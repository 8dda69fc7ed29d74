// Implicit psi step: fused init (b, diag M) + first Jacobi sweep, and the
// Jacobi sweep with its residual (arXiv:1409.8340, Sec. 3.1: matrix M, Eq. b,
// Eq. final, Eq. convergence).
//
// Layout: psi, b, D are complex64 arrays, x fastest.  A block of 32 x 8 threads
// owns a 32 x 8 column of the xy plane and marches along z over KZ planes,
// keeping psi(k-1), psi(k), psi(k+1) in registers; x and y neighbours come
// from global memory through L1.  Every sweep also forms r = b - M psi for its
// input iterate and reduces max |r|^2 per block; the last block to finish
// reduces the block maxima and updates the device control block (sweep count,
// convergence flag, result buffer).  Sweeps launched after convergence exit at
// their first instruction, so the host can enqueue several sweeps ahead.
#include <float.h>
#include <string.h>

#include "tdgl_internal.cuh"

namespace tdgl {

constexpr int kBX = 32;
constexpr int kBY = 8;

static int zchunk(const DevGrid &g)
{
    long long bxy = (long long)((g.nx + kBX - 1) / kBX) * ((g.ny + kBY - 1) / kBY);
    long long kz = (bxy * g.nz) / 2432;
    if (kz < 1) kz = 1;
    if (kz > 32) kz = 32;
    return (int)kz;
}

int sweep_blocks(const DevGrid &g)
{
    int kz = zchunk(g);
    return ((g.nx + kBX - 1) / kBX) * ((g.ny + kBY - 1) / kBY) * ((g.nz + kz - 1) / kz);
}

__device__ __forceinline__ float2 wrap_phase(const DevGrid &g, int j, int k)
{
    return cmul(g.Py[j], g.Pz[k]);
}

// x and y parts of the neighbour sum NS_m (the off-diagonal part of the gauge
// Laplacian of Eq. LaplUV_yz, with the Neumann ghosts of Sec. 3.3.2 at open
// faces and the quasi-periodic wrap phase of Sec. 3.3.1 on the x wrap link).
template <bool GEN>
__device__ __forceinline__ float2 ns_xy(const DevGrid &g, const float2 *__restrict__ psi, int i, int j, int k,
                                        long long m, float2 Ux)
{
    float2 fwd = cmk(0.f, 0.f), bwd = cmk(0.f, 0.f);
    const bool lo = (i == 0), hi = (i == g.nx - 1);
    const bool per = (g.bcx == kPeriodic);
    if (!hi || per) {
        long long mp = hi ? m - (g.nx - 1) : m + 1;
        float2 U = GEN ? cmul(Ux, g.L[m]) : Ux;
        if (!GEN && hi) U = cmulc(wrap_phase(g, j, k), U);
        fwd = cmul(U, psi[mp]);
    }
    if (!lo || per) {
        long long mm = lo ? m + (g.nx - 1) : m - 1;
        float2 U = GEN ? cmul(Ux, g.L[mm]) : Ux;
        if (!GEN && lo) U = cmulc(wrap_phase(g, j, k), U);
        bwd = cmulc(U, psi[mm]);
    }
    float2 tx;
    if (per) tx = cadd(fwd, bwd);
    else tx = lo ? cscale(2.f, fwd) : (hi ? cscale(2.f, bwd) : cadd(fwd, bwd));

    const long long sy = g.nx;
    const bool ylo = (j == 0), yhi = (j == g.ny - 1);
    const bool yper = (g.bcy == kPeriodic);
    float2 fy = cmk(0.f, 0.f), by = cmk(0.f, 0.f);
    if (!yhi || yper) {
        long long mp = yhi ? m - (long long)(g.ny - 1) * sy : m + sy;
        float2 U = GEN ? g.L[g.N + m] : g.Uy[i];
        fy = cmul(U, psi[mp]);
    }
    if (!ylo || yper) {
        long long mm = ylo ? m + (long long)(g.ny - 1) * sy : m - sy;
        float2 U = GEN ? g.L[g.N + mm] : g.Uy[i];
        by = cmulc(U, psi[mm]);
    }
    float2 ty;
    if (yper) ty = cadd(fy, by);
    else ty = ylo ? cscale(2.f, fy) : (yhi ? cscale(2.f, by) : cadd(fy, by));
    return cadd(cscale(g.cx, tx), cscale(g.cy, ty));
}

// z part from register-held neighbours.
template <bool GEN>
__device__ __forceinline__ float2 ns_z(const DevGrid &g, int i, int k, long long m, float2 pzm, float2 pzp)
{
    if (g.nz < 2) return cmk(0.f, 0.f);
    const long long sz = (long long)g.nx * g.ny;
    const bool lo = (k == 0), hi = (k == g.nz - 1);
    const bool per = (g.bcz == kPeriodic);
    float2 Uf, Ub;
    if (GEN) {
        Uf = g.L[2 * g.N + m];
        long long mm = lo ? m + (long long)(g.nz - 1) * sz : m - sz;
        Ub = g.L[2 * g.N + mm];
    } else {
        Uf = g.Uz[i];
        Ub = Uf;
    }
    float2 fwd = cmul(Uf, pzp), bwd = cmulc(Ub, pzm);
    float2 t;
    if (per) t = cadd(fwd, bwd);
    else t = lo ? cscale(2.f, fwd) : (hi ? cscale(2.f, bwd) : cadd(fwd, bwd));
    return cscale(g.cz, t);
}

__device__ __forceinline__ void finish_sweep(const SweepArgs &a, float bmax, bool init)
{
    __shared__ float shf[32];
    __shared__ int flag;
    float m = block_max(bmax, shf);
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const unsigned int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const unsigned int nb = gridDim.x * gridDim.y * gridDim.z;
    if (tid == 0) a.blockred[bid] = (double)m;
    if (!last_block(&a.ctl->ticket, nb, &flag)) return;
    double g = 0.0;
    for (unsigned int q = tid; q < nb; q += blockDim.x * blockDim.y) {
        double v = ((volatile double *)a.blockred)[q];
        g = v > g ? v : g;
    }
    float gf = block_max((float)g, shf);
    if (tid == 0) {
        DevCtl *c = a.ctl;
        c->ticket = 0u;
        int it = init ? 1 : c->iter + 1;
        if (init) c->status = TDGL_OK;
        c->iter = it;
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
}

// Init (Sec. 3.1, Eq. b and diag M with psi_est = psi^-) fused with the first
// Jacobi sweep from psi^(0) = psi^-: both need the same neighbour sum of psi^-.
template <bool GEN>
__global__ void __launch_bounds__(kBX *kBY) init_sweep_kernel(SweepArgs a, int kz)
{
    const DevGrid &g = a.g;
    const int i = blockIdx.x * kBX + threadIdx.x;
    const int j = blockIdx.y * kBY + threadIdx.y;
    const int k0 = blockIdx.z * kz;
    const int k1 = min(k0 + kz, g.nz);
    const float2 Ux = a.ctl->Ux;
    float rmax = 0.f;
    if (i < g.nx && j < g.ny) {
        const long long sz = (long long)g.nx * g.ny;
        const long long base = (long long)i + (long long)g.nx * j;
        const bool zper = (g.bcz == kPeriodic);
        float2 pzm = cmk(0.f, 0.f);
        if (g.nz >= 2) {
            int kp = (k0 == 0) ? (zper ? g.nz - 1 : 1) : k0 - 1;
            pzm = a.src[base + kp * sz];
        }
        float2 pc = a.src[base + k0 * sz];
        for (int k = k0; k < k1; ++k) {
            const long long m = base + k * sz;
            float2 pzp = cmk(0.f, 0.f);
            if (g.nz >= 2) {
                int kn = (k == g.nz - 1) ? (zper ? 0 : g.nz - 2) : k + 1;
                pzp = a.src[base + kn * sz];
            }
            float2 ns = cadd(ns_xy<GEN>(g, a.src, i, j, k, m, Ux), ns_z<GEN>(g, i, k, m, pzm, pzp));
            const float a2 = cabs2(pc);
            const float mu = a.mu[m], al = a.alpha[m];
            const float2 D = cmk(1.f + g.ht2 * (g.beta * a2 + 2.f * g.S - al), g.ht2 * g.u * mu);
            // b = p + (ht/2)[(alpha - i u mu) p - beta|p|^2 p + NS - 2 S p]
            const float cr = al - g.beta * a2 - 2.f * g.S;
            const float ci = -g.u * mu;
            const float2 lin = cmk(cr * pc.x - ci * pc.y, cr * pc.y + ci * pc.x);
            const float2 b = cadd(pc, cscale(g.ht2, cadd(lin, ns)));
            // first sweep: s = b - sum_{m'!=m} M psi = b + (ht/2) NS
            const float2 s = cadd(b, cscale(g.ht2, ns));
            const float2 r = csub(s, cmul(D, pc));
            const float inv = 1.0f / cabs2(D);
            const float2 nxt = cscale(inv, cmulc(D, s));
            a.b[m] = b;
            a.D[m] = D;
            a.dst[m] = nxt;
            float r2 = cabs2(r);
            r2 = (r2 <= FLT_MAX) ? r2 : INFINITY;
            rmax = fmaxf(rmax, r2);
            pzm = pc;
            pc = pzp;
        }
    }
    finish_sweep(a, rmax, true);
}

template <bool GEN>
__global__ void __launch_bounds__(kBX *kBY) sweep_kernel(SweepArgs a, int kz)
{
    if (*(volatile int *)&a.ctl->done) return;
    const DevGrid &g = a.g;
    const int i = blockIdx.x * kBX + threadIdx.x;
    const int j = blockIdx.y * kBY + threadIdx.y;
    const int k0 = blockIdx.z * kz;
    const int k1 = min(k0 + kz, g.nz);
    const float2 Ux = a.ctl->Ux;
    float rmax = 0.f;
    if (i < g.nx && j < g.ny) {
        const long long sz = (long long)g.nx * g.ny;
        const long long base = (long long)i + (long long)g.nx * j;
        const bool zper = (g.bcz == kPeriodic);
        float2 pzm = cmk(0.f, 0.f);
        if (g.nz >= 2) {
            int kp = (k0 == 0) ? (zper ? g.nz - 1 : 1) : k0 - 1;
            pzm = a.src[base + kp * sz];
        }
        float2 pc = a.src[base + k0 * sz];
        for (int k = k0; k < k1; ++k) {
            const long long m = base + k * sz;
            float2 pzp = cmk(0.f, 0.f);
            if (g.nz >= 2) {
                int kn = (k == g.nz - 1) ? (zper ? 0 : g.nz - 2) : k + 1;
                pzp = a.src[base + kn * sz];
            }
            float2 ns = cadd(ns_xy<GEN>(g, a.src, i, j, k, m, Ux), ns_z<GEN>(g, i, k, m, pzm, pzp));
            const float2 D = a.D[m];
            const float2 s = cadd(a.b[m], cscale(g.ht2, ns));
            const float2 r = csub(s, cmul(D, pc));
            const float inv = 1.0f / cabs2(D);
            a.dst[m] = cscale(inv, cmulc(D, s));
            float r2 = cabs2(r);
            r2 = (r2 <= FLT_MAX) ? r2 : INFINITY;
            rmax = fmaxf(rmax, r2);
            pzm = pc;
            pc = pzp;
        }
    }
    finish_sweep(a, rmax, false);
}

// Right-hand side of the Poisson equation (Sec. 3.2): f_m = Im[conj(psi_m) NS_m(psi)],
// the lattice divergence of the supercurrent, with the open-x injection terms
// (Neumann ghosts mu_{-1} = mu_1 + 2 hx J, mu_Nx = mu_{Nx-2} - 2 hx J moved to the
// right-hand side).  Also reduces sum_m w_m f_m in FP64 for the compatibility
// projection (w: trapezoid weights).
template <bool GEN>
__global__ void __launch_bounds__(kBX *kBY) poisson_rhs_kernel(DevGrid g, DevCtl *ctl, double *blockred,
                                                               const float2 *__restrict__ psi, float *__restrict__ f,
                                                               float inj, double wsum, int kz)
{
    const int i = blockIdx.x * kBX + threadIdx.x;
    const int j = blockIdx.y * kBY + threadIdx.y;
    const int k0 = blockIdx.z * kz;
    const int k1 = min(k0 + kz, g.nz);
    const float2 Ux = ctl->Ux;
    float acc = 0.f;
    if (i < g.nx && j < g.ny) {
        const long long sz = (long long)g.nx * g.ny;
        const long long base = (long long)i + (long long)g.nx * j;
        const bool zper = (g.bcz == kPeriodic);
        float wxy = 1.f;
        if (g.bcx == kOpen && (i == 0 || i == g.nx - 1)) wxy *= 0.5f;
        if (g.bcy == kOpen && (j == 0 || j == g.ny - 1)) wxy *= 0.5f;
        float2 pzm = cmk(0.f, 0.f);
        if (g.nz >= 2) {
            int kp = (k0 == 0) ? (zper ? g.nz - 1 : 1) : k0 - 1;
            pzm = psi[base + kp * sz];
        }
        float2 pc = psi[base + k0 * sz];
        for (int k = k0; k < k1; ++k) {
            const long long m = base + k * sz;
            float2 pzp = cmk(0.f, 0.f);
            if (g.nz >= 2) {
                int kn = (k == g.nz - 1) ? (zper ? 0 : g.nz - 2) : k + 1;
                pzp = psi[base + kn * sz];
            }
            float2 ns = cadd(ns_xy<GEN>(g, psi, i, j, k, m, Ux), ns_z<GEN>(g, i, k, m, pzm, pzp));
            float v = pc.x * ns.y - pc.y * ns.x;
            if (g.bcx == kOpen) {
                if (i == 0) v -= inj;
                if (i == g.nx - 1) v += inj;
            }
            f[m] = v;
            float w = wxy;
            if (g.bcz == kOpen && g.nz >= 2 && (k == 0 || k == g.nz - 1)) w *= 0.5f;
            acc += w * v;
            pzm = pc;
            pc = pzp;
        }
    }
    __shared__ double shd[32];
    __shared__ int flag;
    double s = block_sum((double)acc, shd);
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const unsigned int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const unsigned int nb = gridDim.x * gridDim.y * gridDim.z;
    if (tid == 0) blockred[bid] = s;
    if (!last_block(&ctl->ticket, nb, &flag)) return;
    double t = 0.0;
    for (unsigned int q = tid; q < nb; q += blockDim.x * blockDim.y) t += ((volatile double *)blockred)[q];
    t = block_sum(t, shd);
    if (tid == 0) {
        ctl->ticket = 0u;
        ctl->fmean = t / wsum;
    }
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

// Block FP64 sum of w f, finished by the last block into ctl->fmean.
__device__ __forceinline__ void finish_rhs_sum(DevCtl *ctl, double *blockred, double v, double wsum)
{
    __shared__ double shd[32];
    __shared__ int flag;
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const unsigned int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const unsigned int nb = gridDim.x * gridDim.y * gridDim.z;
    double s = block_sum(v, shd);
    if (tid == 0) blockred[bid] = s;
    if (!last_block(&ctl->ticket, nb, &flag)) return;
    double t = 0.0;
    for (unsigned int q = tid; q < nb; q += blockDim.x * blockDim.y) t += ((volatile double *)blockred)[q];
    t = block_sum(t, shd);
    if (tid == 0) {
        ctl->ticket = 0u;
        ctl->fmean = t / wsum;
    }
}

// MODE 0: Jacobi sweep; 1: init + first sweep; 2: Poisson right-hand side
template <int MODE>
__global__ void __launch_bounds__(kBX *kBY) sweep2_kernel(SweepArgs a, int kz)
{
    constexpr bool INIT = (MODE == 1);
    constexpr bool RHS = (MODE == 2);
    constexpr bool ADJ = (MODE == 3);   // adjoint solve M^H lam = g: conj(D), transposed open-face rows
    if ((MODE == 0 || ADJ) && *(volatile int *)&a.ctl->done) return;
    const DevGrid &g = a.g;
    const int tx = threadIdx.x;
    const int x = (blockIdx.x * kBX + tx) * 2;
    const int j = blockIdx.y * kBY + threadIdx.y;
    const int k0 = blockIdx.z * kz;
    const int k1 = min(k0 + kz, g.nz);
    const bool in = (x < g.nx) && (j < g.ny);
    const float2 Ux = a.ctl->Ux;
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
    if (in) {
        const float4 uy = reinterpret_cast<const float4 *>(g.Uy)[x >> 1];
        const float4 uz = reinterpret_cast<const float4 *>(g.Uz)[x >> 1];
        const float sy = g.ht2 * g.cy, szc = g.ht2 * g.cz;
        yf0 = cscale(sy, lo2(uy));
        yf1 = cscale(sy, hi2(uy));
        zf0 = cscale(szc, lo2(uz));
        zf1 = cscale(szc, hi2(uz));
    }
    // x: site x has forward neighbour c1 and backward xl; site x+1 has forward xr and backward c0.
    // Backward coefficients are the conjugates of the forward ones.
    const float2 xf = cscale(g.ht2 * g.cx, Ux);
    const float inv_ht2 = 1.0f / g.ht2;

    auto knext = [&](int k) { return (k == g.nz - 1) ? (zper ? 0 : g.nz - 2) : k + 1; };
    float4 pzm = make_float4(0.f, 0.f, 0.f, 0.f), pc = pzm, pzp_n = pzm, b_n = pzm, D_n = pzm;
    float2 mu_n = cmk(0.f, 0.f), al_n = mu_n;
    if (in) {
        if (zact) pzm = src[q0 + plq * ((k0 == 0) ? (zper ? g.nz - 1 : 1) : k0 - 1)];
        pc = src[q0 + plq * k0];
        if (zact) pzp_n = src[q0 + plq * knext(k0)];
        if (INIT) {
            mu_n = mu2[(q0 + plq * k0)];
            al_n = al2[(q0 + plq * k0)];
        } else if (!RHS) {
            b_n = bq[q0 + plq * k0];
            D_n = Dq[q0 + plq * k0];
        }
    }
    float rmax = 0.f;
    float facc = 0.f;   // RHS: sum of w f over this thread's sites
    float wxy0 = 1.f, wxy1 = 1.f;
    if (RHS) {
        const float wy = (g.bcy == kOpen && (j == 0 || j == g.ny - 1)) ? 0.5f : 1.f;
        wxy0 = wy * ((g.bcx == kOpen && x == 0) ? 0.5f : 1.f);
        wxy1 = wy * ((g.bcx == kOpen && x + 1 == g.nx - 1) ? 0.5f : 1.f);
    }
    for (int k = k0; k < k1; ++k) {
        const float4 pzp = pzp_n;
        const float4 bc = b_n, Dc = D_n;
        const float2 muc = mu_n, alc = al_n;
        const long long q = q0 + plq * k;
        float4 yf = make_float4(0.f, 0.f, 0.f, 0.f), yb = yf;
        float2 xl = cmk(0.f, 0.f), xr = xl;
        if (in) {
            if (k + 1 < k1) {
                if (zact) pzp_n = src[q0 + plq * knext(k + 1)];
                if (INIT) {
                    mu_n = mu2[q + plq];
                    al_n = al2[q + plq];
                } else if (!RHS) {
                    b_n = bq[q + plq];
                    D_n = Dq[q + plq];
                }
            }
            yf = src[(x >> 1) + rowq * jp + plq * k];
            yb = src[(x >> 1) + rowq * jm + plq * k];
        }
        // x neighbours: left of x from lane tx-1, right of x+1 from lane tx+1
        const float2 from_left = make_float2(__shfl_up_sync(0xffffffffu, pc.z, 1), __shfl_up_sync(0xffffffffu, pc.w, 1));
        const float2 from_right =
            make_float2(__shfl_down_sync(0xffffffffu, pc.x, 1), __shfl_down_sync(0xffffffffu, pc.y, 1));
        const long long m = (long long)x + (long long)g.nx * jc + sz * k;   // site index of x
        if (in) {
            if (tx > 0) xl = from_left;
            else if (!xlo) xl = src2[m - 1];
            else if (xper) xl = src2[m + g.nx - 1];
            if (!xhi && tx < kBX - 1) xr = from_right;
            else if (!xhi) xr = src2[m + 2];
            else if (xper) xr = src2[m + 2 - g.nx];
        }
        if (in) {
            const float2 c0 = lo2(pc), c1 = hi2(pc);
            // x neighbours with the boundary rules: open faces double the inner
            // neighbour; the periodic wrap link (i = nx-1 -> 0) carries conj(P_jk).
            float2 xl0 = xl, xr1 = xr, c1x = c1, c0x = c0;
            if (xlo || xhi) {
                if (xper) {
                    const float2 P = cmul(g.Py[jc], g.Pz[k]);
                    if (xlo) xl0 = cmul(P, xl);      // conj(Ux conj(P)) xl = conj(Ux) (P xl)
                    if (xhi) xr1 = cmulc(P, xr);     // Ux conj(P) xr = Ux (conj(P) xr)
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
            if (yedge) {
                yf_0 = cscale(wy_f, yf_0);
                yf_1 = cscale(wy_f, yf_1);
                yb_0 = cscale(wy_b, yb_0);
                yb_1 = cscale(wy_b, yb_1);
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
                const float4 zpp = (wz_f == 1.f) ? pzp : make_float4(wz_f * pzp.x, wz_f * pzp.y, wz_f * pzp.z, wz_f * pzp.w);
                const float4 zmm = (wz_b == 1.f) ? pzm : make_float4(wz_b * pzm.x, wz_b * pzm.y, wz_b * pzm.z, wz_b * pzm.w);
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
                    if (xlo) f0 -= a.inj;
                    if (xhi) f1 += a.inj;
                }
                reinterpret_cast<float2 *>(a.f)[q] = make_float2(f0, f1);
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
                float2 bo[2], Do[2];
#pragma unroll
                for (int s2 = 0; s2 < 2; ++s2) {
                    const float a2 = cabs2(cs[s2]);
                    Do[s2] = cmk(1.f + g.ht2 * (g.beta * a2 + 2.f * g.S - als[s2]), g.ht2 * g.u * mus[s2]);
                    const float cr = als[s2] - g.beta * a2 - 2.f * g.S;
                    const float ci = -g.u * mus[s2];
                    const float2 lin = cmk(cr * cs[s2].x - ci * cs[s2].y, cr * cs[s2].y + ci * cs[s2].x);
                    bo[s2] = cadd(cadd(cs[s2], cscale(g.ht2, lin)), nss[s2]);   // nss = (ht/2) NS
                }
                b0 = bo[0];
                b1 = bo[1];
                D0 = Do[0];
                D1 = Do[1];
                bout[q] = make_float4(b0.x, b0.y, b1.x, b1.y);
                Dout[q] = make_float4(D0.x, D0.y, D1.x, D1.y);
            } else {
                b0 = lo2(bc);
                b1 = hi2(bc);
                D0 = ADJ ? cconj(lo2(Dc)) : lo2(Dc);
                D1 = ADJ ? cconj(hi2(Dc)) : hi2(Dc);
            }
            const float2 s0 = cadd(b0, ns0), s1 = cadd(b1, ns1);
            const float2 r0 = csub(s0, cmul(D0, c0)), r1 = csub(s1, cmul(D1, c1));
            const float2 n0 = cscale(1.0f / cabs2(D0), cmulc(D0, s0));
            const float2 n1 = cscale(1.0f / cabs2(D1), cmulc(D1, s1));
            dst[q] = make_float4(n0.x, n0.y, n1.x, n1.y);
            float r2a = cabs2(r0), r2b = cabs2(r1);
            r2a = (r2a <= FLT_MAX) ? r2a : INFINITY;
            r2b = (r2b <= FLT_MAX) ? r2b : INFINITY;
            rmax = fmaxf(rmax, fmaxf(r2a, r2b));
        }
        pzm = pc;
        pc = pzp;
    }
    if (RHS) {
        finish_rhs_sum(a.ctl, a.blockred, (double)facc, a.wsum);
        return;
    }
    finish_sweep(a, rmax, INIT);
}

static dim3 sweep_grid(const DevGrid &g, int kz)
{
    return dim3((g.nx + kBX - 1) / kBX, (g.ny + kBY - 1) / kBY, (g.nz + kz - 1) / kz);
}

static dim3 sweep2_grid(const DevGrid &g, int kz)
{
    return dim3((g.nx + kPX - 1) / kPX, (g.ny + kBY - 1) / kBY, (g.nz + kz - 1) / kz);
}

static bool use_sweep2(const DevGrid &g) { return g.L == nullptr && (g.nx % 2) == 0; }

cudaError_t launch_init_sweep(const SweepArgs &a, cudaStream_t s)
{
    int kz = zchunk(a.g);
    dim3 block(kBX, kBY);
    if (use_sweep2(a.g)) sweep2_kernel<1><<<sweep2_grid(a.g, kz), block, 0, s>>>(a, kz);
    else if (a.g.L) init_sweep_kernel<true><<<sweep_grid(a.g, kz), block, 0, s>>>(a, kz);
    else init_sweep_kernel<false><<<sweep_grid(a.g, kz), block, 0, s>>>(a, kz);
    return cudaGetLastError();
}

cudaError_t launch_sweep(const SweepArgs &a, cudaStream_t s)
{
    int kz = zchunk(a.g);
    dim3 block(kBX, kBY);
    if (use_sweep2(a.g)) sweep2_kernel<0><<<sweep2_grid(a.g, kz), block, 0, s>>>(a, kz);
    else if (a.g.L) sweep_kernel<true><<<sweep_grid(a.g, kz), block, 0, s>>>(a, kz);
    else sweep_kernel<false><<<sweep_grid(a.g, kz), block, 0, s>>>(a, kz);
    return cudaGetLastError();
}

cudaError_t launch_poisson_rhs(const PoissonArgs &a, const float2 *psi, cudaStream_t s)
{
    int kz = zchunk(a.g);
    dim3 grid = sweep_grid(a.g, kz), block(kBX, kBY);
    float inj = a.inject ? (float)(2.0 * a.Jext / a.hx) : 0.f;
    if (use_sweep2(a.g)) {
        SweepArgs sa;
        memset(&sa, 0, sizeof(sa));
        sa.g = a.g;
        sa.ctl = a.ctl;
        sa.blockred = a.blockred;
        sa.src = psi;
        sa.f = a.f;
        sa.inj = inj;
        sa.wsum = a.wsum;
        sweep2_kernel<2><<<sweep2_grid(a.g, kz), block, 0, s>>>(sa, kz);
    } else if (a.g.L) poisson_rhs_kernel<true><<<grid, block, 0, s>>>(a.g, a.ctl, a.blockred, psi, a.f, inj, a.wsum, kz);
    else poisson_rhs_kernel<false><<<grid, block, 0, s>>>(a.g, a.ctl, a.blockred, psi, a.f, inj, a.wsum, kz);
    return cudaGetLastError();
}

}  // namespace tdgl

namespace tdgl {

// Adjoint Jacobi sweep for M^H lam = g (b = g, D = diag M of the forward step).
cudaError_t launch_adj_sweep(const SweepArgs &a, cudaStream_t s)
{
    if (!use_sweep2(a.g)) return cudaErrorInvalidValue;
    int kz = zchunk(a.g);
    dim3 block(kBX, kBY);
    sweep2_kernel<3><<<sweep2_grid(a.g, kz), block, 0, s>>>(a, kz);
    return cudaGetLastError();
}

bool adj_supported(const DevGrid &g) { return use_sweep2(g); }

}  // namespace tdgl
