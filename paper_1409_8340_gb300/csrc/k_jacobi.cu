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

#include "philox.cuh"
#include "staged_tile.cuh"
#include "sweep_tile.cuh"

namespace tdgl {

__device__ __forceinline__ unsigned int grid_bid() { return blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z); }
__device__ __forceinline__ unsigned int grid_nb() { return gridDim.x * gridDim.y * gridDim.z; }

__device__ __forceinline__ void finish_sweep(const SweepArgs &a, float bmax, bool init)
{
    finish_sweep_at(a, bmax, init, grid_bid(), grid_nb());
}

static int zchunk(const DevGrid &g)
{
    long long bxy = (long long)((g.nx + kBX - 1) / kBX) * ((g.ny + kBY - 1) / kBY);
    long long kz = (bxy * (zhi(g) - zlo(g))) / 2432;
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


// Init (Sec. 3.1, Eq. b and diag M with psi_est = psi^-) fused with the first
// Jacobi sweep from psi^(0) = psi^-: both need the same neighbour sum of psi^-.
template <bool GEN>
__global__ void __launch_bounds__(kBX *kBY) init_sweep_kernel(SweepArgs a, int kz)
{
    const unsigned long long nstep = a.ctl->nstep;
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
            const float mu = a.mu[m] - (a.mu_off ? (float)*a.mu_off : 0.f), al = a.alpha[m];
            const float2 D = cmk(1.f + g.ht2 * (g.beta * a2 + 2.f * g.S - al), g.ht2 * g.u * mu);
            // b = p + (ht/2)[(alpha - i u mu) p - beta|p|^2 p + NS - 2 S p]
            const float cr = al - g.beta * a2 - 2.f * g.S;
            const float ci = -g.u * mu;
            const float2 lin = cmk(cr * pc.x - ci * pc.y, cr * pc.y + ci * pc.x);
            float2 b = cadd(pc, cscale(g.ht2, cadd(lin, ns)));
            if (a.noise_amp != 0.f) {
                // thermal noise h_t zeta_m (Sec. 3.1.2)
                const float2 v = noise_uv(a.noise_seed, m, nstep);
                b = cmk(b.x + a.noise_amp * v.x, b.y + a.noise_amp * v.y);
            }
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
    if (sweep_already_decided(a)) return;
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


template <int MODE, bool XZ = false, bool MASK = false>
__global__ void __launch_bounds__(kBX *kBY, 4) sweep2_kernel(SweepArgs a, int kz)
{
    // MODE 5: a plain sweep that recomputes a known result (no test, no early exit)
    if ((MODE == 0 || MODE == 3) && sweep_already_decided(a)) return;
    float rmax = 0.f, facc = 0.f;
    sweep2_body<MODE, false, XZ, MASK>(a, kz, blockIdx.x, blockIdx.y, blockIdx.z, rmax, facc);
    if (MODE == 2) {
        finish_rhs_sum_at(a.ctl, a.blockred, (double)facc, a.wsum, grid_bid(), grid_nb());
        return;
    }
    if (MODE == 5) return;
    finish_sweep(a, rmax, MODE == 1);
}

static dim3 sweep_grid(const DevGrid &g, int kz)
{
    return dim3((g.nx + kBX - 1) / kBX, (g.ny + kBY - 1) / kBY, (g.nz + kz - 1) / kz);
}

static dim3 sweep2_grid(const DevGrid &g, int kz)
{
    return dim3((g.nx + kPX - 1) / kPX, (g.ny + kBY - 1) / kBY, (zhi(g) - zlo(g) + kz - 1) / kz);
}

// the two-site tiled kernels: Landau links of either plane (tables), even nx
static bool use_sweep2(const DevGrid &g) { return (g.L == nullptr || g.Xj != nullptr) && (g.nx % 2) == 0; }

// the tiled kernel of MODE for the grid's gauge plane and link bits
template <int MODE>
static void launch_sweep2(const SweepArgs &a, int kz, cudaStream_t s)
{
    const dim3 grid = sweep2_grid(a.g, kz), block(kBX, kBY);
    const bool xz = a.g.Xj != nullptr, mk = a.g.lk != nullptr;
    if (xz && mk) sweep2_kernel<MODE, true, true><<<grid, block, 0, s>>>(a, kz);
    else if (xz) sweep2_kernel<MODE, true, false><<<grid, block, 0, s>>>(a, kz);
    else if (mk) sweep2_kernel<MODE, false, true><<<grid, block, 0, s>>>(a, kz);
    else sweep2_kernel<MODE, false, false><<<grid, block, 0, s>>>(a, kz);
}

// P = a (S - offS) + b (P - offP), four sites per thread where the arrays allow 16-byte access
__global__ void mu_guess_kernel(long long N, const float *__restrict__ S, float *__restrict__ P, float ca, float cb,
                                const double *offS, const double *offP)
{
    const float os = offS ? (float)*offS : 0.f, op = offP ? (float)*offP : 0.f;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long n4 = N >> 2;
    const float4 *S4 = reinterpret_cast<const float4 *>(S);
    float4 *P4 = reinterpret_cast<float4 *>(P);
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n4; q += stride) {
        const float4 sv = S4[q], pv = P4[q];
        P4[q] = make_float4(ca * (sv.x - os) + cb * (pv.x - op), ca * (sv.y - os) + cb * (pv.y - op),
                            ca * (sv.z - os) + cb * (pv.z - op), ca * (sv.w - os) + cb * (pv.w - op));
    }
    for (long long m = 4 * n4 + blockIdx.x * (long long)blockDim.x + threadIdx.x; m < N; m += stride)
        P[m] = ca * (S[m] - os) + cb * (P[m] - op);
}

cudaError_t launch_mu_guess(long long N, const float *S, float *P, float a, float b, const double *offS,
                            const double *offP, cudaStream_t s)
{
    long long nb = ((N >> 2) + 255) / 256;
    if (nb < 1) nb = 1;
    if (nb > 4096) nb = 4096;
    mu_guess_kernel<<<(int)nb, 256, 0, s>>>(N, S, P, a, b, offS, offP);
    return cudaGetLastError();
}

// Init + first sweep with the tile staged in shared memory (b, diag M, the first sweep and
// the Poisson guess; yz links, no insulating sites, nx % 4 == 0): the same per-site
// arithmetic as sweep2_kernel<1>, planes of psi and rows of mu, alpha and the previous-but-one
// mu copied ahead through a ring of plane stages.
constexpr size_t kInitRingBytes = kRing * sizeof(IStage);
__global__ void __launch_bounds__(kBX *kBY, 3) init_staged_kernel(SweepArgs a, int kz)
{
    extern __shared__ __align__(16) float init_ring[];
    float rmax = 0.f, facc = 0.f;
    sweep_staged_tile<1>(a, kz, blockIdx.x, blockIdx.y, blockIdx.z, rmax, facc,
                         reinterpret_cast<IStage *>(init_ring));
    finish_sweep(a, rmax, true);
}

bool init_staged_supported(const DevGrid &g)
{
    return use_sweep2(g) && g.Xj == nullptr && g.lk == nullptr && (g.nx & 3) == 0;
}

cudaError_t init_staged_setup()
{
    static const cudaError_t e =
        cudaFuncSetAttribute(init_staged_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kInitRingBytes);
    return e;
}

cudaError_t launch_init_sweep(const SweepArgs &a, cudaStream_t s, bool staged)
{
    int kz = zchunk(a.g);
    dim3 block(kBX, kBY);
    if (staged && init_staged_supported(a.g)) {
        const cudaError_t e = init_staged_setup();
        if (e != cudaSuccess) return e;
        init_staged_kernel<<<sweep2_grid(a.g, kz), block, kInitRingBytes, s>>>(a, kz);
        return cudaGetLastError();
    }
    if (use_sweep2(a.g)) {
        launch_sweep2<1>(a, kz, s);   // forms the Poisson guess too
        return cudaGetLastError();
    }
    if (a.g.L) init_sweep_kernel<true><<<sweep_grid(a.g, kz), block, 0, s>>>(a, kz);
    else init_sweep_kernel<false><<<sweep_grid(a.g, kz), block, 0, s>>>(a, kz);
    if (a.mu_guess) {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        return launch_mu_guess(a.g.N, a.mu, a.mu_guess, a.ex_a, a.ex_b, a.mu_off, a.mu_off_prev, s);
    }
    return cudaGetLastError();
}

cudaError_t launch_sweep(const SweepArgs &a, cudaStream_t s)
{
    int kz = zchunk(a.g);
    dim3 block(kBX, kBY);
    if (use_sweep2(a.g)) launch_sweep2<0>(a, kz, s);
    else if (a.g.L) sweep_kernel<true><<<sweep_grid(a.g, kz), block, 0, s>>>(a, kz);
    else sweep_kernel<false><<<sweep_grid(a.g, kz), block, 0, s>>>(a, kz);
    return cudaGetLastError();
}

cudaError_t launch_sweep_redo(const SweepArgs &a, cudaStream_t s)
{
    if (!use_sweep2(a.g) || a.g.Xj || a.g.lk) return cudaErrorInvalidValue;
    int kz = zchunk(a.g);
    sweep2_kernel<5><<<sweep2_grid(a.g, kz), dim3(kBX, kBY), 0, s>>>(a, kz);
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
        launch_sweep2<2>(sa, kz, s);
    } else if (a.g.L) poisson_rhs_kernel<true><<<grid, block, 0, s>>>(a.g, a.ctl, a.blockred, psi, a.f, inj, a.wsum, kz);
    else poisson_rhs_kernel<false><<<grid, block, 0, s>>>(a.g, a.ctl, a.blockred, psi, a.f, inj, a.wsum, kz);
    return cudaGetLastError();
}

}  // namespace tdgl

namespace tdgl {

// Adjoint Jacobi sweep for M^H lam = g (b = g, D = diag M of the forward step).
cudaError_t launch_adj_sweep(const SweepArgs &a, cudaStream_t s)
{
    if (!adj_supported(a.g)) return cudaErrorInvalidValue;
    int kz = zchunk(a.g);
    dim3 block(kBX, kBY);
    sweep2_kernel<3><<<sweep2_grid(a.g, kz), block, 0, s>>>(a, kz);
    return cudaGetLastError();
}

bool adj_supported(const DevGrid &g) { return g.L == nullptr && g.lk == nullptr && (g.nx % 2) == 0; }

}  // namespace tdgl
