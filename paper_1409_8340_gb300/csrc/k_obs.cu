// J_av and the K ODE (arXiv:1409.8340, Sec. 2.2 Eq. K_ODE, Sec. 3.1.1 J_av), and
// the observables: <|psi|^2>, the discrete free energy with trapezoid face
// weights, and the winding of xy plaquettes.  Bulk arithmetic in FP32, sums in
// FP64, finished on the device by the last block.
#include <float.h>

#include "tdgl_internal.cuh"

namespace tdgl {

constexpr int kRedThreads = 256;

static int red_blocks(long long N)
{
    long long b = (N + kRedThreads * 8 - 1) / (kRedThreads * 8);
    if (b > 4096) b = 4096;
    if (b < 1) b = 1;
    return (int)b;
}

__device__ __forceinline__ void site_ijk(const DevGrid &g, long long m, int &i, int &j, int &k)
{
    i = (int)(m % g.nx);
    long long t = m / g.nx;
    j = (int)(t % g.ny);
    k = (int)(t / g.ny);
}

// Forward link from (i,j,k) along x, including K and the periodic wrap phase.
template <bool GEN>
__device__ __forceinline__ float2 link_x(const DevGrid &g, float2 Ux, int i, int j, int k, long long m)
{
    if (GEN) return cmul(Ux, g.L[m]);
    if (i == g.nx - 1 && g.bcx == kPeriodic) return cmulc(cmul(g.Py[j], g.Pz[k]), Ux);
    return Ux;
}
template <bool GEN>
__device__ __forceinline__ float2 link_y(const DevGrid &g, int i, long long m)
{
    return GEN ? g.L[g.N + m] : g.Uy[i];
}
template <bool GEN>
__device__ __forceinline__ float2 link_z(const DevGrid &g, int i, long long m)
{
    return GEN ? g.L[2 * g.N + m] : g.Uz[i];
}

__device__ __forceinline__ long long wrapped(const DevGrid &g, int i, int j, int k)
{
    i = (i + g.nx) % g.nx;
    j = (j + g.ny) % g.ny;
    k = (k + g.nz) % g.nz;
    return (long long)i + (long long)g.nx * ((long long)j + (long long)g.ny * k);
}

// ---------------------------------------------------------------------------
// J_av (periodic x) and the explicit-Euler K update with the rewind rule.
// ---------------------------------------------------------------------------
template <bool GEN>
__global__ void javg_K_kernel(KArgs a)
{
    const DevGrid &g = a.g;
    const float2 Ux = a.ctl->Ux;
    double acc = 0.0;
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < g.N; m += (long long)gridDim.x * blockDim.x) {
        int i, j, k;
        site_ijk(g, m, i, j, k);
        float2 p = a.psi[m];
        long long mp = wrapped(g, i + 1, j, k), mm = wrapped(g, i - 1, j, k);
        float2 fwd = cmul(link_x<GEN>(g, Ux, i, j, k, m), a.psi[mp]);
        int im = (i - 1 + g.nx) % g.nx;
        float2 bwd = cmulc(link_x<GEN>(g, Ux, im, j, k, mm), a.psi[mm]);
        if (g.lk) {   // links next to insulating sites carry no current
            const unsigned l = g.lk[m];
            if (!(l & kLkXp)) fwd = cmk(0.f, 0.f);
            if (!(l & kLkXm)) bwd = cmk(0.f, 0.f);
        }
        float2 d = csub(fwd, bwd);
        acc += (double)(p.x * d.y - p.y * d.x);   // Im[conj(p) d]
    }
    __shared__ double shd[32];
    __shared__ int flag;
    double s = block_sum(acc, shd);
    if (threadIdx.x == 0) a.blockred[blockIdx.x] = s;
    if (!last_block(&a.ctl->ticket, gridDim.x, &flag)) return;
    double t = 0.0;
    for (unsigned int q = threadIdx.x; q < gridDim.x; q += blockDim.x) t += ((volatile double *)a.blockred)[q];
    t = block_sum(t, shd);
    if (threadIdx.x == 0) {
        a.ctl->ticket = 0u;
        k_ode_update(a.ctl, t / (2.0 * (double)g.N * a.hx), a.hx, a.dtK, a.Jext, a.update_K);
    }
}

cudaError_t launch_javg_K(const KArgs &a, cudaStream_t s)
{
    int nb = red_blocks(a.g.N);
    if (a.g.L) javg_K_kernel<true><<<nb, kRedThreads, 0, s>>>(a);
    else javg_K_kernel<false><<<nb, kRedThreads, 0, s>>>(a);
    return cudaGetLastError();
}

__global__ void set_Ux_kernel(DevCtl *ctl, double hx)
{
    double sn, cs;
    sincos(hx * ctl->K, &sn, &cs);
    ctl->Ux = make_float2((float)cs, (float)sn);
}

cudaError_t launch_set_Ux(DevCtl *ctl, double hx, cudaStream_t s)
{
    set_Ux_kernel<<<1, 1, 0, s>>>(ctl, hx);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Observables: sums[0] = sum |psi|^2, sums[1] = free energy / dV,
// sums[2] = sum |n_p|, sums[3] = sum n_p.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float face_w(int bc, int n, int idx)
{
    return (bc == kOpen && n >= 2 && (idx == 0 || idx == n - 1)) ? 0.5f : 1.0f;
}

__device__ __forceinline__ float phase_of(float2 z) { return atan2f(z.y, z.x); }

template <bool GEN>
__global__ void observables_kernel(DevGrid g, DevCtl *ctl, double *blockred, const float2 *__restrict__ psi,
                                   const float *__restrict__ alpha, float flux)
{
    const float2 Ux = ctl->Ux;
    double s_psi2 = 0.0, s_F = 0.0, s_abs = 0.0, s_sgn = 0.0;
    const float twopi = 6.28318530717958647692f;
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < g.N; m += (long long)gridDim.x * blockDim.x) {
        int i, j, k;
        site_ijk(g, m, i, j, k);
        float2 p = psi[m];
        float a2 = cabs2(p);
        s_psi2 += (double)a2;
        float wx = face_w(g.bcx, g.nx, i), wy = face_w(g.bcy, g.ny, j), wz = face_w(g.bcz, g.nz, k);
        float e = wx * wy * wz * (-alpha[m] * a2 + 0.5f * g.beta * a2 * a2);
        // links along x, y, z leaving this site (without the removed ones next to insulating sites)
        const unsigned l = g.lk ? g.lk[m] : 0x3Fu;
        if ((g.bcx == kPeriodic || i < g.nx - 1) && (l & kLkXp)) {
            float2 d = csub(cmul(link_x<GEN>(g, Ux, i, j, k, m), psi[wrapped(g, i + 1, j, k)]), p);
            e += wy * wz * g.cx * cabs2(d);
        }
        if ((g.bcy == kPeriodic || j < g.ny - 1) && (l & kLkYp)) {
            float2 d = csub(cmul(link_y<GEN>(g, i, m), psi[wrapped(g, i, j + 1, k)]), p);
            e += wx * wz * g.cy * cabs2(d);
        }
        if (g.nz >= 2 && (g.bcz == kPeriodic || k < g.nz - 1) && (l & kLkZp)) {
            float2 d = csub(cmul(link_z<GEN>(g, i, m), psi[wrapped(g, i, j, k + 1)]), p);
            e += wx * wy * g.cz * cabs2(d);
        }
        s_F += (double)e;
        // xy plaquette with lower-left corner (i, j)
        bool has = (g.bcx == kPeriodic || i < g.nx - 1) && (g.bcy == kPeriodic || j < g.ny - 1);
        if (has) {
            int i1 = (i + 1) % g.nx, j1 = (j + 1) % g.ny;
            long long mb = wrapped(g, i1, j, k), mc = wrapped(g, i1, j1, k), md = wrapped(g, i, j1, k);
            // plaquettes with an insulating corner hold no winding
            if (g.lk && ((g.lk[m] | g.lk[mb] | g.lk[mc] | g.lk[md]) & kLkIns)) has = false;
        }
        if (has) {
            int i1 = (i + 1) % g.nx, j1 = (j + 1) % g.ny;
            long long mb = wrapped(g, i1, j, k), mc = wrapped(g, i1, j1, k), md = wrapped(g, i, j1, k);
            float2 pb = psi[mb], pc = psi[mc], pd = psi[md];
            float t_ab = phase_of(cmul(cmulc(p, link_x<GEN>(g, Ux, i, j, k, m)), pb));
            float t_bc = phase_of(cmul(cmulc(pb, link_y<GEN>(g, i1, mb)), pc));
            float t_cd = phase_of(cmul(cmulc(pc, cconj(link_x<GEN>(g, Ux, i, j1, k, md))), pd));
            float t_da = phase_of(cmul(cmulc(pd, cconj(link_y<GEN>(g, i, m))), p));
            float w = (t_ab + t_bc + t_cd + t_da + flux) / twopi;
            float n = floorf(w + 0.5f);
            s_abs += (double)fabsf(n);
            s_sgn += (double)n;
        }
    }
    __shared__ double shd[32];
    __shared__ int flag;
    double v[4] = {s_psi2, s_F, s_abs, s_sgn};
    for (int q = 0; q < 4; ++q) {
        double t = block_sum(v[q], shd);
        if (threadIdx.x == 0) blockred[4 * blockIdx.x + q] = t;
    }
    if (!last_block(&ctl->ticket, gridDim.x, &flag)) return;
    for (int q = 0; q < 4; ++q) {
        double t = 0.0;
        for (unsigned int b = threadIdx.x; b < gridDim.x; b += blockDim.x) t += ((volatile double *)blockred)[4 * b + q];
        t = block_sum(t, shd);
        if (threadIdx.x == 0) ctl->sums[q] = t;
    }
    if (threadIdx.x == 0) ctl->ticket = 0u;
}

cudaError_t launch_observables(const DevGrid &g, DevCtl *ctl, double *blockred, const float2 *psi,
                               const float *alpha, int32_t *, double flux, cudaStream_t s)
{
    int nb = red_blocks(g.N);
    if (g.L) observables_kernel<true><<<nb, kRedThreads, 0, s>>>(g, ctl, blockred, psi, alpha, (float)flux);
    else observables_kernel<false><<<nb, kRedThreads, 0, s>>>(g, ctl, blockred, psi, alpha, (float)flux);
    return cudaGetLastError();
}

}  // namespace tdgl
