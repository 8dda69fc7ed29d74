// Kernels of the reverse (adjoint) time step: gradient of the time-averaged
// voltage with respect to the pinning map alpha.  With H = diag(beta|psi|^2 +
// i u mu - alpha) - Lap_U, the Crank-Nicolson step of arXiv:1409.8340 Sec. 3.1
// is R = psi' - psi + (ht/2) H(psi, mu, alpha)(psi' + psi) = 0; one reverse step
// from (psi^n, mu^n) to (psi^{n-1}, mu^{n-1}) is
//   w            = W * G(mubar^n / W)     (adjoint of the Poisson solve G of Sec. 3.2)
//   g            = psibar^n + i [NS^H(w psi^n) - w NS(psi^n)]
//   M^H lam      = g                      (Jacobi, conj(D), transposed face rows)
//   dJ/dalpha   += (ht/2) Re[conj(lam) s],     s = psi^n + psi^{n-1}
//   mubar^{n-1}  = (ht/2) u Im[conj(lam) s]
//   psibar^{n-1} = 2 lam - g - ht beta Re[conj(lam) s] psi^{n-1}
// (the last line uses (ht/2) H^H lam = M^H lam - lam = g - lam at convergence).
// W are the trapezoid weights (1/2 per open face).  FP32 bulk, FP64 sums.
#include "tdgl_internal.cuh"

namespace tdgl {

constexpr int kAX = 128;   // threads per block along x; grid (x tiles, y, z)

__device__ __forceinline__ float trap_w(int bc, int n, int idx)
{
    return (bc == kOpen && n >= 2 && (idx == 0 || idx == n - 1)) ? 0.5f : 1.f;
}

// forward-operator and transposed-operator weights of the +/- neighbours on an open axis
__device__ __forceinline__ void open_weights(bool adj, int idx, int n, float &wf, float &wb)
{
    if (!adj) {
        wf = (idx == 0) ? 2.f : (idx == n - 1 ? 0.f : 1.f);
        wb = (idx == n - 1) ? 2.f : (idx == 0 ? 0.f : 1.f);
    } else {
        wf = (idx == n - 1) ? 0.f : (idx + 1 == n - 1 ? 2.f : 1.f);
        wb = (idx == 0) ? 0.f : (idx - 1 == 0 ? 2.f : 1.f);
    }
}

__device__ __forceinline__ int wrapn(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// g = psibar + i [NS^H(w psi) - w NS(psi)],  w = W * u   (x open: no wrap phase)
__global__ void __launch_bounds__(kAX) adj_fterm_kernel(DevGrid g, float2 Ux, const float2 *__restrict__ psi,
                                                       const float *__restrict__ u, const float2 *__restrict__ psibar,
                                                       float2 *__restrict__ gout)
{
    const int i = blockIdx.x * kAX + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    if (i >= g.nx) return;
    const long long sy = g.nx, sz = (long long)g.nx * g.ny;
    const long long m = i + sy * j + sz * k;
    const float Wm = trap_w(g.bcx, g.nx, i) * trap_w(g.bcy, g.ny, j) * trap_w(g.bcz, g.nz, k);
    const float wm = Wm * u[m];
    float2 A = cmk(0.f, 0.f), Bh = A;
    // one axis: index idx of n, stride st, coefficient c, link Uf (forward), Ub (from the backward site)
    auto axis = [&](int idx, int n, int bc, long long st, float c, float2 Uf, float2 Ub, int ax) {
        if (n < 2) return;
        const int ip = wrapn(idx + 1, n), im = wrapn(idx - 1, n);
        float wf, wb, af, ab;
        if (bc == kPeriodic) {
            wf = wb = af = ab = 1.f;
        } else {
            open_weights(false, idx, n, wf, wb);
            open_weights(true, idx, n, af, ab);
        }
        const long long mp = m + (long long)(ip - idx) * st, mm = m + (long long)(im - idx) * st;
        const float2 pp = psi[mp], pm = psi[mm];
        // W at the neighbours
        int ci[3] = {i, j, k};
        ci[ax] = ip;
        const float Wp = trap_w(g.bcx, g.nx, ci[0]) * trap_w(g.bcy, g.ny, ci[1]) * trap_w(g.bcz, g.nz, ci[2]);
        ci[ax] = im;
        const float Wn = trap_w(g.bcx, g.nx, ci[0]) * trap_w(g.bcy, g.ny, ci[1]) * trap_w(g.bcz, g.nz, ci[2]);
        const float up = Wp * u[mp], um = Wn * u[mm];
        // forward NS(psi): c [wf Uf psi_+ + wb conj(Ub) psi_-]
        cfma(A, cscale(c * wf, Uf), pp);
        cfmac(A, cscale(c * wb, Ub), pm);
        // transposed NS^H(w psi): c [af Uf (w psi)_+ + ab conj(Ub) (w psi)_-]
        cfma(Bh, cscale(c * af * up, Uf), pp);
        cfmac(Bh, cscale(c * ab * um, Ub), pm);
    };
    axis(i, g.nx, g.bcx, 1, g.cx, Ux, Ux, 0);
    axis(j, g.ny, g.bcy, sy, g.cy, g.Uy[i], g.Uy[i], 1);
    axis(k, g.nz, g.bcz, sz, g.cz, g.Uz[i], g.Uz[i], 2);
    const float2 d = csub(Bh, cscale(wm, A));
    const float2 pb = psibar[m];
    gout[m] = make_float2(pb.x - d.y, pb.y + d.x);   // psibar + i d
}

// D = diag M(psi^{n-1}, mu^{n-1}, alpha); lam0 = g / conj(D)
__global__ void adj_diag_kernel(DevGrid g, const float2 *__restrict__ psi_p, const float *__restrict__ mu_p,
                                const float *__restrict__ alpha, const float2 *__restrict__ gv, float2 *__restrict__ D,
                                float2 *__restrict__ lam0)
{
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < g.N; m += (long long)gridDim.x * blockDim.x) {
        const float a2 = cabs2(psi_p[m]);
        const float2 d = cmk(1.f + g.ht2 * (g.beta * a2 + 2.f * g.S - alpha[m]), g.ht2 * g.u * mu_p[m]);
        D[m] = d;
        lam0[m] = cscale(1.f / cabs2(d), cmul(d, gv[m]));   // g / conj(d) = g d / |d|^2
    }
}

// back-propagation of the step's residual
__global__ void adj_update_kernel(DevGrid g, const float2 *__restrict__ lam, const float2 *__restrict__ psi_n,
                                  const float2 *__restrict__ psi_p, const float2 *__restrict__ gv,
                                  float *__restrict__ grad, float *__restrict__ mubar, float2 *__restrict__ psibar)
{
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < g.N; m += (long long)gridDim.x * blockDim.x) {
        const float2 l = lam[m], pp = psi_p[m];
        const float2 s = cadd(psi_n[m], pp);
        const float2 ls = cmulc(l, s);   // conj(lam) s
        grad[m] += g.ht2 * ls.x;
        mubar[m] = g.ht2 * g.u * ls.y;
        const float2 gg = gv[m];
        const float cb = 2.f * g.ht2 * g.beta * ls.x;   // ht beta Re[conj(lam) s]
        psibar[m] = make_float2(2.f * l.x - gg.x - cb * pp.x, 2.f * l.y - gg.y - cb * pp.y);
    }
}

// mubar += v / nwin on the x faces (E_x = v . mu)
__global__ void adj_voltage_source_kernel(DevGrid g, float *mubar, float s)
{
    const long long nf = (long long)g.ny * g.nz;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nf; q += (long long)gridDim.x * blockDim.x) {
        mubar[q * g.nx] += s;
        mubar[q * g.nx + g.nx - 1] -= s;
    }
}

// r = mubar / W  and  ctl->fmean = sum_m W_m r_m / sum W  (FP64)
__global__ void __launch_bounds__(kAX) adj_rhs_kernel(DevGrid g, const float *__restrict__ mubar, float *__restrict__ r,
                                                     DevCtl *ctl, double *blockred, double wsum)
{
    const int i = blockIdx.x * kAX + threadIdx.x, j = blockIdx.y;
    float acc = 0.f;
    if (i < g.nx) {
        const float wxy = trap_w(g.bcx, g.nx, i) * trap_w(g.bcy, g.ny, j);
        for (int k = 0; k < g.nz; ++k) {
            const long long m = i + (long long)g.nx * (j + (long long)g.ny * k);
            const float W = wxy * trap_w(g.bcz, g.nz, k);
            const float v = mubar[m];
            r[m] = v / W;
            acc += v;
        }
    }
    __shared__ double shd[32];
    __shared__ int flag;
    const unsigned int bid = blockIdx.x + gridDim.x * blockIdx.y, nb = gridDim.x * gridDim.y;
    double s = block_sum((double)acc, shd);
    if (threadIdx.x == 0) blockred[bid] = s;
    if (!last_block(&ctl->ticket, nb, &flag)) return;
    double t = 0.0;
    for (unsigned int q = threadIdx.x; q < nb; q += blockDim.x) t += ((volatile double *)blockred)[q];
    t = block_sum(t, shd);
    if (threadIdx.x == 0) {
        ctl->ticket = 0u;
        ctl->fmean = t / wsum;
    }
}

static int eblocks(long long n)
{
    long long b = (n + 255) / 256;
    return (int)(b > 8192 ? 8192 : (b < 1 ? 1 : b));
}

cudaError_t launch_adj_fterm(const DevGrid &g, float2 Ux, const float2 *psi, const float *u, const float2 *psibar,
                             float2 *gout, cudaStream_t s)
{
    dim3 grid((g.nx + kAX - 1) / kAX, g.ny, g.nz);
    adj_fterm_kernel<<<grid, kAX, 0, s>>>(g, Ux, psi, u, psibar, gout);
    return cudaGetLastError();
}

cudaError_t launch_adj_diag(const DevGrid &g, const float2 *psi_p, const float *mu_p, const float *alpha,
                            const float2 *gv, float2 *D, float2 *lam0, cudaStream_t s)
{
    adj_diag_kernel<<<eblocks(g.N), 256, 0, s>>>(g, psi_p, mu_p, alpha, gv, D, lam0);
    return cudaGetLastError();
}

cudaError_t launch_adj_update(const DevGrid &g, const float2 *lam, const float2 *psi_n, const float2 *psi_p,
                              const float2 *gv, float *grad, float *mubar, float2 *psibar, cudaStream_t s)
{
    adj_update_kernel<<<eblocks(g.N), 256, 0, s>>>(g, lam, psi_n, psi_p, gv, grad, mubar, psibar);
    return cudaGetLastError();
}

cudaError_t launch_adj_voltage_source(const DevGrid &g, float *mubar, float s_val, cudaStream_t s)
{
    long long nf = (long long)g.ny * g.nz;
    adj_voltage_source_kernel<<<eblocks(nf), 256, 0, s>>>(g, mubar, s_val);
    return cudaGetLastError();
}

cudaError_t launch_adj_rhs(const DevGrid &g, const float *mubar, float *r, DevCtl *ctl, double *blockred, double wsum,
                           cudaStream_t s)
{
    dim3 grid((g.nx + kAX - 1) / kAX, g.ny);
    adj_rhs_kernel<<<grid, kAX, 0, s>>>(g, mubar, r, ctl, blockred, wsum);
    return cudaGetLastError();
}

}  // namespace tdgl
