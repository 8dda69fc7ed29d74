// Scalar potential: exact discrete solve of Lap mu = F (arXiv:1409.8340, Sec. 3.2,
// Eq. Poisson; the fixed point of the paper's pseudo-time relaxation) by
// geometric multigrid.
//
// x is never coarsened: every level keeps all Nx points and is smoothed by
// zebra line Gauss-Seidel, each x line solved exactly (Thomas algorithm, or
// Sherman-Morrison for a periodic x line) in shared memory.  y and z are
// coarsened by 2 while the size allows (periodic: even N >= 8; open: odd
// N >= 5), with full weighting and bilinear interpolation.  This pairing
// (x-line relaxation, yz semi-coarsening) is robust to the strong x coupling of
// the coarse levels and to any Nx, including the odd interval count of an open
// x axis.  The zero mode (constants) is removed in FP64: the right-hand side is
// projected onto sum_m w_m F_m = 0 and the solution onto sum_m w_m mu_m = 0, w
// the trapezoid weights (1/2 per open face).
#include <float.h>

#include "tdgl_internal.cuh"

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
// x-line factors (host, FP64): tri = [c' (nx) | 1/pivot (nx) | a (nx) | z (nx) | bg, 1/(1+v.z)]
// for rows a_i u_{i-1} + d u_i + c_i u_{i+1} = rhs_i, d = 2(cx+cy+cz).
// ---------------------------------------------------------------------------
void mg_line_factors(int nx, int bcx, float cx_f, float cy_f, float cz_f, float *tri)
{
    const double cx = cx_f, cy = cy_f, cz = cz_f;
    const double d = 2.0 * (cx + cy + cz);
    double *a = new double[nx], *c = new double[nx], *dd = new double[nx];
    for (int i = 0; i < nx; ++i) {
        a[i] = (i == 0) ? 0.0 : -cx;
        c[i] = (i == nx - 1) ? 0.0 : -cx;
        dd[i] = d;
    }
    double gam = -d, bg = 0.0;
    if (bcx == kOpen) {
        c[0] = -2.0 * cx;
        a[nx - 1] = -2.0 * cx;
    } else {
        // cyclic: T = T' + u v^T, u = (gam, 0.., alpha), v = (1, 0.., beta/gam)
        const double alpha = -cx, beta = -cx;
        dd[0] = d - gam;
        dd[nx - 1] = d - alpha * beta / gam;
        bg = beta / gam;
    }
    double *cp = new double[nx], *ip = new double[nx];
    for (int i = 0; i < nx; ++i) {
        double piv = dd[i] - (i > 0 ? a[i] * cp[i - 1] : 0.0);
        ip[i] = 1.0 / piv;
        cp[i] = c[i] * ip[i];
    }
    for (int i = 0; i < nx; ++i) {
        tri[i] = (float)cp[i];
        tri[nx + i] = (float)ip[i];
        tri[2 * nx + i] = (float)a[i];
        tri[3 * nx + i] = 0.f;
    }
    tri[4 * nx] = 0.f;
    tri[4 * nx + 1] = 0.f;
    if (bcx == kPeriodic) {
        // z = T'^{-1} u
        double *y = new double[nx];
        for (int i = 0; i < nx; ++i) {
            double rhs = (i == 0) ? gam : (i == nx - 1 ? -cx : 0.0);
            y[i] = (rhs - (i > 0 ? a[i] * y[i - 1] : 0.0)) * ip[i];
        }
        for (int i = nx - 2; i >= 0; --i) y[i] -= cp[i] * y[i + 1];
        double vz = y[0] + bg * y[nx - 1];
        for (int i = 0; i < nx; ++i) tri[3 * nx + i] = (float)y[i];
        tri[4 * nx] = (float)bg;
        tri[4 * nx + 1] = (float)(1.0 / (1.0 + vz));
        delete[] y;
    }
    delete[] a;
    delete[] c;
    delete[] dd;
    delete[] cp;
    delete[] ip;
}

// neighbour index along a coarse/fine axis with periodic wrap or Neumann mirror
__device__ __forceinline__ int nb_idx(int j, int d, int n, int bc)
{
    int q = j + d;
    if (bc == kPeriodic) {
        if (q < 0) q += n;
        if (q >= n) q -= n;
    } else {
        if (q < 0) q = -q;
        if (q > n - 1) q = 2 * (n - 1) - q;
    }
    return q;
}

// q-th line of colour c ((j + k) % 2 == c) on an ny x nz line grid
__device__ __forceinline__ void line_jk(long long q, int c, int ny, int nz, int &j, int &k)
{
    if ((ny & 1) == 0) {
        int half = ny >> 1;
        k = (int)(q / half);
        int jj = (int)(q % half);
        j = 2 * jj + ((c + k) & 1);
    } else {
        long long kp = q / ny;
        int rem = (int)(q % ny);
        int cnt0 = (ny + 1 - c) / 2;
        if (rem < cnt0) {
            k = (int)(2 * kp);
            j = 2 * rem + (c & 1);
        } else {
            k = (int)(2 * kp + 1);
            j = 2 * (rem - cnt0) + ((c + 1) & 1);
        }
    }
}

static long long lines_of_colour(int ny, int nz, int c)
{
    long long n = 0;
    for (int k = 0; k < nz; ++k) n += (ny + 1 - ((c + k) & 1)) / 2;
    return n;
}

struct LineArgs {
    MGLevel L;
    int bcx, bcy, bcz;
    int color;
    long long nlines;
    int lpb;
    const DevCtl *ctl;
    int level0;
};

__global__ void __launch_bounds__(kThreads) line_smooth_kernel(LineArgs A)
{
    extern __shared__ float sm[];
    const MGLevel &L = A.L;
    const int nx = L.nx, ny = L.ny, nz = L.nz;
    const int stride = nx + 1;
    float *tri = sm + A.lpb * stride;
    for (int t = threadIdx.x; t < 4 * nx + 2; t += blockDim.x) tri[t] = L.tri[t];
    const long long q0 = (long long)blockIdx.x * A.lpb;
    const float fsub = A.level0 ? (float)A.ctl->fmean : 0.f;
    const long long plane = (long long)nx * ny;
    for (int e = threadIdx.x; e < A.lpb * nx; e += blockDim.x) {
        const int q = e / nx, i = e - q * nx;
        if (q0 + q >= A.nlines) break;
        int j, k;
        line_jk(q0 + q, A.color, ny, nz, j, k);
        const long long base = (long long)nx * j + plane * k;
        float v = -(L.r[base + i] - fsub);
        if (ny >= 2) {
            int jp = nb_idx(j, 1, ny, A.bcy), jm = nb_idx(j, -1, ny, A.bcy);
            v += L.cy * (L.u[(long long)nx * jp + plane * k + i] + L.u[(long long)nx * jm + plane * k + i]);
        }
        if (nz >= 2) {
            int kp = nb_idx(k, 1, nz, A.bcz), km = nb_idx(k, -1, nz, A.bcz);
            v += L.cz * (L.u[(long long)nx * j + plane * kp + i] + L.u[(long long)nx * j + plane * km + i]);
        }
        sm[q * stride + i] = v;
    }
    __syncthreads();
    if (threadIdx.x < A.lpb && q0 + threadIdx.x < A.nlines) {
        float *row = sm + threadIdx.x * stride;
        const float *cp = tri, *ip = tri + nx, *aa = tri + 2 * nx, *zz = tri + 3 * nx;
        float y = row[0] * ip[0];
        row[0] = y;
        for (int i = 1; i < nx; ++i) {
            y = (row[i] - aa[i] * y) * ip[i];
            row[i] = y;
        }
        float x = row[nx - 1];
        for (int i = nx - 2; i >= 0; --i) {
            x = row[i] - cp[i] * x;
            row[i] = x;
        }
        if (A.bcx == kPeriodic) {
            const float fac = (row[0] + tri[4 * nx] * row[nx - 1]) * tri[4 * nx + 1];
            for (int i = 0; i < nx; ++i) row[i] -= fac * zz[i];
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < A.lpb * nx; e += blockDim.x) {
        const int q = e / nx, i = e - q * nx;
        if (q0 + q >= A.nlines) break;
        int j, k;
        line_jk(q0 + q, A.color, ny, nz, j, k);
        L.u[(long long)nx * j + plane * k + i] = sm[q * stride + i];
    }
}

// t = F - L u on one level (level 0: F = f - fmean).  Optionally the max norms.
__global__ void residual_kernel(MGLevel L, int bcx, int bcy, int bcz, const DevCtl *ctl, int level0)
{
    const float fsub = level0 ? (float)ctl->fmean : 0.f;
    const int nx = L.nx, ny = L.ny, nz = L.nz;
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < L.N; m += (long long)gridDim.x * blockDim.x) {
        int i = (int)(m % nx);
        long long t = m / nx;
        int j = (int)(t % ny), k = (int)(t / ny);
        const float u0 = L.u[m];
        float lap = 0.f;
        {
            int ip = nb_idx(i, 1, nx, bcx), im = nb_idx(i, -1, nx, bcx);
            lap += L.cx * (L.u[m - i + ip] + L.u[m - i + im] - 2.f * u0);
        }
        if (ny >= 2) {
            int jp = nb_idx(j, 1, ny, bcy), jm = nb_idx(j, -1, ny, bcy);
            lap += L.cy * (L.u[m + (long long)nx * (jp - j)] + L.u[m + (long long)nx * (jm - j)] - 2.f * u0);
        }
        if (nz >= 2) {
            int kp = nb_idx(k, 1, nz, bcz), km = nb_idx(k, -1, nz, bcz);
            const long long pl = (long long)nx * ny;
            lap += L.cz * (L.u[m + pl * (kp - k)] + L.u[m + pl * (km - k)] - 2.f * u0);
        }
        L.t[m] = (L.r[m] - fsub) - lap;
    }
}

// max |F - L u| and max |F| on level 0 (ctl->res = ratio)
__global__ void residual_norm_kernel(MGLevel L, int bcx, int bcy, int bcz, DevCtl *ctl, double *blockred)
{
    const float fsub = (float)ctl->fmean;
    const int nx = L.nx, ny = L.ny, nz = L.nz;
    float rmax = 0.f, fmax = 0.f;
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < L.N; m += (long long)gridDim.x * blockDim.x) {
        int i = (int)(m % nx);
        long long t = m / nx;
        int j = (int)(t % ny), k = (int)(t / ny);
        const float u0 = L.u[m];
        float lap = 0.f;
        {
            int ip = nb_idx(i, 1, nx, bcx), im = nb_idx(i, -1, nx, bcx);
            lap += L.cx * (L.u[m - i + ip] + L.u[m - i + im] - 2.f * u0);
        }
        if (ny >= 2) {
            int jp = nb_idx(j, 1, ny, bcy), jm = nb_idx(j, -1, ny, bcy);
            lap += L.cy * (L.u[m + (long long)nx * (jp - j)] + L.u[m + (long long)nx * (jm - j)] - 2.f * u0);
        }
        if (nz >= 2) {
            int kp = nb_idx(k, 1, nz, bcz), km = nb_idx(k, -1, nz, bcz);
            const long long pl = (long long)nx * ny;
            lap += L.cz * (L.u[m + pl * (kp - k)] + L.u[m + pl * (km - k)] - 2.f * u0);
        }
        const float F = L.r[m] - fsub;
        rmax = fmaxf(rmax, fabsf(F - lap));
        fmax = fmaxf(fmax, fabsf(F));
    }
    __shared__ float shf[32];
    __shared__ int flag;
    float a = block_max(rmax, shf);
    float b = block_max(fmax, shf);
    if (threadIdx.x == 0) {
        blockred[2 * blockIdx.x] = a;
        blockred[2 * blockIdx.x + 1] = b;
    }
    if (!last_block(&ctl->ticket, gridDim.x, &flag)) return;
    float ra = 0.f, rb = 0.f;
    for (unsigned int q = threadIdx.x; q < gridDim.x; q += blockDim.x) {
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

// r_c = full weighting of t_f (y, z); u_c = 0
__global__ void restrict_kernel(MGLevel F, MGLevel C, int bcy, int bcz)
{
    const int nx = C.nx;
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < C.N; m += (long long)gridDim.x * blockDim.x) {
        int i = (int)(m % nx);
        long long t = m / nx;
        int J = (int)(t % C.ny), K = (int)(t / C.ny);
        float acc = 0.f;
        for (int dk = -1; dk <= 1; ++dk) {
            float wk = (F.fz == 2) ? (dk == 0 ? 0.5f : 0.25f) : (dk == 0 ? 1.f : 0.f);
            if (wk == 0.f) continue;
            int kf = (F.nz >= 2) ? nb_idx(F.fz * K, dk, F.nz, bcz) : 0;
            for (int dj = -1; dj <= 1; ++dj) {
                float wj = (F.fy == 2) ? (dj == 0 ? 0.5f : 0.25f) : (dj == 0 ? 1.f : 0.f);
                if (wj == 0.f) continue;
                int jf = nb_idx(F.fy * J, dj, F.ny, bcy);
                acc += wk * wj * F.t[(long long)nx * (jf + (long long)F.ny * kf) + i];
            }
        }
        C.r[m] = acc;
        C.u[m] = 0.f;
    }
}

// u_f += bilinear interpolation of u_c
__global__ void prolong_kernel(MGLevel F, MGLevel C, int bcy, int bcz)
{
    const int nx = F.nx;
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < F.N; m += (long long)gridDim.x * blockDim.x) {
        int i = (int)(m % nx);
        long long t = m / nx;
        int j = (int)(t % F.ny), k = (int)(t / F.ny);
        int j0, j1, k0, k1;
        float wj1, wk1;
        if (F.fy == 2) {
            j0 = j >> 1;
            j1 = (j & 1) ? ((j0 + 1 < C.ny) ? j0 + 1 : (bcy == kPeriodic ? 0 : j0)) : j0;
            wj1 = (j & 1) ? 0.5f : 0.f;
        } else {
            j0 = j1 = j;
            wj1 = 0.f;
        }
        if (F.fz == 2) {
            k0 = k >> 1;
            k1 = (k & 1) ? ((k0 + 1 < C.nz) ? k0 + 1 : (bcz == kPeriodic ? 0 : k0)) : k0;
            wk1 = (k & 1) ? 0.5f : 0.f;
        } else {
            k0 = k1 = k;
            wk1 = 0.f;
        }
        const long long cpl = (long long)nx * C.ny;
        float v00 = C.u[(long long)nx * j0 + cpl * k0 + i];
        float v10 = C.u[(long long)nx * j1 + cpl * k0 + i];
        float v01 = C.u[(long long)nx * j0 + cpl * k1 + i];
        float v11 = C.u[(long long)nx * j1 + cpl * k1 + i];
        float v = (1.f - wk1) * ((1.f - wj1) * v00 + wj1 * v10) + wk1 * ((1.f - wj1) * v01 + wj1 * v11);
        F.u[m] += v;
    }
}

static cudaError_t smooth(const PoissonArgs &a, int l, int color, cudaStream_t s, long long *nl)
{
    const MGLevel &L = a.lev[l];
    LineArgs A;
    A.L = L;
    A.bcx = a.g.bcx;
    A.bcy = a.g.bcy;
    A.bcz = a.g.bcz;
    A.color = color;
    A.nlines = lines_of_colour(L.ny, L.nz, color);
    A.ctl = a.ctl;
    A.level0 = (l == 0);
    int lpb = (int)((200 * 1024 - 4 * (4 * L.nx + 2)) / (4 * (L.nx + 1)));
    if (lpb > 32) lpb = 32;
    if (lpb < 1) lpb = 1;
    A.lpb = lpb;
    if (A.nlines == 0) return cudaSuccess;
    size_t smem = (size_t)4 * (lpb * (L.nx + 1) + 4 * L.nx + 2);
    int nb = (int)((A.nlines + lpb - 1) / lpb);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(line_smooth_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        attr_set = true;
    }
    line_smooth_kernel<<<nb, kThreads, smem, s>>>(A);
    ++*nl;
    return cudaGetLastError();
}

static cudaError_t vcycle(const PoissonArgs &a, int l, cudaStream_t s, long long *nl)
{
    const int bcx = a.g.bcx, bcy = a.g.bcy, bcz = a.g.bcz;
    if (l == a.nlevels - 1) {
        int n = 2 * (a.lev[l].ny + a.lev[l].nz) + 8;
        for (int it = 0; it < n; ++it) {
            smooth(a, l, 0, s, nl);
            smooth(a, l, 1, s, nl);
        }
        return cudaGetLastError();
    }
    smooth(a, l, 0, s, nl);
    smooth(a, l, 1, s, nl);
    residual_kernel<<<grid_blocks(a.lev[l].N), kThreads, 0, s>>>(a.lev[l], bcx, bcy, bcz, a.ctl, l == 0);
    restrict_kernel<<<grid_blocks(a.lev[l + 1].N), kThreads, 0, s>>>(a.lev[l], a.lev[l + 1], bcy, bcz);
    *nl += 3;
    vcycle(a, l + 1, s, nl);
    prolong_kernel<<<grid_blocks(a.lev[l].N), kThreads, 0, s>>>(a.lev[l], a.lev[l + 1], bcy, bcz);
    smooth(a, l, 1, s, nl);
    smooth(a, l, 0, s, nl);
    return cudaGetLastError();
}

cudaError_t launch_vcycle(const PoissonArgs &a, cudaStream_t s, long long *launches) { return vcycle(a, 0, s, launches); }

cudaError_t launch_poisson_residual(const PoissonArgs &a, cudaStream_t s)
{
    int nb = grid_blocks(a.lev[0].N, 8);
    if (nb > 2048) nb = 2048;
    residual_norm_kernel<<<nb, kThreads, 0, s>>>(a.lev[0], a.g.bcx, a.g.bcy, a.g.bcz, a.ctl, a.blockred);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Zero mode of mu: subtract the weighted mean (FP64 sum).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float site_w(const DevGrid &g, long long m)
{
    int i = (int)(m % g.nx);
    long long t = m / g.nx;
    int j = (int)(t % g.ny), k = (int)(t / g.ny);
    float w = 1.f;
    if (g.bcx == kOpen && (i == 0 || i == g.nx - 1)) w *= 0.5f;
    if (g.bcy == kOpen && (j == 0 || j == g.ny - 1)) w *= 0.5f;
    if (g.bcz == kOpen && g.nz >= 2 && (k == 0 || k == g.nz - 1)) w *= 0.5f;
    return w;
}

__global__ void mu_mean_kernel(DevGrid g, const float *mu, DevCtl *ctl, double *blockred, double wsum)
{
    double acc = 0.0;
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < g.N; m += (long long)gridDim.x * blockDim.x)
        acc += (double)(site_w(g, m) * mu[m]);
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
        ctl->mu_mean = t / wsum;
    }
}

__global__ void mu_shift_kernel(long long N, float *mu, const DevCtl *ctl)
{
    const float c = (float)ctl->mu_mean;
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < N; m += (long long)gridDim.x * blockDim.x)
        mu[m] -= c;
}

cudaError_t launch_project_mu(const PoissonArgs &a, cudaStream_t s)
{
    int nb = grid_blocks(a.g.N, 8);
    if (nb > 2048) nb = 2048;
    mu_mean_kernel<<<nb, kThreads, 0, s>>>(a.g, a.mu, a.ctl, a.blockred, a.wsum);
    mu_shift_kernel<<<grid_blocks(a.g.N, 8), kThreads, 0, s>>>(a.g.N, a.mu, a.ctl);
    return cudaGetLastError();
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
