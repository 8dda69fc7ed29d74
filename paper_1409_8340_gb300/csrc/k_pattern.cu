// Inclusion pattern generator (arXiv:1409.8340, Sec. 3.4: eps(r) modulation by
// inclusions of given shape; here spheres and ellipsoids placed at random).
//
// The paper's sequential rule "add candidates until the volume fraction is
// reached" is evaluated in parallel: every site records the index of the first
// candidate that contains it (atomicMin over candidates rastered inside their
// bounding boxes), a histogram of those indices gives the number of newly
// covered sites per candidate, one block scans it to find how many candidates
// are needed, and a final pass writes alpha.  The result equals the sequential
// rule bit for bit.  The inside test runs in FP64 with every product and sum
// rounded separately (no fused multiply-add), in a fixed evaluation order, so
// that the decision at each site is reproducible.
#include <float.h>

#include "tdgl_internal.cuh"

namespace tdgl {

struct PatternArgs {
    int nx, ny, nz, bcx, bcy, bcz;
    double h[3];
    const double *incl;
    long long n_incl;
    int *first;
};

__device__ __forceinline__ double dm(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double da(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double ds(double a, double b) { return __dsub_rn(a, b); }

// rotation matrix of the unit quaternion (w, x, y, z), row-major R[3*r + c]
__device__ void quat_rot(const double *q, double *R)
{
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = ds(1.0, dm(2.0, da(dm(y, y), dm(z, z))));
    R[1] = dm(2.0, ds(dm(x, y), dm(w, z)));
    R[2] = dm(2.0, da(dm(x, z), dm(w, y)));
    R[3] = dm(2.0, da(dm(x, y), dm(w, z)));
    R[4] = ds(1.0, dm(2.0, da(dm(x, x), dm(z, z))));
    R[5] = dm(2.0, ds(dm(y, z), dm(w, x)));
    R[6] = dm(2.0, ds(dm(x, z), dm(w, y)));
    R[7] = dm(2.0, da(dm(y, z), dm(w, x)));
    R[8] = ds(1.0, dm(2.0, da(dm(x, x), dm(y, y))));
}

__device__ __forceinline__ int wrapi(int a, int n)
{
    int r = a % n;
    return r < 0 ? r + n : r;
}

// One block per candidate (grid-stride): raster the bounding box.
__global__ void raster_kernel(PatternArgs A)
{
    const int n_ax[3] = {A.nx, A.ny, A.nz};
    const int bc[3] = {A.bcx, A.bcy, A.bcz};
    for (long long n = blockIdx.x; n < A.n_incl; n += gridDim.x) {
        const double *inc = A.incl + 10 * n;
        double R[9];
        quat_rot(inc + 6, R);
        double rmax = inc[3];
        if (inc[4] > rmax) rmax = inc[4];
        if (inc[5] > rmax) rmax = inc[5];
        int lo[3], hi[3];
        for (int ax = 0; ax < 3; ++ax) {
            lo[ax] = (int)ceil(__ddiv_rn(ds(inc[ax], rmax), A.h[ax]));
            hi[ax] = (int)floor(__ddiv_rn(da(inc[ax], rmax), A.h[ax]));
            if (bc[ax] == kOpen) {
                if (lo[ax] < 0) lo[ax] = 0;
                if (hi[ax] > n_ax[ax] - 1) hi[ax] = n_ax[ax] - 1;
            } else if (hi[ax] - lo[ax] + 1 > n_ax[ax]) {
                lo[ax] = 0;
                hi[ax] = n_ax[ax] - 1;
            }
        }
        const long long ex = hi[0] - lo[0] + 1, ey = hi[1] - lo[1] + 1, ez = hi[2] - lo[2] + 1;
        if (ex <= 0 || ey <= 0 || ez <= 0) continue;
        const long long tot = ex * ey * ez;
        for (long long e = threadIdx.x; e < tot; e += blockDim.x) {
            const int ii = lo[0] + (int)(e % ex);
            const int jj = lo[1] + (int)((e / ex) % ey);
            const int kk = lo[2] + (int)(e / (ex * ey));
            const int c[3] = {wrapi(ii, A.nx), wrapi(jj, A.ny), wrapi(kk, A.nz)};
            double d[3];
            for (int ax = 0; ax < 3; ++ax) {
                d[ax] = ds(dm((double)c[ax], A.h[ax]), inc[ax]);
                if (bc[ax] == kPeriodic) {
                    const double L = dm((double)n_ax[ax], A.h[ax]);
                    d[ax] = ds(d[ax], dm(L, floor(da(__ddiv_rn(d[ax], L), 0.5))));
                }
            }
            double q = 0.0;
            for (int a = 0; a < 3; ++a) {
                const double eb = da(da(dm(R[a], d[0]), dm(R[3 + a], d[1])), dm(R[6 + a], d[2]));
                const double s = __ddiv_rn(eb, inc[3 + a]);
                q = da(q, dm(s, s));
            }
            if (q <= 1.0) {
                const long long m = (long long)c[0] + (long long)A.nx * ((long long)c[1] + (long long)A.ny * c[2]);
                atomicMin(A.first + m, (int)n);
            }
        }
    }
}

__global__ void histogram_kernel(const int *first, long long N, long long n_incl, unsigned long long *counts)
{
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < N; m += (long long)gridDim.x * blockDim.x) {
        int f = first[m];
        if (f >= 0 && f < n_incl) atomicAdd(counts + f, 1ull);
    }
}

// Sequential rule: candidate n is processed while fewer than `target` sites are marked.
__global__ void select_kernel(const unsigned long long *counts, long long n_incl, long long target, long long *result)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    long long marked = 0, used = 0;
    for (long long n = 0; n < n_incl; ++n) {
        if (target > 0 && marked >= target) break;
        marked += (long long)counts[n];
        used = n + 1;
    }
    result[0] = used;
    result[1] = marked;
}

__global__ void alpha_kernel(const int *first, long long N, const long long *result, float ain, float aout, float *alpha)
{
    const long long used = result[0];
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < N; m += (long long)gridDim.x * blockDim.x)
        alpha[m] = ((long long)first[m] < used) ? ain : aout;
}

cudaError_t launch_pattern(const DevGrid &g, double hx, double hy, double hz, const double *d_incl, long long n_incl,
                           long long target, float alpha_in, float alpha_out, float *alpha, int *first,
                           unsigned long long *counts, long long *result, cudaStream_t s)
{
    cudaError_t e;
    if ((e = cudaMemsetAsync(first, 0x7F, sizeof(int) * (size_t)g.N, s)) != cudaSuccess) return e;
    if (n_incl > 0 && (e = cudaMemsetAsync(counts, 0, sizeof(unsigned long long) * (size_t)n_incl, s)) != cudaSuccess)
        return e;
    PatternArgs A;
    A.nx = g.nx;
    A.ny = g.ny;
    A.nz = g.nz;
    A.bcx = g.bcx;
    A.bcy = g.bcy;
    A.bcz = g.bcz;
    A.h[0] = hx;
    A.h[1] = hy;
    A.h[2] = hz;
    A.incl = d_incl;
    A.n_incl = n_incl;
    A.first = first;
    if (n_incl > 0) {
        int nb = (int)(n_incl < 65535 ? n_incl : 65535);
        raster_kernel<<<nb, 256, 0, s>>>(A);
        long long hb = (g.N + 255) / 256;
        if (hb > 4096) hb = 4096;
        histogram_kernel<<<(int)hb, 256, 0, s>>>(first, g.N, n_incl, counts);
    }
    select_kernel<<<1, 32, 0, s>>>(counts, n_incl, target, result);
    long long ab = (g.N + 255) / 256;
    if (ab > 8192) ab = 8192;
    alpha_kernel<<<(int)ab, 256, 0, s>>>(first, g.N, result, alpha_in, alpha_out, alpha);
    return cudaGetLastError();
}

}  // namespace tdgl
