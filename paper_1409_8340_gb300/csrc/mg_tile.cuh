// Per-site and per-line pieces of the multigrid Poisson solver (Sec. 3.2, the
// exact discrete solve of Lap mu = F), shared by the per-instance kernels and
// the batched persistent kernel.  CG = true: loads of arrays written earlier in
// the same launch go through L2 only.
#pragma once
#include "tdgl_internal.cuh"

namespace tdgl {

constexpr int kR = 16;   // consecutive outputs per thread in a line convolution

// neighbour index along an axis with periodic wrap or Neumann mirror
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

// index of the extended (periodic or mirrored) x line
__device__ __forceinline__ int ext_idx(int j, int nx, int P, int open)
{
    while (j < 0) j += P;
    while (j >= P) j -= P;
    if (open && j > nx - 1) j = P - j;
    return j;
}

__device__ __forceinline__ int pad(int j) { return j + (j >> 5); }

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

// Convolve one padded smem line with the kernel Gs: outputs i0 .. i0+kR-1.
// out[r] = sum_{k=kmin}^{kmax} Gs[k - kmin] * line(ext(i0 + r + k))
__device__ __forceinline__ void line_convolve(const float *__restrict__ line, const float *__restrict__ Gs, int kmin,
                                              int kmax, int i0, int nx, int P, int open, float out[kR])
{
    float w[kR];
#pragma unroll
    for (int r = 0; r < kR; ++r) {
        w[r] = line[pad(ext_idx(i0 + r + kmin, nx, P, open))];
        out[r] = 0.f;
    }
    for (int k = kmin; k <= kmax; ++k) {
        const float g = Gs[k - kmin];
#pragma unroll
        for (int r = 0; r < kR; ++r) out[r] = fmaf(g, w[r], out[r]);
#pragma unroll
        for (int r = 0; r < kR - 1; ++r) w[r] = w[r + 1];
        w[kR - 1] = line[pad(ext_idx(i0 + kR + k, nx, P, open))];
    }
}

// Shared memory (floats) of one zebra line-smoothing tile of lpb lines.
__host__ __device__ inline long long line_tile_floats(int lpb, int nx, int nG)
{
    return (long long)lpb * (nx + nx / 32 + 2) + nG;
}

// Zebra x-line Gauss-Seidel, lines blk*lpb .. blk*lpb+lpb-1 of colour `color`:
// each line solves T u_line = -(F - fsub) + cy (u_{j+1} + u_{j-1}) + cz (u_{k+1} + u_{k-1})
// exactly by convolution with the line Green's function.  Thread tid of nthr
// loads positions r, r + tpl, ... of line q = tid / tpl and computes kR outputs.
template <bool CG>
__device__ __forceinline__ void line_smooth_lines(const MGLevel &L, int bcx, int bcy, int bcz, int color,
                                                  long long nlines, int lpb, int tpl, float fsub, long long blk,
                                                  int tid, int nthr, float *sm)
{
    const int nx = L.nx, ny = L.ny, nz = L.nz;
    const int lstride = pad(nx) + 1;
    float *Gs = sm + lpb * lstride;
    const int nG = L.kmax - L.kmin + 1;
    __syncthreads();   // shared memory may still be read by a previous tile
    for (int t = tid; t < nG; t += nthr) Gs[t] = L.G[t];
    const long long plane = (long long)nx * ny;
    const int q = tid / tpl;
    const int r = tid - q * tpl;
    const long long line = blk * lpb + q;
    const bool active = (q < lpb) && (line < nlines);
    long long base = 0;
    if (active) {
        int j, k;
        line_jk(line, color, ny, nz, j, k);
        base = (long long)nx * j + plane * k;
        const float *rr = L.r + base;
        const float *up = nullptr, *um = nullptr, *zp = nullptr, *zm = nullptr;
        if (ny >= 2) {
            up = L.u + (long long)nx * nb_idx(j, 1, ny, bcy) + plane * k;
            um = L.u + (long long)nx * nb_idx(j, -1, ny, bcy) + plane * k;
        }
        if (nz >= 2) {
            zp = L.u + (long long)nx * j + plane * nb_idx(k, 1, nz, bcz);
            zm = L.u + (long long)nx * j + plane * nb_idx(k, -1, nz, bcz);
        }
        float *row = sm + q * lstride;
#pragma unroll 8
        for (int i = r; i < nx; i += tpl) {
            float v = -(ldx<CG>(rr + i) - fsub);
            if (up) v += L.cy * (ldx<CG>(up + i) + ldx<CG>(um + i));
            if (zp) v += L.cz * (ldx<CG>(zp + i) + ldx<CG>(zm + i));
            row[pad(i)] = v;
        }
    }
    __syncthreads();
    const int i0 = r * kR;
    if (active && i0 < nx) {
        float out[kR];
        line_convolve(sm + q * lstride, Gs, L.kmin, L.kmax, i0, nx, L.P, bcx == kOpen, out);
        float *dst = L.u + base;
#pragma unroll
        for (int rr2 = 0; rr2 < kR; ++rr2)
            if (i0 + rr2 < nx) dst[i0 + rr2] = out[rr2];
    }
}

// (Lap_h u)(i, j, k) on one level, Neumann mirror on open faces.
template <bool CG>
__device__ __forceinline__ float lap_at(const MGLevel &L, const float *u, int i, int j, int k, long long m, int bcx,
                                        int bcy, int bcz)
{
    const int nx = L.nx, ny = L.ny, nz = L.nz;
    const float u0 = ldx<CG>(u + m);
    const int ip = nb_idx(i, 1, nx, bcx), im = nb_idx(i, -1, nx, bcx);
    float lap = L.cx * (ldx<CG>(u + m - i + ip) + ldx<CG>(u + m - i + im) - 2.f * u0);
    if (ny >= 2) {
        const int jp = nb_idx(j, 1, ny, bcy), jm = nb_idx(j, -1, ny, bcy);
        lap += L.cy * (ldx<CG>(u + m + (long long)nx * (jp - j)) + ldx<CG>(u + m + (long long)nx * (jm - j)) - 2.f * u0);
    }
    if (nz >= 2) {
        const int kp = nb_idx(k, 1, nz, bcz), km = nb_idx(k, -1, nz, bcz);
        const long long pl = (long long)nx * ny;
        lap += L.cz * (ldx<CG>(u + m + pl * (kp - k)) + ldx<CG>(u + m + pl * (km - k)) - 2.f * u0);
    }
    return lap;
}

// t = F - L u at one site (level 0: F = f - fmean)
template <bool CG>
__device__ __forceinline__ float residual_at(const MGLevel &L, int bcx, int bcy, int bcz, float fsub, int i, int j,
                                             int k, long long m)
{
    return (ldx<CG>(L.r + m) - fsub) - lap_at<CG>(L, L.u, i, j, k, m, bcx, bcy, bcz);
}

// Full weighting in (y, z) of the fine residual t at coarse site (i, J, K).
template <bool CG>
__device__ __forceinline__ float restrict_at(const MGLevel &F, int bcy, int bcz, int i, int J, int K)
{
    const int nx = F.nx;
    float acc = 0.f;
    for (int dk = -1; dk <= 1; ++dk) {
        const float wk = (F.fz == 2) ? (dk == 0 ? 0.5f : 0.25f) : (dk == 0 ? 1.f : 0.f);
        if (wk == 0.f) continue;
        const int kf = (F.nz >= 2) ? nb_idx(F.fz * K, dk, F.nz, bcz) : 0;
        for (int dj = -1; dj <= 1; ++dj) {
            const float wj = (F.fy == 2) ? (dj == 0 ? 0.5f : 0.25f) : (dj == 0 ? 1.f : 0.f);
            if (wj == 0.f) continue;
            const int jf = nb_idx(F.fy * J, dj, F.ny, bcy);
            acc += wk * wj * ldx<CG>(F.t + (long long)nx * (jf + (long long)F.ny * kf) + i);
        }
    }
    return acc;
}

// Bilinear interpolation in (y, z) of the coarse correction at fine site (i, j, k).
template <bool CG>
__device__ __forceinline__ float prolong_at(const MGLevel &F, const MGLevel &C, int bcy, int bcz, int i, int j, int k)
{
    const int nx = F.nx;
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
    const float v00 = ldx<CG>(C.u + (long long)nx * j0 + cpl * k0 + i);
    const float v10 = ldx<CG>(C.u + (long long)nx * j1 + cpl * k0 + i);
    const float v01 = ldx<CG>(C.u + (long long)nx * j0 + cpl * k1 + i);
    const float v11 = ldx<CG>(C.u + (long long)nx * j1 + cpl * k1 + i);
    return (1.f - wk1) * ((1.f - wj1) * v00 + wj1 * v10) + wk1 * ((1.f - wj1) * v01 + wj1 * v11);
}

// Coarsest level, exact solve.  cw = [W (M x M) | V (M x M) | Gq (M x P)].
// Forward y-z transform: H[q][i] = sum_s W[q][s] * (-(r[s][i] - fsub)), element e = q nx + i.
template <bool CG>
__device__ __forceinline__ float coarse_fwd_at(const MGLevel &L, float fsub, long long e)
{
    const int nx = L.nx, M = L.M;
    const int q = (int)(e / nx), i = (int)(e - (long long)q * nx);
    float acc = 0.f;
    for (int s = 0; s < M; ++s) acc += L.cw[(size_t)q * M + s] * (-(ldx<CG>(L.r + (size_t)s * nx + i) - fsub));
    return acc;
}

// Inverse transform: u[s][i] = sum_q V[s][q] X[q][i] (X in t), element e = s nx + i.
template <bool CG>
__device__ __forceinline__ float coarse_inv_at(const MGLevel &L, long long e)
{
    const int nx = L.nx, M = L.M;
    const float *V = L.cw + (size_t)M * M;
    const int s = (int)(e / nx), i = (int)(e - (long long)s * nx);
    float acc = 0.f;
    for (int q = 0; q < M; ++q) acc += V[(size_t)s * M + q] * ldx<CG>(L.t + (size_t)q * nx + i);
    return acc;
}

// Shared memory (floats) of one coarse mode-line convolution.
__host__ __device__ inline long long coarse_line_floats(int nx, int P) { return (long long)(nx + nx / 32 + 2) + P; }

// Mode line q: X[q][i] = sum_k Gq[q][k] H~[q][i + k] over one period, in place in t.
// The block reads the whole line before writing it (nx <= nthr * kR).
template <bool CG>
__device__ __forceinline__ void coarse_conv_line(const MGLevel &L, int bcx, int q, int tid, int nthr, float *sm)
{
    const int nx = L.nx, M = L.M, P = L.P;
    float *line = sm;
    float *Gs = sm + pad(nx) + 2;
    const float *Gq = L.cw + 2 * (size_t)M * M + (size_t)q * P;
    __syncthreads();   // shared memory may still be read by a previous tile
    for (int t = tid; t < nx; t += nthr) line[pad(t)] = ldx<CG>(L.t + (size_t)q * nx + t);
    for (int t = tid; t < P; t += nthr) Gs[t] = Gq[t];
    __syncthreads();
    const int i0 = tid * kR;
    if (i0 < nx) {
        float out[kR];
        line_convolve(line, Gs, 0, P - 1, i0, nx, P, bcx == kOpen, out);
#pragma unroll
        for (int r = 0; r < kR; ++r)
            if (i0 + r < nx) L.t[(size_t)q * nx + i0 + r] = out[r];
    }
}

}  // namespace tdgl
