// Per-site and per-line pieces of the multigrid Poisson solver (Sec. 3.2, the
// exact discrete solve of Lap mu = F), shared by the per-instance kernels and
// the batched persistent kernel.  CG = true: loads of arrays written earlier in
// the same launch go through L2 only.
#pragma once
#include "tdgl_internal.cuh"

namespace tdgl {

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
__device__ __forceinline__ void line_jk(long long q64, int c, int ny, int nz, int &j, int &k)
{
    const unsigned int q = (unsigned int)q64;   // fewer than 2^31 lines per level
    if ((ny & 1) == 0) {
        const unsigned int half = (unsigned int)(ny >> 1);
        k = (int)(q / half);
        const int jj = (int)(q - (unsigned int)k * half);
        j = 2 * jj + ((c + k) & 1);
    } else {
        const unsigned int kp = q / (unsigned int)ny;
        const int rem = (int)(q - kp * (unsigned int)ny);
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

// Shape of a zebra line-smoothing tile.  Each line is split over tpl threads, each
// computing kLR = 8 consecutive outputs; lpb lines per block of nthr threads.  A
// line is staged in shared memory already extended (periodic wrap or Neumann
// mirror) by the kernel support: E[t] = v_ext(t + koff), t < lext, where koff is
// kmin rounded down to a multiple of 4 (the taps get kmin - koff leading zeros),
// so that the staged line and every 8-tap window sit on 16-byte boundaries.
// Shared layout: the ngp taps, then lpb lines lstride floats apart, each at the
// padded positions pad4(t) = t + 4 (t / 32), which spreads the 16-byte window
// loads of a quarter warp over all banks.
constexpr int kLR = 8;
struct LineShape {
    int tpl, lpb, koff, ngp, lext, lstride;
};
__host__ __device__ inline int pad4(int t) { return t + 4 * (t >> 5); }
__host__ __device__ inline LineShape line_shape(int nx, int kmin, int kmax, int nthr)
{
    LineShape s;
    s.tpl = (nx + kLR - 1) / kLR;
    s.lpb = nthr / s.tpl > 0 ? nthr / s.tpl : 1;
    s.koff = (kmin >= 0) ? kmin / 4 * 4 : -((-kmin + 3) / 4 * 4);
    s.ngp = (kmax - s.koff + 1 + kLR - 1) / kLR * kLR;
    s.lext = s.tpl * kLR + s.ngp + kLR;
    s.lstride = (pad4(s.lext - 1) + 1 + 3) / 4 * 4;
    return s;
}
__host__ __device__ inline long long line_tile_floats(const LineShape &s) { return s.ngp + (long long)s.lpb * s.lstride; }

// Zebra x-line Gauss-Seidel, lines blk*lpb .. blk*lpb+lpb-1 of colour `color`:
// each line solves T u_line = -(F - fsub) + cy (u_{j+1} + u_{j-1}) + cz (u_{k+1} + u_{k-1})
// exactly by convolution with the line Green's function G_k, k = kmin..kmax:
// u_i = sum_k G_k v_ext(i + k), v_ext the periodic or mirrored extension of the line.
// SUM: also this thread's part of the weighted sum of the new values (trapezoid weights 1/2
// per open face, the zero mode of Sec. 3.3.2) in *sw and of their x-face difference (open x:
// values at i = 0 minus those at i = nx - 1) in *sv.
template <bool CG, bool SUM = false>
__device__ __forceinline__ void line_smooth_lines(const MGLevel &L, const LineShape &sh, int bcx, int bcy, int bcz,
                                                  int color, long long nlines, float fsub, long long blk, int tid,
                                                  int nthr, float *sm, float *sw = nullptr, float *sv = nullptr)
{
    const int nx = L.nx, ny = L.ny, nz = L.nz;
    const int nG = L.kmax - L.kmin + 1, lead = L.kmin - sh.koff;
    float *Gs = sm;
    __syncthreads();   // shared memory may still be read by a previous tile
    for (int t = tid; t < sh.ngp; t += nthr) Gs[t] = (t >= lead && t - lead < nG) ? L.G[t - lead] : 0.f;
    const int q = tid / sh.tpl;
    const int r = tid - q * sh.tpl;
    const long long line = blk * sh.lpb + q;
    const bool active = (q < sh.lpb) && (line < nlines);
    float *E = sm + sh.ngp + q * sh.lstride;
    const int off = -sh.koff;   // E position of x = 0, a multiple of 4
    const int i0 = r * kLR;
    const bool vec = (nx & 3) == 0 && i0 + kLR <= nx;   // rows start on 16-byte boundaries
    long long base = 0;
    if (active && i0 < nx) {
        int j, k;
        line_jk(line, color, ny, nz, j, k);
        const long long plane = (long long)nx * ny;
        base = (long long)nx * j + plane * k;
        const bool ya = ny >= 2, za = nz >= 2;
        const float *rr = L.r + base;
        const float *up = ya ? L.u + (long long)nx * nb_idx(j, 1, ny, bcy) + plane * k : rr;
        const float *um = ya ? L.u + (long long)nx * nb_idx(j, -1, ny, bcy) + plane * k : rr;
        const float *zp = za ? L.u + (long long)nx * j + plane * nb_idx(k, 1, nz, bcz) : rr;
        const float *zm = za ? L.u + (long long)nx * j + plane * nb_idx(k, -1, nz, bcz) : rr;
        float v[kLR];
        if (vec) {
#pragma unroll
            for (int h = 0; h < kLR; h += 4) {
                const float4 a = ldx<CG>(reinterpret_cast<const float4 *>(rr + i0 + h));
                const float4 yp = ldx<CG>(reinterpret_cast<const float4 *>(up + i0 + h));
                const float4 ym = ldx<CG>(reinterpret_cast<const float4 *>(um + i0 + h));
                const float4 kp = ldx<CG>(reinterpret_cast<const float4 *>(zp + i0 + h));
                const float4 km = ldx<CG>(reinterpret_cast<const float4 *>(zm + i0 + h));
                const float av[4] = {a.x, a.y, a.z, a.w}, ypv[4] = {yp.x, yp.y, yp.z, yp.w},
                            ymv[4] = {ym.x, ym.y, ym.z, ym.w}, kpv[4] = {kp.x, kp.y, kp.z, kp.w},
                            kmv[4] = {km.x, km.y, km.z, km.w};
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    float x = -(av[c] - fsub);
                    if (ya) x += L.cy * (ypv[c] + ymv[c]);
                    if (za) x += L.cz * (kpv[c] + kmv[c]);
                    v[h + c] = x;
                }
            }
#pragma unroll
            for (int h = 0; h < kLR; h += 4)
                *reinterpret_cast<float4 *>(E + pad4(off + i0 + h)) = make_float4(v[h], v[h + 1], v[h + 2], v[h + 3]);
        } else {
#pragma unroll
            for (int c = 0; c < kLR; ++c) {
                const int i = i0 + c;
                if (i < nx) {
                    float x = -(ldx<CG>(rr + i) - fsub);
                    if (ya) x += L.cy * (ldx<CG>(up + i) + ldx<CG>(um + i));
                    if (za) x += L.cz * (ldx<CG>(zp + i) + ldx<CG>(zm + i));
                    E[pad4(off + i)] = x;
                }
            }
        }
    }
    __syncthreads();
    if (active) {
        // extension outside the line: periodic wrap (P = nx) or Neumann mirror (P = 2(nx-1))
        for (int t = r; t < sh.lext; t += sh.tpl)
            if (t < off || t >= off + nx) E[pad4(t)] = E[pad4(ext_idx(t - off, nx, L.P, bcx == kOpen) + off)];
    }
    __syncthreads();
    if (active && i0 < nx) {
        // out[c] = sum_j Gs[j] E[i0 + j + c]: window of 16 staged values, 8 taps at a time
        float out[kLR], win[2 * kLR];
        {
            const float4 w0 = *reinterpret_cast<const float4 *>(E + pad4(i0));
            const float4 w1 = *reinterpret_cast<const float4 *>(E + pad4(i0 + 4));
            win[0] = w0.x, win[1] = w0.y, win[2] = w0.z, win[3] = w0.w;
            win[4] = w1.x, win[5] = w1.y, win[6] = w1.z, win[7] = w1.w;
        }
#pragma unroll
        for (int c = 0; c < kLR; ++c) out[c] = 0.f;
        for (int j0 = 0; j0 < sh.ngp; j0 += kLR) {
            const float4 w2 = *reinterpret_cast<const float4 *>(E + pad4(i0 + j0 + 8));
            const float4 w3 = *reinterpret_cast<const float4 *>(E + pad4(i0 + j0 + 12));
            win[8] = w2.x, win[9] = w2.y, win[10] = w2.z, win[11] = w2.w;
            win[12] = w3.x, win[13] = w3.y, win[14] = w3.z, win[15] = w3.w;
            const float4 g0 = *reinterpret_cast<const float4 *>(Gs + j0);
            const float4 g1 = *reinterpret_cast<const float4 *>(Gs + j0 + 4);
            const float g[kLR] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
#pragma unroll
            for (int t = 0; t < kLR; ++t) {
#pragma unroll
                for (int c = 0; c < kLR; ++c) out[c] = fmaf(g[t], win[c + t], out[c]);
            }
#pragma unroll
            for (int c = 0; c < kLR; ++c) win[c] = win[kLR + c];
        }
        float *dst = L.u + base + i0;
        if (vec) {
            reinterpret_cast<float4 *>(dst)[0] = make_float4(out[0], out[1], out[2], out[3]);
            reinterpret_cast<float4 *>(dst)[1] = make_float4(out[4], out[5], out[6], out[7]);
        } else {
#pragma unroll
            for (int c = 0; c < kLR; ++c)
                if (i0 + c < nx) dst[c] = out[c];
        }
        if constexpr (SUM) {
            const long long plane = (long long)nx * ny;
            const int k = (int)(base / plane), j = (int)((base - plane * k) / nx);
            const bool ox = bcx == kOpen, oy = bcy == kOpen, oz = bcz == kOpen && nz >= 2;
            const float wyz = ((oy && (j == 0 || j == ny - 1)) ? 0.5f : 1.f) * ((oz && (k == 0 || k == nz - 1)) ? 0.5f : 1.f);
            float acc = 0.f;
#pragma unroll
            for (int c = 0; c < kLR; ++c) {
                const int i = i0 + c;
                if (i < nx) acc += ((ox && (i == 0 || i == nx - 1)) ? 0.5f : 1.f) * out[c];
            }
            *sw += wyz * acc;
            if (ox) {
                if (i0 == 0) *sv += out[0];
                if (i0 <= nx - 1 && nx - 1 < i0 + kLR) {
#pragma unroll
                    for (int c = 0; c < kLR; ++c)
                        if (i0 + c == nx - 1) *sv -= out[c];
                }
            }
        }
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
// zero_color >= 0: the fine rows of that zebra colour hold a zero residual (the colour
// just solved exactly) and are not read
__device__ __forceinline__ float restrict_at(const MGLevel &F, int bcy, int bcz, int i, int J, int K,
                                             int zero_color = -1)
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
            if (zero_color >= 0 && ((jf + kf) & 1) == zero_color) continue;
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

// Four consecutive x sites i0..i0+3 (nx % 4 == 0, so rows start on 16-byte
// boundaries): the same per-site arithmetic as residual_at / restrict_at /
// prolong_at, with 16-byte loads.
template <bool CG>
__device__ __forceinline__ float4 ld4(const float *p)
{
    return ldx<CG>(reinterpret_cast<const float4 *>(p));
}

// t = F - L u at four x sites from values already loaded: the centre c, F (rr), the x
// neighbours xl (of i0) and xr (of i0 + 3), the rows above/below in y (yp, ym; ya: y
// active) and in z (zp, zm; za).  Shared by residual4_at and the fused residual-restriction.
__device__ __forceinline__ float4 residual4_core(const MGLevel &L, float fsub, float4 c, float4 rr, float xl, float xr,
                                                 bool ya, float4 yp, float4 ym, bool za, float4 zp, float4 zm)
{
    const float cv[4] = {c.x, c.y, c.z, c.w};
    const float fwd[4] = {c.y, c.z, c.w, xr};
    const float bwd[4] = {xl, c.x, c.y, c.z};
    float lap[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) lap[q] = L.cx * (fwd[q] + bwd[q] - 2.f * cv[q]);
    if (ya) {
        const float av[4] = {yp.x, yp.y, yp.z, yp.w}, bv[4] = {ym.x, ym.y, ym.z, ym.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) lap[q] += L.cy * (av[q] + bv[q] - 2.f * cv[q]);
    }
    if (za) {
        const float av[4] = {zp.x, zp.y, zp.z, zp.w}, bv[4] = {zm.x, zm.y, zm.z, zm.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) lap[q] += L.cz * (av[q] + bv[q] - 2.f * cv[q]);
    }
    return make_float4((rr.x - fsub) - lap[0], (rr.y - fsub) - lap[1], (rr.z - fsub) - lap[2], (rr.w - fsub) - lap[3]);
}

template <bool CG>
__device__ __forceinline__ float4 residual4_at(const MGLevel &L, int bcx, int bcy, int bcz, float fsub, int i0, int j,
                                               int k)
{
    const int nx = L.nx, ny = L.ny, nz = L.nz;
    const long long pl = (long long)nx * ny;
    const long long row = (long long)nx * j + pl * k;
    const float *u = L.u;
    const float4 c = ld4<CG>(u + row + i0);
    const float4 rr = ld4<CG>(L.r + row + i0);
    const float xl = ldx<CG>(u + row + nb_idx(i0, -1, nx, bcx));
    const float xr = ldx<CG>(u + row + nb_idx(i0 + 3, 1, nx, bcx));
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 yp = zero, ym = zero, zp = zero, zm = zero;
    if (ny >= 2) {
        const int jp = nb_idx(j, 1, ny, bcy), jm = nb_idx(j, -1, ny, bcy);
        yp = ld4<CG>(u + row + (long long)nx * (jp - j) + i0);
        ym = ld4<CG>(u + row + (long long)nx * (jm - j) + i0);
    }
    if (nz >= 2) {
        const int kp = nb_idx(k, 1, nz, bcz), km = nb_idx(k, -1, nz, bcz);
        zp = ld4<CG>(u + row + pl * (kp - k) + i0);
        zm = ld4<CG>(u + row + pl * (km - k) + i0);
    }
    return residual4_core(L, fsub, c, rr, xl, xr, ny >= 2, yp, ym, nz >= 2, zp, zm);
}

template <bool CG>
__device__ __forceinline__ float4 restrict4_at(const MGLevel &F, int bcy, int bcz, int i0, int J, int K,
                                               int zero_color = -1)
{
    const int nx = F.nx;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    const int nk = (F.fz == 2) ? 3 : 1, nj = (F.fy == 2) ? 3 : 1;
    for (int a = 0; a < nk; ++a) {
        const int dk = (nk == 3) ? a - 1 : 0;
        const float wk = (nk == 3) ? (dk == 0 ? 0.5f : 0.25f) : 1.f;
        const int kf = (F.nz >= 2) ? nb_idx(F.fz * K, dk, F.nz, bcz) : 0;
        for (int b = 0; b < nj; ++b) {
            const int dj = (nj == 3) ? b - 1 : 0;
            const float wj = (nj == 3) ? (dj == 0 ? 0.5f : 0.25f) : 1.f;
            const int jf = nb_idx(F.fy * J, dj, F.ny, bcy);
            if (zero_color >= 0 && ((jf + kf) & 1) == zero_color) continue;
            const float4 t = ld4<CG>(F.t + (long long)nx * (jf + (long long)F.ny * kf) + i0);
            acc.x += wk * wj * t.x;
            acc.y += wk * wj * t.y;
            acc.z += wk * wj * t.z;
            acc.w += wk * wj * t.w;
        }
    }
    return acc;
}

template <bool CG>
__device__ __forceinline__ float4 prolong4_at(const MGLevel &F, const MGLevel &C, int bcy, int bcz, int i0, int j, int k)
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
    const float4 a = ld4<CG>(C.u + (long long)nx * j0 + cpl * k0 + i0);
    const float4 b = ld4<CG>(C.u + (long long)nx * j1 + cpl * k0 + i0);
    const float4 c = ld4<CG>(C.u + (long long)nx * j0 + cpl * k1 + i0);
    const float4 d = ld4<CG>(C.u + (long long)nx * j1 + cpl * k1 + i0);
    const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w}, cv[4] = {c.x, c.y, c.z, c.w},
                dv[4] = {d.x, d.y, d.z, d.w};
    float o[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) o[q] = (1.f - wk1) * ((1.f - wj1) * av[q] + wj1 * bv[q]) + wk1 * ((1.f - wj1) * cv[q] + wj1 * dv[q]);
    return make_float4(o[0], o[1], o[2], o[3]);
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

// Coarse mode-line convolution: outputs per thread and shared memory (floats).
constexpr int kCR = 2;
__host__ __device__ inline long long coarse_line_floats(int nx, int P)
{
    const int ngp = (P + kCR - 1) / kCR * kCR;
    const int lext = (nx + kCR - 1) / kCR * kCR + ngp + kCR;
    return (long long)(lext + (lext >> 5) + 1) + ngp;
}

// Mode line q: X[q][i] = sum_k Gq[q][k] H~[q][i + k] over one period for i in
// [ibeg, iend) (ibeg a multiple of kCR), into X (in place in t when X is null: the block
// stages the whole line in shared memory before writing it).
template <bool CG>
__device__ __forceinline__ void coarse_conv_line(const MGLevel &L, int bcx, int q, int tid, int nthr, float *sm,
                                                 float *X = nullptr, int ibeg = 0, int iend = -1)
{
    const int nx = L.nx, M = L.M, P = L.P;
    const int ngp = (P + kCR - 1) / kCR * kCR;
    const int lext = (nx + kCR - 1) / kCR * kCR + ngp + kCR;
    float *E = sm;
    float *Gs = sm + lext + (lext >> 5) + 1;
    const float *Gq = L.cw + 2 * (size_t)M * M + (size_t)q * P;
    __syncthreads();   // shared memory may still be read by a previous tile
    for (int t = tid; t < nx; t += nthr) E[pad(t)] = ldx<CG>(L.t + (size_t)q * nx + t);
    for (int t = tid; t < ngp; t += nthr) Gs[t] = (t < P) ? Gq[t] : 0.f;
    __syncthreads();
    for (int t = nx + tid; t < lext; t += nthr) E[pad(t)] = E[pad(ext_idx(t, nx, P, bcx == kOpen))];
    __syncthreads();
    float *Xo = X ? X : L.t;
    if (iend < 0) iend = nx;
    for (int i0 = ibeg + tid * kCR; i0 < iend; i0 += nthr * kCR) {
        float out[kCR], win[2 * kCR];
#pragma unroll
        for (int c = 0; c < kCR; ++c) {
            win[c] = E[pad(i0 + c)];
            out[c] = 0.f;
        }
        for (int j0 = 0; j0 < ngp; j0 += kCR) {
#pragma unroll
            for (int c = 0; c < kCR; ++c) win[kCR + c] = E[pad(i0 + j0 + kCR + c)];
#pragma unroll
            for (int t = 0; t < kCR; ++t) {
#pragma unroll
                for (int c = 0; c < kCR; ++c) out[c] = fmaf(Gs[j0 + t], win[c + t], out[c]);
            }
#pragma unroll
            for (int c = 0; c < kCR; ++c) win[c] = win[kCR + c];
        }
#pragma unroll
        for (int c = 0; c < kCR; ++c)
            if (i0 + c < iend) Xo[(size_t)q * nx + i0 + c] = out[c];
    }
}

}  // namespace tdgl
