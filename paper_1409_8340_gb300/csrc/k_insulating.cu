// Insulating inclusions (arXiv:1409.8340, Sec. 3.4 (ii): no-current conditions
// across internal grid edges).  A link that touches an insulating site carries
// no current: it is removed from the psi stencil and its diagonal (tiled sweep,
// sweep_tile.cuh), from J_av and the observables (k_obs.cu), and from the
// Poisson operator and right-hand side; insulating sites hold psi = mu = 0.
//
// This file builds the per-site link bits and the connected components of the
// conducting sites (islands enclosed by insulators are components of their own; the
// constants of each component span the Poisson operator's null space), and solves
// the Poisson equation with the removed links.  That operator has variable
// coefficients, so the constant-coefficient multigrid becomes a preconditioner:
// conjugate gradients in the trapezoid-weighted inner product (in which the operator
// is symmetric), each iteration preconditioned by one symmetric V-cycle of the plain
// operator, the right-hand side and the result projected on every component; sums
// in FP64, bulk in FP32.
#include <float.h>

#include "tdgl_internal.cuh"

namespace tdgl {

namespace {

constexpr int kT = 256;

int red_grid(long long N)
{
    long long b = (N + kT * 8 - 1) / (kT * 8);
    if (b > 4096) b = 4096;
    if (b < 1) b = 1;
    return (int)b;
}

__device__ __forceinline__ void ijk_of(const DevGrid &g, long long m, int &i, int &j, int &k)
{
    i = (int)(m % g.nx);
    const long long t = m / g.nx;
    j = (int)(t % g.ny);
    k = (int)(t / g.ny);
}

__device__ __forceinline__ float face_w(int bc, int n, int idx)
{
    return (bc == kOpen && n >= 2 && (idx == 0 || idx == n - 1)) ? 0.5f : 1.0f;
}

// neighbour index one step sgn along axis ax (periodic wrap; callers only use it
// where the link exists)
__device__ __forceinline__ long long nbr(const DevGrid &g, long long m, int i, int j, int k, int ax, int sgn)
{
    const long long sz = (long long)g.nx * g.ny;
    if (ax == 0) return (sgn > 0) ? (i == g.nx - 1 ? m - (g.nx - 1) : m + 1) : (i == 0 ? m + (g.nx - 1) : m - 1);
    if (ax == 1)
        return (sgn > 0) ? (j == g.ny - 1 ? m - (long long)(g.ny - 1) * g.nx : m + g.nx)
                         : (j == 0 ? m + (long long)(g.ny - 1) * g.nx : m - g.nx);
    return (sgn > 0) ? (k == g.nz - 1 ? m - (long long)(g.nz - 1) * sz : m + sz)
                     : (k == 0 ? m + (long long)(g.nz - 1) * sz : m - sz);
}

// Block sum of v into blockred[bid]; the last block writes the total to *out and
// returns true (every other block false).
__device__ __forceinline__ bool finish_sum(DevCtl *ctl, double *blockred, double v, double *out)
{
    __shared__ double shd[32];
    __shared__ int flag;
    double s = block_sum(v, shd);
    if (threadIdx.x == 0) blockred[blockIdx.x] = s;
    if (!last_block(&ctl->ticket, gridDim.x, &flag)) return false;
    double t = 0.0;
    for (unsigned int q = threadIdx.x; q < gridDim.x; q += blockDim.x) t += ((volatile double *)blockred)[q];
    t = block_sum(t, shd);
    if (threadIdx.x == 0) {
        ctl->ticket = 0u;
        *out = t;
    }
    return true;
}

}  // namespace

// ---------------------------------------------------------------------------
// Link bits
// ---------------------------------------------------------------------------
__global__ void link_bits_kernel(DevGrid g, const uint8_t *__restrict__ ins, uint8_t *__restrict__ lk)
{
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < g.N; m += (long long)gridDim.x * blockDim.x) {
        int i, j, k;
        ijk_of(g, m, i, j, k);
        if (ins[m]) {
            lk[m] = (uint8_t)kLkIns;
            continue;
        }
        const int idx[3] = {i, j, k}, n[3] = {g.nx, g.ny, g.nz}, bc[3] = {g.bcx, g.bcy, g.bcz};
        unsigned bits = 0;
        for (int ax = 0; ax < 3; ++ax) {
            if (n[ax] < 2) continue;
            for (int sgn = 1; sgn >= -1; sgn -= 2) {
                const bool inside = bc[ax] == kPeriodic || (sgn > 0 ? idx[ax] < n[ax] - 1 : idx[ax] > 0);
                if (inside && !ins[nbr(g, m, i, j, k, ax, sgn)]) bits |= (sgn > 0 ? 1u : 2u) << (2 * ax);
            }
        }
        lk[m] = (uint8_t)bits;
    }
}

cudaError_t launch_link_bits(const DevGrid &g, const uint8_t *ins, uint8_t *lk, cudaStream_t s)
{
    link_bits_kernel<<<red_grid(g.N) * 8 > 8192 ? 8192 : red_grid(g.N) * 8, kT, 0, s>>>(g, ins, lk);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Connected components of the conducting sites: labels start as the site index
// and drop to the smallest label reachable; each pass takes the minimum over the
// present links, hooks the old representative to it, then follows labels to
// their representatives (pointer jumping).
// ---------------------------------------------------------------------------
__global__ void cc_init_kernel(DevGrid g, long long *lab)
{
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < g.N; m += (long long)gridDim.x * blockDim.x)
        lab[m] = (g.lk[m] & kLkIns) ? -1 : m;
}

__global__ void cc_hook_kernel(DevGrid g, long long *lab, int *changed)
{
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < g.N; m += (long long)gridDim.x * blockDim.x) {
        const unsigned l = g.lk[m];
        if (l & kLkIns) continue;
        int i, j, k;
        ijk_of(g, m, i, j, k);
        const long long cur = lab[m];
        long long best = cur;
        for (int ax = 0; ax < 3; ++ax)
            for (int sgn = 1; sgn >= -1; sgn -= 2) {
                const unsigned bit = (sgn > 0 ? 1u : 2u) << (2 * ax);
                if (l & bit) {
                    const long long v = lab[nbr(g, m, i, j, k, ax, sgn)];
                    best = v < best ? v : best;
                }
            }
        if (best < cur) {
            atomicMin(lab + cur, best);
            atomicMin(lab + m, best);
            *changed = 1;
        }
    }
}

__global__ void cc_jump_kernel(DevGrid g, long long *lab)
{
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < g.N; m += (long long)gridDim.x * blockDim.x) {
        long long v = lab[m];
        if (v < 0) continue;
        for (int t = 0; t < 8; ++t) {
            const long long w = lab[v];
            if (w == v) break;
            v = w;
        }
        lab[m] = v;
    }
}

__global__ void cc_count_kernel(DevGrid g, const long long *lab, DevCtl *ctl, double *blockred)
{
    double roots = 0.0, cond = 0.0;
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < g.N; m += (long long)gridDim.x * blockDim.x) {
        if (lab[m] < 0) continue;
        cond += 1.0;
        if (lab[m] == m) roots += 1.0;
    }
    __shared__ double shd[32];
    __shared__ int flag;
    const double a = block_sum(roots, shd), b = block_sum(cond, shd);
    if (threadIdx.x == 0) {
        blockred[2 * blockIdx.x] = a;
        blockred[2 * blockIdx.x + 1] = b;
    }
    if (!last_block(&ctl->ticket, gridDim.x, &flag)) return;
    double ta = 0.0, tb = 0.0;
    for (unsigned int q = threadIdx.x; q < gridDim.x; q += blockDim.x) {
        ta += ((volatile double *)blockred)[2 * q];
        tb += ((volatile double *)blockred)[2 * q + 1];
    }
    ta = block_sum(ta, shd);
    tb = block_sum(tb, shd);
    if (threadIdx.x == 0) {
        ctl->ticket = 0u;
        ctl->sums[4] = ta;
        ctl->sums[5] = tb;
    }
}

// roots' sizes (one atomic per run of equal roots in a warp)
__global__ void cc_size_kernel(DevGrid g, const long long *lab, int *cnt)
{
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long base = warp * 32; base < g.N; base += nwarps * 32) {
        const long long m = base + lane;
        const long long r = (m < g.N) ? lab[m] : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, r);
        if (r >= 0 && lane == __ffs(peers) - 1) atomicAdd(cnt + r, __popc(peers));
    }
}

// the largest size over roots, then the smallest root of that size (the main component)
__global__ void cc_max_kernel(DevGrid g, const long long *lab, const int *cnt, unsigned long long *mx)
{
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < g.N; m += (long long)gridDim.x * blockDim.x)
        if (lab[m] == m) atomicMax(mx, (unsigned long long)cnt[m]);
}

__global__ void cc_main_kernel(DevGrid g, const long long *lab, const int *cnt, const unsigned long long *mx,
                               unsigned long long *main_root)
{
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < g.N; m += (long long)gridDim.x * blockDim.x)
        if (lab[m] == m && (unsigned long long)cnt[m] == *mx) atomicMin(main_root, (unsigned long long)m);
}

// compact ids: 0 for the main root, 1, 2, ... for the other roots (in no particular order)
__global__ void cc_id_kernel(DevGrid g, const long long *lab, int *cnt, const unsigned long long *main_root,
                             unsigned int *counter)
{
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < g.N; m += (long long)gridDim.x * blockDim.x)
        if (lab[m] == m) cnt[m] = ((unsigned long long)m == *main_root) ? 0 : 1 + (int)atomicAdd(counter, 1u);
}

__global__ void cc_comp_kernel(DevGrid g, const long long *lab, const int *cnt, int *comp)
{
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < g.N; m += (long long)gridDim.x * blockDim.x)
        comp[m] = lab[m] < 0 ? -1 : cnt[lab[m]];
}

// sum of w over the main component (and its x-face sites) into sums[4..6]; per island into isl_w
__global__ void comp_weights_kernel(DevGrid g, const int *comp, DevCtl *ctl, double *blockred, double *isl_w)
{
    double ws = 0.0, f0 = 0.0, f1 = 0.0;
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < g.N; m += (long long)gridDim.x * blockDim.x) {
        const int c = comp[m];
        if (c < 0) continue;
        int i, j, k;
        ijk_of(g, m, i, j, k);
        const double w = (double)(face_w(g.bcx, g.nx, i) * face_w(g.bcy, g.ny, j) * face_w(g.bcz, g.nz, k));
        if (c > 0) {
            atomicAdd(isl_w + (c - 1), w);
            continue;
        }
        ws += w;
        if (i == 0) f0 += 1.0;
        if (i == g.nx - 1) f1 += 1.0;
    }
    __shared__ double shd[32];
    __shared__ int flag;
    const double v[3] = {ws, f0, f1};
    for (int q = 0; q < 3; ++q) {
        const double t = block_sum(v[q], shd);
        if (threadIdx.x == 0) blockred[3 * blockIdx.x + q] = t;
    }
    if (!last_block(&ctl->ticket, gridDim.x, &flag)) return;
    for (int q = 0; q < 3; ++q) {
        double t = 0.0;
        for (unsigned int b = threadIdx.x; b < gridDim.x; b += blockDim.x) t += ((volatile double *)blockred)[3 * b + q];
        t = block_sum(t, shd);
        if (threadIdx.x == 0) ctl->sums[4 + q] = t;
    }
    if (threadIdx.x == 0) ctl->ticket = 0u;
}

int build_components(const DevGrid &g, InsPoisson &ip, DevCtl *ctl, double *blockred, cudaStream_t s)
{
    const int nb = red_grid(g.N) * 8 > 8192 ? 8192 : red_grid(g.N) * 8;
    long long *lab = reinterpret_cast<long long *>(ip.r);   // r and z: 8 bytes per site
    int *cnt = reinterpret_cast<int *>(ip.p);
    int *changed = reinterpret_cast<int *>(&ctl->sums[6]);
    unsigned long long *mx = reinterpret_cast<unsigned long long *>(&ctl->sums[5]);
    unsigned long long *main_root = reinterpret_cast<unsigned long long *>(&ctl->sums[6]);
    unsigned int *counter = reinterpret_cast<unsigned int *>(&ctl->sums[7]);
    cc_init_kernel<<<nb, kT, 0, s>>>(g, lab);
    if (cudaGetLastError() != cudaSuccess) return TDGL_ERR_CUDA;
    // at most a few thousand passes: the labels fall along every path each pass and
    // pointer jumping shortens the chains; an unfinished search is an error
    bool done = false;
    for (int pass = 0; pass < 4096 && !done; ++pass) {
        if (cudaMemsetAsync(changed, 0, sizeof(int), s) != cudaSuccess) return TDGL_ERR_CUDA;
        cc_hook_kernel<<<nb, kT, 0, s>>>(g, lab, changed);
        cc_jump_kernel<<<nb, kT, 0, s>>>(g, lab);
        int h = 0;
        if (cudaMemcpyAsync(&h, changed, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return TDGL_ERR_CUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return TDGL_ERR_CUDA;
        done = (h == 0);
    }
    if (!done) return TDGL_ERR_NOT_CONVERGED;
    cc_count_kernel<<<red_grid(g.N), kT, 0, s>>>(g, lab, ctl, blockred);
    double v[2];
    if (cudaMemcpyAsync(v, &ctl->sums[4], sizeof(v), cudaMemcpyDeviceToHost, s) != cudaSuccess) return TDGL_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return TDGL_ERR_CUDA;
    const long long ncomp = (long long)v[0], ncond = (long long)v[1];
    if (ncond < 1) return TDGL_ERR_INVALID_ARG;
    if (ncomp - 1 > kMaxIslands) return TDGL_ERR_INVALID_ARG;
    ip.n_isl = (int)(ncomp - 1);
    if (cudaMemsetAsync(cnt, 0, 4 * (size_t)g.N, s) != cudaSuccess) return TDGL_ERR_CUDA;
    if (cudaMemsetAsync(mx, 0, 8, s) != cudaSuccess) return TDGL_ERR_CUDA;
    if (cudaMemsetAsync(main_root, 0xFF, 8, s) != cudaSuccess) return TDGL_ERR_CUDA;
    if (cudaMemsetAsync(counter, 0, 4, s) != cudaSuccess) return TDGL_ERR_CUDA;
    cc_size_kernel<<<nb, kT, 0, s>>>(g, lab, cnt);
    cc_max_kernel<<<nb, kT, 0, s>>>(g, lab, cnt, mx);
    cc_main_kernel<<<nb, kT, 0, s>>>(g, lab, cnt, mx, main_root);
    cc_id_kernel<<<nb, kT, 0, s>>>(g, lab, cnt, main_root, counter);
    cc_comp_kernel<<<nb, kT, 0, s>>>(g, lab, cnt, ip.comp);
    if (cudaMemsetAsync(ip.isl_w, 0, 8 * (size_t)kMaxIslands, s) != cudaSuccess) return TDGL_ERR_CUDA;
    comp_weights_kernel<<<red_grid(g.N), kT, 0, s>>>(g, ip.comp, ctl, blockred, ip.isl_w);
    if (cudaGetLastError() != cudaSuccess) return TDGL_ERR_CUDA;
    double w[3];
    if (cudaMemcpyAsync(w, &ctl->sums[4], sizeof(w), cudaMemcpyDeviceToHost, s) != cudaSuccess) return TDGL_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return TDGL_ERR_CUDA;
    ip.wsum_c = w[0];
    ip.n_face0 = w[1];
    ip.n_face1 = w[2];
    return TDGL_OK;
}

// ---------------------------------------------------------------------------
// Poisson operator with removed links: (A u)_m = sum_a c_a [b+ (u+ - u) + b- (u- - u)],
// the ghost doubling the inner link on an open face; rows of insulating sites 0.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float masked_lap(const DevGrid &g, const float *__restrict__ u, long long m, int i, int j,
                                            int k, unsigned l)
{
    const float um = u[m];
    const int idx[3] = {i, j, k}, n[3] = {g.nx, g.ny, g.nz}, bc[3] = {g.bcx, g.bcy, g.bcz};
    const float c[3] = {g.cx, g.cy, g.cz};
    float acc = 0.f;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        if (n[ax] < 2) continue;
        float vp = (l & (1u << (2 * ax))) ? u[nbr(g, m, i, j, k, ax, 1)] - um : 0.f;
        float vm = (l & (2u << (2 * ax))) ? u[nbr(g, m, i, j, k, ax, -1)] - um : 0.f;
        if (bc[ax] == kOpen) {
            if (idx[ax] == 0) vm = vp;
            if (idx[ax] == n[ax] - 1) vp = vm;
        }
        acc += c[ax] * (vp + vm);
    }
    return acc;
}

struct InsArgs {
    DevGrid g;
    DevCtl *ctl;
    double *blockred;
    float *mu, *f, *r, *z, *p, *q;
    const int *comp;
    const double *isl_w;
    double *isl_acc;
    double wsum_c;
    int islands;               // 0: every conducting site is in the main component
    int n_isl;
};

// After a component sum: the last block turns each island's sum into its weighted mean
// (isl_acc, read by the shift that follows), the other blocks' atomics all done.
__device__ __forceinline__ void island_means(const InsArgs &a)
{
    for (int c = threadIdx.x; c < a.n_isl; c += blockDim.x)
        a.isl_acc[c] = ((volatile double *)a.isl_acc)[c] / a.isl_w[c];
}

// Rows (j, k) of the grid spread over the blocks, sites of a row over the threads:
// (i, j, k) and the face weights without per-site division.
template <class F>
__device__ __forceinline__ void for_sites(const DevGrid &g, F &&fn)
{
    const int rows = g.ny * g.nz;
    for (int row = blockIdx.x; row < rows; row += gridDim.x) {
        const int j = row % g.ny, k = row / g.ny;
        const float wyz = face_w(g.bcy, g.ny, j) * face_w(g.bcz, g.nz, k);
        const long long base = (long long)row * g.nx;
        for (int i = threadIdx.x; i < g.nx; i += blockDim.x) fn(base + i, i, j, k, wyz * face_w(g.bcx, g.nx, i));
    }
}

__device__ __forceinline__ int comp_of(const InsArgs &a, long long m)
{
    if (a.islands) return a.comp[m];
    return (a.g.lk[m] & kLkIns) ? -1 : 0;
}

// Component sums of w v: the main component's by blocks into sums[slot], each
// island's by atomics into isl_acc (cleared before the launch).
__global__ void ins_csum_kernel(InsArgs a, const float *v, int slot)
{
    float acc = 0.f;   // FP32 per thread, FP64 over the threads and blocks
    for_sites(a.g, [&](long long m, int, int, int, float w) {
        const int c = comp_of(a, m);
        if (c == 0) acc += w * v[m];
        else if (c > 0) atomicAdd(a.isl_acc + (c - 1), (double)(w * v[m]));
    });
    if (finish_sum(a.ctl, a.blockred, (double)acc, &a.ctl->sums[slot]) && a.islands) island_means(a);
}

// v -= its component's weighted mean (the islands' from island_means), 0 on insulating
// sites.  fmax: also ctl->fmax = max|v| and ctl->fmean = 0 (the level-0 multigrid kernels
// subtract ctl->fmean, which the preconditioner must not).
__global__ void ins_cshift_kernel(InsArgs a, float *v, int mslot, int fmax)
{
    const float cm = (float)(a.ctl->sums[mslot] / a.wsum_c);
    float mx = 0.f;
    for_sites(a.g, [&](long long m, int, int, int, float) {
        const int c = comp_of(a, m);
        if (c < 0) {
            v[m] = 0.f;
            return;
        }
        const float x = v[m] - (c == 0 ? cm : (float)a.isl_acc[c - 1]);
        v[m] = x;
        mx = fmaxf(mx, fabsf(x));
    });
    if (!fmax) return;
    __shared__ float shf[32];
    __shared__ int flag;
    const float bm = block_max(mx, shf);
    if (threadIdx.x == 0) a.blockred[blockIdx.x] = (double)bm;
    if (!last_block(&a.ctl->ticket, gridDim.x, &flag)) return;
    double t = 0.0;
    for (unsigned int q = threadIdx.x; q < gridDim.x; q += blockDim.x) {
        const double w = ((volatile double *)a.blockred)[q];
        t = w > t ? w : t;
    }
    const float tm = block_max((float)t, shf);
    if (threadIdx.x == 0) {
        a.ctl->ticket = 0u;
        a.ctl->fmax = (double)tm;
        a.ctl->fmean = 0.0;
    }
}

// ---------------------------------------------------------------------------
// The same passes four sites at a time (nx a multiple of 4, no islands): 16-byte loads
// of the site values and of the link bits, FP32 partial sums per thread.
// ---------------------------------------------------------------------------
template <class F>
__device__ __forceinline__ void for_quads(const DevGrid &g, F &&fn)
{
    const long long nq = g.N >> 2;
    const int qrow = g.nx >> 2;
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= nq) return;
    // the quad's x index qi, row j and plane k, divided out once and then advanced by the
    // stride's own (dq, dj, dk) with carries: no 64-bit division per quad
    const long long row0 = t / qrow, srow = stride / qrow;
    int qi = (int)(t - row0 * qrow), j = (int)(row0 % g.ny), k = (int)(row0 / g.ny);
    const int dq = (int)(stride - srow * qrow), dj = (int)(srow % g.ny), dk = (int)(srow / g.ny);
    for (; t < nq; t += stride) {
        fn(((long long)k * g.ny + j) * g.nx + 4 * qi, 4 * qi, j, k, face_w(g.bcy, g.ny, j) * face_w(g.bcz, g.nz, k));
        qi += dq;
        j += dj;
        k += dk;
        if (qi >= qrow) {
            qi -= qrow;
            ++j;
        }
        if (j >= g.ny) {
            j -= g.ny;
            ++k;
        }
    }
}

__device__ __forceinline__ float4 ld4f(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void st4f(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }

// masked_lap of the four sites m .. m+3 (i0 = i of site m)
__device__ __forceinline__ float4 masked_lap4(const DevGrid &g, const float *__restrict__ u, long long m, int i0, int j,
                                              int k, uchar4 l4)
{
    const float4 c4 = ld4f(u + m);
    const float c[4] = {c4.x, c4.y, c4.z, c4.w};
    const unsigned l[4] = {l4.x, l4.y, l4.z, l4.w};
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    // x: the quad's own values and one site beyond each end (wrapped; used only where the link exists)
    const float xm = u[i0 == 0 ? m + g.nx - 1 : m - 1];
    const float xp = u[i0 + 4 == g.nx ? m + 4 - g.nx : m + 4];
    const float xs[6] = {xm, c[0], c[1], c[2], c[3], xp};
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        float vp = (l[s] & kLkXp) ? xs[s + 2] - c[s] : 0.f;
        float vm = (l[s] & kLkXm) ? xs[s] - c[s] : 0.f;
        if (g.bcx == kOpen) {
            if (i0 + s == 0) vm = vp;
            if (i0 + s == g.nx - 1) vp = vm;
        }
        acc[s] = g.cx * (vp + vm);
    }
    // y and z: rows at the (wrapped) neighbour indices, whole quads
    const int n[2] = {g.ny, g.nz}, bc[2] = {g.bcy, g.bcz}, idx[2] = {j, k};
    const long long st[2] = {(long long)g.nx, (long long)g.nx * g.ny};
    const float cc[2] = {g.cy, g.cz};
    const unsigned bp[2] = {kLkYp, kLkZp}, bm[2] = {kLkYm, kLkZm};
#pragma unroll
    for (int ax = 0; ax < 2; ++ax) {
        if (n[ax] < 2) continue;
        const long long mp = (idx[ax] == n[ax] - 1) ? m - (long long)(n[ax] - 1) * st[ax] : m + st[ax];
        const long long mm = (idx[ax] == 0) ? m + (long long)(n[ax] - 1) * st[ax] : m - st[ax];
        const float4 p4 = ld4f(u + mp), q4 = ld4f(u + mm);
        const float ps[4] = {p4.x, p4.y, p4.z, p4.w}, qs[4] = {q4.x, q4.y, q4.z, q4.w};
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            float vp = (l[s] & bp[ax]) ? ps[s] - c[s] : 0.f;
            float vm = (l[s] & bm[ax]) ? qs[s] - c[s] : 0.f;
            if (bc[ax] == kOpen) {
                if (idx[ax] == 0) vm = vp;
                if (idx[ax] == n[ax] - 1) vp = vm;
            }
            acc[s] += cc[ax] * (vp + vm);
        }
    }
    return make_float4(acc[0], acc[1], acc[2], acc[3]);
}

// the components of four sites: -1 insulating, 0 the main one, c > 0 island c
template <bool ISL>
__device__ __forceinline__ void comps4(const InsArgs &a, long long m, int cs[4])
{
    if constexpr (ISL) {
        const int4 c = *reinterpret_cast<const int4 *>(a.comp + m);
        cs[0] = c.x, cs[1] = c.y, cs[2] = c.z, cs[3] = c.w;
    } else {
        const uchar4 l = *reinterpret_cast<const uchar4 *>(a.g.lk + m);
        cs[0] = (l.x & kLkIns) ? -1 : 0, cs[1] = (l.y & kLkIns) ? -1 : 0;
        cs[2] = (l.z & kLkIns) ? -1 : 0, cs[3] = (l.w & kLkIns) ? -1 : 0;
    }
}

template <bool ISL>
__global__ void ins_csum4_kernel(InsArgs a, const float *v, int slot)
{
    float acc = 0.f;
    for_quads(a.g, [&](long long m, int i0, int, int, float wyz) {
        const float4 x = ld4f(v + m);
        int cs[4];
        comps4<ISL>(a, m, cs);
        const float xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const float w = wyz * face_w(a.g.bcx, a.g.nx, i0 + s);
            if (cs[s] == 0) acc += w * xs[s];
            else if (ISL && cs[s] > 0) atomicAdd(a.isl_acc + (cs[s] - 1), (double)(w * xs[s]));
        }
    });
    if (finish_sum(a.ctl, a.blockred, (double)acc, &a.ctl->sums[slot]) && ISL) island_means(a);
}

template <bool ISL>
__global__ void ins_cshift4_kernel(InsArgs a, float *v, int mslot, int fmax)
{
    const float cm = (float)(a.ctl->sums[mslot] / a.wsum_c);
    float mx = 0.f;
    for_quads(a.g, [&](long long m, int, int, int, float) {
        const float4 x = ld4f(v + m);
        int cs[4];
        comps4<ISL>(a, m, cs);
        float xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int c = cs[s];
            xs[s] = (c < 0) ? 0.f : xs[s] - ((!ISL || c == 0) ? cm : (float)a.isl_acc[c - 1]);
            mx = fmaxf(mx, fabsf(xs[s]));
        }
        st4f(v + m, make_float4(xs[0], xs[1], xs[2], xs[3]));
    });
    if (!fmax) return;
    __shared__ float shf[32];
    __shared__ int flag;
    const float bmx = block_max(mx, shf);
    if (threadIdx.x == 0) a.blockred[blockIdx.x] = (double)bmx;
    if (!last_block(&a.ctl->ticket, gridDim.x, &flag)) return;
    double t = 0.0;
    for (unsigned int q = threadIdx.x; q < gridDim.x; q += blockDim.x) {
        const double w = ((volatile double *)a.blockred)[q];
        t = w > t ? w : t;
    }
    const float tm = block_max((float)t, shf);
    if (threadIdx.x == 0) {
        a.ctl->ticket = 0u;
        a.ctl->fmax = (double)tm;
        a.ctl->fmean = 0.0;
    }
}

// sums[slot] = sum w r v (r is zero on insulating sites)
__global__ void ins_dot4_kernel(InsArgs a, const float *v, int slot)
{
    float acc = 0.f;
    for_quads(a.g, [&](long long m, int i0, int, int, float wyz) {
        const float4 x = ld4f(v + m), r = ld4f(a.r + m);
        const float xs[4] = {x.x, x.y, x.z, x.w}, rs[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int s = 0; s < 4; ++s) acc += wyz * face_w(a.g.bcx, a.g.nx, i0 + s) * rs[s] * xs[s];
    });
    finish_sum(a.ctl, a.blockred, (double)acc, &a.ctl->sums[slot]);
}

__global__ void ins_dot_kernel(InsArgs a, const float *v, int slot)
{
    float acc = 0.f;   // FP32 per thread, FP64 over the threads and blocks
    for_sites(a.g, [&](long long m, int, int, int, float w) { acc += w * a.r[m] * v[m]; });
    finish_sum(a.ctl, a.blockred, (double)acc, &a.ctl->sums[slot]);
}

__global__ void ins_resid4_kernel(InsArgs a)
{
    for_quads(a.g, [&](long long m, int i0, int j, int k, float) {
        const uchar4 l = *reinterpret_cast<const uchar4 *>(a.g.lk + m);
        const float4 L = masked_lap4(a.g, a.mu, m, i0, j, k, l);
        const float4 f = ld4f(a.f + m);
        st4f(a.r + m, make_float4((l.x & kLkIns) ? 0.f : f.x - L.x, (l.y & kLkIns) ? 0.f : f.y - L.y,
                                  (l.z & kLkIns) ? 0.f : f.z - L.z, (l.w & kLkIns) ? 0.f : f.w - L.w));
    });
}

__global__ void ins_apply4_kernel(InsArgs a, int slot)
{
    float acc = 0.f;
    for_quads(a.g, [&](long long m, int i0, int j, int k, float wyz) {
        const uchar4 l = *reinterpret_cast<const uchar4 *>(a.g.lk + m);
        const float4 L = masked_lap4(a.g, a.p, m, i0, j, k, l);
        const float4 pv = ld4f(a.p + m);
        const float Ls[4] = {L.x, L.y, L.z, L.w}, ps[4] = {pv.x, pv.y, pv.z, pv.w};
        const unsigned ls[4] = {l.x, l.y, l.z, l.w};
        float qs[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            qs[s] = (ls[s] & kLkIns) ? 0.f : Ls[s];
            acc += wyz * face_w(a.g.bcx, a.g.nx, i0 + s) * ps[s] * qs[s];
        }
        st4f(a.q + m, make_float4(qs[0], qs[1], qs[2], qs[3]));
    });
    finish_sum(a.ctl, a.blockred, (double)acc, &a.ctl->sums[slot]);
}

__global__ void ins_dir4_kernel(InsArgs a, int num, int den, int first)
{
    const double d = a.ctl->sums[den];
    const float beta = (first || d == 0.0) ? 0.f : (float)(a.ctl->sums[num] / d);
    const long long nq = a.g.N >> 2;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nq; t += (long long)gridDim.x * blockDim.x) {
        const float4 z = ld4f(a.z + 4 * t);
        if (beta == 0.f) {   // the first direction (or a restart): p = z, the old p not read
            st4f(a.p + 4 * t, z);
            continue;
        }
        const float4 p = ld4f(a.p + 4 * t);
        st4f(a.p + 4 * t, make_float4(z.x + beta * p.x, z.y + beta * p.y, z.z + beta * p.z, z.w + beta * p.w));
    }
}

__global__ void ins_update4_kernel(InsArgs a, int rz, int pq)
{
    const double den = a.ctl->sums[pq];
    const float al = den != 0.0 ? (float)(a.ctl->sums[rz] / den) : 0.f;
    float mx = 0.f;
    const long long nq = a.g.N >> 2;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nq; t += (long long)gridDim.x * blockDim.x) {
        float4 r = ld4f(a.r + 4 * t);
        if (al != 0.f) {
            const float4 p = ld4f(a.p + 4 * t), q = ld4f(a.q + 4 * t);
            float4 u = ld4f(a.mu + 4 * t);
            u = make_float4(u.x + al * p.x, u.y + al * p.y, u.z + al * p.z, u.w + al * p.w);
            r = make_float4(r.x - al * q.x, r.y - al * q.y, r.z - al * q.z, r.w - al * q.w);
            st4f(a.mu + 4 * t, u);
            st4f(a.r + 4 * t, r);
        }
        mx = fmaxf(mx, fmaxf(fmaxf(fabsf(r.x), fabsf(r.y)), fmaxf(fabsf(r.z), fabsf(r.w))));
    }
    __shared__ float shf[32];
    __shared__ int flag;
    const float bm = block_max(mx, shf);
    if (threadIdx.x == 0) a.blockred[blockIdx.x] = (double)bm;
    if (!last_block(&a.ctl->ticket, gridDim.x, &flag)) return;
    double t = 0.0;
    for (unsigned int q = threadIdx.x; q < gridDim.x; q += blockDim.x) {
        const double v = ((volatile double *)a.blockred)[q];
        t = v > t ? v : t;
    }
    const float tm = block_max((float)t, shf);
    if (threadIdx.x == 0) {
        a.ctl->ticket = 0u;
        a.ctl->res = a.ctl->fmax > 0.0 ? (double)tm / a.ctl->fmax : (double)tm;
    }
}

// r = f - A mu
__global__ void ins_resid_kernel(InsArgs a)
{
    for_sites(a.g, [&](long long m, int i, int j, int k, float) {
        const unsigned l = a.g.lk[m];
        a.r[m] = (l & kLkIns) ? 0.f : a.f[m] - masked_lap(a.g, a.mu, m, i, j, k, l);
    });
}

// p = z + beta p, beta = sums[num] / sums[den] (first: beta = 0)
__global__ void ins_dir_kernel(InsArgs a, int num, int den, int first)
{
    const double d = a.ctl->sums[den];
    const float beta = (first || d == 0.0) ? 0.f : (float)(a.ctl->sums[num] / d);   // r = 0 exactly: restart
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < a.g.N;
         m += (long long)gridDim.x * blockDim.x)
        a.p[m] = a.z[m] + beta * a.p[m];
}

// q = A p, sums[slot] = sum_c w p q
__global__ void ins_apply_kernel(InsArgs a, int slot)
{
    float acc = 0.f;   // FP32 per thread, FP64 over the threads and blocks
    for_sites(a.g, [&](long long m, int i, int j, int k, float w) {
        const unsigned l = a.g.lk[m];
        if (l & kLkIns) {
            a.q[m] = 0.f;
            return;
        }
        const float v = masked_lap(a.g, a.p, m, i, j, k, l);
        a.q[m] = v;
        acc += w * a.p[m] * v;
    });
    finish_sum(a.ctl, a.blockred, (double)acc, &a.ctl->sums[slot]);
}

// alpha = sums[rz] / sums[pq] (the operator is negative semi-definite: both sums are
// negative or zero); mu += alpha p, r -= alpha q; ctl->res = max|r| / fmax
__global__ void ins_update_kernel(InsArgs a, int rz, int pq)
{
    const double den = a.ctl->sums[pq];
    const float al = den != 0.0 ? (float)(a.ctl->sums[rz] / den) : 0.f;
    float mx = 0.f;
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < a.g.N;
         m += (long long)gridDim.x * blockDim.x) {
        float r = a.r[m];
        if (al != 0.f) {
            a.mu[m] += al * a.p[m];
            r -= al * a.q[m];
            a.r[m] = r;
        }
        mx = fmaxf(mx, fabsf(r));
    }
    __shared__ float shf[32];
    __shared__ int flag;
    const float bm = block_max(mx, shf);
    if (threadIdx.x == 0) a.blockred[blockIdx.x] = (double)bm;
    if (!last_block(&a.ctl->ticket, gridDim.x, &flag)) return;
    double t = 0.0;
    for (unsigned int q = threadIdx.x; q < gridDim.x; q += blockDim.x) {
        const double v = ((volatile double *)a.blockred)[q];
        t = v > t ? v : t;
    }
    const float tm = block_max((float)t, shf);
    if (threadIdx.x == 0) {
        a.ctl->ticket = 0u;
        a.ctl->res = a.ctl->fmax > 0.0 ? (double)tm / a.ctl->fmax : (double)tm;
    }
}

// Blocks of a quad pass: one resident wave.  Every block's grid-stride walk then moves
// through the grid with the others, so the stencil's neighbours in the planes above and
// below are still in L2 when they are read (with more blocks than fit, the late blocks
// start far behind the early ones and those reads go to DRAM again).
template <class K>
static int wave_blocks(K kern)
{
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 4096;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kT, 0) != cudaSuccess || per < 1) per = 1;
    return per * sms < 4096 ? per * sms : 4096;
}

int masked_poisson_solve(const PoissonArgs &pa, const InsPoisson &ip, double tol, int iters, int max_iters,
                         cudaStream_t s, int *done, long long *launches)
{
    InsArgs a;
    a.g = pa.g;
    a.ctl = pa.ctl;
    a.blockred = pa.blockred;
    a.mu = pa.mu;
    a.f = pa.f;
    a.r = ip.r;
    a.z = ip.z;
    a.p = ip.p;
    a.q = ip.q;
    a.comp = ip.comp;
    a.isl_w = ip.isl_w;
    a.isl_acc = ip.isl_acc;
    a.wsum_c = ip.wsum_c;
    a.islands = ip.n_isl > 0 ? 1 : 0;
    a.n_isl = ip.n_isl;
    // one block per row (up to 4096 blocks, grid-stride beyond): within the partial-sum slots
    const int nb = a.g.ny * a.g.nz < 4096 ? a.g.ny * a.g.nz : 4096;
    // the quad passes: a resident wave each
    const int w_sum = a.islands ? wave_blocks(ins_csum4_kernel<true>) : wave_blocks(ins_csum4_kernel<false>);
    const int w_shift = a.islands ? wave_blocks(ins_cshift4_kernel<true>) : wave_blocks(ins_cshift4_kernel<false>);
    const int w_res = wave_blocks(ins_resid4_kernel), w_dot = wave_blocks(ins_dot4_kernel);
    const int w_app = wave_blocks(ins_apply4_kernel), w_upd = wave_blocks(ins_update4_kernel);
    const int w_dir = wave_blocks(ins_dir4_kernel);
    const size_t bytes = 4 * (size_t)a.g.N;
    // the preconditioner: one V-cycle of the plain operator on r, from z = 0
    PoissonArgs pz = pa;
    pz.lev[0].u = ip.z;
    pz.lev[0].r = ip.r;
    pz.mu = ip.z;
    pz.f = ip.r;
    pz.umap[0] = ip.zmap;
    pz.umap_u[0] = ip.zmap_u;
    long long nl = 0;
    // four sites per thread where rows hold whole 16-byte quads
    const bool quad = (a.g.nx % 4) == 0;
    // v -= the weighted mean of v's component (the constants of each component are the
    // operator's null space)
    auto project = [&](float *v, int fmax) -> bool {
        if (ip.n_isl > 0 && cudaMemsetAsync(ip.isl_acc, 0, 8 * (size_t)ip.n_isl, s) != cudaSuccess) return false;
        if (quad && a.islands) {
            ins_csum4_kernel<true><<<w_sum, kT, 0, s>>>(a, v, 4);
            ins_cshift4_kernel<true><<<w_shift, kT, 0, s>>>(a, v, 4, fmax);
        } else if (quad) {
            ins_csum4_kernel<false><<<w_sum, kT, 0, s>>>(a, v, 4);
            ins_cshift4_kernel<false><<<w_shift, kT, 0, s>>>(a, v, 4, fmax);
        } else {
            ins_csum_kernel<<<nb, kT, 0, s>>>(a, v, 4);
            ins_cshift_kernel<<<nb, kT, 0, s>>>(a, v, 4, fmax);
        }
        nl += 2;
        return cudaGetLastError() == cudaSuccess;
    };
    // z = M r by one V-cycle, and sums[rzslot] = (r, z).  z is not projected: its part in the
    // operator's null space (a constant on each component, any value on insulating sites)
    // is orthogonal to r and to every A p in the weighted inner product, so it changes no
    // step length or direction's image; it only adds null-space parts to mu, which the
    // closing projection removes.
    // Where the cycle's closing finest-level passes can sum (r, z) as they write z, they do.
    const bool fused_dot = vcycle_mean_fusable(pz);
    pz.mean_dot = 1;
    auto precondition = [&](int rzslot) -> bool {
        if (cudaMemsetAsync(ip.z, 0, bytes, s) != cudaSuccess) return false;
        pz.dot_slot = rzslot;
        if (launch_vcycle(pz, s, &nl, false, fused_dot) != cudaSuccess) return false;
        if (fused_dot) return true;
        if (quad) ins_dot4_kernel<<<w_dot, kT, 0, s>>>(a, ip.z, rzslot);
        else ins_dot_kernel<<<nb, kT, 0, s>>>(a, ip.z, rzslot);
        ++nl;
        return cudaGetLastError() == cudaSuccess;
    };
    if (!project(a.f, 1)) return TDGL_ERR_CUDA;   // compatible right-hand side on every component
    if (quad) ins_resid4_kernel<<<w_res, kT, 0, s>>>(a);
    else ins_resid_kernel<<<nb, kT, 0, s>>>(a);
    ++nl;
    if (!precondition(5)) return TDGL_ERR_CUDA;
    if (quad) ins_dir4_kernel<<<w_dir, kT, 0, s>>>(a, 5, 5, 1);
    else ins_dir_kernel<<<nb, kT, 0, s>>>(a, 5, 5, 1);
    ++nl;
    const int cap = iters > 0 ? iters : max_iters;
    int it = 0, rc = TDGL_OK;
    for (; it < cap; ++it) {
        const int rz = (it & 1) ? 6 : 5, rzn = (it & 1) ? 5 : 6;
        if (quad) {
            ins_apply4_kernel<<<w_app, kT, 0, s>>>(a, 7);
            ins_update4_kernel<<<w_upd, kT, 0, s>>>(a, rz, 7);
        } else {
            ins_apply_kernel<<<nb, kT, 0, s>>>(a, 7);
            ins_update_kernel<<<nb, kT, 0, s>>>(a, rz, 7);
        }
        nl += 2;
        if (cudaGetLastError() != cudaSuccess) return TDGL_ERR_CUDA;
        if (iters <= 0) {
            double res = 0.0;
            if (cudaMemcpyAsync(&res, &a.ctl->res, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
                return TDGL_ERR_CUDA;
            if (cudaStreamSynchronize(s) != cudaSuccess) return TDGL_ERR_CUDA;
            if (!(res == res)) {
                rc = TDGL_ERR_NONFINITE;
                ++it;
                break;
            }
            if (res <= tol) {
                ++it;
                break;
            }
        }
        if (it + 1 == cap) {   // the iteration cap ends the solve, as the cycle cap of the plain solver does
            ++it;
            break;
        }
        if (!precondition(rzn)) return TDGL_ERR_CUDA;
        if (quad) ins_dir4_kernel<<<w_dir, kT, 0, s>>>(a, rzn, rz, 0);
        else ins_dir_kernel<<<nb, kT, 0, s>>>(a, rzn, rz, 0);
        ++nl;
    }
    // zero weighted mean on every component, mu = 0 on insulating sites
    if (!project(a.mu, 0)) return TDGL_ERR_CUDA;
    *done = it;
    *launches += nl;
    return rc;
}

// ---------------------------------------------------------------------------
// E_x from the mean mu of each open x face over the sites of the largest conducting
// component (islands carry their own constant and no current from face to face)
// ---------------------------------------------------------------------------
__global__ void voltage_masked_kernel(DevGrid g, const float *mu, const int *comp, DevCtl *ctl, double *blockred,
                                      double hx, double n0, double n1)
{
    const long long nf = (long long)g.ny * g.nz;
    double acc = 0.0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nf; q += (long long)gridDim.x * blockDim.x) {
        const long long m0 = q * g.nx, m1 = q * g.nx + g.nx - 1;
        if (comp[m0] == 0) acc += (double)mu[m0] / n0;
        if (comp[m1] == 0) acc -= (double)mu[m1] / n1;
    }
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
        ctl->Ex = t / ((g.nx - 1) * hx);
    }
}

cudaError_t launch_voltage_masked(const PoissonArgs &a, const InsPoisson &ip, cudaStream_t s)
{
    const long long nf = (long long)a.g.ny * a.g.nz;
    int nb = (int)((nf + kT - 1) / kT);
    if (nb > 256) nb = 256;
    voltage_masked_kernel<<<nb, kT, 0, s>>>(a.g, a.mu, ip.comp, a.ctl, a.blockred, a.hx, ip.n_face0 > 0 ? ip.n_face0 : 1.0,
                                            ip.n_face1 > 0 ? ip.n_face1 : 1.0);
    return cudaGetLastError();
}

}  // namespace tdgl
