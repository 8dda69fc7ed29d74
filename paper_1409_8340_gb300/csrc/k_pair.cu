// Two Jacobi sweeps per pass over memory (temporal blocking of Sec. 3.1, Eq.
// final), with the paper's per-sweep convergence test kept exactly.
//
// A block of 32 x 8 threads owns a tile of 60 x 6 sites (plus a halo of one pair
// in x and one row in y) and marches along z.  At plane k it computes the first
// sweep psi1 = J(psi0) on the whole haloed tile (stage 1, the same per-site
// arithmetic as the single-sweep tile), keeps psi1 of planes k-2..k in registers
// and shares plane k's rows through a three-slot shared ring; then it computes
// the second sweep psi2 = J(psi1) at plane k-1 on the tile interior (stage 2):
// z neighbours from registers, x neighbours from the adjacent lanes, y
// neighbours from the ring.  Global traffic per pass: read psi0, b, diag M,
// write psi2 (32 B per site for two sweeps instead of 64).
//
// Both residuals are reduced: max|r|^2 of psi0 (the first sweep's input) and of
// psi1 (the second's).  The last block decides as two consecutive single sweeps
// would.  If the first sweep already met the test, its output psi1 is the
// result; it was not stored, so the device control block says so (redo) and the
// host recomputes it with one plain sweep from the same input.
#include <float.h>

#include "sweep_tile.cuh"

namespace tdgl {

constexpr int kPW = 8;            // warps per block = tile rows incl. the y halo
constexpr int kPTY = kPW - 2;     // interior rows
constexpr int kPTX = 60;          // interior sites along x (lanes 1..30)

__device__ __forceinline__ int wrap_idx(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

// Jacobi update and residual of a site pair (the single-sweep tile's order of operations).
__device__ __forceinline__ void pair_update(float4 bq, float4 Dq, float2 c0, float2 c1, float2 ns0, float2 ns1,
                                            float4 &out, float &r2)
{
    const float2 b0 = lo2(bq), b1 = hi2(bq), D0 = lo2(Dq), D1 = hi2(Dq);
    const float2 s0 = cadd(b0, ns0), s1 = cadd(b1, ns1);
    const float2 r0 = csub(s0, cmul(D0, c0)), r1 = csub(s1, cmul(D1, c1));
    const float2 n0 = cscale(__frcp_rn(cabs2(D0)), cmulc(D0, s0));
    const float2 n1 = cscale(__frcp_rn(cabs2(D1)), cmulc(D1, s1));
    out = make_float4(n0.x, n0.y, n1.x, n1.y);
    float r2a = cabs2(r0), r2b = cabs2(r1);
    r2a = (r2a <= FLT_MAX) ? r2a : INFINITY;
    r2b = (r2b <= FLT_MAX) ? r2b : INFINITY;
    r2 = fmaxf(r2a, r2b);
}

// (ht/2) NS of a site pair (x, x+1) at row j, plane k from its neighbours: pc the
// pair, xl the site left of x, xr the site right of x+1, yf/yb the pairs of rows
// j+1/j-1, zp/zm the pairs of planes k+1/k-1.  Boundary rules: open faces double
// the inner neighbour, the periodic x wrap link carries conj(P_jk).
struct PairCoef {
    float2 xf, yf0, yf1, zf0, zf1;
};
// Boundary flags of a site pair, fixed along z.
struct PairFlags {
    bool xlo, xhi, xper, yedge, zopen;
    float wy_f, wy_b;
};
__device__ __forceinline__ PairFlags pair_flags(const DevGrid &g, int x, int j)
{
    PairFlags f;
    f.xper = (g.bcx == kPeriodic);
    f.xlo = (x == 0);
    f.xhi = (x + 2 >= g.nx);
    const bool yper = (g.bcy == kPeriodic), ylo = (j == 0), yhi = (j == g.ny - 1);
    f.wy_f = yper ? 1.f : (ylo ? 2.f : (yhi ? 0.f : 1.f));
    f.wy_b = yper ? 1.f : (yhi ? 2.f : (ylo ? 0.f : 1.f));
    f.yedge = (f.wy_f != 1.f) || (f.wy_b != 1.f);
    f.zopen = (g.bcz != kPeriodic);
    return f;
}
__device__ __forceinline__ void pair_ns(const DevGrid &g, const PairCoef &C, const PairFlags &F, int j, int k, float4 pc,
                                        float2 xl, float2 xr, float4 yf, float4 yb, float4 pzp, float4 pzm, float2 &ns0,
                                        float2 &ns1)
{
    const float2 c0 = lo2(pc), c1 = hi2(pc);
    float2 xl0 = xl, xr1 = xr, c1x = c1, c0x = c0;
    if (F.xlo || F.xhi) {
        if (F.xper) {
            const float2 P = cmul(g.Py[j], g.Pz[k]);
            if (F.xlo) xl0 = cmul(P, xl);
            if (F.xhi) xr1 = cmulc(P, xr);
        } else {
            if (F.xlo) {
                c1x = cscale(2.f, c1);
                xl0 = cmk(0.f, 0.f);
            }
            if (F.xhi) {
                c0x = cscale(2.f, c0);
                xr1 = cmk(0.f, 0.f);
            }
        }
    }
    float2 yf_0 = lo2(yf), yf_1 = hi2(yf), yb_0 = lo2(yb), yb_1 = hi2(yb);
    if (F.yedge) {
        yf_0 = cscale(F.wy_f, yf_0);
        yf_1 = cscale(F.wy_f, yf_1);
        yb_0 = cscale(F.wy_b, yb_0);
        yb_1 = cscale(F.wy_b, yb_1);
    }
    ns0 = cmul(C.xf, c1x);
    ns1 = cmulc(C.xf, c0x);
    cfmac(ns0, C.xf, xl0);
    cfma(ns1, C.xf, xr1);
    cfma(ns0, C.yf0, yf_0);
    cfmac(ns0, C.yf0, yb_0);
    cfma(ns1, C.yf1, yf_1);
    cfmac(ns1, C.yf1, yb_1);
    if (g.nz >= 2) {
        float wz_f = 1.f, wz_b = 1.f;
        if (F.zopen) {
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
        cfma(ns0, C.zf0, lo2(zpp));
        cfmac(ns0, C.zf0, lo2(zmm));
        cfma(ns1, C.zf1, hi2(zpp));
        cfmac(ns1, C.zf1, hi2(zmm));
    }
}

// Decision after a pass: the two sweeps' tests in order (Eq. convergence), as
// sweep_decide would take them one at a time.  Run by one thread.
__device__ __forceinline__ void pair_decide(const SweepArgs &a, float g1, float g2)
{
    DevCtl *c = a.ctl;
    c->redo = 0;
    auto one = [&](float gf, int it) -> bool {
        c->iter = it;
        c->r2 = (double)gf;
        c->result = a.dst_index;
        if (!(gf <= FLT_MAX)) {
            c->status = TDGL_ERR_NONFINITE;
            c->done = 1;
        } else if (a.fixed_sweeps > 0) {
            c->done = (it >= a.fixed_sweeps) ? 1 : 0;
        } else if ((it % a.check_every) == 0 && (double)gf < a.eps) {
            c->done = 1;
        } else if (it >= a.max_iter) {
            c->status = TDGL_ERR_NOT_CONVERGED;
            c->done = 1;
        } else {
            c->done = 0;
        }
        return c->done != 0;
    };
    const int it = c->iter + 1;
    if (one(g1, it)) {
        c->redo = 1;   // the first sweep's output is the result
        return;
    }
    one(g2, it + 1);
}

__global__ void __launch_bounds__(32 * kPW, 3) sweep_pair_kernel(SweepArgs a, int kz)
{
    if (*(volatile int *)&a.ctl->done) return;
    const DevGrid &g = a.g;
    __shared__ float4 ring[3][kPW][32];
    const int L = threadIdx.x, w = threadIdx.y;
    const bool xper = (g.bcx == kPeriodic), yper = (g.bcy == kPeriodic);
    const bool zwrap = (g.bcz == kPeriodic) && g.nz >= 3;
    const int nz = g.nz;
    const int x = kPTX * blockIdx.x - 2 + 2 * L;   // unwrapped
    const int y = kPTY * blockIdx.y - 1 + w;
    const int xs = xper ? wrap_idx(x, g.nx) : x;
    const int ys = yper ? wrap_idx(y, g.ny) : y;
    const bool v1 = (xper || (x >= 0 && x <= g.nx - 2)) && (yper || (y >= 0 && y < g.ny));
    const bool v2 = L >= 1 && L <= 30 && w >= 1 && w <= kPW - 2 && x >= 0 && x <= g.nx - 2 && y >= 0 && y < g.ny;
    const int k0 = blockIdx.z * kz, k1 = min(k0 + kz, nz);
    const int ks = zwrap ? k0 - 1 : max(k0 - 1, 0);

    const float4 *__restrict__ src = reinterpret_cast<const float4 *>(a.src);
    const float2 *__restrict__ src2 = a.src;
    const float4 *__restrict__ bq = reinterpret_cast<const float4 *>(a.b);
    const float4 *__restrict__ Dq = reinterpret_cast<const float4 *>(a.D);
    float4 *__restrict__ dst = reinterpret_cast<float4 *>(a.dst);
    const long long rowq = g.nx >> 1, plq = rowq * g.ny, sz = (long long)g.nx * g.ny;

    // stage-1 site pair (wrapped), its row neighbours (face rows read themselves; weight 0)
    const int jc = v1 ? ys : 0;
    const int jp = (jc == g.ny - 1) ? (yper ? 0 : jc) : jc + 1;
    const int jm = (jc == 0) ? (yper ? g.ny - 1 : jc) : jc - 1;
    const int xc = v1 ? xs : 0;
    const long long q0 = (xc >> 1) + rowq * jc;
    const long long qp = (xc >> 1) + rowq * jp, qm = (xc >> 1) + rowq * jm;
    const long long m0 = (long long)xc + (long long)g.nx * jc;
    const PairFlags F1 = pair_flags(g, xc, jc);
    const PairFlags F2 = pair_flags(g, x, y);
    // x neighbours of the edge lanes: offsets from the site x (wrap on periodic x)
    const int dl = (xc > 0) ? -1 : (xper ? g.nx - 1 : 0);
    const int dr = (xc + 2 < g.nx) ? 2 : (xper ? 2 - g.nx : 0);
    PairCoef C;
    {
        const float2 Ux = a.ctl->Ux;
        const float4 uy = reinterpret_cast<const float4 *>(g.Uy)[xc >> 1];
        const float4 uz = reinterpret_cast<const float4 *>(g.Uz)[xc >> 1];
        const float sy = g.ht2 * g.cy, szc = g.ht2 * g.cz;
        C.xf = cscale(g.ht2 * g.cx, Ux);
        C.yf0 = cscale(sy, lo2(uy));
        C.yf1 = cscale(sy, hi2(uy));
        C.zf0 = cscale(szc, lo2(uz));
        C.zf1 = cscale(szc, hi2(uz));
    }
    // plane of stage-1 step kk: wrapped (periodic z) or clamped (its weight is then 0)
    auto znext = [&](int k) { return (k + 1 < nz) ? k + 1 : (zwrap ? 0 : nz - 1); };
    int kw = zwrap ? (ks < 0 ? ks + nz : ks) : ks;     // plane of kk
    int kw1 = znext(kw), kw2 = znext(kw1);             // planes of kk + 1, kk + 2
    const int kwm = zwrap ? (kw == 0 ? nz - 1 : kw - 1) : max(kw - 1, 0);

    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 p_m = zero4, p_c = zero4, p_p = zero4, b_c = zero4, D_c = zero4;
    if (v1) {
        if (nz >= 2) p_m = src[q0 + plq * kwm];
        p_c = src[q0 + plq * kw];
        if (nz >= 2) p_p = src[q0 + plq * kw1];
        b_c = bq[q0 + plq * kw];
        D_c = Dq[q0 + plq * kw];
    }
    float4 q_m = zero4, q_c = zero4, b_s = zero4, D_s = zero4;   // psi1 at kk-2, kk-1; b, D at kk-1
    float rmax1 = 0.f, rmax2 = 0.f;
    int slot = 0, pslot = 2;   // ring slots of kk and kk - 1
    for (int kk = ks; kk <= k1; ++kk) {
        const bool pv = zwrap || (kk >= 0 && kk < nz);
        const long long po = plq * kw;
        // prefetch of the next plane
        float4 p_n = zero4, b_n = zero4, D_n = zero4;
        if (v1 && kk < k1) {
            if (nz >= 2) p_n = src[q0 + plq * kw2];
            const long long po1 = plq * kw1;
            b_n = bq[q0 + po1];
            D_n = Dq[q0 + po1];
        }
        // ---- stage 1: psi1 at plane kk on the haloed tile
        float4 yf = zero4, yb = zero4;
        if (v1 && pv) {
            yf = src[qp + po];
            yb = src[qm + po];
        }
        const float2 from_left = make_float2(__shfl_up_sync(0xffffffffu, p_c.z, 1), __shfl_up_sync(0xffffffffu, p_c.w, 1));
        const float2 from_right = make_float2(__shfl_down_sync(0xffffffffu, p_c.x, 1), __shfl_down_sync(0xffffffffu, p_c.y, 1));
        float4 n1 = zero4;
        float r1 = 0.f;
        if (v1 && pv) {
            const long long m = m0 + sz * kw;
            float2 xl = from_left, xr = from_right;
            if (L == 0) xl = (dl != 0) ? src2[m + dl] : cmk(0.f, 0.f);
            if (L == 31 || F1.xhi) xr = (dr != 0) ? src2[m + dr] : cmk(0.f, 0.f);
            float2 ns0, ns1;
            pair_ns(g, C, F1, jc, kw, p_c, xl, xr, yf, yb, p_p, p_m, ns0, ns1);
            pair_update(b_c, D_c, lo2(p_c), hi2(p_c), ns0, ns1, n1, r1);
        }
        if (v2 && kk >= k0 && kk < k1) rmax1 = fmaxf(rmax1, r1);
        ring[slot][w][L] = n1;
        __syncthreads();
        // ---- stage 2: psi2 at plane km = kk - 1 on the interior
        const int km = kk - 1;
        const float2 l1 = make_float2(__shfl_up_sync(0xffffffffu, q_c.z, 1), __shfl_up_sync(0xffffffffu, q_c.w, 1));
        const float2 r1n = make_float2(__shfl_down_sync(0xffffffffu, q_c.x, 1), __shfl_down_sync(0xffffffffu, q_c.y, 1));
        if (v2 && km >= k0 && km < k1) {
            const float4 yf2 = ring[pslot][w + 1][L], yb2 = ring[pslot][w - 1][L];
            float2 ns0, ns1;
            pair_ns(g, C, F2, y, km, q_c, l1, r1n, yf2, yb2, n1, q_m, ns0, ns1);
            float4 n2;
            float r2;
            pair_update(b_s, D_s, lo2(q_c), hi2(q_c), ns0, ns1, n2, r2);
            dst[(x >> 1) + rowq * y + plq * km] = n2;
            rmax2 = fmaxf(rmax2, r2);
        }
        // rotate registers, ring slots and plane indices
        q_m = q_c;
        q_c = n1;
        b_s = b_c;
        D_s = D_c;
        p_m = p_c;
        p_c = p_p;
        p_p = p_n;
        b_c = b_n;
        D_c = D_n;
        pslot = slot;
        slot = (slot == 2) ? 0 : slot + 1;
        kw = kw1;
        kw1 = kw2;
        kw2 = znext(kw2);
    }
    // block maxima, then the last block decides
    __shared__ float shf[32];
    __shared__ int flag;
    const float m1 = block_max(rmax1, shf);
    const float m2 = block_max(rmax2, shf);
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const unsigned int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const unsigned int nb = gridDim.x * gridDim.y * gridDim.z;
    if (tid == 0) {
        a.blockred[2 * bid] = (double)m1;
        a.blockred[2 * bid + 1] = (double)m2;
    }
    if (!last_block(&a.ctl->ticket, nb, &flag)) return;
    double g1 = 0.0, g2 = 0.0;
    for (unsigned int q = tid; q < nb; q += blockDim.x * blockDim.y) {
        const double v1q = ((volatile double *)a.blockred)[2 * q], v2q = ((volatile double *)a.blockred)[2 * q + 1];
        g1 = v1q > g1 ? v1q : g1;
        g2 = v2q > g2 ? v2q : g2;
    }
    const float f1 = block_max((float)g1, shf);
    const float f2 = block_max((float)g2, shf);
    if (tid == 0) {
        a.ctl->ticket = 0u;
        pair_decide(a, f1, f2);
    }
}

static int pair_kz(const DevGrid &g)
{
    const long long bxy = (long long)((g.nx + kPTX - 1) / kPTX) * ((g.ny + kPTY - 1) / kPTY);
    long long kz = (bxy * g.nz) / 1824;   // about four resident blocks per SM, several waves
    if (kz < 4) kz = 4;
    if (kz > 64) kz = 64;
    return (int)(kz > g.nz ? g.nz : kz);
}

dim3 pair_grid(const DevGrid &g)
{
    const int kz = pair_kz(g);
    return dim3((g.nx + kPTX - 1) / kPTX, (g.ny + kPTY - 1) / kPTY, (g.nz + kz - 1) / kz);
}

size_t pair_blocks(const DevGrid &g)
{
    const dim3 gr = pair_grid(g);
    return (size_t)gr.x * gr.y * gr.z;
}

bool pair_supported(const DevGrid &g) { return g.L == nullptr && g.lk == nullptr && (g.nx % 2) == 0; }

cudaError_t launch_sweep_pair(const SweepArgs &a, cudaStream_t s)
{
    if (!pair_supported(a.g) || a.rel_eps) return cudaErrorInvalidValue;
    sweep_pair_kernel<<<pair_grid(a.g), dim3(32, kPW), 0, s>>>(a, pair_kz(a.g));
    return cudaGetLastError();
}

}  // namespace tdgl
