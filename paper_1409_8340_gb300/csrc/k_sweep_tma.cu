// Jacobi sweep (arXiv:1409.8340, Sec. 3.1, Eq. final and Eq. convergence) with
// its tile staged in shared memory by the tensor memory accelerator.
//
// A block owns 64 x-sites by 8 rows and marches along z.  One producer thread
// streams, per z plane, three boxes into a ring of five plane stages with
// cp.async.bulk.tensor: psi over 68 x-sites (the tile and one site beyond each
// end, on 16-byte boundaries) by 10 rows (the tile and its y halo), and the
// tile's b and diag M; each stage completes an mbarrier by transaction bytes.
// Eight consumer warps (one row each, two sites per lane) read the plane below,
// the plane and the plane above from the ring, write the new iterate to global
// memory and release the plane below through a second mbarrier per stage.  The
// ring keeps three planes in flight ahead of the consumers without holding them
// in registers.  Box parts outside the grid arrive as zeros; the few neighbours
// across a periodic wrap (the x ends of the first and last tiles, the y halo of
// the first and last row tiles) are read from global memory by the lanes that
// need them.  Arithmetic per site is the register-tiled kernel's, in the same
// order, except that 1 / |diag M|^2 comes from the hardware reciprocal
// approximation instead of the correctly rounded one (the new iterate then differs
// by about one FP32 ulp).  Blocks whose tile touches no x or y face run the same
// code with the face tests folded away.  Every wait is bounded by the global timer; a wait that runs out sets
// TDGL_ERR_TIMEOUT and ends the block's planes, the producer drains its copies in
// flight (again bounded), and the block still takes its part in the last-block
// reduction, whose deciding block then ends the solve with that status.
//
// Landau links of either plane (XZ: the j-indexed tables and the y wrap of the
// xz gauge), insulating sites (MASK: link bits, read per site pair), even nx.
//
// RHS: the same tile pipeline for the Poisson right-hand side (Sec. 3.3): only the psi
// box is streamed, through a deeper ring of twelve smaller stages (psi is the only
// stream, so more planes must be in flight), and each site pair writes
// f = Im[conj(psi) NS(psi)] / (ht/2) plus the injected current on the open x faces,
// the register-tiled kernel's arithmetic; the trapezoid-weighted FP64 sum of f is
// reduced over the blocks and the last block stores its mean.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <float.h>

#include <type_traits>

#include "sweep_tile.cuh"
#include "tdgl_internal.cuh"
#include "tma_util.cuh"

namespace tdgl {

namespace {

constexpr int kTR = 8;            // rows per block (consumer warps)
constexpr int kTX = 64;           // x-sites per block
constexpr int kTS = 5;            // ring stages (planes)
constexpr int kRowP = kTX + 4;    // psi row in a stage: [2 halo | 64 | 2 halo]
constexpr int kThreads = (kTR + 1) * 32;
constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s: far beyond any plane's copy time

struct Stage {
    float2 psi[kTR + 2][kRowP];   // 5440 bytes, padded to a 128-byte boundary
    float2 pad[8];
    float2 b[kTR][kTX];
    float2 D[kTR][kTX];
};
static_assert(sizeof(Stage) % 128 == 0, "stages on 128-byte boundaries");
static_assert(offsetof(Stage, b) % 128 == 0 && offsetof(Stage, D) % 128 == 0, "boxes on 128-byte boundaries");
constexpr unsigned kPsiBytes = (kTR + 2) * kRowP * 8;
constexpr unsigned kPlaneBytes = kPsiBytes + 2 * kTR * kTX * 8;
// right-hand side: psi boxes only, twelve stages
struct StageR {
    float2 psi[kTR + 2][kRowP];
    float2 pad[8];
};
static_assert(sizeof(StageR) % 128 == 0, "stages on 128-byte boundaries");
constexpr int kTSR = 12;
template <bool RHS>
using StageT = typename std::conditional<RHS, StageR, Stage>::type;
template <bool RHS>
constexpr int kStages = RHS ? kTSR : kTS;

// 1 / x by the hardware reciprocal approximation (relative error within about 2^-23 in
// the normal range; |diag M|^2 is of order 1 to 10, far from it)
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// one box of a 3-D tensor map at (x, y, z) into shared memory
__device__ __forceinline__ void tma_load3(void *dst, const CUtensorMap *map, int x, int y, int z,
                                         unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            smem_addr(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

}  // namespace

// Tile geometry shared by the producer and the consumers.
struct TmaTile {
    int x0, w;       // first x-site, valid x-sites (even)
    int j0, nr;      // first row, valid rows
};

__device__ __forceinline__ int plane_of(const DevGrid &g, int z)
{
    if (z < 0) return (g.bcz == kPeriodic) ? z + g.nz : (g.nz >= 2 ? 1 : 0);
    if (z >= g.nz) return (g.bcz == kPeriodic) ? z - g.nz : (g.nz >= 2 ? g.nz - 2 : 0);
    return z;
}

// Producer: the three boxes of plane z into stage S (the psi box alone for the
// right-hand side).  x starts two sites before the tile (even, as the tensor memory
// accelerator requires of 8-byte elements).
template <bool RHS>
__device__ __forceinline__ void issue_plane(const TmaTile &T, int zp, StageT<RHS> &S, unsigned long long *full,
                                           const CUtensorMap *mp, const CUtensorMap *mb, const CUtensorMap *md,
                                           unsigned extra_tx)
{
    mbar_expect(full, (RHS ? kPsiBytes : kPlaneBytes) + extra_tx);
    tma_load3(&S.psi[0][0], mp, T.x0 - 2, T.j0 - 1, zp, full);
    if constexpr (!RHS) {
        tma_load3(&S.b[0][0], mb, T.x0, T.j0, zp, full);
        tma_load3(&S.D[0][0], md, T.x0, T.j0, zp, full);
    }
}

template <bool XZ, bool MASK, bool RHS>
__global__ void __launch_bounds__(kThreads, 3)
    sweep_tma_kernel(SweepArgs a, int kz, const __grid_constant__ CUtensorMap map_psi,
                     const __grid_constant__ CUtensorMap map_b, const __grid_constant__ CUtensorMap map_D)
{
    constexpr int NS = kStages<RHS>;
    using St = StageT<RHS>;
    if (!RHS && sweep_already_decided(a)) return;
    extern __shared__ __align__(128) unsigned char tma_smem[];
    St *ring = reinterpret_cast<St *>(tma_smem);
    unsigned long long *full = reinterpret_cast<unsigned long long *>(tma_smem + NS * sizeof(St));
    unsigned long long *empty = full + NS;
    __shared__ int failed;

    const DevGrid &g = a.g;
    TmaTile T;
    T.x0 = blockIdx.x * kTX;
    T.w = min(kTX, g.nx - T.x0);
    T.j0 = blockIdx.y * kTR;
    T.nr = min(kTR, g.ny - T.j0);
    const int k0 = zlo(g) + blockIdx.z * kz, k1 = min(k0 + kz, zhi(g));
    const int nplanes = (k1 - k0) + 2;   // k0 - 1 .. k1
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kTR);
        }
        failed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const unsigned long long wait_ns = a.wait_ns ? a.wait_ns : kWaitNs;
    // timeout test only: the first block's stages expect bytes that never come
    const unsigned xtx = (blockIdx.x | blockIdx.y | blockIdx.z) == 0 ? a.extra_tx : 0u;
    const unsigned long long deadline = gtime() + wait_ns;
    float rmax = 0.f;
    float facc = 0.f;   // RHS: sum of w f over the thread's sites

    if (warp == kTR) {
        // ---------------- producer (one thread) ----------------
        if (lane == 0) {
            int issued = 0;
            for (int t = 0; t < nplanes; ++t) {
                const int s = t % NS;
                if (t >= NS && (!mbar_wait(&empty[s], (unsigned)((t / NS - 1) & 1), deadline) ||
                                *(volatile int *)&failed)) {
                    failed = 1;
                    break;
                }
                issue_plane<RHS>(T, plane_of(g, k0 - 1 + t), ring[s], &full[s], &map_psi, &map_b, &map_D,
                                 xtx);
                issued = t + 1;
            }
            // drain: every issued plane's copies complete before the block can exit
            for (int t = max(0, issued - NS); t < issued; ++t)
                mbar_wait(&full[t % NS], (unsigned)((t / NS) & 1), deadline + wait_ns);
        }
        __syncwarp();
    } else {
        // ---------------- consumers: row `warp`, sites x, x+1 ----------------
        // blocks whose tile touches no x or y face (nor a periodic wrap there) run the
        // same code with the face tests folded away
        const bool edge = T.x0 == 0 || T.x0 + kTX >= g.nx || T.j0 == 0 || T.j0 + kTR >= g.ny;
        auto consume = [&](auto edge_t) {
            constexpr bool EDGE = decltype(edge_t)::value;
            const int r = warp;
            const int x = T.x0 + 2 * lane, j = T.j0 + r;
            const bool in = !EDGE || ((r < T.nr) && (2 * lane < T.w));
            const bool xper = (g.bcx == kPeriodic), yper = (g.bcy == kPeriodic), zper = (g.bcz == kPeriodic);
            const bool xlo = EDGE && (x == 0), xhi = EDGE && (x + 2 >= g.nx);
            const bool ylo = EDGE && (j == 0), yhi = EDGE && (j == g.ny - 1);
            const bool zact = g.nz >= 2;
            const int jc = min(j, g.ny - 1);
            const float wy_f = yper ? 1.f : (ylo ? 2.f : (yhi ? 0.f : 1.f));
            const float wy_b = yper ? 1.f : (yhi ? 2.f : (ylo ? 0.f : 1.f));
            const bool yedge = (wy_f != 1.f) || (wy_b != 1.f);
            float2 yf0 = cmk(0.f, 0.f), yf1 = yf0, zf0 = yf0, zf1 = yf0;
            const bool ywrap = XZ && yper && (ylo || yhi);   // a row next to the xz gauge's y wrap
            float4 wxq = make_float4(1.f, 0.f, 1.f, 0.f);
            if (in) {
                const float sy = g.ht2 * g.cy, szc = g.ht2 * g.cz;
                if (XZ) {
                    yf0 = yf1 = cmk(sy, 0.f);
                    zf0 = zf1 = cscale(szc, g.Zj[jc]);
                    if (ywrap) wxq = reinterpret_cast<const float4 *>(g.Wx)[x >> 1];
                } else {
                    const float4 uy = reinterpret_cast<const float4 *>(g.Uy)[x >> 1];
                    const float4 uz = reinterpret_cast<const float4 *>(g.Uz)[x >> 1];
                    yf0 = cscale(sy, lo2(uy));
                    yf1 = cscale(sy, hi2(uy));
                    zf0 = cscale(szc, lo2(uz));
                    zf1 = cscale(szc, hi2(uz));
                }
            }
            const float2 Ux = ldx<false>(&a.ctl->Ux);
            const float2 xf = cscale(g.ht2 * g.cx, XZ ? cmul(Ux, g.Xj[jc]) : Ux);
            const uchar2 *__restrict__ lk2 = reinterpret_cast<const uchar2 *>(g.lk);
            float4 *__restrict__ dst = reinterpret_cast<float4 *>(a.dst);
            const long long rowq = g.nx >> 1, plq = rowq * g.ny;
            const long long q0 = (x >> 1) + rowq * jc;
            // RHS: trapezoid weights of the pair on open faces, 1 / (ht/2)
            const float wy = (g.bcy == kOpen && (j == 0 || j == g.ny - 1)) ? 0.5f : 1.f;
            const float wxy0 = wy * ((g.bcx == kOpen && x == 0) ? 0.5f : 1.f);
            const float wxy1 = wy * ((g.bcx == kOpen && x + 1 == g.nx - 1) ? 0.5f : 1.f);
            const float inv_ht2 = 1.0f / g.ht2;
            float2 *fdp = reinterpret_cast<float2 *>(a.f) + q0 + plq * k0;
            bool ok = true;
            // stages of planes t - 1, t, t + 1 and the phase parity of plane t + 1's stage,
            // advanced by one plane per iteration
            int sm = 0, sc = 1, sp = 2;
            unsigned php = 0u;
            float4 *dp = dst + q0 + plq * k0;   // plane k0 - 1 + t of this lane's site pair
            // MASK: the link bits of the pair, read one plane ahead (their load overlaps a plane)
            uchar2 lk_next = make_uchar2(0x3f, 0x3f);
            if (MASK && in) lk_next = lk2[q0 + plq * k0];
            for (int t = 1; t + 1 < nplanes; ++t) {
                const int k = k0 - 1 + t;
                if (t == 1) {
                    ok = mbar_wait(&full[0], 0u, deadline) && mbar_wait(&full[1], 0u, deadline);
                }
                ok = ok && mbar_wait(&full[sp], php, deadline);
                if (!__all_sync(0xffffffffu, ok)) {
                    if (lane == 0) failed = 1;
                    break;
                }
                const St &Pm = ring[sm], &Pc = ring[sc], &Pp = ring[sp];
                if (in) {
                    const uchar2 lkc = lk_next;
                    if (MASK && t + 2 < nplanes) lk_next = lk2[q0 + plq * (k + 1)];
                    const int cx = 2 + 2 * lane;
                    const float4 pc = *reinterpret_cast<const float4 *>(&Pc.psi[r + 1][cx]);
                    const float2 c0 = lo2(pc), c1 = hi2(pc);
                    float2 xl = Pc.psi[r + 1][cx - 1], xr = Pc.psi[r + 1][cx + 2];
                    float4 yf = *reinterpret_cast<const float4 *>(&Pc.psi[r + 2][cx]);
                    float4 yb = *reinterpret_cast<const float4 *>(&Pc.psi[r][cx]);
                    // neighbours across a periodic wrap lie outside the boxes: read them directly
                    const long long rowk = (long long)k * g.ny;
                    if (xper && xlo) xl = a.src[(rowk + j) * g.nx + g.nx - 1];
                    if (xper && xhi) xr = a.src[(rowk + j) * g.nx];
                    if (yper && ylo) yb = reinterpret_cast<const float4 *>(a.src)[((rowk + g.ny - 1) * g.nx + x) >> 1];
                    if (yper && yhi) yf = reinterpret_cast<const float4 *>(a.src)[(rowk * g.nx + x) >> 1];
                    float4 bc = make_float4(0.f, 0.f, 0.f, 0.f), Dc = bc;
                    if constexpr (!RHS) {
                        bc = *reinterpret_cast<const float4 *>(&Pc.b[r][2 * lane]);
                        Dc = *reinterpret_cast<const float4 *>(&Pc.D[r][2 * lane]);
                    }
                    // the same boundary rules and arithmetic order as the tiled kernel (MODE 0)
                    float2 xl0 = xl, xr1 = xr, c1x = c1, c0x = c0;
                    if (xlo || xhi) {
                        if (xper) {
                            if (!XZ) {   // the yz gauge's wrap link carries conj(P_jk); the xz gauge's is plain
                                const float2 P = cmul(g.Py[jc], g.Pz[k]);
                                if (xlo) xl0 = cmul(P, xl);
                                if (xhi) xr1 = cmulc(P, xr);
                            }
                        } else {
                            if (xlo) {
                                c1x = cscale(2.f, c1);
                                xl0 = cmk(0.f, 0.f);
                            }
                            if (xhi) {
                                c0x = cscale(2.f, c0);
                                xr1 = cmk(0.f, 0.f);
                            }
                        }
                    }
                    float2 yf_0 = lo2(yf), yf_1 = hi2(yf), yb_0 = lo2(yb), yb_1 = hi2(yb);
                    if (ywrap) {   // xz gauge: wrap link W = Wx[i] Wz[k] from row ny-1 to row 0
                        const float2 wz = g.Wz[k];
                        const float2 W0 = cmul(lo2(wxq), wz), W1 = cmul(hi2(wxq), wz);
                        if (yhi) {
                            yf_0 = cmul(W0, yf_0);
                            yf_1 = cmul(W1, yf_1);
                        }
                        if (ylo) {
                            yb_0 = cmulc(W0, yb_0);
                            yb_1 = cmulc(W1, yb_1);
                        }
                    }
                    if (yedge) {
                        yf_0 = cscale(wy_f, yf_0);
                        yf_1 = cscale(wy_f, yf_1);
                        yb_0 = cscale(wy_b, yb_0);
                        yb_1 = cscale(wy_b, yb_1);
                    }
                    if (MASK) {   // links next to insulating sites removed
                        const unsigned l0 = lkc.x, l1 = lkc.y;
                        c1x = cscale((l0 & kLkXp) ? 1.f : 0.f, c1x);
                        xl0 = cscale((l0 & kLkXm) ? 1.f : 0.f, xl0);
                        xr1 = cscale((l1 & kLkXp) ? 1.f : 0.f, xr1);
                        c0x = cscale((l1 & kLkXm) ? 1.f : 0.f, c0x);
                        yf_0 = cscale((l0 & kLkYp) ? 1.f : 0.f, yf_0);
                        yb_0 = cscale((l0 & kLkYm) ? 1.f : 0.f, yb_0);
                        yf_1 = cscale((l1 & kLkYp) ? 1.f : 0.f, yf_1);
                        yb_1 = cscale((l1 & kLkYm) ? 1.f : 0.f, yb_1);
                    }
                    float2 ns0 = cmul(xf, c1x), ns1 = cmulc(xf, c0x);
                    cfmac(ns0, xf, xl0);
                    cfma(ns1, xf, xr1);
                    cfma(ns0, yf0, yf_0);
                    cfmac(ns0, yf0, yb_0);
                    cfma(ns1, yf1, yf_1);
                    cfmac(ns1, yf1, yb_1);
                    if (zact) {
                        const float4 pzp = *reinterpret_cast<const float4 *>(&Pp.psi[r + 1][cx]);
                        const float4 pzm = *reinterpret_cast<const float4 *>(&Pm.psi[r + 1][cx]);
                        float4 zpp = pzp, zmm = pzm;
                        if (!zper && (k == 0 || k == g.nz - 1)) {   // an open z face (the whole plane)
                            const float wz_f = (k == 0) ? 2.f : 0.f, wz_b = (k == 0) ? 0.f : 2.f;
                            zpp = make_float4(wz_f * pzp.x, wz_f * pzp.y, wz_f * pzp.z, wz_f * pzp.w);
                            zmm = make_float4(wz_b * pzm.x, wz_b * pzm.y, wz_b * pzm.z, wz_b * pzm.w);
                        }
                        if (MASK) {
                            const float f0 = (lkc.x & kLkZp) ? 1.f : 0.f, b0 = (lkc.x & kLkZm) ? 1.f : 0.f;
                            const float f1 = (lkc.y & kLkZp) ? 1.f : 0.f, b1 = (lkc.y & kLkZm) ? 1.f : 0.f;
                            zpp = make_float4(f0 * zpp.x, f0 * zpp.y, f1 * zpp.z, f1 * zpp.w);
                            zmm = make_float4(b0 * zmm.x, b0 * zmm.y, b1 * zmm.z, b1 * zmm.w);
                        }
                        cfma(ns0, zf0, lo2(zpp));
                        cfmac(ns0, zf0, lo2(zmm));
                        cfma(ns1, zf1, hi2(zpp));
                        cfmac(ns1, zf1, hi2(zmm));
                    }
                    if constexpr (RHS) {
                        // f = Im[conj(psi) NS(psi)] plus the open-x injection terms
                        float f0 = (c0.x * ns0.y - c0.y * ns0.x) * inv_ht2;
                        float f1 = (c1.x * ns1.y - c1.y * ns1.x) * inv_ht2;
                        if (!xper) {
                            if (xlo && !(MASK && (lkc.x & kLkIns))) f0 -= a.inj;
                            if (xhi && !(MASK && (lkc.y & kLkIns))) f1 += a.inj;
                        }
                        *fdp = make_float2(f0, f1);
                        const float wz = (g.bcz == kOpen && g.nz >= 2 && (k == 0 || k == g.nz - 1)) ? 0.5f : 1.f;
                        facc += wz * (wxy0 * f0 + wxy1 * f1);
                    } else {
                        const float2 b0 = lo2(bc), b1 = hi2(bc), D0 = lo2(Dc), D1 = hi2(Dc);
                        const float2 s0 = cadd(b0, ns0), s1 = cadd(b1, ns1);
                        const float2 r0 = csub(s0, cmul(D0, c0)), r1 = csub(s1, cmul(D1, c1));
                        const float2 n0 = cscale(rcp_approx(cabs2(D0)), cmulc(D0, s0));
                        const float2 n1 = cscale(rcp_approx(cabs2(D1)), cmulc(D1, s1));
                        *dp = make_float4(n0.x, n0.y, n1.x, n1.y);
                        float r2a = cabs2(r0), r2b = cabs2(r1);
                        r2a = (r2a <= FLT_MAX) ? r2a : INFINITY;
                        r2b = (r2b <= FLT_MAX) ? r2b : INFINITY;
                        rmax = fmaxf(rmax, fmaxf(r2a, r2b));
                    }
                }
                // the plane below is no longer needed by this warp
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[sm]);
                sm = sc;
                sc = sp;
                if (++sp == NS) {
                    sp = 0;
                    php ^= 1u;
                }
                dp += plq;
                if constexpr (RHS) fdp += plq;
            }
        };
        if (edge) consume(std::true_type{});
        else consume(std::false_type{});
    }
    __syncthreads();
    // A block whose wait ran out records the timeout before it takes its ticket, so the
    // deciding block sees it (the ticket's fence orders the write); it still takes the
    // ticket, so the count returns to zero, and the deciding block ends the solve
    // (sweep_decide keeps TDGL_ERR_TIMEOUT and sets done).  Its partial carries no value.
    if (failed) {
        rmax = 0.f;
        facc = 0.f;
        if (threadIdx.x == 0) *(volatile int *)&a.ctl->status = TDGL_ERR_TIMEOUT;
    }
    const unsigned bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const unsigned nb = gridDim.x * gridDim.y * gridDim.z;
    if constexpr (RHS) finish_rhs_sum_at(a.ctl, a.blockred, (double)facc, a.wsum, bid, nb);
    else finish_sweep_at(a, rmax, false, bid, nb);
}

bool tma_sweep_supported(const DevGrid &g) { return (g.L == nullptr || g.Xj != nullptr) && (g.nx % 2) == 0; }

template <bool RHS>
static size_t tma_smem() { return kStages<RHS> * sizeof(StageT<RHS>) + 2 * kStages<RHS> * sizeof(unsigned long long); }
size_t tma_sweep_smem() { return tma_smem<false>(); }

// Tensor map of one complex64 field (nx, ny, nz) with the given box; false on failure.
void *tma_encode_entry()
{
    static void *fn = nullptr;
    if (!fn) {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !f)
            return nullptr;
        fn = f;
    }
    return fn;
}

bool tma_encode_field(const DevGrid &g, const float2 *base, int box_x, int box_y, CUtensorMap *out)
{
    const auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(tma_encode_entry());
    if (!encode) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
    const cuuint64_t strides[2] = {(cuuint64_t)g.nx * 8, (cuuint64_t)g.nx * g.ny * 8};
    const cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return encode(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, const_cast<float2 *>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool tma_encode_maps(const DevGrid &g, float2 *const psi[3], const float2 *b, const float2 *D, TmaMaps *m)
{
    for (int q = 0; q < 3; ++q)
        if (!tma_encode_field(g, psi[q], kRowP, kTR + 2, &m->psi[q])) return false;
    return tma_encode_field(g, b, kTX, kTR, &m->b) && tma_encode_field(g, D, kTX, kTR, &m->D);
}

static int tma_kz(const DevGrid &g)
{
    const long long bxy = (long long)((g.nx + kTX - 1) / kTX) * ((g.ny + kTR - 1) / kTR);
    long long kz = (bxy * (zhi(g) - zlo(g))) / 1824;   // about 1824 blocks (four waves of three per SM) or more
    if (kz < 2) kz = 2;
    if (kz > 32) kz = 32;
    return (int)kz;
}

template <bool XZ, bool MASK, bool RHS = false>
static cudaError_t launch_variant(const SweepArgs &a, const CUtensorMap &map_psi, const TmaMaps &m, cudaStream_t s)
{
    static bool attr = false;
    const size_t smem = tma_smem<RHS>();
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(sweep_tma_kernel<XZ, MASK, RHS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int kz = tma_kz(a.g);
    const dim3 grid((a.g.nx + kTX - 1) / kTX, (a.g.ny + kTR - 1) / kTR, (zhi(a.g) - zlo(a.g) + kz - 1) / kz);
    sweep_tma_kernel<XZ, MASK, RHS><<<grid, kThreads, smem, s>>>(a, kz, map_psi, m.b, m.D);
    return cudaGetLastError();
}

cudaError_t launch_sweep_tma(const SweepArgs &a, const CUtensorMap &map_psi, const TmaMaps &m, cudaStream_t s)
{
    const bool xz = a.g.Xj != nullptr, mk = a.g.lk != nullptr;
    if (xz && mk) return launch_variant<true, true>(a, map_psi, m, s);
    if (xz) return launch_variant<true, false>(a, map_psi, m, s);
    if (mk) return launch_variant<false, true>(a, map_psi, m, s);
    return launch_variant<false, false>(a, map_psi, m, s);
}

cudaError_t launch_poisson_rhs_tma(const PoissonArgs &pa, const float2 *psi, const CUtensorMap &map_psi,
                                   const TmaMaps &m, cudaStream_t s)
{
    SweepArgs a;
    memset(&a, 0, sizeof(a));
    a.g = pa.g;
    a.ctl = pa.ctl;
    a.blockred = pa.blockred;
    a.src = psi;
    a.f = pa.f;
    a.inj = pa.inject ? (float)(2.0 * pa.Jext / pa.hx) : 0.f;
    a.wsum = pa.wsum;
    a.wait_ns = pa.wait_ns;
    a.extra_tx = pa.extra_tx;
    const bool xz = a.g.Xj != nullptr, mk = a.g.lk != nullptr;
    if (xz && mk) return launch_variant<true, true, true>(a, map_psi, m, s);
    if (xz) return launch_variant<true, false, true>(a, map_psi, m, s);
    if (mk) return launch_variant<false, true, true>(a, map_psi, m, s);
    return launch_variant<false, false, true>(a, map_psi, m, s);
}

}  // namespace tdgl
