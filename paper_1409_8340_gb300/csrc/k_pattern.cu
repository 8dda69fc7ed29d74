// Pattern generator (arXiv:1409.8340, Sec. 3.4): eps(r) from shapes (rectangles,
// cuboids, circles, spheres, ellipsoids, crosses, octants, cylinders), lattices
// of a shape (square, triangular, honeycomb, kagome, rectangular, hexagonal),
// shapes that claim their outside (a shaped integration domain) and
// tessellated backgrounds (checkerboard, Voronoi with the Euclidean, absolute
// or maximum distance).
//
// The paper's sequential rule "add shapes in order until the claimed volume
// reaches the target" is evaluated in parallel: every site records the index
// of the first shape that claims it (atomicMin while rastering each shape's
// bounding box, the boxes of all shapes flattened into one balanced index
// space), a histogram of those indices gives the sites each shape newly
// claims, one block scans it to find how many shapes are taken, and a per-site
// pass writes eps (shape value or background) and the insulating mask.  The
// result equals the sequential rule bit for bit.  The inside tests and the
// background distances run in FP64 with every product and sum rounded
// separately (no fused multiply-add) in a fixed order, so each decision is
// reproducible.
#include <float.h>

#include "philox.cuh"
#include "tdgl_internal.cuh"

namespace tdgl {

__device__ __forceinline__ double dm(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double da(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double ds(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dd(double a, double b) { return __ddiv_rn(a, b); }

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

struct PGrid {
    int n[3], bc[3];
    double h[3];
    long long N;
};

// d = r - c with the minimum image on periodic axes.  When |d| < 0.49 L the image
// shift floor(d / L + 0.5) is 0 whatever the rounding, so the division is skipped
// (the result is the same bits).
__device__ __forceinline__ void min_image(const PGrid &G, const double *c, const int *ijk, double *d)
{
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        d[ax] = ds(dm((double)ijk[ax], G.h[ax]), c[ax]);
        if (G.bc[ax] == kPeriodic) {
            const double L = dm((double)G.n[ax], G.h[ax]);
            if (!(fabs(d[ax]) < 0.49 * L)) d[ax] = ds(d[ax], dm(L, floor(da(dd(d[ax], L), 0.5))));
        }
    }
}

// Per-shape raster data: rotation, bounding box of lattice indices, box volume.
struct ShapeBox {
    double R[9];
    int lo[3], ex[3];
};

__device__ __forceinline__ bool shape_contains(const tdgl_shape &S, const double *R, const double *d)
{
    double e[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) e[b] = da(da(dm(R[b], d[0]), dm(R[3 + b], d[1])), dm(R[6 + b], d[2]));
    const double s0 = dd(e[0], S.a[0]), s1 = dd(e[1], S.a[1]), s2 = dd(e[2], S.a[2]);
    switch (S.kind) {
    case TDGL_SHAPE_ELLIPSOID: return da(da(dm(s0, s0), dm(s1, s1)), dm(s2, s2)) <= 1.0;
    case TDGL_SHAPE_CUBOID: return fabs(e[0]) <= S.a[0] && fabs(e[1]) <= S.a[1] && fabs(e[2]) <= S.a[2];
    case TDGL_SHAPE_CYLINDER: return da(dm(s0, s0), dm(s1, s1)) <= 1.0 && fabs(e[2]) <= S.a[2];
    case TDGL_SHAPE_CROSS:
        return (fabs(e[0]) <= S.a[0] && fabs(e[1]) <= S.a[1] && fabs(e[2]) <= S.a[2]) ||
               (fabs(e[0]) <= S.a[1] && fabs(e[1]) <= S.a[0] && fabs(e[2]) <= S.a[2]);
    case TDGL_SHAPE_OCTANT:
        return e[0] >= 0.0 && e[1] >= 0.0 && e[2] >= 0.0 && da(da(dm(s0, s0), dm(s1, s1)), dm(s2, s2)) <= 1.0;
    default: return false;
    }
}

// ---------------------------------------------------------------------------
// Lattice expansion: one thread per lattice point.
// ---------------------------------------------------------------------------
__global__ void lattice_expand_kernel(const tdgl_lattice *lat, long long count, tdgl_shape *out)
{
    const tdgl_lattice L = *lat;
    const int kind = L.kind;
    const double a = L.spacing[0], s3h = dm(__dsqrt_rn(3.0), 0.5);
    double a1[3] = {a, 0.0, 0.0}, a2[3] = {0.0, a, 0.0}, a3[3] = {0.0, 0.0, L.spacing[2]};
    const bool tri = kind == TDGL_LATTICE_TRIANGULAR || kind == TDGL_LATTICE_HONEYCOMB || kind == TDGL_LATTICE_KAGOME ||
                     kind == TDGL_LATTICE_HEXAGONAL;
    if (tri) {
        a2[0] = dm(0.5, a);
        a2[1] = dm(s3h, a);
    }
    if (kind == TDGL_LATTICE_RECTANGULAR) a2[1] = L.spacing[1];
    const int nb = kind == TDGL_LATTICE_HONEYCOMB ? 2 : (kind == TDGL_LATTICE_KAGOME ? 3 : 1);
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < count;
         p += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(p % nb);
        long long r = p / nb;
        const long long k1 = r % L.count[0];
        r /= L.count[0];
        const long long k2 = r % L.count[1];
        const long long k3 = r / L.count[1];
        double basis[3] = {0.0, 0.0, 0.0};
        if (kind == TDGL_LATTICE_HONEYCOMB && b == 1) {
            basis[0] = dm(0.5, a);
            basis[1] = dd(dm(s3h, a), 3.0);
        } else if (kind == TDGL_LATTICE_KAGOME && b == 1) {
            basis[0] = dm(0.5, a);
        } else if (kind == TDGL_LATTICE_KAGOME && b == 2) {
            basis[0] = dm(0.25, a);
            basis[1] = dm(0.5, dm(s3h, a));
        }
        tdgl_shape S = L.motif;
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            double v = da(L.origin[ax], dm((double)k1, a1[ax]));
            v = da(v, dm((double)k2, a2[ax]));
            v = da(v, dm((double)k3, a3[ax]));
            v = da(v, basis[ax]);
            S.c[ax] = da(v, L.motif.c[ax]);
        }
        out[p] = S;
    }
}

// ---------------------------------------------------------------------------
// Boxes: rotation and the axis-aligned box of grid indices that can hold a
// claimed site (the whole grid for inverted shapes); work[n] = box volume.
// ---------------------------------------------------------------------------
__global__ void shape_box_kernel(PGrid G, const tdgl_shape *shapes, long long n_shapes, ShapeBox *boxes,
                                 long long *work)
{
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < n_shapes;
         n += (long long)gridDim.x * blockDim.x) {
        const tdgl_shape S = shapes[n];
        ShapeBox B;
        quat_rot(S.q, B.R);
        double r[3] = {S.a[0], S.a[1], S.a[2]};
        if (S.kind == TDGL_SHAPE_CROSS) r[0] = r[1] = fmax(S.a[0], S.a[1]);
        long long vol = 1;
        for (int ax = 0; ax < 3; ++ax) {
            int lo, hi;
            if (S.flags & TDGL_SHAPE_INVERT) {
                lo = 0;
                hi = G.n[ax] - 1;
            } else {
                // |d_ax| <= sum_b |R_ax,b| r_b, widened far beyond rounding
                double ext = fabs(B.R[3 * ax]) * r[0] + fabs(B.R[3 * ax + 1]) * r[1] + fabs(B.R[3 * ax + 2]) * r[2];
                ext = ext * (1.0 + 1e-9) + 1e-9 * G.h[ax];
                // on a periodic axis the box is placed around the centre's image in [0, L)
                double c = S.c[ax];
                if (G.bc[ax] == kPeriodic) {
                    const double L = G.n[ax] * G.h[ax];
                    c = c - L * floor(c / L);
                }
                const double flo = ceil((c - ext) / G.h[ax]), fhi = floor((c + ext) / G.h[ax]);
                if (G.bc[ax] == kOpen) {
                    // clamp before the conversion: the box may lie far outside the grid
                    lo = (int)fmin(fmax(flo, 0.0), (double)G.n[ax]);
                    hi = (int)fmax(fmin(fhi, (double)(G.n[ax] - 1)), -1.0);
                } else if (!(fhi - flo + 1.0 <= (double)G.n[ax])) {
                    lo = 0;
                    hi = G.n[ax] - 1;
                } else {
                    lo = (int)flo;
                    hi = (int)fhi;
                }
            }
            B.lo[ax] = lo;
            B.ex[ax] = hi >= lo ? hi - lo + 1 : 0;
            vol *= B.ex[ax];
        }
        boxes[n] = B;
        work[n] = vol;
    }
}

// Exclusive scan of work[0..n) into off[0..n] by one block (n up to 2^31).
__global__ void scan_kernel(const long long *work, long long n, long long *off)
{
    __shared__ long long part[1024];
    const int t = threadIdx.x, T = blockDim.x;
    const long long chunk = (n + T - 1) / T;
    const long long b = t * chunk, e = min(n, b + chunk);
    long long s = 0;
    for (long long i = b; i < e; ++i) s += work[i];
    part[t] = s;
    __syncthreads();
    if (t == 0) {
        long long acc = 0;
        for (int i = 0; i < T; ++i) {
            long long v = part[i];
            part[i] = acc;
            acc += v;
        }
        off[n] = acc;
    }
    __syncthreads();
    long long acc = part[t];
    for (long long i = b; i < e; ++i) {
        off[i] = acc;
        acc += work[i];
    }
}

// Raster: every (shape, box cell) pair of the flattened index space.
__global__ void raster_kernel(PGrid G, const tdgl_shape *shapes, const ShapeBox *boxes, const long long *off,
                              long long n_shapes, int *first)
{
    const long long total = off[n_shapes];
    for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < total;
         w += (long long)gridDim.x * blockDim.x) {
        long long lo = 0, hi = n_shapes - 1;   // last n with off[n] <= w
        while (lo < hi) {
            const long long mid = (lo + hi + 1) >> 1;
            if (off[mid] <= w) lo = mid;
            else hi = mid - 1;
        }
        const long long n = lo;
        const ShapeBox &B = boxes[n];
        const long long e = w - off[n];
        const int ii = B.lo[0] + (int)(e % B.ex[0]);
        const int jj = B.lo[1] + (int)((e / B.ex[0]) % B.ex[1]);
        const int kk = B.lo[2] + (int)(e / ((long long)B.ex[0] * B.ex[1]));
        const int ijk[3] = {wrapi(ii, G.n[0]), wrapi(jj, G.n[1]), wrapi(kk, G.n[2])};
        const tdgl_shape &S = shapes[n];
        double d[3];
        min_image(G, S.c, ijk, d);
        const bool in = shape_contains(S, B.R, d);
        if (in != ((S.flags & TDGL_SHAPE_INVERT) != 0)) {
            const long long m = (long long)ijk[0] + (long long)G.n[0] * ((long long)ijk[1] + (long long)G.n[1] * ijk[2]);
            atomicMin(first + m, (int)n);
        }
    }
}

// Sites newly claimed per shape, one atomic per run of equal owners in a warp.
__global__ void histogram_kernel(const int *first, long long N, long long n_shapes, unsigned long long *counts)
{
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long base = warp * 32; base < N; base += nwarps * 32) {
        const long long m = base + lane;
        int f = (m < N) ? first[m] : -1;
        if (f < 0 || (long long)f >= n_shapes) f = -1;
        const unsigned peers = __match_any_sync(0xffffffffu, f);
        if (f >= 0 && lane == __ffs(peers) - 1) atomicAdd(counts + f, (unsigned long long)__popc(peers));
    }
}

// Sequential rule: shape n is taken while fewer than `target` sites are claimed.
__global__ void select_kernel(const unsigned long long *counts, long long n_shapes, long long target, long long *result)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    long long marked = 0, used = 0;
    for (long long n = 0; n < n_shapes; ++n) {
        if (target > 0 && marked >= target) break;
        marked += (long long)counts[n];
        used = n + 1;
    }
    result[0] = used;
    result[1] = marked;
}

// ---------------------------------------------------------------------------
// Voronoi buckets: a uniform grid over the box, about two seeds per bucket.
// ---------------------------------------------------------------------------
struct VoronoiArgs {
    const double *seeds;   // n x (x, y, z, value), as given
    long long n;
    int metric;
    int nb[3];             // buckets per axis
    double bw[3];          // bucket widths
    double bwmin;          // smallest width over axes with more than one bucket (0: none)
    int *start;            // [nbtot + 1] first entry of each bucket in `order`
    int *cursor;           // [nbtot] fill cursor
    int *order;            // [n] seed indices grouped by bucket
};

__device__ __forceinline__ int bucket_of(const VoronoiArgs &V, const PGrid &G, int ax, double x)
{
    if (G.bc[ax] == kPeriodic) {
        const double L = G.n[ax] * G.h[ax];
        x = x - L * floor(x / L);
    }
    int b = (int)floor(x / V.bw[ax]);
    return b < 0 ? 0 : (b >= V.nb[ax] ? V.nb[ax] - 1 : b);
}

__device__ __forceinline__ int seed_bucket(const VoronoiArgs &V, const PGrid &G, long long s)
{
    const double *p = V.seeds + 4 * s;
    return bucket_of(V, G, 0, p[0]) + V.nb[0] * (bucket_of(V, G, 1, p[1]) + V.nb[1] * bucket_of(V, G, 2, p[2]));
}

__global__ void voronoi_count_kernel(VoronoiArgs V, PGrid G)
{
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < V.n; s += (long long)gridDim.x * blockDim.x)
        atomicAdd(V.start + seed_bucket(V, G, s), 1);
}

// exclusive scan of the bucket counts in place (start[nbtot] = n), one block
__global__ void voronoi_scan_kernel(VoronoiArgs V, int nbtot)
{
    __shared__ int part[1024];
    const int t = threadIdx.x, T = blockDim.x;
    const int chunk = (nbtot + T - 1) / T;
    const int b = t * chunk, e = min(nbtot, b + chunk);
    int s = 0;
    for (int i = b; i < e; ++i) s += V.start[i];
    part[t] = s;
    __syncthreads();
    if (t == 0) {
        int acc = 0;
        for (int i = 0; i < T; ++i) {
            int v = part[i];
            part[i] = acc;
            acc += v;
        }
        V.start[nbtot] = acc;
    }
    __syncthreads();
    int acc = part[t];
    for (int i = b; i < e; ++i) {
        const int v = V.start[i];
        V.start[i] = acc;
        V.cursor[i] = acc;
        acc += v;
    }
}

__global__ void voronoi_fill_kernel(VoronoiArgs V, PGrid G)
{
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < V.n; s += (long long)gridDim.x * blockDim.x)
        V.order[atomicAdd(V.cursor + seed_bucket(V, G, s), 1)] = (int)s;
}

__device__ __forceinline__ double metric_value(int metric, const double *d)
{
    if (metric == TDGL_METRIC_EUCLIDEAN) return da(da(dm(d[0], d[0]), dm(d[1], d[1])), dm(d[2], d[2]));
    if (metric == TDGL_METRIC_ABSOLUTE) return da(da(fabs(d[0]), fabs(d[1])), fabs(d[2]));
    return fmax(fmax(fabs(d[0]), fabs(d[1])), fabs(d[2]));
}

// Nearest seed of a site: buckets in Chebyshev shells s = 0, 1, ... around the
// site's bucket.  A seed outside shells 0..s is at least s * bwmin away along
// some axis, so the search ends once the best value is below that bound (with
// a margin far above rounding), or when every bucket has been seen.
__device__ long long voronoi_owner(const VoronoiArgs &V, const PGrid &G, const int *ijk)
{
    int b0[3];
    double r[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        r[ax] = dm((double)ijk[ax], G.h[ax]);
        b0[ax] = bucket_of(V, G, ax, r[ax]);
    }
    const int smax = max(V.nb[0], max(V.nb[1], V.nb[2]));
    long long best = -1;
    double bv = 0.0;
    for (int s = 0; s <= smax; ++s) {
        int olo[3], ohi[3];
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            olo[ax] = -s;
            ohi[ax] = s;
            if (G.bc[ax] != kPeriodic || V.nb[ax] == 1) {   // clip to the axis (open, or a single bucket)
                olo[ax] = max(-s, -b0[ax]);
                ohi[ax] = min(s, V.nb[ax] - 1 - b0[ax]);
            } else if (2 * s + 1 > V.nb[ax]) {               // the shell wraps onto itself: each bucket once
                olo[ax] = -(V.nb[ax] / 2);
                ohi[ax] = olo[ax] + V.nb[ax] - 1;
            }
        }
        for (int oz = olo[2]; oz <= ohi[2]; ++oz)
            for (int oy = olo[1]; oy <= ohi[1]; ++oy)
                for (int ox = olo[0]; ox <= ohi[0]; ++ox) {
                    if (max(abs(ox), max(abs(oy), abs(oz))) != s) continue;
                    const int bx = wrapi(b0[0] + ox, V.nb[0]), by = wrapi(b0[1] + oy, V.nb[1]);
                    const int bz = wrapi(b0[2] + oz, V.nb[2]);
                    const int bk = bx + V.nb[0] * (by + V.nb[1] * bz);
                    for (int q = V.start[bk]; q < V.start[bk + 1]; ++q) {
                        const long long si = V.order[q];
                        double d[3];
                        min_image(G, V.seeds + 4 * si, ijk, d);
                        const double v = metric_value(V.metric, d);
                        if (best < 0 || v < bv || (v == bv && si < best)) {
                            best = si;
                            bv = v;
                        }
                    }
                }
        if (V.bwmin <= 0.0) break;   // one bucket per axis: all seen
        if (best >= 0) {
            const double g = s * V.bwmin;
            const double bound = (V.metric == TDGL_METRIC_EUCLIDEAN) ? g * g : g;
            if (bv < bound * (1.0 - 1e-9)) break;
        }
    }
    return best;
}

// ---------------------------------------------------------------------------
// Per-site output: the claiming shape's value, else the background.
// ---------------------------------------------------------------------------
struct BgArgs {
    int kind;
    double value, cell[3], values[2], p_odd;
    unsigned long long seed;
    long long nc[3];
};

__device__ __forceinline__ double checker_at(const BgArgs &B, const PGrid &G, const int *ijk)
{
    long long ci[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax)
        ci[ax] = B.cell[ax] > 0.0 ? (long long)floor(dd(dm((double)ijk[ax], G.h[ax]), B.cell[ax])) : 0;
    if (B.p_odd < 0.0) return ((ci[0] + ci[1] + ci[2]) & 1) ? B.values[1] : B.values[0];
    const unsigned long long cidx = (unsigned long long)(ci[0] + B.nc[0] * (ci[1] + B.nc[1] * ci[2]));
    unsigned int x[4];
    philox4x32_10((unsigned int)cidx, (unsigned int)(cidx >> 32), 0u, 0x4B434548u, (unsigned int)B.seed,
                  (unsigned int)(B.seed >> 32), x);
    const double u = (double)(x[0] >> 8) * 0x1p-24;
    return (u < B.p_odd) ? B.values[1] : B.values[0];
}

__global__ void output_kernel(PGrid G, const int *first, const long long *result, const tdgl_shape *shapes, BgArgs B,
                              VoronoiArgs V, float *alpha, unsigned char *insulating)
{
    const long long used = result[0];
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < G.N; m += (long long)gridDim.x * blockDim.x) {
        const int f = first[m];
        if ((long long)f < used) {
            alpha[m] = (float)shapes[f].value;
            if (insulating) insulating[m] = (shapes[f].flags & TDGL_SHAPE_INSULATING) ? 1 : 0;
            continue;
        }
        if (insulating) insulating[m] = 0;
        const int ijk[3] = {(int)(m % G.n[0]), (int)((m / G.n[0]) % G.n[1]), (int)(m / ((long long)G.n[0] * G.n[1]))};
        double v = B.value;
        if (B.kind == TDGL_BG_CHECKER) v = checker_at(B, G, ijk);
        else if (B.kind == TDGL_BG_VORONOI) {
            const long long own = voronoi_owner(V, G, ijk);
            if (own >= 0) v = V.seeds[4 * own + 3];
        }
        alpha[m] = (float)v;
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
namespace {

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

int lattice_basis(int kind) { return kind == TDGL_LATTICE_HONEYCOMB ? 2 : (kind == TDGL_LATTICE_KAGOME ? 3 : 1); }

long long lattice_count(const tdgl_lattice &L)
{
    return (long long)L.count[0] * L.count[1] * L.count[2] * lattice_basis(L.kind);
}

bool finite3(const double *v) { return isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]); }

bool shape_ok(const tdgl_shape &S)
{
    if (S.kind < TDGL_SHAPE_ELLIPSOID || S.kind > TDGL_SHAPE_OCTANT) return false;
    if (S.flags & ~(TDGL_SHAPE_INVERT | TDGL_SHAPE_INSULATING)) return false;
    if (!finite3(S.c) || !finite3(S.a) || !isfinite(S.value)) return false;
    if (!(S.a[0] > 0) || !(S.a[1] > 0) || !(S.a[2] > 0)) return false;
    const double n2 = S.q[0] * S.q[0] + S.q[1] * S.q[1] + S.q[2] * S.q[2] + S.q[3] * S.q[3];
    return isfinite(n2) && fabs(n2 - 1.0) <= 1e-6;
}

struct VoronoiPlan {
    int nb[3];
    double bw[3], bwmin;
    long long nbtot;
};

VoronoiPlan voronoi_plan(const PGrid &G, long long n_seeds)
{
    VoronoiPlan P;
    double ext[3];
    int dims = 0;
    double vol = 1.0;
    for (int ax = 0; ax < 3; ++ax) {
        ext[ax] = G.bc[ax] == kPeriodic ? G.n[ax] * G.h[ax] : (G.n[ax] - 1) * G.h[ax];
        if (G.n[ax] >= 2 && ext[ax] > 0) {
            ++dims;
            vol *= ext[ax];
        }
    }
    const double target = n_seeds > 2 ? (double)n_seeds / 2.0 : 1.0;
    const double w = dims > 0 ? pow(vol / target, 1.0 / dims) : 1.0;
    P.nbtot = 1;
    P.bwmin = 0.0;
    for (int ax = 0; ax < 3; ++ax) {
        int nb = 1;
        if (G.n[ax] >= 2 && ext[ax] > 0) {
            double q = floor(ext[ax] / w);
            nb = q < 1 ? 1 : (q > 256 ? 256 : (int)q);
        }
        P.nb[ax] = nb;
        P.bw[ax] = (G.n[ax] >= 2 && ext[ax] > 0) ? ext[ax] / nb : 1.0;
        if (nb > 1 && (P.bwmin == 0.0 || P.bw[ax] < P.bwmin)) P.bwmin = P.bw[ax];
        P.nbtot *= nb;
    }
    return P;
}

struct ExLayout {
    size_t first, counts, work, off, boxes, shapes, lats, result, seeds, start, cursor, order, total;
};

ExLayout ex_layout(const PGrid &G, long long ntot, int n_lattices, long long n_seeds)
{
    ExLayout L;
    size_t o = 0;
    auto take = [&](size_t b) {
        size_t r = o;
        o = al256(o + b);
        return r;
    };
    L.first = take(4 * (size_t)G.N);
    L.counts = take(8 * (size_t)ntot + 8);
    L.work = take(8 * (size_t)ntot + 8);
    L.off = take(8 * (size_t)ntot + 16);
    L.boxes = take(sizeof(ShapeBox) * (size_t)ntot + 8);
    L.shapes = take(sizeof(tdgl_shape) * (size_t)ntot + 8);
    L.lats = take(sizeof(tdgl_lattice) * (size_t)n_lattices + 8);
    L.result = take(16);
    const VoronoiPlan P = voronoi_plan(G, n_seeds);
    L.seeds = take(32 * (size_t)n_seeds + 8);
    L.start = n_seeds > 0 ? take(4 * (size_t)P.nbtot + 8) : take(8);
    L.cursor = n_seeds > 0 ? take(4 * (size_t)P.nbtot + 8) : take(8);
    L.order = take(4 * (size_t)n_seeds + 8);
    L.total = o;
    return L;
}

bool grid_ok(const tdgl_config *g)
{
    if (!g || g->nx < 1 || g->ny < 1 || g->nz < 1) return false;
    if (!(g->hx > 0) || !(g->hy > 0) || !(g->hz > 0)) return false;
    for (int a = 0; a < 3; ++a)
        if (g->bc[a] != TDGL_PERIODIC && g->bc[a] != TDGL_OPEN) return false;
    return true;
}

PGrid pgrid(const tdgl_config *g)
{
    PGrid G;
    G.n[0] = g->nx;
    G.n[1] = g->ny;
    G.n[2] = g->nz;
    for (int a = 0; a < 3; ++a) G.bc[a] = g->bc[a];
    G.h[0] = g->hx;
    G.h[1] = g->hy;
    G.h[2] = g->hz;
    G.N = (long long)g->nx * g->ny * g->nz;
    return G;
}

// total shapes, or -1 on invalid lattices
long long total_shapes(long long n_shapes, const tdgl_lattice *lats, int n_lattices)
{
    if (n_shapes < 0 || n_lattices < 0 || (n_lattices > 0 && !lats)) return -1;
    long long t = n_shapes;
    for (int l = 0; l < n_lattices; ++l) {
        const tdgl_lattice &L = lats[l];
        if (L.kind < TDGL_LATTICE_SQUARE || L.kind > TDGL_LATTICE_HEXAGONAL) return -1;
        if (L.count[0] < 1 || L.count[1] < 1 || L.count[2] < 1) return -1;
        if (!finite3(L.origin) || !finite3(L.spacing) || !(L.spacing[0] > 0)) return -1;
        if (L.kind == TDGL_LATTICE_RECTANGULAR && !(L.spacing[1] > 0)) return -1;
        if (L.count[2] > 1 && !(L.spacing[2] > 0)) return -1;
        if (!shape_ok(L.motif)) return -1;
        const long long c = lattice_count(L);
        if (c > 0x7ffffff0LL) return -1;
        t += c;
        if (t > 0x7ffffff0LL) return -1;
    }
    return t;
}

bool bg_ok(const tdgl_background *bg)
{
    if (!bg) return true;
    if (bg->kind == TDGL_BG_CONSTANT) return isfinite(bg->value);
    if (bg->kind == TDGL_BG_CHECKER)
        return isfinite(bg->values[0]) && isfinite(bg->values[1]) && finite3(bg->cell) && bg->p_odd <= 1.0 &&
               !(bg->p_odd != bg->p_odd);
    if (bg->kind == TDGL_BG_VORONOI) {
        if (bg->n_seeds < 1 || bg->n_seeds > 0x7ffffff0LL || !bg->host_seeds) return false;
        if (bg->metric < TDGL_METRIC_EUCLIDEAN || bg->metric > TDGL_METRIC_MAXIMUM) return false;
        for (long long s = 0; s < 4 * bg->n_seeds; ++s)
            if (!isfinite(bg->host_seeds[s])) return false;
        return true;
    }
    return false;
}

int grid_blocks(long long work, int cap)
{
    long long b = (work + 255) / 256;
    if (b < 1) b = 1;
    return (int)(b > cap ? cap : b);
}

}  // namespace

size_t pattern_ex_scratch(const tdgl_config *grid, int64_t n_shapes, const tdgl_lattice *lats, int32_t n_lattices,
                          const tdgl_background *bg)
{
    if (!grid_ok(grid) || !bg_ok(bg)) return 0;
    const long long ntot = total_shapes(n_shapes, lats, n_lattices);
    if (ntot < 0) return 0;
    const long long ns = (bg && bg->kind == TDGL_BG_VORONOI) ? bg->n_seeds : 0;
    return ex_layout(pgrid(grid), ntot, n_lattices, ns).total;
}

int pattern_ex_run(const tdgl_config *grid, const tdgl_shape *shapes, int64_t n_shapes, const tdgl_lattice *lats,
                   int32_t n_lattices, const tdgl_background *bg, int64_t target, float *d_alpha,
                   uint8_t *d_insulating, void *d_scratch, size_t scratch_bytes, cudaStream_t s, int64_t *n_used,
                   int64_t *n_marked)
{
    if (!grid_ok(grid) || !d_alpha || !bg_ok(bg) || (n_shapes > 0 && !shapes)) return TDGL_ERR_INVALID_ARG;
    const long long ntot = total_shapes(n_shapes, lats, n_lattices);
    if (ntot < 0) return TDGL_ERR_INVALID_ARG;
    for (int64_t n = 0; n < n_shapes; ++n)
        if (!shape_ok(shapes[n])) return TDGL_ERR_INVALID_ARG;
    const PGrid G = pgrid(grid);
    const long long ns = (bg && bg->kind == TDGL_BG_VORONOI) ? bg->n_seeds : 0;
    const ExLayout L = ex_layout(G, ntot, n_lattices, ns);
    if (!d_scratch || ((uintptr_t)d_scratch & 255u) || scratch_bytes < L.total) return TDGL_ERR_WORKSPACE;

    char *base = static_cast<char *>(d_scratch);
    int *first = reinterpret_cast<int *>(base + L.first);
    unsigned long long *counts = reinterpret_cast<unsigned long long *>(base + L.counts);
    long long *work = reinterpret_cast<long long *>(base + L.work);
    long long *off = reinterpret_cast<long long *>(base + L.off);
    ShapeBox *boxes = reinterpret_cast<ShapeBox *>(base + L.boxes);
    tdgl_shape *dsh = reinterpret_cast<tdgl_shape *>(base + L.shapes);
    tdgl_lattice *dlat = reinterpret_cast<tdgl_lattice *>(base + L.lats);
    long long *result = reinterpret_cast<long long *>(base + L.result);

    int rc = TDGL_OK;
    auto chk = [&](cudaError_t e) {
        if (e != cudaSuccess && rc == TDGL_OK) rc = TDGL_ERR_CUDA;
    };
    chk(cudaMemsetAsync(first, 0x7F, 4 * (size_t)G.N, s));
    if (ntot > 0) chk(cudaMemsetAsync(counts, 0, 8 * (size_t)ntot, s));
    if (n_shapes > 0) chk(cudaMemcpyAsync(dsh, shapes, sizeof(tdgl_shape) * (size_t)n_shapes, cudaMemcpyHostToDevice, s));
    if (n_lattices > 0)
        chk(cudaMemcpyAsync(dlat, lats, sizeof(tdgl_lattice) * (size_t)n_lattices, cudaMemcpyHostToDevice, s));
    long long at = n_shapes;
    for (int l = 0; l < n_lattices; ++l) {
        const long long c = lattice_count(lats[l]);
        lattice_expand_kernel<<<grid_blocks(c, 4096), 256, 0, s>>>(dlat + l, c, dsh + at);
        chk(cudaGetLastError());
        at += c;
    }
    if (ntot > 0) {
        shape_box_kernel<<<grid_blocks(ntot, 4096), 256, 0, s>>>(G, dsh, ntot, boxes, work);
        scan_kernel<<<1, 1024, 0, s>>>(work, ntot, off);
        raster_kernel<<<152 * 16, 256, 0, s>>>(G, dsh, boxes, off, ntot, first);
        histogram_kernel<<<grid_blocks(G.N, 152 * 16), 256, 0, s>>>(first, G.N, ntot, counts);
        chk(cudaGetLastError());
    }
    select_kernel<<<1, 32, 0, s>>>(counts, ntot, target, result);

    BgArgs B;
    memset(&B, 0, sizeof(B));
    B.kind = bg ? bg->kind : TDGL_BG_CONSTANT;
    B.value = bg ? bg->value : 1.0;
    if (bg) {
        for (int a = 0; a < 3; ++a) B.cell[a] = bg->cell[a];
        B.values[0] = bg->values[0];
        B.values[1] = bg->values[1];
        B.p_odd = bg->p_odd;
        B.seed = bg->seed;
        for (int a = 0; a < 3; ++a)
            B.nc[a] = B.cell[a] > 0.0 ? (long long)floor(((G.n[a] - 1) * G.h[a]) / B.cell[a]) + 1 : 1;
    }
    VoronoiArgs V;
    memset(&V, 0, sizeof(V));
    if (ns > 0) {
        const VoronoiPlan P = voronoi_plan(G, ns);
        V.seeds = reinterpret_cast<const double *>(base + L.seeds);
        V.n = ns;
        V.metric = bg->metric;
        for (int a = 0; a < 3; ++a) {
            V.nb[a] = P.nb[a];
            V.bw[a] = P.bw[a];
        }
        V.bwmin = P.bwmin;
        V.start = reinterpret_cast<int *>(base + L.start);
        V.cursor = reinterpret_cast<int *>(base + L.cursor);
        V.order = reinterpret_cast<int *>(base + L.order);
        chk(cudaMemcpyAsync(base + L.seeds, bg->host_seeds, 32 * (size_t)ns, cudaMemcpyHostToDevice, s));
        chk(cudaMemsetAsync(V.start, 0, 4 * (size_t)(P.nbtot + 1), s));
        voronoi_count_kernel<<<grid_blocks(ns, 4096), 256, 0, s>>>(V, G);
        voronoi_scan_kernel<<<1, 1024, 0, s>>>(V, (int)P.nbtot);
        voronoi_fill_kernel<<<grid_blocks(ns, 4096), 256, 0, s>>>(V, G);
        chk(cudaGetLastError());
    }
    output_kernel<<<grid_blocks(G.N, 152 * 16), 256, 0, s>>>(G, first, result, dsh, B, V, d_alpha, d_insulating);
    chk(cudaGetLastError());
    long long res[2] = {0, 0};
    chk(cudaMemcpyAsync(res, result, 16, cudaMemcpyDeviceToHost, s));
    chk(cudaStreamSynchronize(s));
    if (rc != TDGL_OK) return rc;
    if (n_used) *n_used = res[0];
    if (n_marked) *n_marked = res[1];
    return TDGL_OK;
}

}  // namespace tdgl
