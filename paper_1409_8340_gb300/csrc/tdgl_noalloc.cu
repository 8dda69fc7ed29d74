// Allocation-free entry point: one Jacobi sweep whose scratch lives in a
// file-scope device array instead of a caller-provided workspace.
//
// Who needs it: callers that cannot call cudaMalloc -- code embedded in a host
// application whose memory manager owns the whole device heap and forbids
// direct allocation, or real-time loops that must not allocate once they run --
// but that already hold device buffers for their inputs and outputs.  The
// sweep needs, besides its inputs and outputs, a small control block, the
// Landau link tables and one partial maximum per thread block; all three live
// in tdgl_noalloc_scratch below, which every GPU that loads this library keeps
// until the process exits.
//
// Set-up: the first call on a device, with that device current, looks up the
// device address of the array (cudaGetSymbolAddress); make that first call
// before any stream capture.  Every call overwrites the whole control block
// and the entries of the link tables that its grid reads, so nothing depends on
// what an earlier call left there.
// All calls share the one array: calls that overlap on the GPU (on different
// streams, or from different host threads) race on it and must not be issued.
#include <math.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "tdgl_internal.cuh"

using namespace tdgl;

namespace {

constexpr int kNaMaxAxis = TDGL_NOALLOC_MAX_AXIS;          // largest nx, ny, nz
constexpr size_t kNaMaxBlocks = TDGL_NOALLOC_MAX_BLOCKS;   // per-block partials

struct NaLayout {
    static constexpr size_t ctl = 0;
    static constexpr size_t tables = 512;                                   // Uy, Uz, Py, Pz
    static constexpr size_t blockred = tables + 4 * 8 * (size_t)kNaMaxAxis;
    static constexpr size_t total = blockred + 8 * kNaMaxBlocks;
};
static_assert(sizeof(DevCtl) <= NaLayout::tables, "control block does not fit");

}  // namespace

// The scratch of tdgl_sweep_noalloc (TDGL_NOALLOC_SCRATCH_BYTES bytes).
static __device__ __align__(256) unsigned char tdgl_noalloc_scratch[NaLayout::total];
static_assert(NaLayout::total == TDGL_NOALLOC_SCRATCH_BYTES, "scratch size and header disagree");

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_addr[kMaxDevices];

constexpr double kTwoPi = 6.283185307179586476925286766559;

// Device address of the scratch array for the current device (set up once).
int scratch_address(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TDGL_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, tdgl_noalloc_scratch) != cudaSuccess || !p) return TDGL_ERR_CUDA;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return TDGL_OK;
}

double axis_len(int n, double h, int bc) { return bc == TDGL_PERIODIC ? n * h : (n - 1) * h; }

bool whole_quanta(double B, double L1, double L2, long long *n)
{
    const double q = B * L1 * L2 / kTwoPi, r = floor(q + 0.5);
    *n = (long long)r;
    return fabs(q - r) <= 1e-9 * (1.0 + fabs(q));
}

}  // namespace

extern "C" int tdgl_sweep_noalloc(const tdgl_config *cfg, const float *d_psi_in, const float *d_b, const float *d_D,
                                  double K, float *d_psi_out, double *r2max, void *stream)
{
    if (!cfg || !d_psi_in || !d_b || !d_D || !d_psi_out || d_psi_in == d_psi_out) return TDGL_ERR_INVALID_ARG;
    const tdgl_config &c = *cfg;
    if (c.nx < 2 || c.ny < 2 || c.nz < 1) return TDGL_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a)
        if (c.bc[a] != TDGL_PERIODIC && c.bc[a] != TDGL_OPEN) return TDGL_ERR_INVALID_ARG;
    if (!(c.hx > 0) || !(c.hy > 0) || !(c.hz > 0) || !(c.g > 0) || !(c.ht > 0) || !(c.u > 0))
        return TDGL_ERR_INVALID_ARG;
    if (c.links_mode != TDGL_LINKS_LANDAU) return TDGL_ERR_INVALID_ARG;
    if ((c.bc[0] == TDGL_PERIODIC && c.nx < 3) || (c.bc[1] == TDGL_PERIODIC && c.ny < 3) ||
        (c.bc[2] == TDGL_PERIODIC && c.nz == 2))
        return TDGL_ERR_INVALID_ARG;
    // the fixed-size scratch bounds the problem
    if (c.nx > kNaMaxAxis || c.ny > kNaMaxAxis || c.nz > kNaMaxAxis) return TDGL_ERR_WORKSPACE;
    DevGrid g;
    memset(&g, 0, sizeof(g));
    g.nx = c.nx;
    g.ny = c.ny;
    g.nz = c.nz;
    g.N = (long long)c.nx * c.ny * c.nz;
    if ((size_t)sweep_blocks(g) > kNaMaxBlocks) return TDGL_ERR_WORKSPACE;
    const double Lx = axis_len(c.nx, c.hx, c.bc[0]);
    long long nzq = 0, nyq = 0;
    const bool qy = c.bc[1] == TDGL_PERIODIC && whole_quanta(c.Bz, Lx, axis_len(c.ny, c.hy, c.bc[1]), &nzq);
    const bool qz = c.bc[2] == TDGL_PERIODIC && c.nz >= 2 && whole_quanta(c.By, Lx, axis_len(c.nz, c.hz, c.bc[2]), &nyq);
    if (c.bc[0] == TDGL_PERIODIC && ((c.bc[1] == TDGL_PERIODIC && !qy) || (c.bc[2] == TDGL_PERIODIC && c.nz >= 2 && !qz)))
        return TDGL_ERR_INVALID_ARG;

    void *base = nullptr;
    int rc = scratch_address(&base);
    if (rc != TDGL_OK) return rc;
    unsigned char *sb = static_cast<unsigned char *>(base);
    float2 *tUy = reinterpret_cast<float2 *>(sb + NaLayout::tables);
    float2 *tUz = tUy + kNaMaxAxis, *tPy = tUz + kNaMaxAxis, *tPz = tPy + kNaMaxAxis;
    DevCtl *ctl = reinterpret_cast<DevCtl *>(sb + NaLayout::ctl);

    // link tables of the Landau gauge and the periodic-x wrap phase, in FP64; only the
    // entries the grid uses are built and copied, each table at its fixed offset
    // (the x tables are read in pairs: an odd nx gets one padding entry, exp(0))
    const size_t nxp = (size_t)c.nx + (c.nx & 1);
    std::vector<float2> hUy(nxp, make_float2(1.f, 0.f)), hUz(nxp, make_float2(1.f, 0.f));
    std::vector<float2> hPy((size_t)c.ny), hPz((size_t)c.nz);
    for (int i = 0; i < c.nx; ++i) {
        const double xbar = i * c.hx - 0.5 * Lx;
        const double ay = fmod(-c.hy * c.Bz * xbar, kTwoPi), az = fmod(c.hz * c.By * xbar, kTwoPi);
        hUy[i] = make_float2((float)cos(ay), (float)sin(ay));
        hUz[i] = make_float2((float)cos(az), (float)sin(az));
    }
    for (int j = 0; j < c.ny; ++j) {
        const double ph = qy ? -kTwoPi * (double)(((nzq * j) % c.ny + c.ny) % c.ny) / c.ny
                             : -fmod(j * c.hy * Lx * c.Bz, kTwoPi);
        hPy[j] = make_float2((float)cos(ph), (float)sin(ph));
    }
    for (int k = 0; k < c.nz; ++k) {
        const double ph = qz ? kTwoPi * (double)(((nyq * k) % c.nz + c.nz) % c.nz) / c.nz
                             : fmod(k * c.hz * Lx * c.By, kTwoPi);
        hPz[k] = make_float2((float)cos(ph), (float)sin(ph));
    }
    DevCtl h;
    memset(&h, 0, sizeof(h));
    h.K = K;
    h.Ux = make_float2((float)cos(c.hx * K), (float)sin(c.hx * K));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const std::vector<float2> *tabs[4] = {&hUy, &hUz, &hPy, &hPz};
    float2 *dtabs[4] = {tUy, tUz, tPy, tPz};
    for (int q = 0; q < 4; ++q)
        if (cudaMemcpyAsync(dtabs[q], tabs[q]->data(), sizeof(float2) * tabs[q]->size(), cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
            return TDGL_ERR_CUDA;
    if (cudaMemcpyAsync(ctl, &h, sizeof(h), cudaMemcpyHostToDevice, s) != cudaSuccess) return TDGL_ERR_CUDA;

    const bool zact = c.nz >= 2;
    g.bcx = c.bc[0];
    g.bcy = c.bc[1];
    g.bcz = c.bc[2];
    g.cx = (float)(1.0 / (c.hx * c.hx));
    g.cy = (float)(1.0 / (c.hy * c.hy));
    g.cz = zact ? (float)(1.0 / (c.g * c.g * c.hz * c.hz)) : 0.f;
    g.S = (float)(1.0 / (c.hx * c.hx) + 1.0 / (c.hy * c.hy) + (zact ? 1.0 / (c.g * c.g * c.hz * c.hz) : 0.0));
    g.ht2 = (float)(0.5 * c.ht);
    g.u = (float)c.u;
    g.beta = (float)c.beta;
    g.Uy = tUy;
    g.Uz = tUz;
    g.Py = tPy;
    g.Pz = tPz;
    g.L = nullptr;

    SweepArgs a;
    memset(&a, 0, sizeof(a));
    a.g = g;
    a.ctl = ctl;
    a.blockred = reinterpret_cast<double *>(sb + NaLayout::blockred);
    a.src = reinterpret_cast<const float2 *>(d_psi_in);
    a.dst = reinterpret_cast<float2 *>(d_psi_out);
    a.b = const_cast<float2 *>(reinterpret_cast<const float2 *>(d_b));
    a.D = const_cast<float2 *>(reinterpret_cast<const float2 *>(d_D));
    a.dst_index = 0;
    a.check_every = 1;
    a.fixed_sweeps = 1;
    a.max_iter = 1;
    a.eps = 0.0;
    if (launch_sweep(a, s) != cudaSuccess) return TDGL_ERR_CUDA;
    DevCtl done;
    if (cudaMemcpyAsync(&done, ctl, sizeof(done), cudaMemcpyDeviceToHost, s) != cudaSuccess) return TDGL_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return TDGL_ERR_CUDA;
    if (r2max) *r2max = done.r2;
    return done.status;
}
