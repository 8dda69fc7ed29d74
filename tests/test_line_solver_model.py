"""Models of the index rules of two multigrid kernels, checked on the CPU.

The recursive x-line solve (zebra line Gauss-Seidel) splits a 512-site line over 32
lanes of 16 sites.  The line operator (2 cx + s) - cx (S- + S+) factors as
(cx / rho)(1 - rho S-)(1 - rho S+), so the solve is a forward and a backward first-order
recursion.  On short-decay levels each lane starts them W values before (after) its
chunk (`lane_model`, with the kernel's choice of source lane and element and the
periodic wrap or Neumann mirror at the ends); elsewhere the exact scan over the lanes
(`scan_model`: local recursions from zero, carries by a lane scan, closed-form seeds at
the ends).  Both run in FP32 and are compared with a dense FP64 solve of the line system.

The fused residual and restriction marches a thread over coarse planes, carrying the
residual of fine plane 2K+1 and a window of u rows; `fused_model` replays its plane and
row bookkeeping (wrap, mirror, carry) and must reproduce the full-weighting restriction
of the residual exactly, summed in the same order.
"""
import numpy as np
import pytest

P, OP = 0, 1


def lane_model(E, cx, s, open_, W, C=16):
    """W <= C: each lane warms up over the previous lane's last W values (the next
    lane's first W for the backward recursion); lane 0 and lane 31 of an open line read
    the mirror from their own registers."""
    t = 1 + s / (2 * cx)
    rho = np.float32(t - np.sqrt(t * t - 1))
    rsc = np.float32(rho / cx)
    e = E.astype(np.float32).reshape(32, C)
    e_next0, e_prevlast = e[1, 0], e[30, C - 1]
    wv = np.zeros((32, C), np.float32)
    for lane in range(32):
        w = np.float32(0)
        for m in range(W):
            v = e[(lane - 1) % 32, C - W + m]
            if open_ and lane == 0:
                v = e_next0 if W - m == C else e[0, (W - m) % C]
            w = np.float32(rho * w + v)
        for m in range(C):
            w = np.float32(rho * w + e[lane, m])
            wv[lane, m] = w
    wext = np.zeros(W, np.float32)         # forward recursion continued past the right end
    wc = wv[31, C - 1]
    for d in range(1, W + 1):
        v = e[31, C - 1 - d] if d <= C - 1 else e_prevlast
        wc = np.float32(rho * wc + v)
        wext[d - 1] = wc
    out = np.zeros((32, C), np.float32)
    for lane in range(32):
        z = np.float32(0)
        for m in range(W - 1, -1, -1):
            v = wext[m] if (open_ and lane == 31) else wv[(lane + 1) % 32, m]
            z = np.float32(rho * z + v)
        for m in range(C - 1, -1, -1):
            z = np.float32(rho * z + wv[lane, m])
            out[lane, m] = z * rsc
    return out.ravel(), float(rho)


def scan_model(E, cx, s, open_, C=16):
    """The exact solve: both recursions from zero per lane, the entering values by a scan
    over the lanes (c_L = rho^C c_(L-1) + end_(L-1)), seeded by w(-1) (a weighted sum
    over the extended line) and z(N) (mirror symmetry, or a weighted sum of w)."""
    f32 = np.float32
    N = E.size
    t = 1 + s / (2 * cx)
    rho_d = t - np.sqrt(t * t - 1)
    rho, rsc = f32(rho_d), f32(rho_d / cx)
    P = 2 * N - 2 if open_ else N
    rhoC = [f32(rho_d ** (C * (1 << q))) for q in range(5)]
    gf, gb, l2 = f32(1 / (1 - rho_d ** P)), f32(1 / (1 - rho_d ** 2)), np.log2(rho_d)
    e = E.astype(f32).reshape(32, C)
    ps = np.zeros(32, f32)
    for L in range(32):
        x0, x1 = C * L, C * L + C - 1
        p1 = f32(2.0 ** (l2 * (x0 - 1)))
        p2 = f32(2.0 ** (l2 * ((2 * N - 3 - x1) if open_ else (N - 1 - x1))))
        for m in range(C):
            if open_ and not (L == 0 and m == 0):
                ps[L] = f32(ps[L] + p1 * e[L, m])
            p1 = f32(p1 * rho)
        for m in range(C - 1, -1, -1):
            if not (open_ and L == 31 and m == C - 1):
                ps[L] = f32(ps[L] + p2 * e[L, m])
            p2 = f32(p2 * rho)
    wm1 = f32(f32(ps.sum(dtype=np.float64)) * gf)
    w = np.zeros((32, C), f32)
    for L in range(32):
        acc = f32(0)
        for m in range(C):
            acc = f32(rho * acc + e[L, m])
            w[L, m] = acc
    S = w[:, C - 1].copy()
    for q in range(5):
        prev = S.copy()
        for L in range(1 << q, 32):
            S[L] = f32(prev[L] + rhoC[q] * prev[L - (1 << q)])
    S = np.array([f32(S[L] + f32(2.0 ** (l2 * C * (L + 1))) * wm1) for L in range(32)], f32)
    cin = np.concatenate([[wm1], S[:-1]]).astype(f32)
    for L in range(32):
        p = rho
        for m in range(C):
            w[L, m] = f32(w[L, m] + p * cin[L])
            p = f32(p * rho)
    z = np.zeros((32, C), f32)
    for L in range(32):
        acc = f32(0)
        for m in range(C - 1, -1, -1):
            acc = f32(rho * acc + w[L, m])
            z[L, m] = acc
    if open_:
        zN = f32((rho * w[31, C - 1] + w[31, C - 2]) * gb)
    else:
        pz = np.zeros(32, f32)
        for L in range(32):
            p = f32(2.0 ** (l2 * C * L))
            for m in range(C):
                pz[L] = f32(pz[L] + p * w[L, m])
                p = f32(p * rho)
        zN = f32(f32(pz.sum(dtype=np.float64)) * gf)
    T = z[:, 0].copy()
    for q in range(5):
        prev = T.copy()
        for L in range(32 - (1 << q)):
            T[L] = f32(prev[L] + rhoC[q] * prev[L + (1 << q)])
    T = np.array([f32(T[L] + f32(2.0 ** (l2 * C * (32 - L))) * zN) for L in range(32)], f32)
    din = np.concatenate([T[1:], [zN]]).astype(f32)
    out = np.zeros((32, C), f32)
    for L in range(32):
        p = rho
        for m in range(C - 1, -1, -1):
            out[L, m] = f32(f32(z[L, m] + p * din[L]) * rsc)
            p = f32(p * rho)
    return out.ravel(), float(rho_d)


def dense_line(E, cx, s, open_):
    n = E.size
    A = np.zeros((n, n))
    for i in range(n):
        A[i, i] = 2 * cx + s
        if open_:
            if i == 0:
                A[i, 1] -= 2 * cx
            elif i == n - 1:
                A[i, n - 2] -= 2 * cx
            else:
                A[i, i - 1] -= cx
                A[i, i + 1] -= cx
        else:
            A[i, (i - 1) % n] -= cx
            A[i, (i + 1) % n] -= cx
    return np.linalg.solve(A, E)


# the finest level of a 512-site line at h = 0.5 (shift s = 16 at cx = 4)
@pytest.mark.parametrize("W", [12, 16])
@pytest.mark.parametrize("open_", [False, True])
def test_warm_up_line_solve_model(W, open_):
    E = np.random.default_rng(W).normal(size=512)
    got, rho = lane_model(E, 4.0, 16.0, open_, W)
    assert rho ** W <= 1e-8
    ref = dense_line(E, 4.0, 16.0, open_)
    assert np.abs(got - ref).max() <= 5e-7 * np.abs(ref).max()


# the coarser levels (rho from 0.17 to 0.98, the last far beyond any warm-up)
@pytest.mark.parametrize("s", [16.0, 4.0, 1.0, 0.25, 0.0625, 0.01, 0.001])
@pytest.mark.parametrize("open_", [False, True])
def test_scan_line_solve_model(s, open_):
    E = np.random.default_rng(int(1000 * s)).normal(size=512)
    got, rho = scan_model(E, 4.0, s, open_)
    ref = dense_line(E, 4.0, s, open_)
    assert np.abs(got - ref).max() <= 1e-6 * np.abs(ref).max(), rho


def nb(j, d, n, bc):
    q = j + d
    if bc == P:
        return q % n
    if q < 0:
        q = -q
    if q > n - 1:
        q = 2 * (n - 1) - q
    return q


def coarse_n(n, bc):
    return n // 2 if bc == P else (n - 1) // 2 + 1


def residual(u, r, j, k, bc, cx, cy, cz):
    nz, ny, nx = u.shape
    c = u[k, j]
    fw, bw = np.roll(c, -1), np.roll(c, 1)
    if bc[0] == OP:
        fw[-1], bw[0] = c[-2], c[1]
    lap = cx * (fw + bw - 2 * c)
    lap = lap + cy * (u[k, nb(j, 1, ny, bc[1])] + u[k, nb(j, -1, ny, bc[1])] - 2 * c)
    lap = lap + cz * (u[nb(k, 1, nz, bc[2]), j] + u[nb(k, -1, nz, bc[2]), j] - 2 * c)
    return r[k, j] - lap


def restricted_residual(u, r, bc, c3):
    nz, ny, nx = u.shape
    out = np.zeros((coarse_n(nz, bc[2]), coarse_n(ny, bc[1]), nx))
    for K in range(out.shape[0]):
        for J in range(out.shape[1]):
            acc = 0
            for dk in (-1, 0, 1):
                for dj in (-1, 0, 1):
                    w = (0.5 if dk == 0 else 0.25) * (0.5 if dj == 0 else 0.25)
                    acc = acc + w * residual(u, r, nb(2 * J, dj, ny, bc[1]), nb(2 * K, dk, nz, bc[2]), bc, *c3)
            out[K, J] = acc
    return out


def fused_model(u, r, bc, c3, rz):
    nz, ny, nx = u.shape
    Cz, Cy = coarse_n(nz, bc[2]), coarse_n(ny, bc[1])
    out = np.full((Cz, Cy, nx), np.nan)
    for J in range(Cy):
        rows = [nb(2 * J, d, ny, bc[1]) for d in (-1, 0, 1)]

        def resid3(k, U, Zm, Zp):
            # the window must hold exactly the planes this residual reads
            assert (U, Zm, Zp) == (k, nb(k, -1, nz, bc[2]), nb(k, 1, nz, bc[2]))
            return [residual(u, r, j, k, bc, *c3) for j in rows]

        for Ka in range(0, Cz, rz):
            Kb = min(Ka + rz, Cz)
            pA = nb(2 * Ka, -1, nz, bc[2])
            uA, uB = pA, 2 * Ka
            zm, zp = nb(pA, -1, nz, bc[2]), nb(pA, 1, nz, bc[2])
            tA = resid3(pA, uA, uB if zm == 2 * Ka else zm, uB if zp == 2 * Ka else zp)
            for K in range(Ka, Kb):
                pB = 2 * K
                pC, pN = nb(pB, 1, nz, bc[2]), nb(nb(pB, 1, nz, bc[2]), 1, nz, bc[2])
                uC = uA if pC == pA else pC
                uN = uB if pN == pB else pN
                acc = 0
                for b, t in enumerate(tA):
                    acc = acc + 0.25 * (0.5 if b == 1 else 0.25) * t
                for b, t in enumerate(resid3(pB, uB, uA, uC)):
                    acc = acc + 0.5 * (0.5 if b == 1 else 0.25) * t
                cm = nb(pC, -1, nz, bc[2])
                tA = resid3(pC, uC, uB if cm == pB else cm, uN)
                for b, t in enumerate(tA):
                    acc = acc + 0.25 * (0.5 if b == 1 else 0.25) * t
                out[K, J] = acc
                if K + 1 < Kb:
                    uA, pA = uC, pC
                    uB = uN if pN == pB + 2 else pB + 2
    return out


@pytest.mark.parametrize("bc,ny,nz", [((OP, P, P), 12, 16), ((P, P, P), 8, 8), ((OP, OP, OP), 9, 13),
                                      ((OP, OP, OP), 17, 5), ((P, OP, P), 9, 16), ((OP, P, OP), 16, 9)])
@pytest.mark.parametrize("rz", [1, 3, 4])
def test_fused_residual_restriction_model(bc, ny, nz, rz):
    rng = np.random.default_rng(ny * nz + rz)
    u = rng.normal(size=(nz, ny, 12))
    r = rng.normal(size=(nz, ny, 12))
    c3 = (1.3, 0.7, 0.9)
    assert np.array_equal(fused_model(u, r, bc, c3, rz), restricted_residual(u, r, bc, c3))
