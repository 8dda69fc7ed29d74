"""Models of the index rules of two multigrid kernels, checked on the CPU.

The recursive x-line solve (zebra line Gauss-Seidel on levels with short decay) splits
a 512-site line over 32 lanes of 16 sites.  The line operator (2 cx + s) - cx (S- + S+)
factors as (cx / rho)(1 - rho S-)(1 - rho S+), so the solve is a forward and a backward
first-order recursion; each lane starts them W values before (after) its chunk, taking
those values from the lanes that hold them, with the periodic wrap or the Neumann mirror
at the line's ends.  `lane_model` follows the kernel's choice of source lane and element
for every warm-up value (one, two or three lanes, both ends) in FP32, and is compared
with a dense FP64 solve of the line system.

The fused residual and restriction marches a thread over coarse planes, carrying the
residual of fine plane 2K+1 and a window of u rows; `fused_model` replays its plane and
row bookkeeping (wrap, mirror, carry) and must reproduce the full-weighting restriction
of the residual exactly, summed in the same order.
"""
import numpy as np
import pytest

P, OP = 0, 1


def lane_model(E, cx, s, open_, W, C=16):
    t = 1 + s / (2 * cx)
    rho = np.float32(t - np.sqrt(t * t - 1))
    rsc = np.float32(rho / cx)
    e = E.astype(np.float32).reshape(32, C)
    e_next0, e_prevlast = e[1, 0], e[30, C - 1]
    wv = np.zeros((32, C), np.float32)
    for lane in range(32):
        w = np.float32(0)
        for m in range(W):
            if W <= C:
                v = e[(lane - 1) % 32, C - W + m]
                if open_ and lane == 0:
                    v = e_next0 if W - m == C else e[0, (W - m) % C]
            else:
                dl = 3 if m < W - 2 * C else (2 if m < W - C else 1)
                v = e[(lane - dl) % 32, m - W + dl * C]
                d = W - m - lane * C      # -x for the mirror
                if open_ and d > 0:
                    v = e[d // C, (W - m) % C]
            w = np.float32(rho * w + v)
        for m in range(C):
            w = np.float32(rho * w + e[lane, m])
            wv[lane, m] = w
    wext = np.zeros(W, np.float32)         # forward recursion continued past the right end
    wc = wv[31, C - 1]
    for d in range(1, W + 1):
        pos = 32 * C - 1 - d
        v = e[pos // C, pos % C] if W > C else (e[31, C - 1 - d] if d <= C - 1 else e_prevlast)
        wc = np.float32(rho * wc + v)
        wext[d - 1] = wc
    out = np.zeros((32, C), np.float32)
    for lane in range(32):
        z = np.float32(0)
        for m in range(W - 1, -1, -1):
            v = wv[(lane + 1 + m // C) % 32, m % C]
            if open_:
                for back in range(3):         # lanes 31, 30, 29 read past the end
                    if lane == 31 - back and m >= back * C:
                        v = wext[m - back * C]
            z = np.float32(rho * z + v)
        for m in range(C - 1, -1, -1):
            z = np.float32(rho * z + wv[lane, m])
            out[lane, m] = z * rsc
    return out.ravel(), float(rho)


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


# (W, shift s at cx = 4): the levels of a 512-site line at h = 0.5 and their warm-ups
@pytest.mark.parametrize("W,s", [(12, 16.0), (16, 16.0), (24, 4.0), (32, 4.0), (40, 1.0), (48, 1.0)])
@pytest.mark.parametrize("open_", [False, True])
def test_recursive_line_solve_model(W, s, open_):
    E = np.random.default_rng(W + int(4 * s)).normal(size=512)
    got, rho = lane_model(E, 4.0, s, open_, W)
    assert rho ** W <= 1e-8
    ref = dense_line(E, 4.0, s, open_)
    assert np.abs(got - ref).max() <= 5e-7 * np.abs(ref).max()


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
