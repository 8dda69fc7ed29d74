"""Thermal noise of the oracle (Sec. 3.1.2) against what the paper fixes.

The noise enters b as h_t zeta, zeta = zeta_max (v1 + i v2) with v1, v2
independent and uniform on [-1, 1), fresh per site and step; zeta_max =
(T_zeta / (h_t hx hy hz))^(1/2).  Pins: the uniform law of the generated values
(moments, histogram), independence across sites, components and steps, and
the paper's diffusion-limit correlator <|psi|^2> = (2/3) zeta_max^2 h_t t / u^2
for noise-only dynamics (Sec. 3.1.2, the discrete correlator G_ii).
"""
import math

import numpy as np
import pytest

P = 0


def noise_values(O, n, seed, step):
    G = O.Grid(n, 1, 1, hx=1.0, hy=1.0, hz=1.0, ht=1.0, noise_T=1.0, noise_seed=seed)   # amp = 1
    b = np.zeros((1, 1, n), dtype=np.complex128)
    O.add_noise(G, b, step)
    return b.ravel()


def test_uniform_law_of_the_generated_values(O):
    from scipy import stats
    z = noise_values(O, 1 << 16, seed=12345, step=7)
    v = np.concatenate([z.real, z.imag])
    assert v.min() >= -1.0 and v.max() < 1.0
    # exact grid of the 24-bit construction
    assert np.all(np.round((v + 1.0) * 2 ** 23) == (v + 1.0) * 2 ** 23)
    n = v.size
    assert abs(v.mean()) < 5 * math.sqrt(1 / 3 / n)
    assert abs(v.var() - 1 / 3) < 5 * math.sqrt(4 / 45 / n)
    hist, _ = np.histogram(v, bins=64, range=(-1, 1))
    assert stats.chisquare(hist).pvalue > 1e-5


def test_independence_across_components_sites_steps_and_seeds(O):
    n = 1 << 15
    a = noise_values(O, n, seed=99, step=0)
    b = noise_values(O, n, seed=99, step=1)
    c = noise_values(O, n, seed=100, step=0)
    lim = 5 / math.sqrt(n)
    corr = lambda x, y: np.corrcoef(x, y)[0, 1]
    assert abs(corr(a.real, a.imag)) < lim
    assert abs(corr(a.real[:-1], a.real[1:])) < lim
    assert abs(corr(a.real, b.real)) < lim
    assert abs(corr(a.real, c.real)) < lim
    # deterministic: the same counter and key give the same values
    assert np.array_equal(a, noise_values(O, n, seed=99, step=0))


def test_diffusion_limit_correlator(O):
    """Noise-only dynamics (alpha = beta = 0, no field, coupling made negligible by a
    huge h, mu and K frozen): psi^n = psi^{n-1} + h_t zeta^n up to O(1/h^2), so
    <|psi|^2> after n steps from psi = 0 is (2/3) zeta_max^2 h_t^2 n = (2/3) zeta_max^2 h_t t."""
    h = 1.0e4
    ht = 0.1
    G = O.Grid(24, 24, 16, hx=h, hy=h, hz=h, bc=(P, P, P), beta=0.0, ht=ht)
    G.noise_T = ht * h ** 3 * 1.0   # zeta_max = 1
    G.noise_seed = 2024
    alpha = np.zeros(G.shape)
    st = O.State(np.zeros(G.shape, dtype=np.complex128), np.zeros(G.shape))
    prev = st.psi.copy()
    n = 25
    incs = []
    for _ in range(n):
        O.step(G, st, alpha, eps=1e-24, max_iter=50, freeze_mu_K=True)
        incs.append((st.psi - prev) / ht)
        prev = st.psi.copy()
    zmax = math.sqrt(G.noise_T / (ht * h ** 3))
    expect = (2 / 3) * zmax ** 2 * ht * (n * ht)
    got = float(np.mean(np.abs(st.psi) ** 2))
    assert abs(got - expect) < 0.06 * expect, (got, expect)
    # each increment is one draw of zeta: uniform components on [-zeta_max, zeta_max)
    z = incs[3].ravel()
    assert np.max(np.abs(z.real)) <= zmax * (1 + 1e-6) and np.max(np.abs(z.imag)) <= zmax * (1 + 1e-6)
    assert abs(np.mean(np.abs(z) ** 2) - (2 / 3) * zmax ** 2) < 0.05 * (2 / 3) * zmax ** 2
    assert abs(np.corrcoef(incs[3].real.ravel(), incs[4].real.ravel())[0, 1]) < 0.05
