"""The quadratic Bezier short-characteristics formal solver (the option
formal = 1; the paper names no scheme) in the oracle, pinned against what
the mathematics fixes:

* its step weights against direct numerical quadrature of the Bezier
  integrals (scipy), in both the series (d < 1) and the closed-form branch,
  with the large-d limits w_u d^2 -> 2, (1 - w_o) d -> 2, w_c d -> 2 and
  (1 - w_o - w_c) d^2 -> 2;
* a source function linear in tau is reproduced exactly (the control point
  falls on the midpoint): I(0, mu) = a + b mu for S = a + b tau;
* for S = exp(-k tau) the emergent intensity 1 / (1 + k mu) is approached at
  third order under grid refinement (the linear scheme: second), and closer
  than the linear scheme on every grid;
* the control point is held between its neighbours: a sharp step in S gives
  no intensity above the largest S."""
import numpy as np
import pytest

scipy_integrate = pytest.importorskip("scipy.integrate")


def test_weights_match_quadrature(orc):
    quad = scipy_integrate.quad
    for d in (1e-8, 1e-4, 1e-2, 0.3, 0.999, 1.0, 1.001, 3.0, 30.0):
        ex, wu, wo, wc, omp = orc.bez_weights(d)
        qu = quad(lambda s: s * s * np.exp(-d * s) * d, 0, 1, epsabs=0, epsrel=1e-13)[0]
        qo = quad(lambda s: (1 - s) ** 2 * np.exp(-d * s) * d, 0, 1, epsabs=0, epsrel=1e-13)[0]
        qc = quad(lambda s: 2 * s * (1 - s) * np.exp(-d * s) * d, 0, 1, epsabs=0, epsrel=1e-13)[0]
        assert abs(wu / qu - 1) < 1e-12 and abs(wo / qo - 1) < 1e-12 and abs(wc / qc - 1) < 1e-12, d
        assert abs(ex - np.exp(-d)) < 1e-15
        assert abs(omp - (1 - wo - wc)) < 1e-14, d
    for d in (1e4, 1e8):
        ex, wu, wo, wc, omp = orc.bez_weights(d)
        assert abs(wu * d * d - 2) < 1e-3 and abs((1 - wo) * d - 2) < 1e-3
        assert abs(wc * d - 2) < 1e-3 and abs(omp * d * d - 2) < 1e-12


def _emergent(orc, S_of, mu, n, bezier, tmax=40.0):
    tau = np.concatenate([[0.0], np.logspace(-4, np.log10(tmax), n)])
    S = S_of(tau)
    dS = np.gradient(S, tau)
    I, _ = orc.sc_sweep(np.diff(tau) / mu, S, S[-1] + mu * dS[-1], -1, bezier=bezier)
    return I[0]


def test_linear_source_is_exact(orc):
    for mu in (0.1, 0.5, 1.0):
        for n in (10, 50):
            assert abs(_emergent(orc, lambda t: 1 + 2 * t, mu, n, True) - (1 + 2 * mu)) < 1e-13


def test_third_order_for_a_smooth_source(orc):
    k, mu = 2.0, 0.5
    exact = 1 / (1 + k * mu)
    eb, el = [], []
    for n in (20, 40, 80, 160):
        eb.append(abs(_emergent(orc, lambda t: np.exp(-k * t), mu, n, True) - exact))
        el.append(abs(_emergent(orc, lambda t: np.exp(-k * t), mu, n, False) - exact))
    rb = [eb[i] / eb[i + 1] for i in range(3)]
    rl = [el[i] / el[i + 1] for i in range(3)]
    assert min(rb) > 6.0, rb          # ~8: third order
    assert max(rl) < 5.0, rl          # ~4: second order
    assert all(b < l for b, l in zip(eb, el))


def test_no_overshoot_at_a_step(orc):
    tau = np.linspace(0, 20, 41)
    S = np.where(tau < 8.0, 0.0, 1.0) + np.where(tau > 12.0, 3.0, 0.0)
    for mu in (0.2, 1.0):
        for direction, I0 in ((-1, 4.0), (1, 0.0)):
            I, lam = orc.sc_sweep(np.diff(tau) / mu, S, I0, direction, bezier=True)
            assert np.all(I <= S.max() + 1e-12) and np.all(I >= -1e-12)
            assert np.all((lam >= 0) & (lam <= 1))


def test_two_point_ray_is_the_linear_step(orc):
    """Without a downwind point the control point is the midpoint, and the
    Bezier step is the linear one (w_u + w_c/2 and w_o + w_c/2 are the
    linear weights): checked on two-point rays across optical thicknesses
    and with the exact linear-source intensity."""
    rng = np.random.default_rng(5)
    for d in (1e-6, 1e-3, 0.2, 0.9, 1.0, 1.5, 7.0, 200.0, 1e6):
        for _ in range(3):
            S = rng.uniform(0.1, 5.0, 2)
            I0 = rng.uniform(0.0, 5.0)
            for direction in (1, -1):
                Ib, lb = orc.sc_sweep(np.array([d]), S, I0, direction, bezier=True)
                Il, ll = orc.sc_sweep(np.array([d]), S, I0, direction, bezier=False)
                k = 1 if direction > 0 else 0
                assert abs(Ib[k] - Il[k]) <= 1e-13 * max(1.0, abs(Il[k])), (d, direction)
