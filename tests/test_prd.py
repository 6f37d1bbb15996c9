"""Angle-averaged partial redistribution on the GPU against the FP64 oracle
(R_II-A kernels computed by the column kernel with its own quadrature).

Cases: Lyman alpha in PRD on a 3-level atom (24 points, 32 depths), and
Lyman alpha and beta together in PRD on the full 5-level atom at the bench's
64 points per line and 82 depths.  Fixed schedules are compared per iterate
(FP64 within 1e-9, FP32 within 1e-3) without Ng (the damped rho update) and
with the Jacobi step on rho (Ng on, its first extrapolation after the
compared iterations); converged solutions with Ng on populations and rho are
compared at the fixed point."""
import numpy as np
import pytest

import rh_synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rh():
    import paper_1411_1079_gb300 as m
    m.build()
    return m


def prd_atom():
    return rh_synth.hydrogen_like_atom(nbound=3, lyman_nlambda=24, line_nlambda=12, cont_nlambda=10, nmu=3,
                                       prd_lines=((1, 2),))


def two_line_atom():
    return rh_synth.hydrogen_like_atom(prd_lines=((1, 2), (1, 3)))


@pytest.fixture(scope="module")
def cols():
    return rh_synth.subset(rh_synth.chromosphere_cube(nx=16, ny=16, ndep=32, seed=3), [0, 5])


@pytest.fixture(scope="module")
def cols82():
    # two moving columns (|v_z| up to 8.6 and 5.2 km/s) that run every compared
    # iteration from LTE (column 5 of this cube stops at iteration 2 with a
    # negative population under PRD, in the oracle and on the GPU alike)
    return rh_synth.subset(rh_synth.chromosphere_cube(nx=16, ny=16, ndep=82, seed=3), [0, 2])


# fixed schedules: (ng_order, ng_delay) -- no Ng (damped update), and Ng on
# with its first extrapolation after the compared iterations (Jacobi update)
SCHEDULES = [(0, 5), (2, 50)]


def _oracle_fixed(orc, atom, cols):
    o = orc.Oracle()
    o.setup_atom(atom)
    o.load_columns(cols)
    out = {}
    for ng, delay in SCHEDULES:
        for k in (3, 6):
            o.iterate(maxiter=k, tol=0.0, ng_order=ng, ng_delay=delay, prd_eps0=0.05)
            out[ng, k] = o.populations()[0]
    return o, out


@pytest.fixture(scope="module")
def oracle_runs(orc, cols):
    o, out = _oracle_fixed(orc, prd_atom(), cols)
    o.iterate(maxiter=400, tol=1e-3)
    out["conv"] = o.populations()
    o.iterate(maxiter=2000, tol=1e-11)
    out["tight"] = o.populations()
    return out


@pytest.fixture(scope="module")
def oracle_two_lines(orc, cols82):
    return _oracle_fixed(orc, two_line_atom(), cols82)[1]


def _fixed(rh, atom, cols, ref, precision, tol):
    g = rh.Context(0)
    g.setup_atom(atom)
    g.load_columns(cols)
    for ng, delay in SCHEDULES:
        for k in (3, 6):
            g.iterate(maxiter=k, tol=0.0, ng_order=ng, ng_delay=delay, precision=precision, prd_eps0=0.05)
            n = g.populations()[0]
            assert np.max(np.abs(n / ref[ng, k] - 1)) < tol, (precision, ng, k)


@pytest.mark.parametrize("precision,tol", [(0, 1e-9), (1, 1e-3)])
def test_prd_fixed_schedule_matches_oracle(rh, cols, oracle_runs, precision, tol):
    _fixed(rh, prd_atom(), cols, oracle_runs, precision, tol)


@pytest.mark.parametrize("precision,tol", [(0, 1e-9), (1, 1e-3)])
def test_two_prd_lines_fixed_schedule_matches_oracle(rh, cols82, oracle_two_lines, precision, tol):
    """Lyman alpha and beta in PRD at 64 points each on 82 depths (the
    bench's PRD case)."""
    _fixed(rh, two_line_atom(), cols82, oracle_two_lines, precision, tol)


def test_prd_fp64_fixed_point_with_ng(rh, cols, oracle_runs):
    """Ng on populations and rho: the FP64 GPU fixed point at 1e-11 equals
    the oracle's within 1e-9 (mid-trajectory comparison with Ng is not
    meaningful: it amplifies rounding differences)."""
    g = rh.Context(0)
    g.setup_atom(prd_atom())
    g.load_columns(cols)
    g.iterate(maxiter=2000, tol=1e-11, precision=0)
    n, it, st, _ = g.populations()
    no, ito, sto, _ = oracle_runs["tight"]
    assert np.all(st == 0) and np.all(sto == 0)
    assert np.max(np.abs(n / no - 1)) < 1e-9
    assert np.all(it < 1000), it


def test_prd_mixed_fixed_point_and_stopping_point(rh, cols, oracle_runs):
    g = rh.Context(0)
    g.setup_atom(prd_atom())
    g.load_columns(cols)
    g.iterate(maxiter=2000, tol=1e-6, precision=1)
    n, it, st, _ = g.populations()
    no = oracle_runs["tight"][0]
    assert np.all(st == 0)
    assert np.max(np.abs(n / no - 1)) < 1e-3
    # at the 1e-3 criterion (the paper's), through rh_solve
    g.load_columns(cols)
    g.solve(precision=1, maxiter=400, tol=1e-3)
    n3, it3, st3, _ = g.populations()
    assert np.all(st3 == 0)
    assert np.max(np.abs(n3 / no - 1)) < 3e-2
    assert np.allclose(n3.sum(axis=1), cols["nH"], rtol=1e-12)
    # PRD changes the solution (against CRD)
    a = prd_atom()
    a["line_prd"] = a["line_prd"] * 0
    h = rh.Context(0)
    h.setup_atom(a)
    h.load_columns(cols)
    h.solve(precision=1, maxiter=400, tol=1e-3)
    assert np.max(np.abs(h.populations()[0] / n3 - 1)) > 1e-2
