"""Host logic of solve (no GPU): the default re-run ladder it hands to
rh_solve for CRD and PRD atoms, and the final pass with the Bezier formal
solver that it runs through rh_iterate over the columns still unconverged,
checked against a stand-in for the library that records the options."""
import paper_1411_1079_gb300 as rh


class FakeLib:
    """records rh_solve's and rh_iterate's options; reports `left`
    unconverged columns after rh_solve and none after rh_iterate"""

    def __init__(self, ncol, left):
        self.ncol, self.left = ncol, left
        self.solve_opts, self.iter_opts = [], []

    def rh_solve(self, p, o, st):
        o, st = o._obj, st._obj
        self.solve_opts.append(o)
        st.n_converged = self.ncol - self.left
        st.n_failed = self.left
        st.iterations_total = 100
        return 6 if self.left else 0

    def rh_iterate(self, p, o, st):
        o, st = o._obj, st._obj
        self.iter_opts.append(o)
        st.n_converged = self.ncol
        st.n_processed = self.left
        st.iterations_total = 7
        return 0


def _ctx(prd, ncol=10, left=0):
    c = object.__new__(rh.Context)
    c._lib = FakeLib(ncol, left)
    c._p = None
    c.ncol = ncol
    c.has_prd = prd
    return c


def _rungs(o):
    return [(o.rerun_crsw[i], o.rerun_ng[i]) for i in range(o.nrerun)]


def test_crd_ladder():
    c = _ctx(False)
    c.solve(start=1)
    o = c._lib.solve_opts[0]
    assert _rungs(o) == [(1.0, 1), (1e3, 0), (1e5, 0), (1e7, 0)] and o.rerun_maxiter == 500
    c.solve(start=0)
    assert _rungs(c._lib.solve_opts[1]) == [(1e3, 0), (1e5, 0), (1e7, 0)]
    assert not c._lib.iter_opts


def test_prd_ladder_keeps_ng_first_and_allows_longer_reruns():
    c = _ctx(True)
    c.solve(start=1, maxiter=400)
    o = c._lib.solve_opts[0]
    assert _rungs(o) == [(1.0, 1), (1e3, 1), (1e5, 1), (1e3, 0)] and o.rerun_maxiter == 1200
    c.solve(start=0)
    assert _rungs(c._lib.solve_opts[1]) == [(1e3, 1), (1e5, 1), (1e3, 0), (1e5, 0)]


def test_prd_rescue_pass_with_the_bezier_solver():
    c = _ctx(True, ncol=10, left=3)
    s = c.solve(start=1, precision=1, prd_eps0=0.05, prd_hybrid=1)
    assert len(c._lib.iter_opts) == 1
    i = c._lib.iter_opts[0]
    assert (i.only_unconverged, i.formal, i.start, i.prd_hybrid, i.ng_order) == (1, 1, 0, 1, 2)
    assert abs(i.prd_eps0 - 0.05) < 1e-15 and i.maxiter == 1500
    assert s["rescue"]["converged_before"] == 7 and s["rescue"]["converged_after"] == 10
    assert s["n_converged"] == 10 and s["iterations_total"] == 107
    # no pass when everything converged, when asked not to, or for CRD atoms
    for kw, prd, left in ((dict(), True, 0), (dict(rescue=False), True, 3), (dict(), False, 3)):
        c = _ctx(prd, left=left)
        c.solve(**kw)
        assert not c._lib.iter_opts, (kw, prd, left)
