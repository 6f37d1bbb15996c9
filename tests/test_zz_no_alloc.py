"""rh_iterate_noalloc: the iteration for callers that cannot allocate device
memory while they solve (their memory belongs to their own pool, or they are
capturing a stream into a graph, or they cannot afford the synchronisation of
cudaMalloc).  It keeps its scratch in a static array inside the library and
writes into buffers the caller owns, and evaluates the line profiles in the
sweep, where rh_iterate reads them from its per-column profile cache.  Its
results must match rh_iterate's on the same columns, on two calls in a row
(the second call finds the scratch holding the first call's contents).  In
FP32 the two paths agree bit for bit, trajectory and stopping included.  In
FP64 the two kernel instantiations may fuse multiply-adds of the Voigt
function differently (1 ulp); Ng extrapolation amplifies such differences
along a trajectory, so FP64 is compared on a fixed schedule without Ng, as
the FP64 parity tests are.  This file is collected last so that a
run stopping at the first failure has run every other test first."""
import numpy as np
import pytest

import rh_synth

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-9        # same bound as the FP64 parity tests


def _columns():
    cube = rh_synth.chromosphere_cube(nx=32, ny=32, seed=11)
    return rh_synth.subset(cube, list(range(0, 1024, 3)))


@pytest.mark.parametrize("precision", [1, 0])
def test_noalloc_matches_rh_iterate_twice(precision):
    import torch

    import paper_1411_1079_gb300 as rh
    rh.build()
    atom = rh_synth.hydrogen_like_atom()
    cols = _columns() if precision == 1 else rh_synth.subset(_columns(), slice(0, 40))
    ncol, ndep = cols["T"].shape
    ctx = rh.Context(0)
    ctx.setup_atom(atom)
    ctx.load_columns(cols)
    if precision == 1:
        kw = dict(maxiter=120, tol=1e-3, precision=precision)
    else:
        kw = dict(maxiter=15, tol=0.0, ng_order=0, precision=precision)
    ref = ctx.iterate(**kw)
    n_ref, it_ref, st_ref, dm_ref = ctx.populations()

    n_out = torch.zeros((ncol, atom["nlev"], ndep), dtype=torch.float64, device="cuda")
    it_out = torch.zeros(ncol, dtype=torch.int32, device="cuda")
    st_out = torch.zeros(ncol, dtype=torch.uint8, device="cuda")
    dm_out = torch.zeros(ncol, dtype=torch.float64, device="cuda")
    for call in range(2):
        s = ctx.iterate_noalloc(n_out, it_out, st_out, dm_out, **kw)
        torch.cuda.synchronize()
        n = n_out.cpu().numpy()
        assert float(np.max(np.abs(n / n_ref - 1))) < FP64_TOL, call
        assert np.array_equal(it_out.cpu().numpy(), it_ref), call
        assert np.array_equal(st_out.cpu().numpy(), st_ref), call
        assert s["n_converged"] == ref["n_converged"] and s["iterations_total"] == ref["iterations_total"]
        assert s["max_dn_final"] == pytest.approx(ref["max_dn_final"], rel=1e-12 if precision == 1 else 1e-6)
        n_out.fill_(-1.0)
        it_out.fill_(-1)
    # the context's own populations are untouched by the no-allocation call
    assert np.array_equal(ctx.populations()[0], n_ref)


def test_noalloc_rejects_bad_arguments():
    import torch

    import paper_1411_1079_gb300 as rh
    rh.build()
    ctx = rh.Context(0)
    ctx.setup_atom(rh_synth.small_atom())
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(rh.RhError) as e:          # nothing loaded yet
        ctx.iterate_noalloc(buf, buf, buf, buf)
    assert e.value.code == rh.RH_ESTATE
    ctx.load_columns(rh_synth.subset(rh_synth.chromosphere_cube(nx=16, ny=16, ndep=12, seed=1), [0, 1]))
    with pytest.raises(rh.RhError) as e:
        ctx.iterate_noalloc(buf, buf, buf, buf, ng_order=3)
    assert e.value.code == rh.RH_EINVAL
