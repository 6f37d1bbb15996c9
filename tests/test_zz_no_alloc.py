"""rh_iterate_noalloc: the iteration for callers that cannot allocate device
memory while they solve (their memory belongs to their own pool or budget,
or they cannot afford the device-wide synchronisation of cudaMalloc).  It
keeps its scratch in a static array inside the library and writes into
buffers the caller owns; here rh_iterate runs first on the same context, so
the no-alloc call reads the line profiles from the profile cache rh_iterate
allocated and runs the same kernel.  Its results must match rh_iterate's on
the same columns, on two calls in a row (the second call finds the scratch
holding the first call's contents), and the second call must leave the
device's free memory and torch's allocation unchanged.  FP32 is compared
bit for bit, trajectory and stopping included; FP64 on a fixed schedule
without Ng within the FP64 parity tests' bound.  The sweep without the
cache is compared with the cached one in the overlapping-lines tests.  This
file is collected last so that a run stopping at the first failure has run
every other test first."""
import ctypes as C

import numpy as np
import pytest

import rh_synth

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-9        # same bound as the FP64 parity tests


def _columns(n=1024, step=3):
    cube = rh_synth.chromosphere_cube(nx=32, ny=32, seed=11)
    return rh_synth.subset(cube, list(range(0, n, step)))


def _buffers(torch, ncol, nlev, ndep):
    return (torch.zeros((ncol, nlev, ndep), dtype=torch.float64, device="cuda"),
            torch.zeros(ncol, dtype=torch.int32, device="cuda"),
            torch.zeros(ncol, dtype=torch.uint8, device="cuda"),
            torch.zeros(ncol, dtype=torch.float64, device="cuda"))


@pytest.mark.parametrize("precision,persistent", [(1, 1), (0, 1), (1, 0)])
def test_noalloc_matches_rh_iterate_twice(precision, persistent):
    import torch

    import paper_1411_1079_gb300 as rh
    rh.build()
    atom = rh_synth.hydrogen_like_atom()
    if precision == 0:
        cols = rh_synth.subset(_columns(), slice(0, 40))
    elif persistent == 0:
        cols = _columns(1024, 1)      # more columns than resident blocks: static split
    else:
        cols = _columns()
    ncol, ndep = cols["T"].shape
    ctx = rh.Context(0)
    ctx.setup_atom(atom)
    ctx.load_columns(cols)
    if precision == 1:
        kw = dict(maxiter=120, tol=1e-3, precision=precision, persistent=persistent)
    else:
        kw = dict(maxiter=15, tol=0.0, ng_order=0, precision=precision, persistent=persistent)
    ref = ctx.iterate(**kw)
    n_ref, it_ref, st_ref, dm_ref = ctx.populations()

    n_out, it_out, st_out, dm_out = _buffers(torch, ncol, atom["nlev"], ndep)
    torch.cuda.synchronize()
    for call in range(2):
        if call == 1:
            free0 = torch.cuda.mem_get_info()[0]
            alloc0 = torch.cuda.memory_allocated()
        s = ctx.iterate_noalloc(n_out, it_out, st_out, dm_out, **kw)
        torch.cuda.synchronize()
        if call == 1:
            assert torch.cuda.mem_get_info()[0] == free0
            assert torch.cuda.memory_allocated() == alloc0
        n = n_out.cpu().numpy()
        if precision == 1:
            assert np.array_equal(n, n_ref), call
        else:
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
    cols = rh_synth.subset(rh_synth.chromosphere_cube(nx=16, ny=16, ndep=12, seed=1), [0, 1])
    ctx.load_columns(cols)
    good = _buffers(torch, 2, ctx.nlev, 12)
    with pytest.raises(rh.RhError) as e:
        ctx.iterate_noalloc(*good, ng_order=3)
    assert e.value.code == rh.RH_EINVAL
    # the binding refuses host arrays, wrong types, short and strided tensors
    bad = [
        (np.zeros((2, ctx.nlev, 12)),) + good[1:],
        (good[0], good[1].to(torch.int64)) + good[2:],
        good[:3] + (torch.zeros(1, dtype=torch.float64, device="cuda"),),
        (torch.zeros((2, 12, ctx.nlev), dtype=torch.float64, device="cuda").transpose(1, 2),) + good[1:],
    ]
    for b in bad:
        with pytest.raises(ValueError):
            ctx.iterate_noalloc(*b)
    # the library itself refuses a pointer that is not device memory
    host = np.zeros(2 * ctx.nlev * 12)
    o = rh.IterOpts(maxiter=1, tol=0.0, ng_order=0, ng_delay=5, ng_period=3, start=0, precision=1, persistent=1,
                    block_warps=0, crsw_init=1.0, only_unconverged=0)
    rc = ctx._lib.rh_iterate_noalloc(ctx._p, C.byref(o), C.c_void_p(host.ctypes.data),
                                     *(C.c_void_p(t.data_ptr()) for t in good[1:]), None)
    assert rc == rh.RH_EINVAL
    assert b"not device memory" in ctx._lib.rh_last_error(ctx._p)
    # a good call still runs after the refusals, and the current device is kept
    torch.cuda.set_device(0)
    ctx.iterate_noalloc(*good, maxiter=3, tol=0.0)
    assert torch.cuda.current_device() == 0
