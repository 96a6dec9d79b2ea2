"""phtl_batch_run_noalloc -- the batched launch that allocates no memory -- against the
allocating entry point phtl_batch_create + phtl_batch_run.

Callers that cannot let the library allocate device memory (an application whose device
memory is owned by its own allocator, a loop that must never pay for cudaMalloc /
cudaFree) use the no-allocation run; it must track exactly like the regular batch.  Both
paths run the same mixed batch twice in a row from the same initial data: particles must
agree bitwise after each call, monitor moments to FP64 rounding (the tolerance the other
batched tests use).  This file is collected last and needs no state from other tests.
"""
import ctypes as C

import numpy as np
import pytest

import helpers

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1610_05801_gb300 import phtl, synth  # noqa: E402

DEV = "cuda:0"
SPECS = [  # n, turns, voltage, integrator, dtype, monitor stride (0 = none), transverse
    (3001, 400, 4.5e6, "ruth4", "f64", 4, True),
    (1000, 900, 2.0e6, "leapfrog", "f32c", 1, False),
    (513, 250, 6.0e6, "euler_cromer", "f32cd", 0, True),
    (7, 1200, 1.0e6, "leapfrog", "f64", 10, False),
]


def _make(spec, seed):
    n, turns, V, integ, dt, stride, tr = spec
    inp = helpers.inputs(n, seed=seed, voltage=V, transverse=True)
    keys = ("z", "dp", "x", "xp", "y", "yp") if tr else ("z", "dp")
    bufs = []
    for k in keys:
        if dt == "f64":
            bufs.append(torch.tensor(inp[k], dtype=torch.float64, device=DEV))
        else:
            bufs.append(torch.tensor(phtl.split_f32c(inp[k]), dtype=torch.float32, device=DEV))
    while len(bufs) < 6:
        bufs.append(None)
    mon = (torch.zeros((turns // stride + 1, 16), dtype=torch.float64, device=DEV)
           if stride else None)
    return phtl.make_job(*bufs, turns=turns, voltage_V=V, integrator=integ, dtype=dt,
                         monitor=mon, stride=stride or 1)


def test_noalloc_matches_allocating_batch_on_two_calls():
    ring = synth.ring(2e6, transverse=True)
    R = phtl.Ring(**ring)
    ref_jobs = [_make(s, 900 + i) for i, s in enumerate(SPECS)]
    new_jobs = [_make(s, 900 + i) for i, s in enumerate(SPECS)]
    B = phtl.Batch(R, ref_jobs, use_graph=True)
    for call in range(2):
        B.run()
        phtl.batch_run_noalloc(R, new_jobs)
        torch.cuda.synchronize()
        for spec, a, b in zip(SPECS, ref_jobs, new_jobs):
            for u, v in zip(a["c"], b["c"]):
                if u is not None:
                    assert torch.equal(u, v), (call, spec)
            if a["monitor"] is not None:
                ma = phtl.moments_from_sums(a["monitor"].cpu().numpy())
                mb = phtl.moments_from_sums(b["monitor"].cpu().numpy())
                assert np.allclose(ma, mb, rtol=1e-11, atol=1e-300), (call, spec)
    B.close()
    R.close()


def test_noalloc_rejects_more_jobs_than_its_table():
    R = phtl.Ring(**synth.ring(2e6))
    z = torch.zeros(4, dtype=torch.float64, device=DEV)
    J = (phtl.Job * (phtl.NOALLOC_MAX_JOBS + 1))()
    for i in range(len(J)):
        J[i].c[0] = J[i].c[1] = z.data_ptr()
        J[i].n, J[i].turns, J[i].voltage_V, J[i].integrator, J[i].dtype = 4, 1, 2e6, 1, 0
    lib = phtl.load()
    rc = lib.phtl_batch_run_noalloc(R.handle, J, len(J), None)
    assert rc == phtl.E_TOOBIG
    assert lib.phtl_strerror(rc).decode().startswith("more jobs than")
    # exactly at the limit is accepted
    rc = lib.phtl_batch_run_noalloc(R.handle, J, phtl.NOALLOC_MAX_JOBS, None)
    torch.cuda.synchronize()
    assert rc == phtl.OK
    R.close()
