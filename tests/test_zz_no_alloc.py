"""phtl_batch_run_noalloc -- the batched launch that allocates no memory -- against the
allocating entry point phtl_batch_create + phtl_batch_run.

Callers that cannot let the library allocate device memory (an application whose device
memory is owned by its own allocator, a loop that must never pay for cudaMalloc /
cudaFree) use the no-allocation run; it must track exactly like the regular batch.  Both
paths run the same mixed batch twice in a row from the same initial data, then a smaller
batch of another arithmetic mix twice: particles must agree bitwise after each call,
monitor moments to FP64 rounding (the tolerance the other batched tests use), and the
device's free memory must not change across a call once the first one is done.  This
file is collected last and needs no state from other tests.
"""
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


# a later, smaller call with another arithmetic mix: its jobs land at the start of the
# table, over entries the earlier call wrote, and must not see anything of them
SPECS_SMALL = [
    (2049, 300, 3.0e6, "ruth4", "f32cs", 3, True),
    (900, 700, 5.0e6, "leapfrog", "f32c", 0, False),
]


def _compare(spec_list, ref_jobs, new_jobs, call):
    for spec, a, b in zip(spec_list, ref_jobs, new_jobs):
        for u, v in zip(a["c"], b["c"]):
            if u is not None:
                assert torch.equal(u, v), (call, spec)
        if a["monitor"] is not None:
            ma = phtl.moments_from_sums(a["monitor"].cpu().numpy())
            mb = phtl.moments_from_sums(b["monitor"].cpu().numpy())
            assert np.allclose(ma, mb, rtol=1e-11, atol=1e-300), (call, spec)


def test_noalloc_matches_allocating_batch_on_two_calls():
    ring = synth.ring(2e6, transverse=True)
    R = phtl.Ring(**ring)
    ref_jobs = [_make(s, 900 + i) for i, s in enumerate(SPECS)]
    new_jobs = [_make(s, 900 + i) for i, s in enumerate(SPECS)]
    B = phtl.Batch(R, ref_jobs, use_graph=True)
    for call in range(2):
        B.run()
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        phtl.batch_run_noalloc(R, new_jobs)
        torch.cuda.synchronize()
        if call > 0:  # the first call may load code and look up the table's address
            assert torch.cuda.mem_get_info()[0] == free0, "the call took device memory"
        _compare(SPECS, ref_jobs, new_jobs, call)
    B.close()
    # fewer jobs, other arithmetic: the allocating batch first (its launches load the
    # kernels), then the no-allocation run over the table's first entries, twice
    ref_small = [_make(s, 950 + i) for i, s in enumerate(SPECS_SMALL)]
    new_small = [_make(s, 950 + i) for i, s in enumerate(SPECS_SMALL)]
    B2 = phtl.Batch(R, ref_small, use_graph=False)
    for call in range(2):
        B2.run()
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        phtl.batch_run_noalloc(R, new_small)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0, "the call took device memory"
        _compare(SPECS_SMALL, ref_small, new_small, 2 + call)
    B2.close()
    R.close()


def test_noalloc_refuses_a_capturing_stream():
    """Its table comes from the call's own stack frame, which a captured copy would read
    at replay after the frame is gone: on a capturing stream the call must return
    PHTL_E_CAPTURE and enqueue nothing (the capture then ends cleanly and holds no node
    of it), and the next ordinary call tracks as before."""
    ring = synth.ring(2e6, transverse=True)
    R = phtl.Ring(**ring)
    spec = SPECS[1]
    ref = [_make(spec, 990)]
    new = [_make(spec, 990)]
    phtl.batch_run_noalloc(R, [_make(spec, 991)])  # the first call on the device, uncaptured
    torch.cuda.synchronize()
    before = [None if t is None else t.clone() for t in new[0]["c"]]
    arr, _keep = phtl.job_array(R, new)
    lib = phtl.load()
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    marker = torch.zeros(1, dtype=torch.float64, device=DEV)
    rcs = []
    with torch.cuda.graph(g, stream=side, capture_error_mode="thread_local"):
        rcs.append(lib.phtl_batch_run_noalloc(R.handle, arr, 1, side.cuda_stream))
        marker.add_(1.0)  # the graph's one node of its own
    torch.cuda.synchronize()
    assert rcs == [phtl.E_CAPTURE]
    g.replay()  # only the marker: nothing of the refused call is in the graph
    torch.cuda.synchronize()
    assert marker.item() == 1.0
    for u, v in zip(before, new[0]["c"]):
        if u is not None:
            assert torch.equal(u, v)
    B = phtl.Batch(R, ref, use_graph=False)
    B.run()
    phtl.batch_run_noalloc(R, new)
    torch.cuda.synchronize()
    _compare([spec], ref, new, 0)
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
