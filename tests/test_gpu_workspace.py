"""Caller-owned device memory (cls_workspace_bytes / cls_bind_workspace): a torch
tensor holds every device buffer of the handle, and the walk gives the same
tallies as the library-owned buffers -- integer counts bit-exact, sums to the
atomics' summation order."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1708_00765_gb300 as cls  # noqa: E402
from paper_1708_00765_gb300 import _native, workloads  # noqa: E402

COUNTS = ("nR", "nT", "nA", "n_coll", "n_interface", "n_reflect", "n_events", "max_events", "n_capped")


def same_tallies(a, b):
    for k in COUNTS:
        assert a[k] == b[k], k
    assert a["sum_t"] == pytest.approx(b["sum_t"], rel=1e-12)
    np.testing.assert_allclose(a["flux"], b["flux"], rtol=1e-12, atol=1e-15 * max(b["flux"].max(), 1e-300))


def run_raw(params, n, seed, batch=False, ws=False, **opts):
    prob = cls.Problem(params, batch=batch)
    for k, v in opts.items():
        prob.set_option(k, v)
    buf = None
    if ws:
        buf = torch.empty(prob.workspace_bytes(), dtype=torch.uint8, device="cuda")
        prob.bind_workspace(buf.data_ptr(), buf.numel())
    prob.run(n, seed)
    prob.run(n // 3, seed)  # a second run (the batch: a graph replay) into the same buffers
    out = [prob.raw_tallies(k) for k in range(prob.params.shape[0])]
    prob.close()
    return out, buf


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("schedule", ["history", "event"])
def test_bound_workspace_gives_the_library_owned_tallies(precision, schedule):
    p = workloads.BOX_L10
    ref, _ = run_raw(p, 30_000, 3, precision=precision, schedule=schedule)
    got, buf = run_raw(p, 30_000, 3, ws=True, precision=precision, schedule=schedule)
    same_tallies(got[0], ref[0])
    # the tallies live in the caller's tensor: its flux block (offset 0) is the run's
    nbs = (int(p[8]) + 1) & ~1
    flux = buf[: 64 * nbs * 8].view(torch.float64).view(64, nbs)[:, : int(p[8])].cpu().numpy()
    np.testing.assert_array_equal(flux, got[0]["flux"])


def test_bound_workspace_batch_through_the_graph():
    cases = workloads.batch_sweep(16, seed=7, nbins=30)
    ref, _ = run_raw(cases, 4000, 5, batch=True)
    got, _ = run_raw(cases, 4000, 5, batch=True, ws=True)
    for a, b in zip(got, ref):
        same_tallies(a, b)


def test_workspace_errors_and_unbinding():
    prob = cls.Problem(workloads.ROD_L10)
    need = prob.workspace_bytes()
    buf = torch.empty(need + 512, dtype=torch.uint8, device="cuda")
    with pytest.raises(cls.ClsError) as e:      # too small
        prob.bind_workspace(buf.data_ptr(), need - 1)
    assert e.value.code == _native.CLS_E_INVAL
    with pytest.raises(cls.ClsError) as e:      # not 256-byte aligned
        prob.bind_workspace(buf.data_ptr() + 8, need)
    assert e.value.code == _native.CLS_E_INVAL
    host = np.zeros(need, dtype=np.uint8)       # host memory, not the device's
    with pytest.raises(cls.ClsError) as e:
        prob.bind_workspace(host.ctypes.data, need)
    assert e.value.code == _native.CLS_E_INVAL
    prob.bind_workspace(buf.data_ptr(), need)
    prob.run(1000, 1)
    with pytest.raises(cls.ClsError) as e:      # results in the tallies: reset first
        prob.bind_workspace(0, 0)
    assert e.value.code == _native.CLS_E_STATE
    bound = prob.raw_tallies()
    prob.reset()
    # a larger statistics layout that no longer fits the workspace is refused
    with pytest.raises(cls.ClsError) as e:
        prob.set_option("nbatch", 1024)
    assert e.value.code == _native.CLS_E_NOMEM
    assert prob.get_option("nbatch") == 64
    prob.bind_workspace(0, 0)                  # back to library-owned buffers
    prob.run(1000, 1)
    same_tallies(prob.raw_tallies(), bound)
    prob.close()


def test_bound_workspace_with_several_event_launch_groups():
    """Rods and boxes, half of each on the event schedule: four launch groups, two of
    them event launches with their own slices of the bank, all in the caller's
    tensor; the same tallies as the library-owned buffers."""
    cases = workloads.batch_sweep(12, seed=7, nbins=20)

    def run(ws):
        prob = cls.Problem(cases, batch=True)
        prob.set_option("schedule", "history")
        for k in range(0, 12, 2):
            prob.set_case_schedule(k, "event")
        buf = None
        if ws:
            buf = torch.empty(prob.workspace_bytes(), dtype=torch.uint8, device="cuda")
            prob.bind_workspace(buf.data_ptr(), buf.numel())
        prob.run(3000, 8)
        out = [prob.raw_tallies(k) for k in range(12)]
        prob.close()
        return out

    for a, b in zip(run(True), run(False)):
        same_tallies(a, b)
