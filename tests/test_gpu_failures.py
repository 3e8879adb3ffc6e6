"""Failure statuses of the C ABI, provoked on the host side (needs a GB300).

No test here faults or hangs the GPU: the potential solve stops at its cycle
cap (a tolerance below what the arithmetic can reach), a non-finite value is
imported through fcd_set_populations (NaN arithmetic does not trap; the
residual test counts it as infinite and the observables flag it), and a
snapshot is offered to a context of another shape. Each call must return its
status and leave the context usable.
"""
import numpy as np
import pytest

from paper_2410_11129_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fcd():
    import torch
    assert torch.cuda.is_available(), "needs a CUDA device"
    from paper_2410_11129_gb300 import fcd as F
    F.load()
    return F


@pytest.mark.parametrize("graph", [True, False])
def test_solve_cap_reports_noconv(fcd, monkeypatch, graph):
    """A 2-cycle cap cannot reach 1e-9 in FP32: every solve runs to its cap,
    the steps still complete, and the next observables call reports
    FCD_ENOCONV once for the capped solves."""
    if not graph:
        monkeypatch.setenv("FCD_NO_GRAPH", "1")
    cfg = dict(W.small(mag_tol=1e-9, mag_max_iter=2), precision="fp32")
    ch = fcd.Channel(cfg)  # create tolerates a capped initial solve
    ch.step(3)
    with pytest.raises(fcd.FcdError) as e:
        ch.observe()
    assert e.value.status == fcd.FCD_ENOCONV
    assert ch.observe()["step"] == 3  # reported once; the context stays usable
    assert ch.solver_stats()["capped"] >= 3
    ch.close()


def test_nonfinite_state_reports_unstable(fcd):
    cfg = dict(W.small(), precision="fp64")
    ch = fcd.Channel(cfg)
    ch.step(2)
    f, g, psi = ch.populations()
    g[0, 0, 10, 20] = np.nan
    ch.set_populations(f, g, psi, step=2)
    with pytest.raises(fcd.FcdError) as e:
        ch.observe()
    assert e.value.status == fcd.FCD_EUNSTABLE
    # the context stays usable: a clean state observes normally again
    g[0, 0, 10, 20] = 0.0
    ch.set_populations(f, g, psi, step=2)
    assert np.isfinite(ch.observe()["T_o"])
    ch.close()


def test_foreign_snapshot_rejected(fcd):
    a = fcd.Channel(dict(W.small(nx=48), precision="fp64"))
    b = fcd.Channel(dict(W.small(nx=40), precision="fp64"))
    snap = np.zeros(a.state_bytes(), np.uint8)
    a.get_state(snap)
    with pytest.raises(fcd.FcdError) as e:
        b.set_state(np.zeros(max(snap.nbytes, b.state_bytes()), np.uint8))
    assert e.value.status == fcd.FCD_ESTATE
    with pytest.raises(fcd.FcdError) as e:
        b.set_state(np.concatenate([snap, np.zeros(b.state_bytes(), np.uint8)]))
    assert e.value.status == fcd.FCD_ESTATE
    b.step(1)  # still usable
    a.close()
    b.close()


def test_unstable_step_is_reported_with_its_index(fcd):
    """A non-finite value imported at step 2 makes the collision of step 2
    produce a non-finite velocity; the steps complete (no trap) and the next
    synchronising calls report FCD_EUNSTABLE naming step 2."""
    cfg = dict(W.small(), precision="fp64")
    ch = fcd.Channel(cfg)
    ch.step(2)
    f, g, psi = ch.populations()
    bad = g.copy()
    bad[0, 0, 10, 20] = np.nan
    ch.set_populations(f, bad, psi, step=2)
    ch.step(3)
    for call in (ch.observe, lambda: ch.field("ux")):
        with pytest.raises(fcd.FcdError) as e:
            call()
        assert e.value.status == fcd.FCD_EUNSTABLE
        assert "first in step 2 " in str(e.value), str(e.value)
    ch.set_populations(f, g, psi, step=2)  # a clean state clears the record
    ch.step(3)
    # the potential solves of the non-finite steps ran to their cap: reported once
    assert ch.observe(allow=(fcd.FCD_ENOCONV,))["step"] == 5
    assert np.isfinite(ch.observe()["T_o"])
    ch.close()


def test_allocation_failure_reports_enomem_and_releases_everything(fcd):
    """fcd_set_allocator with a hook that fails from its k-th call on: every k
    before the context is complete gives FCD_ENOMEM, a NULL handle, and every
    block the hook handed out is released exactly once."""
    import ctypes as C
    import torch
    L = fcd.load()
    params = fcd.make_params(dict(W.small(), precision="fp32_offset"))
    k, seen_ok = 0, False
    try:
        while not seen_ok:
            live, calls = {}, [0]

            def alloc(size, user):
                i = calls[0]
                calls[0] += 1
                if i >= k:
                    return None
                ptr = int(torch.cuda.caching_allocator_alloc(int(size)))
                live[ptr] = size
                return ptr

            def free(ptr, user):
                assert ptr in live
                del live[ptr]
                torch.cuda.caching_allocator_delete(int(ptr))

            hooks = (fcd.ALLOC_FN(alloc), fcd.FREE_FN(free))
            L.fcd_set_allocator(hooks[0], hooks[1], None)
            h = C.c_void_p()
            st = L.fcd_create(C.byref(params), C.byref(h))
            if st == fcd.FCD_OK:
                seen_ok = True
                assert k >= 17 and calls[0] <= k
                L.fcd_step(h, 2)
                L.fcd_destroy(h)
            else:
                assert st == fcd.FCD_ENOMEM, (k, st)
                assert not h.value
                assert "allocation" in L.fcd_last_error(None).decode()
            assert not live, (k, len(live))
            k += 1 if k < 24 else 7
            assert k < 2000
    finally:
        L.fcd_set_allocator(fcd.ALLOC_FN(), fcd.FREE_FN(), None)
        fcd._torch_alloc = None
