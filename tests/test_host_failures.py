"""Host-side failure paths of the C ABI that need no GPU (Sec. 5 of the
design: failure detection without faulting a device).

An allocator hook that fails from its k-th call on makes fcd_create return
FCD_ENOMEM with a NULL handle and release every block it was handed. The
blocks here are fake addresses that the library never dereferences: the
allocation check comes before any use of the pointers. That ordering is what
this test pins, so it runs only where no GPU is present.
"""
import ctypes as C

import pytest

from paper_2410_11129_gb300 import fcd
from paper_2410_11129_gb300 import workloads as W


def _no_gpu():
    try:
        import torch
        return not torch.cuda.is_available()
    except Exception:
        return True


@pytest.mark.skipif(not _no_gpu(), reason="fake device addresses: host-only test")
@pytest.mark.parametrize("prec", ["fp64", "fp32_offset"])
def test_create_reports_enomem_and_releases_every_block(prec):
    L = fcd.load()
    params = fcd.make_params(dict(W.small(), precision=prec))
    try:
        for fail_at in (0, 1, 5, 11, 16):
            live, calls = {}, [0]

            def alloc(size, user):
                i = calls[0]
                calls[0] += 1
                if i >= fail_at:
                    return None
                ptr = 0x100000 * (i + 1)  # never dereferenced
                live[ptr] = size
                return ptr

            def free(ptr, user):
                assert ptr in live, hex(ptr)
                del live[ptr]

            hooks = (fcd.ALLOC_FN(alloc), fcd.FREE_FN(free))
            L.fcd_set_allocator(hooks[0], hooks[1], None)
            h = C.c_void_p()
            st = L.fcd_create(C.byref(params), C.byref(h))
            assert st == fcd.FCD_ENOMEM, (fail_at, st)
            assert not h.value
            assert "allocation failed" in L.fcd_last_error(None).decode()
            assert not live, (fail_at, len(live))
    finally:
        L.fcd_set_allocator(fcd.ALLOC_FN(), fcd.FREE_FN(), None)
        fcd._torch_alloc = None
