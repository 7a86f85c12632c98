"""crm_eval_noalloc: the entry point for callers that cannot allocate device memory.

Callers such as work recorded under stream capture (where cudaMalloc is not allowed),
serving processes with a fixed device-memory budget, or code inside another component's
memory manager use this entry point; it keeps its scratch in a statically reserved
device array instead of allocating.  This test calls it through the C ABI and checks its
output against crm_eval_form's, bit for bit (the tolerance of every parity test here),
on two calls in a row, and checks that oversized calls are rejected.  The file name makes
pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

CRM_F32 = 0
CRM_ERR_SIZE = 11
MAX_ELEMS = 1 << 20  # CRM_NOALLOC_MAX_ELEMS in include/crm.h


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2605_15547_gb300 import _lib as L
    lib = L.lib()
    lib.crm_eval_noalloc.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]
    lib.crm_noalloc_stats.argtypes = [ctypes.c_void_p, ctypes.POINTER(L.crm_stats_t)]
    lib.crm_noalloc_stats_reset.argtypes = [ctypes.c_void_p]
    return lib


def _noalloc_stats(lib):
    from paper_2605_15547_gb300 import _lib as L
    s = L.crm_stats_t()
    assert lib.crm_noalloc_stats(_stream(), ctypes.byref(s)) == 0
    return s


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _inputs(func, n, seed):
    from paper_2605_15547_gb300 import workloads as W
    x = W.domain_bits(func, n, np.random.Generator(np.random.PCG64(seed))).view(np.float32)
    return torch.from_numpy(x).cuda()


def _run(lib, entry, fid, form, x, rows):
    out = torch.full((rows * x.numel(),), float("nan"), dtype=torch.float32, device="cuda")
    fn = lib.crm_eval_noalloc if entry == "noalloc" else lib.crm_eval_form
    st = fn(fid, CRM_F32, form, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
            x.numel(), _stream())
    assert st == 0, st
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("func,fid,rows", [("expf", 0, 1), ("logf", 4, 1), ("sincosf", 10, 2)])
def test_noalloc_matches_allocating_entry_point(lib, func, fid, rows):
    for form in (0, 1, 2):  # auto, plain, double-float (where the function has it)
        probe = torch.ones(4, device="cuda")
        if lib.crm_eval_form(fid, CRM_F32, form, ctypes.c_void_p(probe.data_ptr()),
                             ctypes.c_void_p(torch.empty(8, device="cuda").data_ptr()), 4, _stream()):
            continue
        # two calls in a row, different inputs and sizes (a ragged tail, then the maximum),
        # the second with every lane forced through the queue in the static scratch
        for call, (n, force) in enumerate([(300001, 0), (MAX_ELEMS, 1)]):
            x = _inputs(func, n, 1234 + call)
            assert lib.crm_noalloc_stats_reset(_stream()) == 0
            lib.crm_set_force_slow(force)
            try:
                got = _run(lib, "noalloc", fid, form, x, rows)
                want = _run(lib, "form", fid, form, x, rows)
            finally:
                lib.crm_set_force_slow(0)
            assert np.array_equal(got, want), f"{func} form {form} call {call}: " \
                f"{int(np.count_nonzero(got != want))} mismatches"
            # the static scratch's counters: no lane undecided, no bounded wait gave up,
            # no lane finished inline (the queue holds every lane); a forced call queued
            # every lane that is not a special input
            st = _noalloc_stats(lib)
            assert st.unresolved_total == 0 and st.timeouts == 0 and st.inline_total == 0, \
                (st.unresolved_total, st.timeouts, st.inline_total)
            if force:
                assert st.hard_total > n // 2 and st.last_count == st.hard_total, st.hard_total


def test_noalloc_rejects_oversized_calls(lib):
    x = torch.ones(MAX_ELEMS + 1, device="cuda")
    y = torch.empty_like(x)
    st = lib.crm_eval_noalloc(0, CRM_F32, 0, ctypes.c_void_p(x.data_ptr()),
                              ctypes.c_void_p(y.data_ptr()), MAX_ELEMS + 1, _stream())
    assert st == CRM_ERR_SIZE
    assert b"CRM_NOALLOC_MAX_ELEMS" in lib.crm_status_str(st)


def test_noalloc_under_graph_capture(lib):
    """The entry point's reason to exist: a call recorded in a CUDA graph (global capture
    mode, where allocation is prohibited) and replayed on new inputs gives crm_eval_form's
    bits; an uncaptured call leaves the device's free memory unchanged."""
    n = 300001
    x = _inputs("expf", n, 77)
    y = torch.empty_like(x)

    def call(stream):
        return lib.crm_eval_noalloc(0, CRM_F32, 0, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                    n, stream)

    assert call(_stream()) == 0  # the first call on the device, before any capture
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    assert call(_stream()) == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        st = call(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    for seed in (78, 79):
        x.copy_(_inputs("expf", n, seed))
        y.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        want = _run(lib, "form", 0, 0, x, 1)
        assert np.array_equal(y.cpu().numpy().view(np.uint32), want), seed
