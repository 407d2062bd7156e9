"""fp_rates4_noalloc: the allocation-free rate entry point, checked against fp_rates4.

This entry point exists for callers that must not allocate device memory during the call
(their device memory is owned by another allocator with a fixed budget, or they cannot accept
the synchronisation of cudaFree).  It takes its working memory from a 16 MiB static device
array instead of cudaMalloc.  The test calls it through the C-ABI twice in a row -- the second
call sees the array as the first call left it -- and compares both results with fp_rates4 at
the FP64 parity tolerance.  It lives in its own file, collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_2104_04895_gb300 import synth

from conftest import oracle_modes

pytestmark = pytest.mark.gpu

RTOL_FP64 = 1e-10


def _entry(binding):
    L = binding.load()
    f = L.fp_rates4_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                  ctypes.POINTER(binding.fp_rates_opts), ctypes.c_void_p, ctypes.POINTER(binding.fp_stats)]
    f.restype = ctypes.c_int
    return L, f


def test_noalloc_matches_fp_rates4_on_two_calls():
    """Both calls match fp_rates4; the second call, on a warmed context (the first call has loaded the module and
    looked up the array), changes the device's free memory by nothing and repeats the first result bit for bit."""
    import torch
    from paper_2104_04895_gb300 import binding
    L, f = _entry(binding)
    cr = synth.diamond_si((3, 3, 2))
    w, e, v = oracle_modes(cr)
    temps = np.array([300.0, 800.0])
    with binding.Context.from_crystal(cr) as ctx:
        ctx.set_modes(w, e, v)
        ref, st_ref = ctx.rates4(temps, cr.scalebroad)
        out = torch.full((len(temps) * cr.nq * cr.nb,), float("nan"), dtype=torch.float64, device="cuda")
        T = np.ascontiguousarray(temps)
        results = []
        for call in range(2):
            o, _ = ctx.make_opts()
            st = binding.fp_stats()
            out.fill_(float("nan"))
            torch.cuda.synchronize()
            free_before = torch.cuda.mem_get_info()[0]
            rc = f(ctx.h, len(T), T.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), cr.scalebroad,
                   ctypes.byref(o), ctypes.c_void_p(out.data_ptr()), ctypes.byref(st))
            assert rc == binding.FP_OK, L.fp_last_error(ctx.h)
            torch.cuda.synchronize()
            free_after = torch.cuda.mem_get_info()[0]
            if call == 1:
                assert free_after == free_before, (free_before, free_after)
            got = out.cpu().numpy().reshape(ref.shape)
            results.append(got)
            zero = ref == 0.0
            assert np.all(got[zero] == 0.0)
            rel = np.abs(got[~zero] - ref[~zero]) / np.abs(ref[~zero])
            assert rel.max() <= RTOL_FP64, (call, rel.max())
            assert list(st.accepted) == st_ref["accepted"], call
        assert np.array_equal(results[0], results[1])


def test_noalloc_rejects_problems_beyond_the_static_scratch():
    import torch
    from paper_2104_04895_gb300 import binding
    L, f = _entry(binding)
    cr = synth.licoo2((16, 16, 16))
    temps = np.linspace(300.0, 1000.0, 8)
    with binding.Context.from_crystal(cr) as ctx:
        ctx.modes(copy=False)
        out = torch.zeros(len(temps) * cr.nq * cr.nb, dtype=torch.float64, device="cuda")
        o, _ = ctx.make_opts()
        st = binding.fp_stats()
        rc = f(ctx.h, len(temps), np.ascontiguousarray(temps).ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
               1.0, ctypes.byref(o), ctypes.c_void_p(out.data_ptr()), ctypes.byref(st))
        assert rc == binding.FP_EINVAL
        assert b"static scratch" in L.fp_last_error(ctx.h)
