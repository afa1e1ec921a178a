"""The allocation-free sampler entry point (epll_sample_noalloc).

Callers that cannot allocate device memory while they run use this entry
point: its scratch is a static device array inside the library, so only the
output buffer comes from the caller.  Its anchors must be identical to those
of epll_sample (the allocating entry point) for every sampler, on two calls
in a row (the second call reuses the array the first one left behind).
This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1710_08124_gb300 as ep  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    ep.build()


CASES = [
    (64, 64, ep.SUBSET_FRACTION, 1 / 3),
    (129, 200, ep.SUBSET_FRACTION, 0.05),
    (512, 512, ep.SUBSET_FRACTION, 1 / 3),
    (50, 37, ep.SUBSET_JITTER, 6),
    (1024, 1024, ep.SUBSET_JITTER, 3),
    (1024, 1024, ep.SUBSET_FRACTION, 1 / 3),   # the largest image the static scratch serves
    (1024, 1023, ep.SUBSET_FRACTION, 0.01),
    (50, 37, ep.SUBSET_REGULAR, 4),
    (33, 40, ep.SUBSET_ALL, 0.0),
    (30, 41, ep.SUBSET_VALID, 0.0),
]


@pytest.mark.parametrize("H,W,kind,param", CASES)
def test_matches_allocating_sampler_two_calls(H, W, kind, param):
    L = ep.lib()
    out = torch.full((H * W,), -1, dtype=torch.int32, device="cuda")
    for t in (0, 1):  # two calls in a row; the second reuses the static scratch
        o = ep.Options(subset=kind, subset_param=param, seed=99)
        opt = o._c()
        n = C.c_int(0)
        st = L.epll_sample_noalloc(H, W, C.byref(opt), t, out.data_ptr(), C.byref(n),
                                   torch.cuda.current_stream().cuda_stream)
        assert st == ep.OK, ep.last_error()
        torch.cuda.synchronize()
        got = out[:n.value].cpu().numpy()
        ref = ep.sample(H, W, o, t).cpu().numpy()
        assert np.array_equal(got, ref), (H, W, kind, param, t)


def test_rejects_images_beyond_the_static_scratch():
    L = ep.lib()
    out = torch.empty(16, dtype=torch.int32, device="cuda")
    opt = ep.Options(subset=ep.SUBSET_FRACTION, subset_param=0.5)._c()
    n = C.c_int(0)
    st = L.epll_sample_noalloc(1025, 1024, C.byref(opt), 0, out.data_ptr(), C.byref(n), None)
    assert st == ep.EINVAL
    assert "2^20" in ep.last_error()


def test_binding_rejects_a_short_or_misplaced_output():
    short = torch.empty(64 * 64 - 1, dtype=torch.int32, device="cuda")
    with pytest.raises(ValueError):
        ep.sample_noalloc(64, 64, ep.Options(subset=ep.SUBSET_FRACTION, subset_param=0.5), out=short)
    with pytest.raises(ValueError):
        ep.sample_noalloc(16, 16, ep.Options(), out=torch.empty(256, dtype=torch.int32))
    got = ep.sample_noalloc(64, 64, ep.Options(subset=ep.SUBSET_FRACTION, subset_param=0.5),
                            out=torch.empty(64 * 64, dtype=torch.int32, device="cuda"))
    ref = ep.sample(64, 64, ep.Options(subset=ep.SUBSET_FRACTION, subset_param=0.5))
    assert torch.equal(got, ref)


def test_rejects_what_the_allocating_sampler_rejects():
    L = ep.lib()
    out = torch.empty(256, dtype=torch.int32, device="cuda")
    n = C.c_int(0)
    for bad in (ep.Options(precision=99), ep.Options(cg_iters=-1), ep.Options(select=7),
                ep.Options(subset=ep.SUBSET_JITTER, subset_param=2.5)):
        opt = bad._c()
        assert L.epll_sample_noalloc(16, 16, C.byref(opt), 0, out.data_ptr(), C.byref(n), None) == ep.EINVAL
        assert L.epll_sample(16, 16, C.byref(opt), 0, out.data_ptr(), C.byref(n), None) == ep.EINVAL
