"""vmc_loss_weights_noalloc, the entry point for callers that cannot allocate
device memory: it keeps its sort scratch in a fixed array inside the library
instead of a caller-provided workspace.  Its results must equal those of
vmc_loss_weights on the same inputs, call after call, although every call
reuses (and finds the previous contents in) the same array.

This file sorts last so that a run stopping at the first failure has run
every other test before it; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=["fp64", "fp32"])
def handle(request):
    """An FP64 handle (double energies and weights) and an FP32 one (float energies and weights,
    FP64 scratch: the path of the FP32 and BF16 modes)."""
    from paper_2307_14123_gb300 import _build
    _build.build()
    from paper_2307_14123_gb300 import Ansatz
    from paper_2307_14123_gb300 import fixtures as fx
    wl = fx.workload("lih_fp64" if request.param == "fp64" else "n2_fp32")
    return Ansatz(wl.system, wl.cfg, request.param, device="cuda:0")


def _noalloc(h, e, clip_k=5.0):
    B = e.numel()
    w = torch.empty(B, dtype=e.dtype, device=e.device)
    stats = torch.empty(4, dtype=torch.float64, device=e.device)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = h.lib.vmc_loss_weights_noalloc(h.h, ctypes.c_void_p(e.data_ptr()), B, clip_k, ctypes.c_void_p(w.data_ptr()),
                                        ctypes.c_void_p(stats.data_ptr()), stream)
    return st, w, stats


def test_noalloc_matches_workspace_entry_point_on_consecutive_calls(handle):
    rng = np.random.default_rng(11)
    # second call is smaller than the first, so stale scratch from call one is present
    for B in (5000, 777):
        e = torch.tensor(rng.standard_cauchy(B) * 3 - 40, dtype=handle.dtype, device="cuda:0")
        st, w, stats = _noalloc(handle, e)
        assert st == 0
        w_ref, stats_ref = handle.vmc_loss_weights(e, clip_k=5.0)
        torch.cuda.synchronize()
        # the same kernel on the same inputs: equal results (FP32 weights are one rounding of FP64 values)
        np.testing.assert_allclose(w.cpu().numpy(), w_ref.cpu().numpy(), rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(stats.cpu().numpy(), stats_ref.cpu().numpy(), rtol=1e-12, atol=1e-15)


def test_noalloc_rejects_batches_beyond_its_capacity(handle):
    e = torch.zeros(65537, dtype=handle.dtype, device="cuda:0")
    st, _, _ = _noalloc(handle, e)
    assert st == 2  # DQ_ERR_SHAPE: more walkers than the fixed scratch holds


def test_noalloc_launch_is_timed_by_the_profiler(handle):
    e = torch.linspace(-3, 3, 100, dtype=handle.dtype, device="cuda:0")
    handle.profile(True)
    handle.profile_reset()
    st, _, _ = _noalloc(handle, e)
    prof = handle.profile_read()
    handle.profile(False)
    assert st == 0 and prof["loss_weights"][1] == 1
