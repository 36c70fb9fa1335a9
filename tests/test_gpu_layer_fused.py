"""The fused jet layer (messages of Eq. 17 as the tensor-core operand of the update map W_g,
and the residual tanh jet update of Eq. 18, in one kernel) against the oracle and against
the separate message / W_g GEMM / update kernels of the same library.

Bounds: the FP32 contract of tests/fp32_contract.py against the FP64 oracle for both
paths; between the two paths (the same quantities summed in different orders, both with
three-product TF32 GEMMs) log|psi| within 1e-5 max(1, |log|psi||) and E_loc within
max(1e-4 Ha, 1e-5 S_b) outside the contract's exception class.  The fused path is
deterministic (fixed summation orders) and independent of the walker chunking."""
import dataclasses
import os

import numpy as np
import pytest
import torch

import oracle
from fp32_contract import check_fp32_oracle, near_nodal
from paper_2307_14123_gb300 import fixtures as fx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2307_14123_gb300 import _build
    _build.build()
    oracle.build()
    oracle.Oracle.set_threads(os.cpu_count() or 1)


def _setup(wl, B, precision="fp32", cfg=None, walker_seed=None):
    from paper_2307_14123_gb300 import Ansatz
    cfg = cfg or wl.cfg
    h = Ansatz(wl.system, cfg, precision, device="cuda:0")
    theta = fx.init_params(wl.system, cfg, wl.param_seed).astype(np.float32).astype(np.float64)
    r = fx.init_walkers(wl.system, B, wl.walker_seed if walker_seed is None else walker_seed)
    r = r.astype(np.float32).astype(np.float64)
    th_t = torch.tensor(theta, dtype=torch.float32, device="cuda:0")
    r_t = torch.tensor(r, dtype=torch.float32, device="cuda:0")
    return h, theta, r, th_t, r_t


def _np(ts):
    return [t.cpu().numpy() if t.dtype == torch.int8 else t.cpu().numpy().astype(np.float64) for t in ts]


def test_support_and_mode_switch():
    from paper_2307_14123_gb300.binding import DQError
    h, *_ = _setup(fx.workload("n2_fp32"), 1)
    assert h.layer_kernel_fused()  # the default for N2 in FP32
    h.set_layer_kernel(2)
    assert not h.layer_kernel_fused()
    h.set_layer_kernel(0)
    assert h.layer_kernel_fused()
    wl = fx.workload("lih_fp64")  # width 32: separate kernels only
    h32, *_ = _setup(wl, 1)
    assert not h32.layer_kernel_fused()
    with pytest.raises(DQError):
        h32.set_layer_kernel(1)
    hb, *_ = _setup(fx.workload("n2_bf16"), 1, precision="bf16")
    assert not hb.layer_kernel_fused()


@pytest.mark.parametrize("variant", ["base", "el_init", "edge_update"])
def test_fused_and_separate_against_oracle(variant):
    """N2 (14 electrons, D=128, 3 layers): both layer paths against the oracle, and against each
    other.  el_init runs layer 0 on node channels from the node map (not the spin-embedding
    constants); edge_update feeds the filters from iterated edge embeddings."""
    wl = fx.workload("n2_fp32")
    cfg = wl.cfg if variant == "base" else dataclasses.replace(wl.cfg, **{variant: 1})
    h, theta, r, th_t, r_t = _setup(wl, 48, cfg=cfg)
    o = oracle.Oracle(wl.system, cfg)
    ref = o.local_energy(theta, r, with_grad=True)
    out = {}
    for mode in (1, 2):
        h.set_layer_kernel(mode)
        out[mode] = _np(h.local_energy(th_t, r_t))
        check_fp32_oracle(f"N2 {variant} layer kernel {mode}", *out[mode], o, theta, r, ref=ref)
    (la1, sg1, el1), (la2, sg2, el2) = out[1], out[2]
    nodal = near_nodal(o, theta, r, ref["logabs"])
    S = 0.5 * (np.abs(ref["lap"]) + np.sum(ref["grad"] ** 2, axis=1))
    ok = ~nodal
    print(f"fused vs separate: max |d log|psi|| {np.max(np.abs(la1 - la2)):.2e}, "
          f"max |dE|/S {np.max(np.abs(el1 - el2) / S):.2e}")
    assert np.all(np.abs(la1 - la2)[ok] <= 1e-5 * np.maximum(1, np.abs(ref["logabs"][ok])))
    assert np.all(np.abs(el1 - el2)[ok] <= np.maximum(1e-4, 1e-5 * S[ok]))
    assert np.array_equal(sg1[ok], sg2[ok])


def test_fused_deterministic_and_chunk_independent():
    """Two calls give the same bits; so do walker chunks of 100 (ragged last chunk) and the whole
    batch in one chunk (each walker's tiles run the same operations in the same order)."""
    wl = fx.workload("n2_fp32")
    h, _, _, th_t, r_t = _setup(wl, 300)
    a = h.local_energy(th_t, r_t)
    b = h.local_energy(th_t, r_t)
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    h.set_max_chunk(100)
    c = h.local_energy(th_t, r_t)
    for x, y in zip(a, c):
        assert torch.equal(x, y)


@pytest.mark.parametrize("k", range(3))
def test_fused_small_molecules(k):
    """H2O, NH3 (10 electrons, three tiles per walker) and C2H4 (16 electrons, eight channels
    per tile, seven tiles): the fused path against the oracle."""
    w = fx.batch_workload("mixed_fp32")[k]
    h, theta, r, th_t, r_t = _setup(w, 16)
    assert h.layer_kernel_fused()
    o = oracle.Oracle(w.system, w.cfg)
    check_fp32_oracle(f"{w.name} fused", *_np(h.local_energy(th_t, r_t)), o, theta, r, max_exception_frac=0.13)
