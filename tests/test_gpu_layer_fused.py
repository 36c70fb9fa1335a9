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
    assert hb.layer_kernel_fused()  # BF16 operands in the same kernel
    hb.set_layer_kernel(2)
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


def test_bf16_fused_and_separate_against_oracle():
    """BF16 mode, N2: the fused kernel (electron-electron messages rounded to BF16 as the MMA
    operand, the electron-nucleus part on 3 x TF32) and the separate path (all messages in BF16)
    against the oracle within the BF16 per-walker bounds: |dE| <= max(1e-2 Ha, 2e-2 S_b) outside
    the FP32 contract's exception class, and log|psi| within the larger of 1e-2 relative and the
    first-order bound for one BF16 rounding of the orbital entries (2^-9 sigma_b).  The two paths
    agree with each other within the same bounds, and the fused BF16 path is deterministic."""
    from fp32_contract import bf16_logabs_bound
    wl = fx.workload("n2_fp32")
    h, theta, r, th_t, r_t = _setup(wl, 48, precision="bf16")
    o = oracle.Oracle(wl.system, wl.cfg)
    ref = o.local_energy(theta, r, with_grad=True)
    S = 0.5 * (np.abs(ref["lap"]) + np.sum(ref["grad"] ** 2, axis=1))
    e_tol = np.maximum(1e-2, 2e-2 * S)
    la_tol = bf16_logabs_bound(o, theta, r, ref["logabs"])
    nodal = near_nodal(o, theta, r, ref["logabs"])
    out = {}
    for mode in (1, 2):
        h.set_layer_kernel(mode)
        assert h.layer_kernel_fused() == (mode == 1)
        out[mode] = _np(h.local_energy(th_t, r_t))
        assert h.device_status() & 0x4 == 0
    for mode in (1, 2):
        la, sg, el = out[mode]
        e, dla = np.abs(el - ref["e_loc"]), np.abs(la - ref["logabs"])
        print(f"BF16 layer kernel {mode}: |dE|/tol max {np.max(e / e_tol):.2e} (outside the FP32 exception "
              f"class, {nodal.sum()} of {nodal.size} in it: {np.max((e / e_tol)[~nodal]):.2e}), median |dE|/S "
              f"{np.median(e / S):.2e}; |d log|psi|| / tol max {np.max(dla / la_tol):.2e}, rel. median "
              f"{np.median(dla / np.abs(ref['logabs'])):.2e}")
    for mode in (1, 2):
        la, sg, el = out[mode]
        assert np.all(np.abs(el - ref["e_loc"])[~nodal] <= e_tol[~nodal])
        assert np.all(np.abs(la - ref["logabs"]) <= la_tol)
    assert np.all(np.abs(out[1][2] - out[2][2])[~nodal] <= e_tol[~nodal])
    assert np.all(np.abs(out[1][0] - out[2][0]) <= la_tol)
    h.set_layer_kernel(1)
    a = h.local_energy(th_t, r_t)
    b = h.local_energy(th_t, r_t)
    for x, y in zip(a, b):
        assert torch.equal(x, y)
