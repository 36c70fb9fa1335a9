"""The sender-tiled jet message kernel (messages of Eq. 17 with the product rule, one spin block
of senders at a time with their node channels in registers) against the oracle and against the
general message kernel of the same library.

Bounds: the FP32 contract of tests/fp32_contract.py against the FP64 oracle for both kernels;
between the two (the same sums in different orders) log|psi| within 1e-5 max(1, |log|psi||) and
E_loc within max(1e-4 Ha, 1e-5 S_b) outside the contract's exception class, signs equal there.
Cases: C4H4 (28 electrons, 14 per spin, width 256, four layers: the 14-slot tile), benzene
(42 electrons, 21 per spin: the 24-slot tile), N2 on the separate layer path with the kernel
forced (7 per spin: the 8-slot tile), with node-map channels at layer 0 (el_init) so that every
layer takes it; BF16 message output is covered by the BF16 tests (C4H4)."""
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


def _np(ts):
    return [t.cpu().numpy() if t.dtype == torch.int8 else t.cpu().numpy().astype(np.float64) for t in ts]


def _case(name):
    if name == "c4h4":
        wl = fx.workload("c4h4_bf16")
        return wl.system, wl.cfg, wl.param_seed, wl.walker_seed, 16, 2048
    if name == "c6h6":
        wl = [w for w in fx.batch_workload("mixed_fp32") if w.system.name == "C6H6"][0]
        return wl.system, wl.cfg, wl.param_seed, wl.walker_seed, 4, 4
    wl = fx.workload("n2_fp32")
    return wl.system, dataclasses.replace(wl.cfg, el_init=1), wl.param_seed, wl.walker_seed, 32, 32


@pytest.mark.parametrize("name", ["c4h4", "c6h6", "n2_el_init"])
def test_sender_tiled_against_oracle_and_general(name):
    from paper_2307_14123_gb300 import Ansatz
    system, cfg, pseed, wseed, n_or, B = _case(name)
    h = Ansatz(system, cfg, "fp32", device="cuda:0")
    if name.startswith("n2"):
        h.set_layer_kernel(2)  # the separate path (N2 runs fused by default)
        assert h.msg_kernel() == 1
        h.set_msg_kernel(2)
    assert h.msg_kernel() == 2
    theta = fx.init_params(system, cfg, pseed).astype(np.float32).astype(np.float64)
    r = fx.init_walkers(system, B, wseed).astype(np.float32).astype(np.float64)
    idx = np.linspace(0, B - 1, n_or).astype(int)
    th_t = torch.tensor(theta, dtype=torch.float32, device="cuda:0")
    r_t = torch.tensor(r, dtype=torch.float32, device="cuda:0")
    tiled = _np(h.local_energy(th_t, r_t))
    assert h.device_status() & 0x4 == 0
    again = _np(h.local_energy(th_t, r_t))
    for x, y in zip(tiled, again):  # fixed summation orders
        assert np.array_equal(x, y)
    h.set_msg_kernel(1)
    assert h.msg_kernel() == 1
    general = _np(h.local_energy(th_t, r_t))
    o = oracle.Oracle(system, cfg)
    th64, r64 = theta, r[idx]
    ref = o.local_energy(th64, r64, with_grad=True)
    frac = 0.13 if name == "c4h4" else 0.05
    for lab, out in (("sender-tiled", tiled), ("general", general)):
        check_fp32_oracle(f"{name} {lab}", *[v[idx] for v in out], o, th64, r64, ref=ref, max_exception_frac=frac)
    (la2, sg2, el2), (la1, sg1, el1) = tiled, general
    nodal = near_nodal(o, th64, r64, ref["logabs"])
    ok = ~nodal
    S = 0.5 * (np.abs(ref["lap"]) + np.sum(ref["grad"] ** 2, axis=1))
    d_la = np.abs(la2[idx] - la1[idx])
    d_e = np.abs(el2[idx] - el1[idx])
    print(f"{name}: sender-tiled vs general: max |d log|psi|| {d_la.max():.2e}, max |dE|/S {np.max(d_e / S):.2e}; "
          f"all {B} walkers: max |d log|psi|| {np.max(np.abs(la2 - la1)):.2e}, "
          f"median |dE| {np.median(np.abs(el2 - el1)):.2e}")
    assert np.all(d_la[ok] <= 1e-5 * np.maximum(1, np.abs(ref["logabs"][ok])))
    assert np.all(d_e[ok] <= np.maximum(1e-4, 1e-5 * S[ok]))
    assert np.array_equal(sg2[idx][ok], sg1[idx][ok])


def test_msg_kernel_modes():
    """Mode 2 is refused on FP64 handles; mode 0 takes the sender-tiled kernel above 16
    electrons; out-of-range modes are argument errors."""
    from paper_2307_14123_gb300 import Ansatz
    from paper_2307_14123_gb300.binding import DQError
    wl = fx.workload("lih_fp64")
    h64 = Ansatz(wl.system, wl.cfg, "fp64", device="cuda:0")
    assert h64.msg_kernel() == 1
    with pytest.raises(DQError):
        h64.set_msg_kernel(2)
    with pytest.raises(DQError):
        h64.set_msg_kernel(3)
    c = fx.workload("c4h4_bf16")
    h = Ansatz(c.system, c.cfg, "bf16", device="cuda:0")
    assert h.msg_kernel() == 2
    h.set_msg_kernel(1)
    assert h.msg_kernel() == 1
    h.set_msg_kernel(0)
    assert h.msg_kernel() == 2
