"""Pseudopotential energies (Eqs. 11 and 12) on the GPU against
the oracle's quadrature on the same walkers, rotations and (synthetic) coefficients.

Bounds: FP64 mode 1e-10 relative (of sum |w psi'/psi|, the size of the quadrature
sum; of |V_loc|).  FP32 mode: the psi ratios come from FP32 log|psi| values
(errors up to 1e-4 max(1, |log psi|), the local-energy parity bound), so a ratio
carries a relative error of up to 2e-4 |log psi| and the bound is that times the
quadrature's absolute sum."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2307_14123_gb300 import fixtures as fx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2307_14123_gb300 import _build
    _build.build()
    oracle.build()
    oracle.Oracle.set_threads(os.cpu_count() or 1)


def _run(name, prec, B, pps, seed):
    from paper_2307_14123_gb300 import Ansatz
    wl = fx.workload(name)
    h = Ansatz(wl.system, wl.cfg, prec, device="cuda:0")
    theta = fx.init_params(wl.system, wl.cfg, wl.param_seed)
    r = fx.init_walkers(wl.system, B, wl.walker_seed)
    rot = fx.random_rotations(B, seed)
    if prec != "fp64":
        theta = theta.astype(np.float32).astype(np.float64)
        r = r.astype(np.float32).astype(np.float64)
        rot = rot.astype(np.float32).astype(np.float64)
    dt = torch.float64 if prec == "fp64" else torch.float32
    th_t, r_t = torch.tensor(theta, dtype=dt, device="cuda:0"), torch.tensor(r, dtype=dt, device="cuda:0")
    la, sg = h.ansatz_eval(th_t, r_t)
    v_loc, v_nl = h.pseudopotential_energy(th_t, r_t, pps, torch.tensor(rot, dtype=dt, device="cuda:0"), la, sg)
    o = oracle.Oracle(wl.system, wl.cfg)
    ref_loc, ref_nl, scale = oracle.pseudopotential(o, theta, r, pps, rot, with_abs=True)
    return (v_loc.cpu().numpy().astype(np.float64), v_nl.cpu().numpy().astype(np.float64), ref_loc, ref_nl,
            scale, la.cpu().numpy().astype(np.float64))


def test_pseudopotential_lih_fp64():
    pps = [(0, fx.synthetic_pseudopotential(2, seed=1))]
    v_loc, v_nl, ref_loc, ref_nl, scale, _ = _run("lih_fp64", "fp64", 16, pps, 3)
    np.testing.assert_allclose(v_loc, ref_loc, rtol=1e-10, atol=1e-12)
    assert np.all(np.abs(v_nl - ref_nl) <= 1e-10 * np.maximum(scale, 1e-12))


def test_pseudopotential_lih_two_nuclei_fp64():
    pps = [(0, fx.synthetic_pseudopotential(3, seed=2)), (1, fx.synthetic_pseudopotential(1, seed=3))]
    v_loc, v_nl, ref_loc, ref_nl, scale, _ = _run("lih_fp64", "fp64", 8, pps, 4)
    np.testing.assert_allclose(v_loc, ref_loc, rtol=1e-10, atol=1e-12)
    assert np.all(np.abs(v_nl - ref_nl) <= 1e-10 * np.maximum(scale, 1e-12))


def test_pseudopotential_n2_fp32():
    pps = [(0, fx.synthetic_pseudopotential(2, seed=5)), (1, fx.synthetic_pseudopotential(2, seed=6))]
    v_loc, v_nl, ref_loc, ref_nl, scale, la = _run("n2_fp32", "fp32", 6, pps, 7)
    np.testing.assert_allclose(v_loc, ref_loc, rtol=1e-5, atol=1e-5)
    tol = 2e-4 * np.maximum(1, np.abs(la)) * scale
    err = np.abs(v_nl - ref_nl)
    print("N2 FP32 V_NL: max err / bound %.2e" % np.max(err / tol))
    assert np.all(err <= tol)
