"""mcmc_step_eloc: Metropolis steps whose proposals are evaluated by the jets forward, carrying
E_loc with the positions (one forward per VMC step instead of a value-only forward and a
local_energy call).

* teacher-forced against the oracle's Metropolis step (the same Philox draws): LiH in FP64
  over 10 steps, positions to 1e-12, decisions equal outside a 1e-8 band at the threshold;
* after every step, logabs and e_loc equal local_energy at the new positions bit for bit
  (FP64 and FP32: accepted walkers take the proposal's values from the same forward,
  rejected ones keep theirs);
* FP64: the same chain as mcmc_step (whose value-only forward agrees to rounding);
* the device step counter advances and replays the same draws.
"""
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


def _setup(name, precision, B):
    from paper_2307_14123_gb300 import Ansatz
    wl = fx.workload(name)
    h = Ansatz(wl.system, wl.cfg, precision, device="cuda:0")
    dt = torch.float64 if precision == "fp64" else torch.float32
    theta = fx.init_params(wl.system, wl.cfg, wl.param_seed)
    r = fx.init_walkers(wl.system, B, wl.walker_seed)
    if precision != "fp64":
        theta = theta.astype(np.float32).astype(np.float64)
        r = r.astype(np.float32).astype(np.float64)
    th_t = torch.tensor(theta, dtype=dt, device="cuda:0")
    r_t = torch.tensor(r, dtype=dt, device="cuda:0")
    return wl, h, theta, th_t, r_t


def test_lih_fp64_teacher_forced_and_self_consistent():
    wl, h, theta, th_t, r_t = _setup("lih_fp64", "fp64", 256)
    o = oracle.Oracle(wl.system, wl.cfg)
    la_t, _, el_t = h.local_energy(th_t, r_t)
    step = wl.extra["step_size"]
    for t in range(10):
        r_prev = r_t.cpu().numpy()
        la_prev = la_t.cpu().numpy()
        n_acc = h.mcmc_step_eloc(th_t, r_t, la_t, el_t, n_steps=1, step_size=step, seed=wl.walker_seed,
                                 step_counter=t)
        r_new = r_t.cpu().numpy()
        xi, u = fx.metropolis_draws(wl.walker_seed, r_new.shape[0], wl.system.n_elec, t)
        ro, lo, acc = o.metropolis_step(theta, r_prev, la_prev, xi, u, step)
        gpu_acc = np.any(r_new != r_prev, axis=(1, 2))
        assert int(n_acc.item()) == int(gpu_acc.sum())
        diff = gpu_acc != acc.astype(bool)
        if diff.any():  # only where the decision sits on the threshold
            lp, _ = o.evaluate(theta, r_prev[diff] + step * xi[diff])
            assert np.all(np.abs(np.log(u[diff]) - 2 * (lp - la_prev[diff])) < 1e-8)
        np.testing.assert_allclose(r_new[~diff], ro[~diff], rtol=0, atol=1e-12)
        # the carried values are local_energy's at the new positions, bit for bit
        la_ref, _, el_ref = h.local_energy(th_t, r_t)
        assert torch.equal(la_t, la_ref) and torch.equal(el_t, el_ref)
    assert 0 < int(n_acc.item()) < r_new.shape[0]


def test_fp64_same_chain_as_mcmc_step():
    wl, h, _, th_t, r_t = _setup("lih_fp64", "fp64", 512)
    la_t, _, el_t = h.local_energy(th_t, r_t)
    r2 = r_t.clone()
    la2, _ = h.ansatz_eval(th_t, r2)
    n1 = h.mcmc_step_eloc(th_t, r_t, la_t, el_t, n_steps=5, step_size=0.2, seed=3, step_counter=40)
    n2 = h.mcmc_step(th_t, r2, la2, n_steps=5, step_size=0.2, seed=3, step_counter=40)
    assert torch.equal(r_t, r2) and int(n1.item()) == int(n2.item())
    assert torch.allclose(la_t, la2, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("name", ["n2_fp32"])
def test_fp32_carried_values_equal_local_energy(name):
    wl, h, _, th_t, r_t = _setup(name, "fp32", 2048)
    la_t, _, el_t = h.local_energy(th_t, r_t)
    ctr = torch.zeros(1, dtype=torch.int64, device="cuda:0")
    r0 = r_t.clone()
    for _ in range(3):
        h.mcmc_step_eloc(th_t, r_t, la_t, el_t, n_steps=1, step_size=0.2, seed=wl.walker_seed, step_counter=ctr)
    assert int(ctr.item()) == 3
    la_ref, _, el_ref = h.local_energy(th_t, r_t)
    assert torch.equal(la_t, la_ref) and torch.equal(el_t, el_ref)
    moved = (r_t != r0).any(dim=2).any(dim=1).float().mean().item()
    assert 0.2 < moved < 1.0
    # the host counter gives the same chain as the device counter
    r1 = r0.clone()
    la1, _, el1 = h.local_energy(th_t, r1)
    for t in range(3):
        h.mcmc_step_eloc(th_t, r1, la1, el1, n_steps=1, step_size=0.2, seed=wl.walker_seed, step_counter=t)
    assert torch.equal(r1, r_t) and torch.equal(el1, el_t)
