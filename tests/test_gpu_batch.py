"""Batches of molecules with uneven electron counts (H2O, NH3, C2H4, C6H6) through
the grouped launches of the C ABI (``*_multi``).

Each molecule's results in the batch must equal, bit for bit, those of the
single-molecule calls on its own handle: both launch the same kernels (the
single-molecule calls with a one-entry table) and the same GEMM tiles per
walker.  The single-molecule path is checked against the oracle elsewhere
(tests/test_gpu_parity.py, including every molecule of this batch); the
full-size batch is also sampled against the oracle here, with the FP32 bounds
of the parity tests."""
import os

import numpy as np
import pytest
import torch

import oracle
from fp32_contract import check_fp32, fp32_floor, nodal_sensitivity
from paper_2307_14123_gb300 import fixtures as fx

pytestmark = pytest.mark.gpu
SMALL_B = (40, 33, 17, 6)  # ragged walker counts per molecule


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2307_14123_gb300 import _build
    _build.build()
    oracle.build()
    oracle.Oracle.set_threads(os.cpu_count() or 1)


def _setup(prec="fp32", B=SMALL_B, singles=True):
    from paper_2307_14123_gb300 import Ansatz, AnsatzBatch
    wls = fx.batch_workload("mixed_" + prec)
    batch = AnsatzBatch([w.system for w in wls], [w.cfg for w in wls], prec, device="cuda:0")
    hs = [Ansatz(w.system, w.cfg, prec, device="cuda:0") for w in wls] if singles else None
    th = [torch.tensor(fx.init_params(w.system, w.cfg, w.param_seed), dtype=torch.float32, device="cuda:0")
          for w in wls]
    r = [torch.tensor(fx.init_walkers(w.system, b, w.walker_seed), dtype=torch.float32, device="cuda:0")
         for w, b in zip(wls, B)]
    return wls, batch, hs, th, r


@pytest.mark.parametrize("rounds", [0, 2, 3])
def test_batch_local_energy_equals_single(rounds):
    wls, batch, singles, th, r = _setup()
    batch.set_rounds(rounds)
    la, sg, el, e2 = batch.local_energy(th, r, sums=True)
    for k, h in enumerate(singles):
        la1, sg1, el1, e21 = h.local_energy(th[k], r[k], sums=True)
        d = (el[k].double() - el1.double()).abs().max().item()
        assert torch.equal(la[k], la1) and torch.equal(sg[k], sg1) and torch.equal(el[k], el1), (wls[k].name, d)
        assert torch.equal(e2[k], e21)
        assert torch.isfinite(el[k]).all()


def test_batch_autotune_keeps_results():
    """The autotuner picks a tile shape among its candidates; results stay equal to the
    single-molecule calls (the message kernel's register tile does not change the order
    of any sum)."""
    wls, batch, singles, th, r = _setup()
    ms, rounds, ib = batch.autotune(th, r)
    assert ms > 0 and rounds in (1, 2, 3, 4) and ib in (4, 8)
    assert batch.tuning() == (rounds, ib)
    la, sg, el = batch.local_energy(th, r)
    for k, h in enumerate(singles):
        la1, sg1, el1 = h.local_energy(th[k], r[k])
        assert torch.equal(la[k], la1) and torch.equal(el[k], el1), (wls[k].name, rounds, ib)


def test_batch_eval_and_mcmc_equal_single():
    wls, batch, singles, th, r = _setup()
    la, sg = batch.ansatz_eval(th, r)
    r1 = [t.clone() for t in r]
    la1 = []
    for k, h in enumerate(singles):
        a, s = h.ansatz_eval(th[k], r[k])
        assert torch.equal(la[k], a) and torch.equal(sg[k], s)
        la1.append(a.clone())
    n = batch.mcmc_step(th, r, la, n_steps=3, step_size=0.2, seed=7, step_counter=5)
    for k, h in enumerate(singles):
        n1 = h.mcmc_step(th[k], r1[k], la1[k], n_steps=3, step_size=0.2, seed=7, step_counter=5)
        assert torch.equal(r[k], r1[k]) and torch.equal(la[k], la1[k]), wls[k].name
        assert int(n[k]) == int(n1.item())
    assert int(n.sum()) > 0


def test_batch_loss_weights_and_grad_equal_single():
    wls, batch, singles, th, r = _setup()
    _, _, el = batch.local_energy(th, r)
    w, stats = batch.vmc_loss_weights(el, 5.0)
    g = batch.grad_logpsi(th, r, w)
    for k, h in enumerate(singles):
        w1, st1 = h.vmc_loss_weights(el[k], 5.0)
        assert torch.equal(w[k], w1) and torch.equal(stats[k], st1)
        g1 = h.grad_logpsi(th[k], r[k], w1, 0)
        assert torch.equal(g[k], g1), wls[k].name
        assert g[k].shape == (batch.P[k],)


def test_batch_bf16_equals_single():
    wls, batch, singles, th, r = _setup("bf16")
    la, sg, el = batch.local_energy(th, r)
    for k, h in enumerate(singles):
        la1, sg1, el1 = h.local_energy(th[k], r[k])
        assert torch.equal(la[k], la1) and torch.equal(sg[k], sg1) and torch.equal(el[k], el1), wls[k].name


def test_batch_with_empty_molecule():
    wls, batch, singles, th, r = _setup(B=(12, 0, 9, 3))
    la, sg, el, e2 = batch.local_energy(th, r, sums=True)
    assert la[1].numel() == 0 and float(e2[1].abs().sum()) == 0.0
    for k in (0, 2, 3):
        la1, sg1, el1 = singles[k].local_energy(th[k], r[k])
        assert torch.equal(el[k], el1)
    n = batch.mcmc_step(th, r, la, n_steps=1, seed=1)
    assert int(n[1]) == 0


def test_batch_vmc_step_graph_replay():
    """The batch's VMC step (Metropolis sweep with the counter on the device, local
    energies, loss weights, gradients) captured once as a CUDA graph and replayed
    equals the same steps run eagerly."""
    wls, batch, _, th, r = _setup(singles=False)
    la, _ = batch.ansatz_eval(th, r)
    r_e, la_e = [t.clone() for t in r], [t.clone() for t in la]
    ctr = torch.zeros(1, dtype=torch.int64, device="cuda:0")

    def step(rr, ll, c):
        batch.mcmc_step(th, rr, ll, 1, 0.2, 3, c)
        _, _, el = batch.local_energy(th, rr)
        w, _ = batch.vmc_loss_weights(el, 5.0)
        return el, batch.grad_logpsi(th, rr, w)

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):  # warm-up outside capture (workspace allocated here)
        step([t.clone() for t in r], [t.clone() for t in la], torch.zeros(1, dtype=torch.int64, device="cuda:0"))
    torch.cuda.current_stream().wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        el_g, gr_g = step(r, la, ctr)
    for t in range(2):
        g.replay()
        el_e, gr_e = step(r_e, la_e, t)
        torch.cuda.synchronize()
        for k in range(batch.n):
            assert torch.equal(r[k], r_e[k]) and torch.equal(el_g[k], el_e[k]) and torch.equal(gr_g[k], gr_e[k])
    assert int(ctr.item()) == 2


def test_batch_full_size_sampled():
    """The benchmark batch (8192, 8192, 4096, 2048 walkers) in one call; sampled
    walkers of every molecule against the oracle (FP32 bounds of the parity tests)."""
    full = tuple(w.B for w in fx.batch_workload("mixed_fp32"))
    wls, batch, _, th, r = _setup(B=full, singles=False)
    la, sg, el = batch.local_energy(th, r)
    rng = np.random.default_rng(0)
    for k, w in enumerate(wls):
        n_s = 2 if w.system.n_elec > 40 else 4
        idx = np.unique(np.concatenate([[0, w.B - 1], rng.choice(w.B, n_s, replace=False)]))[: n_s + 1]
        theta = fx.init_params(w.system, w.cfg, w.param_seed).astype(np.float32).astype(np.float64)
        rs = r[k].cpu().numpy().astype(np.float64)[idx]
        o = oracle.Oracle(w.system, w.cfg)
        ref = o.local_energy(theta, rs, with_grad=True)
        oc, oshape = fx.param_offsets(w.system, w.cfg)["c"]
        check_fp32(f"{w.name} ({idx.size} sampled walkers)", la[k].cpu().numpy()[idx], sg[k].cpu().numpy()[idx],
                   el[k].cpu().numpy()[idx], ref, nodal_sensitivity(o, theta, rs, theta[oc:oc + oshape[0]]),
                   max_exception_frac=0.34, f32=fp32_floor(o, theta, rs))
