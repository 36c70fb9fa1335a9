"""GB300-native hot path of real-space VMC with a DeepQMC-style GNN ansatz.

The computation lives in ``libdqmc.so`` (hand-written CUDA for sm_103a behind
the C ABI of ``include/dqmc.h``); :mod:`.binding` is a thin ctypes layer over
it and :mod:`.fixtures` produces seeded synthetic inputs.
"""
from .binding import (DQError, Ansatz, AnsatzBatch, LogAbsPsi, ansatz_eval, grad_logpsi, load_library, local_energy,
                      log_abs_psi, mcmc_step, vmc_loss_weights, vmc_train_step)

__all__ = ["DQError", "Ansatz", "AnsatzBatch", "LogAbsPsi", "ansatz_eval", "local_energy", "mcmc_step", "grad_logpsi",
           "vmc_loss_weights", "vmc_train_step", "log_abs_psi", "load_library"]
