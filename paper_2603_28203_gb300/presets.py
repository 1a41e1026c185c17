"""Optimiser settings (dpf_solve_opts fields) used by the workloads.

TABLE2: the paper's Table 2 (Adam betas, ReduceLROnPlateau), the library's
defaults apart from the learning rate.

N1_WARM: N-1 cases started from the base case's solution (the paper's
warm-start idea of Sec. 5.4.2 applied to contingencies).  Table 2's plateau
rule lowers the rate whenever the loss improves by less than 6.73% within 41
iterations, which on a warm-started 2,000-bus N-1 case stops the progress
within a few thousand iterations.  These values come from a random search of
the kind Sec. 5.3 describes (1,481 seeded draws of optimiser, rate, betas,
eps and scheduler settings, each scored by the cases of a 512-case subset of
the 2,000-bus N-1 batch that reach 1e-6 p.u. within 3,000 iterations, FP32R),
rounded to two or three digits: Adam with a slowly decaying plateau rule
(relative threshold 4.4e-4).
"""
from . import _abi

TABLE2 = dict(optimizer=_abi.OPT_ADAM, beta1=0.979, beta2=0.963, eps=1e-8, sched=_abi.SCHED_PLATEAU, factor=0.547,
              patience=41, threshold=0.0673, cooldown=97)

N1_WARM = dict(optimizer=_abi.OPT_ADAM, lr=7.7e-5, beta1=0.977, beta2=0.983, eps=8.7e-10, sched=_abi.SCHED_PLATEAU,
               factor=0.70, patience=65, threshold=4.4e-4, cooldown=80)
