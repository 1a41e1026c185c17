"""Optimiser settings (dpf_solve_opts fields) used by the workloads.

TABLE2: the paper's Table 2 (Adam betas, ReduceLROnPlateau), the library's
defaults apart from the learning rate.

N1_WARM: N-1 cases started from the base case's solution (the paper's
warm-start idea of Sec. 5.4.2 applied to contingencies).  Table 2's plateau
rule lowers the rate whenever the loss improves by less than 6.73% within 41
iterations, which on a warm-started 2,000-bus N-1 case stops the progress
within a few thousand iterations.  These values come from a search of the
kind Sec. 5.3 describes, in two stages, each candidate scored by the cases of
a subset of the 2,000-bus N-1 batch that reach 1e-6 p.u. within 3,000
refined-FP32 iterations: 1,481 seeded random draws of optimiser (Adam, SGD,
RMSprop), rate, betas, eps and scheduler (plateau, StepLR, constant) on 512
cases, then 1,250 seeded perturbations of the best draw on 1,024 cases (FP64
test every 50 iterations, gate 5e-6), kept to six digits (rounding them to
two or three changes which cases converge: 33 instead of 40 of the 2,379
within 3,000 iterations, a measure of how noisy the count is).  Adam with a
plateau rule that lowers the rate only after ~120 iterations without a 0.2%
improvement.
"""
from . import _abi

TABLE2 = dict(optimizer=_abi.OPT_ADAM, beta1=0.979, beta2=0.963, eps=1e-8, sched=_abi.SCHED_PLATEAU, factor=0.547,
              patience=41, threshold=0.0673, cooldown=97)

N1_WARM = dict(optimizer=_abi.OPT_ADAM, lr=7.68962e-5, beta1=0.988452, beta2=0.987099, eps=3.57398e-9,
               sched=_abi.SCHED_PLATEAU, factor=0.70, patience=69, threshold=2.14818e-3, cooldown=51)
