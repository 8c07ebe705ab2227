"""Plain FP64 CPU oracle for the contrastive-RL (CRL) update step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (the CUDA library and its Python binding) never
imports, links or executes anything here, and this package never imports the
product package: the two share no code.  Inputs come from the seeded
generators in ``paper_2408_11052_gb300.workload`` (which hold none of the
method's arithmetic), and are handed to both sides by the tests.

Every function follows the paper (arXiv 2408.11052, "JaxGCRL"), cited by
section / equation / algorithm.  Where the paper is silent or ambiguous the
reading taken is stated at the function.  Pins for each function live in
``tests/test_oracle_*.py`` (run with ``-m "not gpu"``).

Modules
-------
philox   Philox4x64-10 counter-based generator (Salmon et al., SC'11).
relabel  replay buffer model + hindsight future-goal relabelling (§3.1, §3.2,
         Algorithm 1, the Geom(1-gamma) offset of §3).
mlp      encoder / actor MLPs with optional LayerNorm (§4.3, §5.4) and their
         hand-derived backward.
critic   energy functions and InfoNCE objectives with the logsumexp penalty
         (§3.1, App. A.2, Algorithm 1) and their hand-derived gradient.
actor    tanh-Gaussian DDPG-style actor objective (Eq. 3, §5.1).
adam     Adam update (optimiser of the learning rates in App. B.3).
step     one full CRL update step (Algorithm 1, inner loop body).
"""

from . import philox, relabel, mlp, critic, actor, adam, step, collect  # noqa: F401
