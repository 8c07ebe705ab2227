"""Adam update (Kingma & Ba, 2015), textbook form with bias correction.

Test infrastructure only (see ``oracle/__init__``).

App. B.3 (Table "Hyperparameters") gives the learning rates, policy 6e-4 and
critic 3e-4, but not the optimiser.  Reading: Adam with beta1 = 0.9,
beta2 = 0.999, eps = 1e-8, bias-corrected, no weight decay (App. E reports
weight decay as a failed experiment).
"""

import numpy as np


def adam_update(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step at step number t (1-based); returns new (p, m, v)."""
    p = np.asarray(p, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** t)
    v_hat = v / (1.0 - beta2 ** t)
    return p - lr * m_hat / (np.sqrt(v_hat) + eps), m, v
