"""Adam, the optimiser of the inverse problem (Sec. 4.2: the latent code is
optimised through the renderer; Sec. B.4: Adam with learning rate 1e-2 and
z initialised to 0), in float64.

Adam as published (Kingma & Ba, ICLR 2015, Algorithm 1): exponential moving
averages of the gradient and of its square, bias-corrected by 1 - beta^t,
and the step lr * m_hat / (sqrt(v_hat) + eps).  TEST INFRASTRUCTURE ONLY
(see the package header).
"""

from __future__ import annotations

import numpy as np


def adam_step(z, g, m, v, t, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8):
    """One step (t counts from 1).  Returns new (z, m, v); inputs untouched."""
    z, g, m, v = (np.asarray(a, dtype=np.float64) for a in (z, g, m, v))
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** t)
    v_hat = v / (1.0 - beta2 ** t)
    return z - lr * m_hat / (np.sqrt(v_hat) + eps), m, v
