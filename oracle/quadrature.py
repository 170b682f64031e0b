"""Expected one-step straight-through gradient for two reactions.  Test infrastructure.

With two reactions, the soft sample of Eq. 3 is y~_1 = sigma((log a_1 - log a_2 + L)/T) with
L = G_1 - G_2, and the difference of two independent standard Gumbel variables is standard
logistic: density f(L) = sigma(L) sigma(-L). The straight-through derivative of y~_1 with respect
to log a_1 is y~_1 y~_2 / T, so its expectation over the noise is a one-dimensional integral.
As T -> 0 that expectation tends to f(-d) = pi_1 pi_2 with d = log(a_1/a_2), which is the exact
derivative d pi_1 / d log a_1 of the categorical probability pi_1 = a_1/(a_1 + a_2).
"""
from __future__ import annotations

import numpy as np
from scipy import integrate
from scipy.special import expit


def expected_st_derivative(log_ratio: float, T: float) -> float:
    """E_L[ y~_1 (1 - y~_1) / T ] with y~_1 = sigma((log_ratio + L)/T), L ~ Logistic(0, 1)."""
    def f(L):
        s = expit((log_ratio + L) / T)
        pdf = expit(L) * expit(-L)
        return s * (1.0 - s) / T * pdf

    # the integrand is concentrated near L = -log_ratio with width ~T; split there
    c = -log_ratio
    w = max(T, 1e-3) * 60.0
    parts = [(-np.inf, c - w), (c - w, c + w), (c + w, np.inf)]
    return float(sum(integrate.quad(f, lo, hi, limit=400, epsabs=1e-13, epsrel=1e-11)[0]
                     for lo, hi in parts))


def exact_choice_derivative(log_ratio: float) -> float:
    """d pi_1 / d log a_1 = pi_1 pi_2 for pi_1 = sigma(log_ratio)."""
    p = expit(log_ratio)
    return float(p * (1.0 - p))
