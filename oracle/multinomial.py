"""The paper's multinomial evaluation of the sub-stepped Taylor product (tiny problems).

TEST INFRASTRUCTURE ONLY (part of the oracle; see oracle/__init__.py).

Sec. 2.2 writes exp(tau B) v_1 ~ (P_0 + P_1 + ... + P_m)^s v_1 with
P_j = (tau B / s)^j / j! and expands the product with the multinomial theorem:
a sum over all (k_0, ..., k_m) with k_0 + ... + k_m = s of
s! / (k_0! ... k_m!) * prod_t P_t^{k_t} v_1.  Because every P_t is a power of
the same matrix X = tau B / s, each product equals X^d v_1 / prod_t (t!)^{k_t}
with d = sum_t t k_t, so the method precomputes the powers X^d v_1 and adds
them with the collected coefficients.  This module does exactly that, by
enumerating the compositions in pure Python, so it is only for small s and m.
"""
from __future__ import annotations

import math

import numpy as np


def compositions(total: int, parts: int):
    """All tuples of `parts` non-negative integers summing to `total`."""
    if parts == 1:
        yield (total,)
        return
    for first in range(total + 1):
        for rest in compositions(total - first, parts - 1):
            yield (first,) + rest


def power_coefficients(s: int, m: int) -> np.ndarray:
    """c[d] = sum over compositions with sum_t t k_t = d of s!/prod k_t! / prod (t!)^k_t."""
    c = np.zeros(s * m + 1)
    for k in compositions(s, m + 1):
        coef = math.factorial(s)
        denom = 1
        d = 0
        for t, kt in enumerate(k):
            denom *= math.factorial(kt) * math.factorial(t) ** kt
            d += t * kt
        c[d] += coef / denom
    return c


def phi1_action(problem, un, b, tau: float, s: int, m: int) -> np.ndarray:
    """tau phi1(tau A) b as the top block of sum_d c_d X^d v_1 (augmented B, J inert).

    X [x; a] = (tau / s) [A x + b a; 0]: the augmented component a starts at 1
    and is zero in every power d >= 1 (the J block of B acts on a zero entry).
    """
    shape = np.shape(b)
    c = power_coefficients(s, m)
    h = tau / s
    x = np.zeros(shape)
    a = 1.0
    out = c[0] * x
    for d in range(1, s * m + 1):
        x = h * (problem.apply_A(un, x) + b * a)
        a = 0.0
        out = out + c[d] * x
    return out
