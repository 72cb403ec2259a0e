"""Closed-form characteristic flows used as pins (independent of the oracle)."""

import math

import numpy as np

TWO_PI = 2.0 * math.pi


def exact_flow_cos_t_cos_x(x, t_from, t_to):
    """Exact characteristic of d xi/dt = cos(2 pi t) cos(2 pi xi) from (x, t_from) to time t_to.

    artanh(sin(2 pi xi)) - sin(2 pi t) is constant along the flow; each cell between
    the stagnation points x = -1/4 + k/2 is invariant.
    """
    x = np.asarray(x, dtype=np.float64)
    k = np.floor(x + 0.25)  # period 1: reduce to [-1/4, 3/4)
    xr = x - k
    v = _artanh_sin(xr) + math.sin(TWO_PI * t_to) - math.sin(TWO_PI * t_from)
    a = np.arcsin(np.tanh(v))
    left = xr < 0.25
    xi = np.where(left, a / TWO_PI, (math.pi - a) / TWO_PI)
    return xi + k



def _artanh_sin(xr):
    with np.errstate(divide="ignore"):
        return np.arctanh(np.clip(np.sin(TWO_PI * xr), -1.0, 1.0))
