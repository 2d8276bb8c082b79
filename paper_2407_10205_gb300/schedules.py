"""Schedule heuristic for PHIA runs (host-side convenience, not from the paper).

The paper gives no values for beta, eps or gamma.  The potential jump a spin meets when
its position crosses zero is beta times its local field (Eqs. 4-6), so the useful beta
range scales inversely with the typical field magnitude.  `suggest_schedule` takes that
magnitude as q * rms(k) * sqrt(mean degree) and ends the linear beta schedule where the
typical jump is `jump` (units of the kinetic energy of a unit momentum), starting 20
times lower.  By default the final jump grows with the size, 6 max(1, sqrt(n / 128)):
measured on SK, spin-model and 3-regular max-cut instances of n = 512 and 1024 (the
time-to-solution study), a final jump of 12 reached the best known energies on more
instances than 6 or 3 at these sizes, while 6 suffices up to n = 128.  eps = 0.1,
gamma = 2 and a momentum refresh every 50 iterations are the values the workloads of
this repository use.  These are this project's own choices, not the paper's.
"""
from __future__ import annotations

import math

import numpy as np


def field_scale(inst) -> float:
    """q * rms(k) * sqrt(mean number of couplings per spin)."""
    q = math.ldexp(1.0, -int(getattr(inst, "frac_bits", 0)))
    n = int(np.asarray(inst.kh).shape[0])
    if getattr(inst, "k", None) is not None:
        k = np.asarray(inst.k, dtype=np.float64)
        nz = np.count_nonzero(k)
        rms = math.sqrt(float((k * k).sum()) / max(nz, 1))
        deg = nz / max(n, 1)
    else:
        v = np.asarray(inst.val, dtype=np.float64)
        rms = math.sqrt(float((v * v).mean())) if v.size else 0.0
        deg = v.size / max(n, 1)
    return max(q * rms * math.sqrt(max(deg, 1.0)), 1e-6)


def default_jump(n: int) -> float:
    """Final potential jump of the schedule for n spins: 6 max(1, sqrt(n / 128))."""
    return 6.0 * max(1.0, math.sqrt(n / 128.0))


def suggest_schedule(inst, jump: float | None = None):
    """(beta0, beta1, eps, gamma, refresh) for an instance (jump: the final jump, default
    default_jump(n))."""
    n = int(np.asarray(inst.kh).shape[0])
    beta1 = (default_jump(n) if jump is None else jump) / field_scale(inst)
    return beta1 / 20.0, beta1, 0.1, 2.0, 50
