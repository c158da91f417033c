"""Shared test helpers: the same seeded inputs go to the CUDA library and to the oracle."""
import os

import numpy as np

from oracle import nls


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def oracle_problem(w, V=None, tc="robin", bc="same", m=4):
    return nls.Problem(xl=w.xl, xr=w.xr, yb=w.yb, yu=w.yu, nx=w.nx, ny=w.ny, dt=w.dt,
                       V=w.V() if V is None else V, kappa=w.kappa, lap=w.lap, tc=tc, p=w.p, m=m, bc=bc)


def gpu_params(w, **kw):
    d = dict(xl=w.xl, xr=w.xr, yb=w.yb, yu=w.yu, nx=w.nx, ny=w.ny, n_strips=w.n_strips, dt=w.dt,
             lap=w.lap, kappa=w.kappa, p=w.p, nl_tol=1e-14, max_schwarz=5000)
    d.update(kw)
    return d


def printed_p_table():
    """Sec. 5.1, Table Influence_p_NL_2_32 as printed (tests/golden): p and, per strip count N,
    the classical ("cls") and preconditioned ("pd") counts from the zero interface vector."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table_influence_p_nl_2_32.txt")
    with open(path) as f:
        rows = [[int(v) for v in line.split()] for line in f if line.strip() and not line.startswith("#")]
    return {"p": [r[0] for r in rows],
            "cls": {2: [r[1] for r in rows], 32: [r[5] for r in rows]},
            "pd": {2: [r[2] for r in rows], 32: [r[6] for r in rows]}}
