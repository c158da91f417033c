"""Seeded synthetic workloads: domains, meshes, potentials and initial data.

This module holds inputs only (no step of the method): the tests and the benchmark feed the
same arrays to the CUDA library and to the CPU oracle.  Sign conventions follow eq. (Sch):
    i u_t + lap * Lap u + V u + kappa |u|^2 u = 0,
so the GPE of eq. (GPE) / (GPE_Trans), i u_t + 1/2 Lap u - V_trap u - beta |u|^2 u = 0, is
lap = 1/2, V = -V_trap, kappa = -beta.

Workloads (sizes are cells; nodes are cells + 1 per direction):
* nls_small  -- plain cubic NLS on (-8,8)^2, 128 x 128 cells, 2 strips, Robin p = 2,
                dt = 0.01, 10 steps, u0 = exp(-(x^2+y^2)) exp(2ix), V = 0, focusing.
* nls_well   -- NLS with the Gaussian well V = 5 exp(-(x^2+y^2)/4), focusing, on
                (-32,32)^2, 1024 x 1024 cells, 16 strips, preconditioned, Robin p in
                {1, 2, 4}, dt = 0.005, 200 steps, same u0 (the initial datum is not stated
                for this case; the nls_small datum is used).
* gpe_trap   -- GPE, harmonic trap V_trap = (x^2+y^2)/2, beta = 500, on (-16,16)^2,
                2048 x 2048 cells, 32 strips, dt = 0.001, 500 steps, S_pade^8 transmission,
                preconditioned, rotation omega = 0.4 (isotropic trap: the rotating-frame
                potential does not change, omega enters the energy);
                u0 = pi^{-1/2} exp(-(x^2+y^2)/2) exp(i eps xi), eps = 1e-3, xi ~ U[-1,1]
                per node from numpy's PCG64 with seed 1603.
* gpe_batch  -- 64 independent GPE instances on (-16,16)^2, dt = 0.002, 100 steps, Robin
                p = sqrt(4/dt), classical: instance i draws (numpy PCG64, seed 1603 + i) the
                strip count N ~ U{4..16}, cells per strip c ~ U{ceil(256/N)..floor(1024/N)}
                (a square mesh of N*c cells), beta ~ U[100, 1000] and omega ~ U[0, 0.6]
                (omega leaves the rotating-frame solve unchanged for the isotropic trap and is
                carried as metadata only); u0 as gpe_trap with the instance's seed.
"""
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Workload:
    name: str
    xl: float
    xr: float
    yb: float
    yu: float
    nx: int
    ny: int
    n_strips: int
    dt: float
    steps: int
    lap: float = 1.0
    kappa: float = 1.0
    p: float = 2.0
    algorithm: str = "classical"
    potential: str = "zero"       # zero | well | trap
    datum: str = "gauss_kick"     # gauss_kick | ground_noise
    seed: int = 1603
    extra: dict = field(default_factory=dict)

    def grid(self):
        x = self.xl + (self.xr - self.xl) / self.nx * np.arange(self.nx + 1)
        y = self.yb + (self.yu - self.yb) / self.ny * np.arange(self.ny + 1)
        return np.meshgrid(x, y, indexing="xy")

    def V(self):
        X, Y = self.grid()
        if self.potential == "zero":
            return np.zeros_like(X)
        if self.potential == "well":
            return 5.0 * np.exp(-(X ** 2 + Y ** 2) / 4.0)
        if self.potential == "trap":
            return -0.5 * (X ** 2 + Y ** 2)          # V = -V_trap, eq. (Sch) sign
        raise ValueError(self.potential)

    def u0(self):
        X, Y = self.grid()
        if self.datum == "gauss_kick":
            return np.exp(-(X ** 2 + Y ** 2)) * np.exp(2j * X)
        if self.datum == "ground_noise":
            rng = np.random.default_rng(self.seed)
            xi = rng.uniform(-1.0, 1.0, size=X.shape)
            return np.pi ** -0.5 * np.exp(-(X ** 2 + Y ** 2) / 2.0) * np.exp(1e-3j * xi)
        raise ValueError(self.datum)

    def nodes(self):
        return (self.nx + 1) * (self.ny + 1)


NLS_SMALL = Workload("nls_small", -8.0, 8.0, -8.0, 8.0, 128, 128, 2, 0.01, 10, p=2.0)
NLS_WELL = Workload("nls_well", -32.0, 32.0, -32.0, 32.0, 1024, 1024, 16, 0.005, 200, p=2.0,
                    algorithm="preconditioned", potential="well")
GPE_TRAP = Workload("gpe_trap", -16.0, 16.0, -16.0, 16.0, 2048, 2048, 32, 0.001, 500, lap=0.5,
                    kappa=-500.0, p=2.0 * np.sqrt(1.0 / 0.001), algorithm="preconditioned", potential="trap",
                    datum="ground_noise", extra={"tc": "pade", "pade_m": 8, "omega": 0.4})

WORKLOADS = {w.name: w for w in (NLS_SMALL, NLS_WELL, GPE_TRAP)}


def scaled(w, nx, ny, n_strips=None, **kw):
    """The same physics on another mesh (for parity cases the oracle finishes quickly)."""
    d = dict(w.__dict__)
    d.update(nx=nx, ny=ny, n_strips=n_strips or w.n_strips, **kw)
    d.pop("extra", None)
    return Workload(**d)


def gpe_batch(n_instances=64, seed=1603, dt=0.002, steps=100, max_cells=1024, min_cells=256):
    """The batched GPE instances (see the module docstring)."""
    out = []
    for i in range(n_instances):
        rng = np.random.default_rng(seed + i)
        N = int(rng.integers(4, 17))
        c = int(rng.integers(-(-min_cells // N), max_cells // N + 1))
        beta = float(rng.uniform(100.0, 1000.0))
        omega = float(rng.uniform(0.0, 0.6))
        n = N * c
        out.append(Workload(f"gpe_batch_{i}", -16.0, 16.0, -16.0, 16.0, n, n, N, dt, steps, lap=0.5,
                            kappa=-beta, p=float(np.sqrt(4.0 / dt)), potential="trap", datum="ground_noise",
                            seed=seed + i, extra={"omega": omega, "beta": beta}))
    return out
