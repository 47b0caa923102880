"""Seeded synthetic workloads for the QSGS generator.

Parameter sets only: no QSGS arithmetic lives here, so the CUDA binding,
the CPU oracle and the benchmark can all take their inputs from this one
module.  Every workload is a plain dict with the keys of ``qsgs_params``.

The paper's experiments need no dataset: a realization is defined entirely
by its parameters (Sec. 3.2, Sec. 3.3).  The Fontainebleau benchmark of
Sec. 3.3 enters only through its generation parameters.
"""
from __future__ import annotations

import numpy as np

# Directional reference probabilities used by all workloads below: face,
# edge and corner classes with G_face = 4 G_edge = 16 G_corner.
G_FACE, G_EDGE, G_CORNER = 0.01, 0.0025, 0.000625


def _base(n: int, cd: float, s: int, solid: float, seed: int) -> dict:
    return dict(nx=n, ny=n, nz=n, cd=cd, g_face=G_FACE, g_edge=G_EDGE, g_corner=G_CORNER,
                spacing_s=s, target_solid_fraction=solid, target_count=0, seed=seed,
                max_steps=0)


def small_64() -> dict:
    """64^3, cd = 0.002, no spacing, solid fraction 0.70, seed 1."""
    return _base(64, 0.002, 0, 0.70, 1)


def single_400() -> dict:
    """400^3 (64 M voxels), cd = 1e-4, spacing s = 30, solid fraction 0.80
    (porosity 0.20), seed 1 -- the timing size of Sec. 3.2."""
    return _base(400, 1e-4, 30, 0.80, 1)


# Size sweep in the setting of the paper's throughput figure (Sec. 3.2,
# Fig. 3): seed probability 2e-4, one reference probability 8e-4 for every
# direction class, porosity 0.20, diamond spacing s = 15 (Fig. 3a) or none
# (Fig. 3b), edges 200 .. 1000.
FIG3_EDGES = (200, 300, 400, 500, 600, 700, 800, 900, 1000)


def fig3_size(n: int, spacing: bool, seed: int = 1) -> dict:
    """One realization of the size sweep at n^3 (spacing s = 15 or 0)."""
    return dict(nx=n, ny=n, nz=n, cd=2e-4, g_face=8e-4, g_edge=8e-4, g_corner=8e-4,
                spacing_s=15 if spacing else 0, target_solid_fraction=0.80, target_count=0,
                seed=seed, max_steps=0)


# The Fontainebleau benchmark of Sec. 3.3: seed probability from the grain
# diameter, S_d = 6 phi_s Delta^3 / (pi d^3), with voxel size Delta = 4 um;
# a 500^3 domain, porosity 0.15, one reference probability 8e-4 for every
# class, spacing s = 0 .. 40 in steps of 5, five realizations per s.  The
# paper gives a grain diameter range of 200 .. 250 um, not one value; 225 um
# is taken here.
FONTAINEBLEAU_SPACINGS = tuple(range(0, 41, 5))
FONTAINEBLEAU_VOXEL_UM = 4.0


def fontainebleau_seed_probability(solid_fraction: float, grain_um: float,
                                   voxel_um: float = FONTAINEBLEAU_VOXEL_UM) -> float:
    """S_d = 6 phi_s Delta^3 / (pi d^3)."""
    return 6.0 * solid_fraction * voxel_um**3 / (np.pi * grain_um**3)


def fontainebleau(spacing: int, realization: int, n: int = 500, porosity: float = 0.15,
                  grain_um: float = 225.0) -> dict:
    """One realization of the Fontainebleau sweep (seed = 5 * (s / 5) + realization)."""
    solid = round(1.0 - porosity, 12)
    return dict(nx=n, ny=n, nz=n, cd=fontainebleau_seed_probability(solid, grain_um),
                g_face=8e-4, g_edge=8e-4, g_corner=8e-4, spacing_s=spacing,
                target_solid_fraction=solid, target_count=0,
                seed=5 * (spacing // 5) + realization, max_steps=0)


SWEEP_POROSITY = (0.08, 0.12, 0.16, 0.20, 0.25)
SWEEP_SPACING = (10, 20, 30, 40, 50)


def sweep_500() -> list[dict]:
    """Sandstone-like sweep at 500^3: porosity x spacing, cd = 1e-4, one
    realization per grid point, seed = 5 * i_porosity + i_spacing."""
    out = []
    for ip, por in enumerate(SWEEP_POROSITY):
        for js, s in enumerate(SWEEP_SPACING):
            out.append(_base(500, 1e-4, s, round(1.0 - por, 12), 5 * ip + js))
    return out


def batch_96(rng_seed: int = 2026) -> list[dict]:
    """96 uneven realizations: edge in {128,160,192,256}, porosity
    U[0.10,0.30], spacing U{10..40}, cd = 2e-4, seeds 0..95."""
    rng = np.random.default_rng(rng_seed)
    edges = rng.choice(np.array([128, 160, 192, 256]), size=96)
    por = rng.uniform(0.10, 0.30, size=96)
    sp = rng.integers(10, 41, size=96)
    return [_base(int(edges[i]), 2e-4, int(sp[i]), float(1.0 - por[i]), i) for i in range(96)]


SERVE_EDGES = (64, 128, 256, 400, 512)
SERVE_WEIGHTS = (0.30, 0.30, 0.20, 0.15, 0.05)


def serve_requests(n: int = 2000, rng_seed: int = 2027) -> list[dict]:
    """Request mix for the serving loop: edge from SERVE_EDGES with
    SERVE_WEIGHTS, porosity U[0.08,0.30], spacing U{0..40}, cd = 1e-4,
    seed = request id.  Arrival times are drawn separately
    (``poisson_arrivals``)."""
    rng = np.random.default_rng(rng_seed)
    edges = rng.choice(np.array(SERVE_EDGES), size=n, p=np.array(SERVE_WEIGHTS))
    por = rng.uniform(0.08, 0.30, size=n)
    sp = rng.integers(0, 41, size=n)
    return [_base(int(edges[i]), 1e-4, int(sp[i]), float(1.0 - por[i]), i) for i in range(n)]


def poisson_arrivals(n: int, rate_per_s: float, rng_seed: int = 2027) -> np.ndarray:
    """Arrival times (s) of a Poisson stream with the given rate."""
    rng = np.random.default_rng(rng_seed + 1)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))


def random_small(rng: np.random.Generator, max_edge: int = 20) -> dict:
    """A random small case for parity tests: ragged dims (not multiples of
    32), random probabilities and spacing, possibly degenerate."""
    nx, ny, nz = (int(v) for v in rng.integers(1, max_edge + 1, size=3))
    return dict(nx=nx, ny=ny, nz=nz, cd=float(rng.choice([0.0, 0.002, 0.01, 0.05, 0.3, 1.0])),
                g_face=float(rng.choice([0.0, 0.01, 0.2, 0.7, 1.0])),
                g_edge=float(rng.choice([0.0, 0.0025, 0.05, 0.5, 1.0])),
                g_corner=float(rng.choice([0.0, 0.000625, 0.0125, 0.3, 1.0])),
                spacing_s=int(rng.choice([0, 1, 2, 3, 5, 8])),
                target_solid_fraction=float(rng.uniform(0.0, 1.0)), target_count=0,
                seed=int(rng.integers(0, 2**63)), max_steps=int(rng.choice([0, 0, 0, 3, 20])))
