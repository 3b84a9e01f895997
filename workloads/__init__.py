"""Seeded synthetic workloads shared by the oracle, the tests and ``bench.py``.

This module only *describes* inputs: mesh sizes, subdomain cuts, material
constants, boundary-condition masks, load schedules, tolerances and the seeded
random draws of the irregular-partition workload.  It holds none of the
method's arithmetic (no strains, stresses, stiffness, loads or solves), so that
both the CUDA path and the CPU oracle can take their inputs from here without
sharing any of the computation.

Material (Sec. 5, numerical experiments): E = 206 900, nu = 0.29,
sigma_y = 450, H_m = 10 000.  The paper's benchmark geometry (a plate with a
hole meshed by Ansys and partitioned by Metis) is not available, so seeded
unit-cube hex meshes with box subdomains stand in for it.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
import random

# Sec. 5: material parameters of the benchmark body.
MATERIAL = {"young": 206900.0, "poisson": 0.29, "sigma_y": 450.0, "hardening": 10000.0}

# Face names and their (axis, side) pairs; side 0 = low end, 1 = high end.
FACES = ("x0", "x1", "y0", "y1", "z0", "z1")


def equal_cuts(n_elements: int, n_parts: int) -> tuple:
    """Cut positions splitting ``n_elements`` into ``n_parts`` equal boxes."""
    if n_elements % n_parts:
        raise ValueError("equal split needs n_elements divisible by n_parts")
    a = n_elements // n_parts
    return tuple(a * i for i in range(n_parts + 1))


def irregular_cuts(n_elements: int, rng: random.Random, lo: int = 4, hi: int = 12) -> tuple:
    """Seeded irregular 1-D partition with segment lengths in [lo, hi].

    While more than ``hi`` elements remain, draw a length uniformly from
    {lo .. min(hi, rem - lo)}; the last segment takes the remainder, which
    then lies in [lo, hi].
    """
    cuts = [0]
    rem = n_elements
    while rem > hi:
        length = rng.randint(lo, min(hi, rem - lo))
        cuts.append(cuts[-1] + length)
        rem -= length
    cuts.append(n_elements)
    return tuple(cuts)


@dataclass(frozen=True)
class Workload:
    """One synthetic problem: a box of hex8 elements cut into box subdomains."""

    name: str
    nel: tuple                       # elements per axis (nx, ny, nz)
    cuts: tuple                      # per axis, the subdomain cut positions
    length: tuple = (1.0, 1.0, 1.0)  # box edge lengths
    material: dict = field(default_factory=lambda: dict(MATERIAL))
    # Dirichlet mask per face: bit c set = displacement component c fixed.
    dirichlet: dict = field(default_factory=lambda: {"z0": 7})
    traction_face: str = "z1"
    traction_dir: tuple = (1.0, 0.0, 0.0)
    n_steps: int = 10
    load_factor: float = 1.5         # final load = load_factor x first-yield load
    newton_tol: float = 1e-10
    pcg_rtol: float = 1e-12
    newton_maxit: int = 30
    pcg_maxit: int = 2000
    cyclic: bool = False             # load, unload, reverse, unload in four equal phases

    @property
    def n_sub(self) -> int:
        return (len(self.cuts[0]) - 1) * (len(self.cuts[1]) - 1) * (len(self.cuts[2]) - 1)

    def dirichlet_masks(self) -> tuple:
        """Six masks in FACES order."""
        return tuple(int(self.dirichlet.get(f, 0)) for f in FACES)

    def load_fractions(self, n_steps: int | None = None) -> list:
        """Load level after step k (1-based), as a multiple of the first-yield load.

        Linear ramp: load_factor * k / n_steps.  Cyclic: with t = 4 k / n_steps the
        level is load_factor * (t, 2 - t, 2 - t, t - 4) on the phases t in
        (0,1], (1,2], (2,3], (3,4]: 0 -> +F -> 0 -> -F -> 0, piecewise linear.
        """
        n = self.n_steps if n_steps is None else n_steps
        if not self.cyclic:
            return [self.load_factor * k / self.n_steps for k in range(1, n + 1)]
        out = []
        for k in range(1, n + 1):
            t = 4.0 * k / self.n_steps
            level = t if t <= 1.0 else (2.0 - t if t <= 3.0 else t - 4.0)
            out.append(self.load_factor * level)
        return out

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


def cube(name: str, n: int, parts: int, **kw) -> Workload:
    c = equal_cuts(n, parts)
    return Workload(name=name, nel=(n, n, n), cuts=(c, c, c), **kw)


# Tolerances: in the decomposed Newton of Algorithm 4 the Newton criterion
# cannot fall below roughly 0.03..0.4 x the dual PCG tolerance (the dual
# right-hand side always carries the O(1) interface forces), so a Newton
# tolerance is paired with a PCG tolerance at least ~100x tighter:
# (1e-10, 1e-12) for parity runs, (1e-6, 1e-8) for timed runs.
# 12^3 hex8, 2x2x2 subdomains of 6^3, 10 steps to 1.5x first yield.
CUBE12 = cube("cube12_2x2x2", 12, 2, n_steps=10, newton_tol=1e-10, pcg_rtol=1e-12)
# 64^3 hex8, 8x8x8 subdomains of 8^3, 20 steps to 1.5x first yield, timed at 1e-8 dual residual.
CUBE64 = cube("cube64_8x8x8", 64, 8, n_steps=20, newton_tol=1e-6, pcg_rtol=1e-8)
# 48^3 hex8, 6^3 subdomains of 8^3 (a smaller case of the same box size, for profiler captures).
CUBE48 = cube("cube48_6x6x6", 48, 6, n_steps=20, newton_tol=1e-6, pcg_rtol=1e-8)
# 96^3 hex8, 12^3 subdomains of 8^3.
CUBE96 = cube("cube96_12x12x12", 96, 12, n_steps=20, newton_tol=1e-6, pcg_rtol=1e-8)
# 128^3 hex8, 16^3 subdomains of 8^3, cyclic load (40 steps: load, unload, reverse, unload).
CUBE128 = cube("cube128_16x16x16", 128, 16, n_steps=40, newton_tol=1e-6, pcg_rtol=1e-8, cyclic=True)
# 12^3 with the cyclic schedule (parity case of the cyclic load).
CUBE12_CYCLIC = cube("cube12_cyclic", 12, 2, n_steps=8, newton_tol=1e-10, pcg_rtol=1e-12, cyclic=True)

# Small cases for pins and parity tests.
TINY_1x1x2 = Workload(name="tiny2_1x1x2", nel=(2, 2, 2), cuts=((0, 2), (0, 2), (0, 1, 2)), n_steps=4)
SMALL4 = cube("small4_2x2x2", 4, 2, n_steps=4)
SMALL6_RAGGED = Workload(name="small_ragged", nel=(5, 4, 6), cuts=((0, 2, 5), (0, 4), (0, 3, 4, 6)),
                         length=(1.0, 0.8, 1.2), n_steps=4)

WORKLOADS = {w.name: w for w in (CUBE12, CUBE48, CUBE64, CUBE96, CUBE128, CUBE12_CYCLIC, TINY_1x1x2, SMALL4,
                                  SMALL6_RAGGED)}


def irregular_cube80(seed: int = 0, n: int = 80) -> Workload:
    """80^3 cube with a seeded tensor-product partition into boxes of 4..12 elements."""
    rng = random.Random(seed)
    cuts = tuple(irregular_cuts(n, rng) for _ in range(3))
    return Workload(name=f"cube80_irregular_s{seed}", nel=(n, n, n), cuts=cuts, n_steps=20)


def irregular_cube(n: int, seed: int, n_steps: int = 20, **kw) -> Workload:
    """n^3 cube with a seeded tensor-product partition into boxes of 4..12 elements per edge."""
    rng = random.Random(seed)
    cuts = tuple(irregular_cuts(n, rng) for _ in range(3))
    return Workload(name=f"cube{n}_irregular_s{seed}", nel=(n, n, n), cuts=cuts, n_steps=n_steps, **kw)


def irregular_cases(seed: int = 0, n_cases: int = 16) -> list:
    """Seeded material/load cases: sigma_y ~ U[300,600], H ~ U[1e3,2e4], traction angle ~ U[0, 2pi)."""
    import math
    rng = random.Random(seed + 1000003)
    cases = []
    for _ in range(n_cases):
        sy = rng.uniform(300.0, 600.0)
        hm = rng.uniform(1e3, 2e4)
        th = rng.uniform(0.0, 2.0 * math.pi)
        cases.append({"sigma_y": sy, "hardening": hm, "traction_dir": (math.cos(th), math.sin(th), 0.0)})
    return cases


def direction_cases(n_cases: int = 4) -> list:
    """Load cases of one material whose x-y traction directions split the circle evenly:
    theta_k = 2 pi k / n_cases (four cases: the x, y, -x and -y directions)."""
    import math
    cases = []
    for k in range(n_cases):
        th = 2.0 * math.pi * k / n_cases
        cases.append({"sigma_y": MATERIAL["sigma_y"], "hardening": MATERIAL["hardening"],
                      "traction_dir": (math.cos(th), math.sin(th), 0.0)})
    return cases


def case_workload(w: Workload, case: dict) -> Workload:
    """The workload ``w`` with one case's yield stress, hardening and traction direction."""
    mat = dict(w.material)
    mat["sigma_y"] = case["sigma_y"]
    mat["hardening"] = case["hardening"]
    return w.with_(material=mat, traction_dir=tuple(case["traction_dir"]),
                   name=f"{w.name}_sy{case['sigma_y']:.1f}_h{case['hardening']:.0f}")


def seeded_vector(n: int, seed: int, dtype="float64"):
    """Deterministic standard-normal vector (numpy) for operator parity tests."""
    import numpy as np
    return np.random.default_rng(seed).standard_normal(n).astype(dtype)


def seeded_gauss_point_inputs(n: int, seed: int, scale_strain: float = 1e-3, scale_stress: float = 100.0):
    """Seeded (sigma_k, kappa_k, eta) triples for material-point parity tests.

    sigma_k ~ N(0, scale_stress) per component, kappa_k ~ U[0, 1e-3],
    eta ~ N(0, scale_strain) per component.  A spread that puts points on both
    sides of the yield surface for the Sec. 5 material.
    """
    import numpy as np
    rng = np.random.default_rng(seed)
    sig = rng.standard_normal((n, 6)) * scale_stress
    kap = rng.uniform(0.0, 1e-3, size=n)
    eta = rng.standard_normal((n, 6)) * scale_strain
    return sig, kap, eta


# Batching geometry (config 4): 80^3 in a seeded irregular partition (seed 0: 9 x 10 x 9 = 810 boxes of
# 252 distinct shapes), timed like the 64^3 case; and a 24^3 irregular parity case.
CUBE80_IRREGULAR = irregular_cube(80, 0, newton_tol=1e-6, pcg_rtol=1e-8)
CUBE24_IRREGULAR = irregular_cube(24, 3, n_steps=4)
WORKLOADS[CUBE80_IRREGULAR.name] = CUBE80_IRREGULAR
WORKLOADS[CUBE24_IRREGULAR.name] = CUBE24_IRREGULAR


def box_dof_offsets(w: Workload) -> list:
    """Start of each box's block in the decomposed dof vector (boxes in x-fastest order, three dofs per
    node of a box of (ax+1)(ay+1)(az+1) nodes), plus the total as the last entry."""
    sx, sy, sz = (len(c) - 1 for c in w.cuts)
    off = [0]
    for k in range(sz):
        for j in range(sy):
            for i in range(sx):
                ax = w.cuts[0][i + 1] - w.cuts[0][i]
                ay = w.cuts[1][j + 1] - w.cuts[1][j]
                az = w.cuts[2][k + 1] - w.cuts[2][k]
                off.append(off[-1] + 3 * (ax + 1) * (ay + 1) * (az + 1))
    return off


def seeded_partly_plastic_increment(w: Workload, seed: int, n_hot: int, hot_scale: float = 1.2e-3,
                                    cold_scale: float = 1e-5):
    """Seeded displacement increment whose strains exceed first yield only in a few boxes.

    Every decomposed dof draws N(0, (s h)^2) with h the smallest element edge: s = hot_scale in
    ``n_hot`` boxes picked by the seed (strains of about 1e-3: from a zero state about half of their
    Gauss points lie beyond first yield with the Sec. 5 material) and s = cold_scale elsewhere (far
    below yield).  Returns the vector and the sorted list of hot boxes.
    """
    import numpy as np
    off = box_dof_offsets(w)
    n_sub = len(off) - 1
    rng = np.random.default_rng(seed)
    hot = np.sort(rng.choice(n_sub, size=min(n_hot, n_sub), replace=False))
    h = min(l / n for l, n in zip(w.length, w.nel))
    du = rng.standard_normal(off[-1]) * (cold_scale * h)
    for p in hot:
        du[off[p]:off[p + 1]] *= hot_scale / cold_scale
    return du, [int(p) for p in hot]


def seeded_indices(n: int, k: int, seed: int):
    """k distinct indices in [0, n), sorted, drawn by the seed (sampled outputs of full-size checks)."""
    import numpy as np
    return np.sort(np.random.default_rng(seed).choice(n, size=min(k, n), replace=False))
