"""The synthetic workloads: a scatterer mesh, a frequency, tree/ACA knobs and a
plane-wave incidence sweep.  Shapes follow the paper's test cases (closed
sphere, open square plate, lambda/10-ish meshes, monostatic sweeps), Sec. V.

Angles are returned in radians as three arrays ``theta, phi, pol`` where
``pol`` is 0 for a theta-hat polarised and 1 for a phi-hat polarised incident
field.  At theta = phi = 0 the theta-hat polarisation is x-hat.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .meshes import icosphere, plate, ellipsoid, closed_cylinder


@dataclass(frozen=True)
class Workload:
    name: str
    mesh: tuple                      # ("icosphere", level, radius) | ("plate", side, ncell)
    wavelength: float = 1.0          # metres
    leaf_max: int = 64
    aca_tol: float = 1e-4
    sweep: tuple = ("single",)       # see monostatic_angles
    precision: str = "fp64"
    notes: str = ""

    def build_mesh(self):
        kind = self.mesh[0]
        if kind == "icosphere":
            return icosphere(self.mesh[1], self.mesh[2])
        if kind == "plate":
            return plate(self.mesh[1], self.mesh[2])
        if kind == "ellipsoid":
            return ellipsoid(self.mesh[1], self.mesh[2])
        if kind == "cylinder":
            return closed_cylinder(*self.mesh[1:])
        raise ValueError(kind)

    def angles(self):
        return monostatic_angles(*self.sweep)


def monostatic_angles(kind, *args):
    """Incidence sweeps.

    ("single", theta_deg, phi_deg, pol)          one RHS
    ("theta", start, stop, step, phi, pols)      theta sweep, phi fixed, each pol
    ("phi", start, stop, step, theta, pols)      phi sweep, theta fixed, each pol
    """
    if kind == "single":
        th, ph, pol = (args + (0.0, 0.0, 0))[:3] if args else (0.0, 0.0, 0)
        return (np.array([math.radians(th)]), np.array([math.radians(ph)]),
                np.array([pol], dtype=np.int32))
    start, stop, step, fixed, pols = args
    n = int(round((stop - start) / step)) + 1
    sweep = start + step * np.arange(n, dtype=np.float64)
    th, ph, po = [], [], []
    for p in pols:
        for s in sweep:
            if kind == "theta":
                th.append(s); ph.append(fixed)
            else:
                th.append(fixed); ph.append(s)
            po.append(p)
    return (np.radians(np.array(th)), np.radians(np.array(ph)),
            np.array(po, dtype=np.int32))


WORKLOADS = {
    # 0.5 lambda PEC sphere, 1920 RWG unknowns, one x-polarised RHS from theta=0
    "sphere_r0.5_L3": Workload("sphere_r0.5_L3", ("icosphere", 3, 0.5),
                               leaf_max=64, sweep=("single", 0.0, 0.0, 0)),
    # 2 lambda sphere, 30720 unknowns, 181 theta angles x {theta, phi} pol = 362 RHS
    "sphere_r2_L5": Workload("sphere_r2_L5", ("icosphere", 5, 2.0), leaf_max=128,
                             sweep=("theta", 0.0, 180.0, 1.0, 0.0, (0, 1))),
    "sphere_r2_L5_1rhs": Workload("sphere_r2_L5_1rhs", ("icosphere", 5, 2.0),
                                  leaf_max=128, sweep=("single", 0.0, 0.0, 0)),
    # 8 lambda x 8 lambda plate, lambda/10 cells, 12800 triangles, 19040 unknowns,
    # 360 RHS phi = 0..359 deg at theta = 60 deg
    "plate_8l": Workload("plate_8l", ("plate", 8.0, 80), leaf_max=128,
                         sweep=("phi", 0.0, 359.0, 1.0, 60.0, (0,)),
                         precision="mixed"),
    # small cases for parity tests (oracle finishes in seconds)
    "sphere_r0.25_L2": Workload("sphere_r0.25_L2", ("icosphere", 2, 0.25),
                                leaf_max=32, sweep=("theta", 0.0, 180.0, 30.0, 0.0, (0, 1))),
    "plate_2l": Workload("plate_2l", ("plate", 2.0, 20), leaf_max=32,
                         sweep=("phi", 0.0, 330.0, 30.0, 60.0, (0,))),
    # 10 lambda sphere, 491520 unknowns, 720 RHS
    "sphere_r10_L7": Workload("sphere_r10_L7", ("icosphere", 7, 10.0), leaf_max=256,
                              sweep=("theta", 0.0, 179.75, 0.25, 0.0, (0,)),
                              precision="mixed"),
}


def get_workload(name: str) -> Workload:
    """A named workload, or member s of the seeded scatterer batch as
    ``scatterer_<s>``."""
    if name.startswith("scatterer_") and name[10:].isdigit():
        s = int(name[10:])
        return scatterer_batch(s + 1)[s]
    return WORKLOADS[name]


def scatterer_batch(count: int = 64, wavelength: float = 1.0):
    """Seeded batch of closed scatterers for grouped solves: seed s uses
    numpy.random.default_rng(s); type s % 3 is sphere / prolate ellipsoid /
    closed cylinder; the size targets a log-uniform unknown count in
    [2000, 40000] at a lambda/10 mean edge; the leaf cap is drawn from
    {32, 64, 128, 256}; 91 theta-polarised RHS theta = 0..180 step 2 deg."""
    out = []
    h = wavelength / 10.0
    for s in range(count):
        rng = np.random.default_rng(s)
        target = math.exp(rng.uniform(math.log(2000), math.log(40000)))
        leaf = int(rng.choice([32, 64, 128, 256]))
        kind = s % 3
        if kind == 0 or kind == 1:
            # icosphere level whose unknown count 30 * 4^level is nearest the
            # target in log scale (1920, 7680 or 30720), then radius for edge h
            level = min(5, max(3, int(round(math.log(target / 30.0, 4)))))
            ntri = 20 * 4 ** level
            area = ntri * (math.sqrt(3) / 4) * h * h
            if kind == 0:
                r = math.sqrt(area / (4 * math.pi))
                mesh = ("icosphere", level, r)
            else:
                ratio = rng.uniform(1.0, 4.0)
                # area of a prolate spheroid ~ 4 pi a^2 (1 + 2 ratio)/3 (rough)
                a = math.sqrt(area / (4 * math.pi * (1 + 2 * ratio) / 3))
                mesh = ("ellipsoid", level, (a, a, a * ratio))
        else:
            # side + caps area 2 pi r (r + height); height = 2 r
            ntri = target / 1.5
            area = ntri * (math.sqrt(3) / 4) * h * h
            r = math.sqrt(area / (6 * math.pi))
            mesh = ("cylinder", r, 2 * r, h)
        out.append(Workload(f"scatterer_{s}", mesh, wavelength=wavelength,
                            leaf_max=leaf,
                            sweep=("theta", 0.0, 180.0, 2.0, 0.0, (0,)),
                            precision="mixed"))
    return out
