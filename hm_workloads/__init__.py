"""Seeded, synthetic scatterer workloads: triangle meshes and incidence-angle lists.

This package holds only input generation (surface meshes of spheres, plates,
ellipsoids and cylinders, and the plane-wave incidence sweeps).  It contains
none of the method's arithmetic (no basis functions, no Green's function, no
matrix, no solve); both the CPU oracle and the GPU library consume what it
produces.
"""
from .meshes import icosphere, plate, ellipsoid, closed_cylinder, mesh_stats
from .workloads import (WORKLOADS, Workload, monostatic_angles, get_workload,
                        scatterer_batch)

__all__ = ["icosphere", "plate", "ellipsoid", "closed_cylinder", "mesh_stats",
           "WORKLOADS", "Workload", "monostatic_angles", "get_workload",
           "scatterer_batch"]
