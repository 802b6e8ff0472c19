"""Seeded synthetic inputs shared by the oracle tests, the CUDA-path tests and the benchmark.

This package only *generates inputs*: surface meshes of the test bodies (quadratic 6-node
triangles with their analytic node normals), observation points, wavenumber grids and
sampled incident pulses.  It holds none of the boundary-integral method's arithmetic
(no quadrature, no Green's function, no assembly, no transform), so the oracle and the
GPU library can both consume its arrays without sharing any of the method's code.
"""
from .meshes import (Mesh, octa_sphere, ico_sphere, scale_translate, merge_meshes,
                     ellipsoid_from_sphere, revolution_mesh, bowl_profile, bowl_mesh, linear_from_quadratic,
                     uv_sphere_linear)
from .pulses import gaussian_pulse, ricker_pulse, modulated_gaussian, paper_sine_pulse
from .configs import (config_sphere_fp64, config_two_spheres_mixed, config_spheroid_learned, config_uneven_batch, config_lattice_large,
                      config_paper_sphere, config_paper_two_spheres, config_paper_bowl, bowl_inside,
                      uneven_configuration, shell_points,
                      spheroid_shell_points, plane_grid_points, Workload)

__all__ = [
    "Mesh", "octa_sphere", "ico_sphere", "scale_translate", "merge_meshes",
    "ellipsoid_from_sphere", "gaussian_pulse", "ricker_pulse", "modulated_gaussian",
    "paper_sine_pulse", "config_sphere_fp64", "config_two_spheres_mixed", "config_spheroid_learned",
    "config_uneven_batch", "uneven_configuration", "config_lattice_large", "config_paper_sphere",
    "config_paper_two_spheres", "config_paper_bowl", "bowl_inside", "revolution_mesh", "bowl_profile", "bowl_mesh",
    "linear_from_quadratic", "uv_sphere_linear",
    "shell_points", "spheroid_shell_points",
    "plane_grid_points", "Workload",
]
