"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle's tests.

This package only makes inputs: tetrahedral meshes with tagged boundary faces, and the
closed-form flow fields that the test problems prescribe as data (initial histories and
Dirichlet values).  It holds none of the finite-element method's arithmetic (no element
integrals, no stabilisation, no solver); both the oracle and the CUDA library compute those
on their own.
"""
from .meshes import (Mesh, cube_kuhn, cylinder, stenosis, bifurcation, single_tet, batch,
                     mesh_stats, boundary_faces)
from .flows import beltrami_u, beltrami_p, beltrami_grad_u, poiseuille_u, poiseuille_p, zero_net_flux

__all__ = ["Mesh", "cube_kuhn", "cylinder", "stenosis", "bifurcation", "single_tet", "batch",
           "mesh_stats", "boundary_faces", "beltrami_u", "beltrami_p", "beltrami_grad_u",
           "poiseuille_u", "poiseuille_p", "zero_net_flux"]
