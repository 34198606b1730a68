"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds no arithmetic of the DMRG method: it only draws random numbers
and writes integrals in the layout the library's C ABI takes (h as L*L row-major,
V as L^4 in physics notation V[i,j,k,l] = (ij|V|kl)).
"""
from .synthetic import *  # noqa: F401,F403
