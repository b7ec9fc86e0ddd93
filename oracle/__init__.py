"""CPU oracle for the SHG integral library.

TEST INFRASTRUCTURE ONLY: the product package never imports this module.  Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it.  It shares no code with the CUDA path.

The numerical work is in ``shg_oracle.c`` (plain FP64 C, OpenMP over pairs):
a Cartesian two-center recursion seeded with the s-type integrals of Table S1,
explicit real-solid-harmonic coefficients, contraction and unit-self-overlap
normalisation; (a|r_a^{2n}|b) from the multinomial expansion of r_A^{2n} and
closed-form 1-D Gaussian overlaps.  This module compiles it with gcc and wraps it with ctypes.

Parity pins: every function here is checked in ``tests/test_oracle_*.py``
against closed forms, exact quadrature, symmetry relations and brute force.
"""
from .oracle import (  # noqa: F401
    OP_OVERLAP, OP_COULOMB, OP_ERFC, OP_ERF, OP_GAUSS, OP_GCOUL,
    build, lib_path, boys, ss_deriv, sph_coef, cart_2c, shell_norms,
    eval_2c, eval_2c_grad, eval_2c_ra2n, eval_2c_ra2n_grad, eval_3c_aab, eval_3c_aab_grad, ncart,
)
