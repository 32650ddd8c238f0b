"""Tolerances of the split-precision (BF16 slice) path, shared by the tests.

The method's targets are absolute: 1e-9 on Omega (and on the Jacobian's rho,
whose trial vectors are normalised) and 1e-8 Eh on the triples energy.  On
outputs of small magnitude an absolute bound alone would admit relative errors
of 1e-6, enough to hide a lost slice level, so every comparison also holds the
error to 1e-10 of the largest reference element (of |E_T| for the energy)."""
import numpy as np

ABS_OMEGA = 1e-9
ABS_ENERGY = 1e-8
REL = 1e-10


def split_err(x, ref):
    """(max abs error, max |ref|)"""
    return float(np.abs(np.asarray(x) - ref).max()), float(np.abs(ref).max())


def split_close(x, ref, abs_tol=ABS_OMEGA, rel=REL):
    err, scale = split_err(x, ref)
    return err <= abs_tol and err <= rel * scale


def energy_close(e, ref, abs_tol=ABS_ENERGY, rel=REL):
    d = abs(float(e) - float(ref))
    return d <= abs_tol and d <= rel * abs(float(ref))
