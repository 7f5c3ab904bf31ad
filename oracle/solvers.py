"""Textbook conjugate gradient on the normal equations (oracle, FP64).

Solves A x = b through A^dag A x = A^dag b (CGNR; Hestenes-Stiefel CG on the
Hermitian positive definite normal operator).  The stopping rule is the true
residual ||b - A x|| <= tol ||b||, recomputed from A itself.
"""
import numpy as np


def vdot(a, b):
    return complex(np.vdot(a.reshape(-1), b.reshape(-1)))


def norm2(a):
    return float(np.vdot(a.reshape(-1), a.reshape(-1)).real)


def cgnr(apply_A, apply_Adag, b, tol=1e-14, maxit=100000, x0=None):
    """Return (x, iterations, true relative residual)."""
    bn = np.sqrt(norm2(b))
    if bn == 0.0:
        return np.zeros_like(b), 0, 0.0
    x = np.zeros_like(b) if x0 is None else np.array(x0, copy=True)
    r = b - apply_A(x)
    z = apply_Adag(r)
    p = z.copy()
    zz = norm2(z)
    it = 0
    while it < maxit:
        q = apply_A(p)
        alpha = zz / norm2(q)
        x += alpha * p
        r -= alpha * q
        it += 1
        if np.sqrt(norm2(r)) <= 0.5 * tol * bn:
            rt = b - apply_A(x)            # confirm with the true residual
            if np.sqrt(norm2(rt)) <= tol * bn:
                r = rt
                break
            r = rt
            z = apply_Adag(r)
            p = z.copy()
            zz = norm2(z)
            continue
        z = apply_Adag(r)
        zz_new = norm2(z)
        p = z + (zz_new / zz) * p
        zz = zz_new
    rt = b - apply_A(x)
    return x, it, float(np.sqrt(norm2(rt)) / bn)
