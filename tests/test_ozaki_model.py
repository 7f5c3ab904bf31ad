"""Host-side model of the tensor-core trailing update of the blocked dense LU
(the Ozaki scheme of the exact check path, Sec. 3's exact block
determinants), checked against exact rational arithmetic.

The GPU tests compare the kernel with LAPACK and with the FP64 FMA update;
this file pins the numerical argument on which the kernel rests, on the CPU:
  * every row of [Re L, Im L] and column of [Re U; Im U] (64 reals) is scaled
    by 2^-e (e from frexp of the largest entry) and cut into 8 integer slices
    of 7 bits by round-to-nearest-even, each exact in FP16;
  * for every diagonal d = s + t < 8 the sum over the 64 terms of all slice
    products has absolute sum below 2^22, so an FP32 accumulator holds it
    exactly in any order, and four neighbouring diagonals combined by Horner's
    rule in 2^7 stay below 2^43 (exact in int64 and as an FP64 value);
  * what is left out (pairs with s + t >= 8 and the remainders after 8
    slices) is below 2^-48 of the product of the row and column maxima;
  * complex products as two real products over k = 64:
    C_re = [Re L, Im L] [Re U; -Im U], C_im = [Re L, Im L] [Im U; Re U].
Two mistakes planted in the model (6 slices instead of 8; +Im U instead of
-Im U in the real part) fail the 2^-48 check.
"""
from fractions import Fraction

import numpy as np
import pytest

BETA, S, NB = 7, 8, 32


def split(v, slices=S):
    """Slices of one 64-vector: (q[slices][64] integers, e) with
    v = 2^e sum_s q_s 2^(-BETA (s + 1)) + remainder."""
    mx = float(np.max(np.abs(v)))
    e = int(np.frexp(mx)[1]) if mx > 0.0 else 0
    t = np.ldexp(v, -e)
    q = np.zeros((slices, v.size))
    for s in range(slices):
        t = t * float(1 << BETA)
        q[s] = np.rint(t)
        t = t - q[s]
    return q.astype(np.int64), e


def model_product(L, U, slices=S, re_sign=-1):
    """The kernel's arithmetic for C = L U (L m x 32, U 32 x n complex):
    returns (C as FP64, C as exact rationals before the final FP64 sums,
    the largest absolute diagonal sum, the largest Horner group).  slices
    and re_sign (the sign of Im U in the real part) exist so that a test can
    plant a mistake."""
    m, n = L.shape[0], U.shape[1]
    A = np.concatenate([L.real, L.imag], axis=1)  # m x 64
    sa = [split(A[i], slices) for i in range(m)]
    # the column's exponent is shared by its real and imaginary parts
    sb = [split(np.concatenate([U.real[:, j], U.imag[:, j]]), slices) for j in range(n)]
    C = np.zeros((m, n), dtype=np.complex128)
    Cx = [[None] * n for _ in range(m)]
    diag_max = 0
    group_max = 0
    for i in range(m):
        qa, ea = sa[i]
        for j in range(n):
            qcol, eb = sb[j]
            # slices of [Re U; -Im U] and [Im U; Re U] from the column's slices
            qre = np.concatenate([qcol[:, :NB], re_sign * qcol[:, NB:]], axis=1)
            qim = np.concatenate([qcol[:, NB:], qcol[:, :NB]], axis=1)
            acc = [0.0, 0.0]
            exact = [Fraction(0), Fraction(0)]
            for part, qb in enumerate((qre, qim)):
                g = 0
                for d in range(slices):
                    terms = [qa[s] * qb[d - s] for s in range(d + 1)]
                    f = int(sum(int(np.sum(t)) for t in terms))
                    diag_max = max(diag_max, int(sum(int(np.sum(np.abs(t))) for t in terms)))
                    g = g * (1 << BETA) + f
                    group_max = max(group_max, abs(g))
                    exact[part] += Fraction(f) / Fraction(2) ** (BETA * (d + 2))
                    if d % 4 == 3 or d == slices - 1:
                        # 2^-w g is exact (|g| < 2^43), so this add rounds
                        # as the kernel's fused multiply-add does
                        acc[part] = acc[part] + np.ldexp(float(g), -BETA * (d + 2))
                        g = 0
                sc = Fraction(2) ** (ea + eb) if ea + eb >= 0 else Fraction(1, 2 ** -(ea + eb))
                exact[part] *= sc
            C[i, j] = complex(np.ldexp(acc[0], ea + eb), np.ldexp(acc[1], ea + eb))
            Cx[i][j] = exact
    return C, Cx, diag_max, group_max


def exact_product(L, U):
    """C = L U in exact rational arithmetic (real and imaginary parts)."""
    m, k = L.shape
    n = U.shape[1]
    F = Fraction
    out = []
    for i in range(m):
        row = []
        for j in range(n):
            re = sum(F(L[i, t].real) * F(U[t, j].real) - F(L[i, t].imag) * F(U[t, j].imag) for t in range(k))
            im = sum(F(L[i, t].real) * F(U[t, j].imag) + F(L[i, t].imag) * F(U[t, j].real) for t in range(k))
            row.append((re, im))
        out.append(row)
    return out


def operands(seed, m=5, n=4, spread=40):
    """Complex operands with row and column scales over 2^+-spread, a few
    exact zeros, and entries at the top of their row's binade (first slices
    of magnitude 128)."""
    rng = np.random.default_rng(seed)
    L = rng.standard_normal((m, NB)) + 1j * rng.standard_normal((m, NB))
    U = rng.standard_normal((NB, n)) + 1j * rng.standard_normal((NB, n))
    L *= np.ldexp(1.0, rng.integers(-spread, spread, size=(m, 1)))
    U *= np.ldexp(1.0, rng.integers(-spread, spread, size=(1, n)))
    L[0, 3] = 0.0
    U[5, 0] = 0.0
    L[1, 0] = np.ldexp(0.9999999, int(np.frexp(np.max(np.abs(L[1])))[1]))  # rounds to a first slice of 128
    return L, U


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_ozaki_slices_exact_in_fp32_and_within_2_48(seed):
    L, U = operands(seed)
    C, Cx, diag_max, group_max = model_product(L, U)
    assert diag_max < 2 ** 22
    assert group_max < 2 ** 43
    ref = exact_product(L, U)
    A = np.concatenate([L.real, L.imag], axis=1)
    for i in range(L.shape[0]):
        rmax = float(np.max(np.abs(A[i])))
        for j in range(U.shape[1]):
            cmax = float(max(np.max(np.abs(U.real[:, j])), np.max(np.abs(U.imag[:, j]))))
            scale = Fraction(rmax) * Fraction(cmax)
            for part in (0, 1):
                # what the slices leave out, before any FP64 rounding
                dropped = abs(Cx[i][j][part] - ref[i][j][part])
                assert dropped <= scale / 2 ** 48, (i, j, part, float(dropped / scale))
            # the FP64 result (the dropped part plus the roundings of the two
            # group sums) within the rounding bound of an FP64 dot product of
            # the same 64 terms, 64 x 2^-53 sum_k |a_k b_k|
            got = (C[i, j].real, C[i, j].imag)
            for part, b in enumerate((np.concatenate([U.real[:, j], -U.imag[:, j]]),
                                      np.concatenate([U.imag[:, j], U.real[:, j]]))):
                err = abs(Fraction(got[part]) - ref[i][j][part])
                mag = sum(Fraction(abs(x)) * Fraction(abs(y)) for x, y in zip(A[i], b))
                assert err <= 64 * mag / 2 ** 53, (i, j, part, float(err / mag))


def test_ozaki_model_detects_a_dropped_slice_and_a_sign():
    """The 2^-48 check fails for the model with 6 slices instead of 8, or
    with +Im U instead of -Im U in the real part."""
    L, U = operands(5, m=3, n=3)
    ref = exact_product(L, U)
    A = np.concatenate([L.real, L.imag], axis=1)
    scale = Fraction(float(np.max(np.abs(A[0])))) * Fraction(
        float(max(np.max(np.abs(U.real[:, 0])), np.max(np.abs(U.imag[:, 0])))))
    _, Cx, _, _ = model_product(L, U)
    assert abs(Cx[0][0][0] - ref[0][0][0]) <= scale / 2 ** 48
    _, Cx, _, _ = model_product(L, U, slices=6)
    assert abs(Cx[0][0][0] - ref[0][0][0]) > scale / 2 ** 48
    _, Cx, _, _ = model_product(L, U, re_sign=+1)
    assert abs(Cx[0][0][0] - ref[0][0][0]) > scale / 2 ** 48
