"""Euclidean gamma matrices in the chiral basis (oracle).

The paper names the unimproved Wilson-Dirac operator (Sec. 5) without fixing
a basis.  Reading taken: the chiral basis
    gamma_0 = [[0, -1], [-1, 0]],   gamma_k = [[0, -i sigma_k], [i sigma_k, 0]]
in 2x2 spin blocks, gamma_5 = gamma_0 gamma_1 gamma_2 gamma_3 = diag(1, 1, -1, -1).
gamma index 0 is time, i.e. lattice axis 3; gamma_k (k = 1, 2, 3) belongs to
lattice axis k - 1.  A change of basis is a unitary similarity, so no
determinant depends on this choice, but the Dirac operator's output does, and
the CUDA path uses the same basis.
"""
import numpy as np

SIGMA = np.array([[[0, 1], [1, 0]],
                  [[0, -1j], [1j, 0]],
                  [[1, 0], [0, -1]]], dtype=np.complex128)

_I2 = np.eye(2, dtype=np.complex128)
_Z2 = np.zeros((2, 2), dtype=np.complex128)


def _blocks(a, b, c, d):
    return np.block([[a, b], [c, d]])


GAMMA = np.empty((4, 4, 4), dtype=np.complex128)   # GAMMA[mu] with mu = 0 (time), 1, 2, 3
GAMMA[0] = _blocks(_Z2, -_I2, -_I2, _Z2)
for _k in range(3):
    GAMMA[_k + 1] = _blocks(_Z2, -1j * SIGMA[_k], 1j * SIGMA[_k], _Z2)

GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]

# gamma matrix attached to each lattice axis a = 0, 1, 2, 3 (axis 3 = time)
AXIS_TO_MU = (1, 2, 3, 0)
GAMMA_AXIS = np.stack([GAMMA[AXIS_TO_MU[a]] for a in range(4)])

ONE4 = np.eye(4, dtype=np.complex128)
