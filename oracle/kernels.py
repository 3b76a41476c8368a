"""Entries of the interaction matrix A (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

A_ij is the interaction between target u_i and source v_j (Sec. 2, eq. Ax=b);
sources equal targets in every experiment (Sec. 4).  Off-diagonal entries:
  log2d : log |x_i - x_j|          (Sec. 4.4, Experiment 4 kernel)
  invr2d: 1 / |x_i - x_j|          (Sec. 4.3, Experiment 3)
  invr3d: 1 / |x_i - x_j|          (3D analogue)
  gauss : exp(-|x_i - x_j|^2 / l^2)
The diagonal A_ii is a given constant (e.g. sqrt(1000 N) in Experiments 1-3).
Parity: these are the definitions; pinned by closed-form values in the tests.
"""
from __future__ import annotations

import numpy as np

LOG2D, INVR3D, INVR2D, GAUSS = 0, 1, 2, 3


class Kernel:
    def __init__(self, kind: int, diag: float, length: float = 1.0):
        self.kind, self.diag, self.length = int(kind), float(diag), float(length)

    def offdiag(self, r2: np.ndarray) -> np.ndarray:
        """Kernel value as a function of the squared distance."""
        if self.kind == LOG2D:
            return 0.5 * np.log(r2)
        if self.kind in (INVR2D, INVR3D):
            return 1.0 / np.sqrt(r2)
        if self.kind == GAUSS:
            return np.exp(-r2 / (self.length * self.length))
        raise ValueError(self.kind)

    def block(self, pts: np.ndarray, I, J) -> np.ndarray:
        """A[I, J] for index arrays I, J into ``pts`` (same index = diagonal)."""
        I = np.asarray(I, dtype=np.int64)
        J = np.asarray(J, dtype=np.int64)
        X = pts[I][:, None, :]
        Y = pts[J][None, :, :]
        r2 = ((X - Y) ** 2).sum(axis=-1)
        same = I[:, None] == J[None, :]
        with np.errstate(divide="ignore", invalid="ignore"):
            out = self.offdiag(np.where(same, 1.0, r2))
        if np.any((r2 == 0) & ~same):
            raise ValueError("duplicate points: kernel is singular")
        out[same] = self.diag
        return out

    def dense(self, pts: np.ndarray) -> np.ndarray:
        idx = np.arange(len(pts))
        return self.block(pts, idx, idx)
