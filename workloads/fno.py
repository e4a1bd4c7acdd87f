"""Seeded inputs of the temperature-field surrogate (shared by the oracle and
the CUDA path; holds no surrogate arithmetic, only shapes and random draws).

The surrogate is not in the paper: it is a Fourier neural operator (FNO)
that maps the 7 scalars of a cell instance (5 region conductivities, heater
power q, Dirichlet temperature T_D) to the temperature field after a fixed
number of ADI steps on a fixed grid.

Flat parameter vector (FP32 on the device, FP64 in the oracle), in order:
    P   [C, F]   lift weights,  pb [C]
    per layer l < L:
        W_l [C, C]   pointwise weights,  wb_l [C]
        Rre_l, Rim_l [MZ, MR, C, C]  spectral weights, (kz index, kr, in c, out o)
    Q1 [H, C], q1b [H]   projection hidden layer
    Q2 [2, H], q2b [2]   projection output layer
with F = 16 input features (7 per-sample scalars, r, z, the cell's one-hot
region, ln k and heater source), H = 2 C hidden projection channels,
MZ = 2 mz kept z-modes (kz = 0..mz-1 and Nz-mz..Nz-1), MR = mr kept r-modes.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

N_FEATURES = 16


@dataclass(frozen=True)
class FnoDims:
    Nz: int = 256
    Nr: int = 128
    C: int = 32
    mz: int = 12
    mr: int = 12
    L: int = 4

    @property
    def H(self) -> int:
        return 2 * self.C

    @property
    def MZ(self) -> int:
        return 2 * self.mz

    @property
    def MR(self) -> int:
        return self.mr

    def kz_list(self):
        """The kept z wave numbers in kz-index order."""
        return list(range(self.mz)) + list(range(self.Nz - self.mz, self.Nz))

    def sizes(self):
        """(name, shape) of every block of the flat vector, in order."""
        C, F, H, MZ, MR = self.C, N_FEATURES, self.H, self.MZ, self.MR
        out = [("P", (C, F)), ("pb", (C,))]
        for l in range(self.L):
            out += [(f"W{l}", (C, C)), (f"wb{l}", (C,)), (f"Rre{l}", (MZ, MR, C, C)), (f"Rim{l}", (MZ, MR, C, C))]
        out += [("Q1", (H, C)), ("q1b", (H,)), ("Q2", (2, H)), ("q2b", (2,))]
        return out

    def n_params(self) -> int:
        return int(sum(np.prod(s) for _, s in self.sizes()))


SMALL = FnoDims(Nz=16, Nr=8, C=4, mz=3, mr=3, L=2)     # gradient checks on the CPU
MEDIUM = FnoDims(Nz=64, Nr=32, C=16, mz=6, mr=6, L=3)  # GPU-vs-oracle parity


def init_params(d: FnoDims, seed: int = 0) -> np.ndarray:
    """Seeded initial weights: dense blocks uniform in +-1/sqrt(fan_in), biases
    zero, spectral weights uniform in [0, 1/(C*C)) (re and im), draw order as
    in FnoDims.sizes()."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, shape in d.sizes():
        if name.startswith(("Rre", "Rim")):
            parts.append(rng.uniform(0.0, 1.0 / (d.C * d.C), size=shape))
        elif len(shape) == 2:
            b = 1.0 / np.sqrt(shape[1])
            parts.append(rng.uniform(-b, b, size=shape))
        else:
            parts.append(np.zeros(shape))
    return np.concatenate([p.ravel() for p in parts])


def random_params(d: FnoDims, seed: int) -> np.ndarray:
    """Seeded weights with nonzero biases (for gradient checks)."""
    rng = np.random.default_rng(seed)
    x = init_params(d, seed)
    return x + 0.1 * rng.standard_normal(x.shape) * (np.abs(x) + 0.05)
