"""Pins of the FP64 surrogate oracle (CPU only).

The forward is pinned to a brute-force DFT sum (independent of numpy's FFT),
to closed forms of the spectral convolution (band-limited inputs pass
unchanged through identity mode weights, modes outside the kept set vanish,
z-translation equivariance) and to a pointwise MLP when the spectral weights
are zero.  The backward is pinned to central finite differences of the
forward, block by block; planted mistakes in it must fail that check.  Adam
is pinned to its closed-form first step."""
import numpy as np
import pytest

from oracle.fno_oracle import FnoOracle, gelu, S_Q
from workloads import fno as F

TINY = F.FnoDims(Nz=8, Nr=6, C=2, mz=2, mr=2, L=1)


def _oracle(d, seed=0, masked=False):
    rng = np.random.default_rng(seed)
    rc = np.sort(rng.uniform(0.1, 4.0, d.Nr))
    zc = np.sort(rng.uniform(0.1, 10.0, d.Nz))
    reg = rng.integers(0, 5, size=(d.Nz, d.Nr))
    if masked:
        reg[rng.uniform(size=(d.Nz, d.Nr)) < 0.3] = -1
    return FnoOracle(d, rc, zc, 4.2, 10.2, region=reg)


def _params(n, seed):
    rng = np.random.default_rng(seed)
    k = np.exp(rng.uniform(np.log(0.1), np.log(400.0), size=(n, 5)))
    return np.concatenate([k, rng.uniform(1e5, 1e7, (n, 1)), rng.uniform(250, 350, (n, 1))], axis=1)


def test_spectral_matches_brute_force_dft():
    d = TINY
    o = _oracle(d)
    rng = np.random.default_rng(1)
    v = rng.standard_normal((2, d.C, d.Nz, d.Nr))
    Rre = rng.standard_normal((d.MZ, d.MR, d.C, d.C))
    Rim = rng.standard_normal((d.MZ, d.MR, d.C, d.C))
    s, _ = o.spectral(v, Rre, Rim)
    N = d.Nz * d.Nr
    jj, ii = np.meshgrid(np.arange(d.Nz), np.arange(d.Nr), indexing="ij")
    ref = np.zeros_like(s)
    for b in range(2):
        for zi, kz in enumerate(d.kz_list()):
            for kr in range(d.mr):
                th = 2 * np.pi * (kz * jj / d.Nz + kr * ii / d.Nr)
                Vh = [np.sum(v[b, c] * np.exp(-1j * th)) for c in range(d.C)]
                for oc in range(d.C):
                    Y = sum(Vh[c] * (Rre[zi, kr, c, oc] + 1j * Rim[zi, kr, c, oc]) for c in range(d.C))
                    a = 1.0 if kr == 0 else 2.0
                    ref[b, oc] += a / N * np.real(Y * np.exp(1j * th))
    np.testing.assert_allclose(s, ref, rtol=1e-12, atol=1e-12)


def test_identity_modes_pass_band_limited_fields_and_drop_the_rest():
    d = F.FnoDims(Nz=16, Nr=12, C=1, mz=3, mr=3, L=1)
    o = _oracle(d)
    jj, ii = np.meshgrid(np.arange(d.Nz), np.arange(d.Nr), indexing="ij")
    I_re = np.ones((d.MZ, d.MR, 1, 1))
    I_im = np.zeros_like(I_re)
    kept = np.cos(2 * np.pi * (2 * jj / d.Nz + 1 * ii / d.Nr)) + 0.5 * np.sin(2 * np.pi * (-2 * jj / d.Nz + 2 * ii / d.Nr)) + 3.0
    s, _ = o.spectral(kept[None, None], I_re, I_im)
    np.testing.assert_allclose(s[0, 0], kept, atol=1e-12)
    dropped = np.cos(2 * np.pi * (5 * jj / d.Nz)) + np.sin(2 * np.pi * (4 * ii / d.Nr + jj / d.Nz))
    s, _ = o.spectral(dropped[None, None], I_re, I_im)
    np.testing.assert_allclose(s, 0.0, atol=1e-12)


def test_spectral_is_z_translation_equivariant():
    d = F.MEDIUM
    o = _oracle(d)
    rng = np.random.default_rng(3)
    v = rng.standard_normal((1, d.C, d.Nz, d.Nr))
    w = o.unpack(F.random_params(d, 3))
    s1, _ = o.spectral(np.roll(v, 5, axis=2), w["Rre0"], w["Rim0"])
    s0, _ = o.spectral(v, w["Rre0"], w["Rim0"])
    np.testing.assert_allclose(s1, np.roll(s0, 5, axis=2), atol=1e-12)


def test_zero_spectral_weights_reduce_to_a_pointwise_mlp():
    d = F.SMALL
    o = _oracle(d)
    flat = F.random_params(d, 4)
    w = o.unpack(flat)
    for l in range(d.L):
        w[f"Rre{l}"][:] = 0.0
        w[f"Rim{l}"][:] = 0.0
    flat0 = o.pack(w)
    p = _params(2, 5)
    T = o.forward(flat0, p)
    x = o.features(p)
    for b, j, i in [(0, 0, 0), (1, 7, 3), (0, 15, 7)]:
        h = w["P"] @ x[b, :, j, i] + w["pb"]
        for l in range(d.L):
            h = w[f"W{l}"] @ h + w[f"wb{l}"]
            if l < d.L - 1:
                h = gelu(h)
        u = w["Q2"] @ gelu(w["Q1"] @ h + w["q1b"]) + w["q2b"]
        ref = 300.0 + S_Q * p[b, 5] * u[0] + (p[b, 6] - 300.0) * u[1]
        assert abs(T[b, j, i] - ref) <= 1e-9 * abs(ref)


def test_cell_features_follow_the_region_map():
    d = F.SMALL
    o = _oracle(d, seed=15, masked=True)
    p = _params(2, 16)
    x = o.features(p)
    for b, j, i in [(0, 0, 0), (1, 3, 5), (0, 9, 2), (1, 15, 7)]:
        r = o.region[j, i]
        onehot = [1.0 if r == m else 0.0 for m in range(5)]
        assert list(x[b, 9:14, j, i]) == onehot
        lnk = 2.0 * (np.log(p[b, r]) - np.log(0.1)) / (np.log(400.0) - np.log(0.1)) - 1.0 if r >= 0 else 0.0
        assert abs(x[b, 14, j, i] - lnk) <= 1e-12
        qn = 2.0 * (p[b, 5] - 1e5) / (1e7 - 1e5) - 1.0 if r == 2 else 0.0
        assert abs(x[b, 15, j, i] - qn) <= 1e-12


def test_void_cells_hold_the_initial_temperature():
    d = F.SMALL
    o = _oracle(d, masked=True)
    T = o.forward(F.random_params(d, 13), _params(3, 14))
    assert np.all(T[:, o.m == 0] == 300.0)
    assert np.all(T[:, o.m == 1] != 300.0)


def _fd_check(o, flat, p, Tt, seed, blocks=None):
    L0, g = o.grad(flat, p, Tt)
    rng = np.random.default_rng(seed)
    offs, off = {}, 0
    for name, shape in o.d.sizes():
        n = int(np.prod(shape))
        offs[name] = (off, n)
        off += n
    for name in (blocks or offs):
        a, n = offs[name]
        u = np.zeros_like(flat)
        u[a:a + n] = rng.standard_normal(n)
        eps = 1e-5 / max(np.max(np.abs(u)), 1e-30)
        fd = (o.loss(flat + eps * u, p, Tt) - o.loss(flat - eps * u, p, Tt)) / (2 * eps)
        an = float(g @ u)
        # central differences at eps ~ 1e-5 carry ~1e-11 rounding on an O(1) loss
        assert abs(fd - an) <= 1e-6 * max(abs(fd), abs(an)) + 1e-10 * max(1.0, L0), (name, fd, an)
    return L0


def _fd_case(d=F.SMALL):
    o = _oracle(d, seed=6, masked=True)
    flat = F.random_params(d, 7)
    p = _params(2, 8)
    Tt = 300.0 + S_Q * p[:, 5, None, None] * np.random.default_rng(9).uniform(0, 1, (2, d.Nz, d.Nr))
    return o, flat, p, Tt


def test_backward_matches_finite_differences_block_by_block():
    o, flat, p, Tt = _fd_case()
    _fd_check(o, flat, p, Tt, seed=10)


def test_planted_backward_mistakes_fail_the_finite_difference_check():
    o, flat, p, Tt = _fd_case()
    good = FnoOracle.spectral_backward

    def no_weight(self, gs, Vk, Rre, Rim):  # drops the irfft weight a_kr
        a = self.a
        self.a = np.ones_like(a)
        try:
            return good(self, gs, Vk, Rre, Rim)
        finally:
            self.a = a

    def no_conj(self, gs, Vk, Rre, Rim):  # mixes with R instead of conj(R)
        return good(self, gs, Vk, Rre, -Rim)

    for bad in (no_weight, no_conj):
        FnoOracle.spectral_backward = bad
        try:
            with pytest.raises(AssertionError):
                _fd_check(o, flat, p, Tt, seed=11, blocks=["Rre0", "Rim0", "P"])
        finally:
            FnoOracle.spectral_backward = good


def test_adam_first_step_is_lr_times_sign():
    rng = np.random.default_rng(12)
    x = rng.standard_normal(50)
    g = rng.standard_normal(50)
    m = np.zeros(50)
    v = np.zeros(50)
    x1, m, v = FnoOracle.adam(x, g, m, v, 1, lr=1e-3, eps=0.0)
    np.testing.assert_allclose(x1, x - 1e-3 * np.sign(g), rtol=0, atol=1e-12)
    x2, _, _ = FnoOracle.adam(x1, g, m, v, 2, lr=1e-3, eps=0.0)  # constant gradient: the same step again
    np.testing.assert_allclose(x2, x1 - 1e-3 * np.sign(g), rtol=0, atol=1e-12)
