"""Plain FP64 CPU oracle of the temperature-field surrogate.

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and by the CPU-baseline leg
of ``bench.py``; the CUDA library never imports, links or calls it.

The paper has no surrogate.  This is a Fourier neural operator (FNO, the
architecture of Li et al., "Fourier neural operator for parametric partial
differential equations", 2021) written out in numpy, step by step, for the
map (5 region conductivities k, heater power q, Dirichlet temperature T_D)
-> temperature field after a fixed number of ADI steps of the paper's scheme
(Sec. 3) on a fixed grid.  Spectral transforms use numpy's FFT as a library
primitive; everything else is explicit array arithmetic.

Definition:
  features  x_f (16 channels): 5 x scaled ln k, scaled q, scaled T_D (all
            broadcast over the grid), scaled r and z cell centres, the one-hot
            region of the cell (5 channels, all 0 on void), the cell's own
            scaled ln k (0 on void) and the scaled q on heater cells (0
            elsewhere): the geometry is fixed, so these are positional
            features that tell the network which material each cell holds
  lift      v_0 = P x + pb                                  (C channels)
  layer l   pre_l = K_l(v_l) + W_l v_l + wb_l,
            v_{l+1} = gelu(pre_l) for l < L-1, pre_l for the last layer
  spectral  K(v) = irfft2( pad( R  .  trunc(rfft2(v)) ) ), keeping
            kz in {0..mz-1, Nz-mz..Nz-1} and kr in {0..mr-1}, with a complex
            C x C matrix R per kept mode
  project   h = gelu(Q1 v_L + q1b),  u = Q2 h + q2b          (2 channels)
  output    T = T_init + m (S_Q q u_0 + (T_D - T_init) u_1)
  loss      mean over samples and cells of ((T - T_true) / (S_Q q))^2
The output head is linear in q and T_D because the discrete heat equation
is linear in its source and its Dirichlet value (Sec. 3, eqs.
"scheme_eq_1", "scheme_eq_2"): T - T_init = q G(k) + (T_D - T_init) H(k).
m is the active-cell indicator of the geometry (1 where the cell centre
lies in a region box, 0 on void cells): the scheme keeps void cells at
T_init (identity rows), so the field jumps at the void's edge, a jump the
network is not asked to reproduce.
gelu(x) = x/2 (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))).
"""
from __future__ import annotations

import numpy as np

LNK_LO, LNK_HI = np.log(0.1), np.log(400.0)
Q_LO, Q_HI = 1.0e5, 1.0e7
TD_MID, TD_HALF = 300.0, 50.0
S_Q = 0.02
GELU_C = np.sqrt(2.0 / np.pi)


def gelu(x):
    return 0.5 * x * (1.0 + np.tanh(GELU_C * (x + 0.044715 * x ** 3)))


def gelu_grad(x):
    t = np.tanh(GELU_C * (x + 0.044715 * x ** 3))
    return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t * t) * GELU_C * (1.0 + 3 * 0.044715 * x * x)


class FnoOracle:
    """FNO forward, loss, backward and Adam in FP64.

    d: a ``workloads.fno.FnoDims``; rc [Nr], zc [Nz]: cell centres; R, Z: the
    outer radius and height used to scale the coordinates; region [Nz, Nr]:
    the region of each cell (0..4, -1 on void; all 0 if None), whose
    indicator region >= 0 is the active-cell mask m; heater: the region that
    holds the source q."""

    def __init__(self, d, rc, zc, R, Z, T_init=300.0, region=None, heater=2):
        self.d = d
        self.region = np.zeros((d.Nz, d.Nr), dtype=np.int64) if region is None else np.asarray(region, dtype=np.int64)
        assert self.region.shape == (d.Nz, d.Nr)
        self.m = (self.region >= 0).astype(np.float64)
        self.heater = int(heater)
        self.rc = np.asarray(rc, dtype=np.float64)
        self.zc = np.asarray(zc, dtype=np.float64)
        assert self.rc.shape == (d.Nr,) and self.zc.shape == (d.Nz,)
        self.R, self.Z, self.T_init = float(R), float(Z), float(T_init)
        self.kz = np.array(d.kz_list())
        self.a = np.where(np.arange(d.mr) == 0, 1.0, 2.0)  # irfft weights of the kept kr

    # ---- parameters
    def unpack(self, flat):
        out, o = {}, 0
        for name, shape in self.d.sizes():
            n = int(np.prod(shape))
            out[name] = np.asarray(flat[o:o + n], dtype=np.float64).reshape(shape)
            o += n
        assert o == len(flat)
        return out

    def pack(self, parts):
        return np.concatenate([parts[name].ravel() for name, _ in self.d.sizes()])

    # ---- features: [B, 16, Nz, Nr]
    def features(self, params):
        p = np.asarray(params, dtype=np.float64).reshape(-1, 7)
        B, d = p.shape[0], self.d
        x = np.zeros((B, 16, d.Nz, d.Nr))
        for m in range(5):
            x[:, m] = (2.0 * (np.log(p[:, m]) - LNK_LO) / (LNK_HI - LNK_LO) - 1.0)[:, None, None]
        x[:, 5] = (2.0 * (p[:, 5] - Q_LO) / (Q_HI - Q_LO) - 1.0)[:, None, None]
        x[:, 6] = ((p[:, 6] - TD_MID) / TD_HALF)[:, None, None]
        x[:, 7] = (2.0 * self.rc / self.R - 1.0)[None, None, :]
        x[:, 8] = (2.0 * self.zc / self.Z - 1.0)[None, :, None]
        for m in range(5):
            on = self.region == m
            x[:, 9 + m] = on[None].astype(np.float64)
            x[:, 14] += on[None] * x[:, m]
        x[:, 15] = (self.region == self.heater)[None] * x[:, 5]
        return x

    # ---- spectral convolution and its adjoints
    def _modes(self, v):
        """Kept modes of rfft2 over (z, r): [B, C, MZ, MR] complex."""
        V = np.fft.rfft2(v, axes=(-2, -1))
        return V[:, :, self.kz, :][:, :, :, : self.d.mr]

    def _pad_irfft(self, Y):
        d = self.d
        full = np.zeros(Y.shape[:2] + (d.Nz, d.Nr // 2 + 1), dtype=np.complex128)
        full[:, :, self.kz, : d.mr] = Y
        return np.fft.irfft2(full, s=(d.Nz, d.Nr), axes=(-2, -1))

    def spectral(self, v, Rre, Rim):
        Vk = self._modes(v)
        Rc = Rre + 1j * Rim                               # [MZ, MR, C, O]
        Y = np.einsum("bczr,zrco->bozr", Vk, Rc)
        return self._pad_irfft(Y), Vk

    def spectral_backward(self, gs, Vk, Rre, Rim):
        """(dv, dRre, dRim) from gs = dL/ds and the forward's kept modes Vk."""
        d = self.d
        N = d.Nz * d.Nr
        gY = self._modes(gs) * (self.a / N)[None, None, None, :]
        Rc = Rre + 1j * Rim
        dR = np.einsum("bczr,bozr->zrco", np.conj(Vk), gY)
        gV = np.einsum("bozr,zrco->bczr", gY, np.conj(Rc))
        dv = N * self._pad_irfft(gV / self.a[None, None, None, :])
        return dv, dR.real, dR.imag

    # ---- network
    def forward(self, flat, params, keep=False):
        """Temperature fields [B, Nz, Nr]; with keep=True also the cache for backward."""
        w = self.unpack(flat)
        d = self.d
        p = np.asarray(params, dtype=np.float64).reshape(-1, 7)
        x = self.features(p)
        v = np.einsum("cf,bfzr->bczr", w["P"], x) + w["pb"][None, :, None, None]
        cache = {"x": x, "v": [v], "pre": [], "Vk": []}
        for l in range(d.L):
            s, Vk = self.spectral(v, w[f"Rre{l}"], w[f"Rim{l}"])
            pre = s + np.einsum("oc,bczr->bozr", w[f"W{l}"], v) + w[f"wb{l}"][None, :, None, None]
            v = gelu(pre) if l < d.L - 1 else pre
            cache["pre"].append(pre)
            cache["Vk"].append(Vk)
            cache["v"].append(v)
        hpre = np.einsum("hc,bczr->bhzr", w["Q1"], v) + w["q1b"][None, :, None, None]
        h = gelu(hpre)
        u = np.einsum("oh,bhzr->bozr", w["Q2"], h) + w["q2b"][None, :, None, None]
        q, Td = p[:, 5], p[:, 6]
        T = self.T_init + self.m[None] * ((S_Q * q)[:, None, None] * u[:, 0] + (Td - self.T_init)[:, None, None] * u[:, 1])
        cache.update(hpre=hpre, h=h, u=u, p=p)
        return (T, cache) if keep else T

    def loss(self, flat, params, T_true):
        T = self.forward(flat, params)
        q = np.asarray(params, dtype=np.float64).reshape(-1, 7)[:, 5]
        e = (T - np.asarray(T_true, dtype=np.float64)) / (S_Q * q)[:, None, None]
        return float(np.mean(e * e))

    def grad(self, flat, params, T_true):
        """(loss, dL/dflat) by reverse-mode differentiation of the forward above."""
        d = self.d
        w = self.unpack(flat)
        T, c = self.forward(flat, params, keep=True)
        p = c["p"]
        q, Td = p[:, 5], p[:, 6]
        sc = (S_Q * q)[:, None, None]
        e = (T - np.asarray(T_true, dtype=np.float64)) / sc
        Ntot = e.size
        L = float(np.mean(e * e))
        gT = 2.0 * e / sc / Ntot * self.m[None]
        gu = np.stack([gT * sc, gT * (Td - self.T_init)[:, None, None]], axis=1)
        g = {}
        g["Q2"] = np.einsum("bozr,bhzr->oh", gu, c["h"])
        g["q2b"] = gu.sum(axis=(0, 2, 3))
        gh = np.einsum("oh,bozr->bhzr", w["Q2"], gu) * gelu_grad(c["hpre"])
        vL = c["v"][d.L]
        g["Q1"] = np.einsum("bhzr,bczr->hc", gh, vL)
        g["q1b"] = gh.sum(axis=(0, 2, 3))
        gv = np.einsum("hc,bhzr->bczr", w["Q1"], gh)
        for l in reversed(range(d.L)):
            pre = c["pre"][l]
            gpre = gv * gelu_grad(pre) if l < d.L - 1 else gv
            vl = c["v"][l]
            g[f"W{l}"] = np.einsum("bozr,bczr->oc", gpre, vl)
            g[f"wb{l}"] = gpre.sum(axis=(0, 2, 3))
            dv_s, g[f"Rre{l}"], g[f"Rim{l}"] = self.spectral_backward(gpre, c["Vk"][l], w[f"Rre{l}"], w[f"Rim{l}"])
            gv = np.einsum("oc,bozr->bczr", w[f"W{l}"], gpre) + dv_s
        g["P"] = np.einsum("bczr,bfzr->cf", gv, c["x"])
        g["pb"] = gv.sum(axis=(0, 2, 3))
        return L, self.pack(g)

    @staticmethod
    def adam(flat, grad, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
        """One Adam step (Kingma and Ba, 2015) with bias correction; t counts from 1.
        Returns the new (flat, m, v)."""
        m = b1 * m + (1.0 - b1) * grad
        v = b2 * v + (1.0 - b2) * grad * grad
        mh = m / (1.0 - b1 ** t)
        vh = v / (1.0 - b2 ** t)
        return flat - lr * mh / (np.sqrt(vh) + eps), m, v
