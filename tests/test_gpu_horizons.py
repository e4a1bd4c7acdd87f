"""Parity over the workloads' full horizons, not a few steps.

Config 2 (2048 x 4096, the benchmark's grid and launch configuration) for its
full 1000 steps in FP64 and FP32, against one 1000-step oracle run; config 3's
smallest and largest members and four sampled ones for their full 500 steps
in every precision.  Bars as everywhere (relative max-norm 1e-12 FP64, 1e-5
FP32); the error relative to the temperature rise and the energy change are
printed beside them.  The oracle needs about 40 s of host time for config 2.
"""
import numpy as np
import pytest

from oracle import Oracle
from workloads import heat as H

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5, "fp32_refined": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _norms(Tg, To, T_init):
    d = np.max(np.abs(Tg - To))
    return d / np.max(np.abs(To)), d / max(np.max(np.abs(To - T_init)), 1e-300)


@pytest.fixture(scope="module")
def config2_oracle():
    p = H.config2()
    o = Oracle(p)
    tau = H.DT_FACTOR * o.tau_exp()
    E0 = o.energy()[0]
    o.step(tau, H.STEPS["config2"])
    return p, tau, o.field(), E0, o.energy()[0]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_config2_full_horizon(config2_oracle, precision):
    from paper_1912_03744_gb300 import HeatSolver
    p, tau, To, E0, Eo = config2_oracle
    s = HeatSolver(p, tau, precision=precision)
    s.step(H.STEPS["config2"])
    Tg = s.field()
    E, _, _ = s.energy()
    s.close()
    rel, rise = _norms(Tg, To, p.T_init)
    dE = abs((E - E0) - (Eo - E0)) / abs(Eo - E0)
    print(f"config2 2048x4096 {precision}, {H.STEPS['config2']} steps: rel max {rel:.3e}, "
          f"rise-relative {rise:.3e}, energy change {dE:.3e}")
    assert rel <= TOL[precision], rel


def _pick(members, k, seed):
    cells = [p.Nr * p.Nz for p in members]
    idx = {int(np.argmin(cells)), int(np.argmax(cells))}
    rng = np.random.default_rng(seed)
    for i in rng.permutation(len(members)):
        if len(idx) >= k + 2:
            break
        idx.add(int(i))
    return sorted(idx)


@pytest.fixture(scope="module")
def config3_oracle():
    members = H.config3_members(512)
    sel = _pick(members, 4, seed=9)
    probs = [members[i] for i in sel]
    ref, dts = [], []
    for p in probs:
        o = Oracle(p)
        tau = H.DT_FACTOR * o.tau_exp()
        o.step(tau, H.STEPS["config3"])
        ref.append(o.field())
        dts.append(tau)
    return sel, probs, ref, dts


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_refined"])
def test_config3_members_full_horizon(config3_oracle, precision):
    from paper_1912_03744_gb300 import HeatBatch
    sel, probs, ref, dts = config3_oracle
    b = HeatBatch(probs, dts, precision=precision)
    b.step(H.STEPS["config3"])
    for m, To, i, p in zip(b.members, ref, sel, probs):
        rel, rise = _norms(m.field(), To, p.T_init)
        print(f"config3 member {i} ({p.Nr}x{p.Nz}) {precision}, {H.STEPS['config3']} steps: "
              f"rel max {rel:.3e}, rise-relative {rise:.3e}")
        assert rel <= TOL[precision], (i, rel)
    b.close()
