"""Batched ensemble (heat_batch_*) against the FP64 oracle, member by member.

Every member is compared with its own single-instance oracle run, including
the smallest and largest members of the 512-member ensemble; the schedules
the autotuner can pick must all stay within the FP tolerance."""
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


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _pick(members, k, seed=0):
    """Smallest and largest members by cell count, plus k others."""
    cells = [p.Nr * p.Nz for p in members]
    idx = {int(np.argmin(cells)), int(np.argmax(cells))}
    rng = np.random.default_rng(seed)
    for i in rng.permutation(len(members)):
        if len(idx) >= k + 2:
            break
        idx.add(int(i))
    return sorted(idx)


def _oracle_runs(probs, steps, factor=H.DT_FACTOR):
    out, dts = [], []
    for p in probs:
        o = Oracle(p)
        tau = factor * o.tau_exp()
        o.step(tau, steps)
        out.append(o.field())
        dts.append(tau)
    return out, dts


ENSEMBLE = H.config3_members(512)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_refined"])
def test_members_match_their_oracle_runs(precision):
    from paper_1912_03744_gb300 import HeatBatch
    sel = _pick(ENSEMBLE, 6, seed=1)
    probs = [ENSEMBLE[i] for i in sel]
    steps = 23  # two 10-step graph replays and three 1-step ones
    ref, dts = _oracle_runs(probs, steps)
    b = HeatBatch(probs, dts, precision=precision)
    assert b.launches_per_step() == (7 if precision == "fp32_refined" else 4)
    b.step(steps)
    for m, To, i in zip(b.members, ref, sel):
        assert _rel(m.field(), To) <= TOL[precision], (i, m.Nr, m.Nz)
    b.close()


@pytest.mark.parametrize("tuning", [(2, 0, 1), (2, 4, 2), (2, 64, 1), (1, 0, 1), (1, 1, 2), (1, 16, 1), (8, 1, 1), (16, 2, 2), (16, 0, 1), (32, 4, 2),
                                    (32, 64, 1), (16, 1000, 2)])
def test_every_schedule_gives_the_same_answer(tuning):
    from paper_1912_03744_gb300 import HeatBatch
    sel = _pick(ENSEMBLE, 3, seed=2)
    probs = [ENSEMBLE[i] for i in sel]
    ref, dts = _oracle_runs(probs, 12)
    b = HeatBatch(probs, dts, precision="fp32")
    rK, band, zw = tuning
    if rK >= 4 and max(p.Nr for p in probs) > 32 * rK:  # block lines: one line within one warp
        from paper_1912_03744_gb300.heat import HeatError
        with pytest.raises(HeatError):
            b.set_tuning(rK, band, zw)
        b.close()
        return
    b.set_tuning(rK, band, zw)
    assert b.tuning()[0] == rK and b.tuning()[2] == zw
    b.step(12)
    for m, To in zip(b.members, ref):
        assert _rel(m.field(), To) <= 1e-5
    b.close()


def test_work_list_mixes_tiled_and_plain_members():
    """The batch's z passes run on a work list of (member, chunk, column tile):
    the five-region cell at 512 and 1000 columns is tiled by column class,
    the homogeneous cylinder and the small member are not; members of
    different chunk counts (Nz 130 .. 1024) share one launch."""
    from paper_1912_03744_gb300 import HeatBatch
    probs = [H.config2(512, 256), H.config2(1000, 130), ENSEMBLE[0],
             H.homogeneous_cylinder(300, 1024, R=2.0, Z=3.0, k=5.0, C=2.0e6, bc=(0, 1, 0, 1),
                                    T_bc=(0, 250.0, 0, 310.0), T_init=300.0, q=1e5)]
    ref, dts = _oracle_runs(probs, 9)
    for precision in ("fp32", "fp64"):
        b = HeatBatch(probs, dts, precision=precision)
        b.step(9)
        for m, To in zip(b.members, ref):
            assert _rel(m.field(), To) <= TOL[precision], (precision, m.Nr, m.Nz)
        b.close()


def test_work_list_with_different_chunk_rows():
    """Members whose z chunks differ in rows (Nz 20: one chunk of 20 rows;
    300: chunks of 32; 9000: chunks of 36) share the work list's blocks, so
    warps of different members stage their tables side by side in a block's
    shared memory."""
    from paper_1912_03744_gb300 import HeatBatch
    cyl = dict(R=2.0, Z=3.0, k=5.0, C=2.0e6, bc=(0, 1, 0, 1), T_bc=(0, 250.0, 0, 310.0), T_init=300.0, q=1e5)
    probs = [H.homogeneous_cylinder(100, 20, **cyl), H.homogeneous_cylinder(300, 300, **cyl),
             H.homogeneous_cylinder(64, 9000, **cyl), H.homogeneous_cylinder(36, 20, **cyl)]
    T0 = [H.random_field(p, seed=i, amp=20.0) for i, p in enumerate(probs)]
    ref, dts = [], []
    for p, t in zip(probs, T0):
        o = Oracle(p)
        tau = 5.0 * o.tau_exp()
        o.set_field(t)
        o.step(tau, 6)
        ref.append(o.field())
        dts.append(tau)
    for precision in ("fp32", "fp64"):
        b = HeatBatch(probs, dts, precision=precision)
        for m, t in zip(b.members, T0):
            m.set_field(t)
        b.step(6)
        for m, To in zip(b.members, ref):
            assert _rel(m.field(), To) <= TOL[precision], (precision, m.Nr, m.Nz)
        b.close()


def test_tune_leaves_the_state_unchanged_and_then_steps_correctly():
    from paper_1912_03744_gb300 import HeatBatch
    sel = _pick(ENSEMBLE, 4, seed=3)
    probs = [ENSEMBLE[i] for i in sel]
    ref, dts = _oracle_runs(probs, 7)
    b = HeatBatch(probs, dts, precision="fp32")
    T0 = [H.random_field(p, seed=i, amp=10.0) + 0.0 for i, p in enumerate(probs)]
    for m, t in zip(b.members, T0):
        m.set_field(t)
    before = [m.field() for m in b.members]
    ms = b.tune(trial_steps=2)
    assert ms > 0.0
    after = [m.field() for m in b.members]
    for x, y in zip(before, after):
        np.testing.assert_array_equal(x, y)
    # back to the initial state, then 7 steps under the tuned schedule
    for m, p in zip(b.members, probs):
        m.set_field(np.full((p.Nz, p.Nr), p.T_init))
    b.step(7)
    for m, To in zip(b.members, ref):
        assert _rel(m.field(), To) <= 1e-5
    b.close()


def test_full_ensemble_sampled_members():
    """All 512 members in the launch configuration the benchmark times
    (autotuned schedule, graph replay); sampled members against the oracle."""
    from paper_1912_03744_gb300 import HeatBatch
    steps = 5
    dts = [H.DT_FACTOR * Oracle(p).tau_exp() for p in ENSEMBLE]
    b = HeatBatch(ENSEMBLE, dts, precision="fp32")
    b.tune(trial_steps=2)
    b.step(steps)
    b.sync()
    for i in _pick(ENSEMBLE, 6, seed=4):
        o = Oracle(ENSEMBLE[i])
        o.step(dts[i], steps)
        assert _rel(b.members[i].field(), o.field()) <= 1e-5, i
    b.close()


def test_batch_heat_balance_fp64():
    from paper_1912_03744_gb300 import HeatBatch
    probs = [ENSEMBLE[i] for i in _pick(ENSEMBLE, 2, seed=5)]
    dts = [H.DT_FACTOR * Oracle(p).tau_exp() for p in probs]
    b = HeatBatch(probs, dts, precision="fp64")
    for i, m in enumerate(b.members):
        m.set_field(H.random_field(probs[i], seed=10 + i, amp=30.0))
    before = [m.energy() for m in b.members]
    b.step(1)
    for m, (E0, F0, Q), tau in zip(b.members, before, dts):
        E1, F1, _ = m.energy()
        assert abs((E1 - E0) - (tau * Q + 0.5 * tau * (F0 + F1))) <= 1e-12 * abs(E0)
    b.close()


def test_member_rules():
    from paper_1912_03744_gb300 import HeatBatch
    from paper_1912_03744_gb300.heat import HeatError
    probs = [ENSEMBLE[0], ENSEMBLE[1]]
    b = HeatBatch(probs, [1.0, 1.0], precision="fp32")
    m = b.members[0]
    with pytest.raises(HeatError):
        m.sweep(0)
    with pytest.raises(HeatError):
        m.set_dt(2.0)
    m.close()  # a member view cannot destroy its context
    b.step(2)
    b.sync()
    assert np.isfinite(b.members[0].field()).all()
    b.close()
    big = H.homogeneous_cylinder(1025, 8, R=1.0, Z=1.0, k=1.0, C=1e6, bc=(0, 0, 0, 1), T_bc=(0, 0, 0, 300.0),
                                 T_init=300.0, q=0.0)
    with pytest.raises(HeatError):
        HeatBatch([probs[0], big], [1.0, 1.0], precision="fp32")


def test_batch_set_dt():
    """Created with dt = 1 s, switched to 50 x each member's explicit limit."""
    from paper_1912_03744_gb300 import HeatBatch
    sel = _pick(ENSEMBLE, 2, seed=6)
    probs = [ENSEMBLE[i] for i in sel]
    ref, dts = _oracle_runs(probs, 9)
    b = HeatBatch(probs, [1.0] * len(probs), precision="fp32")
    for m, d in zip(b.members, dts):
        assert abs(H.DT_FACTOR * m.tau_exp - d) <= 1e-12 * d
    b.set_dt(dts)
    b.step(9)
    for m, To in zip(b.members, ref):
        assert _rel(m.field(), To) <= 1e-5
    b.close()
