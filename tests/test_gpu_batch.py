"""The batched persistent step (ledds_batch_*) against independent simulations and the
oracle, on an uneven ensemble (lattices 24..96 per edge, 1..64 spheres, settling and
sheared members)."""
import numpy as np
import pytest

from paper_2512_04997_gb300 import workloads as W

from _helpers import gpu_from_workload, normwise, oracle_from_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_batch_members_match_independent_runs():
    from paper_2512_04997_gb300 import ledds
    ws = W.batched_ensemble(nsim=8, seed_index=55, storage="f32")
    b = ledds.batch_from_workloads(ws)
    b.step(1)
    b.step(24)     # 1- and 2-step graphs, both parities
    for w, m in zip(ws, b.members):
        s = gpu_from_workload(w)
        s.step(25)
        _, u_b = m.fields()
        _, u_s = s.fields()
        assert normwise(u_b.cpu().numpy(), u_s.cpu().numpy()) < 1e-6
        if w.n:
            # FP32 contact arithmetic: hydrodynamic sums that differ in the last FP64 bit
            # (atomic order) may round to forces one FP32 ulp apart
            pb, vb, _, _ = m.particles()
            ps, vs, _, _ = s.particles()
            assert np.abs(pb - ps).max() < 1e-6
            assert normwise(vb, vs) < 1e-5
        st = m.status()
        assert st["rc"] == 0, st
    # members cannot be stepped on their own
    rc = ledds.lib().ledds_step(b.members[0].h, 1)
    assert rc == -6


def test_batch_member_matches_oracle(oracle):
    from paper_2512_04997_gb300 import ledds
    ws = W.batched_ensemble(nsim=4, seed_index=56, storage="f32")
    b = ledds.batch_from_workloads(ws)
    b.step(30)
    for k in (0, 1):     # one settling and one sheared member
        o = oracle_from_workload(oracle, ws[k])
        o.step(30)
        _, u_o = o.moments()
        _, u_b = b.members[k].fields()
        assert normwise(u_b.cpu().numpy(), u_o) < 1e-5
        if ws[k].n:
            po, vo, _, _ = o.particles()
            pb, vb, _, _ = b.members[k].particles()
            assert normwise(vb, vo) < 1e-5


def test_batch_fp16_storage_error():
    """FP16-offset storage in the batch stays within 2e-3 of the FP32 run on the fields."""
    from paper_2512_04997_gb300 import ledds
    ws = W.batched_ensemble(nsim=6, seed_index=57, storage="f16")
    b16 = ledds.batch_from_workloads(ws)
    b32 = ledds.batch_from_workloads(ws, storage="f32")
    b16.step(100)
    b32.step(100)
    for m16, m32 in zip(b16.members, b32.members):
        _, u16 = m16.fields()
        _, u32 = m32.fields()
        assert normwise(u16.cpu().numpy(), u32.cpu().numpy()) < 2e-3


def test_batch_autotune_keeps_the_step():
    """The autotuner's trial steps are ordinary steps: after it (and more steps), every
    member still matches the same simulation stepped on its own as often."""
    from paper_2512_04997_gb300 import ledds
    ws = W.batched_ensemble(nsim=6, seed_index=58, storage="f32")
    b = ledds.batch_from_workloads(ws)
    choice = b.autotune(steps_per_trial=2)
    cfg = b.config()
    assert 0 <= choice < 3 * cfg["ctas_per_sm"] * 2 + 6 and cfg["tile_depth"] in (8, 16, 32)
    b.step(3)
    steps = b.members[0].status()["steps"]
    assert steps >= 4 + 3
    for w, m in zip(ws, b.members):
        assert m.status()["steps"] == steps
        s = gpu_from_workload(w)
        s.step(steps)
        _, u_b = m.fields()
        _, u_s = s.fields()
        assert normwise(u_b.cpu().numpy(), u_s.cpu().numpy()) < 1e-6
        if w.n:
            pb, _, _, _ = m.particles()
            ps, _, _, _ = s.particles()
            assert np.abs(pb - ps).max() < 1e-6


@pytest.mark.parametrize("tile_depth", [8, 16, 32])
def test_batch_tile_depths_match_independent_runs(tile_depth):
    """Every tile shape the autotuner can choose (32 x 8 x depth, with either work order)
    gives each member the results of the same simulation stepped on its own. The tiles'
    FP32 partial sums group a particle's node forces differently for each depth, so the
    forces differ in the last bits and the runs part at the rounding level (fields within
    5e-6 after 13 steps)."""
    from paper_2512_04997_gb300 import ledds
    ws = W.batched_ensemble(nsim=6, seed_index=59, storage="f32")
    b = ledds.batch_from_workloads(ws)
    b.configure(tile_depth=tile_depth, order=tile_depth // 16 % 2)
    assert b.config()["tile_depth"] == tile_depth
    b.step(13)
    for w, m in zip(ws, b.members):
        s = gpu_from_workload(w)
        s.step(13)
        _, u_b = m.fields()
        _, u_s = s.fields()
        assert normwise(u_b.cpu().numpy(), u_s.cpu().numpy()) < 5e-6
        if w.n:
            pb, vb, _, _ = m.particles()
            ps, vs, _, _ = s.particles()
            assert np.abs(pb - ps).max() < 1e-6
            assert normwise(vb, vs) < 1e-5
        assert m.status()["rc"] == 0


def test_batch_autotune_choice_is_cached_by_shape():
    """A second batch of the same shape takes the first one's choice without trial steps."""
    from paper_2512_04997_gb300 import ledds
    ws = W.batched_ensemble(nsim=4, seed_index=60, storage="f16")
    a = ledds.batch_from_workloads(ws)
    c1 = a.autotune(steps_per_trial=1)
    b = ledds.batch_from_workloads(ws)
    c2 = b.autotune(steps_per_trial=1)
    assert c1 == c2 and b.config() == a.config()
    assert b.members[0].status()["steps"] == 0
