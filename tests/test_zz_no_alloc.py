"""The allocation-free cell-list entry point (ledds_cell_list_noalloc) against the cell
list a simulation builds.

Some callers cannot allocate device memory (a pool owns the whole device, or the call
sits on a path where an allocation must not happen); this entry point serves them with
scratch that lives inside the library. This file is collected last so that a run that
stops at the first failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest

from paper_2512_04997_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _call(lib, torch, pos_dev, n, lo, hi, h, stream):
    keys = torch.full((max(n, 1),), -1, dtype=torch.int32, device=pos_dev.device)
    ids = torch.full((max(n, 1),), -1, dtype=torch.int32, device=pos_dev.device)
    g = (C.c_int * 3)()
    rc = lib.ledds_cell_list_noalloc(pos_dev.data_ptr(), n, (C.c_double * 3)(*lo),
                                     (C.c_double * 3)(*hi), h, keys.data_ptr(), ids.data_ptr(), g,
                                     C.c_void_p(stream.cuda_stream))
    torch.cuda.synchronize()
    return rc, keys[:n].cpu().numpy().view(np.uint32), ids[:n].cpu().numpy(), tuple(g)


def test_cell_list_without_allocation_matches_simulation(torch_cuda):
    torch = torch_cuda
    from paper_2512_04997_gb300 import ledds
    lib = ledds.lib()
    stream = torch.cuda.current_stream()
    w = W.granular_box(n_particles=20000, box=(60.0, 60.0, 100.0), seed_index=7)
    h = w.params["dem_h"]
    # reference: the cell list a simulation rebuilds at the start of its first step
    sim = ledds.from_workload(w)
    sim.step(1)
    keys_ref, ids_ref, gn_ref = sim.cell_keys()
    pos = torch.tensor(np.ascontiguousarray(w.pos.T), dtype=torch.float64, device="cuda")
    # two calls in a row: the second reuses the scratch left by the first
    for _ in range(2):
        rc, keys, ids, gn = _call(lib, torch, pos, w.n, w.box_lo, w.box_hi, h, stream)
        assert rc == 0
        assert gn == gn_ref
        assert np.array_equal(keys, keys_ref)
        assert np.array_equal(ids, ids_ref)
    # a different input between calls must not see stale counts
    half = w.n // 2
    pos_half = torch.tensor(np.ascontiguousarray(w.pos[:half].T), dtype=torch.float64, device="cuda")
    rc, keys_h, ids_h, _ = _call(lib, torch, pos_half, half, w.box_lo, w.box_hi, h, stream)
    assert rc == 0
    assert np.array_equal(keys_h, keys_ref[:half])
    assert np.array_equal(ids_h, np.lexsort((np.arange(half), keys_ref[:half])))


def test_cell_list_without_allocation_rejects_oversize(torch_cuda):
    torch = torch_cuda
    from paper_2512_04997_gb300 import ledds
    lib = ledds.lib()
    stream = torch.cuda.current_stream()
    pos = torch.zeros(3, dtype=torch.float64, device="cuda")
    too_many = (1 << 18) + 1
    rc, _, _, _ = _call(lib, torch, pos, too_many, (0, 0, 0), (10, 10, 10), 1.0, stream)
    assert rc == -2     # LEDDS_ERR_CAPACITY, before any device work
    rc, _, _, _ = _call(lib, torch, pos, 1, (0, 0, 0), (100, 100, 100), 1.0, stream)
    assert rc == -2     # 10^6 grid cells exceed the 262144 limit


@pytest.mark.parametrize("n", [32768, 1 << 18])
def test_cell_list_without_allocation_one_cell_and_crowded_cells(torch_cuda, n):
    """Degenerate grids, each cell ordered in bounded time: h larger than the box (one
    cell holds every particle), and a fine grid where non-finite positions all land in
    cell 0 beside ordinary cells; (key, id) order against numpy's lexsort."""
    torch = torch_cuda
    from paper_2512_04997_gb300 import ledds
    lib = ledds.lib()
    stream = torch.cuda.current_stream()
    g = np.random.default_rng(41)
    p = g.uniform(0.0, 10.0, (n, 3))
    pos = torch.tensor(np.ascontiguousarray(p.T), dtype=torch.float64, device="cuda")
    rc, keys, ids, gn = _call(lib, torch, pos, n, (0, 0, 0), (10, 10, 10), 20.0, stream)
    assert rc == 0 and gn == (1, 1, 1)
    assert not keys.any() and np.array_equal(ids, np.arange(n))
    p[g.random(n) < 0.3] = np.nan
    pos = torch.tensor(np.ascontiguousarray(p.T), dtype=torch.float64, device="cuda")
    for _ in range(2):
        rc, keys, ids, gn = _call(lib, torch, pos, n, (0, 0, 0), (10, 10, 10), 0.5, stream)
        assert rc == 0 and gn == (20, 20, 20)
        c = np.where(np.isfinite(p), np.floor(p / 0.5), 0.0).clip(0, 19).astype(np.int64)
        c[~np.isfinite(p).all(axis=1)] = 0
        k = c[:, 0] + 20 * (c[:, 1] + 20 * c[:, 2])
        assert np.array_equal(keys.astype(np.int64), k)
        assert np.array_equal(ids, np.lexsort((np.arange(n), k)))
