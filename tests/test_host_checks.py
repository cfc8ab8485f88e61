"""Host-side argument checks of the C ABI (no GPU: every case here is rejected, or sized,
before the library makes any CUDA call)."""
import ctypes

import pytest

ERR_INVALID, ERR_CAPACITY = -1, -2


@pytest.fixture(scope="module")
def L():
    from paper_2512_04997_gb300 import build, ledds
    build.build()
    return ledds.lib()


def _size(L, d, p):
    n = ctypes.c_size_t(0)
    return L.ledds_workspace_size(ctypes.byref(d), ctypes.byref(p), ctypes.byref(n)), n.value


BAD_PARAMS = [
    dict(tau=0.5), dict(tau=0.2), dict(tau=float("nan")), dict(storage=3), dict(storage=-1),
    dict(voxel=2), dict(subdiv_n=0), dict(subdiv_n=17), dict(law=2), dict(n_sub=0),
    dict(skin=-0.1), dict(dem_h=0.0), dict(dem_h=float("nan")), dict(collision=2),
    dict(collision=-1), dict(force_fp32=2), dict(orient=2), dict(orient=-1), dict(pattern=2),
    dict(pattern=-1), dict(index64=2), dict(psm_route=3), dict(psm_route=-1), dict(ell_screen=2),
    dict(ell_screen=-1),
]


@pytest.mark.parametrize("bad", BAD_PARAMS, ids=[str(b) for b in BAD_PARAMS])
def test_invalid_params_rejected(L, bad):
    from paper_2512_04997_gb300 import ledds
    base = dict(dem_h=2.5)
    base.update(bad)
    p = ledds.make_params(**base)
    d = ledds.make_dims(16, 16, 16, max_particles=4)
    assert _size(L, d, p)[0] == ERR_INVALID


BAD_DIMS = [
    dict(nx=-1, ny=8, nz=8), dict(nx=8, ny=0, nz=8), dict(nx=0, ny=0, nz=0, max_particles=0),
    dict(nx=8, ny=8, nz=8, max_particles=-1), dict(nx=8, ny=8, nz=8, cand_cap=65),
    dict(nx=8, ny=8, nz=8, tile_cap=65), dict(nx=2048, ny=1024, nz=1024),
    dict(nx=0, ny=0, nz=0, max_particles=4, box_lo=(0, 0, 0), box_hi=(1, 0, 1)),
]


@pytest.mark.parametrize("bad", BAD_DIMS, ids=[str(b) for b in BAD_DIMS])
def test_invalid_dims_rejected(L, bad):
    from paper_2512_04997_gb300 import ledds
    p = ledds.make_params(dem_h=2.5)
    d = ledds.make_dims(**bad)
    assert _size(L, d, p)[0] == ERR_INVALID


def test_workspace_grows_with_the_problem(L):
    from paper_2512_04997_gb300 import ledds
    p = ledds.make_params(dem_h=2.5)
    rc, a = _size(L, ledds.make_dims(32, 32, 32, max_particles=10), p)
    rc2, b = _size(L, ledds.make_dims(64, 32, 32, max_particles=10), p)
    rc3, c = _size(L, ledds.make_dims(32, 32, 32, max_particles=10), ledds.make_params(dem_h=2.5, storage=1))
    assert rc == rc2 == rc3 == 0
    assert b - a >= 2 * 19 * 32 ** 3 * 4      # two FP32 population buffers of the extra cells
    assert a - c >= 2 * 19 * 32 ** 3 * 2      # FP16 storage halves the population bytes
    rc4, e = _size(L, ledds.make_dims(32, 32, 32, max_particles=10), ledds.make_params(dem_h=2.5, pattern="aa"))
    assert rc4 == 0 and a - e >= 19 * 32 ** 3 * 4   # the AA pattern keeps one population array


def test_large_lattice_sizes(L):
    """Node indices are 32-bit: 1024^3 nodes (19 N > 2^31 population elements, 64-bit
    offsets in the kernel) are accepted and sized, 2^31 nodes are not; one population
    array (AA) halves the population bytes."""
    from paper_2512_04997_gb300 import ledds
    p = ledds.make_params(dem_h=2.5)
    d = ledds.make_dims(1024, 1024, 1024, max_particles=0)
    rc, n_ab = _size(L, d, p)
    assert rc == 0 and n_ab >= 2 * 19 * 1024 ** 3 * 4
    rc, n_aa = _size(L, d, ledds.make_params(dem_h=2.5, pattern="aa", storage="f16"))
    assert rc == 0 and n_aa < n_ab / 3.9
    assert _size(L, ledds.make_dims(2048, 1024, 1024), p)[0] == ERR_INVALID


def _batch_size(L, dims, params):
    from paper_2512_04997_gb300 import ledds
    n = len(dims)
    D = (ledds.ledds_dims * n)(*dims)
    P = (ledds.ledds_params * n)(*params)
    out = ctypes.c_size_t(0)
    return L.ledds_batch_workspace_size(n, D, P, ctypes.byref(out)), out.value


def test_batch_workspace_rules(L):
    from paper_2512_04997_gb300 import ledds
    p16 = ledds.make_params(dem_h=8.0, storage=1)
    p32 = ledds.make_params(dem_h=8.0, storage=0)
    d1 = ledds.make_dims(24, 40, 32, periodic=(1, 1, 0), max_particles=8)
    d2 = ledds.make_dims(96, 24, 64, periodic=(0, 0, 0), max_particles=64)
    rc, total = _batch_size(L, [d1, d2], [p16, p16])
    assert rc == 0
    s1 = _size(L, d1, p16)[1]
    s2 = _size(L, d2, p16)[1]
    assert total >= s1 + s2
    assert _batch_size(L, [d1, d2], [p16, p32])[0] == ERR_INVALID            # mixed storage
    trt = ledds.make_params(dem_h=8.0, storage=1, collision="trt")
    assert _batch_size(L, [d1, d2], [p16, trt])[0] == ERR_INVALID            # mixed collision
    assert _batch_size(L, [d1, d2], [trt, trt])[0] == 0
    aa = ledds.make_params(dem_h=8.0, storage=1, pattern="aa")
    assert _batch_size(L, [d1, d2], [aa, aa])[0] == ERR_INVALID              # members use two lattices
    no_lattice = ledds.make_dims(0, 0, 0, max_particles=8, box_lo=(0, 0, 0), box_hi=(20, 20, 20))
    assert _batch_size(L, [d1, no_lattice], [p16, p16])[0] == ERR_INVALID    # member without a lattice
    big = ledds.make_dims(32, 32, 32, max_particles=4097)
    assert _batch_size(L, [big], [p16])[0] == ERR_INVALID                    # direct search limit
    out = ctypes.c_size_t(0)
    assert L.ledds_batch_workspace_size(0, None, None, ctypes.byref(out)) == ERR_INVALID


def test_noalloc_cell_list_host_checks(L):
    """Oversized and invalid requests are refused before the scratch is touched."""
    lo = (ctypes.c_double * 3)(0.0, 0.0, 0.0)
    hi = (ctypes.c_double * 3)(100.0, 100.0, 100.0)
    gn = (ctypes.c_int * 3)()
    fake = ctypes.c_void_p(0x1000)   # never dereferenced: every case returns on the host
    # 100/0.3 = 333 cells per axis: 3.7e7 cells > 262144
    assert L.ledds_cell_list_noalloc(fake, 10, lo, hi, ctypes.c_double(0.3), fake, fake, gn, None) == ERR_CAPACITY
    assert list(gn) == [333, 333, 333]
    assert L.ledds_cell_list_noalloc(fake, 262145, lo, hi, ctypes.c_double(10.0), fake, fake, gn, None) == ERR_CAPACITY
    assert L.ledds_cell_list_noalloc(None, 10, lo, hi, ctypes.c_double(10.0), fake, fake, gn, None) == ERR_INVALID
    assert L.ledds_cell_list_noalloc(fake, 10, lo, hi, ctypes.c_double(0.0), fake, fake, gn, None) == ERR_INVALID
    assert L.ledds_cell_list_noalloc(fake, -1, lo, hi, ctypes.c_double(1.0), fake, fake, gn, None) == ERR_INVALID
    bad_hi = (ctypes.c_double * 3)(100.0, 0.0, 100.0)
    assert L.ledds_cell_list_noalloc(fake, 10, lo, bad_hi, ctypes.c_double(1.0), fake, fake, gn, None) == ERR_INVALID
    # no particles: nothing to do, no device work
    assert L.ledds_cell_list_noalloc(None, 0, lo, hi, ctypes.c_double(10.0), None, None, gn, None) == 0
    assert list(gn) == [10, 10, 10]
