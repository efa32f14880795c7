"""Error handling that is decided on the host, before any device work:
invalid graphs and corrupt network files (no GPU needed)."""
import numpy as np
import pytest

from paper_2505_08491_gb300 import _lib as L


@pytest.fixture(scope="module")
def lib():
    from paper_2505_08491_gb300 import build
    return L.load(build.build())


def _assemble(lib, xyz, edges, N=8, elems=2, R=0.02, beta=1.0):
    import ctypes as C
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    edges = np.ascontiguousarray(edges, dtype=np.int32)
    g = L.MdGraph(len(xyz), xyz.ctypes.data_as(C.POINTER(C.c_double)), len(edges),
                  edges.ctypes.data_as(C.POINTER(C.c_int)), elems)
    h = C.c_void_p()
    return lib.md_assemble(N, C.byref(g), R, beta, None, C.byref(h))


def test_cyclic_graph_rejected(lib):
    xyz = [[0.3, 0.3, 0.3], [0.6, 0.3, 0.3], [0.45, 0.6, 0.3]]
    assert _assemble(lib, xyz, [[0, 1], [1, 2], [2, 0]]) == -1
    assert b"cycle" in lib.md_last_error()


def test_bad_inputs_rejected(lib):
    xyz = [[0.3, 0.3, 0.3], [0.6, 0.3, 0.3]]
    assert _assemble(lib, xyz, [[0, 5]]) == -1                       # node id out of range
    assert _assemble(lib, [[0.3, 0.3, 0.3], [1.2, 0.3, 0.3]], [[0, 1]]) == -1  # outside the cube
    assert _assemble(lib, xyz, [[0, 1]], N=1) == -1                  # grid too small
    assert _assemble(lib, xyz, [[0, 1]], R=-1.0) == -1
    assert _assemble(lib, xyz, [[0, 1], [1, 0]]) == -1               # repeated edge


def test_corrupt_network_file(lib, tmp_path):
    import ctypes as C
    n = L.MD_CNN_NPARAMS
    vals = np.random.default_rng(0).standard_normal(n).astype(np.float32)
    h = 1469598103934665603
    for byte in vals.tobytes():
        h = ((h ^ byte) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    good = b"MDCNN001" + np.int64(n).tobytes() + vals.tobytes() + np.uint64(h).tobytes()
    bad = bytearray(good)
    bad[100] ^= 0xFF
    p = tmp_path / "bad.bin"
    p.write_bytes(bytes(bad))
    out = C.c_void_p()
    assert lib.md_cnn_load(str(p).encode(), C.byref(out)) == -6
    assert b"checksum" in lib.md_last_error()
    p.write_bytes(good[:1000])
    assert lib.md_cnn_load(str(p).encode(), C.byref(out)) == -6
    assert lib.md_cnn_load(str(tmp_path / "missing.bin").encode(), C.byref(out)) == -6
    # the reader in the package agrees with the file format
    from paper_2505_08491_gb300.weights import read_network_file
    q = tmp_path / "good.bin"
    q.write_bytes(good)
    assert np.array_equal(read_network_file(str(q)), vals)


def test_smoothing_entries_reject_null_handles(lib):
    assert lib.md_batch_set_smoothing(None, 1, 0.5) == -1
    assert lib.md_precondition_smoothed(None, None, 0, 1, 0.5, None, None, None) == -1
    assert b"md_precondition_smoothed" in lib.md_last_error()


def test_inner_entries_reject_null_handles(lib):
    assert lib.md_batch_set_inner_iters(None, 1) == -1
    assert lib.md_precondition_inner(None, None, 0, 1, None, None, None) == -1
    assert b"md_precondition_inner" in lib.md_last_error()
