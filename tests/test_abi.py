"""The C-ABI library loads without a GPU and exports every function that
include/ccfr.h declares; the header's structs match the binding's layout."""
import ctypes as C
import re
from pathlib import Path

from paper_2607_26901_b300 import build_lib, ccfr

ROOT = Path(__file__).resolve().parent.parent


def declared_functions():
    src = (ROOT / "include" / "ccfr.h").read_text()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ccfr_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    build_lib.build()
    lib = C.CDLL(str(build_lib.LIB))
    names = declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(ccfr.exported_symbols())


def test_status_strings_without_gpu():
    lib = ccfr.lib()
    assert lib.ccfr_status_string(0) == b"ok"
    assert lib.ccfr_status_string(2) == b"output capacity exceeded"


def test_struct_layouts():
    # ccfr_params: 7 floats, 3 ints, 3 floats, 3 floats, float, unsigned
    assert C.sizeof(ccfr.Params) == 4 * 23
    assert C.sizeof(ccfr.Mesh) == 3 * 4 + 4 + 3 * 8
    assert C.sizeof(ccfr.Stats) == 34 * 8 + 8 + 3 * 8
    assert C.sizeof(ccfr.MeshExt) == 40 + 4 + 4 + 8 + 8 + 4 + 4 + 8 + 4 + 4


def test_host_checks_reject_bad_arguments_without_gpu():
    """Argument validation happens before any device work."""
    lib = ccfr.lib()
    h = C.c_void_p()
    # null mesh / params
    assert lib.ccfr_create(None, None, None, C.byref(h)) == 1
    p = ccfr.Params()
    m = ccfr.Mesh(4, 0, 0, None, None, None)
    p.r, p.xi, p.pad, p.eps_dep, p.dt, p.solver_iters = 1e-3, 1e-3, 1.5e-3, 1e-6, 1 / 60, 1
    p.plane_capacity = 33                      # not a multiple of 32
    assert lib.ccfr_create(C.byref(m), C.byref(p), None, C.byref(h)) == 1
    p.plane_capacity = 64
    for bad in (-1, 1025):                     # candidate-pair buffer capacity out of range
        p.pair_capacity = bad
        assert lib.ccfr_create(C.byref(m), C.byref(p), None, C.byref(h)) == 1
    p.pair_capacity = 0
    assert lib.ccfr_destroy(None) == 1
    assert lib.ccfr_step(None, None, None, None) == 1
    # mixed scenes: the extension is checked before any copy to or from the device
    p.plane_capacity = 64
    assert lib.ccfr_create_ext(None, C.byref(p), None, C.byref(h)) == 1
    me = ccfr.MeshExt(m, -1, None, None, 0, None, 0.0)          # negative link count
    assert lib.ccfr_create_ext(C.byref(me), C.byref(p), None, C.byref(h)) == 1
    me = ccfr.MeshExt(m, 2, None, None, 0, None, 0.0)           # links announced, none given
    assert lib.ccfr_create_ext(C.byref(me), C.byref(p), None, C.byref(h)) == 1
    me = ccfr.MeshExt(m, 0, None, None, 3, None, 0.0)           # tetrahedra announced, none given
    assert lib.ccfr_create_ext(C.byref(me), C.byref(p), None, C.byref(h)) == 1
    me = ccfr.MeshExt(m, 0, None, None, 0, None, -1.0)          # negative volume compliance
    assert lib.ccfr_create_ext(C.byref(me), C.byref(p), None, C.byref(h)) == 1


def test_host_checks_of_static_projection_batch_and_server_without_gpu():
    """The no-allocation projection, the batched context and the server
    reject bad arguments on the host, before any CUDA call; the byte estimate
    is host arithmetic."""
    from paper_2607_26901_b300 import scenes as S
    lib = ccfr.lib()
    p = ccfr.make_params(S.default_params(2e-3, 1e-3))
    a = C.c_void_p(256)                      # aligned stand-ins: never dereferenced on these paths
    # ccfr_project_static: pointers, size limit, alignment, capacity, pass budget
    assert lib.ccfr_project_static(None, a, a, a, None, 4, 32, C.byref(p), None, None) == 1
    assert lib.ccfr_project_static(a, a, a, a, None, (1 << 18) + 1, 32, C.byref(p), None, None) == 1
    assert lib.ccfr_project_static(a, C.c_void_p(264), a, a, None, 4, 32, C.byref(p), None, None) == 1
    assert lib.ccfr_project_static(a, a, None, a, None, 4, 32, C.byref(p), None, None) == 1
    assert lib.ccfr_project_static(a, a, a, a, None, 4, 0, C.byref(p), None, None) == 1
    q = ccfr.make_params(S.default_params(2e-3, 1e-3))
    q.max_passes = 65
    assert lib.ccfr_project_static(a, a, a, a, None, 4, 32, C.byref(q), None, None) == 1
    assert lib.ccfr_project_static(a, a, a, a, None, 0, 32, C.byref(p), None, None) == 0   # nothing to do
    # ccfr_create_batch: scene count and parameter blocks
    h = C.c_void_p()
    m = ccfr.Mesh(4, 0, 0, None, None, None)
    assert lib.ccfr_create_batch(None, None, 1, None, C.byref(h)) == 1
    assert lib.ccfr_create_batch(C.byref(m), C.byref(p), 0, None, C.byref(h)) == 1
    assert lib.ccfr_create_batch(C.byref(m), C.byref(p), 2049, None, C.byref(h)) == 1
    bad = ccfr.make_params(S.default_params(2e-3, 1e-3))
    bad.plane_capacity = 33
    assert lib.ccfr_create_batch(C.byref(m), C.byref(bad), 1, None, C.byref(h)) == 1
    # server: slots, timeout, null handles
    sv = C.c_void_p()
    assert lib.ccfr_server_create(1 << 30, 0, 1.0, C.byref(sv)) == 1
    assert lib.ccfr_server_create(1 << 30, 65, 1.0, C.byref(sv)) == 1
    assert lib.ccfr_server_create(1 << 30, 4, 0.0, C.byref(sv)) == 1
    sid, rid = C.c_int(), C.c_long()
    assert lib.ccfr_server_add_scene(None, 4, 0, 0, None, None, a, a, C.byref(p), C.byref(sid)) == 1
    assert lib.ccfr_server_submit(None, 0, 0.0, C.byref(rid)) == 1
    assert lib.ccfr_server_start(None) == 1
    assert lib.ccfr_server_destroy(None) == 1
    # byte estimate: grows with the vertices and the plane capacity
    b = [C.c_size_t() for _ in range(3)]
    assert lib.ccfr_estimate_bytes(1000, 2900, 1900, 64, C.byref(b[0])) == 0
    assert lib.ccfr_estimate_bytes(2000, 5900, 3900, 64, C.byref(b[1])) == 0
    assert lib.ccfr_estimate_bytes(1000, 2900, 1900, 128, C.byref(b[2])) == 0
    assert 0 < b[0].value < b[1].value and b[0].value < b[2].value
    # the planes alone: 16 bytes per plane slot
    assert b[2].value - b[0].value >= 1000 * 64 * 16
    assert lib.ccfr_estimate_bytes(-1, 0, 0, 64, C.byref(b[0])) == 1
    assert lib.ccfr_estimate_bytes(10, 0, 0, 0, C.byref(b[0])) == 1
