"""C ABI checks that need no GPU: the library loads, exports every function
``include/rdcnn.h`` declares, and rejects bad arguments on the host before any
CUDA work (no compute calls are made here)."""
import ctypes
import math
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rdcnn.h")


def header_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rdcnn_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2102_10340_gb300 import _lib, build_library

    build_library()
    return _lib.load()


@pytest.fixture(scope="module")
def L():
    from paper_2102_10340_gb300 import _lib

    return _lib


def test_header_declares_expected_calls():
    names = header_functions()
    for must in ("rdcnn_create", "rdcnn_init", "rdcnn_run", "rdcnn_batch_run", "rdcnn_adjoint",
                 "rdcnn_get_state", "rdcnn_destroy"):
        assert must in names


def test_every_header_symbol_is_exported(lib):
    from paper_2102_10340_gb300.build import LIB

    out = subprocess.run(["nm", "-D", "--defined-only", LIB], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (rdcnn_\w+)", out))
    missing = [n for n in header_functions() if n not in exported]
    assert not missing, missing
    for n in header_functions():
        assert hasattr(lib, n)


def test_binding_covers_header_exactly(L):
    assert sorted(name for name, _, _ in L.SIGNATURES) == header_functions()


def test_struct_layouts(L):
    assert ctypes.sizeof(L.Params) == 7 * 8
    assert ctypes.sizeof(L.Tune) == 8
    assert ctypes.sizeof(L.Instance) == 2 * 8 + 7 * 8 + 4 * 8


def _create(lib, L, nn=8, nm=8, params=None, boundary=0, dtype=0, reaction=0):
    h = ctypes.c_void_p()
    p = L.params_struct(params or {"dt": 0.1, "a": -0.3, "b": 1.3, "eps": -0.1, "c": 1.0, "Du": 0.06, "Dv": 1.0})
    rc = lib.rdcnn_create(ctypes.byref(h), nn, nm, ctypes.byref(p), boundary, dtype, reaction)
    return rc, h


def test_create_validation(lib, L):
    assert _create(lib, L, nn=0)[0] == L.EINVAL
    assert _create(lib, L, nm=-3)[0] == L.EINVAL
    assert _create(lib, L, boundary=2)[0] == L.EINVAL
    assert _create(lib, L, nn=1 << 30, nm=4)[0] == L.EINVAL
    assert _create(lib, L, nn=1 << 21, nm=1 << 20)[0] == L.EINVAL  # 2^41 cells
    rc, h = _create(lib, L, nn=(1 << 30) - 1, nm=4)
    assert rc == L.OK
    lib.rdcnn_destroy(h)
    assert _create(lib, L, dtype=7)[0] == L.EINVAL
    assert _create(lib, L, reaction=5)[0] == L.EINVAL
    bad = {"dt": 0.1, "a": math.nan, "b": 1.3, "eps": -0.1, "c": 1.0, "Du": 0.06, "Dv": 1.0}
    assert _create(lib, L, params=bad)[0] == L.ENONFINITE
    neg = {"dt": 0.1, "a": -0.3, "b": 1.3, "eps": -0.1, "c": 1.0, "Du": -0.06, "Dv": 1.0}
    assert _create(lib, L, params=neg)[0] == L.EINVAL
    assert "diffusion" in L.last_error()
    rc, h = _create(lib, L)
    assert rc == L.OK and h.value
    lib.rdcnn_destroy(h)
    lib.rdcnn_destroy(None)


def test_cfl_warning_still_creates(lib, L):
    hot = {"dt": 0.3, "a": -0.3, "b": 1.3, "eps": -0.1, "c": 1.0, "Du": 0.06, "Dv": 1.0}
    rc, h = _create(lib, L, params=hot)
    assert rc == L.WARN_CFL and h.value
    lib.rdcnn_destroy(h)


def test_unbound_handle_and_workspace(lib, L):
    rc, h = _create(lib, L, nn=6, nm=10, dtype=L.F64)
    n = ctypes.c_size_t()
    assert lib.rdcnn_workspace_bytes(h, ctypes.byref(n)) == L.OK
    plane = 6 * 10 * 8
    assert n.value == ((plane + 255) // 256) * 256 + plane  # second plane 256-byte aligned
    assert lib.rdcnn_run(h, 5, 0, 0) == L.ESTATE
    assert lib.rdcnn_get_state(h, None, None, 0) == L.ESTATE
    assert lib.rdcnn_init(h, None, 1.0, 1) == L.ESTATE
    assert lib.rdcnn_bind(h, None, None, None, 0, None) == L.EINVAL
    assert lib.rdcnn_bind(h, 16, 32, 48, 10, None) == L.ESPACE
    t = L.Tune(9, 0)
    assert lib.rdcnn_set_tune(h, ctypes.byref(t)) == L.EINVAL  # F64 allows k <= 4
    t = L.Tune(3, 16)
    assert lib.rdcnn_set_tune(h, ctypes.byref(t)) == L.OK
    assert lib.rdcnn_set_tune(h, None) == L.OK
    a = ctypes.c_size_t()
    assert lib.rdcnn_adjoint_workspace_bytes(h, 100, 0, ctypes.byref(a)) == L.OK
    assert a.value >= (10 + 10 + 4) * 2 * 6 * 10 * 8 // 2
    lib.rdcnn_destroy(h)


def test_bound_run_rejects_bad_args_before_gpu_work(lib, L):
    rc, h = _create(lib, L, nn=4, nm=6)
    # fake, never-dereferenced addresses: validation must fail before any CUDA call
    assert lib.rdcnn_bind(h, 256, 512, 1024, 256 + 4 * 6 * 4, None) == L.OK
    assert lib.rdcnn_run(h, -1, 0, 0) == L.EINVAL
    assert lib.rdcnn_run(h, 5, 9, 0) == L.EINVAL
    assert lib.rdcnn_run(h, 5, L.VARIANT_TEMPORAL, 0) == L.EINVAL  # NM=6 is not a multiple of 4
    assert "multiple" in L.last_error() or "aligned" in L.last_error()
    assert lib.rdcnn_run(h, 0, 0, 0) == L.OK  # T = 0 is a no-op
    lib.rdcnn_destroy(h)


def test_batch_model_validation(lib, L):
    p = L.params_struct({"dt": 0.1, "a": 0.0, "b": 0.0, "eps": 0.0, "c": 2.0, "Du": -0.5, "Dv": 0.0})
    tab = (L.Instance * 1)()
    tab[0] = L.Instance(8, 8, p, 256, 512, 768, 1024)
    run = lambda dt, rx, bc, ws=1 << 12: lib.rdcnn_batch_run_model(tab, 1, 0, dt, rx, bc, None, 4096, ws, None)
    assert run(L.F32, L.REACTION_CENN, L.BC_ZEROFLUX) == L.OK  # T = 0: validation only
    assert run(L.F32, L.REACTION_CENN, L.BC_PERIODIC) == L.OK
    assert run(L.F32, L.REACTION_FHN, L.BC_ZEROFLUX) == L.EINVAL  # Du < 0 is a diffusion error here
    for dt in (L.F64, L.BF16, L.F16):
        assert run(dt, L.REACTION_CENN, L.BC_ZEROFLUX) == L.OK
    assert run(7, L.REACTION_CENN, L.BC_PERIODIC) == L.EINVAL  # unknown dtype
    assert run(L.F32, L.REACTION_CENN, 2) == L.EINVAL
    assert run(L.F32, 3, L.BC_PERIODIC) == L.EINVAL


def test_batch_validation(lib, L):
    p = L.params_struct({"dt": 0.1, "a": -0.3, "b": 1.3, "eps": -0.1, "c": 1.0, "Du": 0.06, "Dv": 1.0})
    tab = (L.Instance * 2)()
    tab[0] = L.Instance(8, 8, p, 256, 512, 768, 1024)
    tab[1] = L.Instance(8, 6, p, 256, 512, 768, 1024)
    n = ctypes.c_size_t()
    assert lib.rdcnn_batch_workspace_bytes(tab, 2, 0, None, ctypes.byref(n)) == L.OK and n.value > 0
    assert lib.rdcnn_batch_run(tab, 2, 10, 0, 0, None, 4096, n.value, None) == L.EINVAL  # NM=6
    tab[1] = L.Instance(8, 8, p, 256, 0, 768, 1024)
    assert lib.rdcnn_batch_run(tab, 2, 10, 0, 0, None, 4096, n.value, None) == L.EINVAL  # NULL
    tab[1] = L.Instance(8, 8, p, 256, 520, 768, 1024)
    assert lib.rdcnn_batch_run(tab, 2, 10, 0, 0, None, 4096, n.value, None) == L.EINVAL  # misaligned
    # 16-bit planes need 8-byte alignment only (T = 0: validation, no launch)
    assert lib.rdcnn_batch_run(tab, 2, 0, L.BF16, 0, None, 4096, n.value, None) == L.OK
    tab[1] = L.Instance(8, 8, p, 256, 516, 768, 1024)
    assert lib.rdcnn_batch_run(tab, 2, 10, L.F16, 0, None, 4096, n.value, None) == L.EINVAL
    tab[1] = L.Instance(8, 8, p, 256, 512, 768, 1024)
    t = L.Tune(12, 0)
    assert lib.rdcnn_batch_run(tab, 2, 10, 0, 0, ctypes.byref(t), 4096, n.value, None) == L.EINVAL
    assert lib.rdcnn_batch_run(tab, 2, 10, 0, 0, None, 4096, 1, None) == L.ESPACE
    assert lib.rdcnn_batch_run(tab, 0, 10, 0, 0, None, 4096, n.value, None) == L.EINVAL


def test_adjoint_validation(lib, L):
    rc, h = _create(lib, L, nn=4, nm=8)
    g = (ctypes.c_double * 6)()
    assert lib.rdcnn_adjoint(h, 10, 256, 512, 768, 1024, 0, 1280, 1536, g, None, 0) == L.EINVAL
    assert lib.rdcnn_adjoint(h, 10, 256, 512, 768, 1024, 0, 1280, 1540, g, 4096, 1 << 20) == L.EINVAL
    assert lib.rdcnn_adjoint(h, 10, 256, 512, 768, 1024, 0, 1280, 1536, g, 4096, 16) == L.ESPACE
    assert lib.rdcnn_adjoint(h, -2, 256, 512, 768, 1024, 0, 1280, 1536, g, 4096, 1 << 20) == L.EINVAL
    lib.rdcnn_destroy(h)


def test_tape_layout_and_validation(lib, L):
    """Host-side rules of the recorded-forward entry points (no GPU work happens)."""
    rc, h = _create(lib, L, nn=4, nm=8)  # FP32: one plane is 128 bytes, padded to 256
    tb, wb = ctypes.c_size_t(), ctypes.c_size_t()
    assert lib.rdcnn_tape_bytes(h, 100, 0, ctypes.byref(tb), ctypes.byref(wb)) == L.OK
    assert tb.value == 10 * 2 * 256  # ceil(sqrt(100)) = 10 slots of (u, v)
    assert lib.rdcnn_tape_bytes(h, 100, 7, ctypes.byref(tb), ctypes.byref(wb)) == L.OK
    assert tb.value == 7 * 2 * 256  # S = ceil(100 / 7) = 15, ceil(100 / 15) = 7 slots
    assert lib.rdcnn_tape_bytes(h, 100, 100, ctypes.byref(tb), ctypes.byref(wb)) == L.OK
    assert tb.value == 100 * 2 * 256  # every state 0 .. 99
    full_ws = wb.value
    assert lib.rdcnn_tape_bytes(h, 100, 0, ctypes.byref(tb), ctypes.byref(wb)) == L.OK
    assert full_ws < wb.value  # a full tape needs no segment buffers
    a = ctypes.c_size_t()
    assert lib.rdcnn_adjoint_workspace_bytes(h, 100, 0, ctypes.byref(a)) == L.OK
    assert a.value == wb.value + tb.value  # rdcnn_adjoint keeps its checkpoints in the workspace
    assert lib.rdcnn_tape_bytes(h, -1, 0, ctypes.byref(tb), ctypes.byref(wb)) == L.EINVAL
    assert lib.rdcnn_tape_bytes(h, 10, 0, None, ctypes.byref(wb)) == L.EINVAL
    # recording needs a bound handle; the tape must be present, aligned and large enough
    assert lib.rdcnn_run_record(h, 10, 0, 4096, 1 << 20) == L.ESTATE
    g = (ctypes.c_double * 6)()
    assert lib.rdcnn_adjoint_tape(h, 10, 0, None, 0, 256, 512, 768, 1024, g, 4096, 1 << 20) == L.EINVAL
    assert lib.rdcnn_adjoint_tape(h, 10, 0, 4100, 1 << 20, 256, 512, 768, 1024, g, 4096, 1 << 20) == L.EINVAL
    assert lib.rdcnn_adjoint_tape(h, 10, 0, 8192, 16, 256, 512, 768, 1024, g, 4096, 1 << 20) == L.ESPACE
    assert lib.rdcnn_adjoint_tape(h, 10, 0, 8192, 1 << 20, 256, 512, 768, 1024, g, 4096, 16) == L.ESPACE
    assert lib.rdcnn_adjoint_tape(h, -3, 0, 8192, 1 << 20, 256, 512, 768, 1024, g, 4096, 1 << 20) == L.EINVAL
    lib.rdcnn_destroy(h)
    rc, h = _create(lib, L, nn=4, nm=8, dtype=L.BF16)
    assert lib.rdcnn_tape_bytes(h, 10, 0, ctypes.byref(tb), ctypes.byref(wb)) == L.EINVAL
    lib.rdcnn_destroy(h)


def test_version_and_counter(lib):
    assert b"rdcnn" in lib.rdcnn_version()
    assert lib.rdcnn_launch_count() >= 0


def header_enums():
    """Every RDCNN_* enumerator of the header with its value."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    out = {}
    for body in re.findall(r"enum\s*\w*\s*\{(.*?)\}", text, flags=re.S):
        for name, val in re.findall(r"RDCNN_(\w+)\s*=\s*(-?\d+)", body):
            out[name] = int(val)
    return out


def test_binding_constants_match_header(L):
    enums = header_enums()
    for name in ("BC_PERIODIC", "BC_ZEROFLUX", "F32", "F64", "BF16", "F16", "REACTION_FHN", "REACTION_NONE",
                 "REACTION_CENN", "VARIANT_AUTO", "VARIANT_STEP1", "VARIANT_TEMPORAL",
                 "VARIANT_GENERIC", "VARIANT_TEMPORAL2", "VARIANT_TEMPORAL_WIDE"):
        assert getattr(L, name) == enums[name], name


def test_create_accepts_models_and_rejects_bad_enums(lib, L):
    p = L.params_struct({"dt": 0.1, "a": -0.3, "b": 1.3, "eps": -0.1, "c": 1.0, "Du": 0.06, "Dv": 1.0})
    for bc in (L.BC_PERIODIC, L.BC_ZEROFLUX):
        for rx in (L.REACTION_FHN, L.REACTION_NONE, L.REACTION_CENN):
            h = ctypes.c_void_p()
            assert lib.rdcnn_create(ctypes.byref(h), 8, 8, ctypes.byref(p), bc, L.F32, rx) == 0
            lib.rdcnn_destroy(h)
    h = ctypes.c_void_p()
    assert lib.rdcnn_create(ctypes.byref(h), 8, 8, ctypes.byref(p), 2, L.F32, L.REACTION_FHN) == L.EINVAL
    assert lib.rdcnn_create(ctypes.byref(h), 8, 8, ctypes.byref(p), L.BC_PERIODIC, L.F32, 3) == L.EINVAL
    # CeNN feedback arms may be negative; diffusion coefficients may not
    q = L.params_struct({"dt": 0.1, "a": 0.0, "b": 0.0, "eps": 0.0, "c": 2.0, "Du": -0.5, "Dv": 0.0})
    assert lib.rdcnn_create(ctypes.byref(h), 8, 8, ctypes.byref(q), L.BC_ZEROFLUX, L.F32, L.REACTION_CENN) == 0
    lib.rdcnn_destroy(h)
    assert lib.rdcnn_create(ctypes.byref(h), 8, 8, ctypes.byref(q), L.BC_ZEROFLUX, L.F32, L.REACTION_FHN) == L.EINVAL


def test_plan_resolves_without_running(lib, L):
    """rdcnn_plan for the variants whose shape needs no device query (no CUDA work)."""
    h = _create(lib, L, nn=64, nm=64)[1]
    var = ctypes.c_int(L.VARIANT_STEP1)
    tune = L.Tune(0, 0)
    assert lib.rdcnn_plan(h, ctypes.byref(var), ctypes.byref(tune)) == 0
    assert (var.value, tune.k, tune.rows) == (L.VARIANT_STEP1, 1, 2)  # FP32 single step: 2-row strips
    assert lib.rdcnn_set_tune(h, ctypes.byref(L.Tune(0, 16))) == 0
    tune = L.Tune(0, 0)
    assert lib.rdcnn_plan(h, ctypes.byref(var), ctypes.byref(tune)) == 0 and tune.rows == 16
    var = ctypes.c_int(L.VARIANT_GENERIC)
    assert lib.rdcnn_plan(h, ctypes.byref(var), ctypes.byref(tune)) == 0 and (tune.k, tune.rows) == (1, 0)
    var = ctypes.c_int(L.VARIANT_TEMPORAL)
    assert lib.rdcnn_plan(h, ctypes.byref(var), ctypes.byref(L.Tune(9, 0))) == L.EINVAL  # k > 8
    var = ctypes.c_int(17)
    assert lib.rdcnn_plan(h, ctypes.byref(var), ctypes.byref(tune)) == L.EINVAL
    lib.rdcnn_destroy(h)
    h = _create(lib, L, nn=64, nm=64, boundary=L.BC_ZEROFLUX)[1]
    var = ctypes.c_int(L.VARIANT_TEMPORAL2)
    t4 = L.Tune(4, 0)
    assert lib.rdcnn_plan(h, ctypes.byref(var), ctypes.byref(t4)) == 0  # every model, FP32 / FP64
    assert var.value == L.VARIANT_TEMPORAL2 and t4.k == 4 and t4.rows >= 1
    lib.rdcnn_destroy(h)


def test_create_accepts_16bit_storage(lib, L):
    for dt in (L.BF16, L.F16):
        rc, h = _create(lib, L, nn=16, nm=16, dtype=dt)
        assert rc == 0
        nbytes = ctypes.c_size_t()
        assert lib.rdcnn_workspace_bytes(h, ctypes.byref(nbytes)) == 0 and nbytes.value == 512 + 16 * 16 * 2
        var = ctypes.c_int(L.VARIANT_TEMPORAL2)
        assert lib.rdcnn_plan(h, ctypes.byref(var), ctypes.byref(L.Tune(4, 0))) == L.EINVAL
        nbytes = ctypes.c_size_t()
        assert lib.rdcnn_adjoint_workspace_bytes(h, 10, 0, ctypes.byref(nbytes)) == L.EINVAL
        lib.rdcnn_destroy(h)
    assert _create(lib, L, dtype=4)[0] == L.EINVAL


def test_snapshot_summary_and_static_validation(lib, L):
    """Host-side rejections of rdcnn_run_snapshots, rdcnn_batch_summary and rdcnn_run_static
    (fake, never-dereferenced addresses; every case fails before any CUDA work)."""
    p = L.params_struct({"dt": 0.1, "a": -0.3, "b": 1.3, "eps": -0.1, "c": 1.0, "Du": 0.06, "Dv": 1.0})
    assert lib.rdcnn_run_snapshots(None, 10, 2, 256, 512, 1, None, 0) == L.EINVAL
    rc, h = _create(lib, L, nn=4, nm=8)
    assert lib.rdcnn_run_snapshots(h, 10, 2, 256, 512, 1, None, 0) == L.ESTATE  # unbound
    assert lib.rdcnn_bind(h, 256, 512, 1024, 1 << 12, None) == L.OK
    assert lib.rdcnn_run_snapshots(h, 10, 0, 256, 512, 1, None, 0) == L.EINVAL  # every < 1
    assert lib.rdcnn_run_snapshots(h, -1, 2, 256, 512, 1, None, 0) == L.EINVAL
    assert lib.rdcnn_run_snapshots(h, 10, 2, None, 512, 1, None, 0) == L.EINVAL
    assert lib.rdcnn_run_snapshots(h, 10, 2, 256, 512, 0, 4096, 16) == L.ESPACE  # staging too small
    lib.rdcnn_destroy(h)

    tab = (L.Instance * 1)()
    tab[0] = L.Instance(8, 8, p, 256, 512, 0, 0)
    out = (ctypes.c_double * 8)()
    need = ctypes.c_size_t()
    assert lib.rdcnn_summary_workspace_bytes(tab, 0, ctypes.byref(need)) == L.EINVAL
    assert lib.rdcnn_summary_workspace_bytes(tab, 1, ctypes.byref(need)) == L.OK and need.value > 0
    assert lib.rdcnn_batch_summary(tab, 1, 7, 0.05, out, 4096, need.value, None) == L.EINVAL  # dtype
    assert lib.rdcnn_batch_summary(tab, 1, L.F32, 0.05, out, 4096, 8, None) == L.ESPACE
    tab[0] = L.Instance(8, 8, p, 0, 512, 0, 0)
    assert lib.rdcnn_batch_summary(tab, 1, L.F32, 0.05, out, 4096, need.value, None) == L.EINVAL

    assert lib.rdcnn_run_static(0, 8, ctypes.byref(p), L.F32, L.REACTION_FHN, 256, 512, 10, 0, None) == L.EINVAL
    assert lib.rdcnn_run_static(8, 8, ctypes.byref(p), L.BF16, L.REACTION_FHN, 256, 512, 10, 0, None) == L.EINVAL
    assert lib.rdcnn_run_static(8, 8, ctypes.byref(p), L.F32, L.REACTION_CENN, 256, 512, 10, 0, None) == L.EINVAL
    assert lib.rdcnn_run_static(8, 8, ctypes.byref(p), L.F32, L.REACTION_FHN, None, 512, 10, 0, None) == L.EINVAL
    big = L.STATIC_SCRATCH_BYTES // 8 + 1  # one FP32 plane over half the static scratch
    assert lib.rdcnn_run_static(1, big, ctypes.byref(p), L.F32, L.REACTION_FHN, 256, 512, 10, 0, None) == L.EINVAL
    assert lib.rdcnn_run_static(8, 8, ctypes.byref(p), L.F32, L.REACTION_FHN, 256, 512, 10, 9, None) == L.EINVAL
    assert lib.rdcnn_run_static(8, 8, ctypes.byref(p), L.F32, L.REACTION_FHN, 256, 512, 0, 0, None) == L.OK
