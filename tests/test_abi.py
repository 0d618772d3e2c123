"""The C-ABI library loads and exports every symbol include/dags.h declares
(no GPU needed: nothing here launches work)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "dags.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?\w+\s*\**\s*(\w+)\s*\([^;]*\)\s*;", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2602_21644_gb300 import build
    return ctypes.CDLL(build.build())


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("splat_forward", "splat_backward", "pose_step", "dags_create", "dags_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"libdags.so does not export {name}"


def test_binding_covers_every_declared_symbol():
    from paper_2602_21644_gb300 import dags
    assert sorted(dags.EXPORTS) == declared_functions()


def test_host_only_helpers(lib):
    lib.dags_status_string.restype = ctypes.c_char_p
    assert lib.dags_status_string(0) == b"ok"
    assert b"capacity" in lib.dags_status_string(-3)
    assert lib.dags_abi_version() == 1
    from paper_2602_21644_gb300 import dags
    dags.load()
    rc = dags.default_raster_cfg()
    assert rc.tile == 16 and abs(rc.alpha_min - 1 / 255) < 1e-9 and abs(rc.alpha_max - 0.99) < 1e-7
    lc = dags.default_loss_cfg()
    assert abs(lc.lambda_pho - 0.9) < 1e-7 and abs(lc.lambda_depth - 0.1) < 1e-7   # Sec. V-A(c)
    sc = dags.default_sched_cfg()
    assert (sc.w_u, sc.w_r, sc.theta, sc.e_ref, sc.n_max) == (0.5, 0.5, 0.35, 0.05, 10)
    lm = dags.default_lm_cfg()
    assert (lm.mu0, lm.delta, lm.down, lm.up) == (1e-2, 0.01, 0.1, 10.0)
    ec = dags.default_edge_cfg()
    assert abs(ec.edge_rel - 0.05) < 1e-7 and abs(ec.huber - 0.05) < 1e-7 and ec.literal == 0
    h = ctypes.c_void_p()
    lib.dags_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                ctypes.c_int32, ctypes.c_int64]
    assert lib.dags_create(ctypes.byref(h), -1, 16, 16, 1, 0) == -1        # rejected before any CUDA call
    assert lib.dags_create(ctypes.byref(h), 10, 16, 16, 0, 0) == -1
    assert h.value is None


def test_oracle_builds_with_gcc():
    import oracle
    assert os.path.exists(oracle.build())


def _zero_args(fn):
    args = []
    for t in fn.argtypes:
        if t in (ctypes.c_float, ctypes.c_double):
            args.append(0.0)
        elif t in (ctypes.c_int, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64):
            args.append(0)
        else:
            args.append(None)          # pointers, structs by pointer, streams
    return args


def test_entry_points_reject_a_null_context():
    # every call that takes a dags_ctx checks its arguments on the host before
    # any CUDA call: a NULL context is DAGS_E_INVAL (-1), with nothing launched
    from paper_2602_21644_gb300 import dags
    lib = dags.load()
    host_only = {"dags_create", "dags_destroy", "dags_status_string", "dags_abi_version", "splat_forward_static",
                 "dags_measure_alu", "dags_measure_mma"}
    checked = []
    for name in dags.EXPORTS:
        if name in host_only or name.startswith("dags_default_"):
            continue
        fn = getattr(lib, name)
        assert fn.argtypes and fn.argtypes[0] is ctypes.c_void_p, name
        assert fn(*_zero_args(fn)) == -1, name
        checked.append(name)
    assert len(checked) >= 20
    lib.dags_destroy(None)             # destroying NULL is a no-op
    # the ALU probe takes no context; its arguments are checked first too
    ops = ctypes.c_double()
    assert lib.dags_measure_alu(2, 1024, ctypes.byref(ops), None) == -1
    assert lib.dags_measure_alu(0, 0, ctypes.byref(ops), None) == -1
    assert lib.dags_measure_alu(1, 1 << 25, ctypes.byref(ops), None) == -1
    assert lib.dags_measure_alu(0, 1024, None, None) == -1
    # so does the tensor-core probe's (N, warpgroups, repetitions)
    mac = ctypes.c_double()
    for m, n, g, r in [(128, 24, 1, 64), (128, 0, 1, 64), (128, 272, 1, 64), (128, 256, 4, 64), (128, 32, 3, 64),
                       (128, 32, 1, 0), (128, 32, 1, 5000), (96, 32, 1, 64), (256, 32, 1, 64)]:
        assert lib.dags_measure_mma(m, n, g, r, ctypes.byref(mac), None) == -1, (m, n, g, r)
    assert lib.dags_measure_mma(128, 32, 1, 64, None, None) == -1


def test_static_forward_limits_are_checked_on_the_host():
    # splat_forward_static's workspace limits (n <= 16384, width and height
    # <= 256) are argument errors, returned before its first CUDA call; the
    # device pointers are never touched on the host, so stand-ins do
    from paper_2602_21644_gb300 import dags
    lib = dags.load()
    dev = ctypes.c_void_p(256)                     # a 16-byte aligned stand-in device address
    f = lib.splat_forward_static

    def call(n, w, h, image=dev):
        cam = dags.CCamera(200.0, 200.0, w / 2, h / 2, w, h)
        return f(dev, n, ctypes.byref(cam), dev, None, None, None, image, dev, None, None, None)
    assert call(16385, 64, 48) == -1
    assert call(100, 257, 48) == -1
    assert call(100, 64, 257) == -1
    assert call(-1, 64, 48) == -1
    assert call(100, 64, 48, image=None) == -1
