"""The C ABI without a GPU: libdist.so loads, exports every function that
include/dist.h declares, its structs have the layout the ctypes binding
assumes, and host-only entry points behave (defaults, argument checks)."""

import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dist.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1911_13225_b300 import build
    build.build()
    from paper_1911_13225_b300 import _abi
    return _abi.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(dist_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    from paper_1911_13225_b300 import _abi
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), f"{n} declared in dist.h but not exported"
    assert set(names) == set(_abi.EXPORTS)


def test_struct_layouts_match_ctypes(tmp_path):
    from paper_1911_13225_b300 import _abi
    prog = tmp_path / "sizes.c"
    prog.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "dist.h"\n'
        "int main(void) {\n"
        '  printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(dist_decoder_desc), sizeof(dist_camera),\n'
        "         sizeof(dist_trace_params), sizeof(dist_trace_out), sizeof(dist_loss_weights),\n"
        "         sizeof(dist_request));\n"
        '  printf("%zu %zu %zu\\n", offsetof(dist_request, cam), offsetof(dist_request, z),\n'
        "         offsetof(dist_trace_out, queries));\n"
        "  return 0; }\n")
    exe = tmp_path / "sizes"
    subprocess.check_call(["gcc", "-I", os.path.dirname(HEADER), str(prog), "-o", str(exe)])
    out = subprocess.check_output([str(exe)]).decode().split()
    got = [int(x) for x in out]
    want = [ctypes.sizeof(_abi.DecoderDesc), ctypes.sizeof(_abi.Camera),
            ctypes.sizeof(_abi.TraceParams), ctypes.sizeof(_abi.TraceOut),
            ctypes.sizeof(_abi.LossWeights), ctypes.sizeof(_abi.Request),
            _abi.Request.cam.offset, _abi.Request.z.offset, _abi.TraceOut.queries.offset]
    assert got == want


def test_defaults_and_version(lib):
    from paper_1911_13225_b300 import _abi, api
    p = _abi.TraceParams()
    lib.dist_trace_params_default(ctypes.byref(p))
    mine = api.TraceParams().c()
    for f, _ in _abi.TraceParams._fields_:
        assert getattr(p, f) == pytest.approx(getattr(mine, f)), f
    assert p.max_steps == 50 and p.alpha == pytest.approx(1.5) and p.eps == pytest.approx(5e-5)
    assert lib.dist_version().startswith(b"libdist")


def test_argument_checks_without_device(lib):
    from paper_1911_13225_b300 import _abi
    h = ctypes.c_void_p()
    desc = _abi.DecoderDesc(256, 500, 8, 4)          # width not supported
    W = (ctypes.c_void_p * 9)()
    assert lib.dist_decoder_create(ctypes.byref(desc), W, W, ctypes.byref(h)) == _abi.DIST_E_INVALID
    assert b"width" in lib.dist_last_error()
    assert lib.dist_decoder_create(None, W, W, ctypes.byref(h)) == _abi.DIST_E_INVALID
    assert lib.dist_workspace_create(0, 50, ctypes.byref(h)) == _abi.DIST_E_INVALID
    assert lib.dist_trace_fwd(None, None, 1, None, 1, None, None, None, None) == _abi.DIST_E_INVALID
    assert lib.dist_serve_submit(None, None, None) == _abi.DIST_E_INVALID
    assert lib.dist_serve_poll(None, 1, None) == _abi.DIST_E_INVALID
    assert lib.dist_serve_destroy(None) == _abi.DIST_OK
    assert lib.dist_decoder_destroy(None) == _abi.DIST_OK


def test_library_fails_loudly_when_missing(tmp_path, monkeypatch):
    from paper_1911_13225_b300 import _abi
    monkeypatch.setattr(_abi, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_abi, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _abi.lib()
