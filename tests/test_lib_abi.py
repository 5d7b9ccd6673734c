"""The C-ABI library builds, loads and exports every symbol include/fos.h declares.

Runs without a GPU: no compute call is made except ones that must fail
cleanly when no device is present.
"""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fos.h")


@pytest.fixture(scope="module")
def fos():
    from paper_2002_00250_gb300 import build
    build.build()
    from paper_2002_00250_gb300 import fos as f
    f.load()
    return f


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fos_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(fos):
    lib = ctypes.CDLL(fos.LIB_PATH)
    names = declared_functions()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(fos.SIGNATURES), "binding and header disagree"


def test_struct_layout_matches_c(fos, tmp_path):
    # sizeof / offsetof from the C compiler against the ctypes mirrors
    prog = tmp_path / "layout.c"
    fields = [f for f, _ in fos.Params._fields_]
    cfields = [("lambda" if f == "lambda_" else f) for f in fields]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "fos.h"', "int main(void){",
             'printf("%zu\\n", sizeof(fos_params));',
             'printf("%zu\\n", sizeof(fos_state_header));',
             'printf("%zu\\n", sizeof(fos_kernel_timing));']
    lines += [f'printf("%zu\\n", offsetof(fos_params, {c}));' for c in cfields]
    lines.append("return 0;}")
    prog.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    out = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert out[0] == ctypes.sizeof(fos.Params)
    assert out[1] == ctypes.sizeof(fos.StateHeader)
    assert out[2] == ctypes.sizeof(fos.KernelTiming)
    for f, off in zip(fields, out[3:]):
        assert getattr(fos.Params, f).offset == off, f


def test_default_params(fos):
    p = fos.default_params()
    assert p.methods == 3 and p.K_rgb == 3 and p.K_d == 3 and p.N == 20
    assert p.alpha == pytest.approx(0.001)  # Sec. 3.1
    assert p.depth_full_scale_mm == 10000
    assert fos.load().fos_abi_version() == 1


def test_invalid_arguments_rejected_before_any_device_call(fos):
    lib = fos.load()
    p = fos.default_params()
    assert not lib.fos_create(0, 10, ctypes.byref(p))
    assert b"width" in lib.fos_last_error(None)
    p.N = 32
    assert not lib.fos_create(16, 16, ctypes.byref(p))
    assert b"N" in lib.fos_last_error(None)
    p = fos.default_params(K_rgb=4)
    assert not lib.fos_create(16, 16, ctypes.byref(p))
    assert b"K_rgb" in lib.fos_last_error(None)
    assert lib.fos_process_frame(None, None, None, None) == 1
    lib.fos_destroy(None)


def test_create_fails_loudly_without_a_device(fos):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(fos.FosError):
        fos.Segmenter(32, 16)


def test_params_json_round_trip(tmp_path):
    from paper_2002_00250_gb300 import fos
    p = fos.params_from_dict({"alpha": 0.01, "lambda": 3.0, "N": 16, "methods": 2})
    assert p.N == 16 and p.methods == 2 and abs(p.lambda_ - 3.0) < 1e-7
    text = fos.params_to_json(p)
    q = fos.params_from_json(text)
    assert q.as_dict() == p.as_dict()
    f = tmp_path / "p.json"
    f.write_text(text)
    assert fos.params_from_json(str(f)).as_dict() == p.as_dict()
    with pytest.raises(KeyError):
        fos.params_from_dict({"no_such_field": 1})
