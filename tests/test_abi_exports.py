"""The C-ABI library builds, loads and exports every function include/crl.h declares.

Runs without a GPU: only host-side entry points are called (config defaults
and the parameter layout), never a kernel.
"""

import ctypes
import os
import re

import pytest

from paper_2408_11052_gb300 import api, build, workload

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "crl.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return api.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(crl_[a-z0-9_]+)\s*\(", text))
    assert names, "no declarations found"
    return sorted(names)


def test_every_declared_function_is_exported(lib):
    raw = ctypes.CDLL(api.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(raw, n)]
    assert not missing, missing
    assert set(declared_functions()) == set(api._SIGNATURES), "binding signatures out of sync with the header"


def test_config_default_layout_matches_binding(lib):
    c = api.CrlConfig()
    lib.crl_config_default(ctypes.byref(c))
    assert (c.E, c.T, c.D, c.A, c.G, c.B) == (1024, 1000, 29, 8, 2, 256)
    assert (c.hidden, c.layers, c.repr) == (256, 2, 64)
    assert list(c.goal_idx)[:3] == [0, 1, 2]
    assert c.gamma == pytest.approx(0.99) and c.beta_lse == pytest.approx(0.1)
    assert c.lr_critic == pytest.approx(3e-4) and c.lr_actor == pytest.approx(6e-4)
    assert c.adam_eps == pytest.approx(1e-8) and c.offset_min == 1
    assert c.seed == 0 and c.agent == 0
    assert c.alpha_autotune == 0 and c.target_entropy == pytest.approx(-8.0) and c.lr_alpha == pytest.approx(6e-4)


def test_config_struct_layout_matches_the_header(tmp_path):
    """sizeof and every field offset of crl_config as the C compiler lays out the
    header, against the ctypes mirror."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    fields = [f[0] for f in api.CrlConfig._fields_]
    src = tmp_path / "layout.c"
    lines = ["#include <stddef.h>", "#include <stdio.h>", f'#include "{ROOT}/include/crl.h"', "int main(void) {",
             '  printf("%zu\\n", sizeof(crl_config));']
    lines += [f'  printf("%zu\\n", offsetof(crl_config, {f}));' for f in fields]
    lines += ["  return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", str(src), "-o", str(exe)], check=True)
    out = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert out[0] == ctypes.sizeof(api.CrlConfig)
    assert out[1:] == [getattr(api.CrlConfig, f).offset for f in fields]


@pytest.mark.parametrize("w", [workload.ANT_AUTOGRAD, workload.HUMANOID_BF16, workload.LARGE_BATCH])
@pytest.mark.parametrize("net", ["phi", "psi", "pi"])
def test_param_layout_is_consistent(lib, w, net):
    cfg = api.make_config(w)
    n, tensors = api.param_layout(cfg, net)
    ins, out = workload.network_shapes(w, net)
    dims = [ins] + [w.hidden] * w.layers + [out]
    expect = []
    for li in range(w.layers + 1):
        expect.append((li, "W", dims[li + 1], dims[li]))
        expect.append((li, "b", dims[li + 1], 1))
        if w.layernorm and li < w.layers:
            expect += [(li, "ln_g", dims[li + 1], 1), (li, "ln_b", dims[li + 1], 1)]
    assert [(t["layer"], t["kind"], t["rows"], t["cols"]) for t in tensors] == expect
    end = 0
    for t in tensors:
        assert t["offset"] % 64 == 0 and t["offset"] >= end
        end = t["offset"] + t["rows"] * t["cols"]
    assert end <= n


def test_host_side_errors_without_gpu(lib):
    cfg = api.make_config(workload.SMALL_FP32)
    out = ctypes.c_int64()
    assert lib.crl_param_count(ctypes.byref(cfg), 7, ctypes.byref(out)) == api.E_INVALID_ARG
    info = api.CrlTensorInfo()
    assert lib.crl_param_tensor(ctypes.byref(cfg), 0, 99, ctypes.byref(info)) == api.E_INVALID_ARG
    assert b"out of range" in lib.crl_last_error(None)


def test_config_validation_of_objectives_without_gpu(lib):
    """Rejected before any device work: unknown objective and forward-backward
    with B = 1."""
    h = ctypes.c_void_p()
    w = workload.SMALL_FP32
    for cfg, code in ((api.make_config(w, loss=10), api.E_INVALID_ARG),
                      (api.make_config(w.with_(B=1, loss="fb")), api.E_INVALID_ARG)):
        assert lib.crl_create(ctypes.byref(cfg), ctypes.byref(h)) == code
        assert h.value is None


def header_defines():
    text = open(HEADER).read()
    return {m.group(1): int(m.group(2)) for m in re.finditer(r"#define\s+(CRL_[A-Z0-9_]+)\s+\(?(-?\d+)\)?", text)}


@pytest.mark.parametrize("table,prefix", [("ENERGY", "ENERGY"), ("LOSS", "LOSS"), ("PREC", "PREC"), ("PATH", "PATH"),
                                          ("NET", "NET"), ("TRACE", "TRACE"), ("GEMM_KERNEL", "GEMM")])
def test_binding_constants_match_the_header(table, prefix):
    """Every name of the binding's table is the header's CRL_<prefix>_<NAME>, with its value."""
    defines = header_defines()
    for name, value in getattr(api, table).items():
        key = f"CRL_{prefix}_{name.upper()}"
        assert key in defines, key
        assert defines[key] == value, (key, defines[key], value)


def test_error_codes_match_the_header():
    defines = header_defines()
    for name in ("INVALID_ARG", "SHAPE", "BUFFER_EMPTY", "CUDA", "NONFINITE", "TIMEOUT", "NOT_BOUND", "UNSUPPORTED"):
        assert defines[f"CRL_E_{name}"] == getattr(api, f"E_{name}"), name
    assert defines["CRL_OK"] == api.OK
