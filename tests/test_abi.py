"""The C ABI without a GPU: the library builds, loads and exports every declared entry
point; the ctypes struct matches the C layout; the product path has no fallback."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2405_16911_gb300 as pkg
from paper_2405_16911_gb300 import _cyc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    pkg.build()
    return pkg.load()


def test_every_declared_symbol_is_exported(lib):
    names = pkg.declared_functions()
    assert {"cyc_create", "cyc_push", "cyc_read"} <= set(names)
    for n in names:
        assert hasattr(lib, n), n
        assert hasattr(_cyc, n), "binding lacks " + n
    out = subprocess.run(["nm", "-D", "--defined-only", pkg.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (cyc_\w+)", out))
    assert set(names) <= exported
    assert exported <= set(names), "undeclared exports: %s" % (exported - set(names))


def test_params_struct_layout_matches_c(tmp_path):
    src = tmp_path / "lay.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "cyc.h"\nint main(void){'
                   'printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(cyc_params), offsetof(cyc_params, alphas),'
                   'offsetof(cyc_params, n0), offsetof(cyc_params, max_chunk), offsetof(cyc_params, cuda_stream),'
                   'offsetof(cyc_params, device)); return 0; }\n')
    exe = tmp_path / "lay"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    P = _cyc.cyc_params
    assert got == [ctypes.sizeof(P), P.alphas.offset, P.n0.offset, P.max_chunk.offset,
                   P.cuda_stream.offset, P.device.offset]


def test_server_structs_match_c(tmp_path):
    src = tmp_path / "lay2.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "cyc.h"\nint main(void){'
                   'printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(cyc_server_params),'
                   'offsetof(cyc_server_params, mem_budget), offsetof(cyc_server_params, ring_samples),'
                   'offsetof(cyc_server_params, max_items), offsetof(cyc_server_params, item_samples),'
                   'offsetof(cyc_server_params, device), sizeof(cyc_done), offsetof(cyc_done, tag),'
                   'offsetof(cyc_done, done_s)); return 0; }\n')
    exe = tmp_path / "lay2"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    P, D = _cyc.cyc_server_params, _cyc.cyc_done
    assert got == [ctypes.sizeof(P), P.mem_budget.offset, P.ring_samples.offset, P.max_items.offset,
                   P.item_samples.offset, P.device.offset, ctypes.sizeof(D), D.tag.offset, D.done_s.offset]


def test_status_strings_and_no_device_error(lib):
    assert pkg.cyc_strerror(-1) == "invalid argument"
    assert pkg.cyc_strerror(-6).startswith("no data")
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if has_gpu:
        pytest.skip("a GPU is present")
    with pytest.raises(pkg.CycError) as e:
        pkg.cyc_create([0, 1], [0.1])
    assert e.value.code == -3 and "no CUDA device" in str(e.value)


def test_product_path_does_not_touch_the_oracle():
    pkgdir = os.path.join(ROOT, "paper_2405_16911_gb300")
    for dirpath, _, files in os.walk(pkgdir):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", text, re.M), f
                assert "cyc_oracle" not in text and "cyco_" not in text, f


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    monkeypatch.setattr(_cyc, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        _cyc.load(str(tmp_path / "nope.so"))


def test_phase_increment_is_exact_rounding(lib):
    """round(a * 2^64) mod 2^64 in exact rational arithmetic, for awkward doubles."""
    from fractions import Fraction
    import numpy as np
    rng = np.random.default_rng(0)
    vals = [0.0, -0.0, 0.5, -0.5, 0.1, -0.33, 1.0 / 3.0, -1.0 / 3.0, 1e-30, -1e-30, 2.0 ** -64,
            2.0 ** -65, 3 * 2.0 ** -66, 12345.678, -98765.4321, 2.0 ** 60 + 0.5 * 2 ** 8, -0.875, 1 - 2 ** -53]
    vals += list(rng.uniform(-3, 3, 200)) + list(rng.uniform(-1e-12, 1e-12, 50))
    for a in vals:
        exact = Fraction(a) * (1 << 64)
        fl = exact.numerator // exact.denominator
        rem = exact - fl
        want = (fl + (1 if rem > Fraction(1, 2) else 0 if rem < Fraction(1, 2) else 1)) % (1 << 64)
        got = pkg.cyc_phase_increment(a)
        # ties (only possible for a with a bit at 2^-65) may round either way
        assert got == want or (rem == Fraction(1, 2) and got == (fl % (1 << 64))), a
    with pytest.raises(pkg.CycError):
        pkg.cyc_phase_increment(float("inf"))
