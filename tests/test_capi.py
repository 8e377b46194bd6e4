"""CPU-only checks of the C ABI: the library loads and exports every function
declared in include/*.h; argument validation that needs no GPU."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(qsi_\w+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2601_04904_gb300 import build

    build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_entry_points():
    d = _declared()
    for name in ("qsi_create", "qsi_bta_factor", "qsi_bta_selinv", "qsi_bta_selquad", "qsi_bta_selquad_host"):
        assert name in d


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_binding_covers_header(lib):
    from paper_2601_04904_gb300 import qsi

    assert set(_declared()) <= set(qsi.exported_symbols())


def test_factor_bytes_formula(lib):
    from paper_2601_04904_gb300 import qsi

    # factor of a fused solve holds S_A, S_B, 4 arrow arrays, 2 tips and 4 off-diagonal copies
    n, b, a = 8, 32, 16
    nb = qsi.factor_bytes(n, b, a, True)
    exact = 16 * (2 * n * b * b + 4 * n * b * a + 2 * a * a + 4 * (n - 1) * b * b)
    assert exact <= nb <= exact + 16 * 32 * 12
    assert qsi.factor_bytes(n, b, a, False) < nb


def test_null_context_is_rejected(lib):
    from paper_2601_04904_gb300 import qsi

    f = qsi._lib.qsi_bta_factor
    out = ctypes.c_void_p()
    st = f(None, qsi.Shape(1, 1, 0), None, None, 0, ctypes.byref(out))
    assert st == qsi.ERR_ARG
    assert qsi._lib.qsi_synchronize(None) == qsi.ERR_ARG
    assert qsi._lib.qsi_destroy(None) == qsi.OK
    assert qsi._lib.qsi_factor_destroy(None) == qsi.OK


def test_request_bytes_covers_factor(lib):
    from paper_2601_04904_gb300 import qsi

    for n, b, a in [(4, 32, 16), (16, 256, 128), (64, 512, 256)]:
        rb = qsi.request_bytes(n, b, a, True, qsi.FP64)
        assert rb > qsi.factor_bytes(n, b, a, True)
        assert qsi.request_bytes(n, b, a, True, qsi.FP64_EMU) > rb
        assert qsi.request_bytes(n, b, a, False, qsi.FP64) < rb


def test_serve_submit_rejects_bad_args_without_gpu(lib):
    from paper_2601_04904_gb300 import qsi

    t = ctypes.c_uint64()
    assert qsi._lib.qsi_serve_submit(None, None, ctypes.byref(t)) == qsi.ERR_ARG
    assert qsi._lib.qsi_serve_destroy(None) == qsi.OK
    done = ctypes.c_int()
    assert qsi._lib.qsi_serve_poll(None, 1, ctypes.byref(done), None) == qsi.ERR_ARG
    srv = ctypes.c_void_p()
    assert qsi._lib.qsi_serve_create(ctypes.byref(srv), 0, 0, 0) == qsi.ERR_ARG  # zero slots
    assert qsi._lib.qsi_serve_create(ctypes.byref(srv), 0, 65, 0) == qsi.ERR_ARG  # too many slots


def test_zgemm_and_batched_reject_null_context(lib):
    from paper_2601_04904_gb300 import qsi

    assert qsi._lib.qsi_zgemm(None, 0, 1, 1, 1, 0, None, 1, 0, None, 1, 1.0, 0.0, 0.0, None, 1) == qsi.ERR_ARG
    assert qsi._lib.qsi_bta_selquad_batched(None, qsi.Shape(1, 1, 0), None, 1, None, 0.0, None, None, 0, None,
                                            None) == qsi.ERR_ARG


def test_struct_layouts_match_header(tmp_path):
    """ctypes mirrors of the header's structs: same size and field offsets as a
    C compiler gives them (the binding marshals through these)."""
    import shutil
    import subprocess

    from paper_2601_04904_gb300 import qsi

    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    specs = {"qsi_shape": qsi.Shape, "qsi_bta": qsi.BTA, "qsi_stats": qsi.Stats, "qsi_request": qsi.Request,
             "qsi_result": qsi.Result}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "qsi.h"', "int main(void) {"]
    for cname, py in specs.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname}.{fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    seen = 0
    for line in out.splitlines():
        key, val = line.split()
        if "." in key:
            c, f = key.split(".")
            assert getattr(specs[c], f).offset == int(val), key
        else:
            assert ctypes.sizeof(specs[key]) == int(val), key
        seen += 1
    assert seen == len(specs) + sum(len(p._fields_) for p in specs.values())


def test_constants_match_header(tmp_path):
    """The binding's status codes, precisions, flags and limits have the
    header's values (a C compiler prints them)."""
    import shutil
    import subprocess

    from paper_2601_04904_gb300 import qsi

    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    pairs = {"QSI_OK": qsi.OK, "QSI_ERR_ARG": qsi.ERR_ARG, "QSI_ERR_OOM": qsi.ERR_OOM,
             "QSI_ERR_SINGULAR": qsi.ERR_SINGULAR, "QSI_ERR_CUDA": qsi.ERR_CUDA, "QSI_ERR_TIMEOUT": qsi.ERR_TIMEOUT,
             "QSI_ERR_BUSY": qsi.ERR_BUSY, "QSI_ERR_STATE": qsi.ERR_STATE,
             "QSI_ERR_UNSUPPORTED": qsi.ERR_UNSUPPORTED, "QSI_ERR_ACCURACY": qsi.ERR_ACCURACY,
             "QSI_FP64": qsi.FP64, "QSI_FP64_EMU": qsi.FP64_EMU, "QSI_MIXED": qsi.MIXED, "QSI_SPLIT3": qsi.SPLIT3,
             "QSI_MAX_RHS": qsi.MAX_RHS, "QSI_PLAN_ARRAYS": qsi.PLAN_ARRAYS,
             "QSI_ASSUME_ANTIHERMITIAN_B": qsi.ASSUME_ANTIHERMITIAN_B, "QSI_TWISTED_SPLIT": qsi.TWISTED_SPLIT,
             "QSI_NOALLOC_MAX_B": qsi.NOALLOC_MAX_B}
    lines = ["#include <stdio.h>", '#include "qsi.h"', "int main(void) {"]
    lines += [f'printf("{c} %lld\\n", (long long)({c}));' for c in pairs]
    lines.append("return 0; }")
    src = tmp_path / "consts.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "consts"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    got = dict(line.split() for line in out.splitlines())
    assert {c: int(v) for c, v in got.items()} == pairs
    # the flags are distinct bits
    assert qsi.ASSUME_ANTIHERMITIAN_B & qsi.TWISTED_SPLIT == 0
