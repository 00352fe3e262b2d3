"""The C ABI without a GPU: the library builds for sm_103a, loads, exports
every function include/hanf.h declares, and its host-only entry points
(workspace sizing, argument checks, statistics) behave as documented."""
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def H():
    from paper_1011_5599_gb300 import build as B
    B.build()
    import paper_1011_5599_gb300.hanf as H
    return H


def header_functions():
    src = open(os.path.join(ROOT, "include", "hanf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hanf_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_function(H):
    declared = header_functions()
    assert declared, "no functions parsed from hanf.h"
    assert sorted(declared) == sorted(H.EXPORTS)
    for name in declared:
        assert hasattr(H.lib(), name), name


def test_library_has_no_torch_dependency():
    from paper_1011_5599_gb300 import build as B
    B.build()
    data = open(B.LIB, "rb").read()
    assert b"libtorch" not in data and b"libc10" not in data


def test_default_opts(H):
    o = H.default_opts()
    assert (o.runs, o.frontier, o.push_den, o.use_graph) == (1, 2, 4, 0)


def test_workspace_size_and_argument_errors(H):
    o, _ = H.make_opts()
    small = H.workspace_size(1000, 5000, 6, o, True)
    big = H.workspace_size(100000, 500000, 6, o, True)
    assert 0 < small < big
    borrowed = H.workspace_size(100000, 500000, 6, o, False)
    assert borrowed < big
    for bad in [dict(log2m=3), dict(log2m=9), dict(n=-1), dict(n=2**31), dict(arcs=-1)]:
        args = dict(n=10, arcs=10, log2m=6)
        args.update(bad)
        with pytest.raises(H.HanfError) as e:
            H.workspace_size(args["n"], args["arcs"], args["log2m"], o, True)
        assert e.value.code == H.HANF_EINVAL
    o3, _ = H.make_opts(runs=3)
    with pytest.raises(H.HanfError):
        H.workspace_size(10, 10, 6, o3, True)
    o9, _ = H.make_opts(runs=9)
    with pytest.raises(H.HanfError):
        H.workspace_size(10, 10, 6, o9, True)


def test_stats_match_oracle(H, oracle):
    """Host post-processing (Sections 4-5) of the library against the oracle."""
    rng = np.random.default_rng(4)
    for _ in range(20):
        N = np.cumsum(rng.uniform(1, 100, rng.integers(1, 30)))
        for ez in (False, True):
            a = H.stats(N, exclude_zero=ez)
            b = oracle.stats(N, exclude_zero=ez)
            for k in a:
                if math.isnan(b[k]):
                    assert math.isnan(a[k])
                else:
                    assert a[k] == pytest.approx(b[k], rel=1e-13, abs=1e-13)


def test_ed_interval_and_run_stats_match_oracle(H, oracle):
    rng = np.random.default_rng(5)
    for _ in range(30):
        N = np.cumsum(rng.uniform(1, 100, rng.integers(1, 25)))
        for eps in (0.0, 0.01, 0.1):
            assert H.ed_interval(N, 0.9, eps) == oracle.ed_interval(N, 0.9, eps)
    runs = [np.cumsum(rng.uniform(1, 50, rng.integers(2, 15))) for _ in range(7)]
    a, b = H.stats_runs(runs), oracle.stats_runs(runs)
    for k in a:
        assert a[k][0] == pytest.approx(b[k][0], rel=1e-12)
        assert a[k][1] == pytest.approx(b[k][1], rel=1e-9, abs=1e-12)


def test_structs_match_header(H, tmp_path):
    """The binding's ctypes structures have the header's layout: a C program
    compiled against include/hanf.h prints every field's offset and the
    sizes, which must equal the ctypes ones."""
    import ctypes
    import shutil
    import subprocess
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "hanf.h"', "int main(void) {"]
    expect = []
    for cname, ctype in (("hanf_opts", H.Opts), ("hanf_job", H.Job)):
        lines.append(f'printf("%zu\\n", sizeof({cname}));')
        expect.append(ctypes.sizeof(ctype))
        for field, _ in ctype._fields_:
            lines.append(f'printf("%zu\\n", offsetof({cname}, {field}));')
            expect.append(getattr(ctype, field).offset)
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True,
                                          text=True).stdout.split()]
    assert got == expect
