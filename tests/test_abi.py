"""The C-ABI library builds, loads without a GPU and exports every function that
include/*.h declares (no compute calls here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, re.M):
            name = m.group(1)
            if name not in ("if", "while", "for", "return", "sizeof"):
                names.add(name)
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1504_05158_gb300 import build, qap_pso
    build.build()
    return qap_pso.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("qap_create_instance", "pso_init", "pso_step", "pso_best", "pso_stats"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_lists_every_export(lib):
    from paper_1504_05158_gb300 import qap_pso
    assert set(declared_functions()) <= set(qap_pso.EXPORTS)


def test_status_strings(lib):
    from paper_1504_05158_gb300 import qap_pso as Q
    assert Q.status_string(Q.OK) == "ok"
    assert "unsupported" in Q.status_string(Q.ERR_UNSUPPORTED)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_1504_05158_gb300 import qap_pso as Q
    monkeypatch.setattr(Q, "_lib", None)
    monkeypatch.setattr(Q, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        Q.lib()


def test_built_for_sm_103a(lib):
    from paper_1504_05158_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH
    assert os.path.getsize(build.LIB) > 0
