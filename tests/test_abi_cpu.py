"""CPU-only checks of the C ABI library and of the oracle/product separation."""
import ast
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(dda_[a-z0-9_]+)\s*\(", text))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_1202_3424_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    declared = _declared_symbols()
    assert len(declared) >= 14
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing


def test_create_without_gpu_fails_cleanly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    import paper_1202_3424_gb300 as dda
    with pytest.raises(dda.DdaError):
        dda.dda_create(0)


def _imports(path):
    tree = ast.parse(open(path).read())
    out = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            out |= {a.name.split(".")[0] for a in node.names}
        elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
            out.add(node.module.split(".")[0])
    return out


def _py_files(d):
    for base, _, files in os.walk(os.path.join(ROOT, d)):
        for f in files:
            if f.endswith(".py"):
                yield os.path.join(base, f)


def test_oracle_and_product_do_not_import_each_other():
    for f in _py_files("oracle"):
        assert "paper_1202_3424_gb300" not in _imports(f), f
    for f in _py_files("paper_1202_3424_gb300"):
        assert "oracle" not in _imports(f), f
    for f in _py_files("dda_inputs"):
        assert not ({"oracle", "paper_1202_3424_gb300"} & _imports(f)), f


def test_product_sources_reference_no_oracle_code():
    csrc = os.path.join(ROOT, "paper_1202_3424_gb300", "csrc")
    for f in os.listdir(csrc):
        text = open(os.path.join(csrc, f)).read()
        assert "oracle" not in text.lower(), f


def test_scattering_directions_host_code_matches_oracle():
    """The library's host-side direction rule (no GPU needed) against the
    oracle's, including the guide's printed NAVG = 962 case."""
    import numpy as np
    import paper_1202_3424_gb300 as dda
    from oracle import dda as odda
    try:
        dda.load_library(build_if_missing=False)
    except dda.DdaError:
        pytest.skip("library not built")
    for x, eta in ((3.093665, 0.5), (0.3, 1.0), (8.0, 0.25), (20.0, 0.5)):
        t, p, w = dda.dda_scattering_directions(x, eta)
        t2, p2, w2 = odda.scattering_directions(x, eta)
        assert t.size == t2.size
        assert np.abs(t - t2).max() < 1e-13 and np.abs(p - p2).max() < 1e-13 and np.abs(w - w2).max() < 1e-13
    assert dda.dda_scattering_directions(3.093665, 0.5)[0].size == 962


def _header_struct_fields(name):
    """Field names of `typedef struct { ... } name;` in include/dda.h, in order."""
    text = open(os.path.join(ROOT, "include", "dda.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    m = re.search(r"typedef struct\s*\{([^{}]*)\}\s*" + name + r"\s*;", text)
    assert m, name
    return re.findall(r"(\w+)\s*(?=[,;])", m.group(1))


@pytest.mark.parametrize("struct", ["dda_opts", "dda_result", "dda_info"])
def test_binding_structs_match_header(struct):
    """The ctypes mirrors of the ABI structs list the header's fields in order
    (a field added on one side only would shift every later one)."""
    import paper_1202_3424_gb300 as dda
    ours = [name for name, _ in getattr(dda, struct)._fields_]
    assert ours == _header_struct_fields(struct)
