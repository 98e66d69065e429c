"""The C-ABI library builds/loads and exports every symbol include/pifepic.h declares.
No compute call: these run without a GPU."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pifepic.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pifepic_[A-Za-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_2011_10214_gb300 import build
    if not os.path.exists(build.LIB):
        build.build_library()
    from paper_2011_10214_gb300 import capi
    declared = _declared()
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(capi.lib, name), name
    assert sorted(capi.EXPORTED) == declared


def test_binding_has_no_cpu_fallback():
    """The product path never imports the oracle."""
    for fn in ("capi.py", "build.py", "workloads.py", "__init__.py"):
        src = open(os.path.join(ROOT, "paper_2011_10214_gb300", fn)).read()
        code = "\n".join(l for l in src.splitlines() if not l.lstrip().startswith("#"))
        assert "import oracle" not in code and "from oracle" not in code, fn
