"""The C ABI library builds, loads without a GPU and exports every declared call."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sddm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sddm_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_1912_06474_gb300 import build
    build.build()
    from paper_1912_06474_gb300 import sddm
    names = _declared()
    assert len(names) >= 16
    for n in names:
        assert hasattr(sddm.lib, n), n
    assert set(names) == set(sddm.EXPORTED)
    assert sddm.version().startswith("sddm ")


def test_binding_has_no_cpu_fallback():
    """The binding imports nothing from the oracle and refuses to run without the library."""
    src = open(os.path.join(ROOT, "paper_1912_06474_gb300", "sddm.py")).read()
    assert "oracle" not in src
    assert "raise ImportError" in src
    for f in os.listdir(os.path.join(ROOT, "paper_1912_06474_gb300")):
        if f.endswith(".py"):
            assert "import oracle" not in open(os.path.join(ROOT, "paper_1912_06474_gb300", f)).read(), f


def test_every_call_rejects_a_null_context():
    """Argument checks run before any CUDA call: with a NULL context every entry
    point returns a negative status and leaves a message (the library never
    aborts), and sddm_create rejects a NULL output pointer."""
    import ctypes as C
    from paper_1912_06474_gb300 import build
    build.build()
    from paper_1912_06474_gb300 import sddm
    lib = sddm.lib
    skip = {"sddm_last_error", "sddm_version", "sddm_destroy"}
    for name in sddm.EXPORTED:
        if name in skip:
            continue
        f = getattr(lib, name)
        args = []
        for t in f.argtypes:
            if t in (C.c_int, C.c_int64, C.c_uint32):
                args.append(0)
            elif t in (C.c_float, C.c_double):
                args.append(0.0)
            elif t is C.c_char_p:
                args.append(None)
            else:
                args.append(None)
        rc = f(*args)
        assert rc < 0, name
        assert lib.sddm_last_error(), name
    assert lib.sddm_destroy(None) == 0
