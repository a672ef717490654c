"""The C-ABI library builds, loads and exports every entry point the public headers declare (CPU only;
no compute call is made without a GPU)."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(fhash_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return names


def test_library_exports_declared_symbols():
    import __graft_entry__
    path = __graft_entry__._build_module().build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert "fhash_build" in names and "fhash_train_step" in names
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_fails_without_gpu_gracefully():
    # Importing the binding works on a CPU-only host; errors come back as statuses, never aborts.
    import paper_2507_03836_gb300 as fh
    assert callable(fh.fhash_build)
    assert isinstance(fh.fhash_last_error(), str)
