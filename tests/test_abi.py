"""The C-ABI library loads and exports every function include/*.h declares
(no GPU needed: nothing is called)."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_builder():
    """The build script, loaded by path (importing the package would load the library)."""
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "exactmap_build", os.path.join(ROOT, "paper_2404_17084_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(hdr).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?(?:int|void|char|int64_t)\s*\*?\s*(\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    b = load_builder()
    path = b.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert {"map_init", "map_particles_to_cells", "build_pseudo_particles", "solve_h"} <= names
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_and_defaults_without_gpu():
    b = load_builder()
    lib = ctypes.CDLL(b.build())
    lib.map_strerror.restype = ctypes.c_char_p
    assert lib.map_strerror(0) == b"ok"
    assert b"memory" in lib.map_strerror(-2)


def test_binding_wraps_every_declared_symbol():
    """The Python binding has a function of the same name for every entry
    point the header declares (argument marshalling only)."""
    import paper_2404_17084_gb300 as L
    missing = sorted(n for n in declared_functions() if not callable(getattr(L, n, None)))
    assert not missing, missing
