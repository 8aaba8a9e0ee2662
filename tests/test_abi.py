"""The C-ABI library loads and exports every function include/vcsgc.h declares
(no compute calls: runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "vcsgc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:int|void|const char\*)\s+(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for required in ("vcsgc_init", "vcsgc_sweep", "md_steps", "observables", "vcsgc_free"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1012_5082_gb300 import build
    lib = ctypes.CDLL(build.build())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_export():
    from paper_1012_5082_gb300 import vcsgc
    assert set(declared_functions()) == set(vcsgc.EXPORTS)


def test_default_options_without_gpu():
    from paper_1012_5082_gb300 import vcsgc
    o = vcsgc.vcsgc_default_options()
    assert o.n_replicas == 1 and o.schedule == vcsgc.SCHED_SUBLATTICE and abs(o.dt - 2.0) < 1e-15
