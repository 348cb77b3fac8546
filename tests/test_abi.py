"""CPU-side checks of the native library: it builds for sm_103a, loads, and
exports every entry point declared in include/lemps.h (no compute calls)."""
import os
import re
import subprocess

import pytest

from paper_2508_05745_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "lemps.h")).read()
    return sorted(set(re.findall(r"^\s*(?:lemps_status|const char\*)\s+(\w+)\(", src, re.M)))


@pytest.fixture(scope="module")
def lib_path():
    return B.build()


def test_header_declares_the_six_calls():
    names = declared_symbols()
    for n in ["sim_create", "apply_layer", "unravel_opt", "sample_branch", "measure", "destroy"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [n for n in declared_symbols() if n not in exported]
    assert not missing, missing


def test_library_loads_with_ctypes(lib_path):
    from paper_2508_05745_gb300 import lemps
    lib = lemps.load()
    for n in declared_symbols():
        assert hasattr(lib, n)


def test_built_for_sm103a_only(lib_path):
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.getsize(lib_path) > 0


def test_no_cpu_fallback_without_gpu():
    import torch
    from paper_2508_05745_gb300 import lemps
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(RuntimeError):
        lemps.Simulation(4, 4, 2)
