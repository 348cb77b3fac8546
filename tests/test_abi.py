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


def test_misaligned_allocator_blocks_are_refused_and_freed(lib_path):
    """sim_create checks that every block from a user allocator hook is 16-byte
    aligned (the kernels stream workspaces with bulk copies) before anything
    touches device memory: one misaligned block fails the call with
    LEMPS_EINVAL, no handle is returned, and every block handed out goes back
    through the free hook.  Host only: the fake blocks are never dereferenced."""
    import ctypes
    from paper_2508_05745_gb300 import lemps as L
    lib = L.load()
    handed, freed = [], []

    def alloc(nbytes, stream, ctx):
        p = 0x7F0000000000 + 0x1000000 * (len(handed) + 1) + (8 if len(handed) == 3 else 0)
        handed.append(p)
        return p

    def free(ptr, nbytes, stream, ctx):
        freed.append(ptr)

    cb = (L.ALLOC_FN(alloc), L.FREE_FN(free))
    cfg = L.Config(n_qubits=8, chi_max=16, trunc_cutoff=1e-12, n_traj=4, traj_offset=0, seed=1,
                   precision=L.LEMPS_MIXED, unravel_mode=L.LEMPS_UNRAVEL_OPTIMAL, log_capacity=0, eps_max=2.0,
                   cuda_stream=None, alloc=cb[0], free=cb[1], alloc_ctx=None, layering=L.LEMPS_LAYER_LOCAL,
                   max_traj_in_flight=4)
    h = ctypes.c_void_p()
    assert lib.sim_create(ctypes.byref(cfg), ctypes.byref(h)) == L.LEMPS_EINVAL
    assert b"16-byte aligned" in lib.lemps_last_error()
    assert h.value is None
    assert len(handed) > 3 and sorted(freed) == sorted(handed)


def test_eigvec_fp64_flag_is_validated(lib_path):
    """lemps_config.eigvec_fp64 takes 0 or 1; any other value fails sim_create
    with LEMPS_EINVAL before any device call (host only)."""
    import ctypes
    from paper_2508_05745_gb300 import lemps as L
    lib = L.load()
    cfg = L.Config(n_qubits=8, chi_max=16, trunc_cutoff=1e-12, n_traj=4, traj_offset=0, seed=1,
                   precision=L.LEMPS_MIXED, unravel_mode=L.LEMPS_UNRAVEL_OPTIMAL, log_capacity=0, eps_max=2.0,
                   cuda_stream=None, alloc=L.ALLOC_FN(0), free=L.FREE_FN(0), alloc_ctx=None,
                   layering=L.LEMPS_LAYER_LOCAL, max_traj_in_flight=4, eigvec_fp64=2)
    h = ctypes.c_void_p()
    assert lib.sim_create(ctypes.byref(cfg), ctypes.byref(h)) == L.LEMPS_EINVAL
    assert b"eigvec_fp64" in lib.lemps_last_error()
    assert h.value is None


def test_gemm_tile_is_validated(lib_path):
    """lemps_config.gemm_tile takes 0 (autotune) or 1..4 (a fixed tile shape);
    any other value fails sim_create with LEMPS_EINVAL before any device call
    (host only)."""
    import ctypes
    from paper_2508_05745_gb300 import lemps as L
    lib = L.load()
    for bad in (-1, 5):
        cfg = L.Config(n_qubits=8, chi_max=16, trunc_cutoff=1e-12, n_traj=4, traj_offset=0, seed=1,
                       precision=L.LEMPS_FP64, unravel_mode=L.LEMPS_UNRAVEL_OPTIMAL, log_capacity=0, eps_max=2.0,
                       cuda_stream=None, alloc=L.ALLOC_FN(0), free=L.FREE_FN(0), alloc_ctx=None,
                       layering=L.LEMPS_LAYER_LOCAL, max_traj_in_flight=4, eigvec_fp64=0, gemm_tile=bad)
        h = ctypes.c_void_p()
        assert lib.sim_create(ctypes.byref(cfg), ctypes.byref(h)) == L.LEMPS_EINVAL
        assert b"gemm_tile" in lib.lemps_last_error()
        assert h.value is None
