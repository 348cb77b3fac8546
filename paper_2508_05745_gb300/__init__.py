"""GB300 library for batched Monte-Carlo MPS trajectories with the locally
entanglement-optimal unraveling (arXiv 2508.05745).

Submodules: ``lemps`` (binding of the C ABI in include/lemps.h), ``build``
(nvcc build for sm_103a), ``inputs`` (seeded synthetic workloads).  The
binding is imported lazily so that the input generators can be used without
the native library.
"""
__all__ = ["lemps", "build", "inputs"]
