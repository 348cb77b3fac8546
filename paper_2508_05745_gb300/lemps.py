"""Python binding of the C ABI in include/lemps.h (argument marshalling only).

Every numerical step runs in the CUDA library ``_build/liblemps.so``.  There is
no CPU fallback: if the library is missing or no GPU is present the calls
raise.  PyTorch provides device memory (its caching allocator is passed to
``sim_create`` as the allocation hook) and streams.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import build as _build

LEMPS_OK, LEMPS_EINVAL, LEMPS_ENOMEM, LEMPS_ECUDA, LEMPS_ENUMERIC, LEMPS_ESTATE = range(6)
LEMPS_FP64, LEMPS_MIXED = 0, 1
LEMPS_UNRAVEL_OPTIMAL, LEMPS_UNRAVEL_GIVEN, LEMPS_UNRAVEL_HAAR_OPT = 0, 1, 2
LEMPS_LAYER_LOCAL, LEMPS_LAYER_GLOBAL = 0, 1
LAYERINGS = {"local": LEMPS_LAYER_LOCAL, "global": LEMPS_LAYER_GLOBAL}
UNRAVEL_MODES = {"optimal": LEMPS_UNRAVEL_OPTIMAL, "given": LEMPS_UNRAVEL_GIVEN,
                 "haar_optimal": LEMPS_UNRAVEL_HAAR_OPT}

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)

EXPORTED = ["sim_create", "apply_layer", "unravel_opt", "sample_branch", "measure", "sim_export_mps", "sim_waves",
            "sim_sync", "sim_profile", "sim_tiles", "destroy", "unravel_grad", "unravel_descend", "unravel_grad_noalloc",
            "sample_bitstrings", "eps_concentrated", "lemps_last_error"]
KERNEL_KINDS = ["move", "contract", "unravel", "gram", "eig", "split", "other"]


class LempsError(RuntimeError):
    def __init__(self, status, where, msg):
        super().__init__(f"{where}: status {status}: {msg}")
        self.status = status


class Config(ctypes.Structure):
    _fields_ = [("n_qubits", ctypes.c_int32), ("chi_max", ctypes.c_int32), ("trunc_cutoff", ctypes.c_double),
                ("n_traj", ctypes.c_int64), ("traj_offset", ctypes.c_int64), ("seed", ctypes.c_uint64),
                ("precision", ctypes.c_int32), ("unravel_mode", ctypes.c_int32), ("log_capacity", ctypes.c_int32),
                ("eps_max", ctypes.c_double), ("cuda_stream", ctypes.c_void_p), ("alloc", ALLOC_FN),
                ("free", FREE_FN), ("alloc_ctx", ctypes.c_void_p), ("layering", ctypes.c_int32),
                ("max_traj_in_flight", ctypes.c_int64), ("eigvec_fp64", ctypes.c_int32),
                ("gemm_tile", ctypes.c_int32), ("big_kernels", ctypes.c_int32)]


class LayerStruct(ctypes.Structure):
    _fields_ = [("n_gates", ctypes.c_int32), ("left_qubit", ctypes.POINTER(ctypes.c_int32)),
                ("gates", ctypes.POINTER(ctypes.c_double)), ("n_kraus", ctypes.c_int32),
                ("kraus", ctypes.POINTER(ctypes.c_double)), ("coin_p", ctypes.c_double)]


_DP = ctypes.POINTER(ctypes.c_double)


class Measurement(ctypes.Structure):
    _fields_ = [("z", _DP), ("zz", _DP), ("s_half", _DP), ("eps_bound", _DP),
                ("status", ctypes.POINTER(ctypes.c_int32)), ("z_mean", _DP), ("z_stderr", _DP),
                ("zz_mean", _DP), ("zz_stderr", _DP), ("s_half_mean", ctypes.c_double),
                ("s_half_stderr", ctypes.c_double), ("eps_hat", ctypes.c_double), ("eps_buffer", ctypes.c_double),
                ("n_failed", ctypes.c_int64)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load liblemps.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"{path} is missing: build it with paper_2508_05745_gb300.build.build()")
        _build.build()
    lib = ctypes.CDLL(path)
    vp, i32, i64, dp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, _DP
    lib.sim_create.argtypes = [ctypes.POINTER(Config), ctypes.POINTER(vp)]
    lib.apply_layer.argtypes = [vp, ctypes.POINTER(LayerStruct)]
    lib.unravel_opt.argtypes = [vp, vp, i32, i64, vp, vp, vp]
    lib.sample_branch.argtypes = [vp, i64, i32, ctypes.POINTER(i32)]
    lib.measure.argtypes = [vp, ctypes.POINTER(Measurement)]
    lib.sim_export_mps.argtypes = [vp, i64, ctypes.POINTER(i32), dp]
    lib.sample_bitstrings.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_uint8)]
    lib.eps_concentrated.argtypes = [vp, i32, ctypes.c_double, dp, dp]
    lib.sim_sync.argtypes = [vp]
    lib.sim_waves.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i32)]
    lib.sim_profile.argtypes = [vp, i32, dp, ctypes.POINTER(i64)]
    lib.sim_tiles.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), dp]
    lib.destroy.argtypes = [vp]
    lib.unravel_grad.argtypes = [vp, i32, i64, i32, vp, vp, vp, vp, vp, vp]
    lib.unravel_descend.argtypes = [vp, vp, i64, i32, ctypes.c_double, vp, vp, vp]
    lib.unravel_grad_noalloc.argtypes = [vp, i32, i64, i32, vp, vp, vp, vp, vp]
    lib.lemps_last_error.restype = ctypes.c_char_p
    for name in EXPORTED[:-1]:
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(status, where):
    if status != LEMPS_OK:
        raise LempsError(status, where, load().lemps_last_error().decode())


def _require_cuda():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("lemps needs a CUDA GPU; there is no CPU fallback")
    return torch


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


class Simulation:
    """Handle of a batch of MPS trajectories (sim_create ... destroy)."""

    def __init__(self, n_qubits: int, chi_max: int, n_traj: int, seed: int = 0, precision: str = "fp64",
                 unravel: str = "optimal", cutoff: Optional[float] = None, traj_offset: int = 0,
                 log_capacity: int = 0, eps_max: float = 4.0, stream=None, torch_allocator: bool = True,
                 layering: str = "local", max_traj_in_flight: int = 0, eigvec_fp64: bool = False,
                 gemm_tile: int = 0, big_kernels: bool = False):
        torch = _require_cuda()
        lib = load()
        self.n, self.chi, self.B = int(n_qubits), int(chi_max), int(n_traj)
        self.precision = precision
        if cutoff is None:
            cutoff = 1e-20 if precision == "fp64" else 1e-12
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        cfg = Config()
        cfg.n_qubits, cfg.chi_max, cfg.trunc_cutoff = self.n, self.chi, float(cutoff)
        cfg.n_traj, cfg.traj_offset, cfg.seed = self.B, int(traj_offset), int(seed)
        cfg.precision = LEMPS_FP64 if precision == "fp64" else LEMPS_MIXED
        if unravel not in UNRAVEL_MODES:
            raise ValueError(f"unravel must be one of {sorted(UNRAVEL_MODES)}")
        cfg.unravel_mode = UNRAVEL_MODES[unravel]
        if layering not in LAYERINGS:
            raise ValueError(f"layering must be one of {sorted(LAYERINGS)}")
        cfg.layering = LAYERINGS[layering]
        cfg.log_capacity = int(log_capacity)
        cfg.eps_max = float(eps_max)
        cfg.max_traj_in_flight = int(max_traj_in_flight)
        cfg.eigvec_fp64 = 1 if eigvec_fp64 else 0
        cfg.gemm_tile = int(gemm_tile)
        cfg.big_kernels = 1 if big_kernels else 0
        cfg.cuda_stream = self.stream.cuda_stream
        self._cb = None
        if torch_allocator:
            dev = torch.cuda.current_device()

            def _alloc(nbytes, stream, ctx):
                return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream or 0)

            def _free(ptr, nbytes, stream, ctx):
                torch.cuda.caching_allocator_delete(ptr)

            self._cb = (ALLOC_FN(_alloc), FREE_FN(_free))
            cfg.alloc, cfg.free = self._cb
        self._h = ctypes.c_void_p()
        _check(lib.sim_create(ctypes.byref(cfg), ctypes.byref(self._h)), "sim_create")
        self.gates_applied = 0

    def apply_layer(self, layer) -> None:
        q = np.ascontiguousarray(layer.left_qubits, dtype=np.int32)
        g = np.ascontiguousarray(layer.gates, dtype=np.complex128)
        k = np.ascontiguousarray(layer.kraus, dtype=np.complex128)
        ls = LayerStruct(len(q), _ptr(q, ctypes.c_int32), _ptr(g.view(np.float64), ctypes.c_double),
                         k.shape[0], _ptr(k.view(np.float64), ctypes.c_double), float(layer.coin_p))
        _check(load().apply_layer(self._h, ctypes.byref(ls)), "apply_layer")
        self.gates_applied += len(q)

    def run(self, circuit) -> None:
        for layer in circuit.layers:
            self.apply_layer(layer)

    def sample_bitstrings(self, n_shots: int) -> np.ndarray:
        """[n_traj, n_shots, n] uint8 computational-basis samples of every
        trajectory's current state (sample_bitstrings)."""
        out = np.empty((self.B, int(n_shots), self.n), dtype=np.uint8)
        _check(load().sample_bitstrings(self._h, int(n_shots), _ptr(out, ctypes.c_uint8)), "sample_bitstrings")
        return out

    def eps_concentrated(self, kind: str, param: float):
        """(per-trajectory bounds, mean) of the concentration-improved error
        bound; kind "alpha" (param = alpha) or "depolarizing" (param = p)."""
        k = {"alpha": 0, "depolarizing": 1}[kind]
        out = np.empty(self.B, dtype=np.float64)
        hat = ctypes.c_double(0.0)
        _check(load().eps_concentrated(self._h, k, float(param), _ptr(out, ctypes.c_double), ctypes.byref(hat)),
               "eps_concentrated")
        return out, hat.value

    def sample_branch(self, gate: int, slot: int) -> np.ndarray:
        out = np.empty(self.B, dtype=np.int32)
        _check(load().sample_branch(self._h, gate, slot, _ptr(out, ctypes.c_int32)), "sample_branch")
        return out

    def measure(self, per_trajectory: bool = True) -> dict:
        n, B = self.n, self.B
        res = {k: np.zeros(s) for k, s in [("z_mean", n), ("z_stderr", n), ("zz_mean", n - 1), ("zz_stderr", n - 1)]}
        m = Measurement()
        if per_trajectory:
            res.update(z=np.zeros((B, n)), zz=np.zeros((B, n - 1)), s_half=np.zeros(B), eps_bound=np.zeros(B),
                       status=np.zeros(B, dtype=np.int32))
            m.z, m.zz = _ptr(res["z"], ctypes.c_double), _ptr(res["zz"], ctypes.c_double)
            m.s_half, m.eps_bound = _ptr(res["s_half"], ctypes.c_double), _ptr(res["eps_bound"], ctypes.c_double)
            m.status = _ptr(res["status"], ctypes.c_int32)
        for key in ("z_mean", "z_stderr", "zz_mean", "zz_stderr"):
            setattr(m, key, _ptr(res[key], ctypes.c_double))
        st = load().measure(self._h, ctypes.byref(m))
        res.update(s_half_mean=m.s_half_mean, s_half_stderr=m.s_half_stderr, eps_hat=m.eps_hat,
                   eps_buffer=m.eps_buffer, n_failed=m.n_failed, status_code=st)
        if st not in (LEMPS_OK, LEMPS_ENUMERIC):
            _check(st, "measure")
        return res

    def export_mps(self, traj: int):
        bonds = np.zeros(self.n + 1, dtype=np.int32)
        buf = np.zeros(2 * self.n * 2 * self.chi * self.chi, dtype=np.float64)
        _check(load().sim_export_mps(self._h, traj, _ptr(bonds, ctypes.c_int32), _ptr(buf, ctypes.c_double)),
               "sim_export_mps")
        z = buf.view(np.complex128)
        out, off = [], 0
        for k in range(self.n):
            size = bonds[k] * 2 * bonds[k + 1]
            out.append(z[off:off + size].reshape(bonds[k], 2, bonds[k + 1]).copy())
            off += size
        return out, bonds

    def waves(self):
        """(wave size, number of waves) of the handle (sim_waves)."""
        size, count = ctypes.c_int64(0), ctypes.c_int32(0)
        _check(load().sim_waves(self._h, ctypes.byref(size), ctypes.byref(count)), "sim_waves")
        return size.value, count.value

    def sync(self) -> int:
        return load().sim_sync(self._h)

    def tiles(self):
        """GEMM tile shapes of the handle (sim_tiles): {"contract", "gram_left",
        "gram_right"} -> int32 [n-1, 2] (rows, columns of the output tile per
        gate position; (0, 0) where the tensor-core contraction runs), and
        "tune_ms", the time sim_create spent timing candidates."""
        m = np.zeros(3 * (self.n - 1), dtype=np.int32)
        k = np.zeros(3 * (self.n - 1), dtype=np.int32)
        ms = ctypes.c_double(0.0)
        _check(load().sim_tiles(self._h, _ptr(m, ctypes.c_int32), _ptr(k, ctypes.c_int32), ctypes.byref(ms)),
               "sim_tiles")
        shape = np.stack([m, k], axis=1).reshape(3, self.n - 1, 2)
        return {"contract": shape[0], "gram_left": shape[1], "gram_right": shape[2], "tune_ms": ms.value}

    def profile(self, enable: bool, collect: bool = False):
        """Start/stop CUDA-event timing of every kernel launch; with collect=True
        return {kind: (total_ms, launches)}."""
        ms = np.zeros(len(KERNEL_KINDS))
        n = np.zeros(len(KERNEL_KINDS), dtype=np.int64)
        _check(load().sim_profile(self._h, 1 if enable else 0, _ptr(ms, ctypes.c_double) if collect else None,
                                  _ptr(n, ctypes.c_int64) if collect else None), "sim_profile")
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(KERNEL_KINDS)} if collect else None

    def destroy(self) -> None:
        if self._h:
            _check(load().destroy(self._h), "destroy")
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


# --- functions named after the C entry points ---------------------------------------

def sim_create(**kw) -> Simulation:
    return Simulation(**kw)


def apply_layer(sim: Simulation, layer) -> None:
    sim.apply_layer(layer)


def sample_branch(sim: Simulation, gate: int, slot: int) -> np.ndarray:
    return sim.sample_branch(gate, slot)


def sample_bitstrings(sim: Simulation, n_shots: int) -> np.ndarray:
    return sim.sample_bitstrings(n_shots)


def eps_concentrated(sim: Simulation, kind: str, param: float):
    return sim.eps_concentrated(kind, param)


def measure(sim: Simulation, per_trajectory: bool = True) -> dict:
    return sim.measure(per_trajectory)


def sim_tiles(sim: Simulation) -> dict:
    return sim.tiles()


def destroy(sim: Simulation) -> None:
    sim.destroy()


def unravel_opt(rho_a, kraus):
    """rho_a: cuda complex128 [B, 2, 2]; kraus: cuda complex128 [r, 2, 2].
    Returns (kraus_out [B, 4, 2, 2], e_av [B]) as cuda tensors."""
    torch = _require_cuda()
    rho_a = rho_a.contiguous()
    kraus = kraus.contiguous()
    B = rho_a.shape[0]
    kout = torch.empty((B, 4, 2, 2), dtype=torch.complex128, device=rho_a.device)
    e_av = torch.empty(B, dtype=torch.float64, device=rho_a.device)
    st = torch.cuda.current_stream().cuda_stream
    _check(load().unravel_opt(rho_a.data_ptr(), kraus.data_ptr(), kraus.shape[0], B, kout.data_ptr(),
                              e_av.data_ptr(), st), "unravel_opt")
    return kout, e_av


def unravel_grad(theta, p, h, want_grad: bool = True):
    """theta: cuda complex64/complex128 [B, chi, 2, 2, chi]; p: cuda float64 [B];
    h: cuda complex128 [B, 4, 4].  Returns (cost [B], grad [B,4,4] or None, rho [B,2,2])."""
    torch = _require_cuda()
    theta = theta.contiguous()
    B, chi = theta.shape[0], theta.shape[1]
    cost = torch.empty(B, dtype=torch.float64, device=theta.device)
    grad = torch.empty((B, 4, 4), dtype=torch.complex128, device=theta.device) if want_grad else None
    rho = torch.empty((B, 2, 2), dtype=torch.complex128, device=theta.device)
    st = torch.cuda.current_stream().cuda_stream
    _check(load().unravel_grad(theta.data_ptr(), 1 if theta.dtype == torch.complex128 else 0, B, chi,
                               p.contiguous().data_ptr(), h.contiguous().data_ptr(), cost.data_ptr(),
                               grad.data_ptr() if grad is not None else None, rho.data_ptr(), st), "unravel_grad")
    return cost, grad, rho


def unravel_descend(rho, p, h, steps: int, lr: float, trace: bool = True):
    """Gradient descent on the device; returns (h_new, cost_trace [steps, B])."""
    torch = _require_cuda()
    h = h.clone().contiguous()
    B = rho.shape[0]
    tr = torch.empty((steps, B), dtype=torch.float64, device=rho.device) if trace else None
    st = torch.cuda.current_stream().cuda_stream
    _check(load().unravel_descend(rho.contiguous().data_ptr(), p.contiguous().data_ptr(), B, steps, float(lr),
                                  h.data_ptr(), tr.data_ptr() if tr is not None else None, st), "unravel_descend")
    return h, tr


class UnravelCost:
    """torch.autograd.Function exposing E(H) with the hand-written adjoint."""

    @staticmethod
    def function():
        import torch

        class _F(torch.autograd.Function):
            @staticmethod
            def forward(ctx, h, theta, p):
                cost, grad, _ = unravel_grad(theta, p, h.detach(), want_grad=True)
                ctx.save_for_backward(grad)
                return cost

            @staticmethod
            def backward(ctx, gout):
                (grad,) = ctx.saved_tensors
                return gout.to(grad.dtype)[:, None, None] * grad, None, None

        return _F
