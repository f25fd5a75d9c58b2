"""ctypes binding of libhadamag.so (C ABI in include/hadamag.h).

Argument marshalling only: every step of the computation runs in the library's CUDA
kernels.  There is no CPU fallback: if the shared library is missing or no GPU is present,
calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhadamag.so")

C64, C128 = 0, 1
PATH_AUTO, PATH_CUDACORE, PATH_TENSOR = 0, 1, 2

STATUS = {0: "ok", 1: "invalid argument", 2: "unsupported", 3: "out of memory", 4: "CUDA error",
          5: "device wait timed out", 6: "non-finite result"}

EXPORTS = [
    "hadamag_create", "hadamag_destroy", "hadamag_set_path", "hadamag_set_wait_limit",
    "hadamag_launch_count", "hadamag_status_string", "hadamag_last_error", "hadamag_sre",
    "hadamag_sre_host", "hadamag_sre_terms", "hadamag_mc_xstrings", "hadamag_sre_mc",
    "hadamag_mana", "hadamag_mana_sums", "hadamag_sre_grad", "hadamag_sre_batched",
    "hadamag_sre_noalloc", "hadamag_batched_status", "hadamag_sre_ti", "hadamag_mana_mixed",
    "hadamag_reduced_density_matrix", "hadamag_sre_even_sector", "hadamag_mana_qudit", "hadamag_mana_grad",
    "hadamag_mana_mixed_qudit", "hadamag_reduced_density_matrix_qudit", "hadamag_set_fp32_powers",
    "hadamag_sre_chunk", "hadamag_sre_slice", "hadamag_sre_combine", "hadamag_sre_grad_slice",
    "hadamag_sre_grad_combine", "hadamag_set_autotune", "hadamag_twopass_shape", "hadamag_set_twopass_shape",
    "hadamag_set_grad_xbatch",
]


class HadamagError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str = ""):
        self.code = code
        msg = f"{where}: {STATUS.get(code, code)}"
        if detail:
            msg += f" ({detail})"
        super().__init__(msg)


_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Load libhadamag.so (built in-tree by `paper_2601_07824_gb300.build`)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise ImportError(f"{p} is missing: build it with `python -m paper_2601_07824_gb300.build` "
                              "(the CUDA library is required; there is no CPU fallback)")
        lib = ctypes.CDLL(p)
        V, I, D, L, U64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64, ctypes.c_uint64
        PD, PV = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_void_p)
        sig = {
            "hadamag_create": [ctypes.POINTER(V), I],
            "hadamag_destroy": [V],
            "hadamag_set_path": [V, I],
            "hadamag_set_wait_limit": [V, ctypes.c_longlong, ctypes.c_uint],
            "hadamag_set_fp32_powers": [V, I],
            "hadamag_launch_count": [V, ctypes.POINTER(U64)],
            "hadamag_status_string": [I],
            "hadamag_last_error": [V],
            "hadamag_sre": [V, V, I, D, I, PD, PD, V],
            "hadamag_sre_host": [V, V, I, D, I, PD, PD],
            "hadamag_sre_terms": [V, V, I, D, I, V, L, V, V],
            "hadamag_mc_xstrings": [V, U64, L, I, V, V],
            "hadamag_sre_mc": [V, V, I, L, U64, I, PD, PD, V],
            "hadamag_mana": [V, V, I, I, PD, PD, V],
            "hadamag_mana_sums": [V, V, I, I, PD, V],
            "hadamag_sre_grad": [V, V, I, I, PD, V, V],
            "hadamag_sre_batched": [V, I, PV, ctypes.POINTER(I), I, PV, V, V],
            "hadamag_sre_noalloc": [V, I, D, V, V],
            "hadamag_batched_status": [V, V],
            "hadamag_sre_ti": [V, V, I, I, L, L, U64, D, I, I, PD, PD, PD, V, V],
            "hadamag_sre_even_sector": [V, V, I, D, I, PD, PD, V],
            "hadamag_mana_qudit": [V, V, I, I, I, PD, PD, V],
            "hadamag_mana_grad": [V, V, I, I, I, PD, V, V],
            "hadamag_mana_mixed_qudit": [V, V, I, I, I, PD, PD, V],
            "hadamag_reduced_density_matrix_qudit": [V, V, I, I, I, ctypes.POINTER(I), I, V, V],
            "hadamag_mana_mixed": [V, V, I, I, PD, PD, V],
            "hadamag_reduced_density_matrix": [V, V, I, I, ctypes.POINTER(I), I, V, V],
            "hadamag_sre_chunk": [I],
            "hadamag_set_autotune": [V, I],
            "hadamag_twopass_shape": [V, I, D, ctypes.POINTER(I)],
            "hadamag_set_twopass_shape": [V, I, D, I, I, I, I],
            "hadamag_set_grad_xbatch": [V, I, I],
            "hadamag_sre_slice": [V, V, I, D, I, L, L, V, V],
            "hadamag_sre_combine": [I, D, PD, L, PD, PD],
            "hadamag_sre_grad_slice": [V, V, I, I, L, L, PD, V, V],
            "hadamag_sre_grad_combine": [V, V, I, D, I, PD, V, V],
        }
        for name, args in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            if name in ("hadamag_status_string", "hadamag_last_error"):
                f.restype = ctypes.c_char_p
            elif name == "hadamag_sre_chunk":
                f.restype = L
            else:
                f.restype = I
        _lib = lib
        return lib


class Context:
    """Owns one hadamag_ctx_t on one CUDA device."""

    def __init__(self, device: int = 0):
        self.lib = load()
        self.device = device
        h = ctypes.c_void_p()
        rc = self.lib.hadamag_create(ctypes.byref(h), int(device))
        if rc != 0:
            raise HadamagError(rc, "hadamag_create", f"device {device}")
        self.h = h

    def check(self, rc: int, where: str):
        if rc != 0:
            detail = self.lib.hadamag_last_error(self.h)
            raise HadamagError(rc, where, detail.decode() if detail else "")

    def close(self):
        if getattr(self, "h", None):
            self.lib.hadamag_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def launch_count(self) -> int:
        n = ctypes.c_uint64()
        self.check(self.lib.hadamag_launch_count(self.h, ctypes.byref(n)), "hadamag_launch_count")
        return n.value

    def set_path(self, path: int):
        self.check(self.lib.hadamag_set_path(self.h, int(path)), "hadamag_set_path")
        self.path = int(path)

    def set_fp32_powers(self, on: bool):
        """Opt into FP32 powers for non-integer n (see hadamag_set_fp32_powers)."""
        self.check(self.lib.hadamag_set_fp32_powers(self.h, 1 if on else 0), "hadamag_set_fp32_powers")

    def set_autotune(self, on: bool):
        """Launch-shape autotuning on (default) or off (see hadamag_set_autotune)."""
        self.check(self.lib.hadamag_set_autotune(self.h, 1 if on else 0), "hadamag_set_autotune")

    def twopass_shape(self, N: int, n: float = 2.0):
        """[units per pass-1 warp, tiles per pass-2 task, ring slots, X-strings per batch, lag] in
        use for (N, n); zeros before the tuner ran."""
        out = (ctypes.c_int * 5)()
        self.check(self.lib.hadamag_twopass_shape(self.h, int(N), float(n), out), "hadamag_twopass_shape")
        return list(out)

    def set_twopass_shape(self, N: int, n: float, upw: int, tpt: int, R: int = 0, lag: int = 1):
        """Pin the two-pass shape for (N, n) (see hadamag_set_twopass_shape)."""
        self.check(self.lib.hadamag_set_twopass_shape(self.h, int(N), float(n), int(upw), int(tpt), int(R),
                                                      int(lag)), "hadamag_set_twopass_shape")

    def set_grad_xbatch(self, N: int, A: int):
        """Pin the adjoint's X-strings per batch for N (see hadamag_set_grad_xbatch)."""
        self.check(self.lib.hadamag_set_grad_xbatch(self.h, int(N), int(A)), "hadamag_set_grad_xbatch")

    def set_wait_limit(self, spins: int, bias: int = 0):
        self.check(self.lib.hadamag_set_wait_limit(self.h, int(spins), int(bias)), "hadamag_set_wait_limit")


_contexts: dict[int, Context] = {}


def context(device: int = 0) -> Context:
    with _lock:
        c = _contexts.get(device)
    if c is None:
        c = Context(device)
        with _lock:
            _contexts[device] = c
    return c
