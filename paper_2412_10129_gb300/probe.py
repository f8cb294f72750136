"""Python binding of libtgprobe (include/tg_probe.h): measured gather rates
that bound the interpolated projector and its transpose.

``python -m paper_2412_10129_gb300.probe`` prints one JSON line with every
rate on the current device."""
from __future__ import annotations

import ctypes
import json
import os

_lib = None


def load():
    global _lib
    if _lib is None:
        from .build import PROBE_PATH
        if not os.path.exists(PROBE_PATH):
            raise RuntimeError(f"{PROBE_PATH} is missing: run paper_2412_10129_gb300.build.build() first")
        lib = ctypes.CDLL(PROBE_PATH)
        D = ctypes.POINTER(ctypes.c_double)
        lib.tgp_sector_gather.argtypes = [ctypes.c_size_t, ctypes.c_int, D, D]
        lib.tgp_tex_gather.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, D, D]
        lib.tgp_smem_atomic.argtypes = [ctypes.c_int, ctypes.c_int, D, D]
        lib.tgp_smem_atomic_kind.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, D, D]
        _lib = lib
    return _lib


def sector_gather(nbytes: int, reps: int = 10) -> dict:
    """Random 32-byte sectors over a working set of `nbytes` through L2."""
    gbs, ms = ctypes.c_double(), ctypes.c_double()
    rc = load().tgp_sector_gather(int(nbytes), int(reps), ctypes.byref(gbs), ctypes.byref(ms))
    if rc:
        raise RuntimeError(f"tgp_sector_gather failed: cudaError {rc}")
    return {"working_set_bytes": int(nbytes), "gbs": gbs.value, "sectors_per_s": gbs.value * 1e9 / 32.0,
            "ms_per_launch": ms.value}


def tex_gather(nx: int, ny: int, nlayers: int, coherent: bool, reps: int = 10) -> dict:
    """2x2 texture gathers (tld4) from an nx x ny x nlayers layered array."""
    rate, ms = ctypes.c_double(), ctypes.c_double()
    rc = load().tgp_tex_gather(int(nx), int(ny), int(nlayers), 1 if coherent else 0, int(reps), ctypes.byref(rate),
                               ctypes.byref(ms))
    if rc:
        raise RuntimeError(f"tgp_tex_gather failed: cudaError {rc}")
    return {"array": [int(nx), int(ny), int(nlayers)], "bytes": 4 * int(nx) * int(ny) * int(nlayers),
            "coherent": bool(coherent), "gathers_per_s": rate.value, "ms_per_launch": ms.value}


def smem_atomic(random: bool, reps: int = 10, kind: str = "u32") -> dict:
    """Shared-memory atomic adds (u32, u64 or f32 words): conflict-free or random words."""
    rate, ms = ctypes.c_double(), ctypes.c_double()
    k = {"u32": 0, "u64": 1, "f32": 2, "load": 3}[kind]
    rc = load().tgp_smem_atomic_kind(k, 1 if random else 0, int(reps), ctypes.byref(rate), ctypes.byref(ms))
    if rc:
        raise RuntimeError(f"tgp_smem_atomic_kind failed: cudaError {rc}")
    return {"kind": kind, "random": bool(random), "atomics_per_s": rate.value, "ms_per_launch": ms.value}


def gather_rates() -> dict:
    """The rates a projector roofline needs: L2-resident (64 MiB) and
    HBM-resident (2 GiB) random sector gathers; warp-coherent and random
    texture gathers from an L2-resident 64 MiB layered array and from an
    L1-resident 64 KB one; conflict-free and random shared-memory atomics."""
    return {"l2_sector": sector_gather(64 << 20), "hbm_sector": sector_gather(2 << 30, reps=3),
            "tex_coherent": tex_gather(512, 512, 64, True), "tex_random": tex_gather(512, 512, 64, False),
            "tex_coherent_l1": tex_gather(64, 64, 4, True), "tex_random_l1": tex_gather(64, 64, 4, False),
            "smem_atomic_conflict_free": smem_atomic(False), "smem_atomic_random": smem_atomic(True),
            "smem_atomic_u64_conflict_free": smem_atomic(False, kind="u64"),
            "smem_atomic_u64_random": smem_atomic(True, kind="u64"),
            "smem_atomic_f32_conflict_free": smem_atomic(False, kind="f32"),
            "smem_atomic_f32_random": smem_atomic(True, kind="f32"),
            "smem_load_conflict_free": smem_atomic(False, kind="load"),
            "smem_load_random": smem_atomic(True, kind="load")}


if __name__ == "__main__":
    from . import build
    build.build()
    print(json.dumps(gather_rates()), flush=True)
