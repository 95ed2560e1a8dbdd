"""Loader of the OpenMP C reference step (oracle/c/lbm_ref.c): the Shan-Chen
step of Sec. 2 (SRT with the velocity shift, or MRT with Guo forcing) in
plain FP64 C, for timing the method on all host cores beside the numpy
oracle.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``.  `build()` compiles
``oracle/liblbm_ref.so`` with the host C compiler (gcc -fopenmp); `run_srt`
takes populations in the numpy oracle's layout and velocity order.
"""

from __future__ import annotations

import ctypes
import os
import shutil
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "c", "lbm_ref.c")
LIB = os.path.join(HERE, "liblbm_ref.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile liblbm_ref.so if missing or older than its source."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("no C compiler for the C reference")
    tmp = LIB + ".tmp"
    subprocess.run([cc, "-std=c99", "-O2", "-fopenmp", "-fPIC", "-shared", SRC, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, LIB)
    return LIB


def load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.lbm_ref_run_srt.restype = ctypes.c_int
        _lib.lbm_ref_run_srt.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int]
        _lib.lbm_ref_run_mrt.restype = ctypes.c_int
        _lib.lbm_ref_run_mrt.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_double, ctypes.c_void_p, ctypes.c_double, ctypes.c_int]
        _lib.lbm_ref_threads.restype = ctypes.c_int
    return _lib


def threads() -> int:
    return int(load().lbm_ref_threads())


def run_srt(f, steps, G, tau, rho0=1.0):
    """`steps` SRT steps of populations f (19, nz, ny, nx), float64."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty_like(f)
    _, nz, ny, nx = f.shape
    st = load().lbm_ref_run_srt(f.ctypes.data, out.ctypes.data, nx, ny, nz, float(G), float(tau), float(rho0),
                                int(steps))
    if st != 0:
        raise MemoryError("C reference: allocation failed")
    return out


def run_mrt(f, steps, G, rates, rho0=1.0):
    """`steps` MRT steps (Guo forcing, 19 rates in moment order) of
    populations f (19, nz, ny, nx), float64."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    s = np.ascontiguousarray(rates, dtype=np.float64)
    if s.shape != (19,):
        raise ValueError("rates: 19 values")
    out = np.empty_like(f)
    _, nz, ny, nx = f.shape
    st = load().lbm_ref_run_mrt(f.ctypes.data, out.ctypes.data, nx, ny, nz, float(G), s.ctypes.data, float(rho0),
                                int(steps))
    if st != 0:
        raise MemoryError("C reference: allocation failed")
    return out
