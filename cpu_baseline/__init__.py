"""CPU FFT baseline (timing comparison only; not part of the library).

The same loop as the GPU path (Algorithm 1 of Sec. 3.3, Eq. PC, Eqs. 2-3)
with a project-written radix-2 FFT in FP64 or FP32, one frame per host
thread (fft_gerchberg.cpp). bench.py times it beside the direct-DFT oracle;
tests/test_cpu_baseline.py checks it against the oracle. Nothing in the
package imports it: the library has no CPU path.
"""

import ctypes
import os
import shutil
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(_HERE, "fft_gerchberg.cpp")
LIB = os.path.join(_HERE, "_lib", "libfwr_cpufft.so")

_lib = None


def build():
    """Compile fft_gerchberg.cpp with the host C++ compiler (portable flags)."""
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        raise RuntimeError("no C++ compiler for the CPU FFT baseline")
    tmp = LIB + ".tmp"
    cmd = [cxx, "-O3", "-fcx-limited-range", "-std=c++17", "-shared", "-fPIC", "-pthread", SRC, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("CPU FFT baseline build failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


def load():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            build()
        lib = ctypes.CDLL(LIB)
        P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        lib.fwr_cpu_fft_reconstruct.restype = I
        lib.fwr_cpu_fft_reconstruct.argtypes = [I, P, I, I, P, I, I, I, D, D, D, I, P, I]
        lib.fwr_cpu_fft_threads.restype = I
        lib.fwr_cpu_fft_threads.argtypes = []
        _lib = lib
    return _lib


def threads():
    return load().fwr_cpu_fft_threads()


def next_pow2(x):
    p = 1
    while p < x:
        p *= 2
    return p


def reconstruct(slopes, mask, pad_factor, iters, filt=0, noise_var=0.0, r0=1.0, L0=100.0, periodic=0,
                precision=64, n_threads=0):
    """slopes (F, 2, n, n) or (2, n, n); returns the phase (F, N, N) (or
    (N, N)) as float64. filt 0 = LSQ, 1 = Wiener; r0, L0 in lenslet pitches."""
    lib = load()
    s = np.ascontiguousarray(np.asarray(slopes, dtype=np.float64))
    single = s.ndim == 3
    if single:
        s = s[None]
    F, _, n, _ = s.shape
    m = np.ascontiguousarray(np.asarray(mask).astype(np.uint8))
    N = next_pow2(int(np.ceil(pad_factor * n - 1e-9)))
    out = np.empty((F, N, N), dtype=np.float64)
    rc = lib.fwr_cpu_fft_reconstruct(int(precision), s.ctypes.data, F, n, m.ctypes.data, N, int(iters), int(filt),
                                     float(noise_var), float(r0), float(L0), int(periodic), out.ctypes.data,
                                     int(n_threads))
    if rc != 0:
        raise ValueError("fwr_cpu_fft_reconstruct: bad argument")
    return out[0] if single else out
