"""ctypes loader for the oracle's plain C loops (oracle/c/oracle_ilu.c and
its complex counterpart oracle/c/oracle_ilu_z.c).

Compiles the shared object with gcc on first use when it is missing or older
than its source.  -ffp-contract=off keeps every multiply and add separately
rounded so that results do not depend on the host's FMA contraction rules.
"""
import ctypes
import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "c", "oracle_ilu.c"), os.path.join(_HERE, "c", "oracle_ilu_z.c")]
_LIB = os.path.join(_HERE, "_oracle_ilu.so")
_lib = None


def build():
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-std=c99",
           "-o", _LIB, *_SRCS, "-lm"]
    subprocess.run(cmd, check=True)


class Factors(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64),
                ("lrp", ctypes.POINTER(ctypes.c_int64)),
                ("lci", ctypes.POINTER(ctypes.c_int32)),
                ("lv", ctypes.POINTER(ctypes.c_double)),
                ("urp", ctypes.POINTER(ctypes.c_int64)),
                ("uci", ctypes.POINTER(ctypes.c_int32)),
                ("uv", ctypes.POINTER(ctypes.c_double)),
                ("nclamp", ctypes.c_int64)]


def lib():
    global _lib
    if _lib is None:
        if (not os.path.exists(_LIB)) or any(os.path.getmtime(_LIB) < os.path.getmtime(f) for f in _SRCS):
            build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        L.oracle_ilu0.restype = ctypes.POINTER(Factors)
        L.oracle_ilu0.argtypes = [ctypes.c_int64, P, P, P]
        L.oracle_ilut.restype = ctypes.POINTER(Factors)
        L.oracle_ilut.argtypes = [ctypes.c_int64, P, P, P, ctypes.c_double, ctypes.c_int64]
        L.oracle_free_factors.argtypes = [ctypes.POINTER(Factors)]
        L.oracle_free_factors.restype = None
        for f in (L.oracle_lsolve, L.oracle_usolve, L.oracle_lsolve_z, L.oracle_usolve_z):
            f.argtypes = [ctypes.c_int64, P, P, P, P, P]
            f.restype = None
        # complex factors: the same struct, lv/uv holding (re, im) pairs
        L.oracle_ilu0_z.restype = ctypes.POINTER(Factors)
        L.oracle_ilu0_z.argtypes = [ctypes.c_int64, P, P, P]
        L.oracle_ilut_z.restype = ctypes.POINTER(Factors)
        L.oracle_ilut_z.argtypes = [ctypes.c_int64, P, P, P, ctypes.c_double, ctypes.c_int64]
        L.oracle_free_factors_z.argtypes = [ctypes.POINTER(Factors)]
        L.oracle_free_factors_z.restype = None
        _lib = L
    return _lib
