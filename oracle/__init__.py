"""Dense FP64 CPU oracle for the non-iterative type-4/5 NUFFT (test infrastructure).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product library
never imports, links or runs anything here, and this package imports nothing
from the product package.

What it computes (the plain definitions, no fast algorithm):

* ``type1(x, a)``     A_k = sum_p a_p e^{-j2pi k t_p}, k = 0..P-1        (Sec. II, Eq. 32)
* ``type1_at(x,a,ks)`` the same sum at a list of integer frequencies
* ``type2(x, S)``     s_p = sum_m S_m e^{+j2pi m t_p}, m = 0..P-1        (Sec. II, Eq. 34)
* ``type2_at(x,S,ms)`` the same sum with the coefficients at a list of integer frequencies
* ``inv5(x, s)``      solves Eq. 48 for S by Gaussian elimination (LU with
                      partial pivoting, the paper's GE benchmark of Sec. VI)
* ``inv4(x, A)``      solves Eq. 47 for a by the same LU on G^H
* ``kernel_samples``  K_q = L(rho e^{j2pi q/P}) = prod_p (z_q - z_p)     (Eqs. 10, 11)
* ``deriv_samples``   D_p = L'(z_p) = prod_{q!=p} (z_p - z_q)            (Sec. III-D)
* ``weights``         w_p = h(-P t_p + jPa)/(L'(z_p) z_p)                (Eqs. 17, 27, 40)
* ``inv5_vjp``, ``inv4_vjp``  gradients of a real loss through the inverses
                      (dense LU and direct sums; pinned by finite differences)

Nodes are given in radians (x) and canonicalised exactly as
``t = x/(2 pi) mod 1``, ``T = trunc(t 2^64)``; all phases are formed from the
integer ``m*T mod 2^64`` (exact), so only one libm sin/cos rounds per term.

Pins: every function is checked in ``tests/test_oracle_pins.py`` against
closed forms (equispaced nodes reduce every transform to numpy's DFT and the
kernel to z^P - 1), brute-force pure-Python sums on tiny inputs, hand-derived
values in ``tests/golden/``, round trips with known truth, the type-4/5
duality, the translation law, and numpy's independent polynomial routines for
L and L' on small P.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force=False):
    """Compile oracle.c into liboracle.so (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        d = ctypes.c_double
        lib.oracle_canon.argtypes = [i64, P, P, P]
        lib.oracle_type1.argtypes = [i64, P, P, i64, i64, P]
        lib.oracle_type2.argtypes = [i64, i64, P, i64, P, P]
        lib.oracle_matrix.argtypes = [i64, P, P]
        lib.oracle_kernel_samples.argtypes = [i64, P, d, P]
        lib.oracle_deriv_samples.argtypes = [i64, P, P]
        lib.oracle_weights.argtypes = [i64, P, d, P, P]
        lib.oracle_type1_at.argtypes = [i64, P, P, i64, P, P]
        lib.oracle_type2_at.argtypes = [i64, P, P, i64, P, P]
        for f in (lib.oracle_canon, lib.oracle_type1, lib.oracle_type2, lib.oracle_matrix,
                  lib.oracle_kernel_samples, lib.oracle_deriv_samples, lib.oracle_weights, lib.oracle_type1_at,
                  lib.oracle_type2_at):
            f.restype = None
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c128(v):
    return np.ascontiguousarray(np.asarray(v, dtype=np.complex128))


def canon(x):
    """Radians -> (T uint64 fixed-point turns, t float64 in [0,1))."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    T = np.empty(x.size, dtype=np.uint64)
    t = np.empty(x.size, dtype=np.float64)
    _load().oracle_canon(x.size, _ptr(x), _ptr(T), _ptr(t))
    return T, t


def type1(x, a, k0=0, M=None):
    """Eq. 32: A_k = sum_p a_p e^{-j 2 pi k t_p}, k = k0 .. k0+M-1 (default 0..P-1)."""
    T, _ = canon(x)
    a = _c128(a)
    M = T.size if M is None else M
    A = np.empty(M, dtype=np.complex128)
    _load().oracle_type1(T.size, _ptr(T), _ptr(a), k0, M, _ptr(A))
    return A


def type1_at(x, a, ks):
    """Eq. 32 at the integer frequencies ks: A_k = sum_p a_p e^{-j 2 pi k t_p}."""
    T, _ = canon(x)
    a = _c128(a)
    ks = np.ascontiguousarray(np.asarray(ks, dtype=np.int64))
    A = np.empty(ks.size, dtype=np.complex128)
    _load().oracle_type1_at(T.size, _ptr(T), _ptr(a), ks.size, _ptr(ks), _ptr(A))
    return A


def type2(x, S, m0=0):
    """Eq. 34: s_q = sum_m S_m e^{+j 2 pi (m0+m) t_q} at every node."""
    T, _ = canon(x)
    S = _c128(S)
    s = np.empty(T.size, dtype=np.complex128)
    _load().oracle_type2(S.size, m0, _ptr(S), T.size, _ptr(T), _ptr(s))
    return s


def type2_at(x, S, ms):
    """Eq. 34 with coefficient S_i at the integer frequency ms[i]:
    s_q = sum_i S_i e^{+j 2 pi ms[i] t_q} at every node."""
    T, _ = canon(x)
    S = _c128(S)
    ms = np.ascontiguousarray(np.asarray(ms, dtype=np.int64))
    assert ms.size == S.size
    s = np.empty(T.size, dtype=np.complex128)
    _load().oracle_type2_at(ms.size, _ptr(ms), _ptr(S), T.size, _ptr(T), _ptr(s))
    return s


def matrix(x):
    """G_{q,m} = e^{j 2 pi m t_q} (the type-5 system matrix of Eq. 48)."""
    T, _ = canon(x)
    G = np.empty((T.size, T.size), dtype=np.complex128)
    _load().oracle_matrix(T.size, _ptr(T), _ptr(G))
    return G


def inv5(x, s):
    """Type-5 (Eq. 48): S with G S = s, by LU with partial pivoting (GE)."""
    G = matrix(x)
    return np.linalg.solve(G, _c128(s))


def inv4(x, A):
    """Type-4 (Eq. 47): a with G^H a = A (the type-1 matrix is G^H), by LU."""
    G = matrix(x)
    return np.linalg.solve(G.conj().T, _c128(A))


def rho_of_gamma(P, gamma):
    """rho = e^{-2 pi a} with the shift a chosen so that rho^{-P} = gamma."""
    return float(np.exp(-np.log(gamma) / P))


def kernel_samples(x, rho):
    """Eq. 10: K_q = L(z_q), z_q = rho e^{j 2 pi q/P}, L(z) = prod_p (z - z_p) (Eq. 11)."""
    T, _ = canon(x)
    K = np.empty(T.size, dtype=np.complex128)
    _load().oracle_kernel_samples(T.size, _ptr(T), float(rho), _ptr(K))
    return K


def deriv_samples(x):
    """Sec. III-D: D_p = L'(z_p) = prod_{q != p} (z_p - z_q)."""
    T, _ = canon(x)
    D = np.empty(T.size, dtype=np.complex128)
    _load().oracle_deriv_samples(T.size, _ptr(T), _ptr(D))
    return D


def weights(x, rho, D=None):
    """Eqs. 27 / 40: w_p = h(-P t_p + jPa) / (L'(z_p) z_p), h(t) = 1/(e^{j2pi t} - 1)."""
    T, _ = canon(x)
    D = deriv_samples(x) if D is None else _c128(D)
    w = np.empty(T.size, dtype=np.complex128)
    _load().oracle_weights(T.size, _ptr(T), float(rho), _ptr(D), _ptr(w))
    return w


def rel_l2(a, b):
    """The paper's error measure (Sec. VI): ||a - b|| / ||b||."""
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def inv5_vjp(x, f, g_S):
    """Gradient of a real loss through the type-5 inverse S = G^{-1} f (Eq. 48).

    g_S is the loss gradient with respect to S in the convention
    dL = Re<g_S, dS> (PyTorch's).  Returns (g_f, g_x):
      g_f = G^{-H} g_S (the type-4 system of Eq. 47 is G^H),
      dS = -G^{-1} (s' o dt) with s'(t) = sum_m j 2 pi m S_m e^{j 2 pi m t}
      (row q of G depends on t_q only), so dL/dt_q = -Re(conj(g_f[q]) s'(t_q)),
      g_x = dL/dt / (2 pi)  (t = x / 2 pi).
    Dense LU and exact-phase direct sums."""
    G = matrix(x)
    S = np.linalg.solve(G, _c128(f))
    u = np.linalg.solve(G.conj().T, _c128(g_S))
    P = S.size
    sd = type2(x, 2j * np.pi * np.arange(P) * S)
    g_t = -(np.conj(u) * sd).real
    return u, g_t / (2 * np.pi)


def inv4_vjp(x, A, g_a):
    """Gradient of a real loss through the type-4 inverse a = G^{-H} A (Eq. 47).

    dL = Re<g_a, da>.  Returns (g_A, g_x): g_A = G^{-1} g_a; with
    w = g_A and w'(t) = sum_m j 2 pi m w_m e^{j 2 pi m t},
    dL/dt_q = -Re(a_q conj(w'(t_q))) (G^H depends on t_q through column q),
    g_x = dL/dt / (2 pi).  Dense LU and exact-phase direct sums."""
    G = matrix(x)
    a = np.linalg.solve(G.conj().T, _c128(A))
    w = np.linalg.solve(G, _c128(g_a))
    P = a.size
    wd = type2(x, 2j * np.pi * np.arange(P) * w)
    g_t = -(a * np.conj(wd)).real
    return w, g_t / (2 * np.pi)
