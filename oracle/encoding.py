"""Canonical-embedding encode / decode for CKKS, float64 numpy (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Slot j of a plaintext m(X) in Z[X]/(X^N+1) is m(zeta^(5^j mod 2N)) / scale
with zeta = exp(i*pi/N), j < N/2 (CKKS, Cheon-Kim-Kim-Song 2017; the paper's
Sect. 2.1 assumes this SIMD packing and its rotations, App. D).

Derivation used here.  Write w_k = m_k + i*m_(k+N/2) for k < h = N/2.  Since
zeta^(5^j*N/2) = i for every j, slot_j = sum_k w_k * xi_j^k with
xi_j = zeta^(4*l+1), l = (5^j mod 2N - 1)/4.  With b_k = w_k*zeta^k this is a
length-h DFT: A_l = sum_k b_k * exp(2*pi*i*l*k/h), so decode is
twist -> h*ifft -> gather and encode is scatter -> fft/h -> untwist -> round.
``encode_bruteforce`` / ``decode_bruteforce`` evaluate the defining sums directly
(O(N^2)); tests pin the FFT forms to them.
"""
import numpy as np


def slot_to_l(log_n: int) -> np.ndarray:
    """l(j) = (5^j mod 2N - 1)/4 for j < N/2."""
    n = 1 << log_n
    h = n // 2
    out = np.empty(h, dtype=np.int64)
    g = 1
    for j in range(h):
        out[j] = (g - 1) // 4
        g = (g * 5) % (2 * n)
    return out


def _rot_exponents(log_n: int) -> np.ndarray:
    n = 1 << log_n
    h = n // 2
    out = np.empty(h, dtype=np.int64)
    g = 1
    for j in range(h):
        out[j] = g
        g = (g * 5) % (2 * n)
    return out


def encode_real_values(z, log_n: int, scale: float) -> np.ndarray:
    """Slots (complex or real, length <= N/2, zero-filled) -> unrounded coefficients * scale."""
    n = 1 << log_n
    h = n // 2
    zz = np.zeros(h, dtype=np.complex128)
    z = np.asarray(z)
    zz[: len(z)] = z
    A = np.empty(h, dtype=np.complex128)
    A[slot_to_l(log_n)] = zz
    b = np.fft.fft(A) / h
    k = np.arange(h)
    w = b * np.exp(-1j * np.pi * k / n)
    m = np.empty(n, dtype=np.float64)
    m[:h] = w.real * scale
    m[h:] = w.imag * scale
    return m


def encode(z, log_n: int, scale: float) -> np.ndarray:
    """Integer plaintext (integer-valued float64 array of length N), round-half-even."""
    return np.rint(encode_real_values(z, log_n, scale))


def decode(m, log_n: int, scale: float) -> np.ndarray:
    """Coefficients (float64, centred) -> complex slots."""
    n = 1 << log_n
    h = n // 2
    m = np.asarray(m, dtype=np.float64)
    w = m[:h] + 1j * m[h:]
    k = np.arange(h)
    b = w * np.exp(1j * np.pi * k / n)
    A = np.fft.ifft(b) * h
    return A[slot_to_l(log_n)] / scale


def encode_bruteforce(z, log_n: int, scale: float) -> np.ndarray:
    """w_k = (scale/h) * sum_j z_j * xi_j^(-k), by the defining sum (small N only)."""
    n = 1 << log_n
    h = n // 2
    zz = np.zeros(h, dtype=np.complex128)
    z = np.asarray(z)
    zz[: len(z)] = z
    e = _rot_exponents(log_n)
    k = np.arange(h)
    ang = -np.pi * ((np.outer(e, k)) % (2 * n)) / n          # exact integer angles
    w = (zz[:, None] * np.exp(1j * ang)).sum(axis=0) * scale / h
    m = np.empty(n)
    m[:h] = w.real
    m[h:] = w.imag
    return m


def decode_bruteforce(m, log_n: int, scale: float) -> np.ndarray:
    """slot_j = sum_k m_k * zeta^(k * 5^j) / scale, by the defining sum (small N only)."""
    n = 1 << log_n
    e = _rot_exponents(log_n)
    k = np.arange(n)
    ang = np.pi * ((np.outer(e, k)) % (2 * n)) / n
    return (np.exp(1j * ang) * np.asarray(m, dtype=np.float64)[None, :]).sum(axis=1) / scale
