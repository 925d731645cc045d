"""ctypes binding of the C oracle (hc_oracle.c).  TEST INFRASTRUCTURE ONLY.

Definitions followed (arXiv 2506.11586):
  * ring R_q = Z_q[X]/(X^N+1)                                    Sec. 2.1
  * negacyclic product, schoolbook O(N^2) with the X^N = -1 wrap  App. C
  * NTT as evaluation at psi^(2 rev(k) + 1), INTT its inverse      App. C.1
  * primes, psi: deterministic Miller-Rabin, minimal primitive 2N-th root
    (the paper fixes neither; these are the build's readings)
"""
import ctypes as C
import numpy as np

from . import build_oracle

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build_oracle()
        L = C.CDLL(path)
        u64, u32, sz = C.c_uint64, C.c_uint32, C.c_size_t
        p64 = C.POINTER(C.c_uint64)
        p32 = C.POINTER(C.c_uint32)
        pi64 = C.POINTER(C.c_int64)
        L.or_mulmod.restype = u64; L.or_mulmod.argtypes = [u64, u64, u64]
        L.or_addmod.restype = u64; L.or_addmod.argtypes = [u64, u64, u64]
        L.or_submod.restype = u64; L.or_submod.argtypes = [u64, u64, u64]
        L.or_powmod.restype = u64; L.or_powmod.argtypes = [u64, u64, u64]
        L.or_is_prime.restype = C.c_int; L.or_is_prime.argtypes = [u64]
        L.or_ntt_primes.restype = sz; L.or_ntt_primes.argtypes = [u32, u32, sz, p64]
        L.or_min_psi.restype = u64; L.or_min_psi.argtypes = [u64, u32]
        L.or_bitrev.restype = u32; L.or_bitrev.argtypes = [u32, u32]
        L.or_ntt_direct_at.restype = None
        L.or_ntt_direct_at.argtypes = [p64, u32, u64, u64, p32, sz, p64]
        L.or_intt_direct_at.restype = None
        L.or_intt_direct_at.argtypes = [p64, u32, u64, u64, p32, sz, p64]
        L.or_negacyclic_at.restype = None
        L.or_negacyclic_at.argtypes = [p64, p64, u32, u64, p32, sz, p64]
        L.or_negacyclic_batch.restype = None
        L.or_negacyclic_batch.argtypes = [p64, p64, sz, u32, p64, u32, p64]
        L.or_negacyclic_sparse_at.restype = None
        L.or_negacyclic_sparse_at.argtypes = [p64, p32, pi64, sz, u32, u64, p32, sz, p64]
        L.or_negacyclic_ternary_at.restype = None
        L.or_negacyclic_ternary_at.argtypes = [p64, p32, sz, p32, sz, u32, u64, p32, sz, p64]
        _lib = L
    return _lib


def _p64(a):
    return a.ctypes.data_as(C.POINTER(C.c_uint64))


def _p32(a):
    return a.ctypes.data_as(C.POINTER(C.c_uint32))


def _pi64(a):
    return a.ctypes.data_as(C.POINTER(C.c_int64))


def _u64(a):
    return np.ascontiguousarray(a, dtype=np.uint64)


def _idx(ks):
    if ks is None:
        return None, 0
    k = np.ascontiguousarray(ks, dtype=np.uint32)
    return k, k.size


# ---- scalars ---------------------------------------------------------------

def mulmod(a, b, q):
    return int(lib().or_mulmod(a, b, q))


def powmod(a, e, q):
    return int(lib().or_powmod(a, e, q))


def is_prime(n):
    return bool(lib().or_is_prime(n))


def ntt_primes(bits, log2_step, count):
    """The `count` largest primes q < 2^bits with q = 1 mod 2^log2_step, descending."""
    out = np.zeros(count, dtype=np.uint64)
    n = lib().or_ntt_primes(bits, log2_step, count, _p64(out))
    return [int(x) for x in out[:n]]


def min_psi(q, N):
    """Minimal primitive 2N-th root of unity mod q (0 if none)."""
    return int(lib().or_min_psi(q, N))


def bitrev(k, logn):
    return int(lib().or_bitrev(k, logn))


# ---- transforms by definition ---------------------------------------------

def ntt(a, q, psi, ks=None):
    """out[k] = sum_j a[j] psi^((2 rev(k)+1) j) mod q, at indices ks (all if None)."""
    a = _u64(a)
    N = a.size
    k, nk = _idx(ks)
    out = np.zeros(nk if k is not None else N, dtype=np.uint64)
    lib().or_ntt_direct_at(_p64(a), N, q, psi, _p32(k) if k is not None else None, nk, _p64(out))
    return out


def intt(A, q, psi, js=None):
    """Exact inverse of ntt(): natural-order coefficients, N^-1 folded in."""
    A = _u64(A)
    N = A.size
    j, nj = _idx(js)
    out = np.zeros(nj if j is not None else N, dtype=np.uint64)
    lib().or_intt_direct_at(_p64(A), N, q, psi, _p32(j) if j is not None else None, nj, _p64(out))
    return out


# ---- negacyclic products ---------------------------------------------------

def negacyclic(a, b, q, ks=None):
    """Schoolbook c = a*b in Z_q[X]/(X^N+1), at coefficient indices ks (all if None)."""
    a, b = _u64(a), _u64(b)
    assert a.size == b.size
    N = a.size
    k, nk = _idx(ks)
    out = np.zeros(nk if k is not None else N, dtype=np.uint64)
    lib().or_negacyclic_at(_p64(a), _p64(b), N, q, _p32(k) if k is not None else None, nk, _p64(out))
    return out


def negacyclic_batch(a, b, moduli):
    """Batched dense schoolbook over a [..., L, N] layout; limb l uses moduli[l]."""
    a, b = _u64(a), _u64(b)
    assert a.shape == b.shape
    L, N = a.shape[-2], a.shape[-1]
    assert L == len(moduli)
    n = a.size // N
    qs = _u64(moduli)
    out = np.zeros_like(a)
    lib().or_negacyclic_batch(_p64(a), _p64(b), n, N, _p64(qs), L, _p64(out))
    return out


def sparse_of(b_small):
    """(idx, val) lists of the nonzero coefficients of a small-integer polynomial."""
    b_small = np.asarray(b_small, dtype=np.int64)
    idx = np.nonzero(b_small)[0].astype(np.uint32)
    return idx, b_small[idx].astype(np.int64)


def negacyclic_sparse(a, sparse, N, q, ks=None):
    """a * b mod (X^N+1, q) where b = sum val[t] X^idx[t] has small signed integers."""
    a = _u64(a)
    idx, val = sparse
    idx = np.ascontiguousarray(idx, dtype=np.uint32)
    val = np.ascontiguousarray(val, dtype=np.int64)
    k, nk = _idx(ks)
    out = np.zeros(nk if k is not None else N, dtype=np.uint64)
    lib().or_negacyclic_sparse_at(_p64(a), _p32(idx), _pi64(val), idx.size, N, q,
                                  _p32(k) if k is not None else None, nk, _p64(out))
    return out


def lift_small(b_small, q):
    """Small signed integers -> canonical residues mod q (w mod q, i.e. q + w for w < 0)."""
    b = np.asarray(b_small, dtype=np.int64)
    out = np.where(b >= 0, b, 0).astype(np.uint64)
    neg = b < 0
    out[neg] = np.uint64(q) - (-b[neg]).astype(np.uint64)
    return out


def ternary_of(b_ternary):
    """(+1 index list, -1 index list) of a polynomial with coefficients in {-1, 0, 1}."""
    b = np.asarray(b_ternary, dtype=np.int64)
    assert np.all(np.abs(b) <= 1)
    return (np.nonzero(b == 1)[0].astype(np.uint32), np.nonzero(b == -1)[0].astype(np.uint32))


def negacyclic_ternary(a, tern, N, q, ks=None):
    """a * b mod (X^N+1, q) for ternary b given as ternary_of(b); additions only."""
    a = _u64(a)
    assert a.size == 0 or int(a.max()) < q, "ternary product needs canonical residues"
    pos, neg = (np.ascontiguousarray(x, dtype=np.uint32) for x in tern)
    k, nk = _idx(ks)
    out = np.zeros(nk if k is not None else N, dtype=np.uint64)
    lib().or_negacyclic_ternary_at(_p64(a), _p32(pos), pos.size, _p32(neg), neg.size, N, q,
                                   _p32(k) if k is not None else None, nk, _p64(out))
    return out
