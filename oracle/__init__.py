"""CPU oracle for the SecONNds HE-convolution hot path (arXiv 2506.11586).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import anything from this
package.  The GPU library (``paper_2506_11586_gb300``) never imports it, and it
never imports the GPU library: the two share no kernels, headers, helpers,
tables or constants.  Seeded inputs come from ``paper_2506_11586_gb300.inputs``,
which holds random-number generation and workload shapes only.

Contents
  core   -- ctypes binding of ``hc_oracle.c``: Miller-Rabin, prime search,
            minimal psi, NTT/INTT by their O(N^2) definitions, schoolbook
            negacyclic products (dense, sparse-small, sampled coefficients).
  conv   -- Cheetah coefficient packing of a stride-1 convolution, canonical
            partition, plaintext convolution mod t, and the ct x pt conv
            computed by schoolbook products (Sec. 6.1, 6.2).
  layers -- strided convolutions as stride-1 layers of the phase-split input
            (polyphase reading) and fully connected layers by matrix-vector
            packing, with their server steps (Sec. 6.1, Sec. 8.1 networks).
  zp     -- BFV over Z_P with SIMD slots: encoding, Galois automorphisms,
            key-switched slot rotations (one special prime) and the
            multiply-accumulate-rotate iteration of HELiKs-style linear layers
            (SecONNds-P, Sec. 6.1, Sec. 2.3).
  bfv    -- BFV secret-key encryption / decryption (App. C), client-side
            test harness only (Sec. 6.3: the server never holds the key).

Parity status of each function is stated in its module docstring; every
function is pinned by a ``-m "not gpu"`` test under ``tests/``.
"""
import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "hc_oracle.c")


def build_oracle(force: bool = False) -> str:
    """Compile hc_oracle.c with gcc into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(LIB_PATH)
            and os.path.getmtime(LIB_PATH) >= os.path.getmtime(_SRC)):
        return LIB_PATH
    tmp = LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH
