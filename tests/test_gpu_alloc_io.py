"""Host-side plumbing on the GPU: weights checkpoint / resume (hc_weights_save
/ hc_weights_load, every preprocessing mode, bit-exact results, corrupt and
foreign files refused) and the device allocator hook (hc_set_allocator):
PyTorch's caching allocator gives the same bits, and an allocator that runs
out is reported as HC_ERR_OOM without harming the context.  The allocator
cases run in a child process so that no handle outlives the allocator that
made it."""
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from gpu_util import to_dev
from paper_2506_11586_gb300.inputs import CANONICAL_PRIMES, T_PLAIN, Stream, uniform_residues

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_11586_gb300 import _lib
    from paper_2506_11586_gb300.build import build
    build()
    return _lib


def test_weights_save_load_roundtrip(L, tmp_path):
    N, nl = 8192, 3
    ctx = L.hc_ctx_create(N, CANONICAL_PRIMES[:nl], T_PLAIN)
    s = Stream(81, 1)
    C_, H, W, M = 10, 12, 12, 6
    K = s.int8(M * C_ * 9).reshape(M, C_, 3, 3)
    d = L.make_desc(C_, H, W, M, 3, 3, pad=1)
    for mode in range(3):
        w = L.hc_weights_preprocess_ex(ctx, d, K, mode)
        ct = to_dev(uniform_residues(s, CANONICAL_PRIMES[:nl], (w.I, 2), N))
        ref = torch.empty(w.O * 2 * nl * N, dtype=torch.int64, device="cuda")
        L.hc_conv_ct_pt(ctx, w, ct, ref)
        path = tmp_path / ("w%d.bin" % mode)
        L.hc_weights_save(w, path)
        w2 = L.hc_weights_load(ctx, path, like_desc=w.desc)
        assert (w2.I, w2.O) == (w.I, w.O)
        got = torch.empty_like(ref)
        L.hc_conv_ct_pt(ctx, w2, ct, got)
        torch.cuda.synchronize()
        assert torch.equal(got, ref), mode
        # a flipped byte, a truncated file and other ring parameters are refused
        raw = bytearray(path.read_bytes())
        raw[len(raw) // 2] ^= 0x40
        (tmp_path / "bad.bin").write_bytes(bytes(raw))
        with pytest.raises(L.HcError) as e:
            L.hc_weights_load(ctx, tmp_path / "bad.bin")
        assert e.value.status == L.HC_ERR_INVALID_ARG
        (tmp_path / "short.bin").write_bytes(path.read_bytes()[:-20])
        with pytest.raises(L.HcError):
            L.hc_weights_load(ctx, tmp_path / "short.bin")
    other = L.hc_ctx_create(N, CANONICAL_PRIMES[1:nl + 1], T_PLAIN)
    with pytest.raises(L.HcError):
        L.hc_weights_load(other, tmp_path / "w0.bin")
    with pytest.raises(L.HcError):
        L.hc_weights_load(ctx, tmp_path / "missing.bin")


CHILD = textwrap.dedent("""
    import ctypes as C, sys
    import numpy as np, torch
    sys.path.insert(0, sys.argv[1])
    sys.path.insert(0, sys.argv[1] + "/tests")
    from gpu_util import to_dev
    from paper_2506_11586_gb300 import _lib as L
    from paper_2506_11586_gb300.inputs import CANONICAL_PRIMES, T_PLAIN, Stream, uniform_residues

    ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
    FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)
    stats = {"alloc": 0, "free": 0, "refused": 0, "limit": None}

    def torch_alloc(nbytes, stream, user):
        if stats["limit"] is not None and nbytes > stats["limit"]:
            stats["refused"] += 1
            return None
        stats["alloc"] += 1
        return torch.cuda.caching_allocator_alloc(nbytes, 0, stream or 0)

    def torch_free(ptr, stream, user):
        stats["free"] += 1
        torch.cuda.caching_allocator_delete(ptr)

    a, f = ALLOC(torch_alloc), FREE(torch_free)
    N, nl = 8192, 3

    def run(ctx, w, ct):
        out = torch.empty(w.O * 2 * nl * N, dtype=torch.int64, device="cuda")
        L.hc_conv_ct_pt(ctx, w, ct, out)
        torch.cuda.synchronize()
        return out

    s = Stream(82, 1)
    K = s.int8(8 * 16 * 9).reshape(8, 16, 3, 3)
    d = L.make_desc(16, 20, 20, 8, 3, 3, pad=1)
    ctx0 = L.hc_ctx_create(N, CANONICAL_PRIMES[:nl], T_PLAIN)
    w0 = L.hc_weights_preprocess(ctx0, d, K)
    ct = to_dev(uniform_residues(s, CANONICAL_PRIMES[:nl], (w0.I, 2), N))
    ref = run(ctx0, w0, ct)
    w0.close(); ctx0.close()

    L.lib().hc_set_allocator(C.cast(a, C.c_void_p), C.cast(f, C.c_void_p), None)
    ctx = L.hc_ctx_create(N, CANONICAL_PRIMES[:nl], T_PLAIN)
    w = L.hc_weights_preprocess(ctx, d, K)
    assert torch.equal(run(ctx, w, ct), ref)
    assert stats["alloc"] > 0
    stats["limit"] = 1 << 16                       # scratch of this layer is larger (393 KB)
    try:
        run(ctx, w, ct)
        raise SystemExit("expected HC_ERR_OOM")
    except L.HcError as e:
        assert e.status == L.HC_ERR_OOM, e
    assert stats["refused"] >= 1
    stats["limit"] = None
    assert torch.equal(run(ctx, w, ct), ref)       # the context is unharmed
    w.close(); ctx.close()
    assert stats["free"] == stats["alloc"], stats  # every allocation returned
    L.lib().hc_set_allocator(None, None, None)
    print("ok", stats)
""")


def test_allocator_hook_in_child(L):
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", CHILD, root], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "ok" in r.stdout, (r.stdout[-2000:], r.stderr[-4000:])
