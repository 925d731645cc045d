"""Device-side failure detection without a GPU fault: a bounded mbarrier wait
that nothing completes runs out, the kernel records a timeout in the
context's device flag and returns, the host reads HC_ERR_TIMEOUT, and the
context stays usable (an NTT round trip afterwards is still exact)."""
import numpy as np
import pytest

from gpu_util import to_dev, to_host
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


def test_bounded_wait_timeout_is_reported(L):
    ctx = L.hc_ctx_create(4096, CANONICAL_PRIMES[:2], T_PLAIN)
    L.hc_ctx_device_status(ctx)                       # clean to start with
    L.hc_selftest_wait_timeout(ctx, 256)
    with pytest.raises(L.HcError) as e:
        L.hc_ctx_device_status(ctx)
    assert e.value.status == L.HC_ERR_TIMEOUT
    L.hc_ctx_device_status(ctx)                       # reading cleared the flag
    a = uniform_residues(Stream(3, 3), CANONICAL_PRIMES[:2], (2,), 4096)
    d = to_dev(a)
    L.hc_ntt_fwd(ctx, d)
    L.hc_ntt_inv(ctx, d)
    torch.cuda.synchronize()
    assert np.array_equal(to_host(d).reshape(a.shape), a)
    with pytest.raises(L.HcError):
        L.hc_selftest_wait_timeout(ctx, 0)
