"""Helpers shared by the GPU parity tests (marshalling only, no arithmetic)."""
import numpy as np


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).cuda()


def to_host(t):
    return t.detach().cpu().numpy().view(np.uint64)


def sample_indices(N, n_random, seed):
    """Edges plus seeded random coefficient indices (sorted, unique)."""
    from paper_2506_11586_gb300.inputs import Stream
    ks = set(range(8)) | set(range(N - 8, N)) | {N // 2 - 1, N // 2, N // 2 + 1}
    ks |= set(int(k) for k in Stream(seed, 99).below(N, n_random))
    return np.array(sorted(ks), dtype=np.uint32)
