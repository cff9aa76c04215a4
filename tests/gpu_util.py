"""Helpers of the GPU tests: export an oracle case, load it in the library,
move panels between numpy (N, nrhs) and torch (nrhs, N) device tensors."""
import os
import tempfile

import numpy as np

from oracle.export import write_blocks


def load_case(H, S, groups=None, **kw):
    """Export the oracle's H (and scaling S, and supernode groups with their
    T_G) and load it in the library with solve options kw."""
    import paper_2109_04129_gb300 as hp
    fd, path = tempfile.mkstemp(suffix=".hmps")
    os.close(fd)
    try:
        write_blocks(path, H, S, groups=groups)
        return hp.Solver.load(path, **kw)
    finally:
        os.unlink(path)


def to_dev(A):
    import torch
    A = np.asarray(A, dtype=np.complex128).reshape(A.shape[0], -1)
    return torch.from_numpy(np.ascontiguousarray(A.T)).cuda()


def from_dev(T):
    return T.cpu().numpy().T.copy()


def rand_panel(N, nrhs, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((N, nrhs)) + 1j * rng.standard_normal((N, nrhs))


def rel(a, b):
    a = np.asarray(a).reshape(len(a), -1)
    b = np.asarray(b).reshape(len(b), -1)
    return np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)
