"""Helpers for the GPU tests: numpy uint64 words <-> CUDA tensors."""
import numpy as np
import torch

import paper_1708_09746_gb300 as G


def need_gpu():
    assert torch.cuda.is_available(), "this test needs a CUDA GPU"
    from paper_1708_09746_gb300 import build
    build.build()
    G.load()


def to_dev(words):
    w = np.ascontiguousarray(np.asarray(words, dtype=np.uint64))
    if w.size == 0:
        return torch.zeros(1, dtype=torch.int64, device="cuda")
    return torch.from_numpy(w.view(np.int64).copy()).cuda()


def from_dev(t, n=None):
    a = t.detach().cpu().numpy().view(np.uint64)
    return a if n is None else a[:n]


def empty_dev(nwords):
    return torch.zeros(max(1, int(nwords)), dtype=torch.int64, device="cuda")


def pairs_to_ints(words):
    w = np.asarray(words, dtype=np.uint64)
    return [int(w[2 * i]) | (int(w[2 * i + 1]) << 64) for i in range(len(w) // 2)]


def ints_to_pairs(vals):
    out = np.zeros(2 * len(vals), dtype=np.uint64)
    for i, v in enumerate(vals):
        out[2 * i] = v & (2**64 - 1)
        out[2 * i + 1] = v >> 64
    return out


def gpu_mul(a, na, b, nb, sentinel=True):
    """Product through the C-ABI gf2x_mul; checks no word past the product
    is written (the output buffer carries a sentinel tail)."""
    ow = G.gf2x_out_words(na, nb)
    da, db = to_dev(a), to_dev(b)
    out = torch.full((ow + 4,), -0x5A5A5A5A5A5A5A5B, dtype=torch.int64, device="cuda")
    G.gf2x_mul(da, na, db, nb, out)
    torch.cuda.synchronize()
    res = from_dev(out)
    if sentinel:
        assert all(int(x) == 0xA5A5A5A5A5A5A5A5 for x in res[ow:]), "wrote past the product"
    return res[:ow]
