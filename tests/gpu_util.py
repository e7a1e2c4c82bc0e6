"""Helpers for the GPU parity tests (host side only)."""
import numpy as np


def to_dev(V):
    import torch
    import paper_2503_16717_gb300 as rbo
    n, c = V.shape
    Vd = rbo.colmajor(n, c)
    Vd.copy_(torch.from_numpy(np.asarray(V)))
    return Vd


def to_host(Vd):
    return Vd.cpu().numpy()
