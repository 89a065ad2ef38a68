"""Shared helpers for the GPU tests: move generator output to CUDA tensors."""

import numpy as np


def to_cuda(d, keys=("At", "b", "lo", "hi")):
    import torch
    out = {}
    for k in keys:
        if k in d and d[k] is not None:
            out[k] = torch.from_numpy(np.ascontiguousarray(d[k])).cuda()
    return out


def quantize_columns(At_np, m, kind):
    """Per-column symmetric quantisation of A (input preparation for the BF16/FP8 storage).

    Returns (q CUDA tensor (n, lda), scale CUDA float32 (n,), dequantised FP64 numpy (n, m)).
    """
    import torch
    A = torch.from_numpy(np.ascontiguousarray(At_np[:, :m])).to(torch.float64)
    n = A.shape[0]
    amax = A.abs().amax(dim=1).clamp_min(1e-30)
    if kind == "bf16":
        scale = (amax / 1.0).to(torch.float32)
        tdt, elt = torch.bfloat16, 2
    else:
        scale = (amax / 448.0).to(torch.float32)
        tdt, elt = torch.float8_e4m3fn, 1
    per = 16 // elt
    lda = (m + per - 1) // per * per
    q = (A / scale.to(torch.float64)[:, None]).to(torch.float32).to(tdt)
    qp = torch.zeros((n, lda), dtype=tdt)
    qp[:, :m] = q
    deq = q.to(torch.float64) * scale.to(torch.float64)[:, None]
    return qp.cuda(), scale.cuda(), deq.numpy()


def rel_inf(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = max(float(np.abs(b).max(initial=0.0)), 1e-300)
    return float(np.abs(a - b).max(initial=0.0)) / den
