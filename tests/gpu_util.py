"""Helpers for GPU tests: move seeded numpy inputs to the device, read results back."""
import numpy as np


def dev(x):
    import torch
    x = np.ascontiguousarray(x)
    if x.dtype == np.uint16:                    # bf16 bit patterns
        return torch.from_numpy(x.view(np.int16)).cuda().view(torch.bfloat16)
    return torch.from_numpy(x).cuda()


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def empty_c(m, n, fill=np.nan):
    import torch
    return torch.full((m, n), float(fill), dtype=torch.float32, device="cuda")
