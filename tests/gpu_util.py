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


def abs_product_rows(A, B, rows):
    """Rows `rows` of |A| |B| in FP64 by the oracle: the scale each output
    element's rounding errors are measured against."""
    import oracle
    return oracle.gemm_rows(np.abs(np.asarray(A, np.float64)), np.abs(np.asarray(B, np.float64)),
                            rows)


def assert_elementwise(got, ref, scale, rel):
    """|got - ref| <= rel * scale element by element (rel may be a scalar);
    reports the worst element and how many break the bound."""
    got = np.asarray(got, np.float64)
    diff = np.abs(got - ref)
    lim = rel * scale
    bad = ~(diff <= lim)
    if bad.any():
        i = np.unravel_index(np.argmax(np.where(bad, diff / np.maximum(lim, 1e-300), 0)), diff.shape)
        raise AssertionError(f"{int(bad.sum())} elements beyond the bound; worst at {i}: "
                             f"|diff| {diff[i]:.3e} > {lim[i] if np.ndim(lim) else lim:.3e}")


# Element-wise error bounds, relative to the element's (|alpha| |A||B| +
# |beta| |C0|), for a product with inner dimension k.  Each is a worst-case
# bound, not a typical error: accumulation at most one float32 unit
# (2^-23) per addition, doubled (2^-22) to cover a tensor-core accumulator
# that truncates, plus the variant's representation error per product:
#   3xBF16:   a b - (hi hi + hi lo + lo hi) <= (2^-16 + 2^-16 + 2^-34) |a||b|
#             (|x - hi| <= 2^-8|x|, |lo - (x - hi)| <= 2^-17|x|)
#   6-piece:  dropped mid lo + lo mid + lo lo <= (2^-23 + 2^-32) |a||b|
#   3xTF32:   lo lo + r_a b + a r_b with |r| <= 2^-22 |x|: 3.01 * 2^-22
#   TF32:     operands cut to 10 fraction bits (|x - t| < 2^-10 |x|)
# Variants compared against the product of the exact values they multiply
# (BF16 / FP8 tensor-core kinds) have no representation term.
_REPR = {0: 0.0, 1: 0.0, 2: 2.0 ** -9 + 2.0 ** -20, 3: 0.0, 4: 0.0,
         5: 2.0 ** -15 + 2.0 ** -34, 7: 2.0 ** -23 + 2.0 ** -32, 8: 3.01 * 2.0 ** -22,
         9: 2.0 ** -15 + 2.0 ** -34}


def elem_bound(v, k):
    """Relative element-wise bound of variant `v` at inner dimension `k`."""
    accum = (k + 4) * (2.0 ** -24 if v in (0, 1) else 2.0 ** -22)
    return _REPR[v] + accum
