"""Shared helpers for the GPU parity tests (layout conversion, tolerances, the library context)."""
from paper_2405_09233_gb300 import inputs

U64 = 2.0 ** -53  # unit roundoff of FP64


def to_dev(X, device="cuda"):
    import torch
    return torch.from_numpy(inputs.to_device_layout(X)).to(device)


def from_dev(T):
    return inputs.from_device_layout(T.detach().cpu().numpy())


def fp64_product_bound(absA, absB, tprod, length):
    """Rounding bound for an FP64 T-product by DFT + per-slice GEMM + inverse DFT.

    Every entry of A*B is a sum of p * n2 products; the DFT route forms it with
    O(p + n2) additions per entry, each rounding at most u relative to the
    running magnitude, which is bounded by (|A| * |B|)(i, j, k).  With a safety
    factor of 8 the bound is 8 (p + n2) u (|A| * |B|).
    """
    return 8.0 * length * U64 * tprod(absA, absB)
