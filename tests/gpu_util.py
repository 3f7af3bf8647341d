"""Shared helpers of the GPU tests."""
import pytest


def require_gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1110_4623_gb300 import build
    build.build()
    torch.cuda.set_device(0)
