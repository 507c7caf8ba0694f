"""Shared helpers of the GPU tests: library build/load and error bounds."""
import math

import numpy as np
import pytest

U32 = 2.0 ** -24     # unit roundoff, FP32
U64 = 2.0 ** -53


def gpu_lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1011_4764_gb300 import build
    build.build()
    from paper_1011_4764_gb300 import ofm
    return ofm
