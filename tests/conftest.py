import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append(line.split())
    return rows


# ---------------------------------------------------------------------------
# GPU helpers: move oracle-side numpy arrays to and from the device
# ---------------------------------------------------------------------------

def lib_built():
    """Build lib/libhisq.so if needed (nvcc cross-compiles without a GPU)."""
    from paper_1411_4439_gb300 import build_lib
    return build_lib.build()


def to_dev(arr, prec):
    """numpy complex128 [..., 3] -> device tensor of the storage precision."""
    import torch
    import paper_1411_4439_gb300 as H
    t = torch.from_numpy(arr)
    if prec == H.HISQ_F64:
        return t.to("cuda", torch.complex128).contiguous()
    if prec == H.HISQ_F32:
        return t.to("cuda", torch.complex64).contiguous()
    return torch.view_as_real(t.to(torch.complex64)).to("cuda", torch.float16).contiguous()


def from_dev(t):
    import torch
    if t.dtype == torch.float16:
        return torch.view_as_complex(t.float().cpu()).numpy().astype("complex128")
    return t.cpu().numpy().astype("complex128")


def rel_l2(a, b):
    import numpy as np
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="session")
def gpu_lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib_built()
    import paper_1411_4439_gb300 as H
    H.hisq.library()
    return H
