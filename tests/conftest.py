import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the CUDA library)")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture
def torch_side_stream():
    """Run the test under a non-default torch stream.  The library's contexts
    take a stream handle, and handle 0 (torch's default stream) selects the
    context's own stream instead; under a side stream, set_stream(current)
    puts the library's work in order with the tensors the test fills and
    reads."""
    import torch
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        yield side
    torch.cuda.synchronize()
