import os
import sys

import pytest

# Hardware work queues for concurrent streams (read when the CUDA context is created): the
# default 8 makes streams share queues, and work of one stream then waits behind another's
# (the serving tests overlap small requests with large ones).
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")
