import os
import sys

# The oracle's block elimination makes thousands of LAPACK calls on blocks of a
# few hundred rows; with one BLAS thread per process they run several times
# faster than with a thread pool (set before numpy is first imported).
os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libcollo.so")
    config.addinivalue_line("markers", "slow: long-running CPU test")
