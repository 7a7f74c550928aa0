import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU validation")


@pytest.fixture(scope="session")
def gpu_available():
    import torch
    return torch.cuda.is_available()


# Oracle runs of the full-size workloads, shared by the GPU tests that compare
# against them (each is minutes of host CPU work; computed once per session,
# on every host core).

@pytest.fixture(scope="session")
def reion128_oracle():
    """The 128^3 reionisation workload run 100 steps by the oracle:
    (workload, oracle table, library table, (U, xHI, T, hist, err, nclamp))."""
    from paper_1508_07888_b300 import inputs as I
    from _harness import run_oracle, tables
    w = I.reion(steps=100)
    to, tp = tables(w)
    return w, to, tp, run_oracle(w, 100, to, threads=os.cpu_count() or 1)[0]


@pytest.fixture(scope="session")
def reion256_oracle():
    """The 256^3 workload (8 fixed chemistry intervals) run 20 steps by the oracle."""
    from paper_1508_07888_b300 import inputs as I
    from _harness import run_oracle, tables
    w = I.reion_large(steps=20)
    to, tp = tables(w)
    return w, to, tp, run_oracle(w, 20, to, threads=os.cpu_count() or 1)[0]


@pytest.fixture(scope="session")
def ensemble64_oracle():
    """The 64-box ensemble run 100 steps by the oracle (boxes side by side)."""
    from paper_1508_07888_b300 import inputs as I
    from _harness import run_oracle, tables
    w = I.ensemble(steps=100)
    to, tp = tables(w)
    return w, to, tp, run_oracle(w, 100, to, box_parallel=True)
