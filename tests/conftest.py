import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the compiled libvelopir.so")
    config.addinivalue_line("markers", "slow: long-running CPU test")


TOY = dict(n=32, N=256, l=3, bg_bits=7, ks_t=8, ks_base_bits=2)


@pytest.fixture(scope="session")
def paper_keys():
    """Oracle cloud key at the paper's parameters from the master seed."""
    import oracle
    from paper_2506_12761_gb300 import synth
    km = synth.key_material()
    return oracle.keygen(oracle.paper_params(), km)


@pytest.fixture(scope="session")
def toy_keys():
    """Oracle key at a toy parameter set (n=32, N=256) for exhaustive circuit checks."""
    import oracle
    from paper_2506_12761_gb300 import synth
    P = oracle.Params(TOY["n"], TOY["N"], TOY["l"], TOY["bg_bits"], TOY["ks_t"], TOY["ks_base_bits"])
    km = synth.key_material(seed=7, n=P.n, N=P.N, l=P.l, ks_t=P.ks_t, ks_base_bits=P.ks_base_bits)
    return oracle.keygen(P, km)


def read_golden(name):
    rows = {}
    with open(os.path.join(ROOT, "tests", "golden", name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, *v = line.split()
            rows[k] = v
    return rows
