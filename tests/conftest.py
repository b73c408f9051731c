import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: test needs a CUDA GPU (runs the sm_103a library)")
    config.addinivalue_line("markers", "slow: CPU test taking more than a few seconds")


@pytest.fixture(scope="session")
def small_noisefree():
    """1-yr, 1-h-knot sky with 2000 sources and no noise (truth is an exact fixed point)."""
    import synth
    return synth.simulate(synth.config("small1yr", n_src=2000, noise_free=True))


@pytest.fixture(scope="session")
def small_noisy():
    import synth
    return synth.simulate(synth.config("small1yr", n_src=2000))
