import functools
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a) and the built library")


@functools.lru_cache(maxsize=None)
def cached_scene(workload, scale=1.0, seed=None, **kw):
    from paper_2305_07026_b300 import scenes
    return scenes.make_scene(workload, scale=scale, seed=seed, **dict(kw))


@pytest.fixture(scope="session")
def circle():
    return cached_scene("circle")


def rng_for(name):
    return np.random.default_rng(abs(hash(name)) % (2 ** 32))
