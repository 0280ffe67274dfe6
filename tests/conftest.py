"""Shared pytest configuration: the ``gpu`` marker and seeded inputs."""

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the compiled libpdr.so")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


@pytest.fixture(scope="session")
def grid5():
    from paper_2108_07549_gb300 import instances

    return instances.grid5_k10(1.3, seed=0)


@pytest.fixture(scope="session")
def grid5_bad():
    from paper_2108_07549_gb300 import instances

    return instances.grid5_k10(1.3, seed=0).with_factor(0.6)


@pytest.fixture(scope="session")
def knn2500():
    from paper_2108_07549_gb300 import instances

    return instances.knn2500_k500(1.2, seed=0)
