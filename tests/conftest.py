"""Shared pytest configuration: the ``gpu`` marker and cached oracle fixtures."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libfdas")


@pytest.fixture(scope="session")
def bank():
    """Oracle time-domain templates for the default grid (85 x 421), FP64."""
    from oracle import templates

    return templates.template_bank(templates.TemplateGrid())
