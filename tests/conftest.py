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


@pytest.fixture(scope="session")
def fd():
    """The built library's Python binding (GPU tests only)."""
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_01556_gb300 import build

    build.build()
    import paper_1806_01556_gb300 as fdas

    fdas.lib()
    return fdas


@pytest.fixture(scope="session")
def small_case(bank):
    """The N = 2^16 single-tone workload with its FP64 oracle plane."""
    import synth
    from oracle import correlate

    wl = synth.small_workload()
    return wl, correlate.plane_ols(wl.spectrum, bank, 2048)


@pytest.fixture(scope="session")
def ska_case(bank):
    """The N = 2^21 workload (4 tones x 8 harmonics) with its FP64 oracle plane (about 30 s)."""
    import synth
    from oracle import correlate

    wl = synth.ska_workload()
    return wl, correlate.plane_ols(wl.spectrum, bank, 2048)
