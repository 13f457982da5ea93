"""Shared pytest configuration: registers the ``gpu`` marker and puts the repository root on
``sys.path`` so that ``oracle`` and ``paper_2310_08408_gb300`` import from the checkout."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
