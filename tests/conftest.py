import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


_MODELS = {}


def oracle_model(refinement, **kw):
    """Cached oracle models keyed by their parameters (test infrastructure)."""
    from oracle.model import OracleModel, OracleParams
    key = (refinement, tuple(sorted(kw.items())))
    if key not in _MODELS:
        kw.setdefault("lambda_max", 1.0)
        _MODELS[key] = OracleModel(OracleParams(refinement=refinement, **kw))
    return _MODELS[key]


@pytest.fixture(scope="session")
def om():
    return oracle_model
