import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libpfire")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_collection_modifyitems(config, items):
    # A test marked gpu is skipped, not failed, when no GPU is visible; on a GPU machine a
    # missing or unloadable libpfire is an error raised by the test itself.
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device visible")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session", autouse=True)
def _tuning_cache(tmp_path_factory):
    # the autotuner's on-disk cache goes to a per-session file, not the user's cache
    if "PF_TUNE_CACHE" not in os.environ:
        os.environ["PF_TUNE_CACHE"] = str(tmp_path_factory.mktemp("tune") / "tuning.tsv")
    yield
