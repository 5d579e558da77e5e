import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TESTS = os.path.dirname(os.path.abspath(__file__))
for p in (ROOT, TESTS):
    if p not in sys.path:
        sys.path.insert(0, p)


def pytest_configure(config):
    config.addinivalue_line(
        "markers", "gpu: needs a CUDA GPU (GB300) and the built libslqr extension")
    config.addinivalue_line(
        "markers", "full_oracle(*names): compares with oracle outputs of full-size workloads "
                   "(tests/oracle_outputs.py), computed in background processes")


def pytest_collection_finish(session):
    """Start the oracle solves the selected full-size GPU tests need, so that
    they run on the host cores while the GPU tests before them do."""
    names = []
    for item in session.items:
        for mk in item.iter_markers("full_oracle"):
            names += list(mk.args)
    if not names:
        return
    import torch
    if not torch.cuda.is_available():
        return
    import oracle_outputs
    oracle_outputs.start(names)


def pytest_sessionfinish(session, exitstatus):
    mod = sys.modules.get("oracle_outputs")
    if mod is not None:
        mod.shutdown()
